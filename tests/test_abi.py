"""The C ABI without a GPU: the library loads, exports every entry point that
include/bcf.h declares, and rejects invalid arguments on the host before any
CUDA call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(bcf_[a-z0-9_]+)\s*\(", text))
    return names


def _lib():
    from paper_2311_16121_b300 import build

    build.build()
    import paper_2311_16121_b300 as bcf

    return bcf, bcf.lib()


def test_library_exports_every_declared_symbol():
    bcf, L = _lib()
    names = _declared()
    assert {"bcf_decode_bc6h", "bcf_create_material", "bcf_sample_features", "bcf_decode_material"} <= names
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    assert L.bcf_version() >= 100


def test_host_validation_rejects_bad_arguments():
    bcf, L = _lib()
    # negative sizes / null pointers: rejected before any launch
    assert L.bcf_decode_bc6h(None, -1, 4, 0, None, None) == 1
    assert L.bcf_decode_bc6h(None, 4, 4, 0, None, None) == 1
    assert L.bcf_decode_bc6h(None, 0, 7, 0, None, None) == 0  # empty image: no-op
    assert b"null" in L.bcf_last_error()
    d = bcf._MaterialDesc()
    h = ctypes.c_void_p()
    d.num_textures = 0
    assert L.bcf_create_material(ctypes.byref(d), ctypes.byref(h)) == 1
    d.num_textures = 1
    d.res_ref = 64
    d.res[0] = 48  # not a power of two
    d.levels[0] = 1
    assert L.bcf_create_material(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"power of two" in L.bcf_last_error()
    d.res[0] = 64
    d.levels[0] = 6  # 64 -> at most 5 levels (down to one 4x4 block)
    assert L.bcf_create_material(ctypes.byref(d), ctypes.byref(h)) == 1
    d.levels[0] = 5
    d.d_blocks[0] = 8  # misaligned
    assert L.bcf_create_material(ctypes.byref(d), ctypes.byref(h)) == 1
    d.d_blocks[0] = 4096
    d.n_layers = 2
    d.dims[0], d.dims[1], d.dims[2] = 3, 8, 3  # lod_input = 0: 3 inputs
    d.precision = 3
    d.d_weights, d.d_biases = 4096, 8192
    d.act_scale[0], d.act_scale[1] = 0.3, 1.0  # not a power of two
    d.w_scale[0], d.w_scale[1] = 1.0, 1.0
    assert L.bcf_create_material(ctypes.byref(d), ctypes.byref(h)) == 2
    assert L.bcf_decode_material(None, None, None, None, 10, None, 0, None) == 1
    assert L.bcf_sample_features(None, None, None, None, -1, None, None) == 1
    assert L.bcf_status_string(5) == b"device wait timed out"


def test_encoder_host_validation():
    bcf, L = _lib()
    L.bcf_encode_mode10.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert L.bcf_encode_mode10(4096, 3, 48, 1, 4096, 4096, None, None) == 1  # not a power of two
    assert b"power of two" in L.bcf_last_error()
    assert L.bcf_encode_mode10(4096, 3, 64, 6, 4096, 4096, None, None) == 1  # 64 -> at most 5 levels (64 .. 4)
    assert L.bcf_encode_mode10(4096, 3, 64, 0, 4096, 4096, None, None) == 1
    assert L.bcf_encode_mode10(4096, 5, 64, 4, 4096, 4096, None, None) == 1  # texel stride
    assert L.bcf_encode_mode10(None, 3, 64, 4, 4096, 4096, None, None) == 1  # null texels
    assert L.bcf_encode_mode10(4098, 3, 64, 4, 4096, 4096, None, None) == 1  # misaligned texels
    assert b"misaligned" in L.bcf_last_error()
    assert bcf.texture_blocks(64, 4) == 256 + 64 + 16 + 4


def test_compressor_and_packer_host_validation():
    _, L = _lib()
    L.bcf_compress_bc6h.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert L.bcf_compress_bc6h(4096, 3, 48, 1, 4096, None, None, None) == 1  # not a power of two
    assert L.bcf_compress_bc6h(4096, 3, 64, 6, 4096, None, None, None) == 1  # too many levels
    assert L.bcf_compress_bc6h(4096, 2, 64, 4, 4096, None, None, None) == 1  # texel stride
    assert L.bcf_compress_bc6h(4096, 3, 64, 4, 4104, None, None, None) == 1  # blocks not 16-byte aligned
    assert b"misaligned" in L.bcf_last_error()
    L.bcf_pack_mode10.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                  ctypes.c_void_p, ctypes.c_void_p]
    assert L.bcf_pack_mode10(4096, 4096, -1, 0, 4096, None) == 1
    assert L.bcf_pack_mode10(4096, 4096, 0, 0, None, None) == 0  # nothing to do
    assert L.bcf_pack_mode10(4100, 4096, 8, 0, 4096, None) == 1  # params not 16-byte aligned
    assert L.bcf_pack_mode10(4096, None, 8, 0, 4096, None) == 1  # no partitions


def test_material_bytes_reproduce_table2_sizes():
    """The storage the schedule reports for a block-compressed material (16 bytes per 4 x 4 block, full mip
    chains) reproduces the sizes printed for the paper's profiles (Table 2 with Table 1's resolutions)."""
    from paper_2311_16121_b300 import schedule

    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "golden", "table2_sizes.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 4
    for r in rows:
        res = [int(r[1]), int(r[3]), int(r[5]), int(r[7])]
        levels = [int(r[2]), int(r[4]), int(r[6]), int(r[8])]
        mib = schedule.material_bytes(res, levels) / 2 ** 20
        assert round(mib, 2) == float(r[9]), (r[0], mib)
