"""Python binding of libbcf (include/bcf.h): argument marshalling only.

Every computation runs in the CUDA kernels of ``libbcf.so``; this module turns
torch tensors into device pointers and the current torch stream into a CUDA
stream handle, calls the C entry point of the same name and raises
``BcfError`` on a non-OK status.  There is no CPU fallback: importing the
binding without the built library raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_float, c_int, c_int32, c_int64, c_void_p

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbcf.so")

MAX_TEX = 16
MAX_LEVELS = 16
MAX_LAYERS = 8
MAX_WIDTH = 128

FP32, FP16, BF16, FP8_E4M3 = 0, 1, 2, 3
CHECK_PARTITION, CHECK_OFFSETS = 0x1, 0x2  # bits of the device check word
PRECISION = {"fp32": FP32, "fp16": FP16, "bf16": BF16, "fp8": FP8_E4M3}


class BcfError(RuntimeError):
    def __init__(self, status: int, where: str, text: str):
        super().__init__(f"{where}: status {status} ({text})")
        self.status = status


class _MaterialDesc(ctypes.Structure):
    _fields_ = [("num_textures", c_int32), ("res", c_int32 * MAX_TEX), ("levels", c_int32 * MAX_TEX),
                ("res_ref", c_int32), ("is_signed", c_int32), ("wrap", c_int32), ("lod_input", c_int32),
                ("d_blocks", c_void_p * MAX_TEX), ("n_layers", c_int32), ("dims", c_int32 * (MAX_LAYERS + 1)),
                ("precision", c_int), ("d_weights", c_void_p), ("d_biases", c_void_p),
                ("act_scale", c_float * MAX_LAYERS), ("w_scale", c_float * MAX_LAYERS)]


class _TrainerDesc(ctypes.Structure):
    _fields_ = [("num_textures", c_int32), ("res", c_int32 * MAX_TEX), ("levels", c_int32 * MAX_TEX),
                ("res_ref", c_int32), ("lod_input", c_int32), ("d_params", c_void_p * MAX_TEX),
                ("d_partition", c_void_p * MAX_TEX), ("d_grad", c_void_p * MAX_TEX), ("d_adam_m", c_void_p * MAX_TEX),
                ("d_adam_v", c_void_p * MAX_TEX), ("n_layers", c_int32), ("dims", c_int32 * (MAX_LAYERS + 1)),
                ("d_W", c_void_p), ("d_b", c_void_p), ("d_W_grad", c_void_p), ("d_b_grad", c_void_p),
                ("d_W_m", c_void_p), ("d_W_v", c_void_p), ("d_b_m", c_void_p), ("d_b_v", c_void_p),
                ("target_res", c_int32), ("target_levels", c_int32), ("d_target8", c_void_p), ("d_target1", c_void_p),
                ("lr_features", c_float), ("lr_mlp", c_float), ("gamma", c_float), ("beta1", c_float),
                ("beta2", c_float), ("eps", c_float), ("s_max", c_float), ("unconstrained", c_int32),
                ("is_signed", c_int32), ("literal", c_int32), ("batch_grid", c_int32)]


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libbcf.  Raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libbcf is not built ({LIB_PATH} missing); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.bcf_status_string.restype = c_char_p
        L.bcf_status_string.argtypes = [c_int]
        L.bcf_last_error.restype = c_char_p
        L.bcf_last_error.argtypes = []
        L.bcf_version.restype = c_int
        L.bcf_decode_bc6h.restype = c_int
        L.bcf_decode_bc6h.argtypes = [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p]
        L.bcf_texunit_decode_bc6h.restype = c_int
        L.bcf_texunit_decode_bc6h.argtypes = [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p]
        L.bcf_create_material.restype = c_int
        L.bcf_create_material.argtypes = [POINTER(_MaterialDesc), POINTER(c_void_p)]
        L.bcf_destroy_material.restype = c_int
        L.bcf_destroy_material.argtypes = [c_void_p]
        L.bcf_sample_features.restype = c_int
        L.bcf_sample_features.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p]
        L.bcf_set_decode_variant.restype = c_int
        L.bcf_set_decode_variant.argtypes = [c_void_p, c_int32]
        L.bcf_set_mlp_engine.restype = c_int
        L.bcf_set_mlp_engine.argtypes = [c_void_p, c_int32]
        L.bcf_material_refresh.restype = c_int
        L.bcf_material_refresh.argtypes = [c_void_p, c_void_p]
        L.bcf_texunit_fetch_probe.restype = c_int
        L.bcf_texunit_fetch_probe.argtypes = [c_void_p, c_int32, c_int32, c_int64, c_int32, c_void_p, c_void_p]
        L.bcf_decode_material.restype = c_int
        L.bcf_decode_material.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_int, c_void_p]
        L.bcf_create_material_set.restype = c_int
        L.bcf_create_material_set.argtypes = [c_void_p, c_int32, POINTER(c_void_p)]
        L.bcf_destroy_material_set.restype = c_int
        L.bcf_destroy_material_set.argtypes = [c_void_p]
        L.bcf_decode_material_set.restype = c_int
        L.bcf_decode_material_set.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p,
                                              c_int, c_void_p]
        L.bcf_autotune_material_set.restype = c_int
        L.bcf_autotune_material_set.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p,
                                                c_int, c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)]
        L.bcf_material_set_config.restype = c_int
        L.bcf_material_set_config.argtypes = [c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)]
        L.bcf_trainer_create.restype = c_int
        L.bcf_trainer_create.argtypes = [POINTER(_TrainerDesc), POINTER(c_void_p)]
        L.bcf_trainer_destroy.restype = c_int
        L.bcf_trainer_destroy.argtypes = [c_void_p]
        L.bcf_train_step.restype = c_int
        L.bcf_train_step.argtypes = [c_void_p, c_int64, ctypes.c_uint64, c_int64, c_void_p, c_void_p, c_void_p,
                                     c_void_p, c_void_p]
        L.bcf_train_step_noalloc.restype = c_int
        L.bcf_train_step_noalloc.argtypes = [c_void_p, c_int64, ctypes.c_uint64, c_int64, c_void_p, c_void_p,
                                             c_void_p, c_void_p, c_void_p]
        L.bcf_train_forward.restype = c_int
        L.bcf_train_forward.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p]
        L.bcf_train_backward.restype = c_int
        L.bcf_train_backward.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p]
        L.bcf_train_export.restype = c_int
        L.bcf_train_export.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
        L.bcf_decode_material_host.restype = c_int
        L.bcf_decode_material_host.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_int,
                                               c_void_p, c_int64, c_void_p]
        L.bcf_encode_mode10.restype = c_int
        L.bcf_encode_mode10.argtypes = [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]
        L.bcf_compress_bc6h.restype = c_int
        L.bcf_compress_bc6h.argtypes = [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]
        L.bcf_pack_mode10.restype = c_int
        L.bcf_pack_mode10.argtypes = [c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p]
        L.bcf_device_check.restype = c_int
        L.bcf_device_check.argtypes = [POINTER(ctypes.c_uint32)]
        _lib = L
    return _lib


def _check(status: int, where: str) -> None:
    if status != 0:
        L = lib()
        raise BcfError(status, where, (L.bcf_last_error() or b"").decode() or L.bcf_status_string(status).decode())


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libbcf takes CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("libbcf takes contiguous tensors")
    return t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


# --------------------------------------------------------------------------- BC6H

def device_check(raise_on_failure: bool = True) -> int:
    """bcf_device_check: wait for all work on the current device, read and clear its check word
    (CHECK_PARTITION, CHECK_OFFSETS) and return it; raises BcfError naming the checks when a bit is set and
    raise_on_failure holds."""
    word = ctypes.c_uint32(0)
    status = lib().bcf_device_check(ctypes.byref(word))
    if status != 0 and (raise_on_failure or word.value == 0):
        _check(status, "bcf_device_check")
    return word.value


def decode_bc6h(blocks: torch.Tensor, blocks_w: int, blocks_h: int, is_signed: bool = False,
                out: torch.Tensor | None = None) -> torch.Tensor:
    """bcf_decode_bc6h: uint8 [bh * bw * 16] blocks -> int16 [4 bh, 4 bw, 3] half bit patterns."""
    if out is None:
        out = torch.empty((4 * blocks_h, 4 * blocks_w, 3), dtype=torch.int16, device=blocks.device)
    _check(lib().bcf_decode_bc6h(_ptr(blocks), blocks_w, blocks_h, int(is_signed), _ptr(out), _stream()),
           "bcf_decode_bc6h")
    return out


def texture_blocks(res: int, levels: int) -> int:
    """Blocks of a mipmapped texture of `levels` levels from res x res (sum of (W / 4)^2)."""
    return sum(((res >> l) // 4) ** 2 for l in range(levels))


def encode_mode10(texels: torch.Tensor, res: int, levels: int, params: torch.Tensor | None = None,
                  partitions: torch.Tensor | None = None, errors: torch.Tensor | None = None, texel_stride: int = 3):
    """bcf_encode_mode10: RGB texels (levels concatenated, float32, `texel_stride` floats per texel) -> block
    parameters [blocks][32], partitions [blocks] uint8 and per-block squared errors [blocks]."""
    nb = texture_blocks(res, levels)
    n_tex = sum(texel_stride * (res >> l) ** 2 for l in range(levels))
    if texels.dtype != torch.float32 or texels.numel() < n_tex:
        raise ValueError(f"encode_mode10: texels must be float32 with at least {n_tex} values")
    for t, shape_n, dt in ((params, nb * 32, torch.float32), (partitions, nb, torch.uint8), (errors, nb, torch.float32)):
        if t is not None and (t.dtype != dt or t.numel() < shape_n):
            raise ValueError(f"encode_mode10: output of {shape_n} {dt} values expected")
    dev = texels.device
    params = torch.empty((nb, 32), dtype=torch.float32, device=dev) if params is None else params
    partitions = torch.empty(nb, dtype=torch.uint8, device=dev) if partitions is None else partitions
    errors = torch.empty(nb, dtype=torch.float32, device=dev) if errors is None else errors
    _check(lib().bcf_encode_mode10(_ptr(texels), int(texel_stride), int(res), int(levels), _ptr(params), _ptr(partitions),
                                   _ptr(errors), _stream()), "bcf_encode_mode10")
    return params, partitions, errors


def compress_bc6h(texels: torch.Tensor, res: int, levels: int, texel_stride: int = 3):
    """bcf_compress_bc6h: RGB texels (levels concatenated, float32) -> BC6H UF16 blocks uint8 [blocks * 16] (the
    better of a mode-10 and a mode-11 encoding per block), squared errors [blocks] and modes [blocks] (10 / 11)."""
    nb = texture_blocks(res, levels)
    n_tex = sum(texel_stride * (res >> l) ** 2 for l in range(levels))
    if texels.dtype != torch.float32 or texels.numel() < n_tex:
        raise ValueError(f"compress_bc6h: texels must be float32 with at least {n_tex} values")
    dev = texels.device
    blocks = torch.empty(nb * 16, dtype=torch.uint8, device=dev)
    errors = torch.empty(nb, dtype=torch.float32, device=dev)
    modes = torch.empty(nb, dtype=torch.uint8, device=dev)
    _check(lib().bcf_compress_bc6h(_ptr(texels), int(texel_stride), int(res), int(levels), _ptr(blocks),
                                   _ptr(errors), _ptr(modes), _stream()), "bcf_compress_bc6h")
    return blocks, errors, modes


def pack_mode10(params: torch.Tensor, partitions: torch.Tensor, is_signed: bool = False) -> torch.Tensor:
    """bcf_pack_mode10: block-parameter records [blocks][32] float32 and partition ids [blocks] uint8 -> BC6H
    mode-10 blocks as uint8 [blocks * 16]."""
    nb = params.shape[0] if params.dim() == 2 else params.numel() // 32
    if params.dtype != torch.float32 or params.numel() != nb * 32:
        raise ValueError("pack_mode10: params must be float32 [blocks, 32]")
    if partitions.dtype != torch.uint8 or partitions.numel() < nb:
        raise ValueError(f"pack_mode10: {nb} uint8 partition ids expected")
    out = torch.empty(nb * 16, dtype=torch.uint8, device=params.device)
    _check(lib().bcf_pack_mode10(_ptr(params), _ptr(partitions), nb, int(is_signed), _ptr(out), _stream()),
           "bcf_pack_mode10")
    return out


def texunit_decode_bc6h(blocks: torch.Tensor, blocks_w: int, blocks_h: int, is_signed: bool = False) -> torch.Tensor:
    """bcf_texunit_decode_bc6h: the same decode by the GPU texture unit (checking only)."""
    out = torch.empty((4 * blocks_h, 4 * blocks_w, 3), dtype=torch.int16, device=blocks.device)
    _check(lib().bcf_texunit_decode_bc6h(_ptr(blocks), blocks_w, blocks_h, int(is_signed), _ptr(out), _stream()),
           "bcf_texunit_decode_bc6h")
    return out


# --------------------------------------------------------------------------- material

class Material:
    """A bcf_material: BC6H feature textures with mip chains plus the MLP decoder (device tensors, kept alive)."""

    def __init__(self, blocks: list[torch.Tensor], res: list[int], levels: list[int], res_ref: int,
                 dims: list[int], precision: str, weights: torch.Tensor, biases: torch.Tensor,
                 act_scale=None, w_scale=None, is_signed: bool = False, wrap: bool = True, lod_input: bool = True):
        d = _MaterialDesc()
        d.num_textures = len(blocks)
        for t, b in enumerate(blocks):
            d.res[t] = int(res[t])
            d.levels[t] = int(levels[t])
            d.d_blocks[t] = _ptr(b)
        d.res_ref = int(res_ref)
        d.is_signed = int(is_signed)
        d.wrap = int(wrap)
        d.lod_input = int(lod_input)
        d.n_layers = len(dims) - 1
        for i, v in enumerate(dims):
            d.dims[i] = int(v)
        d.precision = PRECISION[precision]
        d.d_weights = _ptr(weights)
        d.d_biases = _ptr(biases)
        for l in range(len(dims) - 1):
            d.act_scale[l] = float(act_scale[l]) if act_scale is not None else 1.0
            d.w_scale[l] = float(w_scale[l]) if w_scale is not None else 1.0
        h = c_void_p()
        _check(lib().bcf_create_material(ctypes.byref(d), ctypes.byref(h)), "bcf_create_material")
        self.handle = h
        self._keep = (list(blocks), weights, biases)
        self.dims = list(dims)
        self.n_tex = len(blocks)
        self.precision = precision

    def decode_host(self, u: torch.Tensor, v: torch.Tensor, s: torch.Tensor | None, out: torch.Tensor,
                    scratch: torch.Tensor) -> torch.Tensor:
        """bcf_decode_material_host: queries and `out` in (preferably pinned) host memory, pipelined through the
        device `scratch` (uint8, 256-byte aligned)."""
        for t in (u, v, s, out):
            if t is not None and (t.is_cuda or not t.is_contiguous()):
                raise ValueError("decode_host takes contiguous host tensors")
        prec = {torch.float32: 0, torch.float16: 1}[out.dtype]
        if out.numel() < u.numel() * self.dims[-1]:
            raise ValueError("decode_host: output too small")
        _check(lib().bcf_decode_material_host(self.handle, u.data_ptr(), v.data_ptr(),
                                              None if s is None else s.data_ptr(), u.numel(), out.data_ptr(), prec,
                                              _ptr(scratch), scratch.numel(), _stream()), "bcf_decode_material_host")
        return out

    def set_decode_variant(self, variant: int) -> None:
        """bcf_set_decode_variant: 0 tile-cooperative (default), 1 per-lane, 2 texture unit (hardware trilinear),
        3 texture-unit texels with the exact FP32 filter."""
        _check(lib().bcf_set_decode_variant(self.handle, int(variant)), "bcf_set_decode_variant")

    def refresh(self) -> None:
        """bcf_material_refresh: the texture-unit copy of the blocks follows a rewrite of the caller's blocks."""
        _check(lib().bcf_material_refresh(self.handle, _stream()), "bcf_material_refresh")

    def set_mlp_engine(self, engine: str) -> None:
        """bcf_set_mlp_engine: "mma_sync" (warp-level MMAs, default) or "tcgen05" (CTA-level MMAs with tensor-memory
        accumulators)."""
        code = {"mma_sync": 0, "tcgen05": 1}[engine]
        _check(lib().bcf_set_mlp_engine(self.handle, code), "bcf_set_mlp_engine")

    def texunit_fetch_probe(self, n_threads: int, rounds: int, texture: int = 0, level: int = 0,
                            sink: torch.Tensor | None = None) -> torch.Tensor:
        """bcf_texunit_fetch_probe (measurement only): 4 x rounds x n_threads point fetches of one level's texels
        in screen-coherent order; returns the float32 sink [n_threads]."""
        if sink is None:
            sink = torch.empty(n_threads, dtype=torch.float32, device="cuda")
        _check(lib().bcf_texunit_fetch_probe(self.handle, int(texture), int(level), int(n_threads), int(rounds),
                                             _ptr(sink), _stream()), "bcf_texunit_fetch_probe")
        return sink

    def close(self) -> None:
        if self.handle:
            _check(lib().bcf_destroy_material(self.handle), "bcf_destroy_material")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sample_features(self, u: torch.Tensor, v: torch.Tensor, s: torch.Tensor | None,
                        out: torch.Tensor | None = None) -> torch.Tensor:
        """bcf_sample_features -> float32 [n, 3 T]."""
        n = u.numel()
        if out is None:
            out = torch.empty((n, 3 * self.n_tex), dtype=torch.float32, device=u.device)
        _check(lib().bcf_sample_features(self.handle, _ptr(u), _ptr(v), _ptr(s), n, _ptr(out), _stream()),
               "bcf_sample_features")
        return out

    def decode(self, u: torch.Tensor, v: torch.Tensor, s: torch.Tensor | None, out_dtype=torch.float32,
               out: torch.Tensor | None = None) -> torch.Tensor:
        """bcf_decode_material -> [n, C] in float32 or float16."""
        n = u.numel()
        if out is None:
            out = torch.empty((n, self.dims[-1]), dtype=out_dtype, device=u.device)
        prec = FP16 if out.dtype == torch.float16 else FP32
        _check(lib().bcf_decode_material(self.handle, _ptr(u), _ptr(v), _ptr(s), n, _ptr(out), prec, _stream()),
               "bcf_decode_material")
        return out


# --------------------------------------------------------------------------- material sets

class MaterialSet:
    """A bcf_material_set: several materials sharing the MLP shape, decoded in one persistent launch."""

    def __init__(self, materials: list[Material]):
        arr = (c_void_p * len(materials))(*[m.handle.value for m in materials])
        h = c_void_p()
        _check(lib().bcf_create_material_set(arr, len(materials), ctypes.byref(h)), "bcf_create_material_set")
        self.handle = h
        self.materials = list(materials)
        self.dims = materials[0].dims

    def close(self):
        if self.handle:
            _check(lib().bcf_destroy_material_set(self.handle), "bcf_destroy_material_set")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def decode(self, offsets: torch.Tensor, u, v, s, out_dtype=torch.float16, out: torch.Tensor | None = None):
        """bcf_decode_material_set: offsets int64 [n_materials + 1] on the device; queries concatenated."""
        n = u.numel()
        if out is None:
            out = torch.empty((n, self.dims[-1]), dtype=out_dtype, device=u.device)
        prec = FP16 if out.dtype == torch.float16 else FP32
        _check(lib().bcf_decode_material_set(self.handle, _ptr(offsets), _ptr(u), _ptr(v), _ptr(s), n, _ptr(out),
                                             prec, _stream()), "bcf_decode_material_set")
        return out

    def autotune(self, offsets, u, v, s, out: torch.Tensor) -> tuple[int, int, int]:
        """bcf_autotune_material_set -> (arena blocks, CTAs per SM, tiles per grab)."""
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        prec = FP16 if out.dtype == torch.float16 else FP32
        _check(lib().bcf_autotune_material_set(self.handle, _ptr(offsets), _ptr(u), _ptr(v), _ptr(s), u.numel(),
                                               _ptr(out), prec, _stream(), ctypes.byref(a), ctypes.byref(b),
                                               ctypes.byref(c)), "bcf_autotune_material_set")
        return a.value, b.value, c.value

    def config(self) -> tuple[int, int, int]:
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().bcf_material_set_config(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "bcf_material_set_config")
        return a.value, b.value, c.value


def decode(target: "Material | MaterialSet", u: torch.Tensor, v: torch.Tensor, s: torch.Tensor | None,
           offsets: torch.Tensor | None = None, out_dtype=torch.float16, out: torch.Tensor | None = None):
    """Decode queries of one material (bcf_decode_material) or of a material set (bcf_decode_material_set,
    `offsets` [n_materials + 1] int64 on the device) -> [n, C] channels."""
    if isinstance(target, MaterialSet):
        if offsets is None:
            raise ValueError("decode: a material set needs the query offsets")
        return target.decode(offsets, u, v, s, out_dtype=out_dtype, out=out)
    if offsets is not None:
        raise ValueError("decode: offsets apply to material sets only")
    return target.decode(u, v, s, out_dtype=out_dtype, out=out)


# --------------------------------------------------------------------------- training

class Trainer:
    """A bcf_trainer: block parameters [blocks, 32] per texture (updated in place), partition ids, the FP32 MLP,
    the FP16 reference mip chain and the Adam state.  Gradient and moment buffers are allocated here (torch)."""

    def __init__(self, params: list[torch.Tensor], partition: list[torch.Tensor], res: list[int], levels: list[int],
                 res_ref: int, dims: list[int], W: torch.Tensor, b: torch.Tensor, target8: torch.Tensor,
                 target1: torch.Tensor, target_res: int, target_levels: int, lr_features: float = 1e-2,
                 lr_mlp: float = 1e-3, gamma: float = 0.9999, beta1: float = 0.9, beta2: float = 0.999,
                 eps: float = 1e-8, s_max: float | None = None, lod_input: bool = True, unconstrained: bool = False,
                 is_signed: bool = False, literal: bool = False, batch_grid: int = 0):
        z = torch.zeros_like
        self.params, self.partition = list(params), list(partition)
        self.grads = [z(p) for p in params]
        self.m = [z(p) for p in params]
        self.v = [z(p) for p in params]
        self.W, self.b = W, b
        self.W_grad, self.b_grad = z(W), z(b)
        self.W_m, self.W_v, self.b_m, self.b_v = z(W), z(W), z(b), z(b)
        self.target = (target8, target1)
        d = _TrainerDesc()
        d.num_textures = len(params)
        for t in range(len(params)):
            d.res[t], d.levels[t] = int(res[t]), int(levels[t])
            d.d_params[t] = _ptr(params[t])
            d.d_partition[t] = _ptr(partition[t]) if partition[t] is not None else None
            d.d_grad[t] = _ptr(self.grads[t])
            d.d_adam_m[t] = _ptr(self.m[t])
            d.d_adam_v[t] = _ptr(self.v[t])
        d.res_ref = int(res_ref)
        d.lod_input = int(lod_input)
        d.n_layers = len(dims) - 1
        for i, x in enumerate(dims):
            d.dims[i] = int(x)
        for name, t in (("d_W", W), ("d_b", b), ("d_W_grad", self.W_grad), ("d_b_grad", self.b_grad),
                        ("d_W_m", self.W_m), ("d_W_v", self.W_v), ("d_b_m", self.b_m), ("d_b_v", self.b_v)):
            setattr(d, name, _ptr(t))
        d.target_res, d.target_levels = int(target_res), int(target_levels)
        d.d_target8, d.d_target1 = _ptr(target8), _ptr(target1)
        d.lr_features, d.lr_mlp, d.gamma = lr_features, lr_mlp, gamma
        d.beta1, d.beta2, d.eps = beta1, beta2, eps
        d.s_max = float(target_levels - 1 if s_max is None else s_max)
        d.unconstrained = int(unconstrained)
        d.is_signed, d.literal = int(is_signed), int(literal)
        d.batch_grid = int(batch_grid)
        self.unconstrained = bool(unconstrained)
        h = c_void_p()
        _check(lib().bcf_trainer_create(ctypes.byref(d), ctypes.byref(h)), "bcf_trainer_create")
        self.handle = h
        self.dims = list(dims)
        self.loss = torch.zeros(1, dtype=torch.float32, device=W.device)

    def state_dict(self) -> dict:
        """Checkpoint of the trainable state: block parameters (or free texels), partitions, MLP weights and both
        Adam moments, as CPU copies.  The step counter is the caller's (bcf_train_step takes it per call), and
        the batch draws are a function of (seed, step), so a run resumed at step t draws what it would have."""
        cpu = lambda xs: [x.detach().cpu().clone() for x in xs]
        return {"params": cpu(self.params), "m": cpu(self.m), "v": cpu(self.v),
                "partition": [None if k is None else k.detach().cpu().clone() for k in self.partition],
                "W": self.W.detach().cpu().clone(), "b": self.b.detach().cpu().clone(),
                "W_m": self.W_m.detach().cpu().clone(), "W_v": self.W_v.detach().cpu().clone(),
                "b_m": self.b_m.detach().cpu().clone(), "b_v": self.b_v.detach().cpu().clone()}

    def load_state_dict(self, state: dict) -> None:
        """Restore a state_dict() into this trainer's buffers in place (same sizes); gradients are zeroed."""
        for dst, src in zip(self.params + self.m + self.v, state["params"] + state["m"] + state["v"]):
            dst.copy_(src)
        for dst, src in zip(self.partition, state["partition"]):
            if dst is not None:
                dst.copy_(src)
        for name in ("W", "b", "W_m", "W_v", "b_m", "b_v"):
            getattr(self, name).copy_(state[name])
        self.zero_grad()

    def close(self):
        if self.handle:
            _check(lib().bcf_trainer_destroy(self.handle), "bcf_trainer_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, batch: int, seed: int, step: int, u=None, v=None, s=None) -> torch.Tensor:
        """bcf_train_step; returns the (device) loss of the batch."""
        _check(lib().bcf_train_step(self.handle, int(batch), int(seed), int(step), _ptr(u), _ptr(v), _ptr(s),
                                    _ptr(self.loss), _stream()), "bcf_train_step")
        return self.loss

    def step_noalloc(self, batch: int, seed: int, step: int, u=None, v=None, s=None) -> torch.Tensor:
        """bcf_train_step_noalloc: the same step with the gradient scratch in the library's device array."""
        _check(lib().bcf_train_step_noalloc(self.handle, int(batch), int(seed), int(step), _ptr(u), _ptr(v),
                                            _ptr(s), _ptr(self.loss), _stream()), "bcf_train_step_noalloc")
        return self.loss

    def forward(self, u, v, s) -> torch.Tensor:
        out = torch.empty((u.numel(), self.dims[-1]), dtype=torch.float32, device=u.device)
        _check(lib().bcf_train_forward(self.handle, _ptr(u), _ptr(v), _ptr(s), u.numel(), _ptr(out), _stream()),
               "bcf_train_forward")
        return out

    def backward(self, u, v, s, grad_out: torch.Tensor) -> None:
        _check(lib().bcf_train_backward(self.handle, _ptr(u), _ptr(v), _ptr(s), u.numel(),
                                        _ptr(grad_out.contiguous()), _stream()), "bcf_train_backward")

    def zero_grad(self) -> None:
        for g in self.grads + [self.W_grad, self.b_grad]:
            g.zero_()

    def export(self):
        """bcf_train_export -> (BC6H mode-10 blocks per texture as uint8 [blocks*16], FP16 weights as int16)."""
        blocks = [torch.empty(p.shape[0] * 16, dtype=torch.uint8, device=p.device) for p in self.params]
        arr = (c_void_p * MAX_TEX)(*[b.data_ptr() for b in blocks])
        w16 = torch.empty(self.W.numel(), dtype=torch.int16, device=self.W.device)
        _check(lib().bcf_train_export(self.handle, arr, _ptr(w16), _stream()), "bcf_train_export")
        return blocks, w16


class BCfTrainFn(torch.autograd.Function):
    """G(u, v, s) of a trainer's block-compressed material as a differentiable function of its block parameters
    and MLP weights: forward = bcf_train_forward, backward = bcf_train_backward (hand-written kernels)."""

    @staticmethod
    def forward(ctx, trainer: Trainer, u, v, s, W, b, *params):
        ctx.trainer = trainer
        ctx.save_for_backward(u, v, s)
        return trainer.forward(u, v, s)

    @staticmethod
    def backward(ctx, grad_out):
        tr = ctx.trainer
        u, v, s = ctx.saved_tensors
        tr.zero_grad()
        tr.backward(u, v, s, grad_out.float())
        return (None, None, None, None, tr.W_grad.clone(), tr.b_grad.clone(), *[g.clone() for g in tr.grads])
