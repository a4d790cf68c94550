"""Python access to the plain CPU oracle (``oracle/bcf_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, obviously-correct FP64 /
integer restatement of the BCf decode and training path of "Real-Time Neural
Materials using Block-Compressed Features" (arXiv 2311.16121) that the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package; the
product path (``paper_2311_16121_b300``) never does, and this package never
imports the product path.

Every wrapper converts numpy arrays to pointers and calls the C function of
the same name; no arithmetic of the method lives in this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from ctypes import POINTER, c_double, c_float, c_int, c_int64, c_uint8, c_uint16, c_uint32, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bcf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MAX_TEX = 16
MAX_LAYERS = 8
PREC = {"fp32": 0, "fp16": 1, "bf16": 2, "fp8": 3}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/liboracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class _Material(ctypes.Structure):
    _fields_ = [("n_tex", c_int), ("res", c_int * MAX_TEX), ("levels", c_int * MAX_TEX),
                ("blocks", c_void_p * MAX_TEX), ("res_ref", c_int), ("is_signed", c_int), ("wrap", c_int),
                ("lod_input", c_int)]


class _Mlp(ctypes.Structure):
    _fields_ = [("n_layers", c_int), ("dims", c_int * (MAX_LAYERS + 1)), ("precision", c_int),
                ("weights", c_void_p), ("biases", c_void_p), ("act_scale", c_void_p), ("w_scale", c_void_p)]


class _TrainFeatures(ctypes.Structure):
    _fields_ = [("n_tex", c_int), ("res", c_int * MAX_TEX), ("levels", c_int * MAX_TEX),
                ("params", c_void_p * MAX_TEX), ("partition", c_void_p * MAX_TEX), ("res_ref", c_int),
                ("lod_input", c_int), ("free_texels", c_int), ("is_signed", c_int), ("literal", c_int)]


class _Target(ctypes.Structure):
    _fields_ = [("res", c_int), ("levels", c_int), ("rgba8", c_void_p), ("ch8", c_void_p)]


class _TrainMlp(ctypes.Structure):
    _fields_ = [("n_layers", c_int), ("dims", c_int * (MAX_LAYERS + 1)), ("W", c_void_p), ("b", c_void_p),
                ("bf16", c_int)]


class _TrainGrads(ctypes.Structure):
    _fields_ = [("feat_grad", c_void_p * MAX_TEX), ("W_grad", c_void_p), ("b_grad", c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.oracle_half_to_double.restype = c_double
        L.oracle_half_to_double.argtypes = [c_uint16]
        L.oracle_bf16_to_double.restype = c_double
        L.oracle_bf16_to_double.argtypes = [c_uint16]
        L.oracle_e4m3_to_double.restype = c_double
        L.oracle_e4m3_to_double.argtypes = [c_uint8]
        for name in ("oracle_round_half", "oracle_round_bf16", "oracle_round_e4m3", "oracle_round_f32", "oracle_eq9",
                     "oracle_eq9_slope"):
            getattr(L, name).restype = c_double
            getattr(L, name).argtypes = [c_double]
        L.oracle_bc6h_decode_block.restype = c_int
        L.oracle_bc6h_decode_block.argtypes = [c_void_p, c_int, c_void_p]
        L.oracle_bc6h_block_mode.restype = c_int
        L.oracle_bc6h_block_mode.argtypes = [c_void_p]
        L.oracle_bc6h_decode_image.restype = None
        L.oracle_bc6h_decode_image.argtypes = [c_void_p, c_int, c_int, c_int, c_void_p]
        L.oracle_bc6h_encode_fields.restype = None
        L.oracle_bc6h_encode_fields.argtypes = [c_int, c_void_p, c_int, c_void_p, c_void_p]
        L.oracle_bc6h_mode_info.restype = None
        L.oracle_bc6h_mode_info.argtypes = [c_int, c_void_p]
        L.oracle_bc6h_header_bits.restype = c_int
        L.oracle_bc6h_header_bits.argtypes = [c_int]
        L.oracle_bc6h_partition_region.restype = c_int
        L.oracle_bc6h_partition_region.argtypes = [c_int, c_int]
        L.oracle_bc6h_anchor2.restype = c_int
        L.oracle_bc6h_anchor2.argtypes = [c_int]
        L.oracle_bc6h_weight.restype = c_int
        L.oracle_bc6h_weight.argtypes = [c_int, c_int]
        L.oracle_sample_features.restype = None
        L.oracle_sample_features.argtypes = [POINTER(_Material), c_int64, c_void_p, c_void_p, c_void_p, c_void_p]
        L.oracle_decode_mt.restype = None
        L.oracle_decode_mt.argtypes = [POINTER(_Material), POINTER(_Mlp), c_int64, c_void_p, c_void_p, c_void_p, c_int,
                                       c_void_p, c_int]
        L.oracle_mlp_one.restype = None
        L.oracle_mlp_one.argtypes = [POINTER(_Mlp), c_void_p, c_int, c_void_p]
        L.oracle_philox4x32_10.restype = None
        L.oracle_philox4x32_10.argtypes = [c_void_p, c_void_p, c_void_p]
        L.oracle_train_query.restype = None
        L.oracle_train_query.argtypes = [c_uint64, c_uint64, c_int64, c_float, POINTER(c_float), POINTER(c_float),
                                         POINTER(c_float)]
        L.oracle_train_query_grid.restype = None
        L.oracle_train_query_grid.argtypes = [c_uint64, c_uint64, c_int64, c_int, c_float, POINTER(c_float),
                                              POINTER(c_float), POINTER(c_float)]
        L.oracle_train_texel.restype = c_double
        L.oracle_train_texel.argtypes = [c_void_p, c_int, c_int, c_int]
        L.oracle_train_texel_relaxed.restype = c_double
        L.oracle_train_texel_relaxed.argtypes = [c_void_p, c_int, c_int, c_int]
        L.oracle_train_texel_grad.restype = None
        L.oracle_train_texel_grad.argtypes = [c_void_p, c_int, c_int, c_int, c_int, c_void_p]
        L.oracle_train_features_one.restype = None
        L.oracle_train_features_one.argtypes = [POINTER(_TrainFeatures), c_float, c_float, c_float, c_int, c_void_p]
        L.oracle_target_sample.restype = None
        L.oracle_target_sample.argtypes = [POINTER(_Target), c_float, c_float, c_float, c_void_p]
        L.oracle_train_loss_grad.restype = c_double
        L.oracle_train_loss_grad.argtypes = [POINTER(_TrainFeatures), POINTER(_TrainMlp), POINTER(_Target), c_int64,
                                             c_void_p, c_void_p, c_void_p, c_int, c_void_p]
        L.oracle_train_outputs.restype = None
        L.oracle_train_outputs.argtypes = [POINTER(_TrainFeatures), POINTER(_TrainMlp), c_int64, c_void_p, c_void_p,
                                           c_void_p, c_void_p]
        L.oracle_train_backward_given.restype = None
        L.oracle_train_backward_given.argtypes = [POINTER(_TrainFeatures), POINTER(_TrainMlp), c_int64, c_void_p,
                                                  c_void_p, c_void_p, c_void_p, c_void_p]
        L.oracle_texture_blocks.restype = c_int64
        L.oracle_texture_blocks.argtypes = [c_int, c_int]
        L.oracle_train_texel_v.restype = c_double
        L.oracle_train_texel_v.argtypes = [c_void_p, c_int, c_int, c_int, c_int, c_int, c_int]
        L.oracle_train_texel_grad_v.restype = None
        L.oracle_train_texel_grad_v.argtypes = [c_void_p, c_int, c_int, c_int, c_int, c_int, c_int, c_void_p]
        L.oracle_train_export_block_v.restype = None
        L.oracle_train_export_block_v.argtypes = [c_void_p, c_int, c_int, c_void_p]
        L.oracle_train_export_block.restype = None
        L.oracle_train_export_block.argtypes = [c_void_p, c_int, c_void_p]
        L.oracle_encode_mode10_block.restype = None
        L.oracle_encode_mode10_block.argtypes = [c_void_p, c_void_p, POINTER(c_int), POINTER(c_double), c_void_p]
        L.oracle_encode_mode10_texture.restype = None
        L.oracle_encode_mode10_texture.argtypes = [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p]
        L.oracle_train_loss_mt.restype = c_double
        L.oracle_train_loss_mt.argtypes = [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_int]
        L.oracle_encode_mode11_block.restype = None
        L.oracle_encode_mode11_block.argtypes = [c_void_p, c_void_p, c_void_p, POINTER(c_double)]
        L.oracle_compress_bc6h_block.restype = None
        L.oracle_compress_bc6h_block.argtypes = [c_void_p, c_void_p, POINTER(c_double), POINTER(c_int)]
        L.oracle_encode_fit_segment.restype = None
        L.oracle_encode_fit_segment.argtypes = [c_void_p, c_int, c_int, c_void_p, c_void_p]
        L.oracle_compress_bc6h_texture.restype = None
        L.oracle_compress_bc6h_texture.argtypes = [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p]
        L.oracle_mlp_explain.restype = c_int
        L.oracle_mlp_explain.argtypes = [POINTER(_Mlp), c_void_p, c_void_p, c_void_p, c_double, c_int, ctypes.c_long]
        L.oracle_train_mlp_explain.restype = c_int
        L.oracle_train_mlp_explain.argtypes = [POINTER(_TrainMlp), c_void_p, c_void_p, c_void_p, c_double,
                                               ctypes.c_long]
        L.oracle_train_backward_bounds.restype = None
        L.oracle_train_backward_bounds.argtypes = [POINTER(_TrainFeatures), POINTER(_TrainMlp), c_int64, c_void_p,
                                                   c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
        L.oracle_adam.restype = None
        L.oracle_adam.argtypes = [c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_double, c_double, c_double,
                                  c_double, c_double, c_double, c_double]
    return _lib


def _ptr(a: np.ndarray | None) -> int | None:
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data


# --------------------------------------------------------------------------- scalars / formats

def half_to_double(h: int) -> float:
    return lib().oracle_half_to_double(int(h))


def bf16_to_double(h: int) -> float:
    return lib().oracle_bf16_to_double(int(h))


def e4m3_to_double(b: int) -> float:
    return lib().oracle_e4m3_to_double(int(b))


def round_half(x: float) -> float:
    return lib().oracle_round_half(float(x))


def round_bf16(x: float) -> float:
    return lib().oracle_round_bf16(float(x))


def round_e4m3(x: float) -> float:
    return lib().oracle_round_e4m3(float(x))


def eq9(y: float) -> float:
    return lib().oracle_eq9(float(y))


def eq9_slope(y: float) -> float:
    return lib().oracle_eq9_slope(float(y))


# --------------------------------------------------------------------------- BC6H

def bc6h_decode_block(block: bytes | np.ndarray, is_signed: bool = False) -> tuple[int, np.ndarray]:
    """Returns (mode 1..14 or 0 for reserved, [16, 3] uint16 half bits)."""
    blk = np.ascontiguousarray(np.frombuffer(bytes(block), dtype=np.uint8) if not isinstance(block, np.ndarray)
                               else block.astype(np.uint8).reshape(16))
    out = np.zeros((16, 3), dtype=np.uint16)
    mode = lib().oracle_bc6h_decode_block(_ptr(blk), int(is_signed), _ptr(out))
    return mode, out


def bc6h_block_mode(block) -> int:
    blk = np.ascontiguousarray(np.asarray(block, dtype=np.uint8).reshape(16))
    return lib().oracle_bc6h_block_mode(_ptr(blk))


def bc6h_decode_image(blocks: np.ndarray, blocks_w: int, blocks_h: int, is_signed: bool = False) -> np.ndarray:
    """blocks: uint8 [blocks_h * blocks_w * 16] -> uint16 [4*bh, 4*bw, 3] half bits."""
    blk = np.ascontiguousarray(blocks, dtype=np.uint8).reshape(-1)
    assert blk.size >= blocks_w * blocks_h * 16
    out = np.zeros((4 * blocks_h, 4 * blocks_w, 3), dtype=np.uint16)
    lib().oracle_bc6h_decode_image(_ptr(blk), blocks_w, blocks_h, int(is_signed), _ptr(out))
    return out


def bc6h_encode_fields(mode: int, raw: list[int], partition: int, indices: list[int]) -> np.ndarray:
    """Pack stored endpoint fields (w,x,y,z x r,g,b), partition and indices into a block."""
    r = np.ascontiguousarray(np.asarray(raw, dtype=np.int32).reshape(12))
    idx = np.ascontiguousarray(np.asarray(indices, dtype=np.int32).reshape(16))
    out = np.zeros(16, dtype=np.uint8)
    lib().oracle_bc6h_encode_fields(int(mode), _ptr(r), int(partition), _ptr(idx), _ptr(out))
    return out


def bc6h_mode_info(mode: int) -> dict:
    info = np.zeros(7, dtype=np.int32)
    lib().oracle_bc6h_mode_info(int(mode), _ptr(info))
    return {"code": int(info[0]), "regions": int(info[1]), "transformed": bool(info[2]), "epb": int(info[3]),
            "delta": (int(info[4]), int(info[5]), int(info[6]))}


def bc6h_header_bits(mode: int) -> int:
    return lib().oracle_bc6h_header_bits(int(mode))


def bc6h_partition_region(k: int, texel: int) -> int:
    return lib().oracle_bc6h_partition_region(int(k), int(texel))


def bc6h_anchor2(k: int) -> int:
    return lib().oracle_bc6h_anchor2(int(k))


def bc6h_weight(index_bits: int, index: int) -> int:
    return lib().oracle_bc6h_weight(int(index_bits), int(index))


# --------------------------------------------------------------------------- materials and decode

class Material:
    """Oracle view of a BCf material: textures (host block arrays) + layout facts."""

    def __init__(self, blocks: list[np.ndarray], res: list[int], levels: list[int], res_ref: int,
                 is_signed: bool = False, wrap: bool = True, lod_input: bool = True):
        assert len(blocks) == len(res) == len(levels) <= MAX_TEX
        self._keep = [np.ascontiguousarray(b, dtype=np.uint8).reshape(-1) for b in blocks]
        m = _Material()
        m.n_tex = len(blocks)
        for t in range(len(blocks)):
            m.res[t] = int(res[t])
            m.levels[t] = int(levels[t])
            m.blocks[t] = self._keep[t].ctypes.data
        m.res_ref = int(res_ref)
        m.is_signed = int(is_signed)
        m.wrap = int(wrap)
        m.lod_input = int(lod_input)
        self.c = m
        self.n_tex = len(blocks)
        self.lod_input = bool(lod_input)


class Mlp:
    """Oracle view of the MLP: dims, stored weights in their format, FP32 biases, FP8 scales."""

    def __init__(self, dims: list[int], precision: str, weights: np.ndarray, biases: np.ndarray,
                 act_scale: np.ndarray | None = None, w_scale: np.ndarray | None = None):
        assert len(dims) - 1 <= MAX_LAYERS
        dt = {"fp32": np.float32, "fp16": np.uint16, "bf16": np.uint16, "fp8": np.uint8}[precision]
        self._w = np.ascontiguousarray(weights).view(dt).reshape(-1)
        self._b = np.ascontiguousarray(biases, dtype=np.float32).reshape(-1)
        self._as = None if act_scale is None else np.ascontiguousarray(act_scale, dtype=np.float32)
        self._ws = None if w_scale is None else np.ascontiguousarray(w_scale, dtype=np.float32)
        c = _Mlp()
        c.n_layers = len(dims) - 1
        for i, d in enumerate(dims):
            c.dims[i] = int(d)
        c.precision = PREC[precision]
        c.weights = self._w.ctypes.data
        c.biases = self._b.ctypes.data
        c.act_scale = None if self._as is None else self._as.ctypes.data
        c.w_scale = None if self._ws is None else self._ws.ctypes.data
        self.c = c
        self.dims = list(dims)


def sample_features(mat: Material, u: np.ndarray, v: np.ndarray, s: np.ndarray | None) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float32)
    s = None if s is None else np.ascontiguousarray(s, dtype=np.float32)
    out = np.zeros((u.size, 3 * mat.n_tex), dtype=np.float64)
    lib().oracle_sample_features(ctypes.byref(mat.c), u.size, _ptr(u), _ptr(v), _ptr(s), _ptr(out))
    return out


def decode(mat: Material, mlp: Mlp, u: np.ndarray, v: np.ndarray, s: np.ndarray | None, quant_aware: bool = False,
           threads: int = 1) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float32)
    s = None if s is None else np.ascontiguousarray(s, dtype=np.float32)
    out = np.zeros((u.size, mlp.dims[-1]), dtype=np.float64)
    lib().oracle_decode_mt(ctypes.byref(mat.c), ctypes.byref(mlp.c), u.size, _ptr(u), _ptr(v), _ptr(s),
                           int(quant_aware), _ptr(out), int(threads))
    return out


def mlp_one(mlp: Mlp, x: np.ndarray, quant_aware: bool = False) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(mlp.dims[-1], dtype=np.float64)
    lib().oracle_mlp_one(ctypes.byref(mlp.c), _ptr(x), int(quant_aware), _ptr(out))
    return out


def mlp_explain(mlp: Mlp, x: np.ndarray, x_err: np.ndarray, y_dev: np.ndarray, tol: float, out_half: bool = False,
                max_leaves: int = 1 << 16) -> int:
    """Whether a device output y_dev that misses the tolerance is a rounding flip (oracle_mlp_explain): 1 if a
    combination of the operand roundings that the device's FP32 error windows allow reproduces y_dev within
    tol, 0 if none does, -1 if the enumeration would exceed max_leaves combinations."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    e = np.ascontiguousarray(x_err, dtype=np.float64)
    y = np.ascontiguousarray(y_dev, dtype=np.float64)
    return int(lib().oracle_mlp_explain(ctypes.byref(mlp.c), _ptr(x), _ptr(e), _ptr(y), float(tol), int(out_half),
                                        int(max_leaves)))


def mlp_inputs(mat: Material, u, v, s) -> tuple[np.ndarray, np.ndarray]:
    """Exact (FP64) MLP inputs of queries -- the filtered features, then the LOD input max(s, 0) with NaN read as
    0 when the material has one -- and a bound on the device's FP32 error in each: 2^-21 + 2^-20 |x| for a
    feature (a few single-precision roundings of a sum of at most 8 texels of magnitude <= 1 per channel of
    the test materials), 0 for the LOD input (the same float on both sides)."""
    f = sample_features(mat, u, v, s)
    e = 2.0 ** -21 + 2.0 ** -20 * np.abs(f)
    if mat.lod_input:
        sq = np.zeros(f.shape[0]) if s is None else np.asarray(s, np.float64)
        lod = np.where(np.isnan(sq), 0.0, np.maximum(sq, 0.0))
        f = np.concatenate([f, lod[:, None]], axis=1)
        e = np.concatenate([e, np.zeros((e.shape[0], 1))], axis=1)
    return f, e


def check_outputs(got: np.ndarray, ref_q: np.ndarray, tol: float, out_half: bool, explain) -> dict:
    """Strict comparison of device outputs with the quantisation-aware oracle: every output within tol
    (plus half an FP16 unit of the reference when the device stored FP16) of ref_q, except in rows that
    explain(rows) -> list of mlp_explain results shows to be operand-rounding flips.  Returns counts: outputs
    beyond the tolerance, rows holding them, rows explained as flips, the unexplained rows (which fail a
    test), and the per-channel maximum error."""
    got = np.asarray(got, np.float64)
    ref_q = np.asarray(ref_q, np.float64)
    if out_half:
        ref_q = ref_q.astype(np.float16).astype(np.float64)
    t = tol + (np.abs(ref_q) * 2.0 ** -11 if out_half else 0.0)
    err = np.abs(got - ref_q)
    beyond = ~(err <= t)
    rows = np.nonzero(beyond.any(axis=1))[0]
    kinds = explain(rows) if rows.size else []
    unexplained = [int(r) for r, k in zip(rows, kinds) if k != 1]
    return {"outputs": int(got.size), "beyond_tol": int(beyond.sum()), "rows_beyond": int(rows.size),
            "flips": int(rows.size - len(unexplained)), "unexplained": unexplained,
            "worst": err.max(axis=0) if err.size else np.zeros(0)}


def decode_explainer(mat: Material, mlp: Mlp, u, v, s, got: np.ndarray, tol: float, out_half: bool):
    """explain(rows) for check_outputs on a decode: mlp_explain of each row with its exact inputs."""
    def explain(rows):
        su = None if s is None else np.asarray(s)[rows]
        x, e = mlp_inputs(mat, np.asarray(u)[rows], np.asarray(v)[rows], su)
        return [mlp_explain(mlp, x[i], e[i], np.asarray(got, np.float64)[r], tol, out_half)
                for i, r in enumerate(rows)]
    return explain


# --------------------------------------------------------------------------- random draws

def philox4x32_10(ctr: list[int], key: list[int]) -> list[int]:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    o = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return [int(x) for x in o]


def train_queries(seed: int, step: int, batch: int, s_max: float,
                  grid: int = 0) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """The step's batch draws: independent (u, v, s) per query, or (grid > 0) a grid x grid uv grid with one
    offset and one s per batch."""
    u = np.zeros(batch, np.float32)
    v = np.zeros(batch, np.float32)
    s = np.zeros(batch, np.float32)
    L = lib()
    cu, cv, cs = c_float(), c_float(), c_float()
    for q in range(batch):
        if grid:
            L.oracle_train_query_grid(seed, step, q, grid, s_max, ctypes.byref(cu), ctypes.byref(cv),
                                      ctypes.byref(cs))
        else:
            L.oracle_train_query(seed, step, q, s_max, ctypes.byref(cu), ctypes.byref(cv), ctypes.byref(cs))
        u[q], v[q], s[q] = cu.value, cv.value, cs.value
    return u, v, s


# --------------------------------------------------------------------------- training

def train_texel(p: np.ndarray, k: int, texel: int, channel: int) -> float:
    """Straight-through emulated BC6 mode-10 texel value (block params p[28])."""
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(28)
    return lib().oracle_train_texel(_ptr(p), int(k), int(texel), int(channel))


def train_texel_relaxed(p: np.ndarray, k: int, texel: int, channel: int) -> float:
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(28)
    return lib().oracle_train_texel_relaxed(_ptr(p), int(k), int(texel), int(channel))


def train_texel_grad(p: np.ndarray, k: int, texel: int, channel: int, relaxed: bool) -> np.ndarray:
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(28)
    g = np.zeros(28, np.float64)
    lib().oracle_train_texel_grad(_ptr(p), int(k), int(texel), int(channel), int(relaxed), _ptr(g))
    return g


class TrainFeatures:
    """Block-parameterised feature textures: params [blocks, 28] (float64) and partition ids per texture; or,
    with free=True, unconstrained features: params [texels, 3] per texture and no partitions."""

    def __init__(self, params: list[np.ndarray], partition: list[np.ndarray] | None, res: list[int],
                 levels: list[int], res_ref: int, lod_input: bool = True, free: bool = False, is_signed: bool = False,
                 literal: bool = False):
        self._p = [np.ascontiguousarray(p, dtype=np.float64).reshape(-1) for p in params]
        self._k = [np.ascontiguousarray(k, dtype=np.uint8).reshape(-1) for k in partition] if not free else \
            [np.zeros(1, np.uint8) for _ in params]
        c = _TrainFeatures()
        c.n_tex = len(params)
        for t in range(len(params)):
            c.res[t] = int(res[t])
            c.levels[t] = int(levels[t])
            c.params[t] = self._p[t].ctypes.data
            c.partition[t] = self._k[t].ctypes.data
        c.res_ref = int(res_ref)
        c.lod_input = int(lod_input)
        c.free_texels = int(free)
        c.is_signed = int(is_signed)
        c.literal = int(literal)
        self.free = free
        self.c = c
        self.n_tex = len(params)


class Target:
    """Reference material mip chain: channels 0..7 interleaved and channel 8 separate, FP16 bits."""

    def __init__(self, rgba8: np.ndarray, ch8: np.ndarray, res: int, levels: int):
        self._a = np.ascontiguousarray(rgba8).view(np.uint16).reshape(-1)
        self._b = np.ascontiguousarray(ch8).view(np.uint16).reshape(-1)
        c = _Target()
        c.res = int(res)
        c.levels = int(levels)
        c.rgba8 = self._a.ctypes.data
        c.ch8 = self._b.ctypes.data
        self.c = c


class TrainMlp:
    def __init__(self, dims: list[int], W: np.ndarray, b: np.ndarray, bf16: bool = True):
        self._W = np.ascontiguousarray(W, dtype=np.float64).reshape(-1)
        self._b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
        c = _TrainMlp()
        c.n_layers = len(dims) - 1
        for i, d in enumerate(dims):
            c.dims[i] = int(d)
        c.W = self._W.ctypes.data
        c.b = self._b.ctypes.data
        c.bf16 = int(bf16)
        self.c = c
        self.dims = list(dims)


def train_features_one(F: TrainFeatures, u: float, v: float, s: float, relaxed: bool = False) -> np.ndarray:
    out = np.zeros(3 * F.n_tex, np.float64)
    lib().oracle_train_features_one(ctypes.byref(F.c), u, v, s, int(relaxed), _ptr(out))
    return out


def target_sample(T: Target, u: float, v: float, s: float) -> np.ndarray:
    out = np.zeros(9, np.float64)
    lib().oracle_target_sample(ctypes.byref(T.c), u, v, s, _ptr(out))
    return out


def train_loss_grad(F: TrainFeatures, P: TrainMlp, T: Target, u, v, s, want_grad: bool = True,
                    relaxed: bool = False):
    """Returns (loss, feature grads per texture [blocks, 28], W grad, b grad) (all float64)."""
    u = np.ascontiguousarray(u, np.float32)
    v = np.ascontiguousarray(v, np.float32)
    s = np.ascontiguousarray(s, np.float32)
    gf = [np.zeros_like(p) for p in F._p]
    gW = np.zeros(P._W.size, np.float64)
    gb = np.zeros(P._b.size, np.float64)
    G = _TrainGrads()
    for t, g in enumerate(gf):
        G.feat_grad[t] = g.ctypes.data
    G.W_grad = gW.ctypes.data
    G.b_grad = gb.ctypes.data
    loss = lib().oracle_train_loss_grad(ctypes.byref(F.c), ctypes.byref(P.c), ctypes.byref(T.c), u.size, _ptr(u),
                                        _ptr(v), _ptr(s), int(relaxed), ctypes.byref(G) if want_grad else None)
    return loss, [g.reshape(-1, 3 if F.free else 28) for g in gf], gW, gb


def train_loss_mt(F: TrainFeatures, P: TrainMlp, T: Target, u, v, s, threads: int | None = None) -> float:
    """The loss of train_loss_grad without gradients, the queries split over POSIX threads (for full-size
    batches)."""
    u = np.ascontiguousarray(u, np.float32)
    v = np.ascontiguousarray(v, np.float32)
    s = np.ascontiguousarray(s, np.float32)
    return lib().oracle_train_loss_mt(ctypes.byref(F.c), ctypes.byref(P.c), ctypes.byref(T.c), u.size, _ptr(u),
                                      _ptr(v), _ptr(s), int(threads or os.cpu_count() or 1))


def adam(p: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, t: int, lr0: float, gamma: float,
         beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, lo: float = 1.0, hi: float = 0.0) -> None:
    """In-place Adam step on float64 arrays (lo > hi: no clamp)."""
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    lib().oracle_adam(p.size, _ptr(p), _ptr(g), _ptr(m), _ptr(v), int(t), lr0, gamma, beta1, beta2, eps, lo, hi)


def texture_blocks(res: int, levels: int) -> int:
    return int(lib().oracle_texture_blocks(int(res), int(levels)))


def train_export_block(p: np.ndarray, k: int, is_signed: bool = False) -> np.ndarray:
    """Mode-10 BC6H block of trained block parameters (with the anchor fix-up); SF16 when is_signed."""
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(28)
    out = np.zeros(16, np.uint8)
    lib().oracle_train_export_block_v(_ptr(p), int(k), int(is_signed), _ptr(out))
    return out


def train_texel_v(p: np.ndarray, k: int, texel: int, channel: int, is_signed: bool = False, literal: bool = False,
                  relaxed: bool = False) -> float:
    """One emulated texel channel: UF16 or SF16, the format's exact steps or Eq. 7-8 as printed, STE or relaxed."""
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(28)
    return lib().oracle_train_texel_v(_ptr(p), int(k), int(texel), int(channel), int(is_signed), int(literal),
                                      int(relaxed))


def train_texel_grad_v(p: np.ndarray, k: int, texel: int, channel: int, is_signed: bool = False,
                       literal: bool = False, relaxed: bool = False) -> np.ndarray:
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(28)
    g = np.zeros(28, np.float64)
    lib().oracle_train_texel_grad_v(_ptr(p), int(k), int(texel), int(channel), int(is_signed), int(literal),
                                    int(relaxed), _ptr(g))
    return g


def train_outputs(F: TrainFeatures, P: TrainMlp, u, v, s) -> np.ndarray:
    u = np.ascontiguousarray(u, np.float32)
    v = np.ascontiguousarray(v, np.float32)
    s = np.ascontiguousarray(s, np.float32)
    out = np.zeros((u.size, P.dims[-1]), np.float64)
    lib().oracle_train_outputs(ctypes.byref(F.c), ctypes.byref(P.c), u.size, _ptr(u), _ptr(v), _ptr(s), _ptr(out))
    return out


def train_backward_given(F: TrainFeatures, P: TrainMlp, u, v, s, grad_out):
    """Gradients (feature grads per texture [blocks, 28], W grad, b grad) for a given dL/dG [n][C]."""
    u = np.ascontiguousarray(u, np.float32)
    v = np.ascontiguousarray(v, np.float32)
    s = np.ascontiguousarray(s, np.float32)
    go = np.ascontiguousarray(grad_out, np.float64)
    gf = [np.zeros_like(p) for p in F._p]
    gW = np.zeros(P._W.size, np.float64)
    gb = np.zeros(P._b.size, np.float64)
    G = _TrainGrads()
    for t, g in enumerate(gf):
        G.feat_grad[t] = g.ctypes.data
    G.W_grad = gW.ctypes.data
    G.b_grad = gb.ctypes.data
    lib().oracle_train_backward_given(ctypes.byref(F.c), ctypes.byref(P.c), u.size, _ptr(u), _ptr(v), _ptr(s),
                                      _ptr(go), ctypes.byref(G))
    return [g.reshape(-1, 3 if F.free else 28) for g in gf], gW, gb


def train_mlp_explain(P: TrainMlp, x: np.ndarray, x_err: np.ndarray, y_dev: np.ndarray, tol: float,
                      max_leaves: int = 1 << 16) -> int:
    """mlp_explain for the training network (bfloat16 operands, FP32 outputs)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    e = np.ascontiguousarray(x_err, dtype=np.float64)
    y = np.ascontiguousarray(y_dev, dtype=np.float64)
    return int(lib().oracle_train_mlp_explain(ctypes.byref(P.c), _ptr(x), _ptr(e), _ptr(y), float(tol),
                                              int(max_leaves)))


def train_explainer(F: TrainFeatures, P: TrainMlp, u, v, s, got: np.ndarray, tol: float, lod_input: bool = True):
    """explain(rows) for check_outputs on a training forward (emulated features, bfloat16 network)."""
    def explain(rows):
        out = []
        for r in rows:
            f = train_features_one(F, float(u[r]), float(v[r]), float(s[r]))
            e = 2.0 ** -21 + 2.0 ** -20 * np.abs(f)
            if lod_input:
                sq = float(s[r])
                f = np.append(f, 0.0 if np.isnan(sq) else max(sq, 0.0))
                e = np.append(e, 0.0)
            out.append(train_mlp_explain(P, f, e, np.asarray(got, np.float64)[r], tol))
        return out
    return explain


def train_backward_bounds(F: TrainFeatures, P: TrainMlp, u, v, s, grad_out):
    """Per-element bounds of the device gradients (oracle_train_backward_bounds): (A, R), each as
    (feature arrays per texture, W array, b array) in the layout of train_backward_given; the device gradient
    lies within c A + R of the oracle's."""
    u = np.ascontiguousarray(u, np.float32)
    v = np.ascontiguousarray(v, np.float32)
    s = np.ascontiguousarray(s, np.float32)
    go = np.ascontiguousarray(grad_out, np.float64)
    out = []
    Gs = []
    for _ in range(2):
        gf = [np.zeros_like(p) for p in F._p]
        gW = np.zeros(P._W.size, np.float64)
        gb = np.zeros(P._b.size, np.float64)
        G = _TrainGrads()
        for t, g in enumerate(gf):
            G.feat_grad[t] = g.ctypes.data
        G.W_grad = gW.ctypes.data
        G.b_grad = gb.ctypes.data
        out.append((gf, gW, gb))
        Gs.append(G)
    lib().oracle_train_backward_bounds(ctypes.byref(F.c), ctypes.byref(P.c), u.size, _ptr(u), _ptr(v), _ptr(s),
                                       _ptr(go), ctypes.byref(Gs[0]), ctypes.byref(Gs[1]))
    return tuple(([g.reshape(-1, 3 if F.free else 28) for g in gf], gW, gb) for gf, gW, gb in out)


# --------------------------------------------------------------------------- mode-10 encoder

def encode_mode10_block(v: np.ndarray) -> tuple[np.ndarray, int, float, np.ndarray]:
    """Encode one 4x4 block of RGB targets (v[16][3], texel t = 4 row + column): block parameters
    (training layout, 28 values), partition, its total error, and the total error of all 32 partitions."""
    v = np.ascontiguousarray(v, dtype=np.float32).reshape(48)
    params = np.zeros(28, np.float64)
    k = ctypes.c_int(0)
    err = ctypes.c_double(0.0)
    errs = np.zeros(32, np.float64)
    lib().oracle_encode_mode10_block(_ptr(v), _ptr(params), ctypes.byref(k), ctypes.byref(err), _ptr(errs))
    return params, int(k.value), float(err.value), errs


def encode_mode10_texture(texels: np.ndarray, res: int, levels: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Encode a mipmapped RGB texture (levels concatenated from level 0, each [W][W][3] float32): block
    parameters [blocks][28], partitions [blocks], errors [blocks]."""
    texels = np.ascontiguousarray(texels, dtype=np.float32).reshape(-1)
    nb = texture_blocks(res, levels)
    params = np.zeros((nb, 28), np.float64)
    part = np.zeros(nb, np.uint8)
    err = np.zeros(nb, np.float64)
    lib().oracle_encode_mode10_texture(_ptr(texels), int(res), int(levels), _ptr(params), _ptr(part), _ptr(err))
    return params, part, err


def encode_fit_segment(y: np.ndarray, k: int, r: int) -> tuple[np.ndarray, np.ndarray]:
    """The encoder's line fit (oracle_encode_fit_segment) of region r of partition k (k < 0: all sixteen
    texels) of interpolation-domain points y[16][3]: the segment ends A, B."""
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(16, 3)
    A = np.zeros(3, np.float64)
    B = np.zeros(3, np.float64)
    lib().oracle_encode_fit_segment(_ptr(y), int(k), int(r), _ptr(A), _ptr(B))
    return A, B


def encode_mode11_block(v: np.ndarray) -> tuple[np.ndarray, np.ndarray, float]:
    """Mode-11 encoding of one 4x4 block of RGB targets (v[16][3]): endpoints e[2][3] (10-bit codes, segment
    start and end), indices [16] (4-bit), total squared error."""
    v = np.ascontiguousarray(v, dtype=np.float32).reshape(48)
    e = np.zeros((2, 3), np.int32)
    idx = np.zeros(16, np.int32)
    err = ctypes.c_double(0.0)
    lib().oracle_encode_mode11_block(_ptr(v), _ptr(e), _ptr(idx), ctypes.byref(err))
    return e, idx, float(err.value)


def compress_bc6h_block(v: np.ndarray) -> tuple[np.ndarray, float, int]:
    """The two-mode (10 / 11) BC6H UF16 compression of one block: (16 bytes, error, mode)."""
    v = np.ascontiguousarray(v, dtype=np.float32).reshape(48)
    blk = np.zeros(16, np.uint8)
    err = ctypes.c_double(0.0)
    mode = ctypes.c_int(0)
    lib().oracle_compress_bc6h_block(_ptr(v), _ptr(blk), ctypes.byref(err), ctypes.byref(mode))
    return blk, float(err.value), int(mode.value)


def compress_bc6h_texture(texels: np.ndarray, res: int, levels: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """The two-mode compression of a mipmapped RGB texture (layout as encode_mode10_texture): blocks
    [blocks][16] uint8, errors [blocks], modes [blocks] (10 or 11)."""
    texels = np.ascontiguousarray(texels, dtype=np.float32).reshape(-1)
    nb = texture_blocks(res, levels)
    blocks = np.zeros((nb, 16), np.uint8)
    err = np.zeros(nb, np.float64)
    modes = np.zeros(nb, np.uint8)
    lib().oracle_compress_bc6h_texture(_ptr(texels), int(res), int(levels), _ptr(blocks), _ptr(err), _ptr(modes))
    return blocks, err, modes
