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
        L.bcf_decode_material.restype = c_int
        L.bcf_decode_material.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_int, c_void_p]
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

def decode_bc6h(blocks: torch.Tensor, blocks_w: int, blocks_h: int, is_signed: bool = False,
                out: torch.Tensor | None = None) -> torch.Tensor:
    """bcf_decode_bc6h: uint8 [bh * bw * 16] blocks -> int16 [4 bh, 4 bw, 3] half bit patterns."""
    if out is None:
        out = torch.empty((4 * blocks_h, 4 * blocks_w, 3), dtype=torch.int16, device=blocks.device)
    _check(lib().bcf_decode_bc6h(_ptr(blocks), blocks_w, blocks_h, int(is_signed), _ptr(out), _stream()),
           "bcf_decode_bc6h")
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

    def set_decode_variant(self, variant: int) -> None:
        """bcf_set_decode_variant: 0 tile-cooperative (default), 1 per-lane."""
        _check(lib().bcf_set_decode_variant(self.handle, int(variant)), "bcf_set_decode_variant")

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
