"""Seeded synthetic inputs for the BCf decode and training workloads.

This module only *draws* inputs: BC6H block bitstreams, query sets, MLP
weights, block parameters and a reference material.  It computes nothing of
the method (no unquantise / interpolate / filter / MLP arithmetic) and is
shared by the tests, the oracle checks and ``bench.py``.  The product path
(libbcf and its binding) does not import it.

Workload shapes stand in for the paper's (Table 1 resolutions and mip
chains, a 9-channel PBR set as in Sec. 6.1, 1-spp screen queries of Table 3
resolutions, random (u, v, s) training batches as in Sec. 5.1); the paper's
Polyhaven materials are not available, so the values are seeded noise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASTER_SEED = 2311161210

# --------------------------------------------------------------------------- BC6H bitstream writer

# Value of the mode field and its width for modes 1..14 (Direct3D BC6H).
MODE_CODE = {1: (0, 2), 2: (1, 2), 3: (2, 5), 4: (6, 5), 5: (10, 5), 6: (14, 5), 7: (18, 5), 8: (22, 5),
             9: (26, 5), 10: (30, 5), 11: (3, 5), 12: (7, 5), 13: (11, 5), 14: (15, 5)}
RESERVED_CODES = (19, 23, 27, 31)

# (endpoint precision, per-channel bits of endpoints 1..3, regions, delta-coded)
MODE_PREC = {1: (10, (5, 5, 5), 2, True), 2: (7, (6, 6, 6), 2, True), 3: (11, (5, 4, 4), 2, True),
             4: (11, (4, 5, 4), 2, True), 5: (11, (4, 4, 5), 2, True), 6: (9, (5, 5, 5), 2, True),
             7: (8, (6, 5, 5), 2, True), 8: (8, (5, 6, 5), 2, True), 9: (8, (5, 5, 6), 2, True),
             10: (6, (6, 6, 6), 2, False), 11: (10, (10, 10, 10), 1, False), 12: (11, (9, 9, 9), 1, True),
             13: (12, (8, 8, 8), 1, True), 14: (16, (4, 4, 4), 1, True)}


def _runs(spec: str):
    """'R0:9-0 G2:4 ...' -> [(endpoint, channel, first_bit, count, step)] in stored order after the mode field.
    Endpoint index 0..3, channel 0..2 (R, G, B); 'P' is the partition field."""
    out = []
    for tok in spec.split():
        name, bits = tok.split(":")
        if "-" in bits:
            a, b = (int(x) for x in bits.split("-"))
        else:
            a = b = int(bits)
        step = 1 if a >= b else -1
        if name == "P":
            out.append((-1, -1, b, abs(a - b) + 1, step))
        else:
            out.append((int(name[1]), "RGB".index(name[0]), b, abs(a - b) + 1, step))
    return out


# Field order after the mode bits (Direct3D BC6H block layouts); R0 = first
# endpoint of region 0, R1 = second, R2/R3 = region 1.
_LAYOUT = {
    1: "G2:4 B2:4 B3:4 R0:9-0 G0:9-0 B0:9-0 R1:4-0 G3:4 G2:3-0 G1:4-0 B3:0 G3:3-0 B1:4-0 B3:1 B2:3-0 R2:4-0 "
       "B3:2 R3:4-0 B3:3 P:4-0",
    2: "G2:5 G3:4 G3:5 R0:6-0 B3:0 B3:1 B2:4 G0:6-0 B2:5 B3:2 G2:4 B0:6-0 B3:3 B3:5 B3:4 R1:5-0 G2:3-0 G1:5-0 "
       "G3:3-0 B1:5-0 B2:3-0 R2:5-0 R3:5-0 P:4-0",
    3: "R0:9-0 G0:9-0 B0:9-0 R1:4-0 R0:10 G2:3-0 G1:3-0 G0:10 B3:0 G3:3-0 B1:3-0 B0:10 B3:1 B2:3-0 R2:4-0 B3:2 "
       "R3:4-0 B3:3 P:4-0",
    4: "R0:9-0 G0:9-0 B0:9-0 R1:3-0 R0:10 G3:4 G2:3-0 G1:4-0 G0:10 G3:3-0 B1:3-0 B0:10 B3:1 B2:3-0 R2:3-0 B3:0 "
       "B3:2 R3:3-0 G2:4 B3:3 P:4-0",
    5: "R0:9-0 G0:9-0 B0:9-0 R1:3-0 R0:10 B2:4 G2:3-0 G1:3-0 G0:10 B3:0 G3:3-0 B1:4-0 B0:10 B2:3-0 R2:3-0 B3:1 "
       "B3:2 R3:3-0 B3:4 B3:3 P:4-0",
    6: "R0:8-0 B2:4 G0:8-0 G2:4 B0:8-0 B3:4 R1:4-0 G3:4 G2:3-0 G1:4-0 B3:0 G3:3-0 B1:4-0 B3:1 B2:3-0 R2:4-0 "
       "B3:2 R3:4-0 B3:3 P:4-0",
    7: "R0:7-0 G3:4 B2:4 G0:7-0 B3:2 G2:4 B0:7-0 B3:3 B3:4 R1:5-0 G2:3-0 G1:4-0 B3:0 G3:3-0 B1:4-0 B3:1 B2:3-0 "
       "R2:5-0 R3:5-0 P:4-0",
    8: "R0:7-0 B3:0 B2:4 G0:7-0 G2:5 G2:4 B0:7-0 G3:5 B3:4 R1:4-0 G3:4 G2:3-0 G1:5-0 G3:3-0 B1:4-0 B3:1 B2:3-0 "
       "R2:4-0 B3:2 R3:4-0 B3:3 P:4-0",
    9: "R0:7-0 B3:1 B2:4 G0:7-0 B2:5 G2:4 B0:7-0 B3:5 B3:4 R1:4-0 G3:4 G2:3-0 G1:4-0 B3:0 G3:3-0 B1:5-0 B2:3-0 "
       "R2:4-0 B3:2 R3:4-0 B3:3 P:4-0",
    10: "R0:5-0 G3:4 B3:0 B3:1 B2:4 G0:5-0 G2:5 B2:5 B3:2 G2:4 B0:5-0 G3:5 B3:3 B3:5 B3:4 R1:5-0 G2:3-0 G1:5-0 "
        "G3:3-0 B1:5-0 B2:3-0 R2:5-0 R3:5-0 P:4-0",
    11: "R0:9-0 G0:9-0 B0:9-0 R1:9-0 G1:9-0 B1:9-0",
    12: "R0:9-0 G0:9-0 B0:9-0 R1:8-0 R0:10 G1:8-0 G0:10 B1:8-0 B0:10",
    13: "R0:9-0 G0:9-0 B0:9-0 R1:7-0 R0:10-11 G1:7-0 G0:10-11 B1:7-0 B0:10-11",
    14: "R0:9-0 G0:9-0 B0:9-0 R1:3-0 R0:10-15 G1:3-0 G0:10-15 B1:3-0 B0:10-15",
}
_RUNS = {m: _runs(s) for m, s in _LAYOUT.items()}

# Second-region anchor texel of the 32 two-region partitions.
_ANCHOR2 = [15] * 17 + [2, 8, 2, 2, 8, 8, 15, 2, 8, 2, 2, 8, 8, 2, 2]


def _put(lo: np.ndarray, hi: np.ndarray, pos: int, nbits: int, val: np.ndarray) -> None:
    """OR `nbits` low bits of `val` into the 128-bit blocks (lo, hi) at bit position `pos`."""
    v = val.astype(np.uint64) & np.uint64((1 << nbits) - 1)
    for j in range(nbits):
        p = pos + j
        bit = (v >> np.uint64(j)) & np.uint64(1)
        if p < 64:
            lo |= bit << np.uint64(p)
        else:
            hi |= bit << np.uint64(p - 64)


def pack_blocks(mode: int, endpoints: np.ndarray, partition: np.ndarray, indices: np.ndarray) -> np.ndarray:
    """Pack n blocks of one mode. endpoints: [n, 4, 3] stored field values (deltas already two's complement),
    partition: [n], indices: [n, 16] (anchor texels must have their top index bit clear). -> uint8 [n, 16]."""
    n = endpoints.shape[0]
    lo = np.zeros(n, np.uint64)
    hi = np.zeros(n, np.uint64)
    code, mbits = MODE_CODE[mode]
    _put(lo, hi, 0, mbits, np.full(n, code))
    pos = mbits
    for ep, ch, first, count, step in _RUNS[mode]:
        src = partition if ep < 0 else endpoints[:, ep, ch]
        for j in range(count):
            b = first + j * step
            _put(lo, hi, pos + j, 1, (src.astype(np.int64) >> b) & 1)
        pos += count
    regions = MODE_PREC[mode][2]
    ib = 3 if regions == 2 else 4
    anchor2 = np.array(_ANCHOR2)[partition] if regions == 2 else np.full(n, -1)
    for t in range(16):
        is_anchor = (t == 0) | (anchor2 == t)
        # anchors carry one bit fewer; write the low bits, with per-block widths
        for j in range(ib):
            write = j < (ib - is_anchor.astype(int))
            bit = ((indices[:, t].astype(np.int64) >> j) & 1) * write
            # position of bit j of texel t: base + sum of widths of earlier texels
            _put_var(lo, hi, _index_pos(regions, anchor2, t) + j, bit, write)
    out = np.empty((n, 16), np.uint8)
    out[:, :8] = lo.view(np.uint8).reshape(n, 8)
    out[:, 8:] = hi.view(np.uint8).reshape(n, 8)
    return out


def _index_pos(regions: int, anchor2: np.ndarray, t: int) -> np.ndarray:
    base, ib = (82, 3) if regions == 2 else (65, 4)
    pos = base + ib * t - (t > 0)
    if regions == 2:
        pos = pos - (anchor2 < t).astype(int)
    return np.asarray(pos)


def _put_var(lo, hi, pos: np.ndarray, bit: np.ndarray, write: np.ndarray) -> None:
    pos = np.broadcast_to(pos, bit.shape).astype(np.int64)
    b = (bit.astype(np.uint64) & np.uint64(1)) * write.astype(np.uint64)
    in_lo = pos < 64
    lo[in_lo] |= b[in_lo] << pos[in_lo].astype(np.uint64)
    hi[~in_lo] |= b[~in_lo] << (pos[~in_lo] - 64).astype(np.uint64)


def random_blocks(rng: np.random.Generator, n: int) -> np.ndarray:
    """n random valid BC6H blocks: mode uniform over the 14 modes, every other bit random. uint8 [n, 16]."""
    out = rng.integers(0, 256, (n, 16), dtype=np.uint8)
    modes = rng.integers(1, 15, n)
    for m in range(1, 15):
        sel = modes == m
        code, mbits = MODE_CODE[m]
        mask = (1 << mbits) - 1
        out[sel, 0] = (out[sel, 0] & ~np.uint8(mask)) | np.uint8(code)
    return out


def bounded_blocks(rng: np.random.Generator, n: int, modes=tuple(range(1, 15)), frac: float = 0.48,
                   signed: bool = False) -> np.ndarray:
    """n BC6H blocks whose endpoints all lie in the lowest `frac` of their mode's range, so every decoded
    texel is at most 1.0 in magnitude for frac <= 0.48.  Unsigned: endpoints in [0, frac 2^epb].  Signed:
    endpoints in [-frac 2^(epb-1), frac 2^(epb-1)], stored as two's complement.  Mode uniform over `modes`;
    partitions and indices random; delta-coded modes get deltas inside both the delta field's range and the
    endpoint bound."""
    out = np.zeros((n, 16), np.uint8)
    mode_of = rng.choice(np.asarray(modes), n)
    for m in modes:
        sel = np.nonzero(mode_of == m)[0]
        k = sel.size
        if k == 0:
            continue
        epb, dbits, regions, delta = MODE_PREC[m]
        emax = int(frac * (1 << (epb - 1 if signed else epb)))
        emin = -emax if signed else 0
        ep = np.zeros((k, 4, 3), np.int64)
        n_ep = 2 * regions
        for c in range(3):
            e0 = rng.integers(emin, emax + 1, k)
            ep[:, 0, c] = e0 & ((1 << epb) - 1)
            for i in range(1, n_ep):
                if delta:
                    d = dbits[c]
                    lo_d = np.maximum(-(1 << (d - 1)), emin - e0)
                    hi_d = np.minimum((1 << (d - 1)) - 1, emax - e0)
                    dv = lo_d + np.floor(rng.random(k) * (hi_d - lo_d + 1)).astype(np.int64)
                    ep[:, i, c] = dv & ((1 << d) - 1)
                else:
                    ep[:, i, c] = rng.integers(emin, emax + 1, k) & ((1 << epb) - 1)
        part = rng.integers(0, 32, k)
        ib = 3 if regions == 2 else 4
        idx = rng.integers(0, 1 << ib, (k, 16))
        idx[:, 0] &= (1 << (ib - 1)) - 1
        if regions == 2:
            a2 = np.array(_ANCHOR2)[part]
            idx[np.arange(k), a2] &= (1 << (ib - 1)) - 1
        out[sel] = pack_blocks(m, ep, part, idx)
    return out


# --------------------------------------------------------------------------- textures

def level_blocks(res: int, levels: int) -> list[int]:
    return [((res >> l) // 4) ** 2 for l in range(levels)]


def full_levels(res: int) -> int:
    """Mip levels down to a single 4x4 block (Table 1: 512 -> 8 levels)."""
    return int(math.log2(res)) - 1


@dataclass
class TextureSet:
    res: list[int]
    levels: list[int]
    blocks: list[np.ndarray]  # uint8 [total_blocks, 16] per texture, mips concatenated from level 0


def make_textures(rng: np.random.Generator, res: list[int], levels: list[int], kind: str = "bounded",
                  pool: int | None = None) -> TextureSet:
    """kind: 'random' (all bits random, any mode) or 'bounded' (values in [0, 1]).  With `pool`, blocks are
    drawn from a pool of that many distinct blocks (for very large texture sets)."""
    gen = random_blocks if kind == "random" else bounded_blocks
    blocks = []
    pool_blocks = gen(rng, pool) if pool else None
    for r, l in zip(res, levels):
        nb = sum(level_blocks(r, l))
        if pool_blocks is not None:
            blocks.append(pool_blocks[rng.integers(0, pool, nb)])
        else:
            blocks.append(gen(rng, nb))
    return TextureSet(list(res), list(levels), blocks)


# --------------------------------------------------------------------------- queries

def uniform_queries(rng: np.random.Generator, n: int, s_range=None):
    u = rng.random(n, dtype=np.float32)
    v = rng.random(n, dtype=np.float32)
    s = None if s_range is None else rng.uniform(s_range[0], s_range[1], n).astype(np.float32)
    return u, v, s


def tile_order(w: int, h: int, tile: int) -> np.ndarray:
    """Permutation of a row-major w x h pixel grid into tile x tile screen tiles (tiles row-major, pixels
    row-major inside a tile, partial tiles at the right / bottom edges), the layout GPU render targets use."""
    ys, xs = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    tiles_x = (w + tile - 1) // tile
    key = ((ys // tile) * tiles_x + xs // tile) * (tile * tile) + (ys % tile) * tile + (xs % tile)
    return np.argsort(key.ravel(), kind="stable")


def plane_queries(rng: np.random.Generator, width: int, height: int, res_ref: int, uv_scale: float = 0.5,
                  x0: int = 0, y0: int = 0, w: int | None = None, h: int | None = None, supersample: int = 1,
                  tile: int = 16):
    """1-spp G-buffer of a perspective-viewed tiled plane.

    Camera 1 unit above the plane z = 0, pitch ~ U[45, 55] degrees below the horizon, yaw ~ U[0, 360),
    vertical FOV 60 degrees, aspect width/height; per-pixel jitter ~ U[-0.5, 0.5]^2.  uv = world_xy * uv_scale
    (repeat addressing wraps it).  s = log2(max(|d uv/dx|, |d uv/dy|) * res_ref) from the FP64 screen
    Jacobian, clamped at 0 (magnification).  An optional sub-rectangle (x0, y0, w, h) of the screen is returned;
    `supersample` renders a (width*ss) x (height*ss) grid.  Returns float32 u, v, s in 16 x 16 screen-tile
    order (`tile`; 0 = row-major pixel order)."""
    W, H = width * supersample, height * supersample
    w = W if w is None else w
    h = H if h is None else h
    pitch = math.radians(rng.uniform(45.0, 55.0))
    yaw = rng.uniform(0.0, 2 * math.pi)
    tan_half = math.tan(math.radians(30.0))
    aspect = W / H
    # camera basis: forward tilted down by `pitch`, rotated by `yaw` about z
    cf, sf = math.cos(pitch), math.sin(pitch)
    cy, sy = math.cos(yaw), math.sin(yaw)
    fwd = np.array([cf * cy, cf * sy, -sf])
    right = np.array([sy, -cy, 0.0])
    up = np.cross(right, fwd)
    px = np.arange(x0, x0 + w, dtype=np.float64)[None, :] + 0.5 + rng.uniform(-0.5, 0.5, (h, w))
    py = np.arange(y0, y0 + h, dtype=np.float64)[:, None] + 0.5 + rng.uniform(-0.5, 0.5, (h, w))
    # ray d = fwd + nx right + ny up hits z = 0 from height 1 at t = -1 / d_z: world = t (d_x, d_y)
    ax, ay = 2.0 * tan_half * aspect / W, -2.0 * tan_half / H  # d nx / d px, d ny / d py
    nx = px * ax - tan_half * aspect
    ny = py * ay + tan_half
    dx_ = fwd[0] + nx * right[0] + ny * up[0]
    dy_ = fwd[1] + nx * right[1] + ny * up[1]
    dz_ = fwd[2] + nx * right[2] + ny * up[2]
    t = -1.0 / dz_
    u = dx_ * t * uv_scale
    v = dy_ * t * uv_scale
    # exact screen Jacobian of (u, v) = uv_scale * (d_x, d_y) / (-d_z)
    def grad(e):  # e: direction derivative per pixel step (3-vector)
        dt = t * t * e[2]
        return uv_scale * (dt * dx_ + t * e[0]), uv_scale * (dt * dy_ + t * e[1])
    gux, gvx = grad(right * ax)
    guy, gvy = grad(up * ay)
    s = np.log2(np.maximum(np.hypot(gux, gvx), np.hypot(guy, gvy)) * res_ref)
    s = np.maximum(s, 0.0)
    u = u - np.floor(u)
    v = v - np.floor(v)
    u, v, s = u.astype(np.float32).ravel(), v.astype(np.float32).ravel(), s.astype(np.float32).ravel()
    if tile:
        perm = tile_order(w, h, tile)
        u, v, s = u[perm], v[perm], s[perm]
    return u, v, s


# --------------------------------------------------------------------------- MLP weights

def mlp_weights(rng: np.random.Generator, dims: list[int]):
    """W_l ~ N(0, 1/fan_in) [out, in] and b_l ~ N(0, 1/fan_in), float32, per layer."""
    Ws, bs = [], []
    for i in range(len(dims) - 1):
        sd = 1.0 / math.sqrt(dims[i])
        Ws.append((rng.standard_normal((dims[i + 1], dims[i])) * sd).astype(np.float32))
        bs.append((rng.standard_normal(dims[i + 1]) * sd).astype(np.float32))
    return Ws, bs


def fp8_scales(Ws, bs, input_bound: float):
    """Per-layer FP8 scales: w_scale = max|W| / 448; act_scale = (interval bound of the layer's input) / 448,
    the bound propagated from `input_bound` through |W| and |b| with ReLU."""
    w_scale, act_scale = [], []
    bound = np.full(Ws[0].shape[1], float(input_bound))
    for l, (W, b) in enumerate(zip(Ws, bs)):
        w_scale.append(float(np.abs(W).max()) / 448.0)
        act_scale.append(float(bound.max()) / 448.0)
        bound = np.abs(W.astype(np.float64)) @ bound + np.abs(b)
    return np.array(act_scale, np.float32), np.array(w_scale, np.float32)


def store_weights(Ws, precision: str, w_scale=None) -> np.ndarray:
    """Concatenated row-major W of every layer in the storage format (library casts, round to nearest even)."""
    import torch

    flat = []
    for l, W in enumerate(Ws):
        t = torch.from_numpy(np.ascontiguousarray(W, np.float32))
        if precision == "fp32":
            flat.append(t.numpy().ravel())
        elif precision == "fp16":
            flat.append(t.to(torch.float16).view(torch.int16).numpy().view(np.uint16).ravel())
        elif precision == "bf16":
            flat.append(t.to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16).ravel())
        elif precision == "fp8":
            q = (t / float(w_scale[l])).to(torch.float8_e4m3fn)
            flat.append(q.view(torch.uint8).numpy().ravel())
        else:
            raise ValueError(precision)
    return np.ascontiguousarray(np.concatenate(flat))


# --------------------------------------------------------------------------- training inputs

def train_block_params(rng: np.random.Generator, n_blocks: int):
    """Eq. 6 parameters per block: 4 RGB endpoints e ~ U[0, 30] (6-bit units), 16 x ~ U[0, 1]; partition k ~ U{0..31}."""
    p = np.empty((n_blocks, 28), np.float32)
    p[:, :12] = rng.uniform(0.0, 30.0, (n_blocks, 12))
    p[:, 12:] = rng.uniform(0.0, 1.0, (n_blocks, 16))
    k = rng.integers(0, 32, n_blocks).astype(np.uint8)
    return p, k


def _value_noise(rng: np.random.Generator, res: int, octaves: int = 6, base: int = 8, gain: float = 0.5):
    """Tileable multi-octave value noise in [0, 1] (smoothstep-interpolated lattice, lacunarity 2)."""
    out = np.zeros((res, res), np.float32)
    amp, total = 1.0, 0.0
    period = base
    x = (np.arange(res, dtype=np.float32) + 0.5) / res
    for _ in range(octaves):
        lat = rng.random((period, period), dtype=np.float32)
        f = x * period
        i0 = np.floor(f).astype(np.int64)
        t = f - i0
        t = t * t * (3 - 2 * t)
        i0 %= period
        i1 = (i0 + 1) % period
        a = lat[np.ix_(i0, i0)]
        b = lat[np.ix_(i0, i1)]
        c = lat[np.ix_(i1, i0)]
        d = lat[np.ix_(i1, i1)]
        ty, tx = t[:, None], t[None, :]
        out += amp * ((a * (1 - tx) + b * tx) * (1 - ty) + (c * (1 - tx) + d * tx) * ty)
        total += amp
        amp *= gain
        period *= 2
    return out / total


def pbr_target(rng: np.random.Generator, res: int):
    """9-channel synthetic PBR material: albedo RGB in [0,1]^3, unit normal xyz from a noise height field,
    roughness / metalness / AO in [0,1].  Returns float32 [res, res, 9]."""
    ch = np.zeros((res, res, 9), np.float32)
    for c in range(3):
        n = _value_noise(rng, res)
        ch[..., c] = 1.0 / (1.0 + np.exp(-6.0 * (n - 0.5)))
    hgt = _value_noise(rng, res) * 0.02 * res / 64
    gx = (np.roll(hgt, -1, axis=1) - np.roll(hgt, 1, axis=1)) * 0.5
    gy = (np.roll(hgt, -1, axis=0) - np.roll(hgt, 1, axis=0)) * 0.5
    nrm = np.stack([-gx, -gy, np.ones_like(hgt)], -1)
    nrm /= np.linalg.norm(nrm, axis=-1, keepdims=True)
    ch[..., 3:6] = nrm
    for c in range(6, 9):
        ch[..., c] = _value_noise(rng, res)
    return ch


def target_mips(img: np.ndarray, levels: int):
    """2x2 box-filtered chain of `levels` levels, stored as FP16: (channels 0..7 [texels, 8], channel 8 [texels])."""
    chain = [img.astype(np.float32)]
    for _ in range(1, levels):
        a = chain[-1]
        chain.append(0.25 * (a[0::2, 0::2] + a[1::2, 0::2] + a[0::2, 1::2] + a[1::2, 1::2]))
    flat = np.concatenate([c.reshape(-1, 9) for c in chain]).astype(np.float16)
    return np.ascontiguousarray(flat[:, :8]), np.ascontiguousarray(flat[:, 8])


# --------------------------------------------------------------------------- the five workloads

CONFIG_NAMES = {
    1: "plain: 2x BC6H 256^2 (random all-mode blocks), no mips, 65,536 uniform uv, MLP 6-16-16-8 FP32",
    2: "screen: 4x BC6H 2048^2 full mips, 3840x2160 perspective-plane queries, MLP 13-32-32-9",
    3: "train: 4x block-parameterised 1024^2 with mips, 2048^2 9-ch target, batch 2^20, MLP 13-32-32-9 BF16",
    4: "batched: 64 materials, res in {256..4096}^2, 4 textures each, 1e4..4e6 queries each, MLP 13-32-32-9 FP16",
    5: "large: 8x BC6H 4096^2 full mips, 7680x4320 (4x supersampled 4K) queries, MLP 25-64-64-9",
}
