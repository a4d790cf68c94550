"""The five BCf workloads as concrete, seeded inputs (host numpy arrays), plus
upload helpers that build a libbcf Material from them.

Shapes follow the paper's profiles (Table 1 resolutions and mip chains,
Table 3 screen resolutions, Sec. 5.1 random training batches).  The paper's
Polyhaven materials are unavailable, so block bitstreams, queries and weights
are seeded synthetic stand-ins (paper_2311_16121_b300.synth).  Nothing here
computes any step of the method.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import synth


@dataclass
class DecodeWorkload:
    name: str
    res: list[int]
    levels: list[int]
    res_ref: int
    blocks: list[np.ndarray]           # uint8 [blocks, 16] per texture
    lod_input: bool
    dims: list[int]
    W: list[np.ndarray]                # float32 [out, in] per layer
    b: list[np.ndarray]                # float32 [out] per layer
    u: np.ndarray
    v: np.ndarray
    s: np.ndarray | None
    is_signed: bool = False
    wrap: bool = True
    input_bound: float = 1.0           # bound on the MLP inputs (features and LOD) for FP8 scales
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.u.size)

    def weights(self, precision: str):
        """(stored weights array, FP32 biases, act_scale, w_scale) for `precision`."""
        bias = np.ascontiguousarray(np.concatenate(self.b).astype(np.float32))
        if precision == "fp8":
            a, w = synth.fp8_scales(self.W, self.b, self.input_bound)
            a = pow2_ceil(a)
            w = pow2_ceil(w)
            return synth.store_weights(self.W, "fp8", w), bias, a, w
        return synth.store_weights(self.W, precision), bias, None, None


def pow2_ceil(x: np.ndarray) -> np.ndarray:
    """Round positive scales up to powers of two (exact scaling on both sides)."""
    return np.exp2(np.ceil(np.log2(np.asarray(x, np.float64)))).astype(np.float32)


def seed_rng(config: int, stream: int) -> np.random.Generator:
    """Independent seeded streams per config and purpose (0 blocks, 1 queries, 2 weights, 3 target, 4 train)."""
    return np.random.Generator(np.random.Philox(key=synth.MASTER_SEED + config, counter=stream))


def config1() -> DecodeWorkload:
    res, levels = [256, 256], [1, 1]
    tex = synth.make_textures(seed_rng(1, 0), res, levels, kind="random")
    u, v, _ = synth.uniform_queries(seed_rng(1, 1), 65536)
    W, b = synth.mlp_weights(seed_rng(1, 2), [6, 16, 16, 8])
    return DecodeWorkload("config1-plain-256", res, levels, 256, tex.blocks, False, [6, 16, 16, 8], W, b, u, v, None,
                          input_bound=65504.0)


def screen_material(config: int, n_tex: int, res: int, dims: list[int], width: int, height: int,
                    supersample: int = 1, pool: int | None = None, modes=tuple(range(1, 15)),
                    tile: int = 16) -> DecodeWorkload:
    levels = synth.full_levels(res)
    rng = seed_rng(config, 0)
    if pool:
        tex = synth.make_textures(rng, [res] * n_tex, [levels] * n_tex, kind="bounded", pool=pool)
    else:
        blocks = [synth.bounded_blocks(rng, sum(synth.level_blocks(res, levels)), modes=modes) for _ in range(n_tex)]
        tex = synth.TextureSet([res] * n_tex, [levels] * n_tex, blocks)
    u, v, s = synth.plane_queries(seed_rng(config, 1), width, height, res_ref=res, supersample=supersample,
                                  tile=tile)
    W, b = synth.mlp_weights(seed_rng(config, 2), dims)
    lod_input = dims[0] == 3 * n_tex + 1  # the paper's own network reads the 3 T features only
    return DecodeWorkload(f"config{config}", [res] * n_tex, [levels] * n_tex, res, tex.blocks, lod_input, dims, W, b,
                          u, v, s, input_bound=max(1.0, float(s.max())))


def config2() -> DecodeWorkload:
    return screen_material(2, 4, 2048, [13, 32, 32, 9], 3840, 2160)


@dataclass
class SetWorkload:
    """Several materials and their concatenated queries (material m: rows offsets[m]..offsets[m+1])."""
    name: str
    materials: list[DecodeWorkload]   # each with its own queries in u, v, s
    offsets: np.ndarray               # int64 [n + 1]

    @property
    def n(self) -> int:
        return int(self.offsets[-1])

    def concat(self):
        u = np.concatenate([m.u for m in self.materials])
        v = np.concatenate([m.v for m in self.materials])
        s = np.concatenate([m.s for m in self.materials])
        return u, v, s


def config4(n_materials: int = 64, q_range=(1e4, 4e6), res_choices=(256, 512, 1024, 2048, 4096),
            dims=(13, 32, 32, 9), pool: int = 1 << 20, config: int = 4) -> SetWorkload:
    """64 materials: resolution uniform over res_choices (4 value-bounded BC6H textures each, full mips),
    query count log-uniform in q_range, each material's queries a contiguous 16:9 patch of the
    perspective-plane screen generator (res_ref = the material's resolution), own MLP weights."""
    rng = seed_rng(config, 0)
    pool_blocks = synth.bounded_blocks(rng, pool)
    mats = []
    offsets = [0]
    rq = seed_rng(config, 1)
    rw = seed_rng(config, 2)
    for m in range(n_materials):
        res = int(rng.choice(np.asarray(res_choices)))
        levels = synth.full_levels(res)
        nb = sum(synth.level_blocks(res, levels))
        blocks = [pool_blocks[rng.integers(0, pool, nb)] for _ in range(4)]
        nq = int(np.floor(np.exp(rng.uniform(np.log(q_range[0]), np.log(q_range[1])))))
        w = int(np.ceil(np.sqrt(nq * 16 / 9)))
        h = int(np.ceil(nq / w))
        x0 = int(rq.integers(0, max(1, 3840 - w)))
        y0 = int(rq.integers(0, max(1, 2160 - h)))
        u, v, s = synth.plane_queries(rq, 3840, 2160, res_ref=res, x0=x0, y0=y0, w=w, h=h)
        u, v, s = u[:nq], v[:nq], s[:nq]
        W, b = synth.mlp_weights(rw, list(dims))
        mats.append(DecodeWorkload(f"material{m}-{res}", [res] * 4, [levels] * 4, res, blocks, True, list(dims), W, b,
                                   u, v, s, input_bound=max(1.0, float(s.max()))))
        offsets.append(offsets[-1] + nq)
    return SetWorkload(f"config{config}-{n_materials}-materials", mats, np.asarray(offsets, np.int64))


def config5() -> DecodeWorkload:
    return screen_material(5, 8, 4096, [25, 64, 64, 9], 3840, 2160, supersample=2, pool=1 << 20)


def small_screen(config: int = 2, n_tex: int = 4, res: int = 64, dims=(13, 32, 32, 9), width: int = 96,
                 height: int = 54, modes=tuple(range(1, 15)), tile: int = 16) -> DecodeWorkload:
    """A reduced screen workload with the structure of configs 2/5 (for parity tests)."""
    w = screen_material(config, n_tex, res, list(dims), width, height, modes=modes, tile=tile)
    w.name = f"small-screen-{n_tex}x{res}-{width}x{height}"
    return w


def upload(w: DecodeWorkload, precision: str, device: str = "cuda"):
    """Build a libbcf Material on the device from a workload."""
    import torch

    from . import Material

    blocks = [torch.from_numpy(np.ascontiguousarray(b).reshape(-1)).to(device) for b in w.blocks]
    Wst, bias, a, ws = w.weights(precision)
    Wt = torch.from_numpy(Wst.view(np.uint8) if Wst.dtype != np.float32 else Wst).to(device)
    if Wst.dtype == np.uint16:
        Wt = torch.from_numpy(Wst.view(np.int16)).to(device)
    bt = torch.from_numpy(bias).to(device)
    return Material(blocks, w.res, w.levels, w.res_ref, w.dims, precision, Wt, bt, act_scale=a, w_scale=ws,
                    is_signed=w.is_signed, wrap=w.wrap, lod_input=w.lod_input)


def queries_to_device(w: DecodeWorkload, device: str = "cuda"):
    import torch

    u = torch.from_numpy(w.u).to(device)
    v = torch.from_numpy(w.v).to(device)
    s = None if w.s is None else torch.from_numpy(w.s).to(device)
    return u, v, s


# --------------------------------------------------------------------------- training (config 3)

@dataclass
class TrainWorkload:
    name: str
    res: list[int]
    levels: list[int]
    params: list[np.ndarray]      # float32 [blocks, 32] (device layout: region r's endpoints at 8 r, x at 16)
    partition: list[np.ndarray]   # uint8 [blocks]
    dims: list[int]
    W: np.ndarray                 # float32, layers concatenated
    b: np.ndarray
    target8: np.ndarray           # float16 [texels, 8]
    target1: np.ndarray           # float16 [texels]
    target_res: int
    target_levels: int
    batch: int

    @property
    def res_ref(self) -> int:
        return self.target_res


def params28_to_32(p28: np.ndarray) -> np.ndarray:
    """[blocks, 28] (e1..e4 RGB, x1..x16) -> the 32-float device record."""
    out = np.zeros((p28.shape[0], 32), np.float32)
    out[:, 0:6] = p28[:, 0:6]
    out[:, 8:14] = p28[:, 6:12]
    out[:, 16:32] = p28[:, 12:28]
    return out


def params32_to_28(p32: np.ndarray) -> np.ndarray:
    return np.concatenate([p32[:, 0:6], p32[:, 8:14], p32[:, 16:32]], axis=1)


def train_workload(res=(1024, 1024, 1024, 1024), target_res: int = 2048, batch: int = 1 << 20,
                   dims=(13, 32, 32, 9), config: int = 3) -> TrainWorkload:
    levels = [synth.full_levels(r) for r in res]
    rng = seed_rng(config, 4)
    params, part = [], []
    for r, l in zip(res, levels):
        p28, k = synth.train_block_params(rng, sum(synth.level_blocks(r, l)))
        p28 = np.concatenate([p28[:, :12], p28[:, 12:]], axis=1)
        params.append(params28_to_32(p28))
        part.append(k)
    tl = synth.full_levels(target_res)
    img = synth.pbr_target(seed_rng(config, 3), target_res)
    t8, t1 = synth.target_mips(img, tl)
    Ws, bs = synth.mlp_weights(seed_rng(config, 2), list(dims))
    W = np.concatenate([w.ravel() for w in Ws]).astype(np.float32)
    b = np.concatenate(bs).astype(np.float32)
    return TrainWorkload(f"train-{len(res)}x{res[0]}-target{target_res}", list(res), levels, params, part, list(dims),
                         W, b, t8, t1, target_res, tl, batch)


def upload_trainer(w: TrainWorkload, device: str = "cuda", **hyper):
    import torch

    from . import Trainer

    P = [torch.from_numpy(p.copy()).to(device) for p in w.params]
    K = [torch.from_numpy(k.copy()).to(device) for k in w.partition]
    W = torch.from_numpy(w.W.copy()).to(device)
    b = torch.from_numpy(w.b.copy()).to(device)
    t8 = torch.from_numpy(w.target8.view(np.int16).copy()).to(device)
    t1 = torch.from_numpy(w.target1.view(np.int16).copy()).to(device)
    return Trainer(P, K, w.res, w.levels, w.res_ref, w.dims, W, b, t8, t1, w.target_res, w.target_levels, **hyper)


def free_texels(w: TrainWorkload, config: int = 3) -> list[np.ndarray]:
    """Initial unconstrained features for the first training stage: [texels][4] float32 per texture (R, G, B,
    unused 0), values ~ U[0, 0.5), mips concatenated."""
    rng = seed_rng(config, 5)
    out = []
    for r, l in zip(w.res, w.levels):
        n = sum((r >> i) ** 2 for i in range(l))
        a = np.zeros((n, 4), np.float32)
        a[:, :3] = rng.random((n, 3), dtype=np.float32) * 0.5
        out.append(a)
    return out


def upload_free_trainer(w: TrainWorkload, texels: list[np.ndarray] | None = None, device: str = "cuda", **hyper):
    """A trainer over unconstrained per-texel features (the MLP, reference and sizes of `w`)."""
    import torch

    from . import Trainer

    tex = free_texels(w) if texels is None else texels
    P = [torch.from_numpy(np.ascontiguousarray(t, np.float32).copy()).to(device) for t in tex]
    W = torch.from_numpy(w.W.copy()).to(device)
    b = torch.from_numpy(w.b.copy()).to(device)
    t8 = torch.from_numpy(w.target8.view(np.int16).copy()).to(device)
    t1 = torch.from_numpy(w.target1.view(np.int16).copy()).to(device)
    return Trainer(P, [None] * len(P), w.res, w.levels, w.res_ref, w.dims, W, b, t8, t1, w.target_res,
                   w.target_levels, unconstrained=True, **hyper)


def paper_bcf1k(width: int = 3840, height: int = 2160, config: int = 6) -> DecodeWorkload:
    """The paper's decode configuration (Table 1 BCf-1K, Table 3): four value-bounded BC6H feature textures of
    1024^2, 512^2, 256^2, 128^2 with 9 / 8 / 7 / 6 levels, the paper's decoder (12 inputs, one hidden layer of
    16, 9 outputs, no LOD input), one sample per pixel of the perspective-plane screen with LODs in units of a
    2048^2 material."""
    res = [1024, 512, 256, 128]
    levels = [synth.full_levels(r) for r in res]
    tex = synth.make_textures(seed_rng(config, 0), res, levels, kind="bounded")
    u, v, s = synth.plane_queries(seed_rng(config, 1), width, height, res_ref=2048)
    dims = [12, 16, 9]
    W, b = synth.mlp_weights(seed_rng(config, 2), dims)
    return DecodeWorkload(f"paper-bcf1k-{width}x{height}", res, levels, 2048, tex.blocks, False, dims, W, b, u, v,
                          s, input_bound=1.0)
