"""The three-stage training schedule (Sec. 5.1, Sec. 6.1) and its evaluation.

Stage 1 trains unconstrained per-texel features with the MLP for a short
while; their compression with the BC6 mode-10 encoder (bcf_encode_mode10)
then fixes every block's partition and initialises its endpoints and
indices; stage 2 trains the block parameters through the emulated BC6
decompression with the MLP; stage 3 freezes the features and fine-tunes
the MLP alone.  Freezing is quantising: the emulated forward already reads
the block parameters rounded to the 6-bit / 3-bit lattice (straight
through), so frozen parameters give exactly the exported block values.

Quality is the PSNR (peak 1) of the mean squared error averaged over the
reference's mip levels, each level compared at its texel centres with the
query LOD equal to the level (Sec. 6.2); the per-level PSNRs are returned
as well.  All sampling and MLP evaluation runs in the library's kernels;
this module only sequences the calls and reduces the error.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import Material, Trainer, compress_bc6h, encode_mode10, pack_mode10, texture_blocks
from . import workloads as wl


@dataclass
class StageLog:
    name: str
    steps: int
    ms_per_step: float
    first_loss: float
    last_loss: float
    psnr: float
    psnr_levels: list[float] = field(default_factory=list)


def eval_psnr(tr: Trainer, w: wl.TrainWorkload, max_queries: int = 1 << 22) -> tuple[float, list[float]]:
    """PSNR of the MSE averaged over the reference mips (texel centres, LOD = level), and per level.  Levels
    with more than `max_queries` texels are evaluated on a regular sub-grid of their texel centres."""
    dev = tr.W.device
    t8 = torch.from_numpy(w.target8.astype(np.float32)).to(dev)
    t1 = torch.from_numpy(w.target1.astype(np.float32)).to(dev)
    mses, off = [], 0
    for l in range(w.target_levels):
        W = w.target_res >> l
        step = 1
        while (W // step) ** 2 > max_queries:
            step *= 2
        idx = torch.arange(0, W, step, device=dev)
        jj, ii = torch.meshgrid(idx, idx, indexing="ij")
        u = ((ii.float() + 0.5) / W).reshape(-1).contiguous()
        v = ((jj.float() + 0.5) / W).reshape(-1).contiguous()
        s = torch.full_like(u, float(l))
        y = tr.forward(u, v, s)
        flat = off + (jj * W + ii).reshape(-1)
        ref = torch.cat([t8[flat], t1[flat, None]], dim=1)
        mses.append(float(((y - ref) ** 2).mean()))
        off += W * W
    psnr = lambda m: 10.0 * math.log10(1.0 / max(m, 1e-30))
    return psnr(float(np.mean(mses))), [psnr(m) for m in mses]


def eval_psnr_exported(tr: Trainer, w: wl.TrainWorkload, is_signed: bool = False,
                       max_queries: int = 1 << 22) -> tuple[float, list[float]]:
    """The same PSNR for what a renderer sees: the trainer's export (BC6H mode-10 blocks and FP16 weights)
    decoded by the decode path (bcf_decode_material, plain FP32 evaluation of the FP16 weights)."""
    blocks, w16 = tr.export()
    Wf = w16.view(torch.float16).float().contiguous()
    mat = Material(blocks, w.res, w.levels, w.res_ref, w.dims, "fp32", Wf, tr.b.contiguous(), is_signed=is_signed)

    class _Decoded:
        W = tr.W

        @staticmethod
        def forward(u, v, s):
            return mat.decode(u, v, s, out_dtype=torch.float32)

    return eval_psnr(_Decoded, w, max_queries)


def _run(tr: Trainer, w: wl.TrainWorkload, name: str, steps: int, batch: int, seed: int, step0: int,
         eval_queries: int) -> StageLog:
    first = float(tr.step(batch, seed, step0).item()) if steps else float("nan")
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for i in range(1, steps):
        tr.step(batch, seed, step0 + i)
    b.record()
    b.synchronize()
    last = float(tr.loss.item()) if steps else float("nan")
    ps, pl = eval_psnr(tr, w, eval_queries)
    return StageLog(name, steps, a.elapsed_time(b) / max(steps - 1, 1), first, last, ps, pl)


def three_stage(w: wl.TrainWorkload, warmup_steps: int = 5000, bc_steps: int = 20000, finetune_steps: int = 1000,
                batch: int | None = None, seed: int = 11, eval_queries: int = 1 << 22, literal: bool = False):
    """Runs the schedule; returns (block trainer after stage 3, partitions, stage logs).  `literal` trains the
    block stages with Eq. 7-8 as printed instead of the format's exact steps."""
    batch = w.batch if batch is None else batch
    logs = []
    # stage 1: unconstrained features (lr 5e-2 / 1e-3, decay 0.9995)
    tr0 = wl.upload_free_trainer(w, lr_features=5e-2, lr_mlp=1e-3, gamma=0.9995)
    logs.append(_run(tr0, w, "unconstrained", warmup_steps, batch, seed, 0, eval_queries))
    # compression of the unconstrained features: partitions and initial block parameters
    params, parts = [], []
    for t in range(len(w.res)):
        p, k, _ = encode_mode10(tr0.params[t].reshape(-1), w.res[t], w.levels[t], texel_stride=4)
        params.append(p)
        parts.append(k)
    W, b = tr0.W.clone(), tr0.b.clone()
    t8, t1 = tr0.target
    del tr0
    # stage 2: block parameters through the emulated BC6 decompression (lr 1e-2 / 1e-3, decay 0.9999)
    tr1 = Trainer(params, parts, w.res, w.levels, w.res_ref, w.dims, W, b, t8, t1, w.target_res, w.target_levels,
                  lr_features=1e-2, lr_mlp=1e-3, gamma=0.9999, literal=literal)
    logs.append(_run(tr1, w, "block", bc_steps, batch, seed, warmup_steps, eval_queries))
    # stage 3: features frozen (on the lattice by construction), MLP fine-tuned
    tr2 = Trainer(tr1.params, parts, w.res, w.levels, w.res_ref, w.dims, tr1.W, tr1.b, t8, t1, w.target_res,
                  w.target_levels, lr_features=0.0, lr_mlp=1e-3, gamma=0.9999, literal=literal)
    logs.append(_run(tr2, w, "finetune", finetune_steps, batch, seed, warmup_steps + bc_steps, eval_queries))
    return tr2, parts, logs


def random_init(w: wl.TrainWorkload, steps: int, batch: int | None = None, seed: int = 11,
                eval_queries: int = 1 << 22):
    """The comparison of Sec. 6.5: block parameters with random partitions and initial values, trained for
    `steps` steps with the stage-2 hyper-parameters."""
    batch = w.batch if batch is None else batch
    tr = wl.upload_trainer(w, lr_features=1e-2, lr_mlp=1e-3, gamma=0.9999)
    return tr, _run(tr, w, "random-partitions", steps, batch, seed, 0, eval_queries)


def material_bytes(res: list[int], levels: list[int]) -> int:
    """Storage of BC6H textures with mips: 16 bytes per 4 x 4 block."""
    return sum(16 * texture_blocks(r, l) for r, l in zip(res, levels))


def classic_bc6h(w: wl.TrainWorkload, res: int, eval_queries: int = 1 << 22, modes: tuple[int, ...] = (10, 11)):
    """The material without the network: the nine reference channels compressed directly as three BC6H
    textures -- albedo, the normal stored as n / 2 + 1 / 2 (the unsigned format holds no negative values),
    roughness / metalness / AO -- at `res` (at most the reference's resolution) with the reference's own box
    mips from that size down, each compressed by bcf_compress_bc6h (per block the better of a mode-10 and a
    mode-11 encoding; modes=(10,) keeps mode 10 alone, the features' own mode).  They are decoded by
    the decode path (BC6H unpack, trilinear filtering at the query LOD) with a single linear output layer that
    undoes the normal encoding, and scored with the same PSNR as the trained materials.
    Returns (PSNR, per-level PSNRs, bytes)."""
    if res > w.target_res or res & (res - 1):
        raise ValueError("classic_bc6h: res must be a power of two no larger than the reference")
    dev = torch.device("cuda")
    lo = int(round(math.log2(w.target_res // res)))
    levels = w.target_levels - lo
    start = sum((w.target_res >> l) ** 2 for l in range(lo))
    ref = np.concatenate([w.target8.astype(np.float32), w.target1.astype(np.float32)[:, None]], axis=1)[start:]
    ref[:, 3:6] = ref[:, 3:6] * 0.5 + 0.5
    blocks = []
    for t in range(3):
        tex = torch.from_numpy(np.ascontiguousarray(ref[:, 3 * t:3 * t + 3])).to(dev)
        if tuple(modes) == (10,):
            params, parts, _ = encode_mode10(tex.reshape(-1), res, levels)
            blocks.append(pack_mode10(params, parts))
        else:
            blocks.append(compress_bc6h(tex.reshape(-1), res, levels)[0])
    Wm = torch.eye(9, device=dev)
    bm = torch.zeros(9, device=dev)
    Wm[3:6, 3:6] *= 2.0
    bm[3:6] = -1.0
    mat = Material(blocks, [res] * 3, [levels] * 3, w.target_res, [9, 9], "fp32", Wm.reshape(-1).contiguous(),
                   bm, lod_input=False)

    class _Decoded:
        W = Wm

        @staticmethod
        def forward(u, v, s):
            return mat.decode(u, v, s, out_dtype=torch.float32)

    ps, pl = eval_psnr(_Decoded, w, eval_queries)
    return ps, pl, material_bytes([res] * 3, [levels] * 3)
