"""Batched multi-material decode (bcf_decode_material_set): one persistent
launch over many materials of different resolutions and query counts."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_16121_b300 import workloads

pytestmark = pytest.mark.gpu


def _bcf():
    import paper_2311_16121_b300 as bcf

    bcf.lib()
    return bcf


def _small_set(precision="fp16", n_materials=7, seed_config=41):
    sw = workloads.config4(n_materials=n_materials, q_range=(300, 6000), res_choices=(32, 64, 128, 256),
                           pool=1 << 14, config=seed_config)
    mats = [workloads.upload(m, precision) for m in sw.materials]
    return sw, mats


def _set_inputs(sw):
    u, v, s = (torch.from_numpy(a).cuda() for a in sw.concat())
    off = torch.from_numpy(sw.offsets).cuda()
    return off, u, v, s


@pytest.mark.parametrize("variant,engine", [(0, "mma_sync"), (0, "tcgen05"), (3, "mma_sync")])
@pytest.mark.parametrize("precision", ["fp16", "fp8"])
def test_set_decode_equals_per_material_decodes(precision, variant, engine):
    """One launch over the set equals the per-material decodes bit for bit: the hand-written single-geometry tile
    decode (materials on variant 0; tiles of a material start at its first query, any alignment) with either MLP
    engine, and the texture-unit decode (materials on variant 3)."""
    bcf = _bcf()
    sw, mats = _small_set(precision)
    for m in mats:
        m.set_decode_variant(variant)
        m.set_mlp_engine(engine)
    S = bcf.MaterialSet(mats)
    off, u, v, s = _set_inputs(sw)
    got = bcf.decode(S, u, v, s, offsets=off).cpu().numpy()
    for m, w in enumerate(sw.materials):
        a, b = int(sw.offsets[m]), int(sw.offsets[m + 1])
        one = bcf.decode(mats[m], u[a:b], v[a:b], s[a:b]).cpu().numpy()
        np.testing.assert_array_equal(got[a:b], one)


def test_set_decode_matches_oracle():
    bcf = _bcf()
    sw, mats = _small_set("fp16", n_materials=3, seed_config=43)
    S = bcf.MaterialSet(mats)
    off, u, v, s = _set_inputs(sw)
    got = S.decode(off, u, v, s, out_dtype=torch.float32).cpu().numpy().astype(np.float64)
    for m, w in enumerate(sw.materials):
        a, b = int(sw.offsets[m]), int(sw.offsets[m + 1])
        Wst, bias, _, _ = w.weights("fp16")
        mat = oracle.Material(w.blocks, w.res, w.levels, w.res_ref, False, True, True)
        P = oracle.Mlp(w.dims, "fp16", Wst, bias)
        ref = oracle.decode(mat, P, w.u, w.v, w.s, quant_aware=True, threads=8)
        r = oracle.check_outputs(got[a:b], ref, 1e-3, False,
                                 oracle.decode_explainer(mat, P, w.u, w.v, w.s, got[a:b], 1e-3, False))
        assert not r["unexplained"], (m, r["unexplained"][:5], r["worst"])


@pytest.mark.parametrize("variant", [0, 3])
def test_set_decode_in_a_cuda_graph_and_autotune(variant):
    bcf = _bcf()
    sw, mats = _small_set("fp16", seed_config=44)
    for m in mats:
        m.set_decode_variant(variant)
    S = bcf.MaterialSet(mats)
    off, u, v, s = _set_inputs(sw)
    ref = S.decode(off, u, v, s).clone()
    cfg = S.autotune(off, u, v, s, torch.empty_like(ref))
    if variant == 0:  # the tile kernel of the single-material decode: its arena is fixed by the tile (cap 0)
        assert cfg[0] == 0 and 1 <= cfg[1] <= 3 and cfg[2] in (1, 2, 4, 8)
    else:  # texture-unit set kernel: CTAs per SM and 32-query warp tiles per grab
        assert cfg[1] in (4, 6, 8) and cfg[2] in (8, 16, 32, 64)
    assert S.config() == cfg
    out = torch.zeros_like(ref)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        S.decode(off, u, v, s, out=out)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S.decode(off, u, v, s, out=out)
    for _ in range(2):  # the work counter is reset inside the graph: replays are repeatable
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        torch.testing.assert_close(out, ref, rtol=0, atol=0)


def test_set_decode_empty_and_clipped_ranges():
    bcf = _bcf()
    sw, mats = _small_set("fp16", n_materials=4, seed_config=45)
    S = bcf.MaterialSet(mats)
    _, u, v, s = _set_inputs(sw)
    n = u.numel()
    # material 1 has no queries; the last offset runs past the end (clipped to n)
    offs = sw.offsets.copy()
    offs[2] = offs[1]
    offs[-1] = n + 1000
    got = S.decode(torch.from_numpy(offs).cuda(), u, v, s).cpu().numpy()
    for m in (0, 2, 3):
        a, b = int(offs[m]), min(int(offs[m + 1]), n)
        one = mats[m].decode(u[a:b], v[a:b], s[a:b], out_dtype=torch.float16).cpu().numpy()
        np.testing.assert_array_equal(got[a:b], one)
    # sets reject mixed MLP shapes
    w2 = workloads.small_screen(res=32, width=8, height=8, dims=(13, 16, 16, 9))
    other = workloads.upload(w2, "fp16")
    with pytest.raises(bcf.BcfError):
        bcf.MaterialSet([mats[0], other])


@pytest.fixture(scope="module")
def full_set():
    return workloads.config4()


@pytest.mark.parametrize("variant", [0, 3])
def test_full_size_batched_decode_sampled_against_oracle(full_set, variant):
    """The 64-material workload at full size (4 textures of 256^2 .. 4096^2 each, 1e4 .. 4e6 queries per
    material, FP16) in the benchmark's launch configuration -- one launch replayed from a CUDA graph, autotuned
    first on variant 0 -- checked on 32 sampled queries per material against the quantisation-aware oracle."""
    bcf = _bcf()
    sw = full_set
    mats = [workloads.upload(m, "fp16") for m in sw.materials]
    for m in mats:
        m.set_decode_variant(variant)
    S = bcf.MaterialSet(mats)
    u, v, s = (torch.from_numpy(a).cuda() for a in sw.concat())
    off = torch.from_numpy(sw.offsets).cuda()
    out = torch.empty((sw.n, 9), dtype=torch.float16, device="cuda")
    if variant == 0:
        S.autotune(off, u, v, s, out)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        S.decode(off, u, v, s, out=out)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S.decode(off, u, v, s, out=out)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    rng = np.random.default_rng(29 + variant)
    su, sv, ss = sw.concat()
    flips = 0
    for m, w in enumerate(sw.materials):
        a, b = int(sw.offsets[m]), int(sw.offsets[m + 1])
        idx = np.sort(rng.choice(np.arange(a, b), 32, replace=False))
        got = out[torch.from_numpy(idx).cuda()].float().cpu().numpy().astype(np.float64)
        Wst, bias, _, _ = w.weights("fp16")
        mat = oracle.Material(w.blocks, w.res, w.levels, w.res_ref, False, True, True)
        P = oracle.Mlp(w.dims, "fp16", Wst, bias)
        ref = oracle.decode(mat, P, su[idx], sv[idx], ss[idx], quant_aware=True, threads=8)
        # FP16 output: within 1e-3 plus half an FP16 unit, every output, except explained rounding flips
        r = oracle.check_outputs(got, ref, 1e-3, True,
                                 oracle.decode_explainer(mat, P, su[idx], sv[idx], ss[idx], got, 1e-3, True))
        assert not r["unexplained"], (m, r["unexplained"][:5], r["worst"])
        flips += r["flips"]
    print(f"rows explained as rounding flips: {flips} of {32 * len(sw.materials)}")


@pytest.mark.parametrize("engine", ["mma_sync", "tcgen05"])
def test_set_decode_tiny_and_unaligned_ranges(engine):
    """Materials with 1, 31, 33 and 513 queries (tiles that end inside a warp, outputs that start at any row
    alignment, a material spanning two tiles) in one launch equal the per-material decodes bit for bit."""
    bcf = _bcf()
    sw, mats = _small_set("fp16", n_materials=4, seed_config=46)
    for m in mats:
        m.set_decode_variant(0)
        m.set_mlp_engine(engine)
    S = bcf.MaterialSet(mats)
    _, u, v, s = _set_inputs(sw)
    sizes = [1, 31, 33, 513]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    assert offs[-1] <= u.numel()
    n = int(offs[-1])
    got = S.decode(torch.from_numpy(offs).cuda(), u[:n], v[:n], s[:n]).cpu().numpy()
    for m in range(len(sizes)):
        a, b = int(offs[m]), int(offs[m + 1])
        one = mats[m].decode(u[a:b], v[a:b], s[a:b], out_dtype=torch.float16).cpu().numpy()
        np.testing.assert_array_equal(got[a:b], one)


@pytest.mark.parametrize("engine", ["mma_sync", "tcgen05"])
@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_set_mixing_formats_and_addressing(precision, engine):
    """One set whose materials differ in what the tile kernel reloads per material: signed (SF16) blocks,
    clamp addressing, textures of one mode (the trained features' mode 10) and plain unsigned repeat-addressed
    all-mode textures.  The launch equals the per-material decodes bit for bit, and every material's rows
    match the oracle."""
    from paper_2311_16121_b300 import synth

    bcf = _bcf()
    sw = workloads.config4(n_materials=4, q_range=(2000, 6000), res_choices=(64, 128), pool=1 << 14, config=47)
    rng = workloads.seed_rng(47, 9)
    w0, w1, w2, _ = sw.materials
    w0.is_signed = True
    w0.blocks = [synth.bounded_blocks(rng, b.shape[0], signed=True) for b in w0.blocks]
    w1.wrap = False
    w1.u = (w1.u * 1.3 - 0.15).astype(np.float32)
    w2.blocks = [synth.bounded_blocks(rng, b.shape[0], modes=(10,)) for b in w2.blocks]
    mats = [workloads.upload(m, precision) for m in sw.materials]
    for m in mats:
        m.set_decode_variant(0)
        m.set_mlp_engine(engine)
    S = bcf.MaterialSet(mats)
    off, u, v, s = _set_inputs(sw)
    got = S.decode(off, u, v, s, out_dtype=torch.float32).cpu().numpy()
    tol = {"fp16": 1e-3, "bf16": 4e-3}[precision]
    for m, w in enumerate(sw.materials):
        a, b = int(sw.offsets[m]), int(sw.offsets[m + 1])
        one = mats[m].decode(u[a:b], v[a:b], s[a:b], out_dtype=torch.float32).cpu().numpy()
        np.testing.assert_array_equal(got[a:b], one)
        Wst, bias, _, _ = w.weights(precision)
        mat = oracle.Material(w.blocks, w.res, w.levels, w.res_ref, w.is_signed, w.wrap, w.lod_input)
        P = oracle.Mlp(w.dims, precision, Wst, bias)
        ref = oracle.decode(mat, P, w.u, w.v, w.s, quant_aware=True, threads=8)
        r = oracle.check_outputs(got[a:b].astype(np.float64), ref, tol, False,
                                 oracle.decode_explainer(mat, P, w.u, w.v, w.s, got[a:b].astype(np.float64), tol,
                                                         False))
        assert not r["unexplained"], (m, r["unexplained"][:5], r["worst"])
