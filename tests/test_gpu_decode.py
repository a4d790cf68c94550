"""GPU parity of the libbcf decode path against the CPU oracle.

Every comparison runs the CUDA kernels through the C ABI (via the thin Python
binding) and the oracle on the same seeded inputs:
  - BC6H unpack: bit-exact, all 14 modes, unsigned and signed, reserved modes;
  - texture-unit BC6H decode (an independent statement of the format) against
    the oracle: pins the per-mode bit layouts;
  - trilinear features: FP32 filtering vs FP64 (relative to the magnitudes);
  - fused decode: FP32 plain path vs FP64; FP16 / BF16 / FP8 tensor-core
    paths vs the quantisation-aware FP64 oracle within 1e-3 (FP16) and 4e-3
    (BF16, FP8) absolute per channel, every output, except rows the oracle
    shows to be operand-rounding flips (counted); error vs the unquantised
    FP64 oracle reported.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2311_16121_b300 import synth, workloads

pytestmark = pytest.mark.gpu

TOL = {"fp16": 1e-3, "bf16": 4e-3, "fp8": 4e-3}


def _bcf():
    import paper_2311_16121_b300 as bcf

    bcf.lib()
    return bcf


def _gpu_blocks(arr):
    return torch.from_numpy(np.ascontiguousarray(arr, np.uint8).reshape(-1)).cuda()


# --------------------------------------------------------------------------- BC6H unpack

@pytest.mark.parametrize("signed", [False, True])
def test_unpack_bit_exact_random_all_modes(signed):
    bcf = _bcf()
    rng = workloads.seed_rng(1, 7)
    bw, bh = 200, 37  # ragged: several 64-block runs and a partial one
    blocks = synth.random_blocks(rng, bw * bh)
    got = bcf.decode_bc6h(_gpu_blocks(blocks), bw, bh, signed).cpu().numpy().view(np.uint16)
    ref = oracle.bc6h_decode_image(blocks, bw, bh, signed)
    assert got.shape == ref.shape
    mism = np.argwhere(got != ref)
    assert mism.size == 0, f"{len(mism)} mismatching values, first at {mism[:3]}"


def test_unpack_reserved_modes_and_edge_sizes():
    bcf = _bcf()
    rng = workloads.seed_rng(1, 8)
    blocks = rng.integers(0, 256, (5 * 3, 16), dtype=np.uint8)
    for i, code in enumerate((19, 23, 27, 31)):
        blocks[i, 0] = (blocks[i, 0] & 0xE0) | code
    got = bcf.decode_bc6h(_gpu_blocks(blocks), 5, 3).cpu().numpy().view(np.uint16)
    np.testing.assert_array_equal(got, oracle.bc6h_decode_image(blocks, 5, 3))
    assert not got[:4, :16].any()
    one = synth.random_blocks(rng, 1)
    np.testing.assert_array_equal(bcf.decode_bc6h(_gpu_blocks(one), 1, 1).cpu().numpy().view(np.uint16),
                                  oracle.bc6h_decode_image(one, 1, 1))
    # empty image: a no-op
    bcf.decode_bc6h(_gpu_blocks(one), 0, 0, out=torch.empty(0, dtype=torch.int16, device="cuda"))


@pytest.mark.parametrize("signed", [False, True])
def test_texture_unit_agrees_with_oracle_on_all_modes(signed):
    """The GPU's BC6H texture decoder as an independent statement of the format
    (bit layouts of the 14 modes, partitions, anchors, weights): it must
    equal the oracle bit for bit on random valid blocks of every mode."""
    bcf = _bcf()
    rng = workloads.seed_rng(1, 9)
    bw, bh = 256, 128
    blocks = synth.random_blocks(rng, bw * bh)
    hw = bcf.texunit_decode_bc6h(_gpu_blocks(blocks), bw, bh, signed).cpu().numpy().view(np.uint16)
    ref = oracle.bc6h_decode_image(blocks, bw, bh, signed)
    modes = np.array([oracle.bc6h_block_mode(b) for b in blocks]).reshape(bh, bw)
    bad = np.any(hw != ref, axis=2)
    if bad.any():
        bad_blocks = np.unique((np.argwhere(bad) // 4) @ np.array([bw, 1]))
        bad_modes = np.bincount(modes.reshape(-1)[bad_blocks], minlength=15)
        pytest.fail(f"texture unit differs from the oracle on {bad_blocks.size} blocks; by mode: {bad_modes.tolist()}")


# --------------------------------------------------------------------------- features

def _oracle_material(w: workloads.DecodeWorkload):
    return oracle.Material(w.blocks, w.res, w.levels, w.res_ref, w.is_signed, w.wrap, w.lod_input)


def test_sample_features_random_blocks_fp32_vs_fp64():
    bcf = _bcf()
    w = workloads.config1()
    m = workloads.upload(w, "fp32")
    u, v, s = workloads.queries_to_device(w)
    got = m.sample_features(u, v, s).cpu().numpy().astype(np.float64)
    ref = oracle.sample_features(_oracle_material(w), w.u, w.v, w.s)
    # non-negative texels, positive weights: relative error of a few FP32 roundings
    err = np.abs(got - ref)
    assert (err <= 8 * 2.0 ** -24 * np.abs(ref) + 1e-30).all(), err.max()


def test_sample_features_screen_trilinear():
    bcf = _bcf()
    w = workloads.small_screen(res=128, width=160, height=90)
    m = workloads.upload(w, "fp16")
    u, v, s = workloads.queries_to_device(w)
    got = m.sample_features(u, v, s).cpu().numpy().astype(np.float64)
    ref = oracle.sample_features(_oracle_material(w), w.u, w.v, w.s)
    assert np.abs(got - ref).max() <= 1e-6


def test_sample_features_edge_inputs():
    """NaN / infinite / out-of-range coordinates and LODs, clamp addressing, negative and huge s."""
    bcf = _bcf()
    w = workloads.small_screen(res=32, width=16, height=9)
    u = np.array([np.nan, np.inf, -np.inf, -0.25, 1.0, 1.75, 7.3e6, -1e-9, 0.5, 0.999999], np.float32)
    v = np.array([0.5, 0.5, 0.1, 1.25, -3.5, np.nan, 0.5, 0.25, 0.0, 1e-20], np.float32)
    s = np.array([0.5, np.nan, -3.0, 1e9, np.inf, 2.5, 3.0, 0.0, -np.inf, 2.0], np.float32)
    for wrap in (True, False):
        w.wrap = wrap
        m = workloads.upload(w, "fp16")
        got = m.sample_features(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(),
                                torch.from_numpy(s).cuda()).cpu().numpy().astype(np.float64)
        ref = oracle.sample_features(_oracle_material(w), u, v, s)
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= 1e-6, (wrap, np.abs(got - ref).max(axis=1))


# --------------------------------------------------------------------------- fused decode

def _abs_bound(w, feat):
    """Magnitude bound of the FP32 MLP: the network with |W|, |b| and |x|."""
    h = np.abs(feat)
    for l, (W, b) in enumerate(zip(w.W, w.b)):
        h = h @ np.abs(W.astype(np.float64)).T + np.abs(b)
    return h


@pytest.mark.parametrize("variant", [0, 3])
def test_decode_fp32_plain_matches_fp64(variant):
    """The plain workload (2 x 256^2 random all-mode blocks, 65,536 queries, FP32 6-16-16-8) whole, through the
    library's BC6H decoder and through the texture unit's texels (the benchmark's launch)."""
    bcf = _bcf()
    w = workloads.config1()
    m = workloads.upload(w, "fp32")
    m.set_decode_variant(variant)
    u, v, s = workloads.queries_to_device(w)
    got = m.decode(u, v, s).cpu().numpy().astype(np.float64)
    Wst, bias, _, _ = w.weights("fp32")
    P = oracle.Mlp(w.dims, "fp32", Wst, bias)
    ref = oracle.decode(_oracle_material(w), P, w.u, w.v, w.s, threads=8)
    feat = oracle.sample_features(_oracle_material(w), w.u, w.v, w.s)
    M = _abs_bound(w, feat)
    tol = 4 * (max(w.dims) + 2) * 2.0 ** -24 * M + 1e-6 * M
    assert (np.abs(got - ref) <= tol).all(), np.max(np.abs(got - ref) / np.maximum(tol, 1e-30))


def _quant_check(got, ref_q, tol, what, mat, P, u, v, s, out_half=False):
    """Strict parity against the quantisation-aware oracle: every output within the absolute tolerance of its
    channel (plus half an FP16 unit when the kernel stored FP16), except where the oracle shows the miss to
    be an operand-rounding flip -- some combination of the roundings that the kernel's FP32 error windows
    leave open reproduces the output within the tolerance (oracle.mlp_explain).  Flips are counted."""
    r = oracle.check_outputs(got, ref_q, tol, out_half, oracle.decode_explainer(mat, P, u, v, s, got, tol, out_half))
    assert not r["unexplained"], (f"{what}: {len(r['unexplained'])} rows beyond {tol} are not rounding flips "
                                  f"(first {r['unexplained'][:5]}); per-channel max {r['worst']}")
    return r["worst"], r


@pytest.mark.parametrize("variant", [0, 3])
@pytest.mark.parametrize("precision", ["fp16", "bf16", "fp8"])
@pytest.mark.parametrize("out_dtype", [torch.float32, torch.float16])
def test_decode_tensor_core_paths_match_quant_aware_oracle(precision, out_dtype, variant):
    bcf = _bcf()
    w = workloads.small_screen(res=128, width=200, height=61)  # 12,200 queries: 381 warp tiles + a ragged tail
    m = workloads.upload(w, precision)
    m.set_decode_variant(variant)
    u, v, s = workloads.queries_to_device(w)
    got = m.decode(u, v, s, out_dtype=out_dtype).cpu().numpy().astype(np.float64)
    Wst, bias, a, ws = w.weights(precision)
    P = oracle.Mlp(w.dims, precision, Wst, bias, a, ws)
    mat = _oracle_material(w)
    ref_q = oracle.decode(mat, P, w.u, w.v, w.s, quant_aware=True, threads=8)
    ref = oracle.decode(mat, P, w.u, w.v, w.s, quant_aware=False, threads=8)
    worst, r = _quant_check(got, ref_q, TOL[precision], precision, mat, P, w.u, w.v, w.s,
                            out_half=out_dtype == torch.float16)
    print(f"{precision} out={out_dtype}: per-channel max |gpu - quant-aware oracle| {np.round(worst, 6)}, "
          f"{r['beyond_tol']} of {r['outputs']} outputs beyond the tolerance, in {r['flips']} rows explained as "
          f"rounding flips; vs unquantised FP64: max {np.abs(got - ref).max(axis=0).round(5)}")


@pytest.mark.parametrize("variant", [0, 3])
@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_decode_edge_sizes(precision, variant):
    """n = 1, a ragged n, and n = 0 (no-op)."""
    bcf = _bcf()
    w = workloads.small_screen(res=32, width=40, height=1)
    m = workloads.upload(w, precision)
    m.set_decode_variant(variant)
    Wst, bias, a, ws = w.weights(precision)
    P = oracle.Mlp(w.dims, precision, Wst, bias, a, ws)
    for n in (1, 33, 40):
        u = torch.from_numpy(w.u[:n].copy()).cuda()
        v = torch.from_numpy(w.v[:n].copy()).cuda()
        s = torch.from_numpy(w.s[:n].copy()).cuda()
        got = m.decode(u, v, s).cpu().numpy()
        ref = oracle.decode(_oracle_material(w), P, w.u[:n], w.v[:n], w.s[:n], quant_aware=True)
        assert got.shape == (n, 9)
        if precision == "fp32":
            assert np.abs(got - ref).max() <= 1e-4
        else:
            _quant_check(got.astype(np.float64), ref, TOL[precision], "edge", _oracle_material(w), P, w.u[:n],
                         w.v[:n], w.s[:n])
    e = torch.empty(0, device="cuda")
    assert m.decode(e, e, e).shape == (0, 9)


def test_invalid_arguments_return_status_without_launching():
    bcf = _bcf()
    w = workloads.small_screen(res=32, width=8, height=4)
    m = workloads.upload(w, "fp16")
    u, v, s = workloads.queries_to_device(w)
    bad_out = torch.empty(w.n * 9 + 1, dtype=torch.float32, device="cuda")[1:]  # 4-byte aligned, not 16
    with pytest.raises(bcf.BcfError):
        m.decode(u, v, s, out=bad_out)
    with pytest.raises(bcf.BcfError):
        bcf.decode_bc6h(_gpu_blocks(np.zeros(16, np.uint8)), -1, 1,
                        out=torch.empty(48, dtype=torch.int16, device="cuda"))


# --------------------------------------------------------------------------- tile-cooperative kernel

def _decode_both(w, precision, u=None, v=None, s=None, out_dtype=torch.float32, also_texunit=False):
    m = workloads.upload(w, precision)
    if u is None:
        u, v, s = workloads.queries_to_device(w)
    m.set_decode_variant(0)
    a = m.decode(u, v, s, out_dtype=out_dtype).cpu().numpy()
    m.set_decode_variant(1)
    b = m.decode(u, v, s, out_dtype=out_dtype).cpu().numpy()
    if also_texunit:  # the texture-unit texels with the exact filter (variant 3) give the same values
        m.set_decode_variant(3)
        c = m.decode(u, v, s, out_dtype=out_dtype).cpu().numpy()
        np.testing.assert_array_equal(c, b)
    return a, b


@pytest.mark.parametrize("precision", ["fp16", "bf16", "fp8"])
def test_tiled_equals_per_lane_bit_for_bit(precision):
    """The tile-cooperative kernel filters the same texel values with the same
    FP32 operation order as the per-lane kernel: identical outputs."""
    _bcf()
    w = workloads.small_screen(res=256, width=230, height=77)  # 17,710 queries: 70 tiles, ragged last tile
    a, b = _decode_both(w, precision)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("case", ["row_order", "random_uv", "wide_lod", "clamp", "signed"])
def test_tiled_fallbacks_and_addressing_match_oracle(case):
    """Incoherent tiles (arena overflow), tiles spanning more than three
    levels, clamp addressing, signed textures and row-major query order, for
    the software decoders and the texture-unit texels (bit-identical)."""
    _bcf()
    kw = {}
    if case == "row_order":
        kw["tile"] = 0
    w = workloads.small_screen(res=128, width=120, height=40, **kw)
    rng = workloads.seed_rng(2, 99)
    if case == "random_uv":
        w.u = rng.random(w.n, dtype=np.float32)
        w.v = rng.random(w.n, dtype=np.float32)
    elif case == "wide_lod":
        w.s = rng.uniform(-1.0, 7.0, w.n).astype(np.float32)
    elif case == "clamp":
        w.wrap = False
        w.u = (w.u * 1.3 - 0.15).astype(np.float32)
    elif case == "signed":
        w.is_signed = True
        w.blocks = [synth.bounded_blocks(rng, b.shape[0], signed=True) for b in w.blocks]
    a, b = _decode_both(w, "fp16", also_texunit=True)
    np.testing.assert_array_equal(a, b)
    Wst, bias, _, _ = w.weights("fp16")
    P = oracle.Mlp(w.dims, "fp16", Wst, bias)
    ref_q = oracle.decode(_oracle_material(w), P, w.u, w.v, w.s, quant_aware=True, threads=8)
    _quant_check(a.astype(np.float64), ref_q, TOL["fp16"], case, _oracle_material(w), P, w.u, w.v, w.s)


def _split_mode_blocks(rng, w, signed=False):
    """Per level, the block columns left of the middle hold mode-10 blocks (the two-region 6-bit format the
    trained features are stored in, Sec. 4.2), the others blocks of any mode: tiles and warps whose blocks
    all have one mode sit beside tiles and warps that mix modes."""
    out = []
    for b, res, levels in zip(w.blocks, w.res, w.levels):
        one = synth.bounded_blocks(rng, b.shape[0], modes=(10,), signed=signed)
        mixed = synth.bounded_blocks(rng, b.shape[0], signed=signed)
        cols = np.concatenate([np.tile(np.arange(max((res >> l) // 4, 1)), max((res >> l) // 4, 1))
                               for l in range(levels)])
        wb = np.concatenate([np.full(max((res >> l) // 4, 1) ** 2, max((res >> l) // 4, 1)) for l in range(levels)])
        out.append(np.where((cols < wb // 2)[:, None], one, mixed))
    return out


@pytest.mark.parametrize("case", ["mode10", "mode10_signed", "mode11", "split", "split_signed", "reserved"])
@pytest.mark.parametrize("engine", ["mma_sync", "tcgen05"])
def test_one_mode_textures_and_mixed_tiles(case, engine):
    """The tile decode's mode sort at its extremes: textures of one mode (the trained features' mode 10, a
    one-region mode, all-reserved blocks: one sort bin holds every block of a round) and textures in which
    tiles of one mode sit beside tiles of all modes.  Against the per-lane decode (bit for bit) and the
    oracle."""
    _bcf()
    w = workloads.small_screen(res=128, width=200, height=61)
    rng = workloads.seed_rng(2, 98)
    signed = case.endswith("signed")
    w.is_signed = signed
    if case.startswith("mode10"):
        w.blocks = [synth.bounded_blocks(rng, b.shape[0], modes=(10,), signed=signed) for b in w.blocks]
    elif case == "mode11":
        w.blocks = [synth.bounded_blocks(rng, b.shape[0], modes=(11,)) for b in w.blocks]
    elif case == "reserved":  # mode field 10011 (reserved): every texel decodes to zero
        blocks = [synth.bounded_blocks(rng, b.shape[0]) for b in w.blocks]
        for b in blocks:
            b[:, 0] = (b[:, 0] & 0xE0) | 0x13
        w.blocks = blocks
    else:
        w.blocks = _split_mode_blocks(rng, w, signed)
    m = workloads.upload(w, "fp16")
    u, v, s = workloads.queries_to_device(w)
    m.set_mlp_engine(engine)
    m.set_decode_variant(0)
    a = m.decode(u, v, s).cpu().numpy()
    m.set_decode_variant(1)
    b = m.decode(u, v, s).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    Wst, bias, _, _ = w.weights("fp16")
    P = oracle.Mlp(w.dims, "fp16", Wst, bias)
    mat = _oracle_material(w)
    ref_q = oracle.decode(mat, P, w.u, w.v, w.s, quant_aware=True, threads=8)
    _quant_check(a.astype(np.float64), ref_q, TOL["fp16"], case, mat, P, w.u, w.v, w.s)


# --------------------------------------------------------------------------- texture-unit comparator (Sec. 5.2)

@pytest.mark.parametrize("precision", ["fp16", "fp8"])
def test_texture_unit_variant_within_hardware_filter_error(precision):
    """Variant 2 samples the feature textures through BC6H texture objects with hardware trilinear filtering
    (the paper's render-time design).  Its filter weights are low-precision fixed point, so it is compared with
    the exact software path (itself parity-checked against the oracle) within a filtering-error bound, and the
    error is reported."""
    bcf = _bcf()
    w = workloads.small_screen(res=256, width=320, height=180)
    m = workloads.upload(w, precision)
    u, v, s = workloads.queries_to_device(w)
    ref = m.decode(u, v, s, out_dtype=torch.float32).cpu().numpy()
    m.set_decode_variant(2)
    hw = m.decode(u, v, s, out_dtype=torch.float32).cpu().numpy()
    err = np.abs(hw - ref)
    print(f"texture unit vs software ({precision}): mean {err.mean():.2e}, p99.9 {np.quantile(err, 0.999):.2e}, "
          f"max {err.max():.2e}")
    assert np.isfinite(hw).all()
    # measured: FP16 mean 2.3e-4, max 4.1e-3; FP8 mean 1.4e-3, max 0.12 (a filtering difference that moves an
    # E4M3 input across a rounding boundary changes it by up to 1/16 relative)
    assert err.mean() < 3e-3 and err.max() < (0.02 if precision == "fp16" else 0.25)
    # FP32 materials have no texture-unit variant
    m32 = workloads.upload(w, "fp32")
    with pytest.raises(bcf.BcfError) as e:
        m32.set_decode_variant(2)
    assert e.value.status == 2


@pytest.mark.parametrize("precision,signed", [("fp16", False), ("fp8", False), ("fp16", True), ("fp32", False)])
def test_texture_unit_texels_with_exact_filter_equal_the_software_decode(precision, signed):
    """Variant 3 fetches every footprint texel from the texture unit with point filtering (the hardware's BC6H
    decoder, bit-exact with the software one) and filters it with the same FP32 operations as the per-lane
    software path (variant 1): the outputs are identical bit for bit."""
    bcf = _bcf()
    w = workloads.small_screen(res=128, width=200, height=61)
    if signed:
        w.is_signed = True
        rng = np.random.default_rng(5)
        w.blocks = [synth.bounded_blocks(rng, b.size // 16, tuple(range(1, 15)), signed=True) for b in w.blocks]
    m = workloads.upload(w, precision)
    u, v, s = workloads.queries_to_device(w)
    m.set_decode_variant(1)
    ref = m.decode(u, v, s, out_dtype=torch.float32)
    m.set_decode_variant(3)
    got = m.decode(u, v, s, out_dtype=torch.float32)
    assert torch.equal(got, ref)


@pytest.mark.parametrize("variant,engine", [(0, "tcgen05"), (0, "mma_sync"), (3, "mma_sync")])
def test_full_size_screen_decode_sampled_against_oracle(variant, engine):
    """The 4 x 2048^2 / 3840x2160 FP16 workload in the launch configurations the benchmark times (whole frame,
    FP16 output; the headline is variant 0 with the tcgen05 MLP), checked on 20,000 sampled queries against the
    quantisation-aware oracle."""
    bcf = _bcf()
    w = workloads.config2()
    m = workloads.upload(w, "fp16")
    m.set_decode_variant(variant)
    m.set_mlp_engine(engine)
    u, v, s = workloads.queries_to_device(w)
    out = torch.empty((w.n, 9), dtype=torch.float16, device="cuda")
    m.decode(u, v, s, out=out)
    idx = np.random.default_rng(17).choice(w.n, 20000, replace=False)
    got = out[torch.from_numpy(idx).cuda()].float().cpu().numpy().astype(np.float64)
    Wst, bias, a, ws = w.weights("fp16")
    P = oracle.Mlp(w.dims, "fp16", Wst, bias, a, ws)
    ref_q = oracle.decode(_oracle_material(w), P, w.u[idx], w.v[idx], w.s[idx], quant_aware=True, threads=8)
    _quant_check(got, ref_q, TOL["fp16"], "fp16", _oracle_material(w), P, w.u[idx], w.v[idx], w.s[idx],
                 out_half=True)


@pytest.fixture(scope="module")
def large_frame():
    return workloads.config5()


@pytest.mark.parametrize("precision,path", [("fp8", "v0_tcgen05"), ("fp16", "v0_tcgen05"), ("fp8", "v3_mma_sync"),
                                            ("fp16", "v3_mma_sync"), ("fp32", "plain")])
def test_full_size_large_frame_sampled_against_oracle(large_frame, precision, path):
    """The 8 x 4096^2 / 7680x4320 workload (MLP 25-64-64-9) at full size in the launch configurations the
    benchmark times (whole frame, FP16 output; FP8 and FP16 on the hand-written decode with the tcgen05 MLP and
    on decode variant 3, FP32 on the plain path), checked on 8,192 sampled queries: the low-precision paths
    against the quantisation-aware oracle, the FP32 path against FP64 within a few FP32 roundings of the
    network's magnitude bound."""
    bcf = _bcf()
    w = large_frame
    m = workloads.upload(w, precision)
    if path == "v0_tcgen05":
        m.set_decode_variant(0)
        m.set_mlp_engine("tcgen05")
    elif path == "v3_mma_sync":
        m.set_decode_variant(3)
    u, v, s = workloads.queries_to_device(w)
    out = torch.empty((w.n, 9), dtype=torch.float16, device="cuda")
    m.decode(u, v, s, out=out)
    idx = np.sort(np.random.default_rng(23).choice(w.n, 8192, replace=False))
    got = out[torch.from_numpy(idx).cuda()].float().cpu().numpy().astype(np.float64)
    del out, u, v, s, m
    Wst, bias, a, ws = w.weights(precision)
    P = oracle.Mlp(w.dims, precision, Wst, bias, a, ws)
    mat = _oracle_material(w)
    if precision != "fp32":
        ref_q = oracle.decode(mat, P, w.u[idx], w.v[idx], w.s[idx], quant_aware=True, threads=8)
        _quant_check(got, ref_q, TOL[precision], precision, mat, P, w.u[idx], w.v[idx], w.s[idx], out_half=True)
        return
    ref = oracle.decode(mat, P, w.u[idx], w.v[idx], w.s[idx], threads=8)
    feat = oracle.sample_features(mat, w.u[idx], w.v[idx], w.s[idx])
    if w.lod_input:
        feat = np.concatenate([feat, np.maximum(w.s[idx].astype(np.float64), 0.0)[:, None]], axis=1)
    M = _abs_bound(w, feat)
    tol = 4 * (max(w.dims) + 2) * 2.0 ** -24 * M + 1e-6 * M + np.abs(ref) * 2.0 ** -11  # FP16 output
    assert (np.abs(got - ref) <= tol).all(), np.max(np.abs(got - ref) / np.maximum(tol, 1e-30))


@pytest.mark.parametrize("n,scratch_kb", [(12200, 64), (12200, 4096), (100, 64), (777, 32)])
def test_host_memory_decode_equals_device_decode(n, scratch_kb):
    """bcf_decode_material_host: pinned host queries in, host channels out, chunked and pipelined over three
    streams through the caller's scratch; the result equals the device-resident decode bit for bit."""
    bcf = _bcf()
    w = workloads.small_screen(res=128, width=200, height=61)
    m = workloads.upload(w, "fp16")
    m.set_decode_variant(3)
    u, v, s = (torch.from_numpy(a[:n].copy()) for a in (w.u, w.v, w.s))
    ref = m.decode(u.cuda(), v.cuda(), s.cuda(), out_dtype=torch.float16)
    uh, vh, sh = (t.pin_memory() for t in (u, v, s))
    oh = torch.zeros((n, 9), dtype=torch.float16).pin_memory()
    scratch = torch.empty(scratch_kb * 1024, dtype=torch.uint8, device="cuda")
    m.decode_host(uh, vh, sh, oh, scratch)
    torch.cuda.synchronize()
    assert torch.equal(oh, ref.cpu())
    with pytest.raises(bcf.BcfError):
        m.decode_host(uh, vh, sh, oh, scratch[:4096])  # too small for one 256-query chunk


@pytest.mark.parametrize("variant,engine", [(0, "mma_sync"), (0, "tcgen05"), (3, "mma_sync")])
def test_single_material_decode_replays_from_a_cuda_graph(variant, engine):
    """bcf_decode_material makes no allocation and no synchronisation once a material has decoded once, so a
    decode captured in a CUDA graph replays with new query values in the captured buffers and gives what a
    direct decode of those values gives."""
    _bcf()
    w = workloads.small_screen(res=128, width=200, height=61)
    m = workloads.upload(w, "fp16")
    m.set_decode_variant(variant)
    m.set_mlp_engine(engine)
    u, v, s = workloads.queries_to_device(w)
    out = torch.empty((w.n, 9), dtype=torch.float16, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        m.decode(u, v, s, out=out)  # warm-up: first-use configuration happens outside the capture
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        m.decode(u, v, s, out=out)
    for shift in (0.0, 0.37):
        u.copy_(torch.from_numpy((w.u + np.float32(shift)) % np.float32(1.0)).cuda())
        g.replay()
        torch.cuda.synchronize()
        ref = m.decode(u, v, s, out_dtype=torch.float16)
        assert torch.equal(out, ref)


@pytest.mark.parametrize("out_dtype", [torch.float16, torch.float32])
@pytest.mark.parametrize("lod_input", [True, False])
def test_host_memory_decode_on_the_headline_kernel(out_dtype, lod_input):
    """bcf_decode_material_host on the hand-written decode (variant 0), FP16 and FP32 channels, with the LOD
    input and without it (the paper's 12-input decoder: no s array is passed or copied); several chunks, the
    last one ragged.  Equal to the device-resident decode bit for bit."""
    _bcf()
    dims = (13, 32, 32, 9) if lod_input else (12, 32, 32, 9)
    w = workloads.small_screen(res=128, width=200, height=61, dims=dims)
    assert w.lod_input == lod_input
    m = workloads.upload(w, "fp16")
    m.set_decode_variant(0)
    n = w.n
    u, v, s = (torch.from_numpy(a[:n].copy()) for a in (w.u, w.v, w.s))
    ref = m.decode(u.cuda(), v.cuda(), s.cuda() if lod_input else None, out_dtype=out_dtype)
    uh, vh = u.pin_memory(), v.pin_memory()
    sh = s.pin_memory() if lod_input else None
    oh = torch.zeros((n, 9), dtype=out_dtype).pin_memory()
    scratch = torch.empty(96 * 1024, dtype=torch.uint8, device="cuda")
    m.decode_host(uh, vh, sh, oh, scratch)
    torch.cuda.synchronize()
    assert torch.equal(oh, ref.cpu())


@pytest.mark.parametrize("precision", ["fp16", "bf16", "fp8"])
def test_paper_decoder_shape_12_16_9(precision):
    """The paper's own decoder: 12 inputs (4 textures, no LOD input), one hidden layer of 16 (Sec. 5.1).  The
    16-bit precisions take the register-chained one-hidden-layer MLP; every variant agrees bit for bit and with
    the oracle."""
    _bcf()
    w = workloads.small_screen(res=128, width=200, height=61, dims=(12, 16, 9))
    assert not w.lod_input
    a, b = _decode_both(w, precision, also_texunit=True)
    np.testing.assert_array_equal(a, b)
    Wst, bias, sa, ws = w.weights(precision)
    P = oracle.Mlp(w.dims, precision, Wst, bias, sa, ws)
    ref_q = oracle.decode(_oracle_material(w), P, w.u, w.v, w.s, quant_aware=True, threads=8)
    _quant_check(a.astype(np.float64), ref_q, TOL[precision], precision, _oracle_material(w), P, w.u, w.v, w.s)


def test_texunit_fetch_probe_sums_the_decoded_footprints():
    """bcf_texunit_fetch_probe (the measured texel-fetch peak of the benchmark): each thread's sum over its
    rounds of (R of (x, y) + G of (x+1, y)) + (B of (x, y+1) + R of (x+1, y+1)), in single precision, equals the
    same sum over the oracle's decode of the level (a ragged thread count, several levels); it needs the
    material's texture objects."""
    bcf = _bcf()
    w = workloads.small_screen(res=64, width=16, height=16)
    m = workloads.upload(w, "fp16")
    with pytest.raises(bcf.BcfError):  # no texture objects before variant 2 / 3
        m.texunit_fetch_probe(64, 2)
    m.set_decode_variant(3)
    with pytest.raises(bcf.BcfError):
        m.texunit_fetch_probe(64, 0)
    n, rounds = 1000, 3
    for level in (0, 2):
        got = m.texunit_fetch_probe(n, rounds, texture=1, level=level).cpu().numpy()
        W = w.res[1] >> level
        start = sum(((w.res[1] >> l) // 4) ** 2 for l in range(level)) * 16
        img = oracle.bc6h_decode_image(w.blocks[1].reshape(-1)[start:], W // 4, W // 4)
        val = img.view(np.float16).astype(np.float32)
        ref = np.zeros(n, np.float32)
        per_row = max(W // 8, 1)
        for t in range(n):
            lane, patch = t & 31, t >> 5
            px = (patch % per_row) * 8 + (lane & 7)
            py = ((patch // per_row) * 4) % W + (lane >> 3)
            acc = np.float32(0.0)
            for r in range(rounds):
                x0, x1 = (px + r) & (W - 1), (px + r + 1) & (W - 1)
                y0, y1 = py & (W - 1), (py + 1) & (W - 1)
                acc = np.float32(acc + np.float32(np.float32(val[y0, x0, 0] + val[y0, x1, 1]) +
                                                  np.float32(val[y1, x0, 2] + val[y1, x1, 0])))
            ref[t] = acc
        np.testing.assert_array_equal(got, ref)


# --------------------------------------------------------------------------- tcgen05 MLP engine

@pytest.mark.parametrize("precision", ["fp16", "bf16", "fp8"])
@pytest.mark.parametrize("shape", ["13-32-32-9", "25-64-64-9"])
def test_tcgen05_mlp_engine_matches_oracle(precision, shape):
    """bcf_set_mlp_engine(BCF_MLP_TCGEN05): the software tile decode with the MLP on tcgen05 (CTA-level MMAs,
    tensor-memory accumulators) against the quantisation-aware oracle under the strict check, and against the
    warp-level MMA engine within the tolerance (the two sum in different orders)."""
    bcf = _bcf()
    if shape == "13-32-32-9":
        w = workloads.small_screen(res=128, width=200, height=61)
    else:
        w = workloads.small_screen(n_tex=8, res=64, dims=(25, 64, 64, 9), width=150, height=53)
    m = workloads.upload(w, precision)
    u, v, s = workloads.queries_to_device(w)
    ref_engine = m.decode(u, v, s, out_dtype=torch.float32).cpu().numpy().astype(np.float64)
    m.set_mlp_engine("tcgen05")
    got = m.decode(u, v, s, out_dtype=torch.float32).cpu().numpy().astype(np.float64)
    again = m.decode(u, v, s, out_dtype=torch.float32).cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(got, again)  # deterministic
    assert bcf.device_check() == 0
    Wst, bias, a, ws = w.weights(precision)
    P = oracle.Mlp(w.dims, precision, Wst, bias, a, ws)
    mat = _oracle_material(w)
    ref_q = oracle.decode(mat, P, w.u, w.v, w.s, quant_aware=True, threads=8)
    worst, r = _quant_check(got, ref_q, TOL[precision], f"tcgen05 {precision} {shape}", mat, P, w.u, w.v, w.s)
    print(f"tcgen05 {precision} {shape}: per-channel max {np.round(worst, 6)}, flips {r['flips']}, "
          f"max |tcgen05 - mma.sync| {np.abs(got - ref_engine).max():.2e}")
    # the texture-unit texels (variant 3) and the per-lane decode (variant 1) with the tcgen05 MLP: the same
    # features and the same MMAs, so the same outputs
    for variant in (3, 1):
        m.set_decode_variant(variant)
        other = m.decode(u, v, s, out_dtype=torch.float32).cpu().numpy().astype(np.float64)
        np.testing.assert_array_equal(other, got)
    m.set_decode_variant(0)
    m.set_mlp_engine("mma_sync")
    np.testing.assert_array_equal(m.decode(u, v, s, out_dtype=torch.float32).cpu().numpy().astype(np.float64),
                                  ref_engine)


def test_tcgen05_mlp_engine_rejects_other_shapes():
    bcf = _bcf()
    w = workloads.small_screen(res=32, width=8, height=8, dims=(13, 16, 16, 9))
    m = workloads.upload(w, "fp16")
    with pytest.raises(bcf.BcfError) as e:
        m.set_mlp_engine("tcgen05")
    assert e.value.status == 2
    m32 = workloads.upload(workloads.small_screen(res=32, width=8, height=8), "fp32")
    with pytest.raises(bcf.BcfError):
        m32.set_mlp_engine("tcgen05")


def test_texture_unit_copy_follows_rewritten_blocks_after_refresh():
    """Decode variants 2 and 3 sample a library-owned copy of the blocks: after the caller rewrites a texture's
    blocks, bcf_material_refresh brings the copy up to date, and variant 3 again equals the software decode of
    the caller's (new) blocks bit for bit; before the refresh it still samples the old blocks."""
    _bcf()
    w = workloads.small_screen(res=64, width=64, height=36)
    m = workloads.upload(w, "fp16")
    u, v, s = workloads.queries_to_device(w)
    m.set_decode_variant(3)
    before = m.decode(u, v, s)
    dev_blocks = m._keep[0][0]
    fresh_blocks = synth.bounded_blocks(workloads.seed_rng(2, 123), w.blocks[0].reshape(-1, 16).shape[0])
    dev_blocks.view(-1).copy_(torch.from_numpy(np.ascontiguousarray(fresh_blocks, np.uint8).reshape(-1)).cuda())
    stale = m.decode(u, v, s)
    assert torch.equal(stale, before)
    m.refresh()
    after = m.decode(u, v, s)
    m.set_decode_variant(0)
    software = m.decode(u, v, s)
    assert torch.equal(after, software) and not torch.equal(after, before)
