"""GPU parity of the training path (emulated BC6 mode 10 + MLP + reference
sampling + Adam) against the CPU oracle, export round trip, the autograd
function, and a training sanity check."""
import math

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


def _oracle_parts(w, params32=None, W=None, b=None):
    p32 = w.params if params32 is None else params32
    F = oracle.TrainFeatures([workloads.params32_to_28(p).astype(np.float64) for p in p32], w.partition, w.res,
                             w.levels, w.res_ref, lod_input=True)
    P = oracle.TrainMlp(w.dims, w.W if W is None else W, w.b if b is None else b, bf16=True)
    T = oracle.Target(w.target8, w.target1, w.target_res, w.target_levels)
    return F, P, T


SMALL = dict(res=(16, 8), target_res=32, batch=384, dims=(7, 8, 8, 9))
MEDIUM = dict(res=(64, 64, 64, 64), target_res=128, batch=600, dims=(13, 32, 32, 9))


def _queries(n, s_max, seed=3):
    rng = np.random.default_rng(seed)
    u = rng.random(n, dtype=np.float32)
    v = rng.random(n, dtype=np.float32)
    s = rng.uniform(0, s_max, n).astype(np.float32)
    return u, v, s


TOL_BF16 = 4e-3  # absolute, per channel (the BF16 tolerance)


def _forward_check(got, F, P, u, v, s, what=""):
    """Every output within 4e-3 of the oracle's BF16-rounded forward, except rows the oracle shows to be
    operand-rounding flips (oracle.train_mlp_explain)."""
    ref = oracle.train_outputs(F, P, u, v, s)
    r = oracle.check_outputs(got, ref, TOL_BF16, False, oracle.train_explainer(F, P, u, v, s, got, TOL_BF16))
    assert not r["unexplained"], (what, len(r["unexplained"]), r["unexplained"][:5], r["worst"])
    return r


def _grad_checks(F, P, u, v, s, go, pairs):
    """Per-element bound on every gradient value: |gpu - oracle| <= c A + R, with A the sum of the absolute
    terms of that value and R the terms that operand-rounding flips leave open (oracle.train_backward_bounds);
    c = (8 n + 16) 2^-23 + 2^-15 covers the single-precision sums of at most 8 terms per query over n queries
    (with a factor 2 for truncating adders) and the two-term bfloat16 split of the output gradient (2^-16
    relative).  pairs: (name, gpu array, oracle array, key) with key 'W', 'b' or a texture index."""
    (Af, AW, Ab), (Rf, RW, Rb) = oracle.train_backward_bounds(F, P, u, v, s, go)
    c = (8 * len(u) + 16) * 2.0 ** -23 + 2.0 ** -15
    for name, got, ref, key in pairs:
        A, R = (AW, RW) if key == "W" else (Ab, Rb) if key == "b" else (Af[key], Rf[key])
        A = A.reshape(ref.shape)
        R = R.reshape(ref.shape)
        d = np.abs(got.astype(np.float64) - ref)
        bound = c * A + R + 1e-12
        bad = d > bound
        assert not bad.any(), (name, int(bad.sum()), float((d / bound).max()))


@pytest.mark.parametrize("shape", ["small", "medium"])
def test_train_forward_matches_oracle(shape):
    _bcf()
    w = workloads.train_workload(**(SMALL if shape == "small" else MEDIUM))
    tr = workloads.upload_trainer(w)
    u, v, s = _queries(w.batch, w.target_levels - 1)
    got = tr.forward(*(torch.from_numpy(a).cuda() for a in (u, v, s))).cpu().numpy().astype(np.float64)
    F, P, _ = _oracle_parts(w)
    r = _forward_check(got, F, P, u, v, s, shape)
    print(f"{shape}: per-channel max {np.round(r['worst'], 6)}, rows explained as rounding flips {r['flips']}")


@pytest.mark.parametrize("shape", ["small", "medium"])
def test_train_backward_matches_oracle_gradient(shape):
    _bcf()
    w = workloads.train_workload(**(SMALL if shape == "small" else MEDIUM))
    tr = workloads.upload_trainer(w)
    u, v, s = _queries(w.batch, w.target_levels - 1, seed=4)
    go = np.random.default_rng(5).standard_normal((w.batch, 9)).astype(np.float32) * 1e-2
    tr.zero_grad()
    tr.backward(*(torch.from_numpy(a).cuda() for a in (u, v, s)), torch.from_numpy(go).cuda())
    F, P, _ = _oracle_parts(w)
    gf, gW, gb = oracle.train_backward_given(F, P, u, v, s, go.astype(np.float64))
    _grad_checks(F, P, u, v, s, go.astype(np.float64),
                 [("W", tr.W_grad.cpu().numpy(), gW, "W"), ("b", tr.b_grad.cpu().numpy(), gb, "b")] +
                 [(f"features{t}", workloads.params32_to_28(tr.grads[t].cpu().numpy()), gf[t], t)
                  for t in range(len(gf))])
    # the unused slots of the parameter records receive nothing
    for g in tr.grads:
        assert not g[:, [6, 7, 14, 15]].any()


def test_train_step_loss_with_philox_draws_and_adam_update():
    bcf = _bcf()
    w = workloads.train_workload(**MEDIUM)
    tr = workloads.upload_trainer(w, lr_features=1e-2, lr_mlp=1e-3, gamma=0.9999)
    seed, step = 1234567, 0
    loss = float(tr.step(w.batch, seed, step).item())
    u, v, s = oracle.train_queries(seed, step, w.batch, float(w.target_levels - 1))
    F, P, T = _oracle_parts(w)
    ref_loss, gf, gW, gb = oracle.train_loss_grad(F, P, T, u, v, s)
    assert loss == pytest.approx(ref_loss, rel=2e-3)
    # first Adam step: p -= lr * g / (|g| + eps) (bias-corrected), projected to the box; compare where |g| is
    # clearly non-zero (sign-like updates), everything else must stay within one learning-rate step
    newW = tr.W.cpu().numpy().astype(np.float64)
    pW, mW, vW = w.W.astype(np.float64).copy(), np.zeros(gW.size), np.zeros(gW.size)
    oracle.adam(pW, gW.copy(), mW, vW, step, 1e-3, 0.9999)
    big = np.abs(gW) > 1e-3 * np.abs(gW).max()
    np.testing.assert_allclose(newW[big], pW[big], rtol=0, atol=2e-6)
    assert np.abs(newW - pW).max() <= 2.0e-3 + 1e-6
    for t in range(len(gf)):
        p28 = workloads.params32_to_28(tr.params[t].cpu().numpy()).astype(np.float64)
        o28 = workloads.params32_to_28(w.params[t]).astype(np.float64)
        ends, xs = o28[:, :12].copy(), o28[:, 12:].copy()
        ge, gx = gf[t][:, :12].copy(), gf[t][:, 12:].copy()
        oracle.adam(ends.reshape(-1), ge.reshape(-1).copy(), np.zeros(ends.size), np.zeros(ends.size), step, 1e-2,
                    0.9999, lo=0.0, hi=63.0)
        oracle.adam(xs.reshape(-1), gx.reshape(-1).copy(), np.zeros(xs.size), np.zeros(xs.size), step, 1e-2, 0.9999,
                    lo=0.0, hi=1.0)
        ref = np.concatenate([ends, xs], axis=1)
        g = np.concatenate([ge, gx], axis=1)
        big = np.abs(g) > 1e-3 * np.abs(g).max()
        np.testing.assert_allclose(p28[big], ref[big], rtol=0, atol=2e-5)
        assert np.abs(p28 - ref).max() <= 2e-2 + 1e-5
    # gradients were zeroed by the optimiser
    assert not tr.W_grad.any() and not any(g.any() for g in tr.grads)


def test_full_size_step_loss_and_sampled_outputs():
    """The timed training configuration at full size (four block-parameterised 1024^2 textures with 9 levels,
    2048^2 reference, batch 2^20, 13-32-32-9 BF16, the bench's launch): outputs of 4,096 sampled queries of the
    batch match the oracle, and the step's loss equals the oracle's loss over the same 2^20 Philox draws."""
    _bcf()
    w = workloads.train_workload()
    tr = workloads.upload_trainer(w)
    seed, step = 987654321, 0
    u, v, s = oracle.train_queries(seed, step, w.batch, float(w.target_levels - 1))
    F, P, T = _oracle_parts(w)
    pick = np.sort(np.random.default_rng(8).choice(w.batch, 4096, replace=False))
    got = tr.forward(*(torch.from_numpy(np.ascontiguousarray(a[pick])).cuda() for a in (u, v, s)))
    _forward_check(got.cpu().numpy().astype(np.float64), F, P, u[pick], v[pick], s[pick], "full size")
    loss = float(tr.step(w.batch, seed, step).item())
    ref_loss = oracle.train_loss_mt(F, P, T, u, v, s)
    assert loss == pytest.approx(ref_loss, rel=2e-3), (loss, ref_loss)


def test_export_is_bit_exact_and_decodes_to_the_emulated_features():
    bcf = _bcf()
    w = workloads.train_workload(**SMALL)
    # include lattice extremes and anchor swaps
    w.params[0][:4, 0:6] = [[0, 63, 0.49, 62.5, 31.5, 7]] * 4
    tr = workloads.upload_trainer(w)
    blocks, w16 = tr.export()
    for t, blk in enumerate(blocks):
        got = blk.cpu().numpy().reshape(-1, 16)
        p28 = workloads.params32_to_28(w.params[t]).astype(np.float64)
        ref = np.stack([oracle.train_export_block(p28[i], int(w.partition[t][i])) for i in range(p28.shape[0])])
        np.testing.assert_array_equal(got, ref)
        # the exported blocks decode (GPU unpack) to the emulated texel values (oracle emulation)
        off = 0
        for l in range(w.levels[t]):
            W = w.res[t] >> l
            nb = (W // 4) ** 2
            img = bcf.decode_bc6h(blk[off * 16:(off + nb) * 16].contiguous(), W // 4, W // 4).cpu().numpy()
            img = img.view(np.uint16).view(np.float16).astype(np.float64)
            for bi in range(nb):
                k = int(w.partition[t][off + bi])
                by, bx = divmod(bi, W // 4)
                for tx in range(16):
                    for c in range(3):
                        assert img[4 * by + tx // 4, 4 * bx + tx % 4, c] == oracle.train_texel(p28[off + bi], k, tx, c)
            off += nb
    np.testing.assert_array_equal(w16.cpu().numpy().view(np.float16), w.W.astype(np.float16))


def test_autograd_function_matches_trainer_backward():
    bcf = _bcf()
    w = workloads.train_workload(**SMALL)
    tr = workloads.upload_trainer(w)
    u, v, s = (torch.from_numpy(a).cuda() for a in _queries(200, w.target_levels - 1, seed=9))
    W = tr.W.clone().requires_grad_(True)
    b = tr.b.clone().requires_grad_(True)
    ps = [p.clone().requires_grad_(True) for p in tr.params]
    y = bcf.BCfTrainFn.apply(tr, u, v, s, W, b, *ps)
    wts = torch.randn_like(y)
    (y * wts).sum().backward()
    tr.zero_grad()
    tr.backward(u, v, s, wts)
    torch.testing.assert_close(W.grad, tr.W_grad)
    torch.testing.assert_close(b.grad, tr.b_grad)
    for p, g in zip(ps, tr.grads):
        torch.testing.assert_close(p.grad, g)
    torch.testing.assert_close(y, tr.forward(u, v, s))


def test_training_reduces_loss_and_beats_linear_decoder():
    """Training sanity: the loss falls, and on held-out queries the trained
    MLP beats both its step-0 state and the best (least-squares) linear
    decoder of the same trained features -- what the network adds over the
    features alone."""
    bcf = _bcf()
    w = workloads.train_workload(res=(32, 32, 32, 32), target_res=64, batch=8192, dims=(13, 32, 32, 9))
    tr = workloads.upload_trainer(w, lr_features=1e-2, lr_mlp=3e-3, gamma=0.9995)
    hu, hv, hs = _queries(4096, w.target_levels - 1, seed=77)
    T = oracle.Target(w.target8, w.target1, w.target_res, w.target_levels)
    tgt = np.stack([oracle.target_sample(T, float(a), float(b_), float(c)) for a, b_, c in zip(hu, hv, hs)])
    hq = [torch.from_numpy(a).cuda() for a in (hu, hv, hs)]
    mse0 = float(((tr.forward(*hq).cpu().numpy() - tgt) ** 2).mean())
    losses = [float(tr.step(w.batch, 42, i).item()) for i in range(400)]
    torch.cuda.synchronize()
    mse1 = float(((tr.forward(*hq).cpu().numpy() - tgt) ** 2).mean())
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:5])
    assert mse1 < 0.5 * mse0
    # features of the trained textures: export, then the decode path's feature sampling
    blocks, _ = tr.export()
    zW = torch.zeros(13 * 16 + 16 * 9, dtype=torch.float16, device="cuda")
    zb = torch.zeros(16 + 9, dtype=torch.float32, device="cuda")
    mat = bcf.Material(blocks, w.res, w.levels, w.res_ref, [13, 16, 9], "fp16", zW, zb)
    feat = mat.sample_features(*hq).cpu().numpy().astype(np.float64)
    X = np.concatenate([feat, hs[:, None].astype(np.float64), np.ones((hs.size, 1))], axis=1)
    coef, *_ = np.linalg.lstsq(X, tgt, rcond=None)
    mse_lin = float(((X @ coef - tgt) ** 2).mean())
    assert mse1 < mse_lin, (mse1, mse_lin)
    print(f"held-out MSE: step 0 {mse0:.4g}, trained {mse1:.4g}, linear decoder on trained features {mse_lin:.4g}")


# --------------------------------------------------------------------------- unconstrained features (Sec. 5.1)

def _free_setup(shape=MEDIUM):
    w = workloads.train_workload(**shape)
    tex = workloads.free_texels(w)
    F = oracle.TrainFeatures([t[:, :3].astype(np.float64) for t in tex], None, w.res, w.levels, w.res_ref,
                             lod_input=True, free=True)
    return w, tex, F


def test_unconstrained_forward_and_backward_match_oracle():
    _bcf()
    w, tex, F = _free_setup()
    tr = workloads.upload_free_trainer(w, tex)
    u, v, s = _queries(w.batch, w.target_levels - 1, seed=21)
    q = [torch.from_numpy(a).cuda() for a in (u, v, s)]
    P = oracle.TrainMlp(w.dims, w.W, w.b, bf16=True)
    got = tr.forward(*q).cpu().numpy().astype(np.float64)
    _forward_check(got, F, P, u, v, s, "unconstrained")
    go = np.random.default_rng(22).standard_normal((w.batch, 9)).astype(np.float32) * 1e-2
    tr.zero_grad()
    tr.backward(*q, torch.from_numpy(go).cuda())
    gf, gW, gb = oracle.train_backward_given(F, P, u, v, s, go.astype(np.float64))
    _grad_checks(F, P, u, v, s, go.astype(np.float64),
                 [("W", tr.W_grad.cpu().numpy(), gW, "W"), ("b", tr.b_grad.cpu().numpy(), gb, "b")] +
                 [(f"texels{t}", tr.grads[t].cpu().numpy()[:, :3], gf[t], t) for t in range(len(gf))])
    assert not any(g[:, 3].any() for g in tr.grads)  # the unused fourth float receives nothing


def test_unconstrained_step_loss_and_unbounded_adam():
    _bcf()
    w, tex, F = _free_setup()
    tr = workloads.upload_free_trainer(w, tex, lr_features=5e-2, lr_mlp=1e-3, gamma=0.9995)
    seed, step = 77, 0
    loss = float(tr.step(w.batch, seed, step).item())
    u, v, s = oracle.train_queries(seed, step, w.batch, float(w.target_levels - 1))
    P = oracle.TrainMlp(w.dims, w.W, w.b, bf16=True)
    T = oracle.Target(w.target8, w.target1, w.target_res, w.target_levels)
    ref_loss, gf, gW, gb = oracle.train_loss_grad(F, P, T, u, v, s)
    assert loss == pytest.approx(ref_loss, rel=2e-3)
    for t in range(len(gf)):
        got = tr.params[t].cpu().numpy().astype(np.float64)
        p = tex[t][:, :3].astype(np.float64).reshape(-1).copy()
        g = gf[t].reshape(-1).copy()
        oracle.adam(p, g.copy(), np.zeros(p.size), np.zeros(p.size), step, 5e-2, 0.9995)  # no box
        big = np.abs(g) > 1e-3 * np.abs(g).max()
        np.testing.assert_allclose(got[:, :3].reshape(-1)[big], p[big], rtol=0, atol=2e-5)
        assert np.abs(got[:, :3].reshape(-1) - p).max() <= 5e-2 + 1e-5
        assert not got[:, 3].any()


def test_unconstrained_trainer_rejects_unsupported_uses():
    bcf = _bcf()
    w = workloads.train_workload(**SMALL)  # 7-8-8-9: no tensor-core path
    with pytest.raises(bcf.BcfError) as e:
        workloads.upload_free_trainer(w)
    assert e.value.status == 2
    w, tex, F = _free_setup()
    tr = workloads.upload_free_trainer(w, tex)
    with pytest.raises(bcf.BcfError):
        tr.export()


def test_three_stage_schedule_runs_and_reports_psnr():
    """Sec. 5.1 schedule on a small problem: unconstrained warm-up, encoder initialisation, block training,
    MLP fine-tuning; compared with block training from random partitions for the same number of steps."""
    _bcf()
    from paper_2311_16121_b300 import schedule

    w = workloads.train_workload(res=(64, 64, 64, 64), target_res=128, batch=1 << 14, dims=(13, 32, 32, 9))
    tr, parts, logs = schedule.three_stage(w, warmup_steps=300, bc_steps=900, finetune_steps=200)
    _, rnd = schedule.random_init(w, 1400)
    for lg in logs + [rnd]:
        print(f"{lg.name:18s} steps {lg.steps:5d} loss {lg.first_loss:.4g} -> {lg.last_loss:.4g} "
              f"PSNR {lg.psnr:.2f} dB ({', '.join(f'{x:.1f}' for x in lg.psnr_levels)}) {lg.ms_per_step:.3f} ms/step")
    assert logs[0].last_loss < 0.5 * logs[0].first_loss
    assert all(math.isfinite(lg.psnr) for lg in logs)
    assert logs[2].psnr >= logs[1].psnr - 0.05  # fine-tuning the MLP alone does not lose quality
    assert len(logs[0].psnr_levels) == w.target_levels
    # Sec. 6.5: partitions and initial blocks from the unconstrained warm-up beat random partitions
    # (measured on this problem: 28.4 dB vs 25.6 dB after 1,400 steps each)
    assert logs[2].psnr > rnd.psnr + 1.0


def test_trained_network_beats_plain_bc6h_storage():
    """What the network gains over the method without it.  The three-stage schedule with the step counts of
    Sec. 6.1 (5k unconstrained, 20k block, 1k fine-tuning) on four 64^2 feature textures (21.8 KB) against the
    nine reference channels stored directly as three BC6H textures and decoded by the same path: in mode 10
    alone (the features' own format) at 3/4 of the bytes, and per block the better of modes 10 and 11 at 3/4
    and at 3x the bytes."""
    _bcf()
    from paper_2311_16121_b300 import schedule

    w = workloads.train_workload(res=(64, 64, 64, 64), target_res=128, batch=1 << 14, dims=(13, 32, 32, 9))
    tr, _, logs = schedule.three_stage(w, warmup_steps=5000, bc_steps=20000, finetune_steps=1000)
    bcf_psnr = logs[-1].psnr
    exported, _ = schedule.eval_psnr_exported(tr, w)
    bytes_bcf = schedule.material_bytes(w.res, w.levels)
    print(f"BCf 4x64^2 {bytes_bcf} B PSNR {bcf_psnr:.2f} dB (exported {exported:.2f})")
    plain = {}
    for r, modes in ((64, (10,)), (64, (10, 11)), (128, (10, 11))):
        ps, pl, nbytes = schedule.classic_bc6h(w, r, modes=modes)
        plain[r, modes] = ps
        print(f"plain BC6H modes {modes} 3x{r}^2 {nbytes} B ({nbytes / bytes_bcf:.2f}x) PSNR {ps:.2f} dB "
              f"({', '.join(f'{x:.1f}' for x in pl)})")
        assert math.isfinite(ps) and len(pl) == w.target_levels
    # the exported blocks and FP16 weights lose nothing against the trainer's BF16 forward (the decode path's
    # FP16 weights and FP32 activations may gain a little: measured +0.0 to +0.13 dB)
    assert exported > bcf_psnr - 0.1
    # measured: 31.3 dB vs 28.6 (mode 10, 0.75x bytes), 29.0 (modes 10 + 11, 0.75x) and 29.2 (3x)
    assert bcf_psnr > plain[64, (10,)] + 2.0
    assert bcf_psnr > plain[128, (10, 11)] + 1.5


# --------------------------------------------------------------------------- SF16 and paper-literal emulation

VARIANTS = [(True, False), (False, True), (True, True)]


def _variant_workload(shape, signed):
    w = workloads.train_workload(**shape)
    if signed:  # SF16 codes in [-15, 15]: decoded values within about [-1, 1] (a = 31/32 doubles the UF16 scale)
        rng = np.random.default_rng(91)
        for p in w.params:
            e = np.r_[0:6, 8:14]
            p[:, e] = rng.uniform(-15, 15, (p.shape[0], 12)).astype(np.float32)
    return w


@pytest.mark.parametrize("shape", ["small", "medium"])
@pytest.mark.parametrize("signed,literal", VARIANTS)
def test_variant_forward_and_backward_match_oracle(shape, signed, literal):
    _bcf()
    w = _variant_workload(SMALL if shape == "small" else MEDIUM, signed)
    tr = workloads.upload_trainer(w, is_signed=signed, literal=literal)
    u, v, s = _queries(w.batch, w.target_levels - 1, seed=31)
    q = [torch.from_numpy(a).cuda() for a in (u, v, s)]
    F = oracle.TrainFeatures([workloads.params32_to_28(p).astype(np.float64) for p in w.params], w.partition, w.res,
                             w.levels, w.res_ref, lod_input=True, is_signed=signed, literal=literal)
    P = oracle.TrainMlp(w.dims, w.W, w.b, bf16=True)
    got = tr.forward(*q).cpu().numpy().astype(np.float64)
    _forward_check(got, F, P, u, v, s, (shape, signed, literal))
    go = np.random.default_rng(32).standard_normal((w.batch, 9)).astype(np.float32) * 1e-2
    tr.zero_grad()
    tr.backward(*q, torch.from_numpy(go).cuda())
    gf, gW, gb = oracle.train_backward_given(F, P, u, v, s, go.astype(np.float64))
    _grad_checks(F, P, u, v, s, go.astype(np.float64),
                 [("W", tr.W_grad.cpu().numpy(), gW, "W"), ("b", tr.b_grad.cpu().numpy(), gb, "b")] +
                 [(f"features{t}", workloads.params32_to_28(tr.grads[t].cpu().numpy()), gf[t], t)
                  for t in range(len(gf))])


def test_signed_export_decodes_to_the_emulated_features_and_adam_box():
    bcf = _bcf()
    w = _variant_workload(SMALL, True)
    w.params[0][:4, 0:6] = [[-32, 31, -0.49, 0.4, -31, 30.6]] * 4  # saturating codes, zero, ties
    tr = workloads.upload_trainer(w, is_signed=True)
    blocks, _ = tr.export()
    for t, blk in enumerate(blocks):
        got = blk.cpu().numpy().reshape(-1, 16)
        p28 = workloads.params32_to_28(w.params[t]).astype(np.float64)
        ref = np.stack([oracle.train_export_block(p28[i], int(w.partition[t][i]), is_signed=True)
                        for i in range(p28.shape[0])])
        np.testing.assert_array_equal(got, ref)
        W0 = w.res[t]
        img = bcf.decode_bc6h(blk[:(W0 // 4) ** 2 * 16].contiguous(), W0 // 4, W0 // 4, is_signed=True)
        img = img.cpu().numpy().view(np.uint16).view(np.float16).astype(np.float64)
        for bi in range((W0 // 4) ** 2):
            by, bx = divmod(bi, W0 // 4)
            for tx in range(16):
                for c in range(3):
                    assert img[4 * by + tx // 4, 4 * bx + tx % 4, c] == oracle.train_texel_v(
                        p28[bi], int(w.partition[t][bi]), tx, c, is_signed=True)
    # the optimiser's box for SF16 codes is [-32, 31]
    tr2 = workloads.upload_trainer(w, is_signed=True, lr_features=5.0)
    tr2.step(w.batch, 5, 0)
    for p in tr2.params:
        e = p[:, [0, 1, 2, 3, 4, 5, 8, 9, 10, 11, 12, 13]]
        assert float(e.min()) >= -32.0 and float(e.max()) <= 31.0 and float(e.min()) < 0.0


def test_literal_emulation_against_the_exact_default_after_export():
    """Eq. 7-8 as printed train a function that the exported blocks do not decode to; the exact emulation's
    export decodes to what it trained.  Both run the three-stage schedule from the same start."""
    _bcf()
    from paper_2311_16121_b300 import schedule

    w = workloads.train_workload(res=(64, 64, 64, 64), target_res=128, batch=1 << 14, dims=(13, 32, 32, 9))
    res = {}
    for literal in (False, True):
        tr, _, logs = schedule.three_stage(w, warmup_steps=300, bc_steps=900, finetune_steps=200, literal=literal)
        exp, _ = schedule.eval_psnr_exported(tr, w)
        res[literal] = (logs[-1].psnr, exp)
        print(f"{'literal' if literal else 'exact  '} emulated {logs[-1].psnr:.2f} dB, exported {exp:.2f} dB")
    assert abs(res[False][0] - res[False][1]) < 0.2  # exact: the export decodes to the trained features
    # literal: about 1 dB lost at export (measured: 28.31 dB emulated, 27.31 dB exported; exact 28.39 dB)
    assert res[True][1] < res[True][0] - 0.5 and res[True][1] < res[False][1] - 0.5


def test_grid_batches_loss_and_step_match_oracle():
    """The paper's batch form (Sec. 5.1): a 32 x 32 jittered uv grid with one scale per step."""
    bcf = _bcf()
    w = workloads.train_workload(**MEDIUM)
    G = 32
    tr = workloads.upload_trainer(w, lr_features=1e-2, lr_mlp=1e-3, gamma=0.9999, batch_grid=G)
    seed, step = 4242, 3
    loss = float(tr.step(G * G, seed, step).item())
    u, v, s = oracle.train_queries(seed, step, G * G, float(w.target_levels - 1), grid=G)
    F, P, T = _oracle_parts(w)
    ref_loss, _, _, _ = oracle.train_loss_grad(F, P, T, u, v, s)
    assert loss == pytest.approx(ref_loss, rel=2e-3)
    with pytest.raises(bcf.BcfError):
        tr.step(G * G + 1, seed, step)


@pytest.mark.parametrize("s_const", [0.3, 1.6, 3.2])
def test_grid_batch_gradients_match_oracle(s_const):
    """Grid trainers (the paper's batch form, Sec. 5.1) sum the endpoint updates of neighbouring lanes that share
    a block and region (a segmented warp scan) before their reductions; at a fine, a middle and a coarse scale
    (few blocks, most lanes sharing them) their gradients match the oracle's element by element."""
    _bcf()
    w = workloads.train_workload(**MEDIUM)
    G = 32
    tr = workloads.upload_trainer(w, batch_grid=G)
    u, v, _ = oracle.train_queries(4242, 3, G * G, float(w.target_levels - 1), grid=G)
    s = np.full(G * G, s_const, np.float32)
    go = np.random.default_rng(6).standard_normal((G * G, 9)).astype(np.float32) * 1e-2
    tr.zero_grad()
    tr.backward(*(torch.from_numpy(a).cuda() for a in (u, v, s)), torch.from_numpy(go).cuda())
    F, P, _ = _oracle_parts(w)
    gf, gW, gb = oracle.train_backward_given(F, P, u, v, s, go.astype(np.float64))
    _grad_checks(F, P, u, v, s, go.astype(np.float64),
                 [("W", tr.W_grad.cpu().numpy(), gW, "W"), ("b", tr.b_grad.cpu().numpy(), gb, "b")] +
                 [(f"features{t}", workloads.params32_to_28(tr.grads[t].cpu().numpy()), gf[t], t)
                  for t in range(len(gf))])


def test_checkpoint_resume_reproduces_the_run():
    """state_dict / load_state_dict: training 6 steps straight equals training 3, checkpointing into a fresh
    trainer, and training 3 more (same draws, since they depend only on seed and step)."""
    _bcf()
    w = workloads.train_workload(**MEDIUM)
    a = workloads.upload_trainer(w, lr_features=1e-2, lr_mlp=1e-3, gamma=0.9999)
    for i in range(6):
        a.step(w.batch, 31, i)
    b = workloads.upload_trainer(w, lr_features=1e-2, lr_mlp=1e-3, gamma=0.9999)
    for i in range(3):
        b.step(w.batch, 31, i)
    state = b.state_dict()
    c = workloads.upload_trainer(w, lr_features=1e-2, lr_mlp=1e-3, gamma=0.9999)
    c.load_state_dict(state)
    for i in range(3, 6):
        c.step(w.batch, 31, i)
    torch.cuda.synchronize()
    # the gradient reductions are atomics (order-free), so compare within the Adam step scale
    np.testing.assert_allclose(c.W.cpu().numpy(), a.W.cpu().numpy(), rtol=0, atol=3e-3)
    for pa, pc in zip(a.params, c.params):
        assert np.abs(pa.cpu().numpy() - pc.cpu().numpy()).max() <= 3e-2


# --------------------------------------------------------------------------- the paper's decoder on the tensor cores

PAPER = dict(res=(64, 32, 16, 16), target_res=128, batch=700, dims=(12, 16, 9))


@pytest.mark.parametrize("free", [False, True])
def test_paper_decoder_trains_on_the_tensor_cores_and_matches_oracle(free):
    """The paper's two-layer decoder (12 inputs, one hidden layer of 16, 9 outputs; Sec. 5.1) runs the
    tensor-core training kernel: forward under the strict output check, every gradient value within its
    per-element bound of the oracle's (block features and unconstrained features)."""
    _bcf()
    w = workloads.train_workload(**PAPER)
    if free:
        tex = workloads.free_texels(w)
        tr = workloads.upload_free_trainer(w, tex, lod_input=False)
        F = oracle.TrainFeatures([t[:, :3].astype(np.float64) for t in tex], None, w.res, w.levels, w.res_ref,
                                 lod_input=False, free=True)
    else:
        tr = workloads.upload_trainer(w, lod_input=False)
        F = oracle.TrainFeatures([workloads.params32_to_28(p).astype(np.float64) for p in w.params], w.partition,
                                 w.res, w.levels, w.res_ref, lod_input=False)
    P = oracle.TrainMlp(w.dims, w.W, w.b, bf16=True)
    u, v, s = _queries(w.batch, w.target_levels - 1, seed=51)
    q = [torch.from_numpy(a).cuda() for a in (u, v, s)]
    got = tr.forward(*q).cpu().numpy().astype(np.float64)
    ref = oracle.train_outputs(F, P, u, v, s)
    r = oracle.check_outputs(got, ref, TOL_BF16, False,
                             oracle.train_explainer(F, P, u, v, s, got, TOL_BF16, lod_input=False))
    assert not r["unexplained"], (r["unexplained"][:5], r["worst"])
    go = np.random.default_rng(52).standard_normal((w.batch, 9)).astype(np.float32) * 1e-2
    tr.zero_grad()
    tr.backward(*q, torch.from_numpy(go).cuda())
    gf, gW, gb = oracle.train_backward_given(F, P, u, v, s, go.astype(np.float64))
    feats = [(f"texels{t}", tr.grads[t].cpu().numpy()[:, :3], gf[t], t) for t in range(len(gf))] if free else \
        [(f"features{t}", workloads.params32_to_28(tr.grads[t].cpu().numpy()), gf[t], t) for t in range(len(gf))]
    _grad_checks(F, P, u, v, s, go.astype(np.float64),
                 [("W", tr.W_grad.cpu().numpy(), gW, "W"), ("b", tr.b_grad.cpu().numpy(), gb, "b")] + feats)
