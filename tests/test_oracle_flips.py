"""Pins of the oracle's rounding-flip explanation (oracle_mlp_explain,
oracle_train_mlp_explain) and of its per-element gradient bounds
(oracle_train_backward_bounds), which the strict GPU parity tests use.

A plain numpy model of a device evaluation -- single-precision inputs a few
units in the last place away from the exact ones, layer inputs rounded by the
library casts (numpy float16, torch bfloat16 / float8_e4m3fn), single-
precision sums in an order of its own -- must always be explained where it
misses the tolerance; outputs with a planted mistake (a shifted channel, a
dropped bias, a wrong-signed weight) must not be.
"""
import numpy as np
import pytest
import torch

import oracle

RNG = np.random.default_rng(20231121)


def _round(prec, a):
    a = np.asarray(a, np.float32)
    if prec == "fp16":
        return a.astype(np.float16).astype(np.float32)
    if prec == "bf16":
        return torch.from_numpy(a).to(torch.bfloat16).float().numpy()
    if prec == "fp8":
        return torch.from_numpy(np.clip(a, -448, 448)).to(torch.float8_e4m3fn).float().numpy()
    return a


def _net(dims, prec, rng):
    Ws, bs = [], []
    for l in range(len(dims) - 1):
        Ws.append(rng.standard_normal((dims[l + 1], dims[l])) / np.sqrt(dims[l]))
        bs.append((rng.standard_normal(dims[l + 1]) * 0.1).astype(np.float32))
    act = np.full(len(Ws), 1.0 / 64.0, np.float32) if prec == "fp8" else None
    wsc = None
    if prec == "fp8":
        wsc = np.array([2.0 ** np.ceil(np.log2(np.abs(W).max() / 448.0)) for W in Ws], np.float32)
        stored = [torch.from_numpy((W / s).astype(np.float32)).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
                  for W, s in zip(Ws, wsc)]
        vals = [torch.from_numpy(st).view(torch.float8_e4m3fn).double().numpy() * s for st, s in zip(stored, wsc)]
        flat = np.concatenate([st.ravel() for st in stored])
    elif prec == "fp16":
        stored = [W.astype(np.float16) for W in Ws]
        vals = [st.astype(np.float64) for st in stored]
        flat = np.concatenate([st.ravel() for st in stored]).view(np.uint16)
    else:
        stored = [torch.from_numpy(W.astype(np.float32)).to(torch.bfloat16) for W in Ws]
        vals = [st.double().numpy() for st in stored]
        flat = np.concatenate([st.view(torch.int16).numpy().ravel() for st in stored]).view(np.uint16)
    P = oracle.Mlp(list(dims), prec, flat, np.concatenate(bs), act, wsc)
    return P, vals, bs, act, wsc


def _device(x, vals, bs, prec, act, wsc, rng, order_seed=0):
    """A single-precision evaluation of the network in its own summation order."""
    h = (x * (1.0 + rng.uniform(-4, 4, x.shape) * 2.0 ** -24)).astype(np.float32)
    for l, (W, b) in enumerate(zip(vals, bs)):
        a = h / np.float32(act[l]) if prec == "fp8" else h
        q = _round(prec, a)
        Wd = (W / wsc[l]).astype(np.float32) if prec == "fp8" else W.astype(np.float32)
        order = np.random.default_rng(order_seed + l).permutation(W.shape[1])
        acc = np.zeros((x.shape[0], W.shape[0]), np.float32)
        for i in order:
            acc = (acc + q[:, i:i + 1] * Wd[:, i][None, :]).astype(np.float32)
        if prec == "fp8":
            acc = (acc * np.float32(act[l] * wsc[l])).astype(np.float32)
        h = (acc + b[None, :]).astype(np.float32)
        if l + 1 < len(vals):
            h = np.maximum(h, np.float32(0))
    return h.astype(np.float64)


@pytest.mark.parametrize("prec,tol", [("fp16", 1e-3), ("bf16", 4e-3), ("fp8", 4e-3)])
def test_device_model_misses_are_all_explained_and_planted_mistakes_are_not(prec, tol):
    dims = (13, 32, 32, 9)
    P, vals, bs, act, wsc = _net(dims, prec, RNG)
    n = 3000
    x = RNG.random((n, dims[0]))
    x[:, -1] *= 8.0
    if prec == "fp8":  # half the rows with input 0 on an E4M3 rounding midpoint (in scaled units)
        grid = torch.arange(0, 127, dtype=torch.uint8).view(torch.float8_e4m3fn).double().numpy()
        mids = (grid[1:] + grid[:-1]) / 2 * act[0]
        x[: n // 2, 0] = RNG.choice(mids[(mids > 0.1) & (mids < 1.0)], n // 2)
    dev = _device(x, vals, bs, prec, act, wsc, RNG, order_seed=5)
    ref = np.stack([oracle.mlp_one(P, x[i], quant_aware=True) for i in range(n)])
    err = np.abs(dev - ref)
    rows = np.nonzero((err > tol).any(axis=1))[0]
    xe = 2.0 ** -20 * np.abs(x) + 2.0 ** -21
    for r in rows:
        assert oracle.mlp_explain(P, x[r], xe[r], dev[r], tol) == 1, (r, err[r].max())
    if prec == "fp8":
        assert rows.size > 0  # E4M3 flips do exceed the tolerance: the pin exercises the enumeration
    # planted mistakes are not explained
    for r in range(20):
        shifted = dev[r].copy()
        shifted[r % 9] += 10 * tol
        assert oracle.mlp_explain(P, x[r], xe[r], shifted, tol) == 0
    nobias = [np.zeros_like(b) for b in bs]
    dev2 = _device(x[:200], vals, nobias, prec, act, wsc, RNG)
    assert sum(oracle.mlp_explain(P, x[i], xe[i], dev2[i], tol) for i in range(200)) == 0
    bad_vals = [W.copy() for W in vals]
    bad_vals[-1][2, :] = -bad_vals[-1][2, :]  # a transposed sign in one output row
    dev3 = _device(x[:200], bad_vals, bs, prec, act, wsc, RNG)
    bad = np.abs(dev3 - ref[:200]).max(axis=1) > 3 * tol
    assert bad.sum() > 100
    assert all(oracle.mlp_explain(P, x[i], xe[i], dev3[i], tol) == 0 for i in np.nonzero(bad)[0])


def test_exact_outputs_and_fp16_storage_are_explained():
    P, vals, bs, act, wsc = _net((6, 16, 8), "fp16", RNG)
    x = RNG.random((50, 6))
    xe = np.full_like(x, 1e-7)
    for i in range(50):
        y = oracle.mlp_one(P, x[i], quant_aware=True)
        assert oracle.mlp_explain(P, x[i], xe[i], y, 1e-3) == 1
        assert oracle.mlp_explain(P, x[i], xe[i], y.astype(np.float16).astype(np.float64), 1e-3, out_half=True) == 1


def test_a_rounding_midpoint_input_admits_both_roundings():
    """An FP16 input exactly halfway between two halves: a device value on either side rounds differently;
    both outputs are explained when the window covers the midpoint, only the exact one when it does not."""
    dims = (2, 9)
    W = np.zeros((9, 2), np.float16)
    W[:, 0] = 1.0
    P = oracle.Mlp(list(dims), "fp16", W.view(np.uint16).ravel(), np.zeros(9, np.float32))
    lo = np.float16(0.5)
    hi = np.nextafter(lo, np.float16(1))
    mid = (float(lo) + float(hi)) / 2
    x = np.array([mid, 0.0])
    for y0 in (float(lo), float(hi)):
        assert oracle.mlp_explain(P, x, np.array([1e-6, 0.0]), np.full(9, y0), 1e-5) == 1
    ties_even = float(lo)  # 0.5 has the even significand
    other = float(hi)
    assert oracle.mlp_explain(P, x, np.zeros(2), np.full(9, ties_even), 1e-5) == 1
    assert oracle.mlp_explain(P, x, np.zeros(2), np.full(9, other), 1e-5) == 0


def test_training_network_explanation_with_bfloat16():
    dims = (13, 32, 32, 9)
    Ws = [RNG.standard_normal((dims[l + 1], dims[l])) / np.sqrt(dims[l]) for l in range(3)]
    bs = [RNG.standard_normal(dims[l + 1]) * 0.1 for l in range(3)]
    P = oracle.TrainMlp(list(dims), np.concatenate([w.ravel() for w in Ws]), np.concatenate(bs), bf16=True)
    vals = [torch.from_numpy(w.astype(np.float32)).to(torch.bfloat16).double().numpy() for w in Ws]
    n = 2000
    x = RNG.random((n, 13))
    dev = _device(x, vals, [b.astype(np.float32) for b in bs], "bf16", None, None, RNG, order_seed=9)
    xe = 2.0 ** -20 * np.abs(x) + 2.0 ** -21
    mlp = oracle.Mlp(list(dims), "bf16",
                     np.concatenate([torch.from_numpy(w.astype(np.float32)).to(torch.bfloat16).view(torch.int16)
                                     .numpy().ravel() for w in Ws]).view(np.uint16),
                     np.concatenate(bs).astype(np.float32))
    ref = np.stack([oracle.mlp_one(mlp, x[i], quant_aware=True) for i in range(n)])
    rows = np.nonzero((np.abs(dev - ref) > 4e-3).any(axis=1))[0]
    for r in rows:
        assert oracle.train_mlp_explain(P, x[r], xe[r], dev[r], 4e-3) == 1
    for r in range(10):
        y = dev[r].copy()
        y[0] -= 0.05
        assert oracle.train_mlp_explain(P, x[r], xe[r], y, 4e-3) == 0


def test_gradient_bounds_are_the_gradients_when_every_term_is_positive():
    """With positive weights, biases, features and output gradients every term of the weight and bias
    gradients is positive, so the absolute-term sums equal the gradients; without operand rounding and away
    from ReLU zeros nothing is left open (R = 0)."""
    from paper_2311_16121_b300 import workloads

    w = workloads.train_workload(res=(16, 8), target_res=32, batch=64, dims=(7, 8, 8, 9))
    F = oracle.TrainFeatures([workloads.params32_to_28(p).astype(np.float64) for p in w.params], w.partition, w.res,
                             w.levels, w.res_ref, lod_input=True)
    Wp = np.abs(w.W.astype(np.float64)) + 0.01
    bp = np.abs(w.b.astype(np.float64)) + 0.1
    rng = np.random.default_rng(3)
    u, v = rng.random(64, dtype=np.float32), rng.random(64, dtype=np.float32)
    s = rng.uniform(0, 3, 64).astype(np.float32)
    go = rng.random((64, 9)) + 0.1
    for bf16 in (False, True):
        P = oracle.TrainMlp(w.dims, Wp, bp, bf16=bf16)
        gf, gW, gb = oracle.train_backward_given(F, P, u, v, s, go)
        (Af, AW, Ab), (Rf, RW, Rb) = oracle.train_backward_bounds(F, P, u, v, s, go)
        np.testing.assert_allclose(AW, gW, rtol=1e-12)
        np.testing.assert_allclose(Ab, gb, rtol=1e-12)
        for a, g in zip(Af, gf):
            assert (a >= np.abs(g) * (1 - 1e-12)).all()
        if not bf16:
            assert not RW.any() and not Rb.any() and not any(r.any() for r in Rf)
        else:
            assert (RW >= 0).all()
