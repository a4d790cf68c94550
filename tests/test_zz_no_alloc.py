"""The allocation-free training step (bcf_train_step_noalloc).

Some callers cannot allocate device memory -- an engine that owns every
device byte through its own budgeted allocator, or a frame loop that must
not call cudaMalloc.  For them the library offers a training step whose
gradient scratch lives in one library-owned device array instead of caller
buffers.  These tests call that entry point through the C ABI twice in a row
and check that it gives what the ordinary bcf_train_step gives on an
identical trainer, within the tolerances of the other training tests, for
the batch forms that change the scratch layout or the kernel chosen:
internally drawn random batches, caller-supplied queries, grid batches and
unconstrained (per-texel) features.  They also check that a trainer too
large for the array, and a grid trainer given a batch that is not its grid,
are refused before any work is launched.  They run alone or after the other
tests (the array keeps the previous call's contents, which the entry point
clears).
"""
import numpy as np
import pytest
import torch

from paper_2311_16121_b300 import workloads

pytestmark = pytest.mark.gpu

SHAPE = dict(res=(64, 64, 64, 64), target_res=128, batch=1024, dims=(13, 32, 32, 9))


def _close(a, b, lr):
    """Element-wise agreement of two Adam-updated arrays: where the gradient is clearly non-zero the updates
    agree to float rounding; everywhere they stay within one learning-rate step of each other."""
    a = a.astype(np.float64)
    b = b.astype(np.float64)
    diff = np.abs(a - b)
    assert diff.max() <= 2 * lr + 1e-6, diff.max()
    assert (diff > 1e-5 + 1e-4 * np.abs(b)).mean() <= 2e-3


def _pair(form, w):
    hyper = dict(lr_features=1e-2, lr_mlp=1e-3, gamma=0.9999)
    if form == "grid":
        hyper["batch_grid"] = 32  # batch 1024 = 32^2
    if form == "unconstrained":
        return workloads.upload_free_trainer(w, **hyper), workloads.upload_free_trainer(w, **hyper)
    return workloads.upload_trainer(w, **hyper), workloads.upload_trainer(w, **hyper)


@pytest.mark.parametrize("form", ["random", "caller_queries", "grid", "unconstrained"])
def test_noalloc_step_matches_train_step_on_two_calls(form):
    import paper_2311_16121_b300 as bcf

    bcf.lib()
    w = workloads.train_workload(**SHAPE)
    ref, new = _pair(form, w)
    before = [g.clone() for g in new.grads]
    q = None
    if form == "caller_queries":
        rng = np.random.default_rng(11)
        q = [torch.from_numpy(a).cuda() for a in (rng.random(w.batch, dtype=np.float32),
                                                  rng.random(w.batch, dtype=np.float32),
                                                  rng.uniform(0, w.target_levels - 1, w.batch).astype(np.float32))]
    for step in (0, 1):
        args = (w.batch, 99, step) + (tuple(q) if q else ())
        l_ref = float(ref.step(*args).item())
        l_new = float(new.step_noalloc(*args).item())
        assert l_new == pytest.approx(l_ref, rel=1e-5)
    torch.cuda.synchronize()
    _close(new.W.cpu().numpy(), ref.W.cpu().numpy(), 1e-3)
    _close(new.b.cpu().numpy(), ref.b.cpu().numpy(), 1e-3)
    for t in range(len(w.params)):
        _close(new.params[t].cpu().numpy(), ref.params[t].cpu().numpy(), 1e-2)
        _close(new.m[t].cpu().numpy(), ref.m[t].cpu().numpy(), 1e-2)
    # the trainer's own gradient arrays are not used by the allocation-free step
    for g0, g1 in zip(before, new.grads):
        assert torch.equal(g0, g1)


def test_noalloc_step_refuses_a_trainer_beyond_the_scratch_size():
    import paper_2311_16121_b300 as bcf

    bcf.lib()
    w = workloads.train_workload(res=(1024,), target_res=128, batch=64, dims=(4, 8, 8, 9))  # 2.8M values
    tr = workloads.upload_trainer(w)
    before = tr.params[0].clone()
    with pytest.raises(bcf.BcfError) as e:
        tr.step_noalloc(w.batch, 1, 0)
    assert e.value.status == 2 and "scratch" in str(e.value)
    torch.cuda.synchronize()
    assert torch.equal(before, tr.params[0])


def test_noalloc_step_refuses_a_grid_batch_that_is_not_the_grid():
    import paper_2311_16121_b300 as bcf

    bcf.lib()
    w = workloads.train_workload(**SHAPE)
    tr = workloads.upload_trainer(w, batch_grid=32)
    before = tr.params[0].clone()
    with pytest.raises(bcf.BcfError) as e:
        tr.step_noalloc(1000, 1, 0)
    assert e.value.status == 1 and "grid" in str(e.value)
    torch.cuda.synchronize()
    assert torch.equal(before, tr.params[0])
