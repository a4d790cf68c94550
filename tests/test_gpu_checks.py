"""Device-side checks: a kernel that meets malformed device data (a partition id above 31, material-set offsets
that decrease) sets a bit of the device's check word, takes the documented reading of the data and carries on;
bcf_device_check reports the bits and clears the word.  Every access of these runs stays in bounds: the ids are
read as id & 31 and the offsets are clipped to the query range."""
import numpy as np
import pytest
import torch

from paper_2311_16121_b300 import workloads

pytestmark = pytest.mark.gpu

SMALL = dict(res=(16, 8), target_res=32, batch=384, dims=(7, 8, 8, 9))
MEDIUM = dict(res=(64, 64, 64, 64), target_res=128, batch=600, dims=(13, 32, 32, 9))


def _bcf():
    import paper_2311_16121_b300 as bcf

    bcf.lib()
    bcf.device_check(raise_on_failure=False)  # start from a clear word
    return bcf


def _queries(n, s_max, seed=3):
    rng = np.random.default_rng(seed)
    return (torch.from_numpy(rng.random(n, dtype=np.float32)).cuda(),
            torch.from_numpy(rng.random(n, dtype=np.float32)).cuda(),
            torch.from_numpy(rng.uniform(0, s_max, n).astype(np.float32)).cuda())


def test_clean_work_leaves_the_word_clear():
    bcf = _bcf()
    w = workloads.train_workload(**SMALL)
    tr = workloads.upload_trainer(w)
    for k in range(3):
        tr.step(w.batch, 7, k)
    tr.export()
    sw = workloads.config4(n_materials=3, q_range=(300, 3000), res_choices=(32, 64), pool=1 << 12, config=46)
    S = bcf.MaterialSet([workloads.upload(m, "fp16") for m in sw.materials])
    u, v, s = (torch.from_numpy(a).cuda() for a in sw.concat())
    S.decode(torch.from_numpy(sw.offsets).cuda(), u, v, s)
    # a decode with the MLP on tcgen05 (its bounded MMA waits are what BCF_CHECK_TIMEOUT reports)
    m = workloads.upload(sw.materials[0], "fp16")
    m.set_decode_variant(0)
    m.set_mlp_engine("tcgen05")
    a, b = int(sw.offsets[0]), int(sw.offsets[1])
    m.decode(u[a:b], v[a:b], s[a:b])
    assert bcf.device_check() == 0


@pytest.mark.parametrize("shape", ["small", "medium"])
def test_partition_above_31_reads_as_its_low_bits_and_sets_the_check(shape):
    """The SIMT (small MLP) and tensor-core (13-32-32-9) training kernels and the export read an id k > 31 as
    k & 31: the outputs, gradients and exported blocks equal those of the valid ids bit for bit.  The export and
    the optimiser of a training step (which see every block once) set the check; forward and backward alone
    only mask."""
    bcf = _bcf()
    w = workloads.train_workload(**(SMALL if shape == "small" else MEDIUM))
    tr = workloads.upload_trainer(w)
    u, v, s = _queries(w.batch, w.target_levels - 1)
    ref = tr.forward(u, v, s).clone()
    go = torch.randn(w.batch, 9, device="cuda") * 1e-2
    tr.zero_grad()
    tr.backward(u, v, s, go)
    torch.cuda.synchronize()
    ref_grads = [g.clone() for g in tr.grads]
    ref_blocks, _ = tr.export()
    assert bcf.device_check() == 0

    rng = np.random.default_rng(9)
    for k in tr.partition:  # every id gets a multiple of 32 added (ids stay below 256)
        k += torch.from_numpy(rng.integers(1, 8, k.numel()).astype(np.uint8) * 32).cuda()
    assert int(min(k.min() for k in tr.partition)) >= 32
    got = tr.forward(u, v, s)
    torch.testing.assert_close(got, ref, rtol=0, atol=0)
    tr.zero_grad()
    tr.backward(u, v, s, go)
    torch.cuda.synchronize()
    for g, r in zip(tr.grads, ref_grads):  # scatter order may differ between runs: FP32 atomics
        torch.testing.assert_close(g, r, rtol=1e-4, atol=1e-5 * float(r.abs().max()) + 1e-12)
    assert bcf.device_check() == 0  # forward and backward mask without checking
    blocks, _ = tr.export()
    for a, b in zip(blocks, ref_blocks):
        assert torch.equal(a, b)
    with pytest.raises(bcf.BcfError) as err:
        bcf.device_check()
    assert err.value.status == 6 and "partition" in str(err.value)
    assert bcf.device_check() == 0  # read and cleared
    tr.zero_grad()
    tr.step(w.batch, 7, 0)
    assert bcf.device_check(raise_on_failure=False) & bcf.CHECK_PARTITION


@pytest.mark.parametrize("variant", [0, 3])
def test_decreasing_set_offsets_set_the_check_and_decode_an_empty_range(variant):
    """Material 1's end offset lies below its start: its range is empty, the other materials decode as they do
    alone (rows that two materials' ranges both cover are skipped), and the offsets bit is set."""
    bcf = _bcf()
    sw = workloads.config4(n_materials=4, q_range=(300, 6000), res_choices=(32, 64, 128), pool=1 << 14, config=47)
    mats = [workloads.upload(m, "fp16") for m in sw.materials]
    for m in mats:
        m.set_decode_variant(variant)
    S = bcf.MaterialSet(mats)
    u, v, s = (torch.from_numpy(a).cuda() for a in sw.concat())
    offs = sw.offsets.copy()
    overlap = 37
    offs[2] = offs[1] - overlap  # material 2 now starts inside material 0's range
    got = S.decode(torch.from_numpy(offs).cuda(), u, v, s).cpu().numpy()
    with pytest.raises(bcf.BcfError) as err:
        bcf.device_check()
    assert err.value.status == 6 and "offsets" in str(err.value)
    ranges = {0: (int(offs[0]), int(offs[1]) - overlap), 2: (int(offs[1]), int(offs[3])),
              3: (int(offs[3]), int(offs[4]))}
    for m, (a, b) in ranges.items():
        one = mats[m].decode(u[a:b], v[a:b], s[a:b], out_dtype=torch.float16).cpu().numpy()
        np.testing.assert_array_equal(got[a:b], one)
    assert bcf.device_check() == 0
