"""Benchmark of the BCf decode hot path (BC6H unpack + trilinear filter + MLP) on B300.

One step = one full decode of the screen workload through ``bcf_decode_material``:
4 BC6H feature textures of 2048^2 with full mip chains (value-bounded random
blocks over all 14 modes), 3840x2160 queries of a perspective-viewed tiled
plane (uv and LOD from the per-pixel screen Jacobian), MLP 13-32-32-9 on the
tensor cores.  The timed configuration is decode variant 0: the library's own
BC6H decoder (16-byte block loads, blocks mode-sorted and decoded into a
shared-memory texel arena per 512-query tile), the exact FP32 trilinear
filter, and the MLP per warp on mma.sync (for this narrow 16-bit network the
faster engine; the tcgen05 engine -- 128-row MMAs, accumulators in tensor
memory -- is timed beside it and runs the FP8 and 25-64-64-9 paths).  Beside
it: the same decode with the texels fetched through the texture unit's BC6H
decoder (variant 3, the paper's render-time design; bit-identical texels) and
the hardware-trilinear comparator.  ``value`` is the
whole-job decode throughput in Gsamples/s with inputs resident in HBM;
``e2e`` is the same metric through the C ABI with the queries in pinned host
memory and the decoded channels read back every step.

Extra keys report the FP32 SIMT plain path and the FP8 path on the same frame,
the batched 64-material launch, the 8x4096^2 frame (FP8 / FP16 / FP32), the
small 2x256^2 launch, training steps/s, the roofline of the dominant kernel
(HBM, with the issue and tensor co-bounds), the measured FP8 and derived FP32
peaks, the CPU oracle on a bounded sample and, from the same oracle run, the
per-channel error of every path against the exact FP64 decode.

Multi-GPU: the decode shards by queries with no exchange step; each rank
decodes its own full frame (replicas, weak scaling), and rank 0 reports the
total samples of all ranks over the slowest rank's time.

``--impl reference`` times the CPU oracle (the only reference implementation
of this method) on the same workload and metric, a bounded sample per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gsamples/s BCf decode (BC6H+filter+MLP) low-prec vs FP32 plain; train steps/s"
HEADLINE_PRECISION = "fp16"
# bcf_set_decode_variant / bcf_set_mlp_engine of the timed low-precision paths: variant 0 = the library's
# BC6H decoder (tile-cooperative, shared-memory texel arena), the exact FP32 filter.  The MLP engine per path is
# the faster of the two measured on it: the per-warp mma.sync MLP for the narrow 16-bit 13-32-32-9 network (no
# per-layer MMA round trip through tensor memory to wait for), tcgen05 for E4M3 operands and for the 64-wide
# 25-64-64-9 network; the other engine is timed beside each.
HEADLINE_VARIANT = 0
HEADLINE_ENGINE = "mma_sync"
FP8_ENGINE = "tcgen05"
LARGE_ENGINE = "tcgen05"
OTHER_ENGINE = {"mma_sync": "tcgen05", "tcgen05": "mma_sync"}
TEXUNIT_VARIANT = 3  # the same decode on the texture unit's BC6H texels (point sampling, bit-exact)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), "measured"
    except Exception:
        return 6400.0, 1800.0, "fallback"


# DRAM traffic and executed warp instructions of one launch of the headline kernel, from one full ncu
# capture of it on the same workload.  They are reported only while the
# kernel's sources hash to the value the capture was taken on; after any change they read as null.
KERNEL_SOURCES = ["bcf_decode_tiled.cu", "bc6h_unpack.cuh", "bcf_sample.cuh", "bcf_mlp.cuh", "bcf_tcmlp.cuh",
                  "bcf_internal.h"]
NCU_CAPTURE = {"engine": "mma_sync", "source_sha256": "de116da64dfaed27", "dram_bytes": 121470464 + 113908992,
               "warp_inst": 561815026, "issue_active_pct": 62.21, "tensor_pipe_pct": 7.35, "warps_active_pct": 46.76}
SM_COUNT, SMSP_PER_SM, FP32_LANES_PER_SM = 148, 4, 128


def _kernel_sha():
    import hashlib

    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2311_16121_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _fp8_tflops(torch, n=8192, iters=20):
    """Dense FP8 E4M3 peak of this GPU, measured with the library GEMM (burst, like the BF16 figure)."""
    try:
        a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()
        one = torch.ones((), device="cuda")
        for _ in range(3):
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(iters):
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        e1.record()
        e1.synchronize()
        return 2.0 * n ** 3 * iters / (e0.elapsed_time(e1) * 1e-3) / 1e12
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_samples(self, n: int, timeout: float = 3.0) -> None:
        """Block until `n` sample lines have arrived (or the timeout passes)."""
        t0 = time.time()
        while self.proc and len(self.lines) < n and time.time() - t0 < timeout:
            time.sleep(0.005)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, first: int = 0):
        """Median SM clock, maximum clock and the throttle reasons seen in the samples from index `first` on."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines[first:]:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _cpu_baseline(w, precision, gpu_out, seconds=12.0):
    """The oracle (plain FP64 C, all host cores) on a seeded uniform sample of the frame's queries.

    The same run also gives the accuracy of the GPU outputs: ``gpu_out`` maps a
    precision to a callable returning that path's FP32 outputs at given query
    indices.  Each path is compared with the exact FP64 decode (FP32 master
    weights, no rounding anywhere) on the first 2^16 sampled queries, and the
    timed path with the quantisation-aware oracle on the whole sample."""
    import oracle

    mat = oracle.Material(w.blocks, w.res, w.levels, w.res_ref, w.is_signed, w.wrap, w.lod_input)
    Wst, bias, a, ws = w.weights(precision)
    P = oracle.Mlp(w.dims, precision, Wst, bias, a, ws)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(7)
    n = 1 << 16
    rate = 0.0
    for _ in range(2):  # calibrate the sample size on the host's actual throughput
        idx = rng.integers(0, w.n, n)
        t = time.perf_counter()
        oracle.decode(mat, P, w.u[idx], w.v[idx], w.s[idx], quant_aware=True, threads=cores)
        rate = n / max(time.perf_counter() - t, 1e-6)
        n = int(min(max(rate * 2.0, 1 << 16), w.n))
    n = int(min(max(rate * seconds, 1 << 16), w.n))
    idx = rng.integers(0, w.n, n)
    t = time.perf_counter()
    ref_q = oracle.decode(mat, P, w.u[idx], w.v[idx], w.s[idx], quant_aware=True, threads=cores)
    dt = time.perf_counter() - t
    cpu = {"value": n / dt / 1e9, "unit": "Gsamples/s", "cores": cores, "kind": "oracle",
           "sample": f"{n} queries drawn uniformly (seed 7) from the {w.n}-query frame, {precision} "
                     f"quantisation-aware FP64 decode, {dt:.1f} s"}

    # accuracy
    W32, b32, _, _ = w.weights("fp32")
    exact = oracle.decode(mat, oracle.Mlp(w.dims, "fp32", W32, b32), w.u[idx[:1 << 16]], w.v[idx[:1 << 16]],
                          w.s[idx[:1 << 16]], quant_aware=False, threads=cores)

    def stats(d):
        return {"max_abs": [float(f"{x:.3g}") for x in np.abs(d).max(axis=0)],
                "rms": [float(f"{x:.3g}") for x in np.sqrt((d * d).mean(axis=0))],
                "p99.9_abs": [float(f"{x:.3g}") for x in np.quantile(np.abs(d), 0.999, axis=0)]}

    acc = {"reference": "exact FP64 decode with the FP32 master weights, 65536 sampled queries, per channel"}
    for prec, get in gpu_out.items():
        acc[prec] = stats(get(idx[:1 << 16]).astype(np.float64) - exact)
    # parity per low precision against the quantisation-aware oracle at the absolute tolerance (FP16 output):
    # outputs beyond it, and how many of their rows the oracle explains as operand-rounding flips
    tols = {"fp16": 1e-3, "bf16": 4e-3, "fp8": 4e-3}
    acc["vs_quantisation_aware_oracle"] = {}
    for prec in [p for p in tols if p in gpu_out]:
        sel = idx if prec == precision else idx[:1 << 16]
        if prec == precision:
            Pq, rq = P, ref_q
        else:
            Wq, bq, aq, wq = w.weights(prec)
            Pq = oracle.Mlp(w.dims, prec, Wq, bq, aq, wq)
            rq = oracle.decode(mat, Pq, w.u[sel], w.v[sel], w.s[sel], quant_aware=True, threads=cores)
        got = gpu_out[prec](sel).astype(np.float64)
        r = oracle.check_outputs(got, rq, tols[prec], True,
                                 oracle.decode_explainer(mat, Pq, w.u[sel], w.v[sel], w.s[sel], got, tols[prec],
                                                         True))
        d = np.abs(got - rq.astype(np.float16).astype(np.float64))
        acc["vs_quantisation_aware_oracle"][prec] = {
            "queries": int(sel.size), "tol_abs": tols[prec], "max_abs": float(f"{d.max():.3g}"),
            "frac_above_tol": float(f"{r['beyond_tol'] / max(r['outputs'], 1):.3g}"),
            "rows_beyond_tol": r["rows_beyond"], "rows_explained_as_flips": r["flips"],
            "rows_unexplained": len(r["unexplained"])}
    return cpu, acc


def run_reference(args):
    """The CPU oracle as the reference arm (bounded sample per step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2311_16121_b300 import workloads

    w = workloads.config2()
    mat = oracle.Material(w.blocks, w.res, w.levels, w.res_ref, w.is_signed, w.wrap, w.lod_input)
    Wst, bias, a, ws = w.weights(HEADLINE_PRECISION)
    P = oracle.Mlp(w.dims, HEADLINE_PRECISION, Wst, bias, a, ws)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(11)
    per_step = 1 << 16
    total_q, total_t = 0, 0.0
    for step in range(args.warmup + args.steps):
        idx = rng.integers(0, w.n, per_step)
        t = time.perf_counter()
        oracle.decode(mat, P, w.u[idx], w.v[idx], w.s[idx], quant_aware=True, threads=cores)
        dt = time.perf_counter() - t
        if step >= args.warmup:
            total_q += per_step
            total_t += dt
    value = total_q / total_t / 1e9
    sample = f"{per_step} queries per step drawn uniformly from the {w.n}-query frame (FP64 oracle, {cores} threads)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gsamples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name + ": " + "4x BC6H 2048^2 full mips, 3840x2160 plane "
                                                                        "queries, MLP 13-32-32-9", "sample": sample},
            "cpu_baseline": {"value": value, "unit": "Gsamples/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "Gsamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _train_bench(torch, workloads, stream, k_train, shape="config3"):
    """Training steps/s: 4 block-parameterised 1024^2 textures with mips, 2048^2 9-channel reference,
    batch 2^20 Philox draws, MLP 13-32-32-9 (BF16 operands), Adam.  shape="paper": the paper's BCf-1K
    textures (1024 / 512 / 256 / 128) and its 12-16-9 decoder without the LOD input.  Returns (ms/step, last
    loss, batch)."""
    if shape == "paper":
        tw = workloads.train_workload(res=(1024, 512, 256, 128), target_res=2048, dims=(12, 16, 9))
        tr = workloads.upload_trainer(tw, lod_input=False)
    elif shape == "grid":  # the paper's batch form: a jittered 1024 x 1024 uv grid with one scale per step
        tw = workloads.train_workload()
        tr = workloads.upload_trainer(tw, batch_grid=1024)
    else:
        tw = workloads.train_workload()
        tr = workloads.upload_trainer(tw)
    for i in range(3):
        tr.step(tw.batch, 7, i)
    torch.cuda.synchronize()
    ta = torch.cuda.Event(enable_timing=True)
    tb = torch.cuda.Event(enable_timing=True)
    ta.record(stream)
    for i in range(k_train):
        tr.step(tw.batch, 7, 3 + i)
    tb.record(stream)
    tb.synchronize()
    return ta.elapsed_time(tb) / k_train, float(tr.loss.item()), tw.batch


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-train", action="store_true",
                    help="time only the training step (for profiler captures); prints a reduced line")
    ap.add_argument("--train-shape", default="config3", choices=["config3", "paper", "grid"],
                    help="with --only-train: the timed workload's decoder (paper = BCf-1K textures, 12-16-9)")
    ap.add_argument("--only-large", action="store_true",
                    help="time only the 8 x 4096^2 frame on the hand-written decode, FP16 and FP8 (for profiler "
                         "captures); prints a reduced line")
    ap.add_argument("--only-batched", action="store_true",
                    help="time only the 64-material set, one graph-replayed launch on the hand-written decode (for "
                         "profiler captures); prints a reduced line")
    ap.add_argument("--only-encode", action="store_true",
                    help="time only the partition-selection encoder, 4 x 1024^2 with 9 levels (for profiler captures); "
                         "prints a reduced line")
    ap.add_argument("--only-headline", action="store_true",
                    help="time only the headline decode (for profiler captures); prints a reduced line")
    ap.add_argument("--only-fp8", action="store_true",
                    help="time only the headline frame in E4M3 on its engine (for profiler captures); prints a "
                         "reduced line")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    import paper_2311_16121_b300 as bcf
    from paper_2311_16121_b300 import workloads

    from paper_2311_16121_b300 import replicas

    rank, world, local = replicas.rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    bcf.lib()
    assert args.warmup >= 3, "at least 3 warm-up steps"

    stream = torch.cuda.current_stream()
    if args.only_encode:
        enc_res, enc_levels = 1024, 9
        n_texels = sum((enc_res >> l) ** 2 for l in range(enc_levels))
        g = torch.Generator(device="cuda").manual_seed(5)
        enc_tex = [torch.rand(n_texels * 3, device="cuda", generator=g) for _ in range(4)]
        enc_out = [bcf.encode_mode10(t, enc_res, enc_levels) for t in enc_tex]
        for _ in range(args.warmup - 1):
            for t, (pp, pk, pe) in zip(enc_tex, enc_out):
                bcf.encode_mode10(t, enc_res, enc_levels, pp, pk, pe)
        torch.cuda.synchronize()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        for _ in range(args.steps):
            for t, (pp, pk, pe) in zip(enc_tex, enc_out):
                bcf.encode_mode10(t, enc_res, enc_levels, pp, pk, pe)
        eb.record(stream)
        eb.synchronize()
        ms = ea.elapsed_time(eb) / args.steps
        blocks = 4 * bcf.texture_blocks(enc_res, enc_levels)
        if rank == 0:
            print(json.dumps({"metric": "blocks/s", "value": blocks / (ms * 1e-3), "unit": "blocks/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                              "note": "capture mode: the encoder only"}))
        return

    if args.only_large or args.only_batched:
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

        def steps(fn, k):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            tot = 0.0
            for _ in range(k):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                b.synchronize()
                tot += a.elapsed_time(b)
            return tot / k

        res = {}
        if args.only_large:
            w5 = workloads.config5()
            u5, v5, s5 = workloads.queries_to_device(w5)
            out5 = torch.empty((w5.n, 9), dtype=torch.float16, device="cuda")
            for prec in ("fp16", "fp8"):
                m5 = workloads.upload(w5, prec)
                m5.set_decode_variant(HEADLINE_VARIANT)
                m5.set_mlp_engine(LARGE_ENGINE)
                res[f"large_{prec}_ms"] = steps(lambda: m5.decode(u5, v5, s5, out=out5), args.steps)
                del m5
        else:
            sw = workloads.config4()
            set_mats = [workloads.upload(m, "fp16") for m in sw.materials]
            for m in set_mats:
                m.set_decode_variant(HEADLINE_VARIANT)
                m.set_mlp_engine(HEADLINE_ENGINE)
            su, sv, ss = (torch.from_numpy(a).cuda() for a in sw.concat())
            soff = torch.from_numpy(sw.offsets).cuda()
            sout = torch.empty((sw.n, 9), dtype=torch.float16, device="cuda")
            S = bcf.MaterialSet(set_mats)
            S.decode(soff, su, sv, ss, out=sout)
            torch.cuda.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                S.decode(soff, su, sv, ss, out=sout)
            res["batched_ms"] = steps(graph.replay, args.steps)
            res["set_config"] = S.config()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "unit": "ms", "n_gpus": world, "steps": args.steps,
                              "warmup": args.warmup, **res, "note": "capture mode: one workload only"}))
        return

    if args.only_train:
        ms, loss, batch = _train_bench(torch, workloads, stream, args.steps, args.train_shape)
        if rank == 0:
            print(json.dumps({"metric": "train steps/s", "value": 1000.0 / ms, "unit": "steps/s", "n_gpus": world,
                              "steps": args.steps, "warmup": 3, "ms_per_step": ms, "batch": batch,
                              "last_loss": loss, "shape": args.train_shape, "note": "training step only"}))
        return

    w = workloads.config2()
    u, v, s = workloads.queries_to_device(w)
    mats = {p: workloads.upload(w, p) for p in (HEADLINE_PRECISION, "fp32", "fp8")}
    for p in (HEADLINE_PRECISION, "fp8"):
        mats[p].set_decode_variant(HEADLINE_VARIANT)
        mats[p].set_mlp_engine(HEADLINE_ENGINE if p == HEADLINE_PRECISION else FP8_ENGINE)
    out = torch.empty((w.n, 9), dtype=torch.float16, device="cuda")
    out32 = torch.empty((w.n, 9), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 126 MB L2
    stream = torch.cuda.current_stream()

    def timed(mat, steps, warmup, out=out):
        for _ in range(warmup):
            mat.decode(u, v, s, out=out)
        torch.cuda.synchronize()
        replicas.barrier()
        total = 0.0
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mat.decode(u, v, s, out=out)
            b.record(stream)
            b.synchronize()
            total += a.elapsed_time(b)
        torch.cuda.synchronize()
        replicas.barrier()
        return total

    if args.only_fp8:
        fp8_only_ms = timed(mats["fp8"], args.steps, args.warmup) / args.steps
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": w.n / (fp8_only_ms * 1e-3) / 1e9, "unit": "Gsamples/s",
                              "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": fp8_only_ms, "mlp_engine": FP8_ENGINE,
                              "note": "capture mode: the headline frame in E4M3 only"}))
        return

    # headline: low-precision path.  Its K steps last milliseconds, shorter than the sampler's 100 ms interval,
    # so the same decode runs back to back for 0.5 s first and the sampling window spans that load, the
    # warm-up and the timed steps, closing with a sample taken after them.
    with ClockSampler(local) as clk:
        clk.wait_samples(1)
        first = len(clk.lines)
        t_load = time.time() + 0.5
        while time.time() < t_load:
            for _ in range(20):
                mats[HEADLINE_PRECISION].decode(u, v, s, out=out)
            torch.cuda.synchronize()
        head_ms = timed(mats[HEADLINE_PRECISION], args.steps, args.warmup)
        clk.wait_samples(len(clk.lines) + 1, timeout=1.0)
    clocks = clk.summary(first)
    clocks["window"] = "0.5 s of back-to-back headline decodes, then the warm-up and the timed steps"
    # whole-job throughput: the queries of all replicas over the slowest rank's time
    head_units, head_ms_max = replicas.aggregate(w.n * args.steps, head_ms, device="cuda")
    value = head_units / (head_ms_max * 1e-3) / 1e9

    if args.only_headline:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "Gsamples/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": head_ms_max / args.steps,
                              "clocks": clocks, "note": "headline decode only"}))
        return

    # the plain FP32 path and FP8 on the same frame
    k_extra = max(3, args.steps // 4)
    fp32_ms = timed(mats["fp32"], k_extra, 3, out=out32) / k_extra
    # the FP32 MLP on the texture unit's texels (variant 3): the same precision gap with the same texel path
    m32t = workloads.upload(w, "fp32")
    m32t.set_decode_variant(TEXUNIT_VARIANT)
    fp32t_ms = timed(m32t, k_extra, 3, out=out32) / k_extra
    del m32t
    fp8_ms = timed(mats["fp8"], k_extra, 3) / k_extra
    # the same decode with the other MLP engine (the texel path bit for bit the same)
    mats[HEADLINE_PRECISION].set_mlp_engine(OTHER_ENGINE[HEADLINE_ENGINE])
    other_engine_ms = timed(mats[HEADLINE_PRECISION], k_extra, 3) / k_extra
    mats[HEADLINE_PRECISION].set_mlp_engine(HEADLINE_ENGINE)
    mats["fp8"].set_mlp_engine(OTHER_ENGINE[FP8_ENGINE])
    fp8_other_ms = timed(mats["fp8"], k_extra, 3) / k_extra
    mats["fp8"].set_mlp_engine(FP8_ENGINE)

    # the texture-unit comparator (decode variant 2: hardware trilinear filtering of BC6H texture objects)
    m_hw = workloads.upload(w, HEADLINE_PRECISION)
    m_hw.set_decode_variant(2)
    hw_out = torch.empty_like(out)
    hw_ms = timed(m_hw, k_extra, 3, out=hw_out) / k_extra
    mats[HEADLINE_PRECISION].decode(u, v, s, out=out)
    hw_err = (hw_out.float() - out.float()).abs()
    hw_stats = {"mean_abs_vs_exact": float(hw_err.mean()), "max_abs_vs_exact": float(hw_err.max())}
    del hw_out, hw_err
    # the texture unit's BC6H decoder for the footprint texels (variant 3, the paper's render-time design), the
    # exact filter: with the warp-level MMA engine (its fastest form; outputs equal to the headline's bit for bit)
    # and with the tcgen05 engine
    m_hw.set_decode_variant(TEXUNIT_VARIANT)
    m_hw.set_mlp_engine("mma_sync")
    tex_ms = timed(m_hw, k_extra, 3) / k_extra
    m_hw.set_mlp_engine("tcgen05")
    tex_tc_ms = timed(m_hw, k_extra, 3) / k_extra
    m_hw.set_mlp_engine(HEADLINE_ENGINE)
    sw_out = torch.empty_like(out)
    m_hw.decode(u, v, s, out=sw_out)
    mats[HEADLINE_PRECISION].decode(u, v, s, out=out)
    tex_identical = bool(torch.equal(out, sw_out))
    del sw_out
    # the same frame on the trained features' own format: every block in BC6H mode 10 (the two-region 6-bit mode
    # of Sec. 4.2); the same seeds give the same queries and weights
    w10 = workloads.screen_material(2, 4, 2048, [13, 32, 32, 9], 3840, 2160, modes=(10,))
    assert np.array_equal(w10.u, w.u) and np.array_equal(w10.s, w.s)
    m10 = workloads.upload(w10, HEADLINE_PRECISION)
    m10.set_decode_variant(HEADLINE_VARIANT)
    m10.set_mlp_engine(HEADLINE_ENGINE)
    mode10_ms = timed(m10, k_extra, 3) / k_extra
    m10.set_mlp_engine(OTHER_ENGINE[HEADLINE_ENGINE])
    mode10_other_ms = timed(m10, k_extra, 3) / k_extra
    del m10, w10

    # the texel-fetch roofline of the headline: the texture unit's point-fetch rate on the same material's
    # level-0 texels in screen-coherent order (bcf_texunit_fetch_probe), against the fetches one headline launch
    # issues -- 4 per texture and sampled level, one level where the LOD is integral or the last one
    probe_rounds = 8
    sink = torch.empty(w.n, dtype=torch.float32, device="cuda")
    for _ in range(3):
        m_hw.texunit_fetch_probe(w.n, probe_rounds, sink=sink)
    torch.cuda.synchronize()
    pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pa.record(stream)
    for _ in range(5):
        m_hw.texunit_fetch_probe(w.n, probe_rounds, sink=sink)
    pb.record(stream)
    pb.synchronize()
    probe_rate = 5 * 4 * probe_rounds * w.n / (pa.elapsed_time(pb) * 1e-3)
    del sink, m_hw
    head_fetches = 0
    s_clean = np.where(np.isnan(w.s), np.float32(0.0), w.s).astype(np.float32)
    for res_t, lev_t in zip(w.res, w.levels):
        bias = np.float32(int(round(np.log2(res_t))) - int(round(np.log2(w.res_ref))))
        st = np.clip(s_clean + bias, np.float32(0.0), np.float32(lev_t - 1))
        fl = np.floor(st)
        head_fetches += int(4 * np.where((st - fl > 0) & (fl + 1 < lev_t), 2, 1).sum())

    def gathered(prec):
        """Outputs of one untimed decode of `prec` (in the timed path's output type) at query indices."""
        o = torch.empty_like(out32 if prec == "fp32" else out)
        mats[prec].decode(u, v, s, out=o)
        return lambda idx: o[torch.from_numpy(idx).cuda()].float().cpu().numpy()

    # small: 2x 256^2 random all-mode textures, 65,536 uniform queries, bilinear at level 0, MLP 6-16-16-8 FP32
    w1 = workloads.config1()
    m1 = workloads.upload(w1, "fp32")
    u1, v1, _ = workloads.queries_to_device(w1)
    o1 = torch.empty((w1.n, 8), dtype=torch.float32, device="cuda")

    def launch_us():
        for _ in range(5):
            m1.decode(u1, v1, None, out=o1)
        torch.cuda.synchronize()
        a1, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a1.record(stream)
        for _ in range(100):
            m1.decode(u1, v1, None, out=o1)
        b1.record(stream)
        b1.synchronize()
        return a1.elapsed_time(b1) * 10.0

    small_sw_us = launch_us()  # the library's per-lane BC6H decoder (random blocks of all 14 modes)
    m1.set_decode_variant(TEXUNIT_VARIANT)  # the texture unit's texels, the same FP32 filter and MLP
    small_us = launch_us()
    del m1, u1, v1, o1

    # end to end through the C ABI with host buffers: bcf_decode_material_host uploads the pinned queries,
    # decodes and downloads the channels chunk by chunk with the three overlapping (128 MB device scratch)
    uh, vh, sh = (torch.from_numpy(a).pin_memory() for a in (w.u, w.v, w.s))
    oh = torch.empty((w.n, 9), dtype=torch.float16).pin_memory()
    scratch = torch.empty(128 << 20, dtype=torch.uint8, device="cuda")
    m = mats[HEADLINE_PRECISION]
    e2e_total = 0.0
    for i in range(3 + k_extra):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m.decode_host(uh, vh, sh, oh, scratch)
        b.record(stream)
        b.synchronize()
        if i >= 3:
            e2e_total += a.elapsed_time(b)
    e2e_value = w.n * world * k_extra / (e2e_total * 1e-3) / 1e9
    # the same copies without overlap (upload, decode, download in sequence), for reference
    ud, vd, sd = torch.empty_like(u), torch.empty_like(v), torch.empty_like(s)
    seq_total = 0.0
    for i in range(3 + k_extra):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ud.copy_(uh, non_blocking=True)
        vd.copy_(vh, non_blocking=True)
        sd.copy_(sh, non_blocking=True)
        m.decode(ud, vd, sd, out=out)
        oh.copy_(out, non_blocking=True)
        b.record(stream)
        b.synchronize()
        if i >= 3:
            seq_total += a.elapsed_time(b)
    e2e_sequential = w.n * world * k_extra / (seq_total * 1e-3) / 1e9
    # the PCIe floor of the same bytes: all uploads and the download concurrently on two streams, no decode
    s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream()
    floor_total = 0.0
    for i in range(3 + k_extra):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s_up.wait_stream(stream)
        s_down.wait_stream(stream)
        with torch.cuda.stream(s_up):
            ud.copy_(uh, non_blocking=True)
            vd.copy_(vh, non_blocking=True)
            sd.copy_(sh, non_blocking=True)
        with torch.cuda.stream(s_down):
            oh.copy_(out, non_blocking=True)
        stream.wait_stream(s_up)
        stream.wait_stream(s_down)
        b.record(stream)
        b.synchronize()
        if i >= 3:
            floor_total += a.elapsed_time(b)
    e2e_copy_floor = w.n * world * k_extra / (floor_total * 1e-3) / 1e9
    del scratch, ud, vd, sd

    train_ms, train_loss, train_batch = _train_bench(torch, workloads, stream, max(3, args.steps // 2))
    ptrain_ms, _, _ = _train_bench(torch, workloads, stream, max(3, args.steps // 4), "paper")
    gtrain_ms, _, _ = _train_bench(torch, workloads, stream, max(3, args.steps // 4), "grid")
    # FP32 atomic-add rate of this GPU for scattered updates into a buffer of the trainer's size (torch
    # index_add_, one atomic per element): the reference for the training scatter's reduction rate
    gbuf = torch.zeros(9_786_368, device="cuda")
    gidx = torch.randint(0, gbuf.numel(), (1 << 24,), device="cuda")
    gval = torch.rand(1 << 24, device="cuda")
    for _ in range(2):
        gbuf.index_add_(0, gidx, gval)
    torch.cuda.synchronize()
    ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ga.record(stream)
    for _ in range(5):
        gbuf.index_add_(0, gidx, gval)
    gb.record(stream)
    gb.synchronize()
    atomic_rate = 5 * (1 << 24) / (ga.elapsed_time(gb) * 1e-3)
    del gbuf, gidx, gval
    # first training stage (unconstrained per-texel features), same sizes and batch
    tw0 = workloads.train_workload()
    tr0 = workloads.upload_free_trainer(tw0, lr_features=5e-2, lr_mlp=1e-3, gamma=0.9995)
    for i in range(3):
        tr0.step(tw0.batch, 7, i)
    torch.cuda.synchronize()
    fa, fb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fa.record(stream)
    k_free = max(3, args.steps // 2)
    for i in range(k_free):
        tr0.step(tw0.batch, 7, 3 + i)
    fb.record(stream)
    fb.synchronize()
    free_ms = fa.elapsed_time(fb) / k_free
    del tr0, tw0

    # partition-selection encoder: 4 textures of 1024^2 with 9 levels (87,381 blocks each), smooth RGB texels
    enc_res, enc_levels = 1024, 9
    n_texels = sum((enc_res >> l) ** 2 for l in range(enc_levels))
    g = torch.Generator(device="cuda").manual_seed(5)
    enc_tex = [torch.rand(n_texels * 3, device="cuda", generator=g) for _ in range(4)]
    enc_out = [bcf.encode_mode10(t, enc_res, enc_levels) for t in enc_tex]
    torch.cuda.synchronize()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    for _ in range(3):
        for t, (pp, pk, pe) in zip(enc_tex, enc_out):
            bcf.encode_mode10(t, enc_res, enc_levels, pp, pk, pe)
    eb.record(stream)
    eb.synchronize()
    enc_ms = ea.elapsed_time(eb) / 3
    enc_blocks = 4 * bcf.texture_blocks(enc_res, enc_levels)
    del enc_tex, enc_out

    # batched multi-material decode: 64 materials, one persistent graph-captured launch, autotuned, against the
    # same materials as 64 separate single-material launches (own 16-byte-aligned outputs); the hand-written
    # decode (variant 0, the headline's engine) and the texture unit's texels (variant 3)
    sw = workloads.config4()
    set_mats = [workloads.upload(m, "fp16") for m in sw.materials]
    su, sv, ss = (torch.from_numpy(a).cuda() for a in sw.concat())
    soff = torch.from_numpy(sw.offsets).cuda()
    sout = torch.empty((sw.n, 9), dtype=torch.float16, device="cuda")
    seq_out = [torch.empty((int(sw.offsets[m + 1] - sw.offsets[m]), 9), dtype=torch.float16, device="cuda")
               for m in range(len(set_mats))]
    seq_q = [tuple(t[int(sw.offsets[m]):int(sw.offsets[m + 1])].clone() for t in (su, sv, ss))
             for m in range(len(set_mats))]

    def time_steps(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(k_extra):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot / k_extra

    def set_vs_sequential(variant, engine):
        for m in set_mats:
            m.set_decode_variant(variant)
            m.set_mlp_engine(engine)
        S = bcf.MaterialSet(set_mats)
        cfg = S.autotune(soff, su, sv, ss, sout)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            S.decode(soff, su, sv, ss, out=sout)
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            S.decode(soff, su, sv, ss, out=sout)
        one_ms = time_steps(graph.replay)
        seq = time_steps(lambda: [mat.decode(*seq_q[m], out=seq_out[m]) for m, mat in enumerate(set_mats)])
        graph.replay()
        torch.cuda.synchronize()
        same = all(torch.equal(sout[int(sw.offsets[m]):int(sw.offsets[m + 1])], seq_out[m])
                   for m in range(len(set_mats)))
        del graph, S
        return one_ms, seq, cfg, same

    set_ms, seq_ms, set_cfg, set_same = set_vs_sequential(HEADLINE_VARIANT, HEADLINE_ENGINE)
    tset_ms, tseq_ms, tex_cfg, tset_same = set_vs_sequential(TEXUNIT_VARIANT, "mma_sync")
    set_n = sw.n
    del set_mats, su, sv, ss, sout, seq_out, seq_q

    # the paper's own decode configuration (Table 1 BCf-1K, decoder 12-16-9) at 3840x2160, FP16, variant 3
    wp = workloads.paper_bcf1k()
    up_, vp_, sp_ = workloads.queries_to_device(wp)
    mp_ = workloads.upload(wp, "fp16")
    outp = torch.empty((wp.n, 9), dtype=torch.float16, device="cuda")
    paper_ms_v = {}
    for var in (TEXUNIT_VARIANT, 0):  # the texture unit's texels, as the paper's shader; the library's decoder
        mp_.set_decode_variant(var)
        for _ in range(3):
            mp_.decode(up_, vp_, sp_, out=outp)
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(k_extra):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mp_.decode(up_, vp_, sp_, out=outp)
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        paper_ms_v[var] = tot / k_extra
    paper_ms = paper_ms_v[TEXUNIT_VARIANT]
    paper_n = wp.n
    del mp_, up_, vp_, sp_, outp, wp

    # large deferred decode: 8 x 4096^2, 7680x4320 queries, MLP 25-64-64-9 (FP8, FP16, FP32)
    w5 = workloads.config5()
    u5, v5, s5 = workloads.queries_to_device(w5)
    out5 = torch.empty((w5.n, 9), dtype=torch.float16, device="cuda")
    cfg5 = {}

    def time5(m5, k5):
        for _ in range(2):
            m5.decode(u5, v5, s5, out=out5)
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(k5):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            m5.decode(u5, v5, s5, out=out5)
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot / k5

    tex5_paths = {}
    for prec in ("fp8", "fp16", "fp32"):
        m5 = workloads.upload(w5, prec)
        if prec != "fp32":
            m5.set_decode_variant(HEADLINE_VARIANT)
            m5.set_mlp_engine(LARGE_ENGINE)
        ms5 = time5(m5, 3 if prec != "fp32" else 2)
        cfg5[prec] = {"value": w5.n / (ms5 * 1e-3) / 1e9, "unit": "Gsamples/s", "ms_per_step": ms5}
        if prec != "fp32":
            # the texture unit's texels (variant 3) with either MLP engine
            m5.set_decode_variant(TEXUNIT_VARIANT)
            for eng in ("mma_sync", "tcgen05"):
                m5.set_mlp_engine(eng)
                ms5 = time5(m5, 3)
                tex5_paths[f"{prec}_{eng}"] = {"value": w5.n / (ms5 * 1e-3) / 1e9, "unit": "Gsamples/s",
                                               "ms_per_step": ms5}
        del m5
    n5 = w5.n
    del u5, v5, s5, out5, w5

    hbm_peak, bf16_peak, peak_kind = _peaks()
    fp8_peak = _fp8_tflops(torch)
    sm_clock_ghz = (clocks.get("sm_max_mhz") or 2032.0) / 1e3
    fp32_simt_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_clock_ghz / 1e3  # TFLOP/s, one FMA per lane per clock
    issue_peak = SM_COUNT * SMSP_PER_SM * sm_clock_ghz  # G warp-instructions/s, one issue per partition per clock
    tex_bytes = sum(int(b.size) for b in w.blocks)
    alg_bytes = w.n * (12 + 18) + tex_bytes  # queries in, FP16 channels out, the texture set once
    head_launch_s = head_ms / args.steps * 1e-3
    achieved = alg_bytes / head_launch_s / 1e9
    counters_valid = _kernel_sha() == NCU_CAPTURE["source_sha256"] and HEADLINE_PRECISION == "fp16"
    counters_valid = counters_valid and HEADLINE_VARIANT == 0 and HEADLINE_ENGINE == NCU_CAPTURE["engine"]
    tex_launch_s = tex_ms * 1e-3
    mlp_flops = 2 * sum(a * b for a, b in zip(w.dims[:-1], w.dims[1:]))  # 3,456 per query for 13-32-32-9

    # large frame: tensor roofline of the MLP (25-64-64-9, 12,544 flop/query) and HBM bytes per path
    flops5 = 2 * (25 * 64 + 64 * 64 + 64 * 9)
    tex5 = 8 * 22369616  # 8 x 4096^2 with full mips, 16 B per 4x4 block
    for prec, peak_tf in (("fp8", fp8_peak), ("fp16", bf16_peak), ("fp32", fp32_simt_peak)):
        t5 = cfg5[prec]["ms_per_step"] * 1e-3
        tf = flops5 * n5 / t5 / 1e12
        cfg5[prec]["tensor" if prec != "fp32" else "fp32_simt"] = {
            "achieved_tflops": tf, "peak_tflops": peak_tf, "frac": (tf / peak_tf) if peak_tf else None}
        cfg5[prec]["hbm_frac"] = (n5 * (12 + 18) + tex5) / t5 / 1e9 / hbm_peak

    if rank == 0:
        cpu, acc = None, None
        if not args.no_cpu_baseline and world == 1:
            mats["bf16"] = workloads.upload(w, "bf16")
            mats["bf16"].set_decode_variant(HEADLINE_VARIANT)
            mats["bf16"].set_mlp_engine(HEADLINE_ENGINE)  # the 16-bit path's engine
            cpu, acc = _cpu_baseline(w, HEADLINE_PRECISION,
                                     {p: gathered(p) for p in ("fp16", "bf16", "fp8", "fp32")})
        line = {
            "metric": METRIC, "value": value, "unit": "Gsamples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": HEADLINE_PRECISION, "data": "synthetic",
            "config": {"workload": "screen decode: 4x BC6H 2048^2 full mips (value-bounded, all 14 modes), "
                                   "3840x2160 perspective-plane queries, MLP 13-32-32-9",
                       "queries_per_step": w.n, "precision": HEADLINE_PRECISION, "out": "fp16 [N][9]",
                       "decode_variant": "0: the library's BC6H decoder (16-byte block loads, mode-sorted blocks "
                                         "decoded into a shared-memory texel arena per 512-query tile), exact "
                                         "FP32 trilinear filter",
                       "mlp_engine": {"mma_sync": "mma.sync per warp (m16n8k16, register-chained layers, FP32 "
                                                  "accumulators in registers)",
                                      "tcgen05": "tcgen05: 128-row MMAs from shared-memory tiles, FP32 accumulators "
                                                 "in tensor memory"}[HEADLINE_ENGINE],
                       "l2": "256 MB buffer written between timed steps",
                       "parallelism": f"replicas x{world}"},
            "fp32_plain": {"value": w.n / (fp32_ms * 1e-3) / 1e9, "unit": "Gsamples/s", "ms_per_step": fp32_ms,
                           "out": "fp32 [N][9]", "kernel": "k_decode_fp32 (plain FP32 SIMT, per-lane)",
                           "fp32_simt": {"achieved_tflops": mlp_flops * w.n / (fp32_ms * 1e-3) / 1e12,
                                         "peak_tflops": fp32_simt_peak, "peak_kind": "derived: 148 SMs x 128 "
                                         "lanes x 2 flop x max SM clock"}},
            "fp8": {"value": w.n / (fp8_ms * 1e-3) / 1e9, "unit": "Gsamples/s", "ms_per_step": fp8_ms,
                    "mlp_engine": FP8_ENGINE,
                    "other_mlp_engine": {"engine": OTHER_ENGINE[FP8_ENGINE], "ms_per_step": fp8_other_ms,
                                         "value": w.n / (fp8_other_ms * 1e-3) / 1e9, "unit": "Gsamples/s"}},
            "fp32_texunit_texels": {"value": w.n / (fp32t_ms * 1e-3) / 1e9, "unit": "Gsamples/s",
                                    "ms_per_step": fp32t_ms, "out": "fp32 [N][9]",
                                    "kernel": "k_decode_fp32 on decode variant 3 (texture-unit texels, exact filter, "
                                              "FP32 SIMT MLP)"},
            "speedup_vs_fp32_plain": fp32_ms / (head_ms / args.steps),
            "speedup_vs_fp32_same_texels": fp32t_ms / (head_ms / args.steps),
            "batched": {"value": set_n / (set_ms * 1e-3) / 1e9, "unit": "Gsamples/s", "ms_per_step": set_ms,
                        "queries": set_n, "materials": 64, "precision": "fp16",
                        "launch": "one persistent launch replayed from a CUDA graph",
                        "decode_variant": HEADLINE_VARIANT, "mlp_engine": HEADLINE_ENGINE,
                        "kernel": "the single-geometry tile kernel over the set's work list (512-query tiles "
                                  "never straddling materials, grabbed from a device counter; a material's "
                                  "description and weights reloaded on change)",
                        "autotuned": {"ctas_per_sm": set_cfg[1], "tiles_per_grab": set_cfg[2]},
                        "identical_to_sequential": set_same,
                        "sequential_64_launches": {"value": set_n / (seq_ms * 1e-3) / 1e9, "unit": "Gsamples/s",
                                                   "ms_per_step": seq_ms},
                        "speedup_vs_sequential": seq_ms / set_ms,
                        "texture_unit_texels": {"value": set_n / (tset_ms * 1e-3) / 1e9, "unit": "Gsamples/s",
                                                "ms_per_step": tset_ms, "decode_variant": TEXUNIT_VARIANT,
                                                "autotuned": {"ctas_per_sm": tex_cfg[1],
                                                              "tiles_per_grab": tex_cfg[2]},
                                                "identical_to_sequential": tset_same,
                                                "sequential_64_launches": {
                                                    "value": set_n / (tseq_ms * 1e-3) / 1e9, "unit": "Gsamples/s",
                                                    "ms_per_step": tseq_ms}}},
            "paper_bcf1k_2160p": {"value": paper_n / (paper_ms * 1e-3) / 1e9, "unit": "Gsamples/s",
                                  "ms_per_step": paper_ms, "queries": paper_n,
                                  "workload": "BC6H 1024/512/256/128 with 9/8/7/6 levels, MLP 12-16-9, FP16, "
                                              "variant 3 (texture-unit texels), 3840x2160 plane queries",
                                  "software_decode": {"value": paper_n / (paper_ms_v[0] * 1e-3) / 1e9,
                                                      "unit": "Gsamples/s", "ms_per_step": paper_ms_v[0]},
                                  "context": "the paper's neural overhead at 2160p: 0.640 ms on an RTX 2070 "
                                             "(hardware trilinear, graphics pipeline)"},
            "large_8x4096": {"queries": n5, "mlp": "25-64-64-9", "flop_per_query": flops5,
                             "paths": "fp8 / fp16: the headline path (variant 0, tcgen05); fp32: the plain SIMT path",
                             **cfg5, "texture_unit_texels": tex5_paths},
            "small_2x256": {"queries": 65536, "mlp": "6-16-16-8 fp32", "us_per_launch": small_us,
                            "value": 65536 / (small_us * 1e-6) / 1e9, "unit": "Gsamples/s",
                            "decode_variant": TEXUNIT_VARIANT,
                            "software_decode_us_per_launch": small_sw_us,
                            "note": "launch-latency bound: 100 back-to-back launches, no flush"},
            "train": {"metric": "train steps/s", "value": 1000.0 / train_ms, "unit": "steps/s",
                      "ms_per_step": train_ms, "batch": train_batch,
                      "samples_per_s": train_batch * 1000.0 / train_ms,
                      "workload": "4x block-parameterised 1024^2 (9 levels), 2048^2 9-ch reference, "
                                  "MLP 13-32-32-9 BF16 operands, Adam", "last_loss": train_loss,
                      "atomic_microbenchmark": {"value": atomic_rate, "unit": "FP32 atomic adds/s",
                                                "workload": "torch index_add_ of 2^24 random updates into "
                                                            "9.79 M floats"},
                      "adam_algorithmic_bytes_per_step": 313_000_000},
            "other_mlp_engine": {"engine": OTHER_ENGINE[HEADLINE_ENGINE],
                                 "value": w.n / (other_engine_ms * 1e-3) / 1e9, "unit": "Gsamples/s",
                                 "ms_per_step": other_engine_ms, "precision": HEADLINE_PRECISION,
                                 "kernel": "the headline decode with the MLP on the other tensor-core engine "
                                           "(tcgen05: 128-row MMAs per 128-query part of the tile, FP32 "
                                           "accumulators in tensor memory; mma.sync: per warp, register-chained)"},
            "texture_unit_texels": {
                "value": w.n / (tex_ms * 1e-3) / 1e9, "unit": "Gsamples/s", "ms_per_step": tex_ms,
                "precision": HEADLINE_PRECISION,
                "kernel": "decode variant 3: every footprint texel fetched through the texture unit's BC6H decoder "
                          "(point sampling, bit-exact), the same exact filter, warp-level MMA MLP (the paper's "
                          "render-time design for the unpack)",
                "identical_to_headline": tex_identical,
                "tcgen05_engine": {"value": w.n / (tex_tc_ms * 1e-3) / 1e9, "unit": "Gsamples/s",
                                   "ms_per_step": tex_tc_ms},
                "roofline": {"bound": "hbm", "achieved": alg_bytes / tex_launch_s / 1e9, "peak": hbm_peak,
                             "unit": "GB/s", "frac": alg_bytes / tex_launch_s / 1e9 / hbm_peak,
                             "peak_kind": peak_kind},
                "texel_fetch": {"unit": "texel fetches/s", "achieved": head_fetches / tex_launch_s,
                                "peak": probe_rate, "frac": head_fetches / tex_launch_s / probe_rate,
                                "fetches_per_launch": head_fetches,
                                "peak_source": "bcf_texunit_fetch_probe: 2x2 point-fetch footprints of the same "
                                               "material's level-0 texels, screen-coherent, measured in this run"}},
            "bcf_mode10_features": {
                "value": w.n / (mode10_ms * 1e-3) / 1e9, "unit": "Gsamples/s", "ms_per_step": mode10_ms,
                "precision": HEADLINE_PRECISION, "decode_variant": HEADLINE_VARIANT, "mlp_engine": HEADLINE_ENGINE,
                "workload": "the headline frame and network with every block in BC6H mode 10 (value-bounded), "
                            "the format trained BCf features are stored in",
                "kernel": "the headline kernel (one mode: every sorted warp decodes one mode's header)",
                "other_mlp_engine": {"engine": OTHER_ENGINE[HEADLINE_ENGINE], "ms_per_step": mode10_other_ms,
                                     "value": w.n / (mode10_other_ms * 1e-3) / 1e9, "unit": "Gsamples/s"}},
            "texunit": {"value": w.n / (hw_ms * 1e-3) / 1e9, "unit": "Gsamples/s", "ms_per_step": hw_ms,
                        "precision": HEADLINE_PRECISION, "kernel": "decode variant 2: hardware trilinear filtering of "
                        "mipmapped BC6H texture objects + tensor-core MLP (per-lane)", **hw_stats},
            "train_grid_batches": {"metric": "train steps/s", "value": 1000.0 / gtrain_ms, "unit": "steps/s",
                                   "ms_per_step": gtrain_ms, "batch": train_batch,
                                   "workload": "the training workload with the paper's batch form: a jittered "
                                               "1024 x 1024 uv grid and one scale per step"},
            "train_paper_decoder": {"metric": "train steps/s", "value": 1000.0 / ptrain_ms, "unit": "steps/s",
                                    "ms_per_step": ptrain_ms, "batch": train_batch,
                                    "workload": "the paper's BCf-1K textures (1024/512/256/128 with mips), 2048^2 "
                                                "reference, its 12-16-9 decoder without the LOD input "
                                                "(tensor-core kernel), Adam"},
            "train_unconstrained": {"metric": "train steps/s", "value": 1000.0 / free_ms, "unit": "steps/s",
                                    "ms_per_step": free_ms, "batch": train_batch,
                                    "workload": "first stage: free per-texel features, 4x 1024^2 with 9 levels"},
            "encode": {"metric": "blocks/s", "value": enc_blocks / (enc_ms * 1e-3), "ms": enc_ms,
                       "blocks": enc_blocks, "workload": "BC6H mode-10 partition selection (32 partitions per "
                                                         "block), 4x 1024^2 RGB textures with 9 levels, uniform texels"},
            "e2e": {"value": e2e_value, "unit": "Gsamples/s", "h2d_bytes_per_step": 12 * w.n,
                    "d2h_bytes_per_step": 18 * w.n, "api": "bcf_decode_material_host (pinned host queries and "
                    "channels, chunked, copies overlapped with the decode)", "sequential_copies": e2e_sequential,
                    "copy_floor": e2e_copy_floor, "copy_floor_note": "the same bytes copied concurrently "
                    "(uploads and download on two streams) with no decode: the PCIe bound of e2e"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak,
                         "traffic": NCU_CAPTURE["dram_bytes"] if counters_valid else None, "peak_kind": peak_kind,
                         "kernel": f"k_decode_geo<{HEADLINE_PRECISION}, 16-32-32-16, {HEADLINE_ENGINE} MLP>",
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "co_bound": {"bound": "issue", "unit": "G warp-instructions/s",
                                      "achieved": (NCU_CAPTURE["warp_inst"] / head_launch_s / 1e9
                                                   if counters_valid else None),
                                      "peak": issue_peak,
                                      "frac": (NCU_CAPTURE["warp_inst"] / head_launch_s / 1e9 / issue_peak
                                               if counters_valid else None),
                                      "note": "executed (not algorithmic) instructions per launch from ncu; "
                                              "peak = 148 SMs x 4 partitions x 1 issue/clock at the max SM clock: "
                                              "the BC6H unpack, filter and MLP epilogue are instruction-issue "
                                              "work, the bytes they move are few"},
                         "tensor": {"achieved_tflops": mlp_flops * w.n / head_launch_s / 1e12,
                                    "peak_tflops": bf16_peak,
                                    "frac": mlp_flops * w.n / head_launch_s / 1e12 / bf16_peak}},
            "peaks": {"hbm_gbs": hbm_peak, "bf16_tflops": bf16_peak, "kind": peak_kind,
                      "fp8_tflops": fp8_peak, "fp8_kind": "measured here: torch._scaled_mm 8192^3 e4m3, burst",
                      "fp32_simt_tflops": fp32_simt_peak, "fp32_simt_kind": "derived from unit counts and clock"},
            "accuracy": acc,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": args.steps,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
