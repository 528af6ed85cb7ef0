#!/usr/bin/env python
"""Throughput of the DPMM sweep (point-sweeps/s = N * sweeps / second) on GB300.

One step is one sweep of Sec. 4.1 -- parameter draws, label step, sufficient
statistics, splits and merges -- over all N points, with the data resident in HBM.
The default workload is the d=32, N=1e6 Gaussian mixture (20 clusters, Dirichlet(1)
weights, means N(0, 25 I), Wishart(I, d+2) covariances, FP32 data, NIW prior with
kappa0=1, m0=0, nu0=d+3, Psi0=I, alpha=10), synthetic and seeded.  The chain is
burned in (untimed) from K=1 until its cluster count has settled, then W warm-up
and K timed sweeps follow.  L2 is flushed (256 MiB write) between timed steps,
outside the timed events.

--impl reference times the FP64 CPU oracle (the paper's method written as plain
loops) on a bounded sample of the same workload, on all of this host's cores (one
independent oracle chain per core on its own slice of the sample).
Multi-GPU (torchrun): independent replicas, one chain per GPU (weak scaling).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))  # synth.py: the seeded input generators

PREC = {"fp64": 0, "tf32": 1, "bf16": 2, "fp32": 3, "bf16x3": 4}
KERNEL = {"tensor": 0, "cuda_core": 1, "auto": 2}
DTYPE = {"fp64": "f64", "tf32": "tf32", "bf16": "bf16", "fp32": "f32", "bf16x3": "bf16x3"}
METRIC = "point-sweeps/s (N*iters/s) d=32 N=1e6, BF16/TF32-TC vs FP64-plain, one GB300"
# ncu DRAM bytes (read + write) per launch of the label kernel, from one capture of it on a
# smaller case (its summary sits with the other profile summaries), as (bytes per point, bytes
# per cluster): the point part scales with N, the factor part with K.  Must be re-taken (or
# removed) whenever that kernel changes.
TRAFFIC_BYTES = {
    # 2 M points, K = 20: 256.227840 MB read + 8.569088 MB written
    ("labels_tc", "gauss_d32"): ((256.227840e6 + 8.569088e6) / 2e6, 0.0),
    # 262,144 points, K = 56: 143.424256 MB read + written, of which the 56 factor images
    # (69,632 B each, read once from DRAM, then from L2) are the cluster part
    ("labels_x3", "gauss_d128"): ((143.424256e6 - 56 * 69632) / 262144, 69632.0),
    # 1 M points: 406.888161 MB read + written (the log theta image is a few KB)
    ("labels_tc_mult", "multinomial"): (406.888161e6 / 1e6, 0.0),
    # the newsgroups shape itself (11,314 documents, K = 20): 23.561 MB read + written per
    # launch (the count atomics and the table reads that miss L2; the rows are L2-resident)
    ("labels_sparse", "newsgroups"): (0.308975e12 * 76.256e-6 / 11314, 0.0),
}
WORKLOADS = {
    "gauss_d32": dict(K_max=64),
    "gauss_d2": dict(K_max=64),
    "multinomial": dict(K_max=128),
    "gauss_d128": dict(K_max=128),
    "batched": dict(K_max=64),
    "newsgroups": dict(K_max=64),
}
# arithmetic of each workload when --prec is not given
DEFAULT_PREC = {"gauss_d32": "tf32", "gauss_d2": "fp64", "multinomial": "bf16", "gauss_d128": "bf16x3",
                "batched": "mixed", "newsgroups": "fp32"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gauss_d32", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default=None, choices=sorted(PREC), help="default: the workload's own (see DEFAULT_PREC)")
    ap.add_argument("--burnin", type=int, default=150)
    ap.add_argument("--n", type=int, default=None, help="override N (smaller cases for profiling)")
    ap.add_argument("--problems", type=int, default=512, help="batched workload: number of problems")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-plain arm on the same state")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--breakdown", action="store_true", help="add a per-kernel time table from a separate profiled pass")
    ap.add_argument("--kernel", default=None, choices=["tensor", "cuda_core", "auto"],
                    help="label-step kernel (dpmm_set_kernel); default: auto for the batched workload, else tensor")
    ap.add_argument("--init-truth", action="store_true",
                    help="start the chain from the generating labels instead of a burn-in from K=1 (profiling runs)")
    return ap.parse_args()


class Clocks:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        time.sleep(0.3)
        if self.p:
            self.p.terminate()
            self.p.wait()

    def summary(self):
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if len(r) > 5 + j and r[5 + j].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def load_workload(name, n, seed_offset):
    """(X, y, prior, options); for the compressed-row workload X is (indptr, indices, counts, d)."""
    import synth

    if name == "newsgroups":
        ip, ix, ct, y = synth.newsgroups_like(seed=1006 + seed_offset, **({} if n is None else {"N": n}))
        d = 20_000
        return (ip, ix, ct, d), y, dict(kind=1, beta=np.ones(d)), dict(alpha=10.0)
    base = {"gauss_d2": 1001, "gauss_d32": 1002, "multinomial": 1003, "gauss_d128": 1004}[name]
    X, y, prior, opt = synth.workload(name, N=n, seed=base + seed_offset)
    return X, y, prior, opt


def dense_rows(X, n):
    """The first n points as a dense FP64 array (the oracle's input)."""
    if isinstance(X, tuple):
        import synth

        ip, ix, ct, d = X
        return synth.csr_to_dense(ip[: n + 1], ix[: ip[n]], ct[: ip[n]], d, dtype=np.float64)
    return X[:n].astype(np.float64)


def n_points(X):
    return X[0].size - 1 if isinstance(X, tuple) else X.shape[0]


def n_dims(X):
    return X[3] if isinstance(X, tuple) else X.shape[1]


def oracle_rate(name, X, y, prior, opt, budget_s=12.0, max_sweeps=4):
    """The FP64 oracle on a bounded sample: its own chain from the generating labels."""
    import oracle as O

    kind = O.NIW if prior["kind"] == 0 else O.DIRICHLET
    kw = {k: v for k, v in prior.items() if k != "kind"}
    K = int(y.max()) + 1
    N = n_points(X)
    o = O.Oracle(kind, n_dims(X), max(64, K), opt["alpha"], burn_out=15, **kw)
    # size the sample from a probe so the whole measurement stays ~budget_s
    n0 = min(N, 2000)
    o.set_data(dense_rows(X, n0))
    o.set_state(K, y[:n0] % K, (np.arange(n0) % 2).astype(np.uint8))
    t0 = time.perf_counter()
    o.sweep(1, 1)
    per_pt = (time.perf_counter() - t0) / n0
    n = int(min(N, max(n0, budget_s / max_sweeps / max(per_pt, 1e-9))))
    o.set_data(dense_rows(X, n))
    o.set_state(K, y[:n] % K, (np.arange(n) % 2).astype(np.uint8))
    sweeps = 0
    t0 = time.perf_counter()
    while sweeps < max_sweeps and (time.perf_counter() - t0) < budget_s:
        o.sweep(1, 1)
        sweeps += 1
    el = time.perf_counter() - t0
    return n * sweeps / el, dict(n=n, sweeps=sweeps, K=K, seconds=el)


def rows_slice(X, a, b):
    """Points [a, b) in the workload's own form (dense rows, or compressed rows rebased)."""
    if isinstance(X, tuple):
        ip, ix, ct, d = X
        return (ip[a: b + 1] - ip[a], ix[ip[a]: ip[b]], ct[ip[a]: ip[b]], d)
    return X[a:b]


def _oracle_chain_worker(job, barrier, out):
    """One oracle chain on its own slice of points (a spawned process): set-up, then the
    timed sweeps once every worker is ready."""
    import oracle as O

    kind, d, kmax, alpha, kw, Xs, ys, sweeps = job
    n = ys.size
    K = int(ys.max()) + 1
    o = O.Oracle(kind, d, kmax, alpha, burn_out=15, **kw)
    o.set_data(dense_rows(Xs, n))
    o.set_state(K, ys % K, (np.arange(n) % 2).astype(np.uint8))
    barrier.wait(timeout=600)
    t0 = time.perf_counter()
    for _ in range(sweeps):
        o.sweep(1, 1)
    out.put((n, sweeps, time.perf_counter() - t0))


def oracle_rate_cores(name, X, y, prior, opt, budget_s=12.0, sweeps=3, cores=None):
    """The FP64 oracle as it stands on every host core: one independent chain per core
    (spawned processes, no threads inside the oracle), each on a contiguous slice of a
    bounded sample and started from the generating labels; the rate is the points swept by
    all chains over the slowest chain's time, the chains starting together."""
    import multiprocessing as mp

    import oracle as O

    cores = cores or len(os.sched_getaffinity(0))
    kind = O.NIW if prior["kind"] == 0 else O.DIRICHLET
    kw = {k: v for k, v in prior.items() if k != "kind"}
    N = n_points(X)
    K = int(y.max()) + 1
    # per-point cost from a one-core probe, then a sample of about budget_s per chain
    n0 = min(N, 1000)
    o = O.Oracle(kind, n_dims(X), max(64, K), opt["alpha"], burn_out=15, **kw)
    o.set_data(dense_rows(X, n0))
    o.set_state(K, y[:n0] % K, (np.arange(n0) % 2).astype(np.uint8))
    t0 = time.perf_counter()
    o.sweep(1, 1)
    per_pt = (time.perf_counter() - t0) / n0
    del o
    n = int(min(N, cores * max(64, budget_s / sweeps / max(per_pt, 1e-9))))
    cuts = np.linspace(0, n, cores + 1).astype(np.int64)
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(cores), ctx.Queue()
    procs = []
    for c in range(cores):
        a, b = int(cuts[c]), int(cuts[c + 1])
        job = (kind, n_dims(X), max(64, K), opt["alpha"], kw, rows_slice(X, a, b), y[a:b].copy(), sweeps)
        p = ctx.Process(target=_oracle_chain_worker, args=(job, barrier, out))
        p.start()
        procs.append(p)
    import queue

    res, deadline = [], time.time() + 900
    while len(res) < cores:
        try:
            res.append(out.get(timeout=2))
        except queue.Empty:
            if any(p.exitcode not in (None, 0) for p in procs) or time.time() > deadline:
                for p in procs:
                    p.terminate()
                raise RuntimeError("an oracle chain process failed")
    for p in procs:
        p.join(timeout=60)
    pts = sum(r[0] * r[1] for r in res)
    el = max(r[2] for r in res)
    return pts / el, dict(n=n, sweeps=sweeps, K=K, seconds=el, cores=cores)


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if a.workload == "batched":  # a bounded sample of the first problem
        import synth

        X, y, d = next(synth.batch_problems(a.problems))
        prior = dict(kind=0, kappa0=1.0, m0=np.zeros(d), nu0=float(d + 3), psi0=np.eye(d))
        opt = dict(alpha=10.0)
    else:
        X, y, prior, opt = load_workload(a.workload, a.n, 0)
    N = n_points(X)
    vals = []
    info = None
    steps = max(1, min(a.steps, 3))
    for _ in range(steps):
        v, info = oracle_rate_cores(a.workload, X, y, prior, opt, budget_s=8.0, sweeps=2)
        vals.append(v)
    v = float(np.median(vals))
    sample = ("first %d of the N=%d points split into %d contiguous slices, one independent oracle chain "
              "per host core, %d sweeps per step from the generating labels (K=%d)" % (
                  info["n"], N, info["cores"], info["sweeps"], info["K"]))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "point-sweeps/s", "n_gpus": a.gpus,
           "steps": steps, "warmup": 0, "ms_per_step": 1e3 * N / v, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": a.workload, "N": N, "d": int(n_dims(X)), "sample": sample,
                      "ms_per_step": "extrapolated: N / value, the sample's rate applied to all N points"},
           "cpu_baseline": {"value": v, "unit": "point-sweeps/s", "cores": info["cores"], "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": "point-sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def job_rate(local_ms, n_points, steps, world, dist=None):
    """Whole-job rate over `world` replicas that each swept n_points `steps` times: the
    slowest rank's time (max over ranks through the process group) bounds the job.
    Returns (point-sweeps per second, max milliseconds)."""
    ms = float(local_ms)
    if dist is not None and world > 1:
        import torch

        t = torch.tensor([ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * n_points * steps / (ms / 1e3), ms


def launch_floor(kernels, step_ms, reps=50):
    """Replay time of a captured CUDA graph of `kernels` trivial kernels: the launch floor a
    step of that many kernels cannot go below (what bounds the small, latency-bound
    configurations)."""
    import torch

    if kernels < 1:
        return None
    t = torch.zeros(1, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(3):
            t.add_(1.0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for _ in range(kernels):
            t.add_(1.0)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):
        e0.record(s)
        for _ in range(reps):
            g.replay()
        e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"kernels_per_step": kernels, "empty_graph_replay_ms": ms, "frac_of_step": ms / step_ms}


def batch_prec(d):
    """Precision of a batched problem: FP32 CUDA cores for d <= 8, TF32 tensor cores for
    d <= 32, split BF16 tensor cores above."""
    return "fp32" if d <= 8 else ("tf32" if d <= 32 else "bf16x3")


def main_batched(a):
    """All problems of the batched workload on one GPU: one chain (context) and one stream
    per problem; a step is one sweep of every problem (dpmm_sweep_batch), timed with events
    on a main stream that every problem stream joins."""
    import torch

    import paper_2204_08988_gb300 as P
    import synth
    from paper_2204_08988_gb300 import _build

    _build.build()
    K_max = WORKLOADS["batched"]["K_max"]
    seed = 0
    chains, streams, sizes = [], [], []
    for p, (X, y, d) in enumerate(synth.batch_problems(a.problems)):
        s = torch.cuda.Stream()
        g = P.DPMM(0, d, K_max, 10.0, prec=PREC[batch_prec(d)], init_K=1, burn_out=15, stream=s.cuda_stream,
                   kappa0=1.0, m0=np.zeros(d), nu0=float(d + 3), psi0=np.eye(d))
        g.set_kernel(KERNEL[a.kernel or "auto"])
        g.set_data(X)
        g.set_problem(p)
        if a.init_truth:
            g.set_state(int(y.max()) + 1, y, (np.arange(len(y)) % 2).astype(np.uint8))
        chains.append(g)
        streams.append(s)
        sizes.append((len(y), d))
    handles = [g.h for g in chains]
    N_tot = sum(n for n, _ in sizes)
    burn = 0 if a.init_truth else a.burnin
    P.dpmm_sweep_batch(handles, burn + a.warmup, seed)
    torch.cuda.synchronize()
    main_s = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    step_ms = []
    for g in chains:  # resets each chain's launch count (no per-kernel events)
        P.dpmm_profile(g.h, 0)
    with Clocks(0) as clk:
        for _ in range(a.steps):
            with torch.cuda.stream(main_s):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(main_s)
            for s in streams:
                s.wait_event(e0)
            P.dpmm_sweep_batch(handles, 1, seed)
            for s in streams:
                ev = torch.cuda.Event()
                ev.record(s)
                main_s.wait_event(ev)
            e1.record(main_s)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    total_ms = float(sum(step_ms))
    gpu_launches = sum(P.dpmm_get_profile(g.h).get("all_kernels", (0, 0))[0] for g in chains)
    Ks = [g.K for g in chains]
    value = N_tot * a.steps / (total_ms / 1e3)
    breakdown = None
    if a.breakdown:  # separate pass: events around every kernel of every chain, summed by kernel
        for g in chains:
            P.dpmm_profile(g.h, 1)
        P.dpmm_sweep_batch(handles, a.steps, seed)
        acc = {}
        for g, (n, d) in zip(chains, sizes):
            for k, (cnt, ms) in P.dpmm_get_profile(g.h).items():
                if k == "all_kernels":
                    continue
                key = "%s@d%d" % (k, d)
                acc.setdefault(key, 0.0)
                acc[key] += ms / a.steps
            P.dpmm_profile(g.h, 0)
        breakdown = {k: round(v, 4) for k, v in sorted(acc.items(), key=lambda x: -x[1])}
    # roofline of the batch: each problem's label-step bound max(flops / the peak of its
    # arithmetic, bytes / HBM), summed over problems, against the measured time of a step
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    bf16 = peaks.get("bf16_tflops", 1900.0) * 1e12
    hbm = peaks.get("hbm_gbs", 6800.0) * 1e9
    peak = {"fp32": 152 * 128 * 2 * 2.07e9, "tf32": bf16 * 1.1 / 2.25, "bf16x3": bf16 / 3.0}
    bound_s = 0.0
    for (n, d), K in zip(sizes, Ks):
        flops = 2.0 * n * d * d * K
        bound_s += max(flops / peak[batch_prec(d)], n * (4 * d + 5) / hbm)
    roof = {"bound": "mixed", "achieved": bound_s * 1e3, "peak": total_ms / a.steps, "unit": "ms (label-step bound / step)",
            "frac": bound_s * 1e3 / (total_ms / a.steps), "traffic": None,
            "note": "sum over problems of max(2 N d^2 K / peak of its precision, N (4d + 5) B / HBM); "
                    "bf16x3 counts one third of the BF16 peak (three products)"}
    mix = {}
    for (n, d) in sizes:
        mix.setdefault(d, [0, 0])
        mix[d][0] += 1
        mix[d][1] += n
    out = {"metric": METRIC, "value": value, "unit": "point-sweeps/s", "n_gpus": 1, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "mixed", "data": "synthetic",
           "config": {"workload": "batched", "problems": len(chains), "N_total": N_tot,
                      "mix": {str(d): {"problems": c, "points": n, "prec": batch_prec(d)} for d, (c, n) in
                              sorted(mix.items())},
                      "K_max": K_max, "K_timed_mean": float(np.mean(Ks)), "burnin_sweeps": burn,
                      "init": "generating labels" if a.init_truth else "K=1", "parallelism": "1gpu, one stream per problem",
                      "device_max_connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS"),
                      "label_kernel": {"requested": a.kernel or "auto",
                                       "tensor": sum(g.kernel()[0] == 0 for g in chains),
                                       "cuda_core": sum(g.kernel()[0] == 1 for g in chains)},
                      "l2": "flushed by a 256 MiB write between timed steps (untimed)"},
           "roofline": roof, "cpu_baseline": None, "e2e": None, "clocks": clk.summary(), "gpu_launches": gpu_launches,
           "step_ms": step_ms}
    if breakdown is not None:
        out["breakdown_stream_ms_per_step"] = breakdown
    print(json.dumps(out))
    for g in chains:
        g.close()


def main():
    a = parse()
    if a.prec is None:
        a.prec = DEFAULT_PREC[a.workload]
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "batched":
        # one hardware work queue per stream (up to 32) instead of the default 8, so that
        # the problems' streams do not serialise behind each other; read when the CUDA
        # context is created, which has not happened yet
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
        return main_batched(a)
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    import paper_2204_08988_gb300 as P
    from paper_2204_08988_gb300 import _build

    _build.build()

    X, y, prior, opt = load_workload(a.workload, a.n, rank)
    N, d = n_points(X), n_dims(X)
    kind = prior["kind"]
    csr = isinstance(X, tuple)
    kw = {k: v for k, v in prior.items() if k != "kind"}
    K_max = WORKLOADS[a.workload]["K_max"]
    stream = torch.cuda.Stream()
    g = P.DPMM(kind, d, K_max, opt["alpha"], prec=PREC[a.prec], init_K=1, burn_out=15,
               stream=stream.cuda_stream, **kw)
    g.set_kernel(KERNEL[a.kernel or "tensor"])
    Xd = None
    if csr:
        g.set_data_csr(*X[:3])
    else:
        Xd = torch.from_numpy(X).cuda()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            g.set_data(Xd)
    seed = 0
    if a.init_truth:
        K_true = int(y.max()) + 1
        g.set_state(K_true, y, (np.arange(N) % 2).astype(np.uint8))
        a.burnin = 0
    g.sweep(a.burnin, seed)
    K0 = g.K
    # the timed sweeps are what a user runs: the captured sweep graph, replayed, no
    # events inside it; dpmm_profile(0) only resets the library's launch counter here
    P.dpmm_profile(g.h, 0)
    g.sweep(a.warmup, seed)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_steps(chain, steps, clocks=None):
        Ks_, ev_ = [], [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                        for _ in range(steps)]
        for s in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()  # L2 flush, outside the timed events
                ev_[s][0].record(stream)
            chain.sweep(1, seed)
            with torch.cuda.stream(stream):
                ev_[s][1].record(stream)
            Ks_.append(chain.K)  # synchronises, outside the events
        return [b.elapsed_time(e) for b, e in ev_], Ks_

    P.dpmm_profile(g.h, 0)
    barrier()
    with Clocks(local) as clk:
        step_ms, Ks = timed_steps(g, a.steps)
        barrier()
    total_ms = float(sum(step_ms))
    gpu_launches = P.dpmm_get_profile(g.h).get("all_kernels", (0, 0))[0]
    value, total_ms = job_rate(total_ms, N, a.steps, world, dist)

    # the label kernel's mean launch time, from a separate pass of the same number of sweeps
    # with CUDA events around that kernel only (those sweeps run eagerly, not replayed)
    P.dpmm_profile(g.h, 2)
    timed_steps(g, a.steps)
    prof = P.dpmm_get_profile(g.h)
    P.dpmm_profile(g.h, 0)
    Kavg = float(np.mean(Ks))
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    # "measured": the pool's own figure from MEASURED_PEAKS.json; "fallback": one earlier
    # GB300 measurement (1.9 PFLOP/s BF16 burst, 6.8 TB/s copy), used when that file is absent
    bf16_src = "measured" if "bf16_tflops" in peaks else "fallback"
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"

    # roofline of the dominant kernel: the label step
    lk = [k for k in prof if k.startswith("labels")]
    roof = None
    if lk:
        launches, ms = prof[lk[0]]
        avg_s = ms / max(launches, 1) / 1e3
        if kind == 0:
            flops = 2.0 * N * d * d * Kavg  # X (N x d) times the K stacked d x d factors
            if a.prec in ("tf32", "bf16", "bf16x3"):
                peak = bf16_peak * (1.1 / 2.25) if a.prec == "tf32" else bf16_peak
                roof = {"bound": "tensor", "achieved": flops / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                        "peak_source": (bf16_src + " bf16 burst x nominal tf32/bf16 ratio 1.1/2.25"
                                        if a.prec == "tf32" else bf16_src + " bf16 burst")}
                if a.prec == "bf16x3":
                    # issued: three BF16 products on the padded dimension plus the one-step -b product
                    dp = 64 if d <= 64 else 128
                    roof["issued_tflops"] = 2.0 * N * Kavg * dp * (3 * dp + 16) / avg_s / 1e12
            else:
                # CUDA-core paths: FMA pipe peak from 152 SMs x 128 FP32 lanes x 2 flop at the max SM clock
                peak = 152 * 128 * 2 * 2.07e9 / 1e12 if a.prec == "fp32" else 1.25
                roof = {"bound": "alu", "achieved": flops / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                        "peak_source": "fp32: 152 SMs x 128 lanes x 2 flop x 2.07 GHz" if a.prec == "fp32"
                        else "fp64: nominal 1.25 TFLOP/s"}
        elif csr:
            # compressed rows: 8 B per nonzero (category, count), the row pointer and the labels
            bytes_ = 8 * int(X[0][-1]) + 8 * (N + 1) + 5 * N
            roof = {"bound": "hbm", "achieved": bytes_ / avg_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "peak_source": hbm_src + " copy bandwidth"}
        else:
            bytes_ = N * d * (2 if a.prec == "bf16" else 4) + 4 * N
            roof = {"bound": "hbm", "achieved": bytes_ / avg_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "peak_source": hbm_src + " copy bandwidth"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        # DRAM bytes per launch from the ncu capture summarised in profiles/ (taken on a smaller
        # case, scaled by the points and clusters processed); null without a current capture
        tb = TRAFFIC_BYTES.get((lk[0], a.workload))
        roof["traffic"] = tb[0] * N + tb[1] * Kavg if tb else None
        roof["kernel"] = lk[0]
        roof["kernel_ms_avg"] = ms / max(launches, 1)
        roof["kernel_timing"] = "CUDA events around the kernel on its stream, separate pass of %d sweeps" % a.steps
        # the whole sweep against its own bound: algorithmic work per point per sweep (Gaussian:
        # d^2 (2K + 5) flop -- cluster scores 2 d^2 K, sub-cluster scores 4 d^2, statistics d^2 --
        # and d x 4 + 5 bytes; multinomial: d x 2 + 5 bytes) at the peak of the path's arithmetic
        step_s = total_ms / a.steps / 1e3
        if kind == 0:
            sw_flops = N * d * d * (2.0 * Kavg + 5.0)
            sw_bytes = N * (4.0 * d + 5.0)
            t_bound = max(sw_flops / (roof["peak"] * 1e12) if roof["unit"] == "TFLOP/s" else 0.0,
                          sw_bytes / (hbm_peak * 1e9))
            roof["sweep"] = {"flop": sw_flops, "bytes": sw_bytes, "bound_ms": t_bound * 1e3,
                             "achieved": sw_flops / step_s / 1e12, "unit": "TFLOP/s"}
        else:
            sw_bytes = (8.0 * int(X[0][-1]) + 13.0 * N) if csr else N * (2.0 * d + 5.0)
            t_bound = sw_bytes / (hbm_peak * 1e9)
            roof["sweep"] = {"bytes": sw_bytes, "bound_ms": t_bound * 1e3, "achieved": sw_bytes / step_s / 1e9,
                             "unit": "GB/s"}
        roof["sweep_frac"] = t_bound / step_s
    floor = launch_floor(gpu_launches // max(a.steps, 1), total_ms / a.steps)

    breakdown = None
    if a.breakdown:  # separate pass, events around every kernel (not the timed steps)
        P.dpmm_profile(g.h, 1)
        for s in range(a.steps):
            g.sweep(1, seed)
        bd = P.dpmm_get_profile(g.h)
        P.dpmm_profile(g.h, 0)
        breakdown = {k: {"launches": v[0], "ms_per_step": v[1] / a.steps} for k, v in bd.items() if k != "all_kernels"}

    # the FP64-plain GPU sweep on the same state: a second chain on the same data, in FP64
    # on CUDA cores (the parity path), started from this chain's current labels, so both
    # arms time sweeps at the same number of clusters
    fp64 = None
    est_s = 2.0 * N * d * d * Kavg / 1e12 if kind == 0 else 2.0 * N * d * Kavg / 1e12
    if a.prec != "fp64" and not a.no_fp64 and world == 1 and (est_s < 2.0 or csr):
        z_now, zb_now = g.labels()
        K_now = g.K
        g64 = P.DPMM(kind, d, K_max, opt["alpha"], prec=PREC["fp64"], init_K=1, burn_out=15,
                     stream=stream.cuda_stream, **kw)
        if csr:
            g64.set_data_csr(*X[:3])
        else:
            with torch.cuda.stream(stream):
                g64.set_data(Xd)
        g64.set_state(K_now, z_now, zb_now)
        g64.sweep(2, seed)  # warm-up (the second sweep captures the graph)
        ms64, K64 = timed_steps(g64, a.fp64_steps)
        v64 = N * len(ms64) / (sum(ms64) / 1e3)
        fp64 = {"value": v64, "unit": "point-sweeps/s", "ms_per_step": float(np.mean(ms64)), "steps": len(ms64),
                "K_start": K_now, "K_timed": K64, "speedup": value / v64,
                "note": "FP64-plain GPU sweep from the timed chain's labels (same data, same K), graph replay, "
                        "L2 flushed between steps"}
        g64.close()

    # end to end through the C ABI: pinned host X in, labels out, every step
    e2e = None
    if not a.no_e2e and not csr:
        Xh = torch.from_numpy(X).pin_memory()
        zh = torch.empty(N, dtype=torch.int32).pin_memory()
        zbh = torch.empty(N, dtype=torch.uint8).pin_memory()
        h2d = Xh.numel() * Xh.element_size()
        d2h = N * 5
        g.stage_data(Xh)  # allocates the staging buffer (untimed)
        g.sweep(1, seed)
        P.dpmm_get_labels(g.h, N, zh, zbh)
        barrier()
        # every step: the step's input from page-locked host memory (its copy overlaps the
        # previous step's sweep: dpmm_stage_data), the sweep, and its labels back to the host
        t0 = time.perf_counter()
        g.stage_data(Xh)
        for s in range(a.steps):
            g.sweep(1, seed)
            if s + 1 < a.steps:
                g.stage_data(Xh)
            P.dpmm_get_labels(g.h, N, zh, zbh)
        barrier()
        el = time.perf_counter() - t0
        if dist:
            t = torch.tensor([el])
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": world * N * a.steps / el, "unit": "point-sweeps/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h,
               "pipeline": "dpmm_stage_data: each step's input copy (copy engine) overlaps the previous step's sweep"}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        v1, i1 = oracle_rate(a.workload, X, y, prior, opt)
        v, info = oracle_rate_cores(a.workload, X, y, prior, opt)
        cpu = {"value": v, "unit": "point-sweeps/s", "cores": info["cores"], "kind": "oracle",
               "sample": "first %d of the N=%d points split into %d contiguous slices, one independent FP64 "
                         "oracle chain per host core, %d sweeps from the generating labels (K=%d)" % (
                             info["n"], N, info["cores"], info["sweeps"], info["K"]),
               "single_core": {"value": v1, "cores": 1,
                               "sample": "first %d of the N=%d points, %d sweep(s) from the generating labels, "
                                         "one oracle chain" % (i1["n"], N, i1["sweeps"])}}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "point-sweeps/s", "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": DTYPE[a.prec], "data": "synthetic",
               "config": {"workload": a.workload, "N": N, "d": d, "K_start": K0, "K_timed": Ks, "K_max": K_max,
                          "prec": a.prec, "burnin_sweeps": a.burnin, "init": "generating labels" if a.init_truth else "K=1", "parallelism": "replicas" if world > 1 else "1gpu",
                          "label_kernel": ["tensor", "cuda_core"][g.kernel()[0]],
                          "l2": "flushed by a 256 MiB write between timed steps (untimed)"},
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
               "gpu_launches": gpu_launches, "launch_floor": floor, "fp64_plain": fp64, "step_ms": step_ms,
               "timing": "CUDA events around each replayed sweep graph on the library's stream; no events "
                         "inside the timed sweeps"}
        if breakdown is not None:
            out["breakdown"] = breakdown
        print(json.dumps(out))
    g.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
