"""Benchmark: Lazy SPCA on one GB300 (and N GPUs under torchrun).

Headline workload (one step = one whole Lazy SPCA fit plus the reduction map
of every row, the paper-scale form of the path): e4m3_binary -- X of
4,600,000 x 4,096 binary features in FP8 E4M3 (column rates p_j ~ Beta(0.5,
9.5), 5 % density; Experiment 1's mostly-binary design matrix, synthetic),
k = 256, very sparse Omega with p = 64.  X (18.8 GB) is larger than L2, so no
flush is needed between steps.  The same JSON line carries, as extra keys, the
precision form (bf16_dense, 1,000,000 x 8,192 BF16, Gaussian Omega, k = 256),
the FP32 form (fp32_sparse, 200,000 x 4,096, k = 128) with the SPCA
comparison path and the Gram on and off, the k x k step on flat and steep
spectra, the TF-IDF-shaped sparse fit and the serving run.

With --gpus N > 1 the step is one fit whose rows are sharded over the N ranks
(each rank holds a 4.6 M-row block of its own, so the work per GPU is fixed:
weak scaling): per rank the sketch and pass F, one exchange of the k x n FP64
partials of F over NCCL (gathered and summed in rank order by the library),
the k x k step replicated, the reduction map of the rank's own rows.  Run
without torchrun, --gpus N starts the N ranks itself.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Lazy SPCA fit samples/s & HBM-roofline frac vs SPCA on GB300; serve p50/p99 ms"
WORKLOAD = "e4m3_binary"


def _peaks():
    """Measured HBM copy bandwidth (GB/s) and BF16 dense TFLOP/s (burst,
    sustained), else the documented fallback figures."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm": d.get("hbm_gbs", 6800.0), "bf16": d.get("bf16_tflops", 1900.0),
                "bf16_sustained": d.get("bf16_tflops_sustained", 1700.0), "kind": "measured"}
    return {"hbm": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "kind": "fallback"}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (model name on x86; implementer
    and part numbers on Arm), else the platform's machine string."""
    import platform
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return platform.machine()
    for line in info:
        if line.lower().startswith("model name"):
            return line.split(":", 1)[1].strip()
    fields = {}
    for line in info:
        if ":" in line:
            key, val = (t.strip() for t in line.split(":", 1))
            fields.setdefault(key, val)
    if "CPU part" in fields:
        return f"{platform.machine()} implementer {fields.get('CPU implementer', '?')} part {fields['CPU part']}"
    return platform.machine()


def _oracle_step(O, X, Om):
    """One oracle step of the headline workload: the FP64 fit and the
    reduction map of the same rows."""
    fit = O.lspca_fit(X, Om, route="eig")
    return O.project(X, fit["V"])


def _oracle_sample(rows: int):
    from oracle import philox as P
    from paper_1709_07175_gb300 import synthetic as S
    w = S.WORKLOADS[WORKLOAD].scaled(m=rows)
    X = S.generate(w).float().double().numpy()
    Om = P.omega_sparse(w.omega_seed, w.n, w.k, w.p)
    return w, X, Om


def cpu_baseline(rows: int, reps_seconds: float = 10.0) -> dict:
    """The FP64 oracle as it stands, on a bounded sample of the workload."""
    import numpy as np

    from oracle import lspca as O
    w, X, Om = _oracle_sample(rows)
    t0 = time.perf_counter()
    reps = 0
    while True:
        _oracle_step(O, X, Om)
        reps += 1
        if time.perf_counter() - t0 >= reps_seconds:
            break
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": rows * reps / dt, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": f"{rows} rows x {w.n} of the {WORKLOAD} workload (same recipe), k={w.k}: "
                      f"{reps} oracle fit(s) plus reduction map of the sample in {dt:.1f} s; FP64 numpy, "
                      f"BLAS threads = host default",
            "cpu": cpu_model(), "np": np.__version__}


def serve_bench(L, S, torch, local: int, seconds: float, loads=(0.5, 0.8, 0.95), seed: int = 5) -> dict:
    """Continuous-batching serving run shaped like the serving workload: three
    resident V (n = 4096, k in {64, 128, 256}) fitted from BF16 low-rank data,
    Poisson arrivals of projection requests (log-uniform 1..65,536 BF16 rows)
    mixed 9:1 with fit requests (m log-uniform 1e4..5e5, n = 4096, k = 128,
    Gaussian Omega), offered at each of `loads` times the measured unbatched
    capacity (the same requests and seed at every load).  Latency = completion
    - arrival on the host clock.  The top-level fields are those of load 0.8."""
    import math
    import numpy as np
    dev = torch.device(f"cuda:{local}")
    n = 4096
    from dataclasses import replace
    wsrc = replace(S.WORKLOADS["bf16_dense"].scaled(m=500_000, n=n, k=128), r=64)
    pool = S.generate(wsrc, device=dev)  # 500k x 4096 BF16 (4.1 GB): fit and projection rows
    ctx = L.Context(local)
    fitV = ctx.fit(pool[:20000], 256, L.omega("gaussian", 0), report=False).V
    Vs = {k: fitV[:, :k].contiguous() for k in (64, 128, 256)}
    rng = np.random.default_rng(seed)
    nreq = 600
    kinds = rng.random(nreq) < 0.1
    prow = S.serving_rows(seed, nreq)
    frow = np.floor(np.exp(rng.uniform(math.log(1e4), math.log(5e5), nreq))).astype(np.int64)
    pk = rng.choice([64, 128, 256], nreq)
    poff = rng.integers(0, 500_000 - 65_536, nreq)
    gaps = rng.exponential(1.0, nreq)  # unit-rate Poisson gaps, scaled per load
    om = L.omega("gaussian", 0)

    def direct(i):
        if kinds[i]:
            ctx.fit(pool[: frow[i]], 128, om, report=False)
        else:
            X = pool[poff[i]: poff[i] + prow[i]]
            ctx.project(X, Vs[int(pk[i])])

    # unbatched plain-launch baseline: service time of each request alone
    for i in range(8):
        direct(i)
    torch.cuda.synchronize()
    svc = np.zeros(nreq)
    for i in range(nreq):
        t0 = time.perf_counter()
        direct(i)
        torch.cuda.synchronize()
        svc[i] = time.perf_counter() - t0

    srv = L.Server(local, 24 << 30, 64)
    vid = {k: srv.register_v(V) for k, V in Vs.items()}
    # warm the server's graphs once per group
    for k in (64, 128, 256):
        r, _ = srv.submit_project(vid[k], pool[:300])
        srv.wait(r)
        srv.release(r)
    torch.cuda.synchronize()

    def run_load(load):
        rate = load / svc.mean()
        arrivals = np.cumsum(gaps / rate)
        # baseline latency: one FIFO server with the measured service times
        done_b = np.zeros(nreq)
        tfree = 0.0
        for i in range(nreq):
            start = max(arrivals[i], tfree)
            tfree = start + svc[i]
            done_b[i] = tfree
        lat_b = (done_b - arrivals) * 1e3
        t_start = time.perf_counter()
        deadline = t_start + seconds
        nxt = 0
        live = {}
        lat = []
        rows_done = 0
        while (nxt < nreq or live) and time.perf_counter() < deadline + 30:
            now = time.perf_counter() - t_start
            while nxt < nreq and arrivals[nxt] <= now:
                if kinds[nxt]:
                    req, V, sig = srv.submit_fit(pool[: frow[nxt]], 128, om)
                    rows = int(frow[nxt])
                else:
                    req, Y = srv.submit_project(vid[int(pk[nxt])], pool[poff[nxt]: poff[nxt] + prow[nxt]])
                    rows = int(prow[nxt])
                live[req] = (arrivals[nxt], rows)
                nxt += 1
            srv.step()
            for req in list(live):
                if srv.done(req):
                    arr, rows = live.pop(req)
                    lat.append((time.perf_counter() - t_start - arr) * 1e3)
                    rows_done += rows
                    srv.release(req)
            if not live and nxt < nreq:
                time.sleep(max(0.0, min(1e-3, arrivals[nxt] - (time.perf_counter() - t_start))))
        wall = time.perf_counter() - t_start
        torch.cuda.synchronize()
        lat = np.array(lat)
        return {"load": load, "requests": int(len(lat)), "mix": "9:1 projections:fits",
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "throughput_req_s": len(lat) / wall, "rows_per_s": rows_done / wall,
                "unbatched": {"p50_ms": float(np.percentile(lat_b, 50)), "p99_ms": float(np.percentile(lat_b, 99)),
                              "capacity_req_s": 1.0 / svc.mean()}}

    runs = [run_load(ld) for ld in loads]
    srv.close()
    ctx.close()
    del pool
    main = next((r for r in runs if abs(r["load"] - 0.8) < 1e-9), runs[0])
    out = dict(main)
    out["loads"] = runs
    return out


# DRAM bytes (read + write) per row of X from one ncu capture of each kernel
# on 400,000 rows of the e4m3_binary recipe (`bench.py --quick --m 400000`;
# dram__bytes_read.sum + dram__bytes_write.sum over 400,000; the kernels
# stream X, so traffic grows with the rows): f8_sketch_kernel 1,641,817,088 +
# 100,861,696, f8_chain_kernel 1,741,043,968 + 225,536, xproj_kernel
# 1,658,828,544 + 379,153,152.
TRAFFIC_PER_ROW = {
    ("e4m3_binary", "sketch"): (1_641_817_088 + 100_861_696) / 400_000,
    ("e4m3_binary", "chain_main"): (1_741_043_968 + 225_536) / 400_000,
}
# (the reduction map's capture, 5,095 B per row, predates its 16-column fold
# segments, so its traffic is reported as null until it is captured again)


def roofline(kernel, ms, bytes_, flops, peak_tflops, pk, m, workload, traffic_key=None):
    """Roofline of one kernel: bound by HBM (bytes / copy bandwidth) or by the
    tensor pipe (flops / peak), whichever is slower; achieved = algorithmic
    work / measured time."""
    t_hbm = bytes_ / (pk["hbm"] * 1e9)
    t_ten = flops / (peak_tflops * 1e12) if flops else 0.0
    sec = ms / 1e3
    tr = TRAFFIC_PER_ROW.get((workload, traffic_key or kernel))
    if t_ten > t_hbm:
        ach = flops / sec / 1e12
        out = {"bound": "tensor", "achieved": ach, "peak": peak_tflops, "unit": "TFLOP/s", "frac": ach / peak_tflops}
    else:
        ach = bytes_ / sec / 1e9
        out = {"bound": "hbm", "achieved": ach, "peak": pk["hbm"], "unit": "GB/s", "frac": ach / pk["hbm"]}
    out.update({"kernel": kernel, "ms_per_launch": ms, "bytes_per_launch": bytes_, "flops_per_launch": flops,
                "traffic": (tr * m if tr else None), "peak_kind": pk["kind"]})
    return out




def run_reference(args):
    """The reference arm: the FP64 oracle (the paper ships no program) on the
    host cores, each step one oracle fit plus reduction map of a bounded
    sample of the headline workload."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import lspca as O
    rows = args.ref_rows
    w, X, Om = _oracle_sample(rows)
    for _ in range(args.warmup):
        _oracle_step(O, X, Om)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_step(O, X, Om)
    dt = time.perf_counter() - t0
    val = rows * args.steps / dt
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    full = S_workload(WORKLOAD)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "samples/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD} {full.m}x{full.n} k={full.k} very sparse p={full.p}, "
                                   f"fit + reduction map of all rows",
                       "m": full.m, "n": full.n, "k": full.k},
            "cpu_baseline": {"value": val, "unit": "samples/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: one oracle fit plus reduction map of {rows} rows x {w.n} "
                                       f"(same recipe)"},
            "e2e": {"value": val, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def S_workload(name):
    from paper_1709_07175_gb300 import synthetic as S
    return S.WORKLOADS[name]


PASS_NAMES = ["omega", "sketch", "chain_main", "chain_reduce", "qr", "small", "total"]


def _events(torch, n):
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def measure_headline(L, S, torch, w, X, ctx, stream, args, dist, pk, ws):
    """The headline step on this rank: the Lazy SPCA fit of X (one GPU) or of
    the row-sharded matrix (N ranks), then the reduction map of the rank's
    rows.  Returns the timing, per-kernel rooflines and launch counts."""
    from paper_1709_07175_gb300 import shard
    dev = X.device
    om = L.omega("sparse", w.omega_seed, w.p)
    V = torch.empty(w.n, w.k, dtype=torch.float32, device=dev)
    sigma = torch.empty(w.k, dtype=torch.float64, device=dev)
    rk = torch.empty(1, dtype=torch.int32, device=dev)
    Y = torch.empty(w.m, w.k, dtype=torch.float32, device=dev)
    steps = max(args.steps, 1)
    pe = _events(torch, 2 * steps)

    def step(i=None):
        if ws == 1:
            rc = L.lspca_fit(ctx.handle, X, w.k, om, 0, V, sigma, None, rk, stream)
            if rc != L.OK:
                raise L.LspcaError(rc, "lspca_fit")
        else:
            V2, s2, r2, _, _ = shard.sharded_fit(ctx, X, w.m * ws, w.k, om)
            V.copy_(V2)
            sigma.copy_(s2)
            rk.copy_(r2)
        if i is not None:
            pe[2 * i].record(stream)
        rc = L.lspca_project(ctx.handle, X, V, w.k, Y, stream)
        if rc != L.OK:
            raise L.LspcaError(rc, "lspca_project")
        if i is not None:
            pe[2 * i + 1].record(stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    L.lspca_profile(ctx.handle, True)
    launches0 = ctx.launch_count()
    clocks = Clocks(dev.index or 0)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = _events(torch, 2)
    e0.record(stream)
    for i in range(steps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = ctx.launch_count() - launches0
    pass_ms, calls = L.lspca_profile_read(ctx.handle)
    L.lspca_profile(ctx.handle, False)
    proj_ms = sum(pe[2 * i].elapsed_time(pe[2 * i + 1]) for i in range(steps)) / steps
    ms = shard.max_over_ranks(ms, dev)
    out = {"ms": ms / steps, "launches": launches // steps, "clocks": clk, "project_ms": proj_ms,
           "rank": int(rk.item()), "sigma_1": float(sigma[0].item())}
    if ws == 1 and calls:
        per = {nm: pass_ms[i] / calls for i, nm in enumerate(PASS_NAMES)}
        per["project"] = proj_ms
        out["passes_ms"] = per
        m, n, k = w.m, w.n, w.k
        f8 = 2.0 * pk["bf16_sustained"]  # FP8 dense peak: the measured BF16 peak x the nominal ratio 2
        kern = {
            "sketch": roofline("sketch", per["sketch"], m * (n + k), 2.0 * m * n * k, f8, pk, m, w.name),
            "chain_main": roofline("chain_main", per["chain_main"], m * (n + k), 2.0 * m * n * k, f8, pk, m, w.name),
            "project": roofline("project", proj_ms, m * (n + 4 * k), 4.0 * m * n * k, pk["bf16_sustained"], pk, m,
                                w.name),
        }
        out["kernels"] = kern
        dom = max(("sketch", "chain_main", "project", "small"), key=lambda nm: per[nm])
        out["dominant"] = dom
        out["roofline"] = kern.get(dom, kern["project"])
    del Y
    return out, V, sigma


def _time(torch, stream, fn, reps):
    fn()
    torch.cuda.synchronize()
    a, b = _events(torch, 2)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _sine(torch, A, B):
    """Largest principal-angle sine between span(A) and span(B) (orthonormal
    columns), ||B - A (A^T B)||_2 in FP64."""
    A = A.double()
    B = B.double()
    return float(torch.linalg.matrix_norm(B - A @ (A.T @ B), ord=2).item())


def measure_spca(L, torch, w, X, ctx, stream, om, V_lazy, ms_lazy, reps):
    """The SPCA comparison path (Alg. 1/3: R of the QR of U by CholeskyQR2,
    F = R^-T U^T X) on the same X, with the QR's time and path and the
    agreement of its span with Lazy SPCA's (Prop. 2).  Both paths' errors
    against the FP64 oracle are asserted by the parity tests, not measured
    here (the bench runs the oracle only for its CPU baseline)."""
    V = torch.empty(w.n, w.k, dtype=torch.float32, device=X.device)
    sig = torch.empty(w.k, dtype=torch.float64, device=X.device)
    rk = torch.empty(1, dtype=torch.int32, device=X.device)

    def fn():
        rc = L.spca_fit(ctx.handle, X, w.k, om, 0, V, sig, None, rk, stream)
        if rc != L.OK:
            raise L.LspcaError(rc, "spca_fit")
    ms = _time(torch, stream, fn, reps)
    rep = L.lspca_report()
    L.spca_fit(ctx.handle, X, w.k, om, 0, V, sig, None, rk, stream, rep)
    out = {"ms_per_fit": ms, "lazy_fit_ms": ms_lazy, "lazy_speedup": ms / ms_lazy,
           "qr_ms": rep.ms_qr, "qr_path": {1: "CholeskyQR2", 2: "Householder TSQR"}.get(rep.qr_path, "?"),
           "sine_spca_vs_lazy": _sine(torch, V, V_lazy),
           "note": "sine: largest principal-angle sine between span(V^s) and span(V^l), equal spans by Prop. 2"}
    return out


def measure_form(L, S, torch, name, stream, local, pk, reps, m=None, spca=False, gram=False):
    """Fit and reduction map of another workload (same process, one GPU)."""
    w = S.WORKLOADS[name]
    if m:
        w = w.scaled(m=m)
    dev = torch.device(f"cuda:{local}")
    X = S.generate(w, device=dev)
    torch.cuda.synchronize()
    ctx = L.Context(local)
    om = L.omega(w.omega, w.omega_seed, w.p)
    V = torch.empty(w.n, w.k, dtype=torch.float32, device=dev)
    sig = torch.empty(w.k, dtype=torch.float64, device=dev)
    rk = torch.empty(1, dtype=torch.int32, device=dev)
    Y = torch.empty(w.m, w.k, dtype=torch.float32, device=dev)

    def fit(flags=0, G=None):
        rc = L.lspca_fit(ctx.handle, X, w.k, om, flags, V, sig, G, rk, stream)
        if rc != L.OK:
            raise L.LspcaError(rc, "lspca_fit")

    def proj():
        rc = L.lspca_project(ctx.handle, X, V, w.k, Y, stream)
        if rc != L.OK:
            raise L.LspcaError(rc, "lspca_project")
    fit()
    fit_ms = _time(torch, stream, fit, reps)
    L.lspca_profile(ctx.handle, True)
    fit()
    pass_ms, calls = L.lspca_profile_read(ctx.handle)
    L.lspca_profile(ctx.handle, False)
    per = {nm: pass_ms[i] / max(calls, 1) for i, nm in enumerate(PASS_NAMES)}
    proj_ms = _time(torch, stream, proj, reps)
    esz = X.element_size()
    xb = w.m * w.n * esz
    out = {"workload": f"{name} {w.m}x{w.n} {w.dtype} k={w.k} {w.omega} omega" + (f" p={w.p}" if w.p else ""),
           "fit_ms": fit_ms, "fit_samples_per_s": w.m / (fit_ms / 1e3), "passes_ms": per,
           "project_ms": proj_ms, "project_samples_per_s": w.m / (proj_ms / 1e3),
           "fit_x_pass_roofline_frac": (xb / (pk["hbm"] * 1e9)) / (fit_ms / 1e3)}
    if name == "bf16_dense":
        # BF16 X: sketch one exact product, pass F two (U split into a BF16 pair), projection two (V pair)
        bf = pk["bf16_sustained"]
        out["kernels"] = {
            "sketch": roofline("sketch", per["sketch"], w.m * (w.n * 2 + w.k * 4), 2.0 * w.m * w.n * w.k, bf, pk,
                               w.m, name),
            "chain_main": roofline("chain_main", per["chain_main"], w.m * (w.n * 2 + w.k * 4),
                                   4.0 * w.m * w.n * w.k, bf, pk, w.m, name),
            "project": roofline("project", proj_ms, w.m * (w.n * 2 + w.k * 4), 4.0 * w.m * w.n * w.k, bf, pk, w.m,
                                name)}
    if name == "fp32_sparse":
        out["kernels"] = {
            "sketch": roofline("sketch", per["sketch"], w.m * (w.n + w.k) * 4, 0, 1.0, pk, w.m, name),
            "chain_main": roofline("chain_main", per["chain_main"], w.m * (w.n + w.k) * 4, 0, 1.0, pk, w.m, name),
            # FP32 X against V split into three exact BF16 pieces: six products
            # (k <= 128, n a multiple of 8), else three; tensor-bound at six
            "project": roofline("project", proj_ms, w.m * (w.n + w.k) * 4,
                                (6 if w.k <= 128 and w.n % 8 == 0 else 3) * 2.0 * w.m * w.n * w.k,
                                pk["bf16_sustained"], pk, w.m, name)}
    if gram:
        G = torch.empty(w.k, w.k, dtype=torch.float64, device=dev)
        out["gram"] = {"ms_per_fit_on": _time(torch, stream, lambda: fit(L.WANT_GRAM, G), reps),
                       "ms_per_fit_off": fit_ms,
                       "note": "the same fit with the optional G = U^T U output (LSPCA_WANT_GRAM) on and off"}
    if spca:
        out["spca"] = measure_spca(L, torch, w, X, ctx, stream, om, V, fit_ms, reps)
    ctx.close()
    del X, Y
    torch.cuda.empty_cache()
    return out


def measure_kxk(L, torch, local, stream, reps=5):
    """The k x k step alone (lspca_decompose, n = 4,096, FP32 V) on a flat
    spectrum (sigma_i(F) = i^-0.2) and a steep one (sigma_i(F) = 2^-i)."""
    import numpy as np
    ctx = L.Context(local)
    out = {}
    for k in (128, 256):
        n = 4096
        rng = np.random.default_rng(k)
        Q, _ = np.linalg.qr(rng.standard_normal((n, k)))
        P, _ = np.linalg.qr(rng.standard_normal((k, k)))
        i = np.arange(1, k + 1, dtype=np.float64)
        for spec, s in (("flat", i ** -0.2), ("steep", 2.0 ** -i)):
            F = torch.from_numpy((P * s) @ Q.T).to(f"cuda:{local}").contiguous()
            out[f"k{k}_{spec}_ms"] = _time(torch, stream, lambda: ctx.decompose(F, 200000, torch.float32), reps)
    ctx.close()
    return out


def measure_sparse(L, S, torch, local, stream):
    """A sparse X in CSR form, the shape of the paper's TF-IDF experiment."""
    sw_ = S.SPARSE_TFIDF
    dev = torch.device(f"cuda:{local}")
    rp_, c_, v_ = (t.to(dev) for t in S.sparse_csr(sw_["m"], sw_["n"], sw_["density"], sw_["seed"]))
    om_s = L.omega("sparse", sw_["omega_seed"], sw_["p"])
    ctx = L.Context(local)
    ms = _time(torch, stream, lambda: ctx.fit_csr(rp_, c_, v_, sw_["n"], sw_["k"], om_s, report=False,
                                                  stream=stream), 5)
    ctx.close()
    return {"workload": f"CSR {sw_['m']}x{sw_['n']} density {sw_['density']} nnz {v_.numel()} "
                        f"k={sw_['k']} very sparse p={sw_['p']}",
            "ms_per_fit": ms, "samples_per_s": sw_["m"] / (ms / 1e3), "nnz_per_s": v_.numel() / (ms / 1e3),
            "api": "lspca_fit_csr"}


def measure_e2e(L, torch, w, X, ctx, stream, reps):
    """The headline step end to end through the public API with host buffers:
    lspca_fit_project_host streams X from pinned host memory into device
    memory while the slices already copied are sketched and folded into F
    (Alg. 4), runs the k x k step, and projects every row slice by slice while
    the previous slice of Y is copied back; then V and sigma are copied back."""
    dev = X.device
    Xh = torch.empty(X.shape, dtype=X.dtype, pin_memory=True)
    Xh.copy_(X)
    om = L.omega("sparse", w.omega_seed, w.p)
    V = torch.empty(w.n, w.k, dtype=torch.float32, device=dev)
    sig = torch.empty(w.k, dtype=torch.float64, device=dev)
    rk = torch.empty(1, dtype=torch.int32, device=dev)
    Vh = torch.empty(V.shape, dtype=V.dtype, pin_memory=True)
    sh = torch.empty(sig.shape, dtype=sig.dtype, pin_memory=True)
    Yh = torch.empty((w.m, w.k), dtype=torch.float32, pin_memory=True)

    def step():
        rc = L.lspca_fit_project_host(ctx.handle, Xh, w.k, om, 0, 0, X, V, sig, Yh, rk, stream)
        if rc != L.OK:
            raise L.LspcaError(rc, "lspca_fit_project_host")
        Vh.copy_(V, non_blocking=True)
        sh.copy_(sig, non_blocking=True)
    h2d_ms = _time(torch, stream, lambda: X.copy_(Xh, non_blocking=True), 1)
    ms = _time(torch, stream, step, reps)
    xb = Xh.numel() * Xh.element_size()
    out = {"value": w.m / (ms / 1e3), "unit": "samples/s", "h2d_bytes_per_step": xb,
           "d2h_bytes_per_step": Vh.numel() * 4 + sh.numel() * 8 + Yh.numel() * 4, "ms_per_step": ms,
           "api": "lspca_fit_project_host (X from pinned host memory, Y to pinned host memory), then V and sigma "
                  "copied back",
           "h2d_copy_ms": h2d_ms, "h2d_copy_gbs": xb / (h2d_ms / 1e3) / 1e9}
    del Xh, Yh
    return out


def run_gpu(args):
    import torch

    from paper_1709_07175_gb300 import build as B
    from paper_1709_07175_gb300 import lspca as L
    from paper_1709_07175_gb300 import shard
    from paper_1709_07175_gb300 import synthetic as S

    ws, rank, local = _dist()
    B.build()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    pk = _peaks()
    stream = torch.cuda.current_stream()
    w = S.WORKLOADS[WORKLOAD]
    if args.m:
        w = w.scaled(m=args.m)
    from dataclasses import replace
    w = replace(w, data_seed=w.data_seed + 1000 * rank)  # each rank its own block of rows
    X = S.generate(w, device=f"cuda:{local}")
    torch.cuda.synchronize()
    ctx = L.Context(local)
    head, V, sigma = measure_headline(L, S, torch, w, X, ctx, stream, args, dist, pk, ws)
    value = w.m * ws / (head["ms"] / 1e3)
    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "e4m3", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD} {w.m}x{w.n} k={w.k} very sparse p={w.p}: fit + reduction map of "
                                   f"all rows" + (f", rows sharded over {ws} ranks (one NCCL exchange of F)"
                                                  if ws > 1 else ""),
                       "m": w.m * ws, "n": w.n, "k": w.k, "x_bytes": w.m * w.n * ws,
                       "l2": "inputs larger than L2 (no flush)"},
            "roofline": head.get("roofline"), "kernels": head.get("kernels"), "passes_ms": head.get("passes_ms"),
            "dominant_kernel": head.get("dominant"), "project_ms": head["project_ms"],
            "gpu_launches": head["launches"], "clocks": head["clocks"], "fit_rank": head["rank"]}
    if rank == 0 and ws == 1:
        if not args.quick:
            om = L.omega("sparse", w.omega_seed, w.p)
            lazy_ms = head["passes_ms"]["total"]
            line["spca"] = measure_spca(L, torch, w, X, ctx, stream, om, V, lazy_ms, 3)
            line["e2e"] = measure_e2e(L, torch, w, X, ctx, stream, 3)
        ctx.close()
        del X, V, sigma
        torch.cuda.empty_cache()
        if not args.quick:
            for key, name, m, extra in (("bf16_dense", "bf16_dense", None, {}),
                                        ("fp32_sparse", "fp32_sparse", None, {"spca": True, "gram": True})):
                try:
                    line[key] = measure_form(L, S, torch, name, stream, local, pk, 5, m=m, **extra)
                except Exception as e:  # the headline line stands on its own
                    line[key] = {"error": f"{type(e).__name__}: {e}"}
            line["kxk"] = measure_kxk(L, torch, local, stream)
            try:
                line["sparse"] = measure_sparse(L, S, torch, local, stream)
            except Exception as e:
                line["sparse"] = {"error": f"{type(e).__name__}: {e}"}
            if args.serve_seconds > 0:
                try:
                    line["serve"] = serve_bench(L, S, torch, local, args.serve_seconds)
                except Exception as e:
                    line["serve"] = {"error": f"{type(e).__name__}: {e}"}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_rows, args.cpu_seconds)
    else:
        ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()




def launch_ranks(n: int, argv: list) -> int:
    """Start n ranks of this script on this node (torch.distributed.run, one
    process per GPU, rendezvous on 127.0.0.1) and return their exit status."""
    import socket
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    port = sk.getsockname()[1]
    sk.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *argv]
    return subprocess.call(cmd)


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--m", type=int, default=0, help="override the rows per rank (smaller runs)")
    ap.add_argument("--cpu-rows", type=int, default=20_000)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-rows", type=int, default=2_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="the headline line only (no extra keys)")
    ap.add_argument("--serve-seconds", type=float, default=5.0, help="serving run length (0 = skip)")
    args = ap.parse_args(argv)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(launch_ranks(args.gpus, argv))
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
