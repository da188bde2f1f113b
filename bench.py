"""Benchmark: Lazy SPCA fit throughput on one GB300 (and N replicas under torchrun).

Workload (one step = one whole Lazy SPCA fit, every pass of the hot path):
fp32_sparse -- X of 200,000 x 4,096 FP32 (sigma_i = 1/i over rank 512 plus
N(0, 1e-3^2) noise), k = 128, very sparse Omega with p = 64.  X (3.28 GB)
is larger than L2, so no flush is needed between steps.

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
WORKLOAD = "fp32_sparse"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


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


def cpu_baseline(rows: int, reps_seconds: float = 10.0) -> dict:
    """The FP64 oracle as it stands, on a bounded sample of the workload."""
    import numpy as np

    from oracle import lspca as O
    from oracle import philox as P
    from paper_1709_07175_gb300 import synthetic as S
    w = S.WORKLOADS[WORKLOAD].scaled(m=rows)
    X = S.generate(w).double().numpy()
    Om = P.omega_sparse(w.omega_seed, w.n, w.k, w.p)
    t0 = time.perf_counter()
    reps = 0
    while True:
        O.lspca_fit(X, Om, route="eig")
        reps += 1
        if time.perf_counter() - t0 >= reps_seconds:
            break
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": rows * reps / dt, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": f"{rows} rows x {w.n} of the {WORKLOAD} workload (same recipe), k={w.k}, "
                      f"{reps} fit(s) in {dt:.1f} s; FP64 numpy, BLAS threads = host default",
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


# DRAM bytes (read + write) per row of X of one launch, from one ncu capture
# (--set full) at 50,000 rows of the same workload; traffic grows in
# proportion to the rows.  Set an entry to None when its kernel changes, until
# it is captured again.
TRAFFIC_PER_ROW = {
    "sketch": (822.426624e6 + 23.101952e6) / 50000,
    "chain_main": (844.953088e6 + 25.067264e6) / 50000,
}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import lspca as O
    from oracle import philox as P
    from paper_1709_07175_gb300 import synthetic as S
    rows = args.ref_rows
    w = S.WORKLOADS[WORKLOAD].scaled(m=rows)
    X = S.generate(w).double().numpy()
    Om = P.omega_sparse(w.omega_seed, w.n, w.k, w.p)
    for _ in range(args.warmup):
        O.lspca_fit(X, Om, route="eig")
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.lspca_fit(X, Om, route="eig")
    dt = time.perf_counter() - t0
    val = rows * args.steps / dt
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    full = S.WORKLOADS[WORKLOAD]
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "samples/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD} {full.m}x{full.n} k={full.k} very sparse p={full.p}",
                       "m": full.m, "n": full.n, "k": full.k},
            "cpu_baseline": {"value": val, "unit": "samples/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: one oracle fit of {rows} rows x {w.n} (same recipe)"},
            "e2e": {"value": val, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch

    from paper_1709_07175_gb300 import build as B
    from paper_1709_07175_gb300 import lspca as L
    from paper_1709_07175_gb300 import synthetic as S

    ws, rank, local = _dist()
    B.build()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl")
        dist = dist_mod

    def barrier():
        if dist is not None:
            dist.barrier()

    w = S.WORKLOADS[WORKLOAD]
    if args.m:
        w = w.scaled(m=args.m)
    # weak scaling: each rank fits its own independent problem (different data seed)
    from dataclasses import replace
    w = replace(w, data_seed=w.data_seed + 1000 * rank)
    X = S.generate(w, device=f"cuda:{local}")
    torch.cuda.synchronize()
    ctx = L.Context(local)
    om = L.omega("sparse", w.omega_seed, w.p)
    stream = torch.cuda.current_stream()
    V = torch.empty(w.n, w.k, dtype=torch.float32, device=X.device)
    sigma = torch.empty(w.k, dtype=torch.float64, device=X.device)
    rk = torch.empty(1, dtype=torch.int32, device=X.device)

    def step(fn=L.lspca_fit):
        rc = fn(ctx.handle, X, w.k, om, 0, V, sigma, None, rk, stream)
        if rc != L.OK:
            raise L.LspcaError(rc, fn.__name__)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs
    L.lspca_profile(ctx.handle, True)
    launches0 = ctx.launch_count()
    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = ctx.launch_count() - launches0
    pass_ms, calls = L.lspca_profile_read(ctx.handle)
    L.lspca_profile(ctx.handle, False)
    if dist is not None:
        t = torch.tensor([ms], device=X.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / args.steps
    value = w.m * ws * args.steps / (ms / 1e3)

    # ---- the same fit with the optional Gram G = U^T U (Lemma 1 / Prop. 1) on
    G = torch.empty(w.k, w.k, dtype=torch.float64, device=X.device)

    def step_gram():
        rc = L.lspca_fit(ctx.handle, X, w.k, om, L.WANT_GRAM, V, sigma, G, rk, stream)
        if rc != L.OK:
            raise L.LspcaError(rc, "lspca_fit")

    for _ in range(2):
        step_gram()
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    ngr = max(3, min(args.steps, 10))
    g0.record(stream)
    for _ in range(ngr):
        step_gram()
    g1.record(stream)
    torch.cuda.synchronize()
    gram_ms = g0.elapsed_time(g1) / ngr
    del G

    # ---- SPCA comparison path (same workload, same launch configuration)
    for _ in range(2):
        step(L.spca_fit)
    torch.cuda.synchronize()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    nsp = max(3, min(args.steps, 10))
    s0.record(stream)
    for _ in range(nsp):
        step(L.spca_fit)
    s1.record(stream)
    torch.cuda.synchronize()
    spca_ms = s0.elapsed_time(s1) / nsp

    # ---- the reduction map Y = X V (Sec. III-B.2) of the fitted V over the same X
    Y = torch.empty(w.m, w.k, dtype=torch.float32, device=X.device)

    def proj():
        rc = L.lspca_project(ctx.handle, X, V, w.k, Y, stream)
        if rc != L.OK:
            raise L.LspcaError(rc, "lspca_project")

    for _ in range(3):
        proj()
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    npj = max(3, min(args.steps, 10))
    p0.record(stream)
    for _ in range(npj):
        proj()
    p1.record(stream)
    torch.cuda.synchronize()
    proj_ms = p0.elapsed_time(p1) / npj
    del Y

    # ---- a sparse X in CSR form, the shape of the paper's TF-IDF experiment
    sparse = None
    if rank == 0:
        try:
            sw_ = S.SPARSE_TFIDF
            rp_, c_, v_ = (t.to(X.device) for t in S.sparse_csr(sw_["m"], sw_["n"], sw_["density"], sw_["seed"]))
            om_s = L.omega("sparse", sw_["omega_seed"], sw_["p"])
            for _ in range(2):
                ctx.fit_csr(rp_, c_, v_, sw_["n"], sw_["k"], om_s, report=False)
            torch.cuda.synchronize()
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            for _ in range(5):
                ctx.fit_csr(rp_, c_, v_, sw_["n"], sw_["k"], om_s, report=False, stream=stream)
            q1.record(stream)
            torch.cuda.synchronize()
            sms = q0.elapsed_time(q1) / 5
            sparse = {"workload": f"CSR {sw_['m']}x{sw_['n']} density {sw_['density']} nnz {v_.numel()} "
                                  f"k={sw_['k']} very sparse p={sw_['p']}",
                      "ms_per_fit": sms, "samples_per_s": sw_["m"] / (sms / 1e3),
                      "nnz_per_s": v_.numel() / (sms / 1e3), "api": "lspca_fit_csr"}
            del rp_, c_, v_
        except Exception as e:  # the fit line above stands on its own
            sparse = {"error": f"{type(e).__name__}: {e}"}

    # ---- end to end through the public API: a host-resident (pinned) X, fitted
    # by lspca_fit_host (row slices copied to the device while the previous
    # slice is computed, Algorithm 4), V and sigma copied back
    Xh = torch.empty(X.shape, dtype=X.dtype, pin_memory=True)
    Xh.copy_(X)
    Vh = torch.empty(V.shape, dtype=V.dtype, pin_memory=True)
    sh = torch.empty(sigma.shape, dtype=sigma.dtype, pin_memory=True)
    ne2e = max(3, min(args.steps, 5))

    def e2e_step():
        rc = L.lspca_fit_host(ctx.handle, Xh, w.k, om, 0, 0, V, sigma, rk, stream)
        if rc != L.OK:
            raise L.LspcaError(rc, "lspca_fit_host")
        Vh.copy_(V, non_blocking=True)
        sh.copy_(sigma, non_blocking=True)

    # the host -> device copy floor of this node: one plain copy of the same bytes
    X.copy_(Xh, non_blocking=True)
    torch.cuda.synchronize()
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    X.copy_(Xh, non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize()
    h2d_ms = c0.elapsed_time(c1)

    e2e_step()
    torch.cuda.synchronize()
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(ne2e):
        e2e_step()
    t1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = t0.elapsed_time(t1) / ne2e
    if dist is not None:
        t = torch.tensor([e2e_ms], device=X.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())

    # ---- roofline of the dominant kernel
    names = ["omega", "sketch", "chain_main", "chain_reduce", "qr", "small", "total"]
    per = {nm: pass_ms[i] / max(calls, 1) for i, nm in enumerate(names)}
    x_bytes = w.m * w.n * 4
    u_bytes = w.m * w.k * 4
    alg = {"sketch": x_bytes + u_bytes, "chain_main": x_bytes + u_bytes}
    dom = max(alg, key=lambda nm: per[nm])
    peak, peak_kind = _peaks()
    achieved = alg[dom] / (per[dom] / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind,
            "traffic": (TRAFFIC_PER_ROW[dom] * w.m if TRAFFIC_PER_ROW.get(dom) else None),
            "bytes_per_launch": alg[dom], "ms_per_launch": per[dom]}

    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD} {w.m}x{w.n} k={w.k} very sparse p={w.p}", "m": w.m, "n": w.n,
                       "k": w.k, "x_bytes": x_bytes, "l2": "inputs larger than L2 (no flush)"},
            "roofline": roof,
            "fit_roofline_frac": {"lazy": (x_bytes / (peak * 1e9)) / (ms_step / 1e3),
                                  "spca": (x_bytes / (peak * 1e9)) / (spca_ms / 1e3)},
            "spca": {"ms_per_step": spca_ms, "samples_per_s": w.m * ws / (spca_ms / 1e3),
                     "lazy_speedup": spca_ms / ms_step},
            "passes_ms": per,
            "gram": {"ms_per_step_on": gram_ms, "ms_per_step_off": ms_step,
                     "note": "the same fit with the optional G = U^T U output (LSPCA_WANT_GRAM) on and off"},
            "project": {"ms_per_call": proj_ms, "samples_per_s": w.m / (proj_ms / 1e3),
                        "achieved_gbs": (x_bytes + u_bytes) / (proj_ms / 1e3) / 1e9,
                        "frac": (x_bytes + u_bytes) / (proj_ms / 1e3) / 1e9 / peak,
                        "bytes_per_call": x_bytes + u_bytes, "kernel": "tmem_a_kernel (FP32 X and V in three exact BF16 pieces, k=128)"},
            "e2e": {"value": w.m * ws / (e2e_ms / 1e3), "unit": "samples/s",
                    "h2d_bytes_per_step": x_bytes, "d2h_bytes_per_step": w.n * w.k * 4 + w.k * 8,
                    "ms_per_step": e2e_ms, "api": "lspca_fit_host (pinned host X, row slices overlapped)",
                    "h2d_copy_ms": h2d_ms, "h2d_copy_gbs": x_bytes / (h2d_ms / 1e3) / 1e9},
            "sparse": sparse,
            "gpu_launches": launches,
            "clocks": clk}
    if rank == 0 and args.serve_seconds > 0:
        del Xh
        X = None
        torch.cuda.empty_cache()
        try:
            line["serve"] = serve_bench(L, S, torch, local, args.serve_seconds)
        except Exception as e:  # the fit line above stands on its own
            line["serve"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_rows, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--m", type=int, default=0, help="override the row count (smaller runs)")
    ap.add_argument("--cpu-rows", type=int, default=50_000)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-rows", type=int, default=20_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=5.0, help="serving run length (0 = skip)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
