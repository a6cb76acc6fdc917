#!/usr/bin/env python3
"""Benchmark of the implicit distance-matrix product on GB300.

Workload: n = 2^20 points in d = 32 dimensions from a 16-cluster Gaussian
mixture (cluster means N(0, 10^2) per coordinate, within-cluster sd 1), FP32,
and a block of k = 16 FP32 N(0, 1) query columns -- synthetic stand-ins of the
shape of the paper's Gaussian-mixture experiment (Section 4), scaled up.

One step = the whole hot path on that input, inputs already resident in HBM:
  l1:   dm_prepare (radix sort of the 32 columns, Algorithm 1)
        + dm_matmat (prefix-scan query of Algorithm 2, k = 16 columns);
  l2sq: dm_prepare (column means, squared norms)
        + dm_matmat (rank-(d+2) identity of Appendix A).
Metric: point*query*dim per second, counting n*k*d units for each of the two
products (2 n k d per step).  Between timed steps the L2 cache is flushed
(a 512 MiB write); the flush is outside the per-step CUDA-event spans.

Also reported: the per-part breakdown, the on-the-fly GPU brute force (the
plain method) and speedups against it, the relative error of sampled output
rows against the CPU oracle, the roofline of the dominant kernel (live CUDA
events inside the library), an end-to-end number through the C ABI with host
buffers, SM clocks sampled during the timed region, and the CPU oracle timed
on a bounded sample of the workload.

`--impl reference` times the CPU oracle instead (the reference arm).
Under torchrun (N > 1) every rank runs an independent replica (the product is
not sharded; no collective is on the data path): value = all ranks' units / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "point*query*dim/s (l1 + l2sq products, prepare included)"
UNIT = "point*query*dim/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--d", type=int, default=32)
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--no-brute", action="store_true", help="skip the brute-force comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end run")
    ap.add_argument("--no-grad", action="store_true", help="skip the gradient measurement")
    ap.add_argument("--no-krylov", action="store_true", help="skip the block Krylov measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch measurement")
    ap.add_argument("--no-variants", action="store_true", help="skip the variant measurements")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the error study of the two accumulation modes")
    ap.add_argument("--grad-n", type=int, default=1 << 21)
    ap.add_argument("--grad-d", type=int, default=64)
    ap.add_argument("--engine", choices=["auto", "cuda", "tensor"], default="auto",
                    help="units of the squared-l2 contraction (dm_set_engine)")
    ap.add_argument("--profile-only", action="store_true",
                    help="run warmup + steps only (for profiler captures); print nothing else")
    return ap.parse_args()


def workload_config(a):
    # identical in both arms: the driver compares the two config objects
    return {"workload": f"gaussian-mixture-16 n={a.n} d={a.d} k={a.k} fp32",
            "n": a.n, "d": a.d, "k": a.k, "clusters": 16, "dtype": "fp32",
            "products": ["l1", "l2sq"], "prepare_in_step": True,
            "l2_flush": "GPU arm: 512 MiB write between timed steps (outside the step events); "
                        "CPU arm: none",
            "l1_accumulation": "L2 reductions (dm_set_deterministic off)",
            "l2_engine": getattr(a, "engine", "auto")}


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replicas_value(ms_local, units_per_rank, world, device):
    """Whole-job throughput of `world` independent replicas: every rank does
    `units_per_rank` units per step; the job's step time is the slowest
    rank's (max over ranks).  Returns (ms per step, units per second)."""
    ms = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_rank / (ms / 1e3)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------- clocks
class NvmlClockSampler:
    """SM clock and clock-event reasons read in-process through NVML (read-only
    queries) on a background thread every `interval_s`, between start() and
    stop() -- enough samples even for a timed region of a few tens of ms."""
    # clock-event reason bits (nvml.h)
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_device, interval_s: float = 0.01):
        import ctypes
        import threading
        self.ok = False
        self.interval = interval_s
        self.samples = []          # (sm_mhz, reasons bitmask, power_mw)
        self.stop_evt = threading.Event()
        self.thread = None
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            self.lib = lib
            self.h = ctypes.c_void_p()
            import torch
            uuid = "GPU-" + str(torch.cuda.get_device_properties(torch_device).uuid)
            if lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) != 0:
                idx = torch_device.index or 0
                vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
                ids = [v for v in vis.split(",") if v.strip()]
                if ids and ids[min(idx, len(ids) - 1)].strip().isdigit():
                    idx = int(ids[min(idx, len(ids) - 1)])
                if lib.nvmlDeviceGetHandleByIndex_v2(idx, ctypes.byref(self.h)) != 0:
                    return
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) != 0:   # NVML_CLOCK_SM
                return
            self.max_mhz = mx.value
            self.ok = True
        except (OSError, AttributeError, RuntimeError):
            self.ok = False

    def _read(self):
        import ctypes
        mhz, rs, mw = ctypes.c_uint(), ctypes.c_ulonglong(), ctypes.c_uint()
        if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(mhz)) != 0:
            return None
        if self.lib.nvmlDeviceGetCurrentClocksEventReasons(self.h, ctypes.byref(rs)) != 0:
            rs.value = 0
        if self.lib.nvmlDeviceGetPowerUsage(self.h, ctypes.byref(mw)) != 0:
            mw.value = 0
        return mhz.value, rs.value, mw.value

    def _loop(self):
        while True:
            r = self._read()
            if r is not None:
                self.samples.append(r)
            if self.stop_evt.wait(self.interval):
                return

    def start(self):
        import threading
        if not self.ok:
            return False
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()
        return True

    def stop(self):
        if self.thread is None:
            return None
        self.stop_evt.set()
        self.thread.join(timeout=5)
        r = self._read()            # one reading at the end of the region as well
        if r is not None:
            self.samples.append(r)
        if not self.samples:
            return None
        reasons = set()
        for _, bits, _ in self.samples:
            for b, nm in self.REASONS.items():
                if bits & b:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(s[0] for s in self.samples), "sm_max_mhz": self.max_mhz,
                "samples": len(self.samples), "source": "nvml", "interval_ms": self.interval * 1e3,
                "power_w_median": statistics.median(s[2] for s in self.samples) / 1e3,
                "reasons": sorted(reasons)}


class ClockSampler:
    """Fallback when NVML cannot be loaded: `nvidia-smi -lms`, started before
    the timed region (its first line awaited) and stopped after it."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="dm_clocks_", suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 5 and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "samples": len(sm),
                "source": "nvidia-smi", "reasons": sorted(reasons)}


def start_clock_sampler(dev):
    s = NvmlClockSampler(dev)
    if s.start():
        return s
    return ClockSampler(dev.index or 0)


# ------------------------------------------------------------- CPU oracle
_WORKLOAD_CACHE = {}


def cpu_oracle_sample(n, d, d_sample, k, pool=None, workers=1):
    """Time the CPU oracle on the workload: the sort-based l1 form of
    Algorithms 1-2 on the first d_sample coordinates (blocks of coordinates on
    `workers` processes of `pool`) and the p = 2 identity on all coordinates,
    in this process.  Returns seconds."""
    import oracle
    from oracle import parallel
    from paper_2210_15114_gb300 import inputs
    key = (n, d, k)
    if key not in _WORKLOAD_CACHE:
        _WORKLOAD_CACHE.clear()
        _WORKLOAD_CACHE[key] = inputs.workload_mixture_f32(n=n, d=d, k=k)
    X, Z = _WORKLOAD_CACHE[key]
    t0 = time.perf_counter()
    parallel.l1_sort(X[:, :d_sample], Z, workers, pool)
    oracle.l2sq_identity(X, Z)
    return time.perf_counter() - t0


def cpu_baseline(n, d, k):
    """The oracle as it stands on all host cores, in a spawned subprocess (no
    CUDA context): the whole workload, every coordinate, at full n."""
    cores = os.cpu_count() or 1
    code = ("import sys, json; sys.path.insert(0, %r); import bench\n"
            "from oracle import parallel\n"
            "if __name__ == '__main__':\n"
            "    with parallel.executor(%d) as pool:\n"
            "        print(json.dumps(bench.cpu_oracle_sample(%d, %d, %d, %d, pool, %d)))\n"
            % (ROOT, cores, n, d, d, k, cores))
    with tempfile.NamedTemporaryFile("w", suffix=".py", delete=False) as f:
        f.write(code)
        path = f.name
    try:
        r = subprocess.run([sys.executable, path], capture_output=True, text=True, timeout=900)
    finally:
        os.unlink(path)
    if r.returncode != 0:
        return {"value": None, "error": r.stderr[-300:]}
    secs = float(r.stdout.strip().splitlines()[-1])
    units = 2 * n * d * k
    return {"value": units / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
            "seconds": secs,
            "sample": f"the whole workload (all {d} coordinates, n={n}, k={k}): numpy sort-based l1 "
                      f"form (Algorithms 1-2) with the coordinates on {cores} processes + p=2 "
                      f"identity (BLAS threads), FP64"}


# ------------------------------------------------------------- algorithmic bytes
def algorithmic_bytes(group, n, d, k, launches):
    """Bytes the method itself moves per launch of a kernel group (FP32
    elements), from the per-step figure of the group divided by the group's
    launches per step."""
    nd = n * d
    per_step = {
        # key 4 + perm 4 + gathered Z row 4k + per-coordinate contribution 4k, + out 4k
        "l1_query": nd * (8 + 8 * k) + 4 * n * k,
        # read key(+payload) and write key+payload: 12 B on the first pass, 16 on the others
        "sort_onesweep": 16 * nd * launches - 4 * nd,
        "sort_keygen_hist": 8 * nd,                 # read X, write keys
        "l2_reduce": 4 * nd + 4 * n * k,            # X and Z once
        "l2_apply": 4 * nd + 4 * n * k,             # X once, out written
        "l1_aggregate": nd * (8 + 4 * k),           # key + perm + gathered Z row (tile sums)
        "l1_prologue": 8 * n * k + 4 * n,           # read Z and R, write the group-major copy
        "l1_finalize": 8 * n * k + 4 * n,           # read the partial output and R, write out
        "l1_rowsum": 4 * nd + 4 * d + 4 * n,
        "l2_prepare": 4 * nd,                       # column sums: X once
    }.get(group)
    if per_step is None:
        return None
    return per_step / max(launches, 1)


def traffic_record(group):
    """ncu DRAM bytes per launch for a kernel group, if recorded for the
    current source of the kernel (profiles/traffic.json)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f).get(group)
    if not rec:
        return None
    src = os.path.join(ROOT, rec["source"])
    with open(src, "rb") as f:
        if hashlib.sha256(f.read()).hexdigest()[:16] != rec["source_sha"]:
            return None
    return rec["bytes_per_launch"]


def measure_gradient(dm, ctx, stream, flush, dev, peak, n=1 << 21, d=64, reps=10):
    """dm_grad on its own workload, timed with CUDA events per call (L2
    flushed between calls), with the library's per-kernel-group events."""
    import numpy as np
    import torch
    import oracle
    from paper_2210_15114_gb300 import inputs
    X, W, Z = inputs.workload_gradient(n=n, d=d)
    Xd, Wd, Zd = (torch.from_numpy(t).to(dev) for t in (X, W, Z))
    G = torch.empty((n, d), dtype=torch.float32, device=dev)
    res = {"workload": f"uniform [0,1) n={n} d={d} k=1 fp32, w and z N(0,1)",
           "units": "point*dim per second (n d per call)"}
    rows = inputs.sample_rows(n, 4)
    for metric in ("l1", "l2sq"):
        plan = dm.dm_prepare(ctx, metric, Xd)
        for _ in range(3):
            dm.dm_grad(plan, Wd, Zd, out=G)
        torch.cuda.synchronize(dev)
        dm.dm_profile_enable(ctx, True)
        ev = []
        for _ in range(reps):
            flush.zero_()
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s_.record(stream)
            dm.dm_grad(plan, Wd, Zd, out=G)
            e_.record(stream)
            ev.append((s_, e_))
        torch.cuda.synchronize(dev)
        prof = dm.dm_profile_read(ctx)
        dm.dm_profile_enable(ctx, False)
        ms = statistics.mean(s_.elapsed_time(e_) for s_, e_ in ev)
        kern = {g: {"launches_per_call": l // reps, "ms_per_call": t / reps} for g, (l, t) in prof.items()}
        ref = (oracle.l1_grad_rows if metric == "l1" else oracle.l2sq_grad_rows)(X, W, Z, rows)
        err = oracle.relative_error(G.cpu().numpy()[rows], ref)
        entry = {"ms": ms, "value": n * d / (ms * 1e-3), "kernels": kern, "rel_err_sampled_rows": err}
        if metric == "l1" and "grad_l1_eval" in kern:
            # the evaluation pass alone moves the method's bytes: sorted value
            # 4 + perm 4 + gathered (z, w) 8 + gradient write 4 per element
            b = n * d * 20
            t_ms = kern["grad_l1_eval"]["ms_per_call"]
            entry["roofline_eval"] = {"bound": "hbm", "alg_bytes": b, "achieved": b / (t_ms * 1e-3) / 1e9,
                                      "peak": peak, "frac": b / (t_ms * 1e-3) / 1e9 / peak}
            b_all = n * d * 20
            entry["roofline_all"] = {"alg_bytes": b_all, "achieved": b_all / (ms * 1e-3) / 1e9,
                                     "frac": b_all / (ms * 1e-3) / 1e9 / peak}
        if metric == "l2sq":
            # reduce reads X and (z, w); apply reads X and (z, w) and writes G
            b = 4 * n * d * 3 + 16 * n
            entry["roofline_all"] = {"bound": "hbm", "alg_bytes": b, "achieved": b / (ms * 1e-3) / 1e9,
                                     "peak": peak, "frac": b / (ms * 1e-3) / 1e9 / peak}
        res[metric] = entry
        del plan
    return res


def measure_krylov(dm, ctx, stream, dev, n=1 << 22, d=16, k=40, q=8, rank=32, reps=2):
    """Top-32 singular values / rank-32 approximation by block Krylov
    iteration (q + 1 products of k columns each), timed end to end with CUDA
    events (prepare included), plus accuracy checks outside the timing."""
    import numpy as np
    import torch
    from paper_2210_15114_gb300 import inputs
    from paper_2210_15114_gb300.krylov import block_krylov
    X, Pi = inputs.workload_krylov(n=n, d=d, k=k)
    Xd, Pid = torch.from_numpy(X).to(dev), torch.from_numpy(Pi).to(dev)
    res = {"workload": f"10-cluster mixture n={n} d={d} fp32; k={k}, q={q}, rank={rank}",
           "products_per_run": q + 1}
    for metric in ("l1", "l2sq"):
        plan = dm.dm_prepare(ctx, metric, Xd)
        block_krylov(plan, Pid, q, rank)            # warm-up
        torch.cuda.synchronize(dev)
        dm.dm_profile_enable(ctx, True)
        times = []
        for _ in range(reps):
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s_.record(stream)
            plan = dm.dm_prepare(ctx, metric, Xd)
            theta, U = block_krylov(plan, Pid, q, rank)
            e_.record(stream)
            e_.synchronize()
            times.append(s_.elapsed_time(e_))
        prof = dm.dm_profile_read(ctx)
        dm.dm_profile_enable(ctx, False)
        prep = ("sort_keygen_hist", "sort_onesweep", "l1_rowsum") if metric == "l1" else ("l2_prepare",)
        dense = ("dense_tn", "dense_nn")
        prod_ms = sum(t for g, (l, t) in prof.items() if g not in prep and g not in dense) / reps
        prep_ms = sum(t for g, (l, t) in prof.items() if g in prep) / reps
        dense_ms = {g: prof[g][1] / reps for g in dense if g in prof}
        ms = statistics.mean(times)
        entry = {"ms": ms, "prepare_ms": prep_ms, "products_ms": prod_ms,
                 "dense_linear_algebra_ms": ms - prod_ms - prep_ms,
                 "dense_kernels_ms": dense_ms,
                 "top_singular_values": [abs(float(t)) for t in theta[:8].cpu()]}
        if metric == "l2sq":
            Xc = X.astype(np.float64)
            Xc -= Xc.mean(axis=0)
            B = np.concatenate([np.ones((n, 1)), (Xc * Xc).sum(1, keepdims=True), Xc], axis=1)
            C = np.zeros((d + 2, d + 2))
            C[0, 1] = C[1, 0] = 1.0
            C[2:, 2:] = -2 * np.eye(d)
            L = np.linalg.cholesky(B.T @ B)
            ev = np.linalg.eigvalsh(L.T @ C @ L)
            ev = ev[np.argsort(-np.abs(ev))]
            th = theta.cpu().numpy()
            entry["max_rel_err_vs_compressed_form"] = float(np.max(np.abs(th[:d + 2] - ev) / np.abs(ev)))
            entry["max_tail_over_top"] = float(np.max(np.abs(th[d + 2:])) / abs(th[0]))
        else:
            AU = dm.dm_matmat(plan, U.contiguous()).double()
            r = torch.linalg.norm(AU[:, :8] - U.double()[:, :8] * theta[:8].to(AU.device), dim=0)
            entry["top8_residual_over_theta1"] = float(r.max().item() / abs(theta[0].item()))
        res[metric] = entry
        del plan, U
    return res


def measure_batch(dm, ctx, stream, dev, reps=5):
    """512 point sets (n log-uniform in [1024, 262144], d in 2..64, k in
    1..32, FP32 uniform [-1, 1), Z N(0, 1)): prepare + product of every set
    per graph run, lanes chosen by the library's autotuner; the same sets as
    one dm_prepare + dm_matmat call each, for comparison."""
    import torch
    from paper_2210_15114_gb300 import inputs
    sets = inputs.workload_batch()
    Xs = [torch.from_numpy(X).to(dev) for X, _ in sets]
    Zs = [torch.from_numpy(Z).to(dev) for _, Z in sets]
    units = sum(X.shape[0] * X.shape[1] * Z.shape[1] for X, Z in sets)
    res = {"workload": "512 sets, n log-uniform [1024, 262144], d 2..64, k 1..32, fp32 U[-1,1), Z N(0,1)",
           "sum_n": sum(X.shape[0] for X, _ in sets), "sum_ndk": units,
           "units": "point*query*dim per second (sum over sets of n d k per run)"}
    for metric in ("l1", "l2sq"):
        t0 = time.perf_counter()
        b = dm.dm_batch_create(ctx, metric, Xs, Zs, lanes=0)
        torch.cuda.synchronize(dev)
        create_s = time.perf_counter() - t0
        dm.dm_batch_run(b)
        torch.cuda.synchronize(dev)
        l0 = dm.dm_launch_count(ctx)
        ev = []
        for _ in range(reps):
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s_.record(stream)
            dm.dm_batch_run(b)
            e_.record(stream)
            ev.append((s_, e_))
        torch.cuda.synchronize(dev)
        launches = (dm.dm_launch_count(ctx) - l0) // reps
        ms = statistics.mean(s_.elapsed_time(e_) for s_, e_ in ev)
        dm.dm_sync(ctx)
        lanes = dm.dm_batch_lanes(b)
        dm.dm_batch_destroy(b)
        # one call per set, no graph (dm_prepare for l1 synchronizes once per set)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for Xd, Zd in zip(Xs, Zs):
            plan = dm.dm_prepare(ctx, metric, Xd)
            dm.dm_matmat(plan, Zd)
            del plan
        torch.cuda.synchronize(dev)
        single_ms = (time.perf_counter() - t0) * 1e3
        res[metric] = {"ms_per_run": ms, "value": units / (ms * 1e-3), "lanes": lanes,
                       "gpu_launches_per_run": launches, "create_and_autotune_s": create_s,
                       "one_call_per_set_ms_wall": single_ms}
    return res


def measure_variants(dm, ctx, stream, dev, X, Z, Xd, Zd, reps=5):
    """Prepare and query times of the variants on the step's workload
    (n d k units per query), with sampled-row errors against the oracle."""
    import numpy as np
    import torch
    import oracle
    from paper_2210_15114_gb300 import inputs
    n, d = X.shape
    k = Z.shape[1]
    rows = inputs.sample_rows(n, 8)
    P = inputs.simplex_points(n, d)
    Pd = torch.from_numpy(P).to(dev)
    G = inputs.embedding_matrix(256, d)
    Gd = torch.from_numpy(G).to(dev)
    cases = {
        "tv": (lambda: dm.dm_prepare(ctx, "tv", Pd), lambda: oracle.tv_rows(P, Z, rows)),
        "lpp_p4": (lambda: dm.dm_prepare_lpp(ctx, Xd, 4), lambda: oracle.lpp_rows(X, Z, 4, rows)),
        "lpp_p3": (lambda: dm.dm_prepare_lpp(ctx, Xd, 3), lambda: oracle.lpp_rows(X, Z, 3, rows)),
        "lpp_p5": (lambda: dm.dm_prepare_lpp(ctx, Xd, 5), lambda: oracle.lpp_rows(X, Z, 5, rows)),
        "l2_embed_m256": (lambda: dm.dm_prepare_l2_embed(ctx, Xd, Gd),
                          lambda: oracle.l1_rows(oracle.l2_embed(X, G), Z, rows)),
    }
    res = {"workload": f"n={n} d={d} k={k} fp32 (tv: Dirichlet(1) rows; others: the step's mixture)",
           "units": "point*query*dim per second of the query (n d k)"}
    for name, (prep, ref) in cases.items():
        plan = prep()
        out = dm.dm_matmat(plan, Zd)
        torch.cuda.synchronize(dev)
        pe, qe = [], []
        for _ in range(reps):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            plan = prep()
            e1.record(stream)
            dm.dm_matmat(plan, Zd, out=out)
            e2.record(stream)
            pe.append((e0, e1))
            qe.append((e1, e2))
        torch.cuda.synchronize(dev)
        p_ms = statistics.mean(a.elapsed_time(b) for a, b in pe)
        q_ms = statistics.mean(a.elapsed_time(b) for a, b in qe)
        err = oracle.relative_error(out.cpu().numpy()[rows], ref())
        res[name] = {"prepare_ms": p_ms, "query_ms": q_ms, "value": n * d * k / (q_ms * 1e-3),
                     "rel_err_sampled_rows": err}
        del plan
    return res


def measure_accumulation_error(dm, dev, n=1 << 18):
    """Relative error of the l1 product against the FP64 oracle (whole block)
    in both accumulation modes of the sum over the coordinates: vector
    reductions of FP32 values in L2 (default) and the ordered FP64 partial
    output (dm_set_deterministic), at d in {32, 64} and k in {16, 40}, on the
    step's mixture and on the same mixture shifted by 1000 per coordinate."""
    import torch
    import oracle
    from oracle import parallel
    from paper_2210_15114_gb300 import inputs
    ctxs = {"l2_reductions_fp32": dm.dm_create(dev.index or 0), "ordered_fp64": dm.dm_create(dev.index or 0)}
    dm.dm_set_deterministic(ctxs["ordered_fp64"], True)
    res = {"n": n, "metric": "||out - AZ||_F / ||AZ||_F, whole block, FP64 oracle on the same FP32 values"}
    for data in ("mixture", "mixture_offset_1000"):
        for d in (32, 64):
            for k in (16, 40):
                if data == "mixture":
                    X, Z = inputs.workload_mixture_f32(n=n, d=d, k=k)
                else:
                    X, Z = inputs.workload_offset_mixture(n, d, k)
                want = parallel.l1_sort(X, Z)
                Xd, Zd = torch.from_numpy(X).to(dev), torch.from_numpy(Z).to(dev)
                entry = {}
                for mode, ctx in ctxs.items():
                    plan = dm.dm_prepare(ctx, "l1", Xd)
                    out = dm.dm_matmat(plan, Zd)
                    dm.dm_sync(ctx)
                    entry[mode] = oracle.relative_error(out.cpu().numpy(), want)
                    del plan
                res[f"{data} d={d} k={k}"] = entry
    return res


# ------------------------------------------------------------- reference arm
def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import parallel
    cores = os.cpu_count() or 1
    # one coordinate per core per step: a bounded sample of the l1 part, the
    # whole squared-l2 part
    d_sample = max(1, min(a.d, cores))
    units = a.n * d_sample * a.k + a.n * a.d * a.k
    with parallel.executor(min(cores, d_sample)) as pool:
        for _ in range(a.warmup):
            cpu_oracle_sample(a.n, a.d, d_sample, a.k, pool, d_sample)
        times = [cpu_oracle_sample(a.n, a.d, d_sample, a.k, pool, d_sample) for _ in range(a.steps)]
    ms = 1e3 * statistics.mean(times)
    value = units / (ms / 1e3)
    sample = (f"per step: the l1 sort-based form (Algorithms 1-2) on {d_sample} of {a.d} coordinates "
              f"(one process per coordinate) + the p=2 identity on all {a.d}, full n={a.n}, k={a.k}, FP64")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(a),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- our arm
def main():
    a = parse_args()
    if a.impl == "reference":
        run_reference(a)
        return
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2210_15114_gb300 import binding as dm
    from paper_2210_15114_gb300 import build, inputs
    build.build()
    dm.load()

    X, Z = inputs.workload_mixture_f32(n=a.n, d=a.d, k=a.k)
    Xd = torch.from_numpy(X).to(dev)
    Zd = torch.from_numpy(Z).to(dev)
    o1 = torch.empty((a.n, a.k), dtype=torch.float32, device=dev)
    o2 = torch.empty_like(o1)
    flush = torch.empty(128 << 20, dtype=torch.float32, device=dev)   # 512 MiB > L2
    stream = torch.cuda.current_stream(dev)
    ctx = dm.dm_create(local, stream.cuda_stream)
    dm.dm_set_engine(ctx, a.engine)

    def step():
        p1 = dm.dm_prepare(ctx, "l1", Xd)
        dm.dm_matmat(p1, Zd, out=o1)
        p2 = dm.dm_prepare(ctx, "l2sq", Xd)
        dm.dm_matmat(p2, Zd, out=o2)
        return p1, p2

    for _ in range(a.warmup):
        plans = step()
        del plans
    torch.cuda.synchronize(dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # ---- timed region
    clocks = start_clock_sampler(dev) if not a.profile_only else None
    dm.dm_profile_enable(ctx, True)
    launches0 = dm.dm_launch_count(ctx)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    barrier()
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter()
    for i in range(a.steps):
        flush.zero_()
        starts[i].record(stream)
        plans = step()
        ends[i].record(stream)
        del plans
    torch.cuda.synchronize(dev)
    barrier()
    t_wall = time.perf_counter() - t_wall
    launches = dm.dm_launch_count(ctx) - launches0
    prof = dm.dm_profile_read(ctx)
    dm.dm_profile_enable(ctx, False)
    clk = clocks.stop() if clocks else None
    dm.dm_sync(ctx)
    if a.profile_only:
        return

    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    units_step = 2 * a.n * a.d * a.k
    ms, value = replicas_value(statistics.mean(step_ms), units_step, world, dev)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- parts, per-kernel groups, roofline
    per_step = {g: t / a.steps for g, (l, t) in prof.items()}
    parts = {
        "l1_prepare_ms": sum(per_step.get(g, 0) for g in ("sort_keygen_hist", "sort_onesweep",
                                                          "l1_rowsum")),
        "l1_query_ms": sum(per_step.get(g, 0) for g in ("l1_prologue", "l1_aggregate", "l1_query",
                                                         "l1_finalize")),
        "l2_prepare_ms": per_step.get("l2_prepare", 0.0),
        "l2_query_ms": sum(per_step.get(g, 0) for g in ("l2_reduce", "l2_apply")),
    }
    peak, peak_kind = load_peaks()
    kernels = {}
    for g, (l, t) in prof.items():
        nl = l // a.steps if l else 0
        per_launch_ms = t / l if l else None
        b = algorithmic_bytes(g, a.n, a.d, a.k, max(nl, 1))
        if b is not None and per_launch_ms:
            kernels[g] = {"launches_per_step": nl, "ms_per_launch": per_launch_ms,
                          "alg_bytes_per_launch": b,
                          "alg_gbs": b / (per_launch_ms * 1e-3) / 1e9}
    dominant = max(kernels, key=lambda g: kernels[g]["ms_per_launch"] * kernels[g]["launches_per_step"])
    # the whole l1 query (prologue, tile sums and scan, sorted pass, finalize)
    # against the same algorithmic bytes as the sorted pass alone
    q_all_ms = parts["l1_query_ms"]
    q_bytes = algorithmic_bytes("l1_query", a.n, a.d, a.k, 1)
    l1_query_all = {"ms": q_all_ms, "alg_gbs": q_bytes / (q_all_ms * 1e-3) / 1e9,
                    "frac": q_bytes / (q_all_ms * 1e-3) / 1e9 / load_peaks()[0]}
    dk = kernels[dominant]
    roofline = {"kernel": dominant, "bound": "hbm", "achieved": dk["alg_gbs"], "peak": peak,
                "unit": "GB/s", "frac": dk["alg_gbs"] / peak,
                "peak_kind": peak_kind + " HBM copy bandwidth",
                "traffic": traffic_record(dominant)}

    # ---- gradient of w^T A(X) z (n = 2^21, d = 64, k = 1, FP32 uniform [0, 1))
    grad = None
    if not a.no_grad:
        grad = measure_gradient(dm, ctx, stream, flush, dev, peak, n=a.grad_n, d=a.grad_d)

    # ---- block Krylov rank-32 (n = 2^22, d = 16, k = 40, q = 8)
    krylov = None
    if not a.no_krylov:
        krylov = measure_krylov(dm, ctx, stream, dev)

    # ---- 512 independent point sets replayed from one graph
    batch = None
    if not a.no_batch:
        batch = measure_batch(dm, ctx, stream, dev)

    # ---- variants: total variation, ||.||_4^4, approximate l2 (m = 256)
    variants = None
    if not a.no_variants:
        variants = measure_variants(dm, ctx, stream, dev, X, Z, Xd, Zd)

    # ---- error of the sum over the coordinates in both accumulation modes
    precision = None
    if not a.no_precision:
        precision = measure_accumulation_error(dm, dev)

    # ---- brute force (the plain method) and accuracy
    brute = None
    if not a.no_brute:
        brute = {}
        for metric in ("l1", "l2sq"):
            ob = torch.empty_like(o1)
            dm.dm_bruteforce(ctx, metric, Xd, Zd, out=ob)       # warm
            torch.cuda.synchronize(dev)
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            dm.dm_bruteforce(ctx, metric, Xd, Zd, out=ob)
            e.record(stream)
            dm.dm_sync(ctx)
            bms = s.elapsed_time(e)
            qms = parts["l1_query_ms"] if metric == "l1" else parts["l2_query_ms"]
            pms = parts["l1_prepare_ms"] if metric == "l1" else parts["l2_prepare_ms"]
            brute[metric] = {"ms": bms, "speedup_query": bms / qms, "speedup_prepare_query": bms / (qms + pms)}
            del ob
    import oracle
    rows = inputs.sample_rows(a.n, 16)
    err = {}
    got1, got2 = o1.cpu().numpy(), o2.cpu().numpy()
    err["l1"] = oracle.relative_error(got1[rows], oracle.l1_rows(X, Z, rows))
    err["l2sq"] = oracle.relative_error(got2[rows], oracle.l2sq_rows(X, Z, rows))

    # ---- end to end through the C ABI with host buffers: the step's two
    # products of the same X and Z in one dm_matmat_host_multi call (X and Z
    # cross the host link once, the products run side by side on two
    # contexts, both results come back).  Reported beside it: the two
    # products as two dm_matmat_host_async calls on two contexts issued from
    # this thread (X and Z copied once per product), and as two blocking
    # dm_matmat_host calls one after the other.
    e2e = None
    if not a.no_e2e:
        Xh = torch.from_numpy(X).pin_memory().numpy()
        Zh = torch.from_numpy(Z).pin_memory().numpy()
        out_h = torch.empty((a.n, a.k), dtype=torch.float32).pin_memory().numpy()
        out_h2 = torch.empty((a.n, a.k), dtype=torch.float32).pin_memory().numpy()
        stream2 = torch.cuda.Stream(device=dev)
        ctx2 = dm.dm_create(local, stream2.cuda_stream)

        def multi_step():
            dm.dm_matmat_host_multi(ctx, ["l1", "l2sq"], Xh, Zh, outs=[out_h, out_h2])

        def two_call_step():
            # the l1 product has the longer chain (copy, sort, query): its
            # copies go first
            dm.dm_matmat_host_async(ctx, "l1", Xh, Zh, out_h)
            dm.dm_matmat_host_async(ctx2, "l2sq", Xh, Zh, out_h2)
            dm.dm_sync(ctx)
            dm.dm_sync(ctx2)

        def sequential_step():
            dm.dm_matmat_host(ctx, "l1", Xh, Zh, out_h)
            dm.dm_matmat_host(ctx, "l2sq", Xh, Zh, out_h2)

        def timed(step_fn):
            for _ in range(2):
                step_fn()
            ms_list = []
            for _ in range(min(10, max(3, a.steps // 2))):
                flush.zero_()
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record(stream)
                step_fn()
                e.record(stream)
                e.synchronize()
                ms_list.append(s.elapsed_time(e))
            return statistics.mean(ms_list)

        em = timed(multi_step)
        # the results of the timed form, checked on sampled rows
        e2e_err = {"l1": oracle.relative_error(out_h[rows], oracle.l1_rows(X, Z, rows)),
                   "l2sq": oracle.relative_error(out_h2[rows], oracle.l2sq_rows(X, Z, rows))}
        em_two = timed(two_call_step)
        em_seq = timed(sequential_step)
        e2e = {"value": units_step / (em / 1e3), "unit": UNIT, "ms_per_step": em,
               "h2d_bytes_per_step": X.nbytes + Z.nbytes,
               "d2h_bytes_per_step": out_h.nbytes + out_h2.nbytes,
               "calls": "one dm_matmat_host_multi call (l1 and squared l2 of the same X and Z)",
               "rel_err_sampled_rows": e2e_err,
               "two_calls": {"ms_per_step": em_two, "value": units_step / (em_two / 1e3),
                             "h2d_bytes_per_step": 2 * (X.nbytes + Z.nbytes),
                             "calls": "two dm_matmat_host_async calls (l1, then squared l2) on two contexts from one host thread, then dm_sync on each"},
               "sequential_ms_per_step": em_seq,
               "sequential_value": units_step / (em_seq / 1e3)}
        dm.dm_destroy(ctx2)

    cpu = None
    if not a.no_cpu and world == 1:
        cpu = cpu_baseline(a.n, a.d, a.k)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(a),
            "parallelism": "replicas" if world > 1 else "single GPU",
            "gpu_launches": launches, "launches_per_step": launches / a.steps,
            "wall_s_timed_region": t_wall,
            "parts_ms": parts, "kernels": kernels, "roofline": roofline, "l1_query_all_kernels": l1_query_all,
            "bruteforce": brute, "rel_err_sampled_rows": err, "gradient": grad, "krylov": krylov, "batch": batch, "variants": variants,
            "l1_accumulation_error": precision,
            "clocks": clk, "e2e": e2e, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
