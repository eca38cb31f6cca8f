#!/usr/bin/env python3
"""Benchmark of the dense Krylov hot path on GB300.

One step = one full solve of each system of the n = 16384 FP64 workload to
relative residual 1e-10 (x0 = 0): conjugate gradient on the SPD matrix
A = G G^T / n + 1e-3 I (cond ~ 4e3) and GMRES(50) on A = 2 I + G / (2 sqrt n),
x* ~ U[-1, 1], b = A x*.  Each A is 2 GiB of FP64, far larger than the L2
cache, so no flush is needed between steps.

  value        whole-job solves per second (device-resident inputs, CUDA events)
  e2e          the same through the C ABI with pinned HOST buffers: the copy of
               A and b to the device and of x back are inside the timed region
  roofline     the dominant kernel (the FP64 matrix-vector product, formed on the
               FP32 pipe from the FP32 pair hi + lo of A), timed with CUDA
               events on its stream as back-to-back launches of the same
               kernel and grid the solvers use; HBM-bound
  cpu_baseline the oracle (plain C, FP64) on this host's cores: one full
               solve of each of the step's two systems (about 7 s)
  accuracy     the same solves at rtol 1e-10 and at the accuracy gate
               rtol 1e-12, with FP32-pair and native FP64 products: error
               against x* and against the oracle's x (solved to the same rtol)
  small_n512   the n = 512 systems: time to 1e-10 and microseconds per
               iteration (latency-bound)

--impl reference times the oracle itself as the reference arm.
Multi-GPU: the path does not shard; every rank solves its own replica
(weak scaling, no collective on the data path).
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
sys.path.insert(0, ROOT)

METRIC = ("time-to-1e-10 residual & GEMV HBM GB/s (mixed vs FP64); served solves/s, p99")
N = 16384
SIGMA = 1e-3
RESTART = 50
RTOL = 1e-10
WORKLOAD = ("n=16384 dense FP64, x0=0, rtol 1e-10: CG on SPD GG^T/n+1e-3I (seed 0) and "
            "GMRES(50) on 2I+G/(2sqrt n) (seed 1); x*~U[-1,1], b=Ax*")


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# FP64 FMA pipe of GB300: 2 DFMA per clock per SM (measured 0.598 T DFMA/s at
# 1.98 GHz on 152 SMs); one DFMA per 8-byte element of A.
def dfma_peak_tflops(sm_mhz_max):
    return 152 * 2 * 2 * sm_mhz_max * 1e6 / 1e12


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)], stdout=self.tmp,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.split(",") for r in self.tmp.read().strip().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for k, v in zip(names, r[5:9]):
                    if "Active" in v and "Not" not in v:
                        reasons.add(k)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def fp32_issue_peak():
    """FP32 instructions per second of the whole GPU: SMs x 128 lanes x max SM clock."""
    import torch
    props = torch.cuda.get_device_properties(0)
    mhz = 2070.0
    try:
        import subprocess
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=10).stdout.split()
        mhz = float(out[0]) if out else mhz
    except Exception:
        pass
    return props.multi_processor_count * 128 * mhz * 1e6


# ---------------------------------------------------------------------------
# profile evidence for the roofline's traffic field
# ---------------------------------------------------------------------------
def gemv_source_hash():
    """Hash of the GEMV kernel's device source: k_gemv.cu up to its host-side
    section, the device helpers (ls_device.cuh, the double-single arithmetic of
    ls_ds.cuh) and the GEMV_* constants of ls_internal.h."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1511_07207_gb300", "csrc")
    with open(os.path.join(csrc, "k_gemv.cu"), "rb") as fh:
        h.update(fh.read().split(b"// ---- host side", 1)[0])
    for name in ("ls_device.cuh", "ls_ds.cuh"):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "ls_internal.h")) as fh:
        h.update("".join(l for l in fh if "GEMV_" in l).encode())
    return h.hexdigest()[:16]


def profiled_traffic(name):
    """DRAM bytes per launch recorded next to a committed ncu summary (a small
    JSON file in profiles/), if it was taken on the current kernel source
    (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            vals = json.load(f)
    except (OSError, ValueError):
        return None
    if vals.get("source_sha256_16") != gemv_source_hash():
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, TypeError, ValueError):
        return None


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------
def max_over_ranks(value, world, device):
    """The largest of the ranks' values (each rank's own time: the job ends with
    the slowest rank).  An all-reduce (MAX) over the default process group
    when world > 1, the value itself otherwise."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms_max):
    """Units all ranks processed per second over the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1e3)


def make_inputs(device):
    import torch
    from paper_1511_07207_gb300 import inputs
    A_spd = inputs.spd_matrix(N, SIGMA, seed=0, device=device)
    xs1 = torch.from_numpy(inputs.solution(N, seed=0)).to(device)
    b_spd = A_spd @ xs1
    A_ns = inputs.nonsym_matrix(N, seed=1, device=device)
    xs2 = torch.from_numpy(inputs.solution(N, seed=1)).to(device)
    b_ns = A_ns @ xs2
    torch.cuda.synchronize(device)
    return A_spd, b_spd, xs1, A_ns, b_ns, xs2


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# ---------------------------------------------------------------------------
def oracle_full_solves(A_spd, b_spd, A_ns, b_ns, rtol=RTOL):
    """Full oracle solves of the step's two systems on this host's cores: CG on
    the SPD system and GMRES(50) on the nonsymmetric one, to `rtol`.  Returns
    (solves/s, threads, seconds, the CG result, the GMRES result); the results
    carry the oracle's x and iteration counts."""
    import oracle
    nt = os.cpu_count() or 1
    t0 = time.perf_counter()
    cg = oracle.cg(A_spd, b_spd, rtol=rtol, nthreads=nt)
    t1 = time.perf_counter()
    gm = oracle.gmres(A_ns, b_ns, m=RESTART, rtol=rtol, nthreads=nt)
    t2 = time.perf_counter()
    return 2.0 / (t2 - t0), nt, t2 - t0, cg, gm


def config_dict(world=1):
    """The workload description shared by both arms."""
    return {"workload": WORKLOAD, "n": N, "restart": RESTART, "rtol": RTOL,
            "matvec": ("FP64 A as the FP32 pair hi + lo (A kept to 2^-48), double-single "
                       "accumulation, FP64 vectors and scalars"),
            "l2": "inputs larger than L2 (each A is 2 GiB)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def accuracy_runs(B, ctx, dev, A_spd, b_spd, xs1, A_ns, b_ns, xs2):
    """CG and GMRES(50) on the step's systems at rtol 1e-10 and 1e-12, with
    FP32-pair and native FP64 products: status, iterations, device time, true
    residual, error against x* and the bound kappa * true residual (kappa
    estimated from the recipe: (4 + sigma) / sigma for G G^T/n + sigma I,
    3 / 1 for 2 I + G/(2 sqrt n)).  Returns (dict, {key: host x})."""
    import torch
    out, xs_host = {}, {}
    for method, A, b, xs, kappa in (("cg", A_spd, b_spd, xs1, (4 + SIGMA) / SIGMA),
                                    ("gmres", A_ns, b_ns, xs2, 3.0)):
        fn = B.ls_cg_solve if method == "cg" else B.ls_gmres_solve
        out[method] = {"kappa_est": kappa}
        for rt in (1e-10, 1e-12):
            row = {}
            for mode, f64 in (("fp32_pair", 0), ("native_f64", 1)):
                x = torch.zeros(N, dtype=torch.float64, device=dev)
                st, inf = fn(ctx, A, b, x, B.make_opts(rtol=rt, restart=RESTART, f64_matvec=f64))
                row[mode] = {"status": B.ls_strerror(st), "iters": inf["iters"],
                             "time_ms": round(inf["time_ms"], 3), "true_rel_res": inf["true_rel_res"],
                             "rel_err_vs_xstar": rel_err(x, xs),
                             "bound_kappa_x_rel_res": kappa * inf["true_rel_res"]}
                xs_host[(method, rt, mode)] = x.cpu().numpy()
                del x
            out[method]["rtol_%g" % rt] = row
    out["gate"] = "rtol 1e-12: rel. error <= 1e-8 against x* and against the oracle's x"
    return out, xs_host


def run_small(B, ctx, dev, reps=20):
    """The n = 512 systems (seed 0): CG on G G^T/n + 0.1 I and GMRES(30) on
    2 I + G/(2 sqrt n), rtol 1e-10, device-resident; latency-bound, so the
    figures are time to solution and microseconds per iteration (best of
    `reps` solves after one warm-up).  The default path runs each solve as one
    fused kernel with A's rows in shared memory; `general` is the same solve
    on the per-step graph path (ls_opts.fused = 0), for comparison."""
    import torch
    from paper_1511_07207_gb300 import inputs
    n = 512
    out = {"n": n, "workload": "seed 0: CG on GG^T/n+0.1I, GMRES(30) on 2I+G/(2sqrt n); x*~U[-1,1], "
                               "b=Ax*, x0=0, rtol 1e-10"}
    for method, A, restart in (("cg", inputs.spd_matrix(n, 0.1, seed=0), 30),
                               ("gmres", inputs.nonsym_matrix(n, seed=0), 30)):
        xs = inputs.solution(n, seed=0)
        Ad = torch.from_numpy(A).to(dev)
        bd = torch.from_numpy(A @ xs).to(dev)
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        fn = B.ls_cg_solve if method == "cg" else B.ls_gmres_solve
        for path, fused in (("fused", 1), ("general", 0)):
            o = B.make_opts(rtol=RTOL, restart=restart, fused=fused)
            fn(ctx, Ad, bd, x, o)
            best = None
            for _ in range(reps):
                x.zero_()
                st, inf = fn(ctx, Ad, bd, x, o)
                if best is None or inf["time_ms"] < best["time_ms"]:
                    best = inf
            r = {"status": B.ls_strerror(st), "iters": best["iters"],
                 "time_to_1e-10_us": round(best["time_ms"] * 1e3, 1),
                 "us_per_iter": round(best["time_ms"] * 1e3 / max(best["iters"], 1), 2),
                 "launches": best["launches"],
                 "true_rel_res": best["true_rel_res"], "rel_err_vs_xstar": rel_err(x, xs)}
            if path == "fused":
                out[method] = r
            else:
                out[method + "_general"] = r
    return out


def rel_err(x, ref):
    """||x - ref|| / ||ref|| in FP64 on the host."""
    import numpy as np
    x = x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)
    ref = ref.cpu().numpy() if hasattr(ref, "cpu") else np.asarray(ref)
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------
def run_native(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1511_07207_gb300 import binding as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    B.load()
    ctx = B.ls_create(local, stream)

    A_spd, b_spd, xs1, A_ns, b_ns, xs2 = make_inputs(dev)
    x1 = torch.zeros(N, dtype=torch.float64, device=dev)
    x2 = torch.zeros(N, dtype=torch.float64, device=dev)
    o_cg = B.make_opts(rtol=RTOL)
    o_gm = B.make_opts(rtol=RTOL, restart=RESTART)

    def step():
        st1, i1 = B.ls_cg_solve(ctx, A_spd, b_spd, x1, o_cg)
        st2, i2 = B.ls_gmres_solve(ctx, A_ns, b_ns, x2, o_gm)
        assert st1 == B.LS_OK and st2 == B.LS_OK, (B.ls_strerror(st1), B.ls_strerror(st2))
        return i1, i2

    for _ in range(args.warmup):
        i1, i2 = step()

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    launches = 0
    infos = []
    for _ in range(args.steps):
        i1, i2 = step()
        launches += i1["launches"] + i2["launches"]
        infos.append((i1, i2))
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms, world, dev)
    ms_per_step = ms_max / args.steps
    value = whole_job_rate(2 * args.steps, world, ms_max)

    # BiCGSTAB (the paper's fastest iterative method) on the nonsymmetric
    # system, timed outside the step: time to 1e-10 and products
    x3 = torch.zeros(N, dtype=torch.float64, device=dev)
    st3, i3 = B.ls_bicgstab_solve(ctx, A_ns, b_ns, x3, B.make_opts(rtol=RTOL))
    bicgstab = {"status": B.ls_strerror(st3), "time_to_1e-10_ms": round(i3["time_ms"], 3),
                "products": i3["iters"], "true_rel_res": i3["true_rel_res"],
                "rel_err_vs_xstar": float(torch.linalg.norm(x3 - xs2) / torch.linalg.norm(xs2))}
    del x3
    peaks_hbm = load_peaks()[0]["hbm_gbs"]
    # Jacobi (the paper's stationary method) on the same nonsymmetric system:
    # its iteration matrix I - D^-1 A has spectral radius about 1/4
    x4 = torch.zeros(N, dtype=torch.float64, device=dev)
    st4, i4 = B.ls_jacobi_solve(ctx, A_ns, b_ns, x4, B.make_opts(rtol=RTOL))
    jacobi = {"status": B.ls_strerror(st4), "time_to_1e-10_ms": round(i4["time_ms"], 3),
              "products": i4["iters"], "rel_res": i4["rel_res"],
              "rel_err_vs_xstar": float(torch.linalg.norm(x4 - xs2) / torch.linalg.norm(xs2)),
              "ms_per_product": round(i4["time_ms"] / max(i4["iters"], 1), 4),
              "hbm_frac_whole_solve": round(i4["bytes_moved"] / i4["time_ms"] / 1e6 / peaks_hbm, 4)}
    del x4
    # forward Gauss-Seidel on the same system: a residual product and a
    # blocked triangular solve over the lower half of A per sweep
    x5 = torch.zeros(N, dtype=torch.float64, device=dev)
    st5, i5 = B.ls_gauss_seidel_solve(ctx, A_ns, b_ns, x5, B.make_opts(rtol=RTOL))
    gauss_seidel = {"status": B.ls_strerror(st5), "time_to_1e-10_ms": round(i5["time_ms"], 3),
                    "residual_tests": i5["iters"], "rel_res": i5["rel_res"],
                    "rel_err_vs_xstar": float(torch.linalg.norm(x5 - xs2) / torch.linalg.norm(xs2)),
                    "A_passes": round(i5["bytes_moved"] / (8.0 * N * N), 1),
                    "hbm_frac_whole_solve": round(i5["bytes_moved"] / i5["time_ms"] / 1e6 / peaks_hbm, 4)}
    del x5
    # block CG (the deflating form, the default) with 8 right-hand sides on
    # the SPD system: one block product Q = A P per step reads A once for all
    # columns
    S_BCG = 8
    from paper_1511_07207_gb300 import inputs as _inputs
    Xs8 = torch.from_numpy(_inputs.solution(N, seed=2, nrhs=S_BCG).T.copy()).to(dev)   # rows = columns of X*
    B8 = (A_spd @ Xs8.t()).t().contiguous().t()
    X8 = torch.zeros((S_BCG, N), dtype=torch.float64, device=dev).t()
    st6, i6 = B.ls_block_cg_solve(ctx, A_spd, B8, X8, B.make_opts(rtol=RTOL))
    block_cg = {"status": B.ls_strerror(st6), "rhs": S_BCG, "time_to_1e-10_ms": round(i6["time_ms"], 2),
                "block_steps": i6["iters"], "ms_per_rhs": round(i6["time_ms"] / S_BCG, 2),
                "max_true_rel_res": i6["true_rel_res"],
                "rel_err_vs_xstar": float(torch.linalg.norm(X8 - Xs8.t()) / torch.linalg.norm(Xs8)),
                "ms_per_step": round(i6["time_ms"] / max(i6["iters"], 1), 3),
                "fp32_issue_frac": round(12.0 * N * N * S_BCG / (i6["time_ms"] / max(i6["iters"], 1) * 1e-3)
                                         / fp32_issue_peak(), 4),
                "note": "block product: 12 FP32 instructions per element of A and column (double-single); "
                        "peak = 152 SMs x 128 lanes x SM max clock"}
    del X8, B8, Xs8
    # block GMRES(10) with 8 right-hand sides on the nonsymmetric system
    Xs8 = torch.from_numpy(_inputs.solution(N, seed=3, nrhs=S_BCG).T.copy()).to(dev)
    B8 = (A_ns @ Xs8.t()).t().contiguous().t()
    X8 = torch.zeros((S_BCG, N), dtype=torch.float64, device=dev).t()
    st7, i7 = B.ls_block_gmres_solve(ctx, A_ns, B8, X8, B.make_opts(rtol=RTOL, restart=10))
    block_gmres = {"status": B.ls_strerror(st7), "rhs": S_BCG, "restart": 10,
                   "time_to_1e-10_ms": round(i7["time_ms"], 2), "block_steps": i7["iters"],
                   "cycles": i7["outer_iters"], "ms_per_rhs": round(i7["time_ms"] / S_BCG, 3),
                   "max_true_rel_res": i7["true_rel_res"],
                   "rel_err_vs_xstar": float(torch.linalg.norm(X8 - Xs8.t()) / torch.linalg.norm(Xs8))}
    del X8, B8, Xs8
    # the paper's direct method (LU with partial pivoting) at n = 8192
    lu_direct = lu_measure(B, ctx, dev, 8192)
    chol_direct = chol_measure(B, ctx, dev, 8192)

    # accuracy of the timed results (checked, not assumed)
    err_cg = float(torch.linalg.norm(x1 - xs1) / torch.linalg.norm(xs1))
    err_gm = float(torch.linalg.norm(x2 - xs2) / torch.linalg.norm(xs2))
    # the same solves at rtol 1e-10 and at the accuracy gate rtol 1e-12, with
    # the default FP32-pair products and with native FP64 products; the error
    # against the oracle's x is filled in by the CPU leg below
    accuracy, acc_x = (None, {}) if args.no_accuracy else accuracy_runs(
        B, ctx, dev, A_spd, b_spd, xs1, A_ns, b_ns, xs2)
    small = run_small(B, ctx, dev) if not args.no_small else None

    # dominant kernel: the FP64 GEMV through the FP32 pair (the solvers'
    # default), same kernel/grid as inside the solves
    p = torch.from_numpy(np.random.default_rng(0).standard_normal(N)).to(dev)
    y = torch.empty(N, dtype=torch.float64, device=dev)
    pair = torch.empty((2 * N, N), dtype=torch.float32, device=dev)
    assert B.ls_split_f64(ctx, A_spd, pair) == B.LS_OK
    st, gemv_ms = B.ls_gemv_timed(ctx, B.LS_F64_PAIR, pair[:N], p, y, 30)
    assert st == B.LS_OK
    del pair
    st, native_ms = B.ls_gemv_timed(ctx, B.LS_F64, A_spd, p, y, 30)
    assert st == B.LS_OK
    peaks, peak_src = load_peaks()
    gemv_bytes = 8.0 * N * N + 16.0 * N
    gemv_gbs = gemv_bytes / (gemv_ms * 1e-3) / 1e9
    native_gbs = gemv_bytes / (native_ms * 1e-3) / 1e9
    native_tflops = 2.0 * N * N / (native_ms * 1e-3) / 1e12
    sm_max = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    alu_peak = dfma_peak_tflops(sm_max)
    traffic = profiled_traffic("gemv_pair_n16384.json")
    roofline = {"bound": "hbm", "achieved": round(gemv_gbs, 1), "peak": round(peaks["hbm_gbs"], 1),
                "unit": "GB/s", "frac": round(gemv_gbs / peaks["hbm_gbs"], 4),
                "traffic": traffic,
                "kernel": "gemv_kernel<DS,TMA> (K1: FP64 A as the FP32 pair hi + lo, double-single FMA)",
                "note": ("algorithmic bytes 8n^2 + 16n per launch (hi and lo are 4 + 4 bytes per element); "
                         "peak = %s copy bandwidth" % peak_src)}
    gemv_native = {"ms": round(native_ms, 4), "GB/s": round(native_gbs, 1),
                   "hbm_frac": round(native_gbs / peaks["hbm_gbs"], 4),
                   "dfma_frac": round(native_tflops / alu_peak, 4),
                   "note": "native FP64 FMA (f64_matvec = 1): bound by the FP64 pipe, "
                           "peak = 152 SMs x 2 DFMA/clk x 2 flop x SM max clock"}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        hA1 = torch.empty((N, N), dtype=torch.float64, pin_memory=True)
        hA1.copy_(A_spd)
        hA2 = torch.empty((N, N), dtype=torch.float64, pin_memory=True)
        hA2.copy_(A_ns)
        hb1 = b_spd.cpu().pin_memory()
        hb2 = b_ns.cpu().pin_memory()
        hx1 = torch.zeros(N, dtype=torch.float64).pin_memory()
        hx2 = torch.zeros(N, dtype=torch.float64).pin_memory()

        # the host link's rate in this run: one plain copy of the same pinned buffer
        probe_dst = torch.empty((N, N), dtype=torch.float64, device=dev)
        probe_dst.copy_(hA1, non_blocking=True)
        barrier()
        tp = time.perf_counter()
        probe_dst.copy_(hA1, non_blocking=True)
        barrier()
        h2d_gbs = 8.0 * N * N / (time.perf_counter() - tp) / 1e9
        del probe_dst
        walls = []

        def step_e2e():
            t = time.perf_counter()
            s1, i1 = B.ls_cg_solve(ctx, hA1, hb1, hx1, o_cg)
            t1 = time.perf_counter()
            s2, i2 = B.ls_gmres_solve(ctx, hA2, hb2, hx2, o_gm)
            t2 = time.perf_counter()
            assert s1 == B.LS_OK and s2 == B.LS_OK
            walls.append((t1 - t, t2 - t1, i1["time_ms"], i2["time_ms"]))

        step_e2e()
        barrier()
        walls.clear()
        t0 = time.perf_counter()
        k_e2e = max(1, min(args.steps, 3))
        for _ in range(k_e2e):
            step_e2e()
        barrier()
        te = time.perf_counter() - t0
        te_max = max_over_ranks(te, world, dev)
        e2e = {"value": round(whole_job_rate(2 * k_e2e, world, te_max * 1e3), 4), "unit": "solves/s",
               "h2d_bytes_per_step": int(2 * (8 * N * N + 8 * N)),
               "d2h_bytes_per_step": int(2 * 8 * N),
               "per_solve_ms": {"cg_wall": round(statistics.median(w[0] for w in walls) * 1e3, 2),
                                "gmres_wall": round(statistics.median(w[1] for w in walls) * 1e3, 2),
                                "cg_device": round(statistics.median(w[2] for w in walls), 2),
                                "gmres_device": round(statistics.median(w[3] for w in walls), 2)},
               "h2d_GBs_plain_copy": round(h2d_gbs, 1),
               "note": ("each call copies its A (2 GiB) from pinned host memory, solves, and copies x "
                        "back; h2d_GBs_plain_copy is one plain copy of the same buffer in this run")}

    # mixed vs FP64: n = 32768 SPD system (cond ~ 4e3), time to 1e-10 and GEMV GB/s
    mixed = None
    if not args.no_mixed:
        mixed = run_mixed_compare(B, ctx, dev, stream, args)
    batch = run_batch_compare(B, ctx, dev, args) if not args.no_batch else None
    serve = run_serve(B, ctx, dev, args) if not args.no_serve else None

    # CPU baseline: the oracle's full solves of the step's two systems (rank 0,
    # N = 1 only); the accuracy gate's oracle solves (rtol 1e-12) follow,
    # untimed, and give the error of every GPU result against the oracle's x
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        hA1, hb1 = A_spd.cpu().numpy(), b_spd.cpu().numpy()
        hA2, hb2 = A_ns.cpu().numpy(), b_ns.cpu().numpy()
        v, nt, secs, or_cg, or_gm = oracle_full_solves(hA1, hb1, hA2, hb2, rtol=RTOL)
        cpu = {"value": round(v, 6), "unit": "solves/s", "cores": nt, "kind": "oracle",
               "sample": ("one full oracle CG solve (%d iterations) + one full oracle GMRES(50) solve "
                          "(%d steps) of the same n=16384 systems to rtol 1e-10, %.1f s"
                          % (or_cg["iters"], or_gm["iters"], secs)),
               "ms_per_cg_iter": round(secs * 1e3 / (or_cg["iters"] + or_gm["iters"]), 3)}
        oracle_x = {("cg", 1e-10): or_cg, ("gmres", 1e-10): or_gm}
        if accuracy is not None:
            _, _, secs12, or_cg12, or_gm12 = oracle_full_solves(hA1, hb1, hA2, hb2, rtol=1e-12)
            oracle_x[("cg", 1e-12)] = or_cg12
            oracle_x[("gmres", 1e-12)] = or_gm12
            for (method, rt, mode), xh in acc_x.items():
                ref = oracle_x[(method, rt)]
                e = accuracy[method]["rtol_%g" % rt][mode]
                e["rel_err_vs_oracle"] = rel_err(xh, ref["x"])
                e["oracle_iters"] = ref["iters"]
            accuracy["oracle_seconds_rtol_1e-12"] = round(secs12, 2)
        del hA1, hA2

    if rank == 0:
        i1, i2 = infos[-1]
        out = {
            "metric": METRIC, "value": round(value, 4), "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_per_step, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(world),
            "time_to_1e-10_ms": {"cg": round(i1["time_ms"], 3), "gmres": round(i2["time_ms"], 3)},
            "iters": {"cg": i1["iters"], "gmres": i2["iters"]},
            "true_rel_res": {"cg": i1["true_rel_res"], "gmres": i2["true_rel_res"]},
            "rel_err_vs_xstar": {"cg": err_cg, "gmres": err_gm},
            "accuracy": accuracy,
            "small_n512": small,
            "bicgstab_nonsym": bicgstab,
            "jacobi_nonsym": jacobi,
            "gauss_seidel_nonsym": gauss_seidel,
            "block_cg_spd": block_cg,
            "block_gmres_nonsym": block_gmres,
            "lu_direct": lu_direct,
            "cholesky_direct": chol_direct,
            "gemv_f64_native": gemv_native,
            "gemv_f64": {"ms": round(gemv_ms, 4), "GB/s": round(gemv_gbs, 1),
                         "hbm_frac": round(gemv_gbs / peaks["hbm_gbs"], 4),
                         "peak_source": peak_src},
            "roofline": roofline,
            "mixed_vs_fp64": mixed,
            "batch_512": batch,
            "serve": serve,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        print(json.dumps(out))
    B.ls_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


def run_mixed_compare(B, ctx, dev, stream, args, n=32768):
    """Plain FP64 CG vs BF16 / FP8 storage + FP64 flexible CG on one SPD
    system A = G G^T / n + 1e-3 I (n = 32768, A is 8 GiB in FP64), and the
    matrix-vector product of each storage format on that A."""
    import torch
    from paper_1511_07207_gb300 import inputs
    A = inputs.spd_matrix(n, SIGMA, seed=2, device=dev)
    xs = torch.from_numpy(inputs.solution(n, seed=2)).to(dev)
    b = A @ xs
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    out = {"n": n, "workload": "SPD GG^T/n+1e-3I (seed 2), x*~U[-1,1], b=Ax*, x0=0, rtol 1e-10",
           "inner_iters": 25}
    runs = {"fp64": B.make_opts(rtol=RTOL),
            "bf16_fcg": B.make_opts(rtol=RTOL, precision=B.LS_BF16_IR),
            "fp8_fcg": B.make_opts(rtol=RTOL, precision=B.LS_FP8_IR, max_iter=60)}
    reps = max(1, min(args.steps, 3))
    for name, o in runs.items():
        st, info = B.ls_cg_solve(ctx, A, b, x, o)            # warm-up (graph build)
        t = []
        for _ in range(reps):
            x.zero_()
            st, info = B.ls_cg_solve(ctx, A, b, x, o)
            t.append(info["time_ms"])
        err = float(torch.linalg.norm(x - xs) / torch.linalg.norm(xs))
        out[name] = {"status": B.ls_strerror(st), "time_to_tol_ms": round(min(t), 3),
                     "iters": info["iters"], "outer_iters": info["outer_iters"],
                     "true_rel_res": info["true_rel_res"], "rel_err_vs_xstar": err,
                     "A_bytes_streamed": info["bytes_moved"]}
    if out["fp64"]["status"] == "converged" and out["bf16_fcg"]["status"] == "converged":
        out["speedup_bf16_vs_fp64"] = round(out["fp64"]["time_to_tol_ms"] /
                                            out["bf16_fcg"]["time_to_tol_ms"], 3)
    # accuracy gate: rtol 1e-12, error against x* and between the two solutions
    if not args.no_accuracy:
        gate, xg = {}, {}
        for name, o in (("fp64", B.make_opts(rtol=1e-12)),
                        ("bf16_fcg", B.make_opts(rtol=1e-12, precision=B.LS_BF16_IR))):
            x.zero_()
            st, info = B.ls_cg_solve(ctx, A, b, x, o)
            gate[name] = {"status": B.ls_strerror(st), "iters": info["iters"],
                          "outer_iters": info["outer_iters"], "time_ms": round(info["time_ms"], 3),
                          "true_rel_res": info["true_rel_res"],
                          "rel_err_vs_xstar": float(torch.linalg.norm(x - xs) / torch.linalg.norm(xs))}
            xg[name] = x.clone()
        gate["rel_diff_bf16_vs_fp64"] = float(torch.linalg.norm(xg["bf16_fcg"] - xg["fp64"]) /
                                              torch.linalg.norm(xg["fp64"]))
        gate["gate"] = "rtol 1e-12: rel. error <= 1e-8 against x*"
        out["accuracy_rtol_1e-12"] = gate
        del xg
    # GEMV per storage format on this A
    peaks, src = load_peaks()
    gb = {}
    xv = torch.randn(n, dtype=torch.float64, device=dev)
    yv = torch.empty(n, dtype=torch.float64, device=dev)
    st, ms = B.ls_gemv_timed(ctx, B.LS_F64, A, xv, yv, 10)
    gb["f64"] = round((8.0 * n * n + 16.0 * n) / ms / 1e6, 1)
    xf = xv.float()
    yf = torch.empty(n, dtype=torch.float32, device=dev)
    for name, dt, tdt, esz in (("bf16", B.LS_BF16_IR, torch.int16, 2),
                               ("fp8", B.LS_FP8_IR, torch.uint8, 1)):
        Q = torch.empty((n, n), dtype=tdt, device=dev)
        sc = torch.empty(n, dtype=torch.float32, device=dev) if dt == B.LS_FP8_IR else None
        B.ls_quantize(ctx, dt, A, Q, sc)
        st, ms = B.ls_gemv_timed(ctx, dt, Q, xf, yf, 20, scale=sc)
        gb[name] = round((esz * n * n + 8.0 * n + (4.0 * n if sc is not None else 0)) / ms / 1e6, 1)
        del Q
    out["gemv_GBs"] = gb
    out["gemv_hbm_frac"] = {k: round(v / peaks["hbm_gbs"], 4) for k, v in gb.items()}
    del A
    torch.cuda.empty_cache()
    return out


def run_batch_compare(B, ctx, dev, args, count=512):
    """512 independent systems, n log-uniform in [64, 2048], half SPD (CG),
    half nonsymmetric (GMRES(30)), 1..32 right-hand sides, FP64 refinement
    to 1e-10 around FP32 inner solves, in one ls_batch_solve call."""
    import numpy as np
    import torch
    from paper_1511_07207_gb300 import inputs
    specs = inputs.batch_specs(count, seed=0)
    systems, keep = [], []
    for sp in specs:
        A = sp.matrix(device=dev)
        Xs = torch.from_numpy(sp.solution()).to(dev)
        Bm = (A @ Xs).T.contiguous().T                      # column-major n x s
        X = torch.zeros_like(Bm).T.contiguous().T
        method = B.LS_METHOD_CG if sp.kind == "spd" else B.LS_METHOD_GMRES
        systems.append(B.make_system(method, A, Bm, X, B.make_opts(rtol=RTOL, restart=30)))
        keep.append((A, Bm, X, Xs))
    torch.cuda.synchronize(dev)
    reps = max(1, min(args.steps, 3))

    def timed():
        B.ls_batch_solve(ctx, systems)                       # warm-up (engine + graph set-up)
        best = None
        for _ in range(reps):
            for (_, _, X, _) in keep:
                X.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            st_, inf_ = B.ls_batch_solve(ctx, systems)
            t = (time.perf_counter() - t0, inf_[0]["time_ms"])
            if best is None or t[1] < best[0][1]:
                best = (t, inf_)
        return best

    # default tile shapes, then the autotuner's, then FP32-pipe products
    B.ls_tune_reset()
    (_, dev_default), _ = timed()
    tune_s = None
    if not args.no_tune:
        t0 = time.perf_counter()
        assert B.ls_autotune(ctx, None, 0) == B.LS_OK
        tune_s = time.perf_counter() - t0
    (wall, dev_ms), infos = timed()
    ok = sum(i["status"] == B.LS_OK for i in infos)
    cols = sum(sp.nrhs for sp in specs)
    worst_res = max(i["true_rel_res"] for i in infos)
    err = max(float(torch.linalg.norm(X - Xs) / torch.linalg.norm(Xs)) for (_, _, X, Xs) in keep)
    bytes_moved = sum(i["bytes_moved"] for i in infos)
    out = {"systems": count, "rhs_columns": cols, "n_range": [64, 2048],
           "status_ok": ok, "batch_ms_device": round(dev_ms, 3), "batch_ms_wall": round(wall * 1e3, 3),
           "tile_shapes": "autotuned" if tune_s is not None else "default",
           "autotune_s": round(tune_s, 2) if tune_s is not None else None,
           "batch_ms_device_default_shapes": round(dev_default, 3),
           "systems_per_s": round(count / (dev_ms * 1e-3), 2),
           "rhs_solves_per_s": round(cols / (dev_ms * 1e-3), 1),
           "A_bytes_streamed_GB": round(bytes_moved / 1e9, 3),
           "A_stream_GBs": round(bytes_moved / (dev_ms * 1e-3) / 1e9, 1),
           "max_true_rel_res": worst_res, "max_rel_err_vs_xstar": err,
           "inner_iters_max": max(i["iters"] for i in infos),
           "outer_iters_max": max(i["outer_iters"] for i in infos),
           "gpu_launches": infos[0]["launches"],
           "inner_products": "tcgen05 kind::tf32, three products of a TF32 head/tail split, for 9-32 "
                             "right-hand sides (where the tuner keeps them); FP32 pipe for 1-8"}
    # the same batch with every inner product on the FP32 pipe (for comparison)
    os.environ["LS_ENGINE_TC"] = "0"
    try:
        (_, dev32), infos2 = timed()
        out["batch_ms_device_fp32_pipe_products"] = round(dev32, 3)
        out["status_ok_fp32_pipe_products"] = sum(i["status"] == B.LS_OK for i in infos2)
    finally:
        del os.environ["LS_ENGINE_TC"]
    del keep, systems
    torch.cuda.empty_cache()
    return out


def run_serve(B, ctx, dev, args):
    """Poisson arrivals at 2000 requests/s; each request draws a matrix from a
    resident pool (64 SPD + 64 nonsymmetric, n log-uniform in [128, 8192]),
    asks for 1e-6 or 1e-10, with 1..8 right-hand sides; 120 GB HBM budget."""
    import threading
    import numpy as np
    import torch
    from paper_1511_07207_gb300 import inputs
    reqs, pool = inputs.serve_requests(rate=2000.0, duration=args.serve_seconds, seed=0)
    mats = [p.matrix(device=dev) for p in pool]
    key = {p.seed: i for i, p in enumerate(pool)}
    # right-hand sides B = A X* per request, prepared before the clock starts
    prepared = []
    for rq in reqs:
        A = mats[key[rq.spec.seed]]
        xs = torch.from_numpy(inputs.solution(rq.spec.n, seed=rq.spec.seed + 7, nrhs=rq.spec.nrhs)).to(dev)
        Bh = np.asfortranarray((A @ xs).cpu().numpy())
        Xh = np.zeros((rq.spec.n, rq.spec.nrhs), order="F")
        method = B.LS_METHOD_CG if rq.spec.kind == "spd" else B.LS_METHOD_GMRES
        o = B.make_opts(rtol=rq.spec.rtol, restart=30)
        prepared.append((rq.t_arrival, B.make_system(method, A, Bh, Xh, o), Bh, Xh))
    torch.cuda.synchronize(dev)
    srv = B.ls_server_start(ctx, hbm_budget_bytes=120 * (1 << 30), max_slots=args.serve_slots, merge_rhs=1,
                            step_iters=args.serve_step)
    import collections
    tickets = [None] * len(prepared)
    lat = [None] * len(prepared)
    fresh = collections.deque()
    done_evt = threading.Event()
    t_start = time.perf_counter()

    def poller():
        pending = set()
        while not done_evt.is_set() or pending or fresh:
            while fresh:
                pending.add(fresh.popleft())
            for i in list(pending):
                st, done, info = B.ls_server_poll(srv, tickets[i])
                if done:
                    lat[i] = info
                    pending.discard(i)
            time.sleep(0.0005)

    th = threading.Thread(target=poller)
    th.start()
    busy = 0
    for i, (ta, sysd, _, _) in enumerate(prepared):
        now = time.perf_counter() - t_start
        if ta > now:
            time.sleep(ta - now)
        while True:
            st, t = B.ls_server_submit(srv, sysd)
            if st != B.LS_ERR_BUSY:
                break
            busy += 1
            time.sleep(0.001)
        tickets[i] = t
        fresh.append(i)
    done_evt.set()
    th.join(timeout=600)
    t_end = time.perf_counter()
    B.ls_server_stop(srv)
    infos = [x for x in lat if x is not None]
    ms = np.array([x["time_ms"] for x in infos])
    ok = sum(x["status"] == B.LS_OK for x in infos)
    out = {"arrival_rate_per_s": 2000, "duration_s": args.serve_seconds, "requests": len(prepared),
           "completed": len(infos), "status_ok": ok,
           "solves_per_s": round(len(infos) / (t_end - t_start), 1),
           "latency_ms": {"p50": round(float(np.percentile(ms, 50)), 3),
                          "p90": round(float(np.percentile(ms, 90)), 3),
                          "p99": round(float(np.percentile(ms, 99)), 3),
                          "max": round(float(ms.max()), 3)} if len(ms) else None,
           "max_slots": args.serve_slots, "step_ticks": args.serve_step, "hbm_budget_GB": 120, "merge_rhs": 1,
           "queue_full_retries": busy,
           "max_rel_res": max((x["true_rel_res"] for x in infos), default=None),
           "pool": "64 SPD + 64 nonsymmetric matrices, n log-uniform in [128, 8192], resident on the device"}
    del mats, prepared
    torch.cuda.empty_cache()
    return out


def run_reference(args):
    """Reference arm: the oracle on this host's cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch
    dev = torch.device("cuda", 0) if torch.cuda.is_available() else None
    if dev is not None:
        A_spd, b_spd, _, A_ns, b_ns, _ = make_inputs(dev)
        A1, b1 = A_spd.cpu().numpy(), b_spd.cpu().numpy()
        A2, b2 = A_ns.cpu().numpy(), b_ns.cpu().numpy()
        del A_spd, A_ns
    else:
        from paper_1511_07207_gb300 import inputs
        A1 = inputs.spd_matrix(N, SIGMA, seed=0)
        b1 = A1 @ inputs.solution(N, seed=0)
        A2 = inputs.nonsym_matrix(N, seed=1)
        b2 = A2 @ inputs.solution(N, seed=1)
    nt = os.cpu_count() or 1
    times, iters = [], None
    for i in range(args.warmup + args.steps):
        _, nt, secs, cg, gm = oracle_full_solves(A1, b1, A2, b2, rtol=RTOL)
        if i >= args.warmup:
            times.append(secs)
        iters = (cg["iters"], gm["iters"])
    total = sum(times)
    value = 2.0 * args.steps / total
    sample = ("per step: one full oracle CG solve (%d iterations) + one full oracle GMRES(50) solve "
              "(%d steps) of the n=16384 FP64 systems to rtol 1e-10, %d threads" % (iters[0], iters[1], nt))
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "solves/s",
           "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": config_dict(int(os.environ.get("WORLD_SIZE", "1"))),
           "cpu_baseline": {"value": round(value, 6), "unit": "solves/s", "cores": nt,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_small_only(args):
    """The n = 512 latency line alone (one JSON line)."""
    import torch
    from paper_1511_07207_gb300 import binding as B
    dev = torch.device("cuda", 0)
    ctx = B.ls_create(0, torch.cuda.current_stream(dev))
    print(json.dumps({"small_n512": run_small(B, ctx, dev, reps=max(args.reps, 1))}))
    B.ls_destroy(ctx)


def run_kernel(args):
    """Kernel-only mode (used for ncu captures on small cases): time the
    y = A x kernel on a random n x n matrix of the given storage format."""
    import numpy as np
    import torch
    from paper_1511_07207_gb300 import binding as B
    dev = torch.device("cuda", 0)
    ctx = B.ls_create(0, torch.cuda.current_stream(dev))
    n = args.n
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    A64 = torch.randn((n, n), dtype=torch.float64, device=dev, generator=g)
    dt = {"f64": B.LS_F64, "pair": B.LS_F64_PAIR, "bf16": B.LS_BF16_IR, "fp8": B.LS_FP8_IR,
          "f32": B.LS_F32_IR}[args.dtype]
    scale = None
    extra = {}
    if dt == B.LS_F64_PAIR:
        A = torch.empty((2 * n, (n + 3) // 4 * 4), dtype=torch.float32, device=dev)
        assert B.ls_split_f64(ctx, A64, A[:, :n]) == B.LS_OK
        # the split itself (once per solve): 8 bytes read and 8 written per element
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        assert B.ls_split_f64(ctx, A64, A[:, :n]) == B.LS_OK
        e1.record()
        torch.cuda.synchronize()
        sms = e0.elapsed_time(e1)
        extra = {"split_ms": round(sms, 4), "split_GB/s": round(16.0 * n * n / sms / 1e6, 1)}
        del A64
        A = A[:n, :n]
        x = torch.randn(n, dtype=torch.float64, device=dev, generator=g)
        y = torch.empty(n, dtype=torch.float64, device=dev)
        esz = 8
    elif dt == B.LS_F64:
        A = A64
        x = torch.randn(n, dtype=torch.float64, device=dev, generator=g)
        y = torch.empty(n, dtype=torch.float64, device=dev)
        esz = 8
    else:
        tdt = {B.LS_BF16_IR: torch.int16, B.LS_FP8_IR: torch.uint8, B.LS_F32_IR: torch.float32}[dt]
        A = torch.empty((n, n), dtype=tdt, device=dev)
        scale = torch.empty(n, dtype=torch.float32, device=dev) if dt == B.LS_FP8_IR else None
        assert B.ls_quantize(ctx, dt, A64, A, scale) == B.LS_OK
        del A64
        x = torch.randn(n, dtype=torch.float32, device=dev, generator=g)
        y = torch.empty(n, dtype=torch.float32, device=dev)
        esz = {B.LS_BF16_IR: 2, B.LS_FP8_IR: 1, B.LS_F32_IR: 4}[dt]
    st, ms = B.ls_gemv_timed(ctx, dt, A, x, y, args.reps, scale=scale)
    assert st == B.LS_OK
    byts = esz * n * n + (8 if dt in (B.LS_F64, B.LS_F64_PAIR) else 4) * 2 * n + (4 * n if scale is not None else 0)
    peaks, src = load_peaks()
    print(json.dumps({"kernel": "gemv", "dtype": args.dtype, "n": n, "reps": args.reps,
                      "ms": round(ms, 5), "GB/s": round(byts / ms / 1e6, 1),
                      "hbm_frac": round(byts / ms / 1e6 / peaks["hbm_gbs"], 4),
                      "peak_source": src, **extra}))
    B.ls_destroy(ctx)


def run_stationary(args):
    """Jacobi or Gauss-Seidel alone (timing and ncu captures): the
    nonsymmetric bench matrix 2I + G/(2 sqrt n) at --n, one solve with one
    residual test and one with 1 + --reps; the difference is --reps sweeps
    (Jacobi: the product with its fused update; Gauss-Seidel: the residual
    product and the triangular solve)."""
    import torch
    from paper_1511_07207_gb300 import binding as B
    from paper_1511_07207_gb300 import inputs
    dev = torch.device("cuda", 0)
    ctx = B.ls_create(0, torch.cuda.current_stream(dev))
    n = args.n
    A = inputs.nonsym_matrix(n, seed=1, device=dev)
    b = A @ torch.ones(n, dtype=torch.float64, device=dev)
    solve = B.ls_jacobi_solve if args.method == "jacobi" else B.ls_gauss_seidel_solve
    times = {}
    for k in (1, 1, 1 + args.reps):     # the first solve warms the graph up
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        st, info = solve(ctx, A, b, x, B.make_opts(rtol=1e-300, max_iter=k))
        assert st == B.LS_NOT_CONVERGED and info["iters"] == k, (st, info)
        times[k] = info["time_ms"]
    sweep = (times[1 + args.reps] - times[1]) / args.reps
    byts = 8.0 * n * n + (4.0 * n * n if args.method == "gauss_seidel" else 0.0)
    peaks, src = load_peaks()
    print(json.dumps({"kernel": "stationary", "method": args.method, "n": n, "reps": args.reps,
                      "setup_and_first_test_ms": round(times[1], 4), "ms_per_sweep": round(sweep, 4),
                      "A_bytes_per_sweep": byts, "GB/s": round(byts / sweep / 1e6, 1),
                      "hbm_frac": round(byts / sweep / 1e6 / peaks["hbm_gbs"], 4), "peak_source": src}))
    B.ls_destroy(ctx)


def run_block_cg_steps(args):
    """Block CG alone (timing and ncu captures): the SPD matrix G G^T/n + 1e-3 I
    at --n with --rhs right-hand sides; one solve of one step and one of
    1 + --reps steps; the difference is --reps steps (block product Q = A P
    and the step kernels), in the deflating form (the default) and in
    O'Leary's form."""
    import torch
    from paper_1511_07207_gb300 import binding as B
    from paper_1511_07207_gb300 import inputs
    dev = torch.device("cuda", 0)
    ctx = B.ls_create(0, torch.cuda.current_stream(dev))
    n, s = args.n, args.rhs
    A = inputs.spd_matrix(n, 1e-3, seed=0, device=dev)
    Xs = torch.from_numpy(inputs.solution(n, seed=2, nrhs=s).T.copy()).to(dev)
    Bm = (A @ Xs.t()).t().contiguous().t()
    out = {"kernel": "block_cg", "n": n, "rhs": s, "reps": args.reps,
           "note": "12 FP32 operations per element of A and column (double-single)"}
    for name, deflate in (("deflating", 1), ("oleary", 0)):
        times = {}
        for k in (1, 1, 1 + args.reps):
            X = torch.zeros((s, n), dtype=torch.float64, device=dev).t()
            st, info = B.ls_block_cg_solve(ctx, A, Bm, X, B.make_opts(rtol=1e-300, max_iter=k, deflate=deflate))
            assert st == B.LS_NOT_CONVERGED and info["iters"] == k, (st, info)
            times[k] = info["time_ms"]
        step = (times[1 + args.reps] - times[1]) / args.reps
        mac = float(n) * n * s
        out[name] = {"ms_per_step": round(step, 4), "A_GB/s": round(8.0 * n * n / step / 1e6, 1),
                     "fp32_ops_per_s": round(12.0 * mac / step / 1e9, 1)}
    print(json.dumps(out))
    B.ls_destroy(ctx)


def lu_measure(B, ctx, dev, n):
    """The direct method on the nonsymmetric family 2I + G/(2 sqrt n) at n: time
    and the share of the FP64 pipe it uses (the elimination is n^3/3 updates,
    each a separate FP64 multiply and subtract, 2 n^3/3 instructions)."""
    import torch
    from paper_1511_07207_gb300 import inputs
    A = inputs.nonsym_matrix(n, seed=5, device=dev)
    xs = torch.from_numpy(inputs.solution(n, seed=5)).to(dev)
    b = A @ xs
    for _ in range(2):   # the first call sizes the workspace
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        st, info = B.ls_lu_solve(ctx, A, b, x)
    peaks, src = load_peaks()
    instr = 2.0 * n ** 3 / 3.0
    # FP64 instructions per second the pipe issues: 152 SMs x 2 per clock x SM max clock
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    dp_peak = 152 * 2 * sm_max * 1e6
    return {"status": B.ls_strerror(st), "n": n, "time_ms": round(info["time_ms"], 2),
            "fp64_instr_per_s": round(instr / (info["time_ms"] * 1e-3) / 1e12, 4),
            "fp64_issue_frac": round(instr / (info["time_ms"] * 1e-3) / dp_peak, 4),
            "true_rel_res": info["true_rel_res"],
            "rel_err_vs_xstar": float(torch.linalg.norm(x - xs) / torch.linalg.norm(xs)),
            "note": ("blocked right-looking elimination (panels of 32 columns), bit for bit the plain "
                     "elimination: 2 n^3/3 unfused FP64 multiply/subtract instructions, bound by the FP64 "
                     "pipe (peak 152 SMs x 2 per clock x SM max clock, fp64_instr_per_s in T/s)")}


def chol_measure(B, ctx, dev, n):
    """The Cholesky method on the SPD family G G^T/n + 0.1 I at n: time and the
    share of the FP64 pipe (n^3/6 updates, each a separate FP64 multiply and
    subtract: n^3/3 instructions)."""
    import torch
    from paper_1511_07207_gb300 import inputs
    A = inputs.spd_matrix(n, 0.1, seed=6, device=dev)
    xs = torch.from_numpy(inputs.solution(n, seed=6)).to(dev)
    b = A @ xs
    for _ in range(2):   # the first call sizes the workspace
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        st, info = B.ls_chol_solve(ctx, A, b, x)
    peaks, src = load_peaks()
    instr = n ** 3 / 3.0
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    dp_peak = 152 * 2 * sm_max * 1e6
    return {"status": B.ls_strerror(st), "n": n, "time_ms": round(info["time_ms"], 2),
            "fp64_instr_per_s": round(instr / (info["time_ms"] * 1e-3) / 1e12, 4),
            "fp64_issue_frac": round(instr / (info["time_ms"] * 1e-3) / dp_peak, 4),
            "true_rel_res": info["true_rel_res"],
            "rel_err_vs_xstar": float(torch.linalg.norm(x - xs) / torch.linalg.norm(xs)),
            "note": ("blocked Cholesky (panels of 32 columns, lower triangle), bit for bit the column "
                     "factorization: n^3/3 unfused FP64 multiply/subtract instructions, bound by the FP64 pipe")}


def run_lu_only(args):
    """The direct method alone (timing and ncu captures) at --n."""
    import torch
    from paper_1511_07207_gb300 import binding as B
    dev = torch.device("cuda", 0)
    ctx = B.ls_create(0, torch.cuda.current_stream(dev))
    print(json.dumps(dict(kernel="lu", **lu_measure(B, ctx, dev, args.n))))
    B.ls_destroy(ctx)


def run_batch_only(args):
    """The batched engine alone (ncu captures of its kernels): the first
    --count systems of the 512-system recipe, one ls_batch_solve."""
    import torch
    from paper_1511_07207_gb300 import binding as B
    dev = torch.device("cuda", 0)
    ctx = B.ls_create(0, torch.cuda.current_stream(dev))

    class _A:
        steps = 1
        no_tune = args.no_tune
    print(json.dumps(run_batch_compare(B, ctx, dev, _A, count=args.count)))
    B.ls_destroy(ctx)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-system batched solve")
    ap.add_argument("--no-serve", action="store_true", help="skip the served workload")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the Poisson arrival window (60 s in the full workload)")
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--serve-step", type=int, default=8)
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the n=32768 mixed-vs-FP64 comparison (its matrix takes ~1 min to form)")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the rtol 1e-10 / 1e-12 accuracy runs (both product modes)")
    ap.add_argument("--no-small", action="store_true", help="skip the n = 512 latency line")
    ap.add_argument("--no-tune", action="store_true", help="batched engine with its default tile shapes")
    ap.add_argument("--kernel", choices=["gemv", "batch", "stationary", "block_cg", "lu", "small"],
                    default=None,
                    help="kernel-only timing (small cases for ncu captures): one GEMV format, "
                         "the batched engine alone on --count systems, --reps sweeps of a "
                         "stationary method, or the n = 512 solves alone")
    ap.add_argument("--method", choices=["jacobi", "gauss_seidel"], default="gauss_seidel",
                    help="--kernel stationary: which method")
    ap.add_argument("--rhs", type=int, default=8, help="--kernel block_cg: right-hand sides")
    ap.add_argument("--count", type=int, default=128, help="--kernel batch: systems in the batch")
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--dtype", choices=["f64", "pair", "bf16", "fp8", "f32"], default="f64")
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "native":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.kernel == "gemv":
        run_kernel(args)
    elif args.kernel == "batch":
        run_batch_only(args)
    elif args.kernel == "stationary":
        run_stationary(args)
    elif args.kernel == "block_cg":
        run_block_cg_steps(args)
    elif args.kernel == "lu":
        run_lu_only(args)
    elif args.kernel == "small":
        run_small_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
