#!/usr/bin/env python
"""Benchmark: 2D db4 reconstructions/s to a 1e-6 relative normal-equation residual,
and the T / T^H apply bandwidth against the HBM roofline.

Workload (one step = one reconstruction, gs_solve in mixed precision from x = 0):
  db4 (p = 4), J = 8 (256 x 256 coefficients), radial sampling 256 spokes x 1024
  points (M = 262144, |xi| <= 255.75), polar cell areas as density weights, data
  y = T X* + 1% complex Gaussian noise with X* a random 10-ellipse phantom.
  Four noise draws are resident in HBM and cycled; L2 is flushed (256 MiB write)
  before every step, outside the per-step CUDA-event interval.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gs|reference]
Under torchrun (N > 1) every rank runs K independent reconstructions on its own
GPU (weak scaling); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

# more hardware work queues than CUDA's default 8, so that the batch section's 16
# solve streams do not share queues (a per-process setting, read at context creation)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "2D db4 reconstructions/s to 1e-6 rel. residual; T/T^H apply GB/s vs HBM peak"
UNIT = "reconstructions/s"
J, P_VM, SPOKES, POINTS, DR = 8, 4, 256, 1024, 0.5
NDRAWS = 4
TOL = 1e-6
WORKLOAD = ("2D db4 J=8 (256x256 coefficients), radial 256 spokes x 1024 points (M=262144), "
            "polar-cell density weights, 10-ellipse phantom + 1% complex noise, CGLS to 1e-6 "
            "relative normal-equation residual")
ORACLE_SAMPLE = 4096  # rows of T the CPU oracle applies per timed sample
# FP64 CGLS iterations of this workload (the oracle's CGLS does the same arithmetic);
# the GPU arm measures it live, the reference arm uses this recorded count.
FP64_ITERS_RECORDED = 224  # GB300, float64 CGLS on this workload (bench fp64_cgls.iterations)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks sampler
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev, self.rows, self.proc = dev, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------ workload
def workload():
    xi, mu = synth.radial_2d(SPOKES, POINTS, DR)
    g = synth.rng(1003)
    xstar = synth.ellipse_phantom(2**J, g) + 0j
    noise = [synth.complex_gaussian(xi.shape[0], synth.rng(1003 + 100 * (i + 1))) for i in range(NDRAWS)]
    return xi, mu, xstar, noise


# bytes one launch of each kernel must move (tables it streams + its input and
# output vectors; the oversampled grids are method-internal and not counted)
def kernel_bytes(name, M, N, b, m_lo=4, m_hi=8):
    """Algorithmic bytes of one launch of a per-sample 2D kernel, by the byte model
    of the method's representation: per sample the interior factors phi-hat_x,
    phi-hat_y (2 complex), the boundary factors L_x, R_x, L_y, R_y (4b complex),
    the sample value (1 complex) and xi_x, xi_y, sqrt(mu) (3 reals): 164 B in
    float32, 328 B in float64.  The oversampled grid is method-internal."""
    f32 = "<f32>" in name
    sc, sr = (8, 4) if f32 else (16, 8)
    if name.startswith("interp2d") or name.startswith("spread2d"):
        return M * (sc * (2 + 4 * b + 1) + sr * 3)
    return None


def streamed_bytes(name, M, b, m_lo=4):
    """Bytes the kernel actually streams per launch in this implementation: per
    sample the grid cell (2 int32), the precomputed float32 window values (2 x 2m)
    or float64 fractional coordinates, the interior and boundary factors and the
    sample value (more than kernel_bytes: window values replace xi)."""
    f32 = "<f32>" in name
    sc = 8 if f32 else 16
    coord = 2 * (2 * m_lo) * 4 if f32 else 2 * 8
    return M * (2 * 4 + coord + 2 * sc + 2 * (2 * b) * sc + sc)


def apply_bytes(M, N, b, f32=True):
    """Algorithmic bytes of one 2D apply (T or T^H): the coefficient vector (N^2
    complex) plus the per-sample tables of kernel_bytes."""
    sc, sr = (8, 4) if f32 else (16, 8)
    return sc * (N * N + M * (2 + 4 * b) + M) + sr * 3 * M


# ------------------------------------------------------------------ oracle baseline
def oracle_time_per_iteration(xi, mu, y, sample=ORACLE_SAMPLE, min_s=3.0):
    """Seconds per full-size CGLS iteration (one T, one T^H) of the FP64 oracle,
    measured on `sample` rows of T and scaled by M / sample (rows are independent)."""
    from oracle.operator import Basis1D, Operator2D

    M = xi.shape[0]
    idx = np.random.default_rng(7).choice(M, size=sample, replace=False)
    op = Operator2D(Basis1D(P_VM, J), xi[idx], mu[idx])
    x = np.random.default_rng(8).standard_normal(4**J) + 0j
    ys = y[idx]
    reps, t = 0, 0.0
    while reps == 0 or t < min_s:
        t0 = time.perf_counter()
        op.apply(x)
        op.adjoint(ys)
        t += time.perf_counter() - t0
        reps += 1
    return (t / reps) * (M / sample), reps


def oracle_probe(threads):
    """Oracle timings with `threads` BLAS/OpenMP threads (set by the caller's
    environment before numpy loads): full FP64 CGLS solves of the 1D
    configurations (Haar J=6 on the 128 integer frequencies, to 1e-12; db4 J=10
    on 4096 jittered samples with Voronoi weights, to TOL) and the sampled
    per-iteration time of the 2D radial workload."""
    from oracle.operator import Basis1D, Operator1D
    from oracle.solvers import cgls
    from oracle.weights import voronoi_1d

    out = {"threads": threads}
    xi, xt = synth.haar_integers()
    t0 = time.perf_counter()
    op = Operator1D(Basis1D(1, 6), xi)
    t1 = time.perf_counter()
    y = op.apply(xt)
    x, it, _ = cgls(op.apply, op.adjoint, y, tol=1e-12, maxit=1000)
    t2 = time.perf_counter()
    out["haar_J6"] = {"init_s": t1 - t0, "solve_s": t2 - t1, "iterations": it, "tol": 1e-12,
                      "max_err": float(np.max(np.abs(x - xt)))}
    g = synth.rng(1002)
    xi = synth.jitter_1d(2048, g)
    mu = voronoi_1d(xi, 2048.0)
    xs = synth.piecewise_smooth(2**10, g) + 0j
    t0 = time.perf_counter()
    op = Operator1D(Basis1D(4, 10), xi, mu)
    t1 = time.perf_counter()
    y = op.apply(xs) + 1e-3 * synth.complex_gaussian(xi.size, g) * np.sqrt(mu)
    x, it, _ = cgls(op.apply, op.adjoint, y, tol=TOL, maxit=5000)
    t2 = time.perf_counter()
    out["db4_J10_jitter"] = {"init_s": t1 - t0, "solve_s": t2 - t1, "iterations": it, "tol": TOL}
    xi2, mu2, _, noise = workload()
    tpi, reps = oracle_time_per_iteration(xi2, mu2, noise[0], min_s=2.0)
    out["radial_J8_per_iteration_s"] = tpi
    out["radial_J8_reps"] = reps
    return out


def oracle_probe_run(threads):
    """oracle_probe in a fresh interpreter with the thread count fixed in its environment."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-probe", str(threads)],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(f"oracle probe failed: {r.stderr[-500:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


# ------------------------------------------------------------------ multi-rank timing
def max_over_ranks(ms, dist=None, device="cpu"):
    """The largest of the ranks' `ms` (an all-reduce MAX; one process returns its own)."""
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, max_ms):
    """Whole-job throughput: the reconstructions of all ranks / the slowest rank's time."""
    return world * steps / (max_ms / 1e3)


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gs", choices=["gs", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--batch", type=int, default=512,
                    help="also time gs_solve_batch on this many problems of the mixed 1D/2D batch workload "
                         "(0: skip; single-GPU runs only)")
    ap.add_argument("--learned", type=int, default=512,
                    help="also train the warm-start CNN on this many method-generated pairs and time "
                         "zero / adjoint / learned starts and the learned + batched + mixed solve against "
                         "plain float64 CGLS on held-out problems (0: skip; single-GPU runs only)")
    ap.add_argument("--table1", type=int, default=1,
                    help="also time plan and solve on the five problem shapes of the paper's Table 1 (0: skip)")
    ap.add_argument("--probe-apply", type=int, default=0,
                    help="only run this many float32 T^H and T applies on the workload (for profilers)")
    ap.add_argument("--oracle-probe", type=int, default=0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_probe:
        print(json.dumps(oracle_probe(args.oracle_probe)), flush=True)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank)
    if args.probe_apply:
        return probe_apply(args.probe_apply)

    import torch
    import paper_1607_04091_gb300 as gs

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    xi, mu, xstar, noise = workload()
    M = xi.shape[0]
    dev = torch.device("cuda", local)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = gs.Plan.plan_2d(xi, P_VM, J, weights=mu)
    torch.cuda.synchronize()
    init_ms = (time.perf_counter() - t0) * 1e3
    y_clean = plan.T(torch.tensor(xstar, device=dev)).cpu().numpy()
    sig = 0.01 * np.sqrt(np.mean(np.abs(y_clean) ** 2))
    ys = [torch.tensor(y_clean + sig * nz, device=dev) for nz in noise]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def solve(y, mode=gs.GS_SOLVE_MIXED):
        x = torch.zeros(plan.ncoef, dtype=torch.complex128, device=dev)
        return x, gs.gs_solve(plan.handle, y, x, tol=TOL, mode=mode, maxit=5000)

    for i in range(args.warmup):
        solve(ys[i % NDRAWS])
    torch.cuda.synchronize()

    # ---- timed region: device time per step with CUDA events, L2 flushed before each
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos = []
    with Clocks(local) as clk:
        barrier()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record()
            _, info = solve(ys[k % NDRAWS])
            ev[k][1].record()
            infos.append(info)
        barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    value = job_value(world, args.steps, total_ms)
    iters = [i["iterations"] for i in infos]
    ok = all(i["status"] == gs.GS_OK and i["rel_normres"] <= TOL for i in infos)

    # ---- e2e through the public API from pinned host buffers
    yh = [y.cpu().pin_memory() for y in ys]
    xh = torch.empty(plan.ncoef, dtype=torch.complex128).pin_memory()
    yd = torch.empty(M, dtype=torch.complex128, device=dev)
    ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush.zero_()
        ee[k][0].record()
        yd.copy_(yh[k % NDRAWS], non_blocking=True)
        x, _ = solve(yd)
        xh.copy_(x, non_blocking=True)
        ee[k][1].record()
    barrier()
    e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ee), dist, dev)
    e2e = {"value": job_value(world, args.steps, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": M * 16,
           "d2h_bytes_per_step": plan.ncoef * 16}

    # ---- second identical pass with per-launch events: kernel shares and roofline
    gs.gs_profile(True)
    barrier()
    for k in range(args.steps):
        flush.zero_()
        solve(ys[k % NDRAWS])
    barrier()
    gs.gs_profile(False)
    prof = gs.gs_profile_report()
    launches = sum(v[0] for v in prof.values())
    b = P_VM
    ranked = sorted(prof.items(), key=lambda kv: -kv[1][1])
    prof_total = sum(v[1] for v in prof.values())
    dom = next(((k, v) for k, v in ranked if kernel_bytes(k, M, 2**J, b) is not None), ranked[0])
    name, (cnt, ms) = dom
    bytes_launch = kernel_bytes(name, M, 2**J, b)
    peak, peak_kind = measured_peaks()
    avg_s = ms / cnt / 1e3
    achieved = bytes_launch / avg_s / 1e9 if bytes_launch else None
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if os.path.exists(tfile):
        try:
            tr = json.load(open(tfile))
            ent = tr.get(name)
            import hashlib
            src = open(os.path.join(ROOT, "paper_1607_04091_gb300", "csrc", ent["source"]), "rb").read() if ent else b""
            if ent and ent.get("source_sha1") == hashlib.sha1(src).hexdigest():
                traffic = ent["dram_bytes_per_launch"]
        except Exception:
            traffic = None
    roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured" else
                "fallback 6.8 TB/s", "bytes_per_launch": bytes_launch,
                "bytes_model": "164 B per sample (float32): phi-hat x/y, 4b boundary factors, sample value, "
                               "xi x/y, sqrt(mu)",
                "streamed_bytes_per_launch": streamed_bytes(name, M, b), "avg_launch_us": avg_s * 1e6,
                "launches": cnt, "share_of_step": ms / prof_total,
                "note": "per-launch CUDA events over a second identical pass of the timed steps; tables are "
                        "L2-resident across the CGLS iterations of one reconstruction"}
    shares = {k: round(v[1] / prof_total, 4) for k, v in ranked[:12]}
    apply = apply_timings(gs, plan, flush, M, 2**J, b, peak)

    # ---- plain float64 CGLS on the same problem (what the mixed solve is measured against)
    fp64 = None
    if args.fp64_steps > 0:
        fe = []
        fit = []
        for k in range(args.fp64_steps):
            flush.zero_()
            a, bq = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            _, inf = solve(ys[k % NDRAWS], mode=gs.GS_SOLVE_FP64)
            bq.record()
            torch.cuda.synchronize()
            fe.append(a.elapsed_time(bq))
            fit.append(inf["iterations"])
        fp64 = {"value": 1e3 / np.mean(fe), "unit": UNIT, "iterations": fit, "ms_per_step": float(np.mean(fe))}

    table1 = table1_bench(dev) if args.table1 and world == 1 else None
    batch = batch_bench(args.batch, dev) if args.batch > 0 and world == 1 else None
    learned = learned_bench(plan, xi, mu, args.learned, 16, dev) if args.learned > 0 and world == 1 else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        it_ref = fp64["iterations"][0] if fp64 else int(np.median(iters))
        allc = oracle_probe_run(os.cpu_count())
        one = oracle_probe_run(1)
        tpi = allc["radial_J8_per_iteration_s"]
        cpu = {"value": 1.0 / (it_ref * tpi), "unit": UNIT, "cores": allc["threads"], "kind": "oracle",
               "sample": f"extrapolated: FP64 oracle T and T^H on {ORACLE_SAMPLE} of {M} rows "
                         f"({allc['radial_J8_reps']} reps, {allc['threads']} BLAS threads), scaled by "
                         f"M/{ORACLE_SAMPLE} and by the {it_ref} FP64 CGLS iterations of this workload",
               "single_thread_value": 1.0 / (it_ref * one["radial_J8_per_iteration_s"]),
               "full_solves": {"all_threads": {k: allc[k] for k in ("haar_J6", "db4_J10_jitter")},
                               "one_thread": {k: one[k] for k in ("haar_J6", "db4_J10_jitter")},
                               "threads": allc["threads"],
                               "note": "timed whole oracle CGLS solves (not extrapolated) of the two 1D "
                                       "configurations; init = building the dense T"}}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "solver": "mixed: f32 CG passes, f64 scalars and residual",
                   "tol": TOL, "l2": "flushed before every step (256 MiB write), outside the step interval",
                   "parallelism": f"{world} independent GPU(s)", "init_ms": init_ms},
        "iterations": iters, "converged": ok, "rel_normres": [i["rel_normres"] for i in infos],
        "outer": [i["outer"] for i in infos],
        "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline, "apply": apply, "kernel_shares": shares,
        "fp64_cgls": fp64, "batch": batch, "learned": learned, "table1": table1, "cpu_baseline": cpu,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def batch_bench(count, dev):
    """Mixed batch: half 1D (db2/db4, J 8..13, oversampling 2..4, jittered, Voronoi
    weights), half 2D (db4, J 6..8, jittered grid or spiral, unit weights); data
    T x* + 0.1% noise from the library's own float64 forward apply.  Times
    gs_solve_batch (one graph per problem, 16 streams) against the same problems
    solved one after another with gs_solve."""
    import torch
    import paper_1607_04091_gb300 as gs

    probs = synth.batch_specs(count=count, seed=4004)
    t0 = time.perf_counter()
    plans = []
    for pr in probs:
        if pr.dim == 1:
            plans.append(gs.Plan.plan_1d(pr.xi, pr.p, pr.J, bandwidth=pr.bandwidth))
        else:
            plans.append(gs.Plan.plan_2d(pr.xi, pr.p, pr.J))
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0
    g = synth.rng(4005)
    ys = []
    for pr, pl in zip(probs, plans):
        yc = pl.T(torch.tensor(pr.x_true, device=dev)).cpu().numpy()
        ys.append(torch.tensor(yc + 1e-3 * np.sqrt(np.mean(np.abs(yc) ** 2)) * synth.complex_gaussian(yc.size, g),
                               device=dev))
    xs = [torch.zeros(pl.ncoef, dtype=torch.complex128, device=dev) for pl in plans]
    handles = [pl.handle for pl in plans]
    # warm-up: the first call builds each problem's solve graph and schedules the
    # streams on a common iteration guess; the second schedules on the measured
    # iteration counts, as the timed call does
    t0 = time.perf_counter()
    gs.gs_solve_batch(handles, ys, xs, tol=TOL, maxit=5000)
    t_first = time.perf_counter() - t0
    gs.gs_solve_batch(handles, ys, xs, tol=TOL, maxit=5000)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    flush.zero_()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    infos = gs.gs_solve_batch(handles, ys, xs, tol=TOL, maxit=5000)
    b.record()
    torch.cuda.synchronize()
    t_batch = a.elapsed_time(b) / 1e3
    flush.zero_()
    torch.cuda.synchronize()
    a.record()
    for pl, y, x in zip(plans, ys, xs):
        gs.gs_solve(pl.handle, y, x, tol=TOL, maxit=5000)
    b.record()
    torch.cuda.synchronize()
    t_seq = a.elapsed_time(b) / 1e3
    ok = sum(1 for i in infos if i["status"] == gs.GS_OK and i["rel_normres"] <= TOL)
    return {"problems": count, "value": count / t_batch, "unit": "reconstructions/s", "seconds": t_batch,
            "one_at_a_time": {"value": count / t_seq, "seconds": t_seq}, "converged": ok,
            "iterations_total": int(sum(i["iterations"] for i in infos)), "init_s": init_s,
            "first_call_s": t_first, "launch": "one CUDA graph per problem, assigned to 16 streams longest-first by measured iterations",
            "workload": "mixed batch: 1D db2/db4 J 8..13 jittered + 2D db4 J 6..8 jittered/spiral, "
                        "oversampling 2..4, tol 1e-6, mixed precision"}


def learned_bench(plan, xi, mu, ntrain, ntest, dev, epochs=12, batch=8, lr=1e-3):
    """Learned warm start on the radial workload: pairs (T^H y, method solution)
    from random ellipse and tensor piecewise-smooth phantoms with 1% noise; a
    6-layer, 32-channel residual CNN trained by the library's kernels; then
    iterations and time to the 1e-6 tolerance from zero, from the adjoint
    (the untrained, identity net) and from the trained net on held-out data."""
    import torch
    import paper_1607_04091_gb300 as gs

    N = 2**J

    def problem(seed):
        g = synth.rng(5000 + seed)
        xs = (synth.ellipse_phantom(N, g) if seed % 2 == 0 else synth.tensor_phantom(N, g)) + 0j
        yc = plan.T(torch.tensor(xs, device=dev)).cpu().numpy()
        sig = 0.01 * np.sqrt(np.mean(np.abs(yc) ** 2))
        return torch.tensor(yc + sig * synth.complex_gaussian(yc.size, g), device=dev)

    t0 = time.perf_counter()
    U = torch.empty((ntrain, 2, N, N), dtype=torch.float32, device=dev)
    X = torch.empty_like(U)
    for k in range(ntrain):
        y = problem(k)
        x, _ = plan.solve(y, tol=TOL, maxit=5000)
        u, xi_ = gs.gs_cnn_pair(plan.handle, y, x)
        U[k].copy_(u[0])
        X[k].copy_(xi_[0])
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = gs.Cnn(N, N, channels=32, depth=6, max_batch=batch, seed=11)
    ident = gs.Cnn(N, N, channels=32, depth=6, max_batch=1, seed=11)
    g = np.random.default_rng(12)
    losses = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        order = g.permutation(ntrain)
        for s0 in range(0, ntrain - batch + 1, batch):
            idx = torch.tensor(order[s0:s0 + batch], device=dev)
            losses.append(net.train_step(U[idx].contiguous(), X[idx].contiguous(), lr=lr))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    res = {"zero": [], "adjoint": [], "learned": []}
    used = 0
    for k in range(ntest):
        y = problem(100000 + k)
        for key in res:
            x = torch.zeros(plan.ncoef, dtype=torch.complex128, device=dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            if key == "zero":
                info = gs.gs_solve(plan.handle, y, x, tol=TOL, maxit=5000)
            else:
                info, u = gs.gs_solve_learned(plan.handle, ident if key == "adjoint" else net, y, x, tol=TOL,
                                              maxit=5000)
                used += int(u and key == "learned")
            b.record()
            torch.cuda.synchronize()
            res[key].append((info["iterations"], a.elapsed_time(b), info["rel_normres"]))
    summ = {k: {"iterations": float(np.mean([r[0] for r in v])), "ms": float(np.mean([r[1] for r in v])),
                "max_rel_normres": float(max(r[2] for r in v))} for k, v in res.items()}
    # the headline comparison on the same held-out problems: learned start +
    # batched (one graph, one plan per problem) + mixed precision, against plain
    # float64 CGLS from zero one problem at a time
    tests = [problem(100000 + k) for k in range(ntest)]
    bplans = [gs.Plan.plan_2d(xi, P_VM, J, weights=mu) for _ in range(ntest)]
    bh = [p.handle for p in bplans]
    bx = [torch.zeros(plan.ncoef, dtype=torch.complex128, device=dev) for _ in range(ntest)]
    for _ in range(2):  # graph builds, then the schedule from measured iterations
        gs.gs_solve_batch_learned(bh, net, tests, bx, tol=TOL, maxit=5000)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    binf = gs.gs_solve_batch_learned(bh, net, tests, bx, tol=TOL, maxit=5000)
    b.record()
    torch.cuda.synchronize()
    t_lbm = a.elapsed_time(b) / ntest
    nf = 4
    t64 = []
    for k in range(nf):
        x = torch.zeros(plan.ncoef, dtype=torch.complex128, device=dev)
        a.record()
        gs.gs_solve(plan.handle, tests[k], x, tol=TOL, maxit=5000, mode=gs.GS_SOLVE_FP64)
        b.record()
        torch.cuda.synchronize()
        t64.append(a.elapsed_time(b))
    del bplans
    versus = {"learned_batched_mixed_ms_per_problem": t_lbm, "fp64_cgls_ms_per_problem": float(np.mean(t64)),
             "speedup": float(np.mean(t64)) / t_lbm, "problems": ntest, "fp64_problems": nf,
             "converged": sum(1 for i in binf if i["status"] == gs.GS_OK and i["rel_normres"] <= TOL),
             "note": "gs_solve_batch_learned on the held-out problems (one graph) vs gs_solve float64 CGLS "
                     "from zero on the first fp64_problems of them"}
    return {"train_pairs": ntrain, "test_problems": ntest, "epochs": epochs, "batch": batch,
            "loss_first": losses[0], "loss_last": float(np.mean(losses[-max(1, ntrain // batch):])),
            "data_s": t_data, "train_s": t_train, "warm_start_used": used, **summ, "vs_fp64_cgls": versus,
            "net": "6 conv3x3 layers 2-32-32-32-32-32-2, ReLU, residual, bf16 inference weights"}


# Table 1 of the paper (Sec. 6.3): its GeneralizedSampling (Julia) timings on a
# 2.6 GHz laptop, for context: (init s, sol s, iterations).  All db4.
TABLE1 = [
    ("Uniform 1D", "8192x4096", (0.34, 0.04, 12)),
    ("Jitter 1D", "5463x2048", (0.23, 0.08, 20)),
    ("Uniform 2D", "512^2x256^2", (0.15, 17.6, 16)),
    ("Jitter 2D", "26244x32^2", (2.4, 2.4, 18)),
    ("Spiral", "27681x32^2", (2.8, 2.2, 16)),
]


def table1_problem(name):
    """Synthetic stand-ins of Table 1's sampling patterns at its sizes (the paper
    does not give its jitter or spiral parameters): (dims, p, J, xi, bandwidth)."""
    g = synth.rng(6001)
    if name == "Uniform 1D":
        return 1, 4, 12, synth.grid_1d(8192, 0.5), 0.0
    if name == "Jitter 1D":
        xi = synth.jitter_grid_1d(5463, 0.75, g)
        return 1, 4, 11, xi, float(np.ceil(np.abs(xi).max()))
    if name == "Uniform 2D":
        return 2, 4, 8, synth.uniform_2d(512, 0.5), 0.0
    if name == "Jitter 2D":
        return 2, 4, 5, synth.jitter_grid_2d(162, 0.5, g), 0.0
    return 2, 4, 5, synth.spiral_2d(27681, 0.5), 0.0


def table1_bench(dev, reps=3):
    """Each Table 1 shape: plan time (the paper's "init"), the mixed-precision solve
    to TOL and the float64 CGLS to TOL (the paper's "sol"), with iterations and time
    per iteration; data T x* + 1% noise, x* piecewise smooth (1D) or 10 ellipses (2D)."""
    import torch
    import paper_1607_04091_gb300 as gs

    out = []
    for name, size, paper in TABLE1:
        dims, p, Jt, xi, bw = table1_problem(name)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan = (gs.Plan.plan_1d(xi, p, Jt, bandwidth=bw) if dims == 1 else gs.Plan.plan_2d(xi, p, Jt))
        torch.cuda.synchronize()
        init_ms = (time.perf_counter() - t0) * 1e3
        g = synth.rng(6002)
        N = 2**Jt
        xs = (synth.piecewise_smooth(N, g) if dims == 1 else synth.ellipse_phantom(N, g)) + 0j
        yc = plan.T(torch.tensor(xs, device=dev)).cpu().numpy()
        y = torch.tensor(yc + 0.01 * np.sqrt(np.mean(np.abs(yc) ** 2)) * synth.complex_gaussian(yc.size, g),
                         device=dev)
        res = {}
        for mode, key, nrep in [(gs.GS_SOLVE_MIXED, "mixed", reps), (gs.GS_SOLVE_FP64, "fp64", 1)]:
            x = torch.zeros(plan.ncoef, dtype=torch.complex128, device=dev)
            gs.gs_solve(plan.handle, y, x, tol=TOL, maxit=5000, mode=mode)  # warm-up (graph build)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ms, it = [], []
            for _ in range(nrep):
                x.zero_()
                a.record()
                info = gs.gs_solve(plan.handle, y, x, tol=TOL, maxit=5000, mode=mode)
                b.record()
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
                it.append(info["iterations"])
            res[key] = {"ms": float(np.median(ms)), "iterations": int(np.median(it)),
                        "ms_per_iteration": float(np.median(ms)) / max(1, int(np.median(it))),
                        "rel_normres": info["rel_normres"], "status": info["status"]}
        out.append({"problem": name, "size": size, "M": int(xi.shape[0]), "J": Jt,
                    "path": "exact lattice FFT" if np.all(2 * xi == np.rint(2 * xi)) else "NFFT",
                    "init_ms": init_ms, **res,
                    "paper_julia_laptop": {"init_s": paper[0], "sol_s": paper[1], "iterations": paper[2]}})
        del plan
    return out


def apply_timings(gs, plan, flush, M, N, b, peak, reps=20):
    """float32 T and T^H applies through the public API (caller's sample order):
    warm = `reps` back-to-back applies, cold = L2 flushed before each (median);
    GB/s of the apply's algorithmic bytes (apply_bytes)."""
    import torch

    g = np.random.default_rng(0)
    y = torch.tensor(g.standard_normal(M) + 1j * g.standard_normal(M), dtype=torch.complex64, device="cuda")
    x = torch.tensor(g.standard_normal(plan.ncoef) + 1j * g.standard_normal(plan.ncoef), dtype=torch.complex64,
                     device="cuda")
    z, q = torch.empty_like(x), torch.empty_like(y)
    fns = {"T": lambda: gs.gs_apply_T(plan.handle, gs.GS_FP32, x, q),
           "TH": lambda: gs.gs_apply_TH(plan.handle, gs.GS_FP32, y, z)}
    B = apply_bytes(M, N, b)
    out = {"bytes_per_apply": B, "unit": "GB/s", "peak": peak,
           "note": "float32 applies, user sample order; warm: back to back, cold: L2 flushed before each"}
    for name, fn in fns.items():
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        warm_us = e0.elapsed_time(e1) * 1e3 / reps
        cold = []
        for _ in range(reps):
            flush.zero_()
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            cold.append(e0.elapsed_time(e1) * 1e3)
        cold_us = float(np.median(cold))
        out[name] = {"warm_us": warm_us, "cold_us": cold_us, "warm_gbs": B / warm_us / 1e3,
                     "cold_gbs": B / cold_us / 1e3, "warm_frac": B / warm_us / 1e3 / peak,
                     "cold_frac": B / cold_us / 1e3 / peak}
    return out


def probe_apply(reps):
    """float32 T^H then T on the workload's plan, `reps` times; CUDA-event timings."""
    import torch
    import paper_1607_04091_gb300 as gs

    xi, mu, _, _ = workload()
    plan = gs.Plan.plan_2d(xi, P_VM, J, weights=mu)
    g = np.random.default_rng(0)
    y = torch.tensor(g.standard_normal(plan.M) + 1j * g.standard_normal(plan.M), dtype=torch.complex64, device="cuda")
    x = torch.tensor(g.standard_normal(plan.ncoef) + 1j * g.standard_normal(plan.ncoef), dtype=torch.complex64,
                     device="cuda")
    z, q = torch.empty_like(x), torch.empty_like(y)
    for r in range(reps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        gs.gs_apply_TH(plan.handle, gs.GS_FP32, y, z)
        e[1].record()
        gs.gs_apply_T(plan.handle, gs.GS_FP32, x, q)
        e[2].record()
        torch.cuda.synchronize()
        log(f"apply {r}: T^H {e[0].elapsed_time(e[1]) * 1e3:.1f} us, T {e[1].elapsed_time(e[2]) * 1e3:.1f} us")


def reference_arm(args, rank):
    """The FP64 CPU oracle on the same workload, bounded samples per step."""
    if rank != 0:
        return
    xi, mu, xstar, noise = workload()
    it_ref = FP64_ITERS_RECORDED
    y = np.zeros(xi.shape[0], dtype=np.complex128)
    for _ in range(max(0, args.warmup)):  # untimed: one sampled T and T^H each
        oracle_time_per_iteration(xi, mu, y, min_s=0.0)
    times = []
    for k in range(args.steps):
        tpi, reps = oracle_time_per_iteration(xi, mu, y, min_s=1.0)
        times.append(tpi * it_ref)
    value = 1.0 / float(np.mean(times))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"extrapolated, each step: FP64 oracle T and T^H on {ORACLE_SAMPLE} of "
                                       f"{xi.shape[0]} rows, scaled by M/{ORACLE_SAMPLE} and by {it_ref} CGLS "
                                       f"iterations (numpy's default BLAS threads)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
