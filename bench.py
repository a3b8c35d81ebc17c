"""Benchmark: EOFA Dirac-equation solve to true residual 1e-10 on one GB300.

A step is one complete EOFA solve (H form, Eq. generic_eofa_system) of the
16^3x32, Ls=16 Moebius workload (b=1.5, c=0.5, M5=1.8, m1=0.04, m2=1.0,
m3=0.04, shift chirality +, beta=-1, antiperiodic time, random SU(3) links
exp(i 0.5 H)) with mixed-precision defect correction: FP32 inner CGNR on the
even-odd Cayley-form Schur complement, FP64 outer residual and update.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--inner f32|f16|bf16|f64]
    python bench.py --impl reference ...     # the FP64 CPU oracle, bounded sample

Prints one JSON line (rank 0).  value = seconds per solve over the whole job
(max over ranks of the timed region / solves done by all ranks); with N > 1
every rank solves its own right-hand side on its own GPU (replicas, weak
scaling).  Inputs are resident in HBM before the timed region; the solver's
working set (~1.2 GB of FP32/FP64 fields) is far larger than L2, so no flush
is needed.  e2e repeats the solve through the public API with the
right-hand side copied from pinned host memory and the solution copied back
inside the timed region.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "EOFA solve sec to r=1e-10 & dslash HBM GB/s: mixed/learned vs plain FP64 CG"
WORKLOAD = dict(name="16^3x32_Ls16", dims=(16, 16, 16, 32), Ls=16, eps=0.5, gauge_seed=1, rhs_seed=1001,
                action=dict(M5=1.8, b=1.5, c=0.5, m1=0.04, m2=1.0, m3=0.04, beta=-1.0, pm=1, t_bc=-1))
TOL = 1e-10
KERNEL_SOURCES = ["paper_1706_05843_gb300/csrc/dslash.cuh", "paper_1706_05843_gb300/csrc/common.cuh"]


def workload_desc(inner):
    w = WORKLOAD
    a = w["action"]
    return (f"EOFA H-form solve {'x'.join(map(str, w['dims']))} Ls={w['Ls']} Moebius b={a['b']} c={a['c']} "
            f"M5={a['M5']} m1={a['m1']} m2={a['m2']} m3={a['m3']} shift + beta={a['beta']}, random SU(3) "
            f"eps={w['eps']}, eo Cayley-form CGNR, {inner} inner / FP64 defect correction to r=1e-10")


def config_of(args, ws):
    """The workload of a bench line (the same for both arms)."""
    return {"workload": workload_desc(args.inner), "lattice": "16x16x16x32", "Ls": 16,
            "inner": args.inner, "tol": TOL, "parallelism": f"replicas{ws}",
            "l2": "working set > L2 (about 1.2 GB of fields); no flush"}


def kernel_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def bf16_peaks():
    """(burst, sustained) dense BF16 TFLOP/s from MEASURED_PEAKS.json, else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", d["bf16_tflops"]))
    return 1900.0, 1700.0


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# --- the multi-GPU path: independent replicas (every rank solves its own
# right-hand side; no collective touches the data path) -------------------
def replica_rhs_seed(rank):
    """Each rank draws its own right-hand side."""
    return WORKLOAD["rhs_seed"] + rank


def max_over_ranks(x, ws, device):
    """Wall time of the job: the slowest rank's timed region."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(elapsed_max, steps, ws):
    """Seconds per solve over the whole job: every rank does `steps` solves."""
    return elapsed_max / (steps * ws)


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.proc = None
        self.buf = None
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.out = open(os.devnull, "w")
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r for r in csv.reader(io.StringIO(out)) if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def ncu_traffic():
    """DRAM bytes per hop launch from the committed ncu summary, if it was
    taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "hop_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_hash") != kernel_hash():
        return None
    return d


def oracle_setup():
    """The FP64 CPU oracle on the full workload, its right-hand side, and the
    oracle's recorded CGNR iteration count to r=1e-10 (None if not recorded)."""
    import oracle
    from paper_1706_05843_gb300 import inputs as I
    oracle.build()
    w = WORKLOAD
    U = I.gauge_field(w["dims"], w["eps"], w["gauge_seed"])
    phi = I.gaussian_fermion(w["dims"], w["Ls"], w["rhs_seed"])
    o = oracle.Oracle(oracle.Action(dims=w["dims"], Ls=w["Ls"], **w["action"]), U)
    counts = os.path.join(ROOT, "oracle", "iteration_counts.json")
    n_iter = None
    if os.path.exists(counts):
        n_iter = json.load(open(counts)).get(w["name"], {}).get("iters")
    return o, phi, n_iter, oracle.num_threads()


def oracle_time(o, phi, iters):
    """Seconds per oracle CGNR iteration over a bounded run of `iters`."""
    t0 = time.perf_counter()
    _, st = o.solve_h(phi, tol=1e-300, maxit=iters)
    return (time.perf_counter() - t0) / max(st.iters, 1)


def oracle_sample(iters_per_sample):
    """Time the FP64 CPU oracle's CGNR on the full workload (bounded sample)
    and scale to seconds per solve with the oracle's recorded iteration count."""
    o, phi, n_iter, cores = oracle_setup()
    return oracle_time(o, phi, iters_per_sample), n_iter, cores


FLOPS_PER_SITE = 1520


def event_times(torch, stream, reps, fn):
    """Seconds of `reps` calls of fn, each bracketed by CUDA events on the
    solve stream; returns (times, last result)."""
    out = None
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return times, out


def _timed(torch, fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, out


def run_batched(B, I, torch, dev):
    """16 right-hand sides over uneven lattices -- 8 systems on 16^4 Ls=16
    (gauge seed 1) and 8 on 12^3x24 Ls=12 (gauge seed 2), links
    exp(i 0.5 H) -- in one eofa_solve_batched call (FP32 inner, FP64
    correction, one graph with a device-driven loop), against the same 16
    solves one after another."""
    act = dict(WORKLOAD["action"])
    groups = [((16, 16, 16, 16), 16, 1), ((12, 12, 12, 24), 12, 2)]
    solvers, rhs = [], []
    k = 0
    for dims, Ls, gseed in groups:
        U = torch.from_numpy(I.gauge_field(dims, 0.5, gseed)).to(dev)
        for _ in range(8):
            solvers.append(B.Solver(U, dims, Ls, **act))
            rhs.append(torch.from_numpy(I.gaussian_fermion(dims, Ls, 1001 + k)).to(dev))
            k += 1
        del U
    sols = [torch.empty_like(r) for r in rhs]
    opts = B.make_opts(tol=TOL, inner="f32")
    ctxs = [s.ctx for s in solvers]
    B.eofa_solve_batched(ctxs, rhs, sols, opts)  # warm-up
    t_b, st = _timed(torch, lambda: B.eofa_solve_batched(ctxs, rhs, sols, opts))
    t_s, _ = _timed(torch, lambda: [s.solve(r, out=o, tol=TOL, inner="f32") for s, r, o in zip(solvers, rhs, sols)])
    res = {"systems": len(solvers), "s_batched": t_b, "s_one_by_one": t_s, "speedup": t_s / t_b,
           "max_true_res": max(x.true_res for x in st), "inner_iters": [x.inner_iters for x in st],
           "status": [x.status for x in st]}
    for s in solvers:
        s.close()
    return res


def run_multi_rhs(B, I, torch, dev):
    """24^3x64 Ls=12, m1 = m3 = 0.0362, links exp(i 0.7 H): four right-hand
    sides with FP16 and BF16 (and FP32) inner storage, FP64 correction."""
    dims, Ls = (24, 24, 24, 64), 12
    act = dict(WORKLOAD["action"], m1=0.0362, m3=0.0362)
    U = torch.from_numpy(I.gauge_field(dims, 0.7, 1)).to(dev)
    s = B.Solver(U, dims, Ls, **act)
    del U
    out = {}
    rhs = [torch.from_numpy(I.gaussian_fermion(dims, Ls, 1001 + i)).to(dev) for i in range(4)]
    sol = torch.empty_like(rhs[0])
    for inner in ["f16", "bf16", "f32"]:
        s.solve(rhs[0], out=sol, tol=TOL, inner=inner)  # warm-up (allocation, graph)
        times, its, resid = [], [], []
        for r in rhs:
            dt, (_, st) = _timed(torch, lambda: s.solve(r, out=sol, tol=TOL, inner=inner))
            times.append(dt)
            its.append(st.inner_iters)
            resid.append(st.true_res)
        out[inner] = {"s_per_solve": statistics.mean(times), "inner_iters": its, "max_true_res": max(resid)}
    s.close()
    return out


def run_heatbath(B, I, torch, dev, solver):
    """EOFA heatbath phi = M_EOFA(m1, m2)^(-1/2) eta (Eq. eofa_heatbath) on the
    benchmark lattice: the largest eigenvalue of M_EOFA by power iteration,
    the Zolotarev approximation with relative error <= 1e-11 on
    [0.5, 1.2 lambda_max], then 2 N_p FP32-inner solves to 1e-10 without
    and with the chronological guess over the last 4 solutions of each term;
    epsilon of Eq. (heatbath_rel_err) from a further M_EOFA application; then
    the pseudofermion force at the drawn phi (two solves and the link
    kernel) with its RMS and largest Frobenius norm over links (Sec. VI
    force norms)."""
    from paper_1706_05843_gb300 import heatbath as H
    from paper_1706_05843_gb300 import rational
    a = WORKLOAD["action"]
    m1, m2 = a["m1"], a["m2"]
    eta = torch.from_numpy(I.heatbath_noise(WORKLOAD["dims"], 31)).to(dev)
    lam, _ = H.largest_eigenvalue(solver, m1, m2, eta.clone(), iters=6, tol=1e-8, inner="f32")
    r = rational.poles_for(1e-11, 0.5, 1.2 * lam)
    out = {"lambda_max": lam, "interval": [0.5, 1.2 * lam], "poles": r.poles, "approx_err": r.err}
    for fc in (0, 4):
        dt, (phi, st) = _timed(torch, lambda: solver.heatbath(eta, m1, m2, r, forecast=fc, tol=TOL, inner="f32"))
        mphi, _ = solver.apply_meofa(phi, m1, m2, tol=1e-12, inner="f32")
        out[f"forecast_{fc}"] = {"s": dt, "eps": H.heatbath_error(solver, eta, phi, mphi),
                                 "inner_iters": [x.inner_iters for x in st],
                                 "max_true_res": max(x.true_res for x in st)}
    # the pseudofermion force of S = phi^dag M_EOFA phi at the drawn phi (Eq. eofa_force)
    dt, (f, st) = _timed(torch, lambda: solver.force(phi, m1, m2, tol=TOL, inner="f32"))
    f_rms, f_max = solver.force_norms(f)
    out["force"] = {"s": dt, "inner_iters": [x.inner_iters for x in st], "F_RMS": f_rms, "F_max": f_max}
    return out


def run_gparity(B, I, torch, dev):
    """G-parity boundary conditions in x, y and z (Sec. I) on the benchmark
    lattice and action: the two-flavour system (FP32 inner, FP64
    correction, 1e-10), one warm-up solve then one timed solve."""
    w = WORKLOAD
    U = torch.from_numpy(I.gauge_field(w["dims"], w["eps"], w["gauge_seed"])).to(dev)
    s = B.Solver(U, w["dims"], w["Ls"], gparity=7, **w["action"])
    del U
    rhs = torch.from_numpy(np.stack([I.gaussian_fermion(w["dims"], w["Ls"], 1001 + i) for i in (0, 1)])).to(dev)
    sol = torch.empty_like(rhs)
    s.solve(rhs, out=sol, tol=TOL, inner="f32")
    dt, (_, st) = _timed(torch, lambda: s.solve(rhs, out=sol, tol=TOL, inner="f32"))
    s.close()
    return {"gparity_dirs": "xyz", "flavours": 2, "s_per_solve": dt, "inner_iters": st.inner_iters,
            "outer": st.outer_iters, "true_res": st.true_res, "status": st.status}


def run_learned(B, I, torch, dev):
    """Learned preconditioner: trained on 2000 (residual, error) pairs from
    16^3x32 Ls=16 solves (gauge seed 3; a further 200 pairs held out to
    measure the trained network's error on unseen pairs), used in flexible
    GCR at 32^3x64 Ls=12 (FP32 inner, FP64 correction to 1e-10), against
    plain CGNR, the untrained network and plain FP64 CG (estimated from two
    capped FP64 solves); the convolution's tensor-core rate from the forward
    passes of one application."""
    act = dict(WORKLOAD["action"])
    rng = np.random.default_rng(17)
    w0 = np.concatenate([rng.standard_normal(81 * co * ci) * np.sqrt(2.0 / (81 * ci))
                         for ci, co in [(24, 32), (32, 32), (32, 24)]]).astype(np.float32)
    dims_t, Ls_t = (16, 16, 16, 32), 16
    Ut = torch.from_numpy(I.gauge_field(dims_t, 0.5, 3)).to(dev)
    st_ = B.Solver(Ut, dims_t, Ls_t, **act)
    srcs = [torch.from_numpy(I.gaussian_fermion(dims_t, Ls_t, 5000 + i)).to(dev) for i in range(60)]
    opts = B.make_train_opts(pairs=2000, snapshot_every=8, epochs=3, batch=8, lr=1e-3, solve_tol=1e-6, holdout=200)
    t_train, (w, tst) = _timed(torch, lambda: B.eofa_train_preconditioner(st_.ctx, srcs, w0, opts))
    st_.close()
    del srcs, Ut
    dims, Ls = (32, 32, 32, 64), 12
    U = torch.from_numpy(I.gauge_field(dims, 0.5, 3)).to(dev)
    s = B.Solver(U, dims, Ls, **act)
    del U
    rhs = torch.from_numpy(I.gaussian_fermion(dims, Ls, 1001)).to(dev)
    sol = torch.empty_like(rhs)
    res = {"train": dict(tst.as_dict(), wall_s=t_train,
                         holdout_gain=(1.0 - tst.holdout_loss_final / tst.holdout_loss_init)
                         if tst.holdout_loss_init > 0 else None)}
    s.solve(rhs, out=sol, tol=TOL, inner="f32")
    dt, (_, st) = _timed(torch, lambda: s.solve(rhs, out=sol, tol=TOL, inner="f32"))
    res["cgnr"] = {"s": dt, "inner_iters": st.inner_iters, "true_res": st.true_res}
    # plain FP64 CG on the same system (about 80 s in full): two capped FP64
    # solves give the time per iteration and the fixed cost (source,
    # reconstruction, true residual); the estimate takes the mixed solve's
    # iteration count (the FP64 and FP32-inner solves of the 16^3x32 workload
    # take 632 and 638 iterations)
    s.solve(rhs, out=sol, tol=TOL, inner="f64", max_iter=16, max_outer=1, check=False)  # tunes the FP64 kinds
    t_lo, (_, s_lo) = _timed(torch, lambda: s.solve(rhs, out=sol, tol=TOL, inner="f64", max_iter=16, max_outer=1,
                                                    check=False))
    t_hi, (_, s_hi) = _timed(torch, lambda: s.solve(rhs, out=sol, tol=TOL, inner="f64", max_iter=64, max_outer=1,
                                                    check=False))
    per_it = (t_hi - t_lo) / max(1, s_hi.inner_iters - s_lo.inner_iters)
    fixed = max(0.0, t_lo - per_it * s_lo.inner_iters)
    res["fp64_cg_estimate"] = {"s": fixed + per_it * st.inner_iters, "s_per_iter": per_it, "s_fixed": fixed,
                               "iters": st.inner_iters, "timed_iters": [s_lo.inner_iters, s_hi.inner_iters]}
    for name, weights in [("trained", w), ("untrained", w0)]:
        B.eofa_set_preconditioner(s.ctx, weights)
        dt, (_, st) = _timed(torch, lambda: s.solve(rhs, out=sol, tol=TOL, inner="f32", precond=1))
        res[name] = {"s": dt, "inner_iters": st.inner_iters, "gcr_steps": st.precond_iters,
                     "fallbacks": st.precond_fallbacks, "true_res": st.true_res,
                     "net_ms": st.precond_ms, "net_applications": st.precond_iters}
        if st.precond_iters and st.precond_ms > 0:
            # executed tensor-core work of one application: 3 layers of 81 taps, 32 x 32 padded
            # channels, on every site of the full lattice and every slice
            rows = int(np.prod(dims)) * Ls
            flops = 2.0 * rows * 3 * 81 * 32 * 32
            tf = flops * st.precond_iters / (st.precond_ms * 1e-3) / 1e12
            res[name]["net_tflops"] = tf
            res[name]["net_frac_of_bf16_sustained"] = tf / bf16_peaks()[1]
        res[name]["speedup_vs_fp64_cg"] = res["fp64_cg_estimate"]["s"] / dt
    s.close()
    return res


def run_profile_net(args):
    """One forward pass of the learned preconditioner's network at 16^3x32
    with 16 slices (2,097,152 rows; three tcgen05 convolutions), after a
    warm-up pass, timed with CUDA events; prints one JSON line (the command
    the ncu captures of k_conv_tc run)."""
    import torch
    from paper_1706_05843_gb300 import binding as B
    from paper_1706_05843_gb300 import build as BLD
    torch.cuda.set_device(0)
    if not os.path.exists(B.LIB_PATH):
        BLD.build()
    B.lib()
    dims, S = (16, 16, 16, 32), 16
    rng = np.random.default_rng(17)
    w = np.concatenate([rng.standard_normal(81 * co * ci) * np.sqrt(2.0 / (81 * ci))
                        for ci, co in [(24, 32), (32, 32), (32, 24)]]).astype(np.float32)
    X, Y, Z, T = dims
    x = torch.from_numpy(rng.standard_normal((S, T, Z, Y, X, 24)).astype(np.float32)).cuda()
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    B.eofa_net_forward(w, dims, x, out, stream=stream)  # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    B.eofa_net_forward(w, dims, x, out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rows = X * Y * Z * T * S
    flops = 2.0 * rows * 3 * 81 * 32 * 32  # executed: 3 layers, 81 taps, 32 x 32 padded channels
    print(json.dumps({"profile_net": True, "rows": rows, "ms": ms, "tflops": flops / (ms * 1e-3) / 1e12,
                      "frac_of_bf16_burst": flops / (ms * 1e-3) / 1e12 / bf16_peaks()[0]}))


def run_fma_peaks(args):
    """FP64 and FP32 FMA throughput of GPU 0 (eofa_measure_fma, best of 5
    launches each, repeated for about 4 s) with nvidia-smi clock samples
    taken meanwhile; prints one JSON line."""
    import torch
    from paper_1706_05843_gb300 import binding as B
    from paper_1706_05843_gb300 import build as BLD
    torch.cuda.set_device(0)
    if not os.path.exists(B.LIB_PATH):
        BLD.build()
    B.lib()
    uuid = "GPU-" + str(torch.cuda.get_device_properties(0).uuid)
    sampler = ClockSampler(uuid)
    time.sleep(0.3)
    res = {"f64": [], "f32": []}
    t0 = time.time()
    while time.time() - t0 < 4.0:
        for k in res:
            res[k].append(B.eofa_measure_fma(k, reps=5))
    clocks = sampler.stop()
    print(json.dumps({k + "_tflops": {"best": max(v), "median": statistics.median(v), "runs": len(v)}
                      for k, v in res.items()} | {"clocks": clocks}))


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    o, phi, n_iter, cores = oracle_setup()
    per = []
    for i in range(warm + steps):
        pi = oracle_time(o, phi, args.ref_iters)
        if i >= warm:
            per.append(pi)
    per_iter = statistics.median(per)
    if n_iter is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle iteration count not recorded"}))
        return
    val = per_iter * n_iter
    sample = (f"{args.ref_iters} oracle CGNR iterations per step on the full workload, "
              f"scaled by the oracle's recorded {n_iter} iterations to r=1e-10")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "s/solve", "n_gpus": ws,
        "steps": steps, "warmup": warm, "ms_per_step": per_iter * args.ref_iters * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(args, ws),
        "solver": "FP64 CPU oracle: unpreconditioned CGNR on the full-lattice H-form system to r=1e-10",
        "cpu_baseline": {"value": val, "unit": "s/solve", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "s/solve", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1706_05843_gb300 import binding as B
    from paper_1706_05843_gb300 import build as BLD
    from paper_1706_05843_gb300 import inputs as I
    if not os.path.exists(B.LIB_PATH):
        BLD.build()
    B.lib()

    w = WORKLOAD
    U = I.gauge_field(w["dims"], w["eps"], w["gauge_seed"])
    phi = I.gaussian_fermion(w["dims"], w["Ls"], replica_rhs_seed(rank))
    solver = B.Solver(U, w["dims"], w["Ls"], **w["action"])
    rhs = torch.from_numpy(phi).to(dev)
    sol = torch.empty_like(rhs)
    stream = torch.cuda.current_stream()
    opts = dict(tol=TOL, inner=args.inner)
    if args.profile:
        _, st = solver.solve(rhs, out=sol, max_iter=16, max_outer=1, check=False, kernel_timing=True, **opts)
        torch.cuda.synchronize()
        print(json.dumps({"profile": True, "inner_iters": st.inner_iters, "status": st.status}))
        solver.close()
        return

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        solver.solve(rhs, out=sol, **opts)
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid) if rank == 0 else None
    time.sleep(0.3)
    stats = []
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        # the production path (graph-captured CG loop); the solver times a
        # sample of its hop launches with events recorded inside the graph
        _, st = solver.solve(rhs, out=sol, kernel_timing=args.host_loop, **opts)
        stats.append(st.as_dict())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    elapsed = max_over_ranks(e0.elapsed_time(e1) / 1e3, ws, dev)
    clocks = sampler.stop() if sampler else None
    value = whole_job_value(elapsed, args.steps, ws)
    ms_per_step = elapsed / args.steps * 1e3
    hop_ms = sum(s["hop_ms"] for s in stats)
    hop_bytes = sum(s["hop_bytes"] for s in stats)
    hop_n = sum(s["hop_launches"] for s in stats)
    launches = int(statistics.median([s["kernel_launches"] for s in stats]))
    tiles = [B.lib().eofa_tile_variant(solver.ctx, B.PREC[args.inner], k) for k in range(4)]

    # end to end through the public API: eofa_solve_host takes the pinned
    # host right-hand side and returns the solution in host memory; the two
    # copies run inside the call, on the timed stream
    host_rhs = torch.from_numpy(phi).pin_memory()
    host_sol = torch.empty_like(host_rhs).pin_memory()
    e2e_steps = max(3, args.steps)  # as many solves as the device-resident measurement
    solver.solve_host(host_rhs, host_sol, stream=stream, **opts)  # allocates the context's host-solve fields
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(e2e_steps):
        solver.solve_host(host_rhs, host_sol, stream=stream, **opts)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_val = whole_job_value(max_over_ranks(e0.elapsed_time(e1) / 1e3, ws, dev), e2e_steps, ws)

    # the other precisions outside the timed region: repeated solves timed
    # with CUDA events on the solve stream, median and spread
    extra = {}
    if rank == 0 and not args.quick:
        for inner in ["f64", "f32", "f16", "bf16"]:
            if inner == args.inner:
                continue
            solver.solve(rhs, out=sol, tol=TOL, inner=inner, check=False)  # tunes and captures this precision
            reps = args.cmp_reps
            times, st = event_times(torch, stream, reps,
                                    lambda: solver.solve(rhs, out=sol, tol=TOL, inner=inner, check=False)[1])
            extra[inner] = {"s_per_solve": statistics.median(times), "s_min": min(times), "s_max": max(times),
                            "repeats": reps, "true_res": st.true_res, "outer": st.outer_iters,
                            "inner_iters": st.inner_iters, "status": st.status,
                            "hop_GBps": st.hop_bytes / (st.hop_ms * 1e-3) / 1e9 if st.hop_ms else None,
                            "hop_ms_per_launch": st.hop_ms / st.hop_launches if st.hop_launches else None}

    # the dslash sweep over storage precision x CTA tile shape (cfg 2): the
    # autotuner's own launch times of every tile variant of the four inner-CG
    # hop kinds on this lattice, as algorithmic GB/s
    sweep = {}
    for name, p in B.PREC.items():
        row = {}
        for k in range(4):
            nbytes = solver.hop_bytes(p, 1 if k in (1, 3) else 0)
            cells = {}
            for v in range(4):
                ms = B.lib().eofa_tile_time(solver.ctx, p, k, v)
                if ms > 0:
                    cells[f"v{v}"] = {"us": ms * 1e3, "GBps": nbytes / (ms * 1e-3) / 1e9}
            if cells:
                row[f"kind{k}"] = dict(cells, chosen=B.lib().eofa_tile_variant(solver.ctx, p, k))
        if row:
            sweep[name] = row

    workloads = {}
    if rank == 0 and not args.quick:
        # the paper's comparison (Sec. V.B): even-odd on the unpreconditioned
        # system with the dense Ls x Ls site block, same outer loop and inner precision
        solver.solve(rhs, out=sol, tol=TOL, inner=args.inner, method=1, check=False)  # set-up and capture
        reps = max(5, args.cmp_reps)
        times, st = event_times(torch, stream, reps,
                                lambda: solver.solve(rhs, out=sol, tol=TOL, inner=args.inner, method=1,
                                                     check=False)[1])
        dt = statistics.median(times)
        cay = [s_["seconds"] for s_ in stats]
        workloads["dense_vs_cayley"] = {
            "inner": args.inner,
            "dense": {"s_per_solve": dt, "s_min": min(times), "s_max": max(times), "repeats": reps,
                      "inner_iters": st.inner_iters, "outer": st.outer_iters,
                      "true_res": st.true_res, "status": st.status,
                      "hop_GBps": st.hop_bytes / (st.hop_ms * 1e-3) / 1e9 if st.hop_ms else None},
            "cayley": {"s_per_solve": value, "repeats": args.steps, "host_s_min": min(cay), "host_s_max": max(cay),
                       "inner_iters": stats[-1]["inner_iters"], "outer": stats[-1]["outer_iters"]},
            "cayley_speedup": dt / value if value else None}
        workloads["heatbath"] = run_heatbath(B, I, torch, dev, solver)
        solver.close()
        workloads["gparity_xyz"] = run_gparity(B, I, torch, dev)
        workloads["batched_16rhs_uneven"] = run_batched(B, I, torch, dev)
        workloads["24^3x64_Ls12_4rhs"] = run_multi_rhs(B, I, torch, dev)
        if not args.no_learned:
            workloads["learned_32^3x64_Ls12"] = run_learned(B, I, torch, dev)

    if rank != 0:
        return
    main = stats[-1]
    peak, peak_kind = peaks()
    achieved = hop_bytes / (hop_ms * 1e-3) / 1e9 if hop_ms > 0 else None
    tr = ncu_traffic()
    traffic = None
    if tr is not None:
        traffic = tr.get(f"{args.inner}_bytes_per_launch")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "kernel": f"hop_kernel<{args.inner}, Ls=16> (4 kinds: Schur and Schur^dag halves)",
                "bytes_per_launch": hop_bytes / hop_n if hop_n else None,
                "launch_ms": hop_ms / hop_n if hop_n else None, "launches_timed": hop_n,
                "timing": "CUDA events recorded inside the solver's CUDA graph on the solve stream around the "
                          "four hop launches of one CG iteration per inner solve, over the timed steps",
                "tile_variants": tiles,
                "peak_kind": f"of {peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                # the same launches by their measured DRAM traffic (ncu bytes per
                # launch / CUDA-event time) and against the nominal HBM3e rate
                "dram_achieved": traffic / (hop_ms / hop_n * 1e-3) / 1e9 if traffic and hop_n and hop_ms else None,
                "frac_of_nominal_7900": achieved / 7900.0 if achieved else None}
    cpu = None
    if ws == 1 and not args.no_cpu:
        pi, n_iter, cores = oracle_sample(args.ref_iters)
        if n_iter:
            cpu = {"value": pi * n_iter, "unit": "s/solve", "cores": cores, "kind": "oracle",
                   "sample": f"{args.ref_iters} FP64 oracle CGNR iterations (unpreconditioned) on the full "
                             f"workload, {pi:.3f} s/iteration, scaled by the oracle's recorded {n_iter} "
                             f"iterations to r=1e-10"}
    f64 = extra.get("f64", {}).get("s_per_solve")
    # the FP64 hop (the plain FP64 CG comparator) against the measured FP64
    # FMA throughput: an algorithmic count of 1520 flops per 5D output site per
    # launch (1320 Wilson hop, 50 for b5 + c5 L, 150 for the s-space inverse)
    roofline_f64 = None
    if rank == 0 and not args.quick and extra.get("f64", {}).get("hop_ms_per_launch"):
        pk64 = B.eofa_measure_fma("f64", reps=5, stream=stream)
        pk32 = B.eofa_measure_fma("f32", reps=5, stream=stream)
        n5 = int(np.prod(w["dims"])) // 2 * w["Ls"]
        tf = FLOPS_PER_SITE * n5 / (extra["f64"]["hop_ms_per_launch"] * 1e-3) / 1e12
        roofline_f64 = {"bound": "alu", "kernel": "hop_kernel<double, Ls=16> (4 kinds)", "achieved": tf,
                        "peak": pk64, "unit": "TFLOP/s", "frac": tf / pk64, "flops_per_site": FLOPS_PER_SITE,
                        "peak_kind": "measured here: eofa_measure_fma FP64 (independent FMA chains, CUDA events)",
                        "fp32_fma_peak_tflops": pk32}
    line = {
        "metric": METRIC, "value": value, "unit": "s/solve", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.inner != "f64" else "f64", "data": "synthetic",
        "config": config_of(args, ws),
        "e2e": {"value": e2e_val, "unit": "s/solve", "h2d_bytes_per_step": int(host_rhs.numel() * 16),
                "d2h_bytes_per_step": int(host_sol.numel() * 16)},
        "gpu_launches": launches * args.steps,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "solve": {"true_res": main["true_res"], "outer_iters": main["outer_iters"],
                  "inner_iters": main["inner_iters"], "kernel_launches_per_solve": launches},
        "other_precisions": extra,
        "dslash_sweep": sweep,
        "roofline_f64": roofline_f64,
        "speedup_vs_fp64": (f64 / value) if f64 and ws == 1 else None,
        "speedup_vs_fp64_repeats": extra.get("f64", {}).get("repeats"),
        "other_workloads": workloads,
    }
    print(json.dumps(line))
    if args.quick:
        solver.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--inner", default="f32", choices=["f64", "f32", "f16", "bf16"])
    ap.add_argument("--ref-iters", type=int, default=4, help="oracle iterations per CPU sample")
    ap.add_argument("--quick", action="store_true", help="skip the other-precision solves")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip training the learned preconditioner and timing it at 32^3x64 Ls=12")
    ap.add_argument("--cmp-reps", type=int, default=5,
                    help="repeats of each comparison solve (other precisions, dense scheme)")
    ap.add_argument("--profile", action="store_true",
                    help="one solve capped at 16 inner iterations, nothing else (for ncu captures)")
    ap.add_argument("--host-loop", action="store_true",
                    help="timed solves with the host-driven CG loop and every hop timed (ncu launch lists: "
                         "ncu does not profile the kernels inside the solver's conditional graph nodes)")
    ap.add_argument("--profile-net", action="store_true",
                    help="only one forward pass of the learned preconditioner's network at 16^3x32, 16 slices "
                         "(for ncu captures of the tcgen05 convolution)")
    ap.add_argument("--fma-peaks", action="store_true",
                    help="only measure the FP64/FP32 FMA throughput with clock samples and print it")
    args = ap.parse_args()
    if args.fma_peaks:
        run_fma_peaks(args)
        return
    if args.profile_net:
        run_profile_net(args)
        return
    if args.profile:
        args.quick, args.no_cpu, args.steps, args.warmup, args.no_learned = True, True, 1, 0, True
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
