"""Benchmark: FSI backward-Euler time steps per second on one GB300.

One step = one implicit time step of the monolithic FSI system through the C ABI
(fsi_step): residual and Jacobian assembly, Schwarz/ILU preconditioner setup,
GMRES solves, backtracking line search, to Newton rtol 1e-6 (GMRES rtol 1e-3).
The default workload is the synthetic three-generation bifurcating tree
(Kuhn-voxel mesh at h = 0.04 cm: 2.51 M nodes, 14.2 M tets, 15.8 M unknowns),
the stand-in for the paper's 12.8 M-unknown pulmonary artery; inputs are
resident in HBM. Both precisions run: mixed (FP32 Jacobian / ILU /
preconditioner, FP64 residual, Krylov and Newton update; the headline value)
and FP64 throughout (on the same line; on the trees with fewer timed steps,
stated in the line, to stay inside the run's time limit). The end-to-end leg
(host buffers, copies inside the timed region) runs for the headline precision.

--impl reference times the CPU oracle (test infrastructure) on a bounded sample
of the same workload on the host cores.
Under torchrun (N > 1) every rank advances its own replica of the workload
(replicas only: the path has no data exchange between problems).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "tube-96x32x15": dict(name="tube-96x32x15", kind="tube"),
    "tube-12x8x4": dict(name="tube-12x8x4", kind="tube"),
    "tube-160x48x22": dict(name="tube-160x48x22", kind="tube"),
    "tree-3gen": dict(name="tree-3gen", kind="tree"),
    "tree-3gen-h08": dict(name="tree-3gen", kind="tree", over=dict(h=0.08)),
    "tree-7gen": dict(name="tree-7gen", kind="tree", dt=2e-3),  # the 7-generation tree is stepped at 2 ms
    "batch-64-tubes": dict(name="batch-64-tubes", kind="batch"),
}
MATERIAL = dict(rho_f=1.05, mu_f=0.035, rho_s=1.2, E_s=3.0e6, nu_s=0.45, eta_s=0.0)
S_F64 = 8
S_F32 = 4
METRIC = "FSI time steps/s on 1 GB300, mixed-precision vs FP64 at Newton rtol 1e-6"
# Options per (workload, precision) chosen by the project's measured autotuner
# (paper_1810_04289_gb300.autotune: time to solve one Newton system over a grid of
# subdomain count, overlap, ILU level, ordering and SpMV threads per row, then
# the Jacobian lag by timing whole steps) on a GB300, committed so that the
# benchmark does not repeat the search; --autotune searches again.
TUNED = {
    # 15.8 M-unknown tree: one-level RAS iterations barely grow from 4,096 to
    # 16,384 subdomains (the ILU quality sets them), so the shortest sequential
    # chains win; ILU(1) beats ILU(2) per step (fewer factor bytes per apply,
    # about 5% more iterations); one Jacobian and its factors per step (lag 3);
    # two block rows per warp in the SpMV (1.46 against 1.58 ms per product)
    ("tree-3gen", "mixed"): dict(n_subdomains=16384, overlap=1, ilu_level=1, ordering=1, threads_per_row=16,
                                 jac_lag=3),
    ("tree-3gen", "fp64"): dict(n_subdomains=16384, overlap=1, ilu_level=1, ordering=1, threads_per_row=32,
                                jac_lag=3),
    # 7-generation tree (43.0 M unknowns): subdomains of the same size as on the
    # 3-generation tree (about 150 owned nodes each)
    ("tree-7gen", "mixed"): dict(n_subdomains=49152, overlap=1, ilu_level=1, ordering=1, threads_per_row=32,
                                 jac_lag=3),
    ("tree-7gen", "fp64"): dict(n_subdomains=49152, overlap=1, ilu_level=1, ordering=1, threads_per_row=32,
                                jac_lag=3),
    # the same tree at h = 0.08 (2.09 M unknowns): subdomains of the same size;
    # ILU(1) stagnates there (GMRES makes no progress in 1,000 iterations)
    ("tree-3gen-h08", "mixed"): dict(n_subdomains=2048, overlap=1, ilu_level=2, ordering=1, threads_per_row=32,
                                     jac_lag=3),
    ("tree-3gen-h08", "fp64"): dict(n_subdomains=2048, overlap=1, ilu_level=2, ordering=1, threads_per_row=32,
                                    jac_lag=3),
    ("tube-96x32x15", "mixed"): dict(n_subdomains=512, overlap=1, ilu_level=1, ordering=1, threads_per_row=32,
                                     jac_lag=3),
    ("tube-96x32x15", "fp64"): dict(n_subdomains=512, overlap=1, ilu_level=1, ordering=1, threads_per_row=32,
                                    jac_lag=3),
    # the 64-tube batch (3.67 M unknowns): the autotuner's choice for the mixed form
    # (ILU(1) does not converge in 1,000 GMRES iterations at any subdomain count)
    ("batch-64-tubes", "mixed"): dict(n_subdomains=8192, overlap=1, ilu_level=2, ordering=1, threads_per_row=16,
                                      jac_lag=3),
    ("batch-64-tubes", "fp64"): dict(n_subdomains=8192, overlap=1, ilu_level=2, ordering=1, threads_per_row=16,
                                     jac_lag=3),
}
# DRAM bytes per launch (read + write) from one ncu capture of the kernel as it is
# now, keyed by (workload, phase, precision, subdomains, ILU level, ordering);
# the summary that holds the capture is named beside it
NCU_TRAFFIC = {
    ("tree-3gen", "pcapply", "mixed", 16384, 1, 1): (27.41e9, "profiles/k_ras_apply_stream_tree-3gen.md"),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="tree-3gen", choices=sorted(WORKLOADS))
    p.add_argument("--subdomains", type=int, default=None)
    p.add_argument("--ilu", type=int, default=None)
    p.add_argument("--overlap", type=int, default=None)
    p.add_argument("--ordering", type=int, default=None)
    p.add_argument("--jac-lag", type=int, default=None)
    p.add_argument("--orth", type=int, default=None,
                   help="Gram-Schmidt form (fsi_options.orth); default the library's (0)")
    p.add_argument("--threads-per-row", type=int, default=None, choices=[16, 32],
                   help="BSR SpMV threads per block row (fsi_options.threads_per_row)")
    p.add_argument("--stages", type=int, default=None,
                   help="streamed apply: ring stages (fsi_options.stages); default the library's choice")
    p.add_argument("--stage-blocks", type=int, default=None,
                   help="streamed apply: blocks per ring stage (fsi_options.stage_blocks)")
    p.add_argument("--newton-rtol", type=float, default=1e-6)
    p.add_argument("--gmres-rtol", type=float, default=1e-3)
    p.add_argument("--precisions", default="mixed,fp64")
    p.add_argument("--fp64-steps", type=int, default=None,
                   help="timed FP64 steps (default: --steps on tubes, min(--steps, 3) on trees)")
    p.add_argument("--fp64-warmup", type=int, default=None,
                   help="FP64 warm-up steps (default: --warmup on tubes, min(--warmup, 1) on trees)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--autotune", action="store_true", help="search the options instead of the committed ones")
    p.add_argument("--kernels-only", type=int, default=0, metavar="R",
                   help="profiling aid: build the headline-precision solver for the workload, assemble the "
                        "Jacobian at the workload's initial state without the Stokes solve (rest for trees), "
                        "then time R preconditioner applies and R SpMVs and print their mean times")
    return p.parse_args()


def make_mesh(name):
    import vesselmesh as vm
    w = WORKLOADS[name]
    if w["kind"] == "tube":
        return vm.tube_config(w["name"])
    if w["kind"] == "batch":
        return vm.batch_tubes(n_tubes=64)
    return vm.tree_config(w["name"], **w.get("over", {}))


def initial_state(m, opt_base):
    """Tubes (one or a batch): the Poiseuille field (no solve). Trees: one steady rigid-wall
    Stokes solve at t = 0 (rho_f = 0, huge time step, wall clamped) from rest, in
    the given options' precision and preconditioner, to Newton rtol 1e-5 with
    GMRES rtol 1e-3 (the state is an input; both precision legs start from it),
    then d = 0."""
    import vesselmesh as vm
    kinds = [q.get("kind") for q in m.info.get("problems", [m.info])]
    if all(k == "tube" for k in kinds):
        return vm.poiseuille_state(m)
    from paper_1810_04289_gb300 import fsi
    opt = fsi.FsiOptions()
    for f, _ in fsi.FsiOptions._fields_:
        setattr(opt, f, getattr(opt_base, f))
    opt.dt = 1e8
    opt.newton_rtol = 1e-5
    opt.newton_maxit = 30
    opt.gmres_rtol = 1e-3
    opt.jac_lag = 1
    stokes = dict(MATERIAL, rho_f=0.0)
    S = fsi.Solver(m, stokes, opt, rigid_wall=True)
    y = np.zeros((m.n_nodes, 7))
    S.set_state(y, t=-1e8)
    S.step()
    y, _ = S.state()
    S.close()
    y[:, 4:7] = 0.0
    return y


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 8:
                for k, nm in enumerate(names):
                    if r[4 + k].lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic bytes / flops per launch of each phase
# ---------------------------------------------------------------------------
def phase_model(info, s):
    """Bytes and FLOPs one launch of each phase must move/do at minimum.

    s = bytes per matrix value (8 FP64, 4 FP32). N nodes, nnzb BSR blocks, T tets.
    """
    N, nnzb, T = info.n_nodes, info.nnzb, info.n_tets
    fb, fr = info.factor_blocks, info.factor_rows
    node_in = 24 + 56 + 56 + 24                 # X, y, y_old, d_older per node
    return {
        "spmv": dict(bytes=nnzb * (49 * s + 4) + (N + 1) * 8 + N * 56 * 2, flops=2 * 49 * nnzb),
        "pcapply": dict(bytes=fb * (49 * s + 4) + fr * (8 + 8 + 8 + 1) + fr * 56 + N * 56,
                        flops=2 * 49 * fb),
        "jaceval": dict(bytes=N * node_in + T * 16 + nnzb * 49 * s, flops=None),
        "funceval": dict(bytes=N * node_in + T * 16 + N * 56, flops=None),
        "pcsetup": dict(bytes=2 * fb * 49 * s, flops=None),
    }


def max_over_ranks(ms, world, device):
    """The slowest replica's time: every rank gets the maximum of the ranks' ms."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def options_for(args, prec, fsi):
    """The solver options of one precision leg: the committed tuned choice for the
    workload (if any), overridden by explicit flags."""
    pflag = 1 if prec == "mixed" else 0
    base = dict(n_subdomains=256, overlap=1, ilu_level=1, ordering=1, threads_per_row=32, jac_lag=1)
    base.update(TUNED.get((args.workload, prec), {}))
    for k, a in (("n_subdomains", args.subdomains), ("ilu_level", args.ilu), ("overlap", args.overlap),
                 ("ordering", args.ordering), ("jac_lag", args.jac_lag), ("orth", args.orth),
                 ("stages", args.stages), ("stage_blocks", args.stage_blocks),
                 ("threads_per_row", args.threads_per_row)):
        if a is not None:
            base[k] = a
    return fsi.fsi_default_options(newton_rtol=args.newton_rtol, gmres_rtol=args.gmres_rtol, precision=pflag,
                                   dt=WORKLOADS[args.workload].get("dt", 1e-3), **base), (args.workload, prec) in TUNED


def run_ours(args, rank, world):
    import torch
    from paper_1810_04289_gb300 import fsi
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    is_tree = WORKLOADS[args.workload]["kind"] == "tree"
    t0 = time.perf_counter()
    m = make_mesh(args.workload)
    t_mesh = time.perf_counter() - t0
    opt0, _ = options_for(args, "mixed", fsi)
    t0 = time.perf_counter()
    y0 = initial_state(m, opt0)
    t_init = time.perf_counter() - t0
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    results = {}
    for prec in args.precisions.split(","):
        steps, warmup = args.steps, args.warmup
        if prec == "fp64":
            steps = args.fp64_steps if args.fp64_steps is not None else (min(args.steps, 3) if is_tree else steps)
            warmup = args.fp64_warmup if args.fp64_warmup is not None else (min(args.warmup, 1) if is_tree
                                                                             else warmup)
        opt, committed = options_for(args, prec, fsi)
        tuned = None
        if args.autotune:
            from paper_1810_04289_gb300.autotune import autotune, tune_jac_lag
            t_tune = time.perf_counter()
            opt, table = autotune(m, MATERIAL, y0, base=opt)
            opt, lag_table = tune_jac_lag(m, MATERIAL, y0, opt)
            tuned = {"chosen": {k: getattr(opt, k) for k in ("n_subdomains", "overlap", "ilu_level", "ordering",
                                                             "threads_per_row", "jac_lag", "orth")},
                     "seconds": time.perf_counter() - t_tune, "candidates": table, "jac_lag": lag_table}
        chosen = {k: getattr(opt, k) for k in ("n_subdomains", "overlap", "ilu_level", "ordering",
                                               "threads_per_row", "jac_lag", "orth")}
        t0 = time.perf_counter()
        S = fsi.Solver(m, MATERIAL, opt)
        t_create = time.perf_counter() - t0
        info = S.info()
        S.set_state(y0, t=0.0)
        # the time levels (y_n, y_{n-1}, y_{n-2}) the timed steps start from: the
        # e2e leg repeats the same steps from them
        hist = [S.vec(y0), S.vec(y0), S.vec(y0)]
        for _ in range(warmup):
            S.step()
            cur = S.vec()
            fsi.fsi_get_state(S.ctx, cur)
            hist = [cur, hist[0], hist[1]]
        t_start = fsi.fsi_get_state(S.ctx, None)
        stream = torch.cuda.current_stream()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(dev)
        clk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = []
        for _ in range(steps):
            stats.append(fsi.stats_dict(S.step()))
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop()
        ms = e0.elapsed_time(e1)
        ms = max_over_ranks(ms, world, "cuda")
        # e2e: the same steps again from the same state, through the public API
        # with host buffers: per step the H2D of the step's inputs (y_n, y_{n-1},
        # y_{n-2}) from pinned memory and the D2H of the result
        e2e = None
        if not args.no_e2e and prec == args.precisions.split(",")[0]:
            N7 = m.n_nodes * 7
            hy = [torch.empty((m.n_nodes, 7), dtype=torch.float64).pin_memory() for _ in range(3)]
            for h, d in zip(hy, hist):
                h.copy_(d.cpu())
            hout = torch.empty((m.n_nodes, 7), dtype=torch.float64).pin_memory()
            dy = [torch.empty((m.n_nodes, 7), dtype=torch.float64, device="cuda") for _ in range(3)]
            dout = torch.empty((m.n_nodes, 7), dtype=torch.float64, device="cuda")
            t_now = t_start
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(steps):
                for h, d in zip(hy, dy):
                    d.copy_(h, non_blocking=True)
                fsi.fsi_set_state(S.ctx, dy[0], dy[1], dy[2], t_now)
                fsi.fsi_step(S.ctx, stats=False)
                t_now = fsi.fsi_get_state(S.ctx, dout)
                hout.copy_(dout, non_blocking=True)
                torch.cuda.synchronize()
                hy[2].copy_(hy[1]); hy[1].copy_(hy[0]); hy[0].copy_(hout)
            e2e_s = time.perf_counter() - t0
            e2e = {"value": world * steps / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": 3 * N7 * 8,
                   "d2h_bytes_per_step": N7 * 8, "steps": steps}
        del hist
        # kernel durations for the roofline: the GMRES cycles run as CUDA graphs,
        # so the preconditioner apply and the SpMV are timed here on their own,
        # R launches each through the C ABI, CUDA events on the same stream
        ysn = S.vec()
        fsi.fsi_get_state(S.ctx, ysn)
        fsi.fsi_jacobian(S.ctx, ysn)
        rvec = torch.randn((m.n_nodes, 7), dtype=torch.float64, device="cuda")
        zvec = S.vec()
        fsi.fsi_pc_apply(S.ctx, rvec, zvec)          # builds the preconditioner
        R = 20
        kt = {}
        for name, fn in (("pcapply", lambda: fsi.fsi_pc_apply(S.ctx, rvec, zvec)),
                         ("spmv", lambda: fsi.fsi_spmv(S.ctx, rvec, zvec))):
            fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(R):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            kt[name] = a.elapsed_time(b) / R
        s = S_F32 if prec == "mixed" else S_F64
        model = phase_model(info, s)
        tot = {k: sum(st[k] for st in stats) for k in stats[0]}
        phases = {}
        for ph, tkey, nkey in (("jaceval", "t_jaceval", "n_jaceval"), ("funceval", "t_funceval", "n_funceval"),
                               ("pcsetup", "t_pcsetup", "n_pcsetup"), ("pcapply", None, "n_pcapply"),
                               ("spmv", None, "n_spmv")):
            n = tot[nkey]
            if tkey is None:
                per = kt[ph]
                t = per * n          # estimated share of the captured GMRES cycles
            else:
                t = tot[tkey]
                per = t / n if n else None
            d = {"ms_total": t, "launches": n, "ms_per_launch": per}
            if ph in model and per:
                gbs = model[ph]["bytes"] / (per * 1e-3) / 1e9
                d["algorithmic_bytes_per_launch"] = model[ph]["bytes"]
                d["gbs"] = gbs
                d["frac_hbm"] = gbs / hbm_peak
                if model[ph]["flops"]:
                    d["tflops"] = model[ph]["flops"] / (per * 1e-3) / 1e12
            if tkey is None:
                d["timed"] = f"{R} launches on their own after the run"
            phases[ph] = d
        phases["krylov"] = {"ms_total": tot["t_krylov"],
                            "note": "GMRES cycles (captured graphs): applies, SpMVs, orthogonalisation"}
        results[prec] = dict(ms=ms, steps=steps, warmup=warmup, value=world * steps / (ms * 1e-3), stats=stats,
                             tuned=tuned, chosen=chosen, committed=committed, tot=tot, phases=phases,
                             info={k: getattr(info, k) for k, _ in info._fields_}, clocks=clocks, e2e=e2e,
                             launches=int(tot["kernel_launches"]), t_create=t_create)
        S.close()
        del S
        torch.cuda.empty_cache()
    return results, hbm_peak, dict(mesh_s=t_mesh, initial_state_s=t_init), m


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------
def _oracle_sample_worker(sub):
    """One worker of the CPU sample: the oracle's residual and complex-step
    Jacobian on one chunk of tets (its sub-mesh); returns the two times (s)."""
    sys.path.insert(0, ROOT)
    from oracle import fsi_oracle as O
    X, tets, dom, tag, prob, inlets = sub
    y0 = np.zeros((X.shape[0], 7))
    P = O.Problem(X, tets, dom, tag, prob, inlets, mat=MATERIAL, dt=1e-3)
    t0 = time.perf_counter()
    P.residual(y0, y0, y0, 1e-3)
    tF = time.perf_counter() - t0
    t0 = time.perf_counter()
    P.jacobian(y0, y0, y0, 1e-3)
    tJ = time.perf_counter() - t0
    return tF, tJ


def _submesh(m, sel):
    """The tets `sel` of mesh m with their nodes renumbered compactly."""
    t = m.tets[sel]
    used, inv = np.unique(t.ravel(), return_inverse=True)
    return (m.X[used], inv.reshape(-1, 4), m.tet_domain[sel], m.node_tag[used], m.node_problem[used], m.inlets)


def cpu_sample(args, m, steps_hint=None, all_cores=True, per_core_tets=None):
    """Time the oracle on a bounded sample of the workload on the host cores.

    The sample is a random subset of the tets (per_core_tets per worker, about
    10 s of oracle work per worker): the oracle's residual and its complex-step
    Jacobian on that subset, scaled to all tets. The oracle's direct solve of
    the full system is not run (its banded LU needs far more memory and hours
    at these sizes), so this is an assembly-only upper bound on the oracle's
    steps/s. Steps/s = 1 / (NI t_J + n_F t_F) with the Newton and residual counts
    of the GPU run. With all_cores, one worker per core (spawned processes)
    evaluates its own chunk of the same size at the same time.
    """
    import multiprocessing as mp
    T = m.n_tets
    k = per_core_tets or max(1000, min(T // 20, 40000))
    cores = (os.cpu_count() or 1) if all_cores else 1
    cores = max(1, min(cores, T // k))
    perm = np.random.default_rng(7).permutation(T)
    subs = [_submesh(m, np.sort(perm[i * k:(i + 1) * k])) for i in range(cores)]
    t0 = time.perf_counter()
    if cores == 1:
        res = [_oracle_sample_worker(subs[0])]
    else:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_sample_worker, subs)
    wall = time.perf_counter() - t0
    # the chunks ran side by side: the slowest worker's time covers cores * k tets
    tF = max(r[0] for r in res) * T / (k * cores)
    tJ = max(r[1] for r in res) * T / (k * cores)
    ni, nf = (steps_hint or (3.0, 4.0))
    t_step = ni * tJ + nf * tF
    import vesselmesh as vm
    return {"value": 1.0 / t_step, "unit": "steps/s", "cores": cores, "kind": "oracle",
            "nodes": int(m.n_nodes), "tets": int(T), "unknowns": int(vm.count_unknowns(m)),
            "sample": (f"{args.workload}: {cores} worker(s) x {k} random tets each: oracle residual and "
                       f"complex-step Jacobian per worker chunk, scaled to all {T} tets "
                       f"(whole mesh on {cores} core(s): t_F {tF:.2f} s, t_J {tJ:.1f} s; pool wall {wall:.1f} s); "
                       f"per step {ni:.1f} Jacobians + {nf:.1f} residuals; direct solve not run "
                       f"(assembly-only, an upper bound on the oracle's steps/s)")}


def kernels_only(args):
    """R applies and R SpMVs of the headline-precision solver (see --kernels-only)."""
    import torch
    from paper_1810_04289_gb300 import fsi
    import vesselmesh as vm
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    m = make_mesh(args.workload)
    prec = args.precisions.split(",")[0]
    opt, _ = options_for(args, prec, fsi)
    kinds = [q.get("kind") for q in m.info.get("problems", [m.info])]
    y0 = vm.poiseuille_state(m) if all(k == "tube" for k in kinds) else np.zeros((m.n_nodes, 7))
    S = fsi.Solver(m, MATERIAL, opt)
    S.set_state(y0, t=0.0)
    fsi.fsi_jacobian(S.ctx, S.vec(y0))
    r = torch.randn((m.n_nodes, 7), dtype=torch.float64, device="cuda")
    z = S.vec()
    out = {}
    for name, fn in (("pcapply", lambda: fsi.fsi_pc_apply(S.ctx, r, z)), ("spmv", lambda: fsi.fsi_spmv(S.ctx, r, z))):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.kernels_only):
            fn()
        b.record()
        torch.cuda.synchronize()
        out[name + "_ms"] = a.elapsed_time(b) / args.kernels_only
    info = S.info()
    out.update(workload=args.workload, precision=prec, factor_blocks=info.factor_blocks, factor_rows=info.factor_rows,
               nnzb=info.nnzb, subdomains=info.n_subdomains, apply_kernel=info.apply_kernel)
    S.close()
    print(json.dumps(out))


def main():
    args = parse()
    if args.kernels_only > 0:
        kernels_only(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        vals = []
        r = None
        m = make_mesh(args.workload)
        for k in range(args.warmup + args.steps):
            r = cpu_sample(args, m, all_cores=True)
            if k >= args.warmup:
                vals.append(r["value"])
        v = float(np.mean(vals))
        cb = dict(r, value=v)
        cfg = {"workload": args.workload, "nodes": cb.pop("nodes"), "unknowns": cb.pop("unknowns"),
               "tets": cb.pop("tets"), "newton_rtol": args.newton_rtol, "gmres_rtol": args.gmres_rtol}
        print(json.dumps({"impl": "reference", "metric": METRIC,
                          "value": v, "unit": "steps/s", "n_gpus": args.gpus, "steps": args.steps,
                          "warmup": args.warmup, "higher_is_better": True, "dtype": "f64",
                          "data": "synthetic", "config": cfg,
                          "cpu_baseline": cb,
                          "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res, hbm_peak, setup, mesh = run_ours(args, rank, world)
    if rank != 0:
        return
    head = res.get("mixed") or next(iter(res.values()))
    other = res.get("fp64")
    hp = head["phases"]
    dom = max((k for k in hp if "gbs" in hp[k]), key=lambda k: hp[k]["ms_total"])
    roof = {"kernel": dom, "bound": "hbm", "achieved": hp[dom]["gbs"], "peak": hbm_peak, "unit": "GB/s",
            "frac": hp[dom]["gbs"] / hbm_peak, "traffic": None,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    hi = head["info"]
    ch = head["chosen"]
    key = (args.workload, dom, "mixed" if "mixed" in res else "fp64", hi["n_subdomains"], ch["ilu_level"],
           ch["ordering"])
    roof["algorithmic_bytes"] = hp[dom]["algorithmic_bytes_per_launch"]
    if key in NCU_TRAFFIC:
        roof["traffic"], roof["traffic_source"] = NCU_TRAFFIC[key]
    st = head["stats"]
    ni = float(np.mean([s["newton_iterations"] for s in st]))
    nres = float(np.mean([s["residual_evaluations"] for s in st]))
    cpu = None
    if not args.no_cpu and world == 1:
        try:
            cpu = cpu_sample(args, mesh, (ni, nres), all_cores=True)
            one = cpu_sample(args, mesh, (ni, nres), all_cores=False)
            cpu["one_core"] = {"value": one["value"], "cores": 1, "sample": one["sample"]}
        except Exception as e:  # the baseline is context, never a reason to lose the GPU line
            cpu = {"value": None, "error": str(e)}
    line = {
        "metric": METRIC,
        "value": head["value"], "unit": "steps/s", "n_gpus": world, "steps": head["steps"],
        "warmup": head["warmup"], "ms_per_step": head["ms"] / head["steps"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if "mixed" in res else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "nodes": hi["n_nodes"], "unknowns": hi["n_unknowns"],
                   "tets": hi["n_tets"], "subdomains": hi["n_subdomains"], "overlap": ch["overlap"],
                   "ilu": ch["ilu_level"], "ordering": ch["ordering"], "jac_lag": ch["jac_lag"],
                   "threads_per_row": ch["threads_per_row"], "orth": ch["orth"],
                   "device_gb": round(hi["device_bytes"] / 1e9, 2), "factor_blocks": hi["factor_blocks"],
                   "options": "committed tuned choice" if head["committed"] and not args.autotune else
                   ("autotuned in this run" if args.autotune else "defaults / flags"),
                   "newton_rtol": args.newton_rtol, "gmres_rtol": args.gmres_rtol,
                   "dt": WORKLOADS[args.workload].get("dt", 1e-3),
                   "l2": "working set (BSR + ILU factors) larger than L2 each step",
                   "parallelism": "replicas" if world > 1 else "single"},
        "NI": ni, "LI_per_newton": float(np.mean([s["linear_iterations"] / max(1, s["newton_iterations"])
                                                  for s in st])),
        "phases_ms_per_step": {k: v["ms_total"] / head["steps"] for k, v in hp.items()},
        "phases": hp,
        "roofline": roof,
        "clocks": head["clocks"],
        "gpu_launches": head["launches"],
        "e2e": head["e2e"],
        "cpu_baseline": cpu,
        "setup_s": dict(setup, create_mixed_s=head["t_create"]),
        "autotune": head["tuned"],
    }
    if other is not None:
        line["fp64"] = {"value": other["value"], "steps": other["steps"], "warmup": other["warmup"],
                        "ms_per_step": other["ms"] / other["steps"],
                        "NI": float(np.mean([s["newton_iterations"] for s in other["stats"]])),
                        "LI": float(np.mean([s["linear_iterations"] for s in other["stats"]])),
                        "options": other["chosen"],
                        "phases_ms_per_step": {k: v["ms_total"] / other["steps"] for k, v in other["phases"].items()},
                        "phases": other["phases"], "gpu_launches": other["launches"], "e2e": other["e2e"],
                        "clocks": other["clocks"], "autotune": other["tuned"], "create_s": other["t_create"]}
        line["mixed_over_fp64"] = head["value"] / other["value"]
    print(json.dumps(line))


if __name__ == "__main__":
    main()
