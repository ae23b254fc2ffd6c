"""Benchmark: FSI backward-Euler time steps per second on one GB300.

One step = one implicit time step of the monolithic FSI system through the C ABI
(fsi_step): residual and Jacobian assembly, Schwarz/ILU preconditioner setup,
GMRES solves, backtracking line search, to Newton rtol 1e-6 (GMRES rtol 1e-3).
The workload is a synthetic straight compliant tube (96 axial x 32 around x
(12 fluid + 3 wall) radial cells, 46,657 nodes, 289,351 unknowns), inputs
resident in HBM. Both precisions run: FP64 throughout, and mixed (FP32
Jacobian / ILU / preconditioner, FP64 residual, Krylov and Newton update); the
headline value is the mixed form.

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
    "tree-7gen": dict(name="tree-7gen", kind="tree"),
    "batch-64-tubes": dict(name="batch-64-tubes", kind="batch"),
}
MATERIAL = dict(rho_f=1.05, mu_f=0.035, rho_s=1.2, E_s=3.0e6, nu_s=0.45, eta_s=0.0)
S_F64 = 8
S_F32 = 4
METRIC = "FSI time steps/s on 1 GB300, mixed-precision vs FP64 at Newton rtol 1e-6"
# DRAM bytes per launch (read + write) from one ncu capture of the kernel as it is
# now, keyed by (workload, phase, precision, subdomains, ILU level, ordering);
# the summary that holds the capture is named beside it
NCU_TRAFFIC = {
    ("tube-96x32x15", "pcapply", "mixed", 512, 1, 1): (585.6e6, "profiles/k_ras_apply_stream_tube-96x32x15.md"),
    ("tube-96x32x15", "spmv", "mixed", 512, 1, 1): (142.9e6, "profiles/k_bsr_spmv_tube-96x32x15.md"),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="tube-96x32x15", choices=sorted(WORKLOADS))
    p.add_argument("--subdomains", type=int, default=256)
    p.add_argument("--ilu", type=int, default=1)
    p.add_argument("--overlap", type=int, default=1)
    p.add_argument("--newton-rtol", type=float, default=1e-6)
    p.add_argument("--gmres-rtol", type=float, default=1e-3)
    p.add_argument("--precisions", default="mixed,fp64")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-autotune", action="store_true", help="use --subdomains/--overlap/--ilu as given")
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
    Stokes solve at t = 0 (rho_f = 0, huge time step, wall clamped) from rest,
    d = 0."""
    import vesselmesh as vm
    kinds = [q.get("kind") for q in m.info.get("problems", [m.info])]
    if all(k == "tube" for k in kinds):
        return vm.poiseuille_state(m)
    from paper_1810_04289_gb300 import fsi
    opt = fsi.FsiOptions()
    for f, _ in fsi.FsiOptions._fields_:
        setattr(opt, f, getattr(opt_base, f))
    opt.dt = 1e8
    opt.newton_rtol = 1e-8
    opt.newton_maxit = 30
    opt.gmres_rtol = 1e-6
    opt.precision = 0
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


def run_ours(args, rank, world):
    import torch
    from paper_1810_04289_gb300 import fsi
    import vesselmesh as vm
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    m = make_mesh(args.workload)
    y0 = initial_state(m, fsi.fsi_default_options(precision=1, n_subdomains=args.subdomains, ilu_level=args.ilu))
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    results = {}
    for prec in args.precisions.split(","):
        pflag = 1 if prec == "mixed" else 0
        opt = fsi.fsi_default_options(newton_rtol=args.newton_rtol, gmres_rtol=args.gmres_rtol,
                                      n_subdomains=args.subdomains, ilu_level=args.ilu, overlap=args.overlap,
                                      precision=pflag)
        tuned = None
        if not args.no_autotune:
            from paper_1810_04289_gb300.autotune import autotune, tune_jac_lag
            t_tune = time.perf_counter()
            opt, table = autotune(m, MATERIAL, y0, base=opt)
            opt, lag_table = tune_jac_lag(m, MATERIAL, y0, opt)
            tuned = {"chosen": {k: getattr(opt, k) for k in ("n_subdomains", "overlap", "ilu_level", "ordering",
                                                             "threads_per_row", "jac_lag")},
                     "seconds": time.perf_counter() - t_tune, "candidates": table, "jac_lag": lag_table}
        S = fsi.Solver(m, MATERIAL, opt)
        info = S.info()
        S.set_state(y0, t=0.0)
        for _ in range(args.warmup):
            S.step()
        stream = torch.cuda.current_stream()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(dev)
        clk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = []
        for _ in range(args.steps):
            stats.append(fsi.stats_dict(S.step()))
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop()
        ms = e0.elapsed_time(e1)
        ms = max_over_ranks(ms, world, "cuda")
        # e2e: through the public API with host buffers, per step H2D of the step's
        # inputs (y_n, y_{n-1}, y_{n-2}) from pinned memory and D2H of the result
        e2e = None
        if not args.no_e2e:
            N7 = m.n_nodes * 7
            ysnap = S.vec()
            fsi.fsi_get_state(S.ctx, ysnap)
            hy = [torch.empty((m.n_nodes, 7), dtype=torch.float64).pin_memory() for _ in range(3)]
            for h in hy:
                h.copy_(ysnap.cpu())
            hout = torch.empty((m.n_nodes, 7), dtype=torch.float64).pin_memory()
            dy = [torch.empty((m.n_nodes, 7), dtype=torch.float64, device="cuda") for _ in range(3)]
            dout = torch.empty((m.n_nodes, 7), dtype=torch.float64, device="cuda")
            t_now = fsi.fsi_get_state(S.ctx, None)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(args.steps):
                for h, d in zip(hy, dy):
                    d.copy_(h, non_blocking=True)
                fsi.fsi_set_state(S.ctx, dy[0], dy[1], dy[2], t_now)
                fsi.fsi_step(S.ctx, stats=False)
                t_now = fsi.fsi_get_state(S.ctx, dout)
                hout.copy_(dout, non_blocking=True)
                torch.cuda.synchronize()
                hy[2].copy_(hy[1]); hy[1].copy_(hy[0]); hy[0].copy_(hout)
            e2e_s = time.perf_counter() - t0
            e2e = {"value": args.steps / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": 3 * N7 * 8,
                   "d2h_bytes_per_step": N7 * 8}
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
        s = S_F32 if pflag else S_F64
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
        phases["krylov"] = {"ms_total": tot["t_krylov"], "note": "GMRES cycles (captured graphs): applies, SpMVs, orthogonalisation"}
        results[prec] = dict(ms=ms, steps=args.steps, value=world * args.steps / (ms * 1e-3), stats=stats, tuned=tuned,
                             tot=tot, phases=phases, info={k: getattr(info, k) for k, _ in info._fields_},
                             clocks=clocks, e2e=e2e, launches=int(tot["kernel_launches"]))
        S.close()
        del S
        torch.cuda.empty_cache()
    return results, hbm_peak


def cpu_sample(args, steps_hint=None):
    """Time the oracle on a bounded sample of the workload (host cores).

    Sample: one full residual evaluation and the complex-step Jacobian of a 5%
    subset of the tets (scaled to all tets) on the benchmark mesh. The oracle's
    direct solve of the full system is not run (hours and tens of GB at this
    size), so the estimate counts assembly only and is an upper bound on the
    oracle's steps/s. Steps/s = 1 / (NI * (t_F * (1 + line-search evaluations)
    + t_J)) with the Newton and line-search counts of the GPU run.
    """
    from oracle import fsi_oracle as O
    m = make_mesh(args.workload)
    import vesselmesh as vm
    y0 = vm.poiseuille_state(m)
    P = O.Problem(m.X, m.tets, m.tet_domain, m.node_tag, m.node_problem, m.inlets, mat=MATERIAL, dt=1e-3)
    t0 = time.perf_counter()
    P.residual(y0, y0, y0, 1e-3)
    tF = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(m.n_tets, size=max(1, m.n_tets // 20), replace=False))
    Ps = O.Problem(m.X, m.tets[sel], m.tet_domain[sel], m.node_tag, m.node_problem, m.inlets, mat=MATERIAL,
                   dt=1e-3)
    t0 = time.perf_counter()
    Ps.jacobian(y0, y0, y0, 1e-3)
    tJ = (time.perf_counter() - t0) * m.n_tets / len(sel)
    ni, nf = (steps_hint or (3.0, 4.0))
    t_step = ni * tJ + nf * tF
    return {"value": 1.0 / t_step, "unit": "steps/s", "cores": 1, "kind": "oracle",
            "nodes": int(m.n_nodes), "tets": int(m.n_tets), "unknowns": int(vm.count_unknowns(m)),
            "sample": (f"{args.workload}: one residual ({tF:.2f} s) + complex-step Jacobian of 5% of the tets "
                       f"scaled to all ({tJ:.1f} s), per step {ni:.1f} Jacobians + {nf:.1f} residuals; "
                       f"direct solve not run (assembly-only, an upper bound on the oracle's steps/s)")}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    if args.impl == "reference":
        if rank != 0:
            return
        vals = []
        for k in range(args.warmup + args.steps):
            r = cpu_sample(args)
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
    res, hbm_peak = run_ours(args, rank, world)
    if rank != 0:
        return
    head = res.get("mixed") or next(iter(res.values()))
    other = res.get("fp64")
    hp = head["phases"]
    dom = max((k for k in hp if "gbs" in hp[k]), key=lambda k: hp[k]["ms_total"])
    roof = {"kernel": dom, "bound": "hbm", "achieved": hp[dom]["gbs"], "peak": hbm_peak, "unit": "GB/s",
            "frac": hp[dom]["gbs"] / hbm_peak, "traffic": None, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    hi = head["info"]
    ch = (head["tuned"] or {}).get("chosen", {})
    key = (args.workload, dom, "mixed" if "mixed" in res else "fp64", hi["n_subdomains"],
           ch.get("ilu_level", args.ilu), ch.get("ordering", 1))
    if key in NCU_TRAFFIC:
        roof["traffic"], roof["traffic_source"] = NCU_TRAFFIC[key]
        roof["algorithmic_bytes"] = hp[dom]["algorithmic_bytes_per_launch"]
    st = head["stats"]
    ni = float(np.mean([s["newton_iterations"] for s in st]))
    nres = float(np.mean([s["residual_evaluations"] for s in st]))
    cpu = None
    if not args.no_cpu and world == 1:
        try:
            cpu = cpu_sample(args, (ni, nres))
        except Exception as e:  # the baseline is context, never a reason to lose the GPU line
            cpu = {"value": None, "error": str(e)}
    line = {
        "metric": METRIC,
        "value": head["value"], "unit": "steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if "mixed" in res else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "nodes": head["info"]["n_nodes"],
                   "unknowns": head["info"]["n_unknowns"], "tets": head["info"]["n_tets"],
                   "subdomains": head["info"]["n_subdomains"],
                   "overlap": (head["tuned"] or {}).get("chosen", {}).get("overlap", args.overlap),
                   "ilu": (head["tuned"] or {}).get("chosen", {}).get("ilu_level", args.ilu),
                   "ordering": (head["tuned"] or {}).get("chosen", {}).get("ordering", 1),
                   "jac_lag": (head["tuned"] or {}).get("chosen", {}).get("jac_lag", 1),
                   "newton_rtol": args.newton_rtol, "gmres_rtol": args.gmres_rtol,
                   "l2": "working set (BSR + ILU factors) larger than L2 each step",
                   "parallelism": "replicas" if world > 1 else "single"},
        "NI": ni, "LI_per_newton": float(np.mean([s["linear_iterations"] / max(1, s["newton_iterations"]) for s in st])),
        "phases_ms_per_step": {k: v["ms_total"] / args.steps for k, v in hp.items()},
        "phases": hp,
        "roofline": roof,
        "clocks": head["clocks"],
        "gpu_launches": head["launches"],
        "e2e": head["e2e"],
        "cpu_baseline": cpu,
        "autotune": head["tuned"],
    }
    if other is not None:
        line["fp64"] = {"value": other["value"], "ms_per_step": other["ms"] / args.steps,
                        "NI": float(np.mean([s["newton_iterations"] for s in other["stats"]])),
                        "LI": float(np.mean([s["linear_iterations"] for s in other["stats"]])),
                        "phases_ms_per_step": {k: v["ms_total"] / args.steps for k, v in other["phases"].items()},
                        "phases": other["phases"], "gpu_launches": other["launches"], "e2e": other["e2e"],
                        "clocks": other["clocks"], "autotune": other["tuned"]}
        line["mixed_over_fp64"] = head["value"] / other["value"]
    print(json.dumps(line))


if __name__ == "__main__":
    main()
