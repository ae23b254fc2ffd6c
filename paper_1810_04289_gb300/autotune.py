"""Measured autotuner for the solver's data-parallel knobs.

For a mesh and a representative state it times, on the GPU and through the C
ABI, one Newton linear system per candidate: preconditioner setup (extraction,
ILU factorisation, packing) plus the GMRES solve to the candidate's tolerance.
Candidates vary the Schwarz subdomain count, the overlap, the ILU fill level, the
subdomain ordering and the SpMV threads per block row (search space: see
default_grid; searched knob by knob, or as a full grid); the fastest converged
time to solution wins. tune_jac_lag then picks the Jacobian lag (how
many Newton iterations reuse one Jacobian and its factors, Eq. 12 and the
paper's Table 3) by timing whole time steps. The solver
arithmetic itself is unchanged by any choice (only the preconditioner and the
launch mapping change), so the tuned options solve the same equations.
"""
import itertools
import time

from . import fsi

def default_grid(n_nodes):
    """The search space: subdomain counts (powers of two giving 40..1000 nodes per
    subdomain), overlap 1 and 2 (Sec. 4.6), ILU(1) and ILU(2) (the paper's levels
    for its small and large meshes, Sec. 4.3, 4.7), RCM, lumen-first RCM and nested
    dissection inside the subdomains (Sec. 4.5), one or two block rows per warp
    in the SpMV. Small subdomains stay in the space because each subdomain's
    triangular solve is a sequential chain on the GPU: more, shorter chains can
    win despite more Krylov iterations."""
    nps = [2 ** k for k in range(4, 16) if 40 <= n_nodes / 2 ** k <= 1000] or [max(1, n_nodes // 400)]
    return dict(n_subdomains=tuple(nps), overlap=(1, 2), ilu_level=(1, 2), ordering=(1, 2, 3),
                threads_per_row=(32, 16))


# order in which the coordinate search visits the knobs (most influential first)
KNOBS = ("n_subdomains", "ilu_level", "ordering", "overlap", "threads_per_row")


def _time_linear_system(S, y, torch):
    """Setup + solve time (s) and iterations for J(y) dy = -F(y) on solver S."""
    yv = S.vec(y)
    F = S.vec()
    fsi.fsi_residual(S.ctx, yv, F)
    F.neg_()
    fsi.fsi_jacobian(S.ctx, yv)
    x = S.vec()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = fsi.fsi_linear_solve(S.ctx, F, x, raise_on_divergence=False)
    torch.cuda.synchronize()
    return time.perf_counter() - t0, st.iterations, st.converged


def _candidate(mesh, material, y0, opt, t0, torch):
    """Setup + solve seconds, iterations and convergence of one candidate, or an error."""
    try:
        S = fsi.Solver(mesh, material, opt)
    except fsi.FsiError as e:          # e.g. factor rows too long for shared memory
        return dict(error=str(e))
    S.set_state(y0, t=t0)
    try:
        # first solve builds the graph and warms the caches; the second is timed
        _time_linear_system(S, y0, torch)
        secs, its, conv = _time_linear_system(S, y0, torch)
    except fsi.FsiError as e:          # e.g. a singular pivot block of this ILU
        return dict(error=str(e))
    finally:
        S.close()
    return dict(seconds=secs, iterations=its, converged=bool(conv))


def autotune(mesh, material, y0, base=None, grid=None, t0=0.0, verbose=False, search="coordinate"):
    """Return (best FsiOptions, list of result dicts) for the given state.

    base: FsiOptions used for every field the grid does not vary (default
    fsi_default_options()). grid: dict of option name -> tuple of values.
    search: "grid" times every combination; "coordinate" starts from the first
    value of every knob (the middle subdomain count) and sweeps the knobs one at
    a time in KNOBS order, each over all its values with the others at their best
    so far, twice (the second sweep re-checks every knob with the others
    settled; candidates already timed are not repeated).
    """
    import torch
    grid = dict(default_grid(mesh.n_nodes) if grid is None else grid)
    base = base if base is not None else fsi.fsi_default_options()
    names = list(grid)
    results = []
    seen = {}

    def make(values):
        opt = fsi.FsiOptions()
        for f, _ in fsi.FsiOptions._fields_:
            setattr(opt, f, getattr(base, f))
        for k, v in values.items():
            setattr(opt, k, v)
        return opt

    def run(values):
        key = tuple(values[k] for k in names)
        if key not in seen:
            rec = dict(values, **_candidate(mesh, material, y0, make(values), t0, torch))
            seen[key] = rec
            results.append(rec)
            if verbose:
                print("autotune", rec, flush=True)
        rec = seen[key]
        return rec["seconds"] if rec.get("converged") else None

    best = None
    if search == "grid":
        for values in itertools.product(*(grid[k] for k in names)):
            v = dict(zip(names, values))
            t = run(v)
            if t is not None and (best is None or t < best[0]):
                best = (t, v)
    else:
        cur = {k: grid[k][0] for k in names}
        if "n_subdomains" in grid:
            nps = grid["n_subdomains"]
            cur["n_subdomains"] = nps[len(nps) // 2]
        order = [k for k in KNOBS if k in grid] + [k for k in names if k not in KNOBS]
        for _ in range(2):
            for k in order:
                for val in grid[k]:
                    v = dict(cur, **{k: val})
                    t = run(v)
                    if t is not None and (best is None or t < best[0]):
                        best = (t, v)
                if best is not None:
                    cur = dict(best[1])
    if best is None:
        raise RuntimeError(f"no candidate converged: {results}")
    return make(best[1]), results


def tune_jac_lag(mesh, material, y0, base, lags=(1, 2, 3), steps=2, t0=0.0, verbose=False):
    """Return (best FsiOptions, list of result dicts): for each Jacobian lag, one
    untimed time step from y0, then `steps` timed steps; the fastest run whose
    steps all converged wins. The Newton tolerance is the same for every lag, so
    each run solves the same steps to the same accuracy."""
    import torch
    results = []
    best = None
    for lag in lags:
        opt = fsi.FsiOptions()
        for f, _ in fsi.FsiOptions._fields_:
            setattr(opt, f, getattr(base, f))
        opt.jac_lag = lag
        S = fsi.Solver(mesh, material, opt)
        S.set_state(y0, t=t0)
        try:
            S.step()
            torch.cuda.synchronize()
            tic = time.perf_counter()
            its = []
            for _ in range(steps):
                st = S.step()
                its.append((st.newton_iterations, st.linear_iterations))
            torch.cuda.synchronize()
            secs = (time.perf_counter() - tic) / steps
        except fsi.FsiError as e:
            results.append(dict(jac_lag=lag, error=str(e)))
            S.close()
            continue
        S.close()
        rec = dict(jac_lag=lag, seconds_per_step=secs, newton_linear_iterations=its)
        results.append(rec)
        if verbose:
            print("jac_lag", rec, flush=True)
        if best is None or secs < best[0]:
            best = (secs, opt)
    if best is None:
        raise RuntimeError(f"no Jacobian lag ran: {results}")
    return best[1], results
