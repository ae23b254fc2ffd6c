"""bench.py's option plumbing, on the CPU: the committed per-workload choices,
the time step of each workload, and the flags that override them."""
import argparse

import pytest

import bench


def _args(**over):
    base = dict(workload="tree-3gen", subdomains=None, ilu=None, overlap=None, ordering=None, jac_lag=None,
                orth=None, stages=None, stage_blocks=None, threads_per_row=None, newton_rtol=1e-6, gmres_rtol=1e-3)
    base.update(over)
    return argparse.Namespace(**base)


def test_committed_choice_and_time_step():
    from paper_1810_04289_gb300 import fsi
    opt, committed = bench.options_for(_args(), "mixed", fsi)
    assert committed and opt.precision == 1 and opt.dt == 1e-3
    t = bench.TUNED[("tree-3gen", "mixed")]
    assert (opt.n_subdomains, opt.ilu_level, opt.ordering, opt.jac_lag, opt.threads_per_row) == \
        (t["n_subdomains"], t["ilu_level"], t["ordering"], t["jac_lag"], t["threads_per_row"])
    opt7, _ = bench.options_for(_args(workload="tree-7gen"), "fp64", fsi)
    assert opt7.dt == 2e-3 and opt7.precision == 0 and opt7.n_subdomains == 49152


def test_flags_override_the_committed_choice():
    from paper_1810_04289_gb300 import fsi
    opt, _ = bench.options_for(_args(subdomains=128, ilu=2, orth=2, stages=3, stage_blocks=20, threads_per_row=32,
                                     jac_lag=1), "mixed", fsi)
    assert (opt.n_subdomains, opt.ilu_level, opt.orth, opt.stages, opt.stage_blocks, opt.threads_per_row,
            opt.jac_lag) == (128, 2, 2, 3, 20, 32, 1)


@pytest.mark.parametrize("name", sorted(bench.WORKLOADS))
def test_every_workload_has_a_kind(name):
    assert bench.WORKLOADS[name]["kind"] in ("tube", "tree", "batch")
