"""Host-side configuration of bench.py (no GPU): which wall rule each
workload runs and which library flags a command line selects.  The wall rule
is chosen by packing name, so a renamed workload would silently run Eq. (CLI)
without the corner safeguards on a packing where it grows; these tests tie
the names to the workload recipes."""
import argparse

import pytest

import bench
import paper_1507_06565_gb300 as L
from paper_1507_06565_gb300 import workloads as W


def _args(**kw):
    base = dict(workload="channel", wall_rule="auto", odd="auto", even="auto", bounce_back=False,
                plane_references="auto")
    base.update(kw)
    return argparse.Namespace(**base)


def test_unstable_packing_names_are_real_workloads():
    names = {W.W2(phi).name for phi in W.W2_POROSITIES} | {W.W3_LARGE.name}
    names |= {W.W4_cube(i).name for i in range(64)}
    assert bench.PAPER_CLI_UNSTABLE <= names, bench.PAPER_CLI_UNSTABLE - names


@pytest.mark.parametrize("phi,rule", [(0.4, "safeguards"), (0.6, "paper"), (0.8, "paper"), (0.9, "paper")])
def test_channel_sweep_wall_rule(phi, rule):
    assert bench.wall_rule(_args(), [W.W2(phi)]) == rule
    # the four solvers of the sweep each take their own rule
    flags = bench.odd_flags(_args(), [W.W2(phi)])
    assert bool(flags & L.LBM_FLAG_CLI_SAFEGUARDS) == (rule == "safeguards")


def test_safeguarded_workloads_and_forced_rules():
    assert bench.wall_rule(_args(), [W.W3_LARGE]) == "safeguards"
    for wl in ("rev", "surrogate", "grid-study", "re-sweep"):
        assert bench.wall_rule(_args(workload=wl), [W.W2(0.9)]) == "safeguards"
    assert bench.wall_rule(_args(), [W.W1]) == "paper"
    assert bench.wall_rule(_args(wall_rule="paper"), [W.W2(0.4)]) == "paper"
    assert bench.wall_rule(_args(wall_rule="safeguards"), [W.W2(0.9)]) == "safeguards"


@pytest.mark.parametrize("odd,flag", [("auto", 0), ("table", L.LBM_FLAG_NEIGHBOUR_TABLE),
                                      ("rows", L.LBM_FLAG_ROW_NEIGHBOURS),
                                      ("staged", L.LBM_FLAG_STAGED_NEIGHBOURS),
                                      ("derived", L.LBM_FLAG_DERIVED_NEIGHBOURS)])
def test_odd_neighbour_flags(odd, flag):
    assert bench.odd_flags(_args(odd=odd), [W.W2(0.9)]) == flag


def test_other_flags():
    c = [W.W2(0.9)]
    assert bench.odd_flags(_args(even="staged"), c) == L.LBM_FLAG_STAGED_EVEN
    assert bench.odd_flags(_args(bounce_back=True), c) == L.LBM_FLAG_SIMPLE_BOUNCE_BACK
    assert bench.odd_flags(_args(plane_references="on"), c) == L.LBM_FLAG_PLANE_REFERENCES
    assert bench.odd_flags(_args(plane_references="off"), c) == L.LBM_FLAG_NO_PLANE_REFERENCES
