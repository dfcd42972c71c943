"""Host-side counting used by the benchmark and the refinement study, checked
against the schedule's own arithmetic: the F_E evaluations of an MLSDC step
(the initialisation evaluates node 0 once per level; each sweep evaluates
the nodes after the first; step B evaluates the restricted coarse nodes), the
observed order of an exact power law, and the algorithmic bytes of a node
update.  CPU only (imports the modules without touching a GPU)."""
import math
import sys
from pathlib import Path

import pytest

sys.path.insert(0, str(Path(__file__).resolve().parents[1]))

import bench  # noqa: E402

study = pytest.importorskip("paper_1805_07923_gb300.study")


def test_headline_evaluation_counts():
    w = bench.WORKLOAD
    # 4 iterations: fine 1 + 4 x 4; coarse 1 + 4 x (2 restricted + 2 sweeps x 2 nodes)
    assert bench.evals_per_step(w) == (17, 25)
    # a third level: the middle level adds one up-sweep (2 nodes) per iteration
    assert bench.evals_per_step_levels(w) == (17, 1 + 4 * 2 * 4, 1 + 4 * 1 * 3)


def test_study_evaluation_counts():
    assert study.fe_evals_per_step("SDC(5,8)") == [33]
    assert study.fe_evals_per_step("SDC(3,4)") == [9]
    assert study.fe_evals_per_step("MLSDC(5,3,4,1/2)") == [17, 17]
    assert study.fe_evals_per_step("MLSDC(3,2,2,1/2)") == [5, 5]
    assert study.fe_evals_per_step("MLSDC(5,3,2,4)") == [17, 25, 9]


def test_observed_order_of_a_power_law():
    dts = [1200.0, 900.0, 600.0, 450.0]
    for p in (2.0, 4.0, 8.0):
        errs = [3.0e-5 * dt ** p for dt in dts]
        orders = study.observed_orders(dts, errs)
        assert orders[0] is None
        assert all(abs(o - p) < 1e-12 for o in orders[1:])
    assert study.observed_orders([2.0, 1.0], [1.0, 0.0]) == [None, None]


def test_node_update_bytes():
    R, n = 3, 5
    nc = (R + 1) * (R + 2) // 2
    field3 = 3 * nc * 16
    # m = 0: Theta^0, old F_I and F_E at 5 nodes; writes Theta, F_I at node 1, node 0 of the new F
    # and the sweep-constant arrays S_2..S_4
    assert bench.node_update_bytes(R, n, 0, False) == field3 * 11 + field3 * 7 + (R + 1) * 16 + nc * 4
    # m = 2: S_3 and the new F_I, F_E at nodes 1..2; writes Theta, F_I at node 3
    assert bench.node_update_bytes(R, n, 2, False) == field3 * 5 + field3 * 2 + (R + 1) * 16 + nc * 4
    # m = 2 with implicit Coriolis: also new F_I, F_E at nodes 1..2, and the chains' tables
    assert bench.node_update_bytes(R, n, 2, True) == field3 * 15 + field3 * 2 + nc * 160
    assert math.isclose(bench.node_update_bytes(170, 5, 0, True) / 1e6, 12.94128, rel_tol=1e-6)
