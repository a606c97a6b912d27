"""Adaptive barrier stiffness (tx_params.kappa_adapt_max; IPC's kappa update applied between steps)
through the C ABI against the FP64 oracle: the sphere press of the 10x13x4 gel with kappa at 1 %
of the fixed rule fails on both sides with a fixed kappa (the indenter's placement becomes
infeasible at step 4), and with adaptation both sides double kappa after the same steps, to the
same values, and keep every vertex within the parity gate of the oracle's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2411_04776_gb300 import binding as B  # noqa: E402
from paper_2411_04776_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import PARITY_NEWTON_TOL, POS_TOL  # noqa: E402

STEPS = 10
DMIN = 1e-5


def scene():
    wl = W.small_gel_sphere(1)
    k0 = O.OracleGel.from_workload(wl).info()["kappa"] * 0.01
    return wl, k0


def test_fixed_weak_kappa_fails_like_the_oracle():
    wl, k0 = scene()
    gel = B.Gel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL, kappa=k0)
    og = O.OracleGel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL, kappa=k0)
    for s in range(6):
        st, info = gel.step(wl.poses[s], wl.dt), og.step(wl.poses[s], wl.dt)
        assert st == info["status"], (s, st, info)
        if st:
            break
    assert st == 4  # TX_ERR_INFEASIBLE on both sides


def test_adaptive_kappa_matches_oracle():
    O.set_threads(0)
    wl, k0 = scene()
    gel = B.Gel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL, kappa=k0, kappa_adapt_max=100.0,
                              kappa_adapt_dmin=DMIN)
    og = O.OracleGel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL, kappa=k0, kappa_adapt_max=100.0,
                                   kappa_adapt_dmin=DMIN)
    worst, kaps, prev = 0.0, [], np.inf
    for s in range(STEPS):
        st = gel.step(wl.poses[s], wl.dt)
        info = og.step(wl.poses[s], wl.dt)
        assert st == 0 and info["status"] == 0, (s, st, info)
        d = info["min_distance"]
        # the rule's decision must not sit on a tie the two sides could round differently
        assert abs(d - DMIN) > 1e-3 * DMIN and (not np.isfinite(prev) or abs(d - prev) > 1e-4 * d), (s, d, prev)
        prev = d
        stats = gel.stats()
        assert abs(stats["kappa"] - info["kappa"]) <= 1e-12 * info["kappa"], (s, stats["kappa"], info["kappa"])
        kaps.append(info["kappa"] / k0)
        worst = max(worst, float(np.abs(gel.state()[0] - og.state()[0]).max()))
    print("adaptive kappa: kappa / kappa0 per step %s, max vertex error %.3e m" % (kaps, worst))
    assert kaps[-1] >= 8.0  # the rule acted
    assert worst <= POS_TOL, worst
    gel.reset()  # back to the initial stiffness
    assert gel.step(wl.poses[0], wl.dt) == 0 and abs(gel.stats()["kappa"] - k0) <= 1e-12 * k0
