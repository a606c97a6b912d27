"""IPC lagged friction through the C ABI (tx_params.friction) against the FP64 oracle's friction
(the same lagged pairs, closest-point weights, tangent bases and normal forces, fixed at the start
of each (sub)step): a sphere pressed into the 10x13x4 gel and then slid across it, every step
compared vertex by vertex (4 nm) with the contact force, friction included, in FP64 and in mixed
precision; the slide must produce a real tangential force (Coulomb: about mu_f times the normal
force), which the frictionless run does not."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2411_04776_gb300 import binding as B  # noqa: E402
from paper_2411_04776_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import PARITY_NEWTON_TOL, POS_TOL  # noqa: E402

MU = 0.5
EPS_V = 1e-3


def press_slide():
    return W.mini_gel(seed=4, grid=W.GRID_SMALL, kind="sphere", depth=0.4e-3, n_press=10, slide=1.0e-3,
                      n_slide=10)


@pytest.fixture(scope="module")
def oracle_run():
    O.set_threads(0)
    wl = press_slide()
    og = O.OracleGel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL, friction=MU, eps_v=EPS_V)
    out = []
    for s in range(len(wl.poses)):
        info = og.step(wl.poses[s], wl.dt)
        assert info["status"] == 0, (s, info)
        x, _, fc, _ = og.state()
        out.append((x.copy(), fc.copy(), info["substeps"]))
    return wl, out


@pytest.mark.parametrize("precision", [B.TX_PREC_FP64, B.TX_PREC_MIXED], ids=["fp64", "mixed"])
def test_friction_matches_oracle(oracle_run, precision):
    wl, ref = oracle_run
    gel = B.Gel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL, precision=precision, friction=MU,
                              friction_eps_v=EPS_V)
    worst, fworst = 0.0, 0.0
    for s in range(len(wl.poses)):
        assert gel.step(wl.poses[s], wl.dt) == 0, s
        x, _, fc, st = gel.state()
        xo, fo, sub = ref[s]
        assert st.substeps == sub, s
        worst = max(worst, float(np.abs(x - xo).max()))
        if np.abs(fo).max() > 0:
            fworst = max(fworst, float(np.abs(fc - fo).max() / np.abs(fo).max()))
    gel.close()
    print("friction (mu %.1f) vs oracle: max vertex error %.3e m, max relative contact-force error %.2e"
          % (MU, worst, fworst))
    assert worst <= POS_TOL
    assert fworst <= 2e-3
    # sliding along +x: the indenter drags the gel with a tangential force of about mu times the
    # normal force (the contact force is the indenter's force on the gel)
    fo = ref[-1][1]
    assert fo[0] > 0.8 * MU * abs(fo[2]), fo


def test_frictionless_slide_has_no_tangential_force():
    wl = press_slide()
    gel = B.Gel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL)
    for s in range(len(wl.poses)):
        assert gel.step(wl.poses[s], wl.dt) == 0
    fc = gel.state()[2]
    gel.close()
    assert abs(fc[0]) < 0.1 * abs(fc[2]), fc
