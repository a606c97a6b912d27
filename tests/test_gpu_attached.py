"""Attachment-driven steps (TacEx, Sec. "General GIPC Simulation Pipeline": the attachment targets
are set from the sensor-case pose, then the solver runs) through the C ABI against the FP64
oracle's attachment-driven step: the attached (Dirichlet) vertices ride on a case that translates
and turns while the indenter presses, every step compared vertex by vertex (4 nm), with the
substep count and the contact force; a rigid carry of the gel with its case; a batch of
attachment-driven gels equal to each gel alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2411_04776_gb300 import binding as B  # noqa: E402
from paper_2411_04776_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import PARITY_NEWTON_TOL, POS_TOL  # noqa: E402


def case_trajectory(n, shift=(60e-6, -25e-6, 12e-6), turn=4e-4):
    """Case poses of n steps: a translation per step and a turn about z (axis through the gel's
    rest-frame origin) per step."""
    out = []
    for s in range(1, n + 1):
        q = W.quat_axis_angle((0.0, 0.0, 1.0), turn * s)
        out.append(W.pose(tuple(np.array(shift) * s), q))
    return np.array(out)


def test_attached_steps_match_oracle():
    wl = W.small_gel_sphere(1)
    n = 14
    cases = case_trajectory(n)
    gel = B.Gel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL)
    og = O.OracleGel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL)
    worst, contact = 0.0, 0
    for s in range(n):
        st = gel.step_attached(wl.poses[s], cases[s], wl.dt)
        info = og.step_attached(wl.poses[s], cases[s], wl.dt)
        assert st == 0 and info["status"] == 0, (s, st, info)
        xg, vg, fg, sg = gel.state()
        xo, vo, fo, _ = og.state()
        assert sg.substeps == info["substeps"], s
        worst = max(worst, float(np.abs(xg - xo).max()))
        assert np.abs(vg - vo).max() <= POS_TOL / wl.dt
        if np.abs(fo).max() > 0:
            contact += 1
            # the contact force of runs stopped at Newton tolerance 1e-7 agrees to ~1e-3 (the
            # oracle's own force moves by up to 7e-4 when the tolerance is tightened)
            assert np.abs(fg - fo).max() <= 2e-3 * np.abs(fo).max(), (s, fg, fo)
    print("attachment-driven steps vs oracle: max vertex error %.3e m over %d steps (%d in contact)"
          % (worst, n, contact))
    assert worst <= POS_TOL and contact > 3
    # the attached vertices sit exactly at their carried rest positions
    fixed = wl.gel.dirichlet == 1
    c = cases[-1]
    R = np.array([[1 - 2 * (c[2] ** 2 + c[3] ** 2), 2 * (c[1] * c[2] - c[0] * c[3]), 2 * (c[1] * c[3] + c[0] * c[2])],
                  [2 * (c[1] * c[2] + c[0] * c[3]), 1 - 2 * (c[1] ** 2 + c[3] ** 2), 2 * (c[2] * c[3] - c[0] * c[1])],
                  [2 * (c[1] * c[3] - c[0] * c[2]), 2 * (c[2] * c[3] + c[0] * c[1]), 1 - 2 * (c[1] ** 2 + c[2] ** 2)]])
    want = wl.gel.verts[fixed] @ R.T + c[4:]
    assert np.abs(gel.state()[0][fixed] - want).max() <= 1e-15
    assert np.allclose(gel.case_pose(), c, rtol=0, atol=0)
    gel.close()


def test_rigid_carry_with_the_case():
    """No contact, gel moving with its case at constant velocity: a rigid translation, met to the
    Newton tolerance."""
    wl = W.small_gel_sphere(0)
    gel = B.Gel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL)
    far = W.pose((0.009, 0.012, 0.05))
    v0 = np.array([2e-3, -1e-3, 3e-3])
    X = wl.gel.verts
    gel.set_state(X, np.tile(v0, (len(X), 1)), far)
    for s in range(1, 6):
        t = v0 * wl.dt * s
        assert gel.step_attached(far, W.pose(t), wl.dt) == 0
        x, v, fc, _ = gel.state()
        assert np.abs(x - (X + t)).max() <= 1e-9
        assert np.abs(v - v0).max() <= 1e-9 / wl.dt
        assert np.all(fc == 0)
    gel.close()


def test_batch_of_attached_gels_equals_alone():
    wls = [W.small_gel_sphere(s) for s in (2, 3)]
    descs = [B.GelDesc.from_workload(w, newton_tol=PARITY_NEWTON_TOL) for w in wls]
    b = B.tx_batch_create(descs)
    alone = [B.Gel.from_workload(w, newton_tol=PARITY_NEWTON_TOL) for w in wls]
    cases = [case_trajectory(10, shift=(20e-6 * (g + 1), 0.0, -10e-6), turn=3e-4 * (g + 1)) for g in range(2)]
    try:
        for s in range(10):
            st, sts = B.tx_batch_step_attached(b, np.stack([w.poses[s] for w in wls]),
                                               np.stack([cases[g][s] for g in range(2)]), np.full(2, wls[0].dt))
            assert st == 0 and np.all(sts == 0)
            for g, w in enumerate(wls):
                assert alone[g].step_attached(w.poses[s], cases[g][s], w.dt) == 0
                d = np.abs(B.tx_batch_state(b, g, len(w.gel.verts))[0] - alone[g].state()[0]).max()
                assert d <= POS_TOL, (s, g, d)
    finally:
        B.tx_batch_destroy(b)
