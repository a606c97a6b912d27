"""Gel-level parity of the CUDA path against the FP64 oracle: energy and gradient of the
incremental potential at seeded states, whole-step trajectories, invariants and error paths."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2411_04776_gb300 import binding as B  # noqa: E402
from paper_2411_04776_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import PARITY_NEWTON_TOL, POS_TOL, smooth_state  # noqa: E402


def contact_pose(wl, depth):
    p = wl.poses[-1].copy()
    p[6] += (0.6e-3 - depth) if wl.name.startswith("gel10") else 0.0
    return p


@pytest.mark.parametrize("make", [lambda: W.small_gel_sphere(0), lambda: W.small_gel_sphere(3),
                                  lambda: W.mini_gel(1, kind="cylinder", n_press=60, n_slide=0)])
def test_energy_and_gradient_match_oracle(make):
    wl = make()
    gel = B.Gel.from_workload(wl)
    ref = O.OracleGel.from_workload(wl)
    x, xt, h = smooth_state(wl, 5)
    # indenter lowered so that it overlaps the barrier zone but not the (displaced) gel
    pose = wl.pose0.copy()
    pose[6] -= 0.95 * W.DHAT
    eg, pg = gel.energy(x, xt, h, pose)
    eo, po = ref.energy(x, xt, h, pose)
    assert np.isfinite(eo) and po["active"] > 0
    assert pg["active"] == po["active"]
    assert abs(eg - eo) <= 1e-12 * abs(eo)
    for k in ("inertia", "elastic", "barrier"):
        assert abs(pg[k] - po[k]) <= 1e-11 * abs(po[k]) + 1e-30, k
    gg, fg = gel.gradient(x, xt, h, pose)
    go, fo = ref.gradient(x, xt, h, pose)
    free = wl.gel.dirichlet == 0
    scale = np.abs(go[free]).max()
    assert np.abs(gg[free] - go[free]).max() <= 1e-10 * scale
    assert np.abs(fg - fo).max() <= 1e-10 * np.abs(fo).max()


def test_rest_state_is_a_fixed_point():
    wl = W.small_gel_sphere(0)
    gel = B.Gel.from_workload(wl)
    far = W.pose((0.009, 0.012, 0.05))
    gel.set_state(wl.gel.verts, np.zeros_like(wl.gel.verts), far)
    assert gel.step(far, wl.dt) == 0
    x, v, fc, st = gel.state()
    assert st.newton_iters == 0 and np.array_equal(x, wl.gel.verts) and np.all(v == 0)


def run_pair(wl, steps, tol=PARITY_NEWTON_TOL):
    gel = B.Gel.from_workload(wl, newton_tol=tol)
    ref = O.OracleGel.from_workload(wl, newton_tol=tol)
    errs = []
    for s in range(steps):
        st = gel.step(wl.poses[s], wl.dt)
        info = ref.step(wl.poses[s], wl.dt)
        assert st == 0, B.STATUS_NAMES[st]
        assert info["status"] == 0
        xg, vg, fg, sg = gel.state()
        xo, vo, fo, _ = ref.state()
        errs.append(np.abs(xg - xo).max())
        assert sg.substeps == info["substeps"]
        assert sg.min_distance > 0
    return gel, ref, np.array(errs), fg, fo


def test_small_gel_trajectory_matches_oracle():
    """All 30 steps of the 10x13x4 gel pressed 0.6 mm by the r = 5 mm sphere."""
    wl = W.small_gel_sphere(0)
    gel, ref, errs, fg, fo = run_pair(wl, 30)
    assert errs.max() <= POS_TOL, errs
    assert np.abs(fg - fo).max() <= 1e-4 * np.abs(fo).max()


def test_gelsight_mini_steps_match_oracle():
    """First contact steps of the GelSight-Mini gel (41x51x9: 18,819 vertices, 96,000 tets) pressed
    by the seeded prism indenter, in the launch configuration the bench times (one gel, FP64):
    the prism starts d_hat above the gel and travels 33 um per step, contact from step 4 on."""
    wl = W.mini_gel(seed=3, kind="prism", depth=0.3e-3, n_press=12, slide=0.0, n_slide=0)
    gel, ref, errs, fg, fo = run_pair(wl, 6)
    assert gel.state()[3].active_pairs > 0
    assert errs.max() <= POS_TOL, errs
    assert np.abs(fg - fo).max() <= 1e-4 * max(np.abs(fo).max(), 1e-12)


def test_mixed_precision_trajectory_matches_oracle():
    """FP32 Hessian blocks + FP32 Krylov solve with FP64 residual refinement; the gradient,
    barrier, CCD and energy stay FP64, so the converged minimiser is the FP64 one."""
    wl = W.small_gel_sphere(0)
    gel = B.Gel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL, precision=B.TX_PREC_MIXED)
    ref = O.OracleGel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL)
    errs = []
    for s in range(30):
        st = gel.step(wl.poses[s], wl.dt)
        info = ref.step(wl.poses[s], wl.dt)
        assert st == 0 and info["status"] == 0, B.STATUS_NAMES[st]
        errs.append(np.abs(gel.state()[0] - ref.state()[0]).max())
    errs = np.array(errs)
    print("mixed precision max / rms error over steps: %.3e / %.3e m" % (errs.max(), np.sqrt(np.mean(errs ** 2))))
    assert errs.max() <= POS_TOL


def test_forcing_terms_keep_the_minimiser():
    """The loose PCG forcing term far from Newton convergence (0.1, the default) changes the
    iterates but not the converged state: every step of the 10x13x4 gel pressed by the sphere
    matches a fixed 1e-3 forcing term within the parity gate, with fewer PCG iterations."""
    wl = W.small_gel_sphere(0)
    loose = B.Gel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL)
    fixed = B.Gel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL, pcg_rel_tol_far=0.0)
    it_loose = it_fixed = 0
    for s in range(30):
        assert loose.step(wl.poses[s], wl.dt) == 0
        assert fixed.step(wl.poses[s], wl.dt) == 0
        xl, _, fl, sl = loose.state()
        xf, _, ff, sf = fixed.state()
        it_loose += sl.pcg_iters
        it_fixed += sf.pcg_iters
        assert np.abs(xl - xf).max() <= POS_TOL
    assert it_loose < it_fixed, (it_loose, it_fixed)


def test_batch_equals_alone():
    wls = [W.small_gel_sphere(s) for s in range(3)]
    descs = [B.GelDesc.from_workload(w, newton_tol=PARITY_NEWTON_TOL) for w in wls]
    b = B.tx_batch_create(descs)
    alone = [B.Gel.from_workload(w, newton_tol=PARITY_NEWTON_TOL) for w in wls]
    try:
        for s in range(8):
            poses = np.stack([w.poses[s] for w in wls])
            st, sts = B.tx_batch_step(b, poses, np.full(3, wls[0].dt))
            assert st == 0 and np.all(sts == 0)
            for g, w in enumerate(wls):
                assert alone[g].step(w.poses[s], w.dt) == 0
                xb = B.tx_batch_state(b, g, len(w.gel.verts))[0]
                xa = alone[g].state()[0]
                assert np.abs(xb - xa).max() <= POS_TOL
    finally:
        B.tx_batch_destroy(b)


def test_error_paths():
    wl = W.small_gel_sphere(0)
    bad = wl.gel.tets.copy()
    bad[0, [2, 3]] = bad[0, [3, 2]]
    with pytest.raises(B.TxError) as e:
        B.Gel(B.GelDesc(wl.gel.verts, bad, wl.gel.dirichlet, wl.material, wl.indenter.verts, wl.indenter.tris, wl.pose0))
    assert e.value.status == 3
    bad = wl.gel.tets.copy()
    bad[1, 1] = 99999
    with pytest.raises(B.TxError) as e:
        B.Gel(B.GelDesc(wl.gel.verts, bad, wl.gel.dirichlet, wl.material, wl.indenter.verts, wl.indenter.tris, wl.pose0))
    assert e.value.status == 1
    # indenter teleported deep into the gel: no split depth can make this feasible
    gel = B.Gel.from_workload(wl)
    deep = wl.pose0.copy()
    deep[6] -= 3e-3
    st = gel.step(deep, wl.dt)
    assert st == 4
    x, v, _, _ = gel.state()
    assert np.array_equal(x, wl.gel.verts)  # transactional
    assert gel.step(wl.poses[0], wl.dt) == 0


def test_autotuned_split_keeps_the_minimiser():
    """The opt-in PCG work-split autotuner (pcg_cta_slices = -1) tries other CTA splits on live
    Newton rounds; the split changes only the order of the PCG's sums, so the stepped states stay
    within the parity gate of the default split."""
    wls = [W.small_gel_sphere(s) for s in range(3)] + [W.mini_gel(7, grid=W.GRID_MID, depth=0.5e-3)]
    tuned = B.tx_batch_create([B.GelDesc.from_workload(w, newton_tol=PARITY_NEWTON_TOL, pcg_cta_slices=-1)
                               for w in wls])
    plain = B.tx_batch_create([B.GelDesc.from_workload(w, newton_tol=PARITY_NEWTON_TOL) for w in wls])
    try:
        for s in range(12):
            poses = np.stack([w.poses[s] for w in wls])
            dts = np.array([w.dt for w in wls])
            for h in (tuned, plain):
                st, sts = B.tx_batch_step(h, poses, dts)
                assert st == 0 and np.all(sts == 0)
        for g, w in enumerate(wls):
            d = np.abs(B.tx_batch_state(tuned, g, len(w.gel.verts))[0] - B.tx_batch_state(plain, g, len(w.gel.verts))[0])
            assert d.max() <= POS_TOL, (g, d.max())
    finally:
        B.tx_batch_destroy(tuned)
        B.tx_batch_destroy(plain)
