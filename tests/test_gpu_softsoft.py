"""Soft-to-soft contact (a mesh of two bodies: the gelpad and a soft ball, pressed by a rigid plate)
through the C ABI: every step against the FP64 oracle (positions, active pairs, the plate's force
on the mesh, no pair left out of the matrix); the energy, gradient and active pairs at a squeezed
state; a ball dropped on a gel whose vertices are all held against the same ball dropped on a
rigid copy of that gel's surface (both on the GPU: soft-soft pairs against rigid pairs); and the
readouts, which see the gelpad's top surface only."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2411_04776_gb300 import binding as B  # noqa: E402
from paper_2411_04776_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import PARITY_NEWTON_TOL, POS_TOL  # noqa: E402

STEPS = 6
# No friction: with IPC friction on the plate-ball pairs and none on the ball-gel pairs (R25) the
# squeezed ball's sideways motion is nearly free once the plate slides over it, and the state a
# solve converges to depends on its path (the GPU's inexact Newton with its Galerkin start against
# the oracle's exact solves: 38 um apart after the second step; from the same start state, the same
# point to 5e-12 m)
MU = 0.0


def ball_scene():
    """Both contacts in place from the first step (gaps of d_hat / 2), a slow squeeze: a ball that
    the plate first knocks loose flies free and is caught again, and where it lands then depends on
    rounding (tens of microns, every outcome converged) — not a parity case."""
    return W.gel_ball(6, grid=W.GRID_SMALL, n_press=20, n_slide=4, depth=0.6e-3, gap_below=0.5 * W.DHAT,
                      gap_above=0.5 * W.DHAT)


@pytest.fixture(scope="module")
def reference():
    O.set_threads(0)
    wl = ball_scene()
    og = O.OracleGel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL, newton_max=400, friction=MU)
    assert og.components()[0] == 2
    out = []
    for s in range(STEPS):
        info = og.step(wl.poses[s], wl.dt)
        assert info["status"] == 0, info
        x, _, fc, _ = og.state()
        out.append((x.copy(), fc.copy(), info))
    return wl, out


@pytest.mark.parametrize("plan,coarse_off", [(0, 0), (1, 0), (1, 1)],
                         ids=["automatic", "streaming", "streaming-no-coarse"])
def test_soft_ball_matches_oracle(reference, plan, coarse_off):
    """FP64, with the automatic plan and with the streaming PCG forced, with and without its
    coarse space over the ball's six rigid motions."""
    precision = B.TX_PREC_FP64
    wl, ref = reference
    gel = B.Gel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL, newton_max_iter=400, precision=precision,
                              pcg_plan=plan, pcg_coarse_off=coarse_off, friction=MU,
                              stream=torch.cuda.current_stream())
    B.tx_gel_profile(gel.h, True)
    worst, ss_active, cut, errs, acts, fdev, subs = 0.0, 0, 0, [], [], [], []
    pcg = newton = 0
    try:
        for s in range(STEPS):
            assert gel.step(wl.poses[s], wl.dt) == 0
            x, _, fc, st = gel.state()
            xo, fo, info = ref[s]
            # pairs whose distance ends within rounding of d_hat may count on one side only
            acts.append((st.active_pairs, info["active_pairs"]))
            subs.append((st.substeps, info["substeps"], st.newton_iters, info["newton_iters"]))
            cut += st.soft_pairs_cut
            errs.append(float(np.abs(x - xo).max()))
            worst = max(worst, errs[-1])
            # the plate's force: its normal (z) part to 2e-3, what the barrier's stiffness near
            # d = 50 um makes of the position gate; its tangential part (a frictionless flat plate:
            # only the edge-edge pairs' common normals tilt, nearly cancelling) to 2e-2 of the force
            fn = max(1e-3, float(np.linalg.norm(fo)))
            fcv = np.asarray(fc)
            fdev.append((abs(fcv[2] - fo[2]) / fn, float(np.abs(fcv[:2] - fo[:2]).max()) / fn))
            ss_active = max(ss_active, info["active_pairs"])
            pcg += st.pcg_iters
            newton += st.newton_iters
        prof = B.tx_gel_profile(gel.h, False)
    finally:
        gel.close()
    print("soft ball (%s, %s PCG) vs oracle: max vertex error per step %s m, active pairs (GPU, oracle) %s, "
          "pair assemblies cut %d, %d Newton and %d PCG iterations"
          % ("fp64" if precision == B.TX_PREC_FP64 else "mixed",
             ("streaming" + (" without coarse space" if coarse_off else "")) if plan else "automatic",
             ["%.2e" % e for e in errs], acts, cut, newton, pcg))
    print("  substeps and Newton iterations per step (GPU, oracle):", subs)
    if plan == 1:
        assert prof["pcg_streaming_launches"] > 0 and prof["pcg_resident_launches"] == 0, prof
    assert worst <= POS_TOL, worst
    assert all(abs(a - b) <= max(3, b // 10) for a, b in acts), acts
    assert all(n <= 2e-3 and t <= 2e-2 for n, t in fdev), fdev
    assert cut == 0, cut  # every cross-body block found a spare position


def test_mixed_precision_refuses_a_free_body():
    """Mixed precision is not offered for a mesh with a body held by no vertex (measured: its FP32
    inner solves end the soft ball's first step 30 um from the oracle's state): TX_ERR_ARG with a
    message; FP64, and mixed precision once the ball is held, are accepted."""
    wl = ball_scene()
    with pytest.raises(B.TxError) as e:
        B.Gel.from_workload(wl, precision=B.TX_PREC_MIXED)
    assert e.value.status == 1 and "free body" in B.load().tx_last_error().decode()  # TX_ERR_ARG
    B.Gel.from_workload(wl).close()
    held = wl.gel.dirichlet.copy()
    held[-1] = 1  # one ball vertex held
    B.Gel(B.GelDesc(wl.gel.verts, wl.gel.tets, held, wl.material, wl.indenter.verts, wl.indenter.tris, wl.pose0,
                    dhat=wl.dhat, precision=B.TX_PREC_MIXED)).close()


def test_soft_ball_energy_and_gradient_match_oracle(reference):
    """At the oracle's state after the squeeze (soft-soft pairs within d_hat): the GPU's energy
    parts, active-pair count (indenter and soft-soft pairs together) and gradient of the step's
    incremental potential, evaluated at that state, against the oracle's."""
    wl, ref = reference
    og = O.OracleGel.from_workload(wl)
    xo = ref[-1][0]
    pose = wl.poses[STEPS - 1]
    counts = og.pair_counts(xo, pose)
    assert counts[8] > 0 and counts[9] > 0, counts  # soft-soft pairs in contact
    xt = xo + 1e-6  # any predictor
    eo, po = og.energy(xo, xt, wl.dt, pose)
    go, fo = og.gradient(xo, xt, wl.dt, pose)
    gel = B.Gel.from_workload(wl)
    try:
        eg, pg = gel.energy(xo, xt, wl.dt, pose)
        gg, fg = gel.gradient(xo, xt, wl.dt, pose)
    finally:
        gel.close()
    assert pg["active"] == po["active"] == int(counts[5:].sum()), (pg, po, counts)
    assert abs(pg["barrier"] - po["barrier"]) <= 1e-11 * abs(po["barrier"]), (pg, po)
    assert abs(eg - eo) <= 1e-11 * abs(eo), (eg, eo)
    free = wl.gel.dirichlet == 0
    scale = np.abs(go[free]).max()
    err = np.abs(gg - go) * free[:, None]
    i = int(np.argmax(err.max(axis=1)))
    print("soft ball gradient vs oracle: %.2e of its scale, worst at vertex %d" % (err.max() / scale, i))
    # the flat contact patch holds nearly parallel edge pairs, whose line-line closest points lose
    # digits (both sides: the energy still agrees to 1e-11)
    assert err.max() <= 1e-7 * scale, err.max() / scale
    assert np.abs(np.asarray(fg) - fo).max() <= 1e-9 * max(np.abs(fo).max(), 1e-12), (fg, fo)


def _held_gel_scene():
    gel = W.gel_grid(*W.GRID_SMALL[0], W.GRID_SMALL[1])
    c = (0.009, 0.012, gel.top + 2 * W.DHAT + 3e-3)
    ball = W.ball_mesh(6, 3e-3, c)
    gel.dirichlet[:] = 1
    return gel, ball


def test_ball_on_held_gel_equals_ball_on_rigid_copy():
    """GPU against GPU: a ball dropped (gravity, initial velocity) on a gel whose vertices are all
    held moves as the ball alone dropped on a rigid indenter made of that gel's surface at rest,
    to the Newton tolerance (soft-soft pairs against the rigid pair path)."""
    gel, ball = _held_gel_scene()
    both = W.join_meshes(gel, ball)
    far = np.array([1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0])
    plate = W.flat_plate(0.004, 3)
    f = np.concatenate([gel.tets[:, [1, 2, 3]], gel.tets[:, [0, 2, 3]], gel.tets[:, [0, 1, 3]], gel.tets[:, [0, 1, 2]]])
    key, cnt = np.unique(np.sort(f, axis=1), axis=0, return_counts=True)
    st = key[cnt == 1]
    sv = np.unique(st)
    remap = np.full(len(gel.verts), -1)
    remap[sv] = np.arange(len(sv))
    ident = np.array([1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0])

    def diag(v):
        return float(np.linalg.norm(v.max(axis=0) - v.min(axis=0)))

    kw = dict(dhat=W.DHAT, kappa=500.0, gravity=(0.0, 0.0, -9.81), newton_max_iter=2000,
              stream=torch.cuda.current_stream())
    tol = 1e-7
    a = B.Gel(B.GelDesc(both.verts, both.tets, both.dirichlet, (W.YOUNG, W.POISSON, W.DENSITY), plate.verts,
                        plate.tris, far, newton_tol=tol, **{k: v for k, v in kw.items() if k != "stream"}),
              kw["stream"])
    b = B.Gel(B.GelDesc(ball.verts, ball.tets, ball.dirichlet, (W.YOUNG, W.POISSON, W.DENSITY), gel.verts[sv],
                        remap[st].astype(np.int32), ident, newton_tol=tol * diag(both.verts) / diag(ball.verts),
                        **{k: v for k, v in kw.items() if k != "stream"}), kw["stream"])
    v = np.tile([0.01, 0.0, -0.05], (len(ball.verts), 1))
    a.set_state(both.verts, np.concatenate([np.zeros_like(gel.verts), v]), far)
    b.set_state(ball.verts, v, ident)
    err, act = 0.0, 0
    try:
        for s in range(6):
            assert a.step(far, W.DT) == 0 and b.step(ident, W.DT) == 0
            sa, sb = a.stats(), b.stats()
            assert sa["active_pairs"] == sb["active_pairs"], (s, sa, sb)
            act = max(act, sa["active_pairs"])
            err = max(err, float(np.abs(a.state()[0][len(gel.verts):] - b.state()[0]).max()))
    finally:
        a.close()
        b.close()
    print("ball on a held gel vs on its rigid copy (GPU): max difference %.3e m, most active pairs %d" % (err, act))
    assert act > 20, act
    assert err < 1e-9, err


def test_readout_sees_the_gelpad_only(reference):
    """Markers and the height map of the two-body mesh use the gelpad's top surface (body 0): the
    ball above it never shows, and both readouts equal the oracle's of the same state."""
    wl, ref = reference
    xo = ref[-1][0]
    og = O.OracleGel.from_workload(wl)
    gel = B.Gel.from_workload(wl)
    try:
        gel.set_state(xo, np.zeros_like(xo), wl.poses[STEPS - 1])
        rng = np.random.default_rng(3)
        m = np.column_stack([rng.uniform(0.0, 0.018, 80), rng.uniform(0.0, 0.024, 80)])
        pg, fg = gel.markers(m)
        po, fo = og.markers(xo, m)
        assert np.array_equal(fg, fo) and fg.all()
        assert np.abs(pg - po).max() <= 1e-15
        grid = dict(nx=64, ny=80, x0=-0.5e-3, y0=-0.6e-3, dx=0.3e-3, dy=0.315e-3)
        hg = gel.height_map(**grid)
        ho = og.height_map(xo, grid["nx"], grid["ny"], grid["x0"], grid["y0"], grid["dx"], grid["dy"])
    finally:
        gel.close()
    assert np.array_equal(np.isnan(hg), np.isnan(ho))
    ok = ~np.isnan(ho)
    assert np.abs(hg[ok] - ho[ok]).max() <= 1e-15
    # the gel bulges by microns around the ball; the ball itself (from 2 d_hat above the top face
    # up) never shows
    assert np.nanmax(hg) < W.gel_grid(*W.GRID_SMALL[0], W.GRID_SMALL[1]).top + W.DHAT


def test_full_size_soft_ball_state_matches_oracle():
    """The benchmark's soft-ball scene at full size (the 41x51x9 gel + a 20^3 ball + plate): after
    the GPU's first steps of the squeeze, the oracle evaluates the GPU's state itself -- its
    brute-force pair scan gives the active pairs by type (rigid and soft-soft) that the GPU counts,
    and the energy and gradient of the step's potential there agree."""
    O.set_threads(0)
    wl = W.gel_ball(20)
    og = O.OracleGel.from_workload(wl)
    gel = B.Gel.from_workload(wl, stream=torch.cuda.current_stream())
    try:
        for s in range(30):  # the first step that ends with the ball pressed on the gel
            assert gel.step(wl.poses[s], wl.dt) == 0
            x = gel.state()[0]
            pose = wl.poses[s]
            counts = og.pair_counts(x, pose)
            if counts[8] + counts[9] > 0:
                break
        xt = x + 1e-6
        eg, pg = gel.energy(x, xt, wl.dt, pose)
        gg, _ = gel.gradient(x, xt, wl.dt, pose)
    finally:
        gel.close()
    eo, po = og.energy(x, xt, wl.dt, pose)
    go, _ = og.gradient(x, xt, wl.dt, pose)
    print("full-size soft ball after %d steps: active pairs by type (PT, TP, EE, SPT, SEE) %s, GPU %d"
          % (s + 1, list(counts[5:]), pg["active"]))
    assert counts[8] + counts[9] > 0, counts  # the ball presses on the gel
    assert pg["active"] == po["active"] == int(counts[5:].sum()), (pg, po, counts)
    assert abs(pg["barrier"] - po["barrier"]) <= 1e-11 * abs(po["barrier"]), (pg, po)
    assert abs(eg - eo) <= 1e-11 * abs(eo), (eg, eo)
    free = wl.gel.dirichlet == 0
    scale = np.abs(go[free]).max()
    assert np.abs(gg - go)[free].max() <= 1e-7 * scale, np.abs(gg - go)[free].max() / scale
