"""Pins of the FP64 CPU oracle against facts it does not compute itself: finite differences,
textbook linear elasticity, closed-form mesh counts, brute-force closest points, library
eigen-solvers and linear solvers, closed-form ACCD impact times, and physical invariants."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_04776_gb300 import workloads as W

E_, NU_, RHO_ = W.YOUNG, W.POISSON, W.DENSITY
MU = E_ / (2 * (1 + NU_))
LAM = E_ * NU_ / ((1 + NU_) * (1 - 2 * NU_))
HERE = os.path.dirname(os.path.abspath(__file__))


def rand_rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


# ------------------------------------------------------------------ elasticity
def test_rest_tensor_is_isotropic_linear_elasticity():
    """At F = I the Hessian of any consistent hyperelastic model is the linear-elasticity tensor
    C_ijkl = mu (d_ik d_jl + d_il d_jk) + lambda d_ij d_kl (textbook), and Psi = P = 0."""
    s, psi, P, C = O.psi(np.eye(3).ravel(), MU, LAM)
    assert s == 0 and psi == 0.0 and np.all(P == 0.0)
    d = np.eye(3)
    ref = np.zeros((9, 9))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    ref[3 * i + j, 3 * k + l] = MU * (d[i, k] * d[j, l] + d[i, l] * d[j, k]) + LAM * d[i, j] * d[k, l]
    np.testing.assert_allclose(C, ref, rtol=1e-12, atol=1e-9 * MU)


def test_rest_tensor_recovers_young_and_poisson():
    """Uniaxial stress through the rest tensor gives back E and nu (checks the Lame conversion)."""
    _, _, _, C = O.psi(np.eye(3).ravel(), MU, LAM)
    sym = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    Cv = np.array([[C[3 * a + b, 3 * c + d] for (c, d) in sym] for (a, b) in sym])
    Cv[:, 3:] *= 2.0  # engineering shear strains
    S = np.linalg.inv(Cv)
    assert abs(1.0 / S[0, 0] - E_) < 1e-6 * E_
    assert abs(-S[1, 0] / S[0, 0] - NU_) < 1e-9


def test_small_strain_energy_matches_linear_elasticity():
    rng = np.random.default_rng(1)
    for _ in range(5):
        A = rng.normal(size=(3, 3))
        eps = 1e-5 * 0.5 * (A + A.T)
        _, psi, _, _ = O.psi((np.eye(3) + eps).ravel(), MU, LAM)
        lin = MU * np.sum(eps * eps) + 0.5 * LAM * np.trace(eps) ** 2
        assert abs(psi - lin) < 1e-4 * abs(lin)


def test_frame_indifference_and_inversion():
    rng = np.random.default_rng(2)
    for _ in range(5):
        F = np.eye(3) + 0.3 * rng.normal(size=(3, 3))
        if np.linalg.det(F) <= 0.1:
            continue
        R = rand_rot(rng)
        _, a, _, _ = O.psi(F.ravel(), MU, LAM)
        _, b, _, _ = O.psi((R @ F).ravel(), MU, LAM)
        assert abs(a - b) <= 1e-10 * abs(a)
    F = np.diag([1.0, 1.0, -0.5])
    s, _, _, _ = O.psi(F.ravel(), MU, LAM)
    assert s == 1  # det F <= 0 has no energy


def random_tet(rng, scale=1e-3, strain=0.2):
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float) * scale
    X += rng.normal(scale=0.1 * scale, size=(4, 3))
    if np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)) < 0:
        X[[2, 3]] = X[[3, 2]]
    F = np.eye(3) + strain * rng.normal(size=(3, 3))
    while np.linalg.det(F) < 0.3:
        F = np.eye(3) + strain * rng.normal(size=(3, 3))
    x = X @ F.T + rng.normal(scale=scale, size=3)
    return X, x


def test_tet_gradient_and_hessian_central_differences():
    rng = np.random.default_rng(3)
    for _ in range(6):
        X, x = random_tet(rng)
        s, e, g, H = O.tet(X, x, MU, LAM, project=False)
        assert s == 0
        h = 1e-9
        gfd = np.zeros(12)
        Hfd = np.zeros((12, 12))
        for k in range(12):
            xp = x.ravel().copy()
            xm = x.ravel().copy()
            xp[k] += h
            xm[k] -= h
            ep = O.tet(X, xp.reshape(4, 3), MU, LAM, derivs=False)[1]
            em = O.tet(X, xm.reshape(4, 3), MU, LAM, derivs=False)[1]
            gfd[k] = (ep - em) / (2 * h)
            Hfd[:, k] = (O.tet(X, xp.reshape(4, 3), MU, LAM, project=False)[2] -
                         O.tet(X, xm.reshape(4, 3), MU, LAM, project=False)[2]) / (2 * h)
        assert np.max(np.abs(g - gfd)) <= 1e-6 * np.max(np.abs(g))
        assert np.max(np.abs(H - Hfd)) <= 1e-5 * np.max(np.abs(H))
        # translation invariance: forces of one element sum to zero
        assert np.max(np.abs(g.reshape(4, 3).sum(0))) <= 1e-9 * np.max(np.abs(g))


def test_tet_projection_is_psd_and_exact_when_already_psd():
    rng = np.random.default_rng(4)
    n_clamped = 0
    for _ in range(20):
        X, x = random_tet(rng, strain=0.35)
        _, _, _, Hr = O.tet(X, x, MU, LAM, project=False)
        _, _, _, Hp = O.tet(X, x, MU, LAM, project=True)
        w = np.linalg.eigvalsh(Hp)
        assert w.min() >= -1e-10 * w.max()
        if np.linalg.eigvalsh(Hr).min() < -1e-8 * w.max():
            n_clamped += 1
    assert n_clamped > 0  # compression cases exercise the clamp
    X, x = random_tet(rng, strain=0.0)  # pure rigid motion: rest Hessian is PSD
    _, _, _, Hr = O.tet(X, x, MU, LAM, project=False)
    _, _, _, Hp = O.tet(X, x, MU, LAM, project=True)
    np.testing.assert_allclose(Hp, Hr, atol=1e-9 * np.abs(Hr).max())


# ------------------------------------------------------------------ eigen / projection / solver
def test_psd_projection_matches_library_eigh():
    rng = np.random.default_rng(5)
    for n in (3, 6, 9, 12):
        A = rng.normal(size=(n, n))
        A = A + A.T
        w, V = np.linalg.eigh(A)
        ref = (V * np.maximum(w, 0)) @ V.T
        P = O.psd_project(A)
        np.testing.assert_allclose(P, ref, atol=1e-12 * np.abs(A).max())
        np.testing.assert_allclose(O.psd_project(P), P, atol=1e-12 * np.abs(A).max())  # idempotent
        wo, _ = O.eigh(A)
        np.testing.assert_allclose(np.sort(wo), w, atol=1e-12 * np.abs(A).max())


def test_pcg_matches_dense_solve():
    import scipy.sparse as sp
    rng = np.random.default_rng(6)
    n = 60
    B = sp.random(n, n, density=0.1, random_state=7, format="csr")
    A = (B @ B.T + sp.eye(n) * 2.0).tocsr()
    b = rng.normal(size=n)
    it, x = O.pcg_csr(A.indptr, A.indices, A.data, b, tol=1e-13)
    assert it > 0
    np.testing.assert_allclose(x, np.linalg.solve(A.toarray(), b), rtol=1e-9, atol=1e-11)


# ------------------------------------------------------------------ distances
def brute_pt(P, n=240):
    p, t0, t1, t2 = P
    u = np.linspace(0, 1, n)
    a, b = np.meshgrid(u, u)
    m = a + b <= 1
    q = t0 + a[m, None] * (t1 - t0) + b[m, None] * (t2 - t0)
    return np.min(np.sum((q - p) ** 2, 1))


def brute_ee(P, n=600):
    a0, a1, b0, b1 = P
    u = np.linspace(0, 1, n)
    s, t = np.meshgrid(u, u)
    pa = a0 + s.ravel()[:, None] * (a1 - a0)
    pb = b0 + t.ravel()[:, None] * (b1 - b0)
    return np.min(np.sum((pa - pb) ** 2, 1))


def refine_min(fun, x0, bounds, cons=()):
    from scipy.optimize import minimize
    r = minimize(fun, x0, bounds=bounds, constraints=cons, method="SLSQP",
                 options=dict(ftol=1e-30, maxiter=500))
    return r.fun


def test_point_triangle_distance_against_brute_force():
    rng = np.random.default_rng(8)
    types = set()
    for k in range(60):
        P = rng.normal(size=(4, 3))
        d2, ty = O.distance2(0, P)
        types.add(ty[0])
        bf = brute_pt(P)
        p, t0, t1, t2 = P

        def f(l):
            q = t0 + l[0] * (t1 - t0) + l[1] * (t2 - t0)
            return float(np.sum((q - p) ** 2))
        ex = refine_min(f, [1 / 3, 1 / 3], [(0, 1), (0, 1)],
                        ({"type": "ineq", "fun": lambda l: 1 - l[0] - l[1]},))
        assert d2 <= bf + 1e-12
        assert abs(d2 - min(ex, bf)) <= 1e-7 * max(1.0, d2)
    assert types == {0, 1, 2}  # PP, PE and PT regions all reached


def test_edge_edge_distance_against_brute_force():
    rng = np.random.default_rng(9)
    types = set()
    for k in range(60):
        P = rng.normal(size=(4, 3))
        d2, ty = O.distance2(1, P)
        types.add(ty[0])
        a0, a1, b0, b1 = P

        def f(st):
            return float(np.sum((a0 + st[0] * (a1 - a0) - b0 - st[1] * (b1 - b0)) ** 2))
        bf = brute_ee(P)
        ex = refine_min(f, [0.5, 0.5], [(0, 1), (0, 1)])
        assert d2 <= bf + 1e-12
        assert abs(d2 - min(ex, bf)) <= 1e-7 * max(1.0, d2)
    assert types == {0, 1, 3}
    # exactly parallel edges never use the (singular) line-line formula
    P = np.array([[0, 0, 0], [1, 0, 0], [0.2, 0.3, 0.0], [1.4, 0.3, 0.0]], float)
    d2, ty = O.distance2(1, P)
    assert ty[0] != 3 and abs(d2 - 0.09) < 1e-15


# ------------------------------------------------------------------ barrier
def fd_pair(kind, P, dhat, eps_x, h=1e-10):
    s, b, g, H = O.pair_barrier(kind, P, dhat, eps_x)
    gfd = np.zeros(12)
    Hfd = np.zeros((12, 12))
    for k in range(12):
        Pp = P.ravel().copy()
        Pm = P.ravel().copy()
        Pp[k] += h
        Pm[k] -= h
        rp = O.pair_barrier(kind, Pp.reshape(4, 3), dhat, eps_x)
        rm = O.pair_barrier(kind, Pm.reshape(4, 3), dhat, eps_x)
        gfd[k] = (rp[1] - rm[1]) / (2 * h)
        Hfd[:, k] = (rp[2] - rm[2]) / (2 * h)
    return s, b, g, H, gfd, Hfd


PAIR_CASES = {
    # kind, points (metres), expected formula
    "PT": (0, [[0.3e-3, 0.3e-3, 5e-5], [0, 0, 0], [1e-3, 0, 0], [0, 1e-3, 0]], 2),
    "PE": (0, [[0.5e-3, -4e-5, 3e-5], [0, 0, 0], [1e-3, 0, 0], [0, 1e-3, 0]], 1),
    "PP": (0, [[-3e-5, -4e-5, 2e-5], [0, 0, 0], [1e-3, 0, 0], [0, 1e-3, 0]], 0),
    "LL": (1, [[0, 0, 0], [1e-3, 0.1e-3, 0], [0.5e-3, -0.5e-3, 6e-5], [0.4e-3, 0.5e-3, 6e-5]], 3),
    "EE-PE": (1, [[0, 0, 0], [1e-3, 0, 0], [1.02e-3, -0.5e-3, 5e-5], [1.03e-3, 0.5e-3, 6e-5]], 1),
}


@pytest.mark.parametrize("name", sorted(PAIR_CASES))
def test_barrier_central_differences(name):
    kind, P, ftype = PAIR_CASES[name]
    P = np.asarray(P, float)
    d2, ty = O.distance2(kind, P)
    assert ty[0] == ftype and d2 < W.DHAT ** 2
    for eps_x in ([0.0] if kind == 0 else [1e-30, 1e-3 * 1e-6 * 1e-6]):
        s, b, g, H, gfd, Hfd = fd_pair(kind, P, W.DHAT, eps_x)
        assert s == 0 and b > 0
        assert np.max(np.abs(g - gfd)) <= 1e-5 * np.max(np.abs(g))
        assert np.max(np.abs(H - Hfd)) <= 1e-4 * np.max(np.abs(H))
        assert np.max(np.abs(g.reshape(4, 3).sum(0))) <= 1e-9 * np.max(np.abs(g))


def test_barrier_vanishes_smoothly_at_dhat_and_blows_up_at_contact():
    base = np.array([[0.3e-3, 0.3e-3, 0.0], [0, 0, 0], [1e-3, 0, 0], [0, 1e-3, 0]])
    vals = []
    for hgt in (W.DHAT * (1 + 1e-9), W.DHAT * (1 - 1e-4), W.DHAT * 1e-3, W.DHAT * 1e-9):
        P = base.copy()
        P[0, 2] = hgt
        s, b, g, H = O.pair_barrier(0, P, W.DHAT)
        vals.append((s, b, np.abs(g).max()))
    assert vals[0][0] == 1 and vals[0][1] == 0.0
    assert vals[1][1] < 1e-8 * W.DHAT ** 2 and vals[1][2] < 1e-3 * W.DHAT  # C1 at dhat
    assert vals[3][1] > vals[2][1] > 0  # grows toward contact
    P = base.copy()
    P[0, 2] = 0.0
    assert O.pair_barrier(0, P, W.DHAT)[0] == 2


def test_edge_mollifier_kills_parallel_and_leaves_crossing_edges():
    par = np.array([[0, 0, 0], [1e-3, 0, 0], [0.2e-3, 0, 5e-5], [0.8e-3, 1e-12, 5e-5]])
    eps = 1e-3 * 1e-6 * 0.36e-6
    assert O.pair_barrier(1, par, W.DHAT, eps)[1] < 1e-12 * O.pair_barrier(1, par, W.DHAT, 0.0)[1]
    cross = PAIR_CASES["LL"][1]
    a = O.pair_barrier(1, np.asarray(cross), W.DHAT, eps)[1]
    b = O.pair_barrier(1, np.asarray(cross), W.DHAT, 0.0)[1]
    assert a == b


# ------------------------------------------------------------------ ACCD
def test_accd_head_on_closed_form():
    """Point-point head-on approach at speed v from gap d0: the first additive step covers
    (1-s) d0 = 0.9 d0 and the next one would cross below s d0, so toi = 0.9 d0 / v exactly."""
    P = np.array([[0, 0, 1e-4], [0, 0, 0], [1, 0, 0], [0, 1, 0]])  # point above vertex t0
    P[2:] = [[-1e-3, -1e-3, -1e-3], [-1e-3, 1e-3, -1e-3]]  # triangle far below except t0
    P = np.array([[0, 0, 1e-4], [0, 0, 0], [1e-3, -1e-3, -1e-3], [-1e-3, 1e-3, -1e-3]])
    dP = np.zeros((4, 3))
    dP[0, 2] = -2e-4  # closes the 1e-4 gap at t = 0.5
    r, t = O.accd(0, P, dP)
    assert r == 1 and abs(t - 0.9 * 0.5) < 1e-12


def min_dist_along(kind, P, dP, t1, n=2000):
    return min(math.sqrt(O.distance2(kind, P + t * dP)[0]) for t in np.linspace(0, t1, n))


def test_accd_is_conservative():
    rng = np.random.default_rng(10)
    hits = 0
    for k in range(60):
        kind = k % 2
        P = rng.normal(size=(4, 3)) * 1e-3
        dP = rng.normal(size=(4, 3)) * 2e-3
        r, t = O.accd(kind, P, dP)
        assert r in (0, 1)
        if r == 1:
            hits += 1
            assert 0 <= t <= 1
            assert min_dist_along(kind, P, dP, t) > 0
        else:
            assert min_dist_along(kind, P, dP, 1.0) > 0
    assert hits > 5


# ------------------------------------------------------------------ mesh and scene
def load_counts():
    rows = []
    with open(os.path.join(HERE, "golden", "grid_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v) for v in line.split()])
    return rows


@pytest.mark.parametrize("row", load_counts())
def test_surface_counts_and_mass(row):
    nx, ny, nz, nv, nt, sv, st, se = row
    size = (0.02, 0.025, 0.004)
    gel = W.gel_grid(nx, ny, nz, size)
    assert gel.verts.shape[0] == nv and gel.tets.shape[0] == nt
    ind = W.icosphere(0.002, 1)
    og = O.OracleGel(gel.verts, gel.tets, gel.dirichlet, (E_, NU_, RHO_), ind.verts, ind.tris,
                     W.pose((0.01, 0.01, 0.1)))
    info = og.info()
    assert (info["surf_verts"], info["surf_tris"], info["surf_edges"]) == (sv, st, se)
    assert abs(info["total_mass"] - RHO_ * np.prod(size)) < 1e-12 * RHO_ * np.prod(size)
    assert info["ind_edges"] == 120  # icosphere level 1: 80 faces -> 120 edges
    assert abs(info["bbox_diag"] - math.sqrt(sum(s * s for s in size))) < 1e-15


def test_inverted_and_bad_meshes_are_rejected():
    gel = W.gel_grid(3, 3, 2, (0.002, 0.002, 0.001))
    ind = W.icosphere(0.001, 0)
    bad = gel.tets.copy()
    bad[0, [2, 3]] = bad[0, [3, 2]]
    with pytest.raises(O.OracleError) as e:
        O.OracleGel(gel.verts, bad, gel.dirichlet, (E_, NU_, RHO_), ind.verts, ind.tris, W.pose((0, 0, 1)))
    assert e.value.status == 3
    bad = gel.tets.copy()
    bad[0, 0] = 10 ** 6
    with pytest.raises(O.OracleError) as e:
        O.OracleGel(gel.verts, bad, gel.dirichlet, (E_, NU_, RHO_), ind.verts, ind.tris, W.pose((0, 0, 1)))
    assert e.value.status == 1


# ------------------------------------------------------------------ whole-step invariants
def small_scene(depth=0.3e-3, steps=6, seed=0, grid=(6, 6, 3), size=(0.01, 0.01, 0.003), r=0.004):
    gel = W.gel_grid(*grid, size)
    ind = W.icosphere(r, 1)
    c = (0.5 * size[0] + 0.3e-3 * seed, 0.5 * size[1])
    p0, poses = W.press_slide_poses(ind, gel, c, depth, steps)
    return W.Workload("tiny", gel, ind, p0, poses, W.DT)


def test_rest_state_is_a_fixed_point():
    wl = small_scene()
    og = O.OracleGel.from_workload(wl)
    far = W.pose((0.005, 0.005, 0.05))
    og.set_state(wl.gel.verts, np.zeros_like(wl.gel.verts), far)
    info = og.step(far, W.DT)
    x, v, fc, _ = og.state()
    assert info["status"] == 0 and info["newton_iters"] == 0
    assert np.array_equal(x, wl.gel.verts) and np.all(v == 0) and np.all(fc == 0)


def test_step_invariants_and_minimiser():
    """Each step: status OK, no penetration, no inversion, dirichlet vertices untouched, and the
    result is a stationary point of E (free-DOF gradient tiny against the inertia scale)."""
    wl = small_scene()
    og = O.OracleGel.from_workload(wl, newton_tol=1e-7)
    m = og.mass()
    for s in range(len(wl.poses)):
        x0, v0, _, _ = og.state()
        info = og.step(wl.poses[s], wl.dt)
        assert info["status"] == 0
        x, v, fc, pose = og.state()
        assert np.array_equal(x[wl.gel.dirichlet == 1], wl.gel.verts[wl.gel.dirichlet == 1])
        assert info["min_distance"] > 0
        t = wl.gel.tets
        J = np.linalg.det(np.stack([x[t[:, 1]] - x[t[:, 0]], x[t[:, 2]] - x[t[:, 0]], x[t[:, 3]] - x[t[:, 0]]], 2))
        assert J.min() > 0
        h = wl.dt / (2 ** 0)
        if info["substeps"] == 1:
            xt = x0 + h * v0
            g, _ = og.gradient(x, xt, h, pose)
            free = wl.gel.dirichlet == 0
            # stationarity: residual force below the force of moving a vertex by 1e-9 m
            assert np.abs(g[free]).max() <= 1e-9 * (m.max() / h ** 2 + 1e3) + 1e-9
    assert fc[2] < 0  # the indenter pushes the gel down


def test_elastic_forces_are_balanced_by_supports():
    """Translation invariance of the elastic energy: the support reactions at the fixed bottom
    face balance the sum of all other forces at a converged quasi-static state."""
    wl = small_scene(depth=0.2e-3, steps=12)
    og = O.OracleGel.from_workload(wl, newton_tol=1e-10)
    # quasi-static: huge time steps so inertia is negligible
    for p in wl.poses:
        info = og.step(p, 100.0)
        assert info["status"] == 0
    x, v, fc, pose = og.state()
    xt = x.copy()  # inertia term zero at xt = x
    g, fcon = og.gradient(x, xt, 100.0, pose)
    fixed = wl.gel.dirichlet == 1
    reaction = g[fixed].sum(0)  # force the supports exert on the gel (= dE/dx at fixed nodes)
    np.testing.assert_allclose(reaction + fcon, 0.0, atol=1e-6 * abs(fcon[2]))
    assert fcon[2] < 0


def test_affine_patch_test():
    """Linear tets reproduce an affine deformation prescribed on the whole boundary."""
    gel = W.gel_grid(5, 5, 5, (0.004, 0.004, 0.004))
    X = gel.verts
    onb = np.any((X <= 1e-12) | (X >= 0.004 - 1e-12), axis=1).astype(np.uint8)
    A = np.array([[1.02, 0.01, -0.005], [0.0, 0.99, 0.01], [0.003, 0.0, 1.01]])
    xa = X @ A.T + np.array([1e-4, 0, 0])
    ind = W.icosphere(0.001, 0)
    far = W.pose((0.0, 0.0, 1.0))
    og = O.OracleGel(X, gel.tets, onb, (E_, NU_, RHO_), ind.verts, ind.tris, far, newton_tol=1e-9)
    x0 = np.where(onb[:, None] == 1, xa, X)
    og.set_state(x0, np.zeros_like(X), far)
    info = og.step(far, 1e4)
    x, _, _, _ = og.state()
    assert info["status"] == 0
    assert np.abs(x - xa).max() < 1e-10  # vs affine displacements of ~1e-4 m


def test_newton_matches_direct_minimisation():
    """The oracle's Newton step reaches the same minimiser as a general-purpose quasi-Newton
    minimiser (scipy L-BFGS-B) applied to the oracle's own energy and gradient."""
    from scipy.optimize import minimize
    wl = small_scene(depth=0.25e-3, steps=12, grid=(4, 4, 3), size=(0.006, 0.006, 0.003), r=0.003)
    og = O.OracleGel.from_workload(wl, newton_tol=1e-7)
    for s in range(12):
        x0, v0, _, p_prev = og.state()
        info = og.step(wl.poses[s], wl.dt)
        assert info["status"] == 0
        if s >= 6 and info["substeps"] == 1 and info["active_pairs"] > 0:
            break
    x, v, _, pose = og.state()
    # replay that step with L-BFGS from x_n on the same energy
    assert info["substeps"] == 1 and info["active_pairs"] > 0
    h = wl.dt
    xt = x0 + h * v0
    free = wl.gel.dirichlet == 0

    S = 1e-6  # optimise in micrometres around the oracle's answer, energies in micro-joules

    def f(z):
        y = x0.copy()
        y[free] = x[free] + S * z.reshape(-1, 3)
        e, _ = og.energy(y, xt, h, pose)
        if not np.isfinite(e):
            return 1e30, np.zeros_like(z)
        g, _ = og.gradient(y, xt, h, pose)
        return e * 1e6, g[free].ravel() * S * 1e6
    z0 = np.full(3 * int(free.sum()), 0.1)  # start 0.1 um away along every coordinate
    r = minimize(f, z0, jac=True, method="L-BFGS-B",
                 options=dict(maxiter=5000, ftol=1e-30, gtol=1e-16, maxcor=50))
    assert np.abs(r.x).max() * S < 1e-10


# ------------------------------------------------------------------ contact mechanics


def hertz_force(uc, radius):
    """Hertz's solution for a rigid frictionless sphere of `radius` pressed to a depth uc into an
    elastic half-space (Johnson, Contact Mechanics, 1985, Sec. 4.2): F = 4/3 E* sqrt(R) uc^(3/2),
    E* = E / (1 - nu^2)."""
    return 4.0 / 3.0 * E_ / (1.0 - NU_ ** 2) * math.sqrt(radius) * uc ** 1.5


def test_hertz_sphere_indentation_coarse():
    """Rigid spherical cap (R = 3 mm) pressed quasi-statically (time step 1 s) into a 16 x 16 x 8 mm
    block (a >> the 80 um cells under the contact, a << the block): the contact force follows
    Hertz's u^(3/2) law.  A displacement-based mesh this coarse is stiffer than the continuum
    (a lower bound on compliance), so the force may exceed Hertz but not fall below it; the
    refinement study that brings it within 15 % runs on the GPU library (test_gpu_hertz)."""
    half = 8e-3
    wl = W.hertz_block(h0=80e-6, ratio=1.5, half=half, thick=half, dhat=15e-6, step=12e-6)
    X = wl.gel.verts
    c = np.where((np.abs(X[:, 0] - half) < 1e-9) & (np.abs(X[:, 1] - half) < 1e-9) & (X[:, 2] > half - 1e-9))[0]
    assert len(c) == 1
    og = O.OracleGel.from_workload(wl)
    u, F = [], []
    for s in range(len(wl.poses)):
        assert og.step(wl.poses[s], wl.dt)["status"] == 0
        x, _, fc, _ = og.state()
        u.append(X[c[0], 2] - x[c[0], 2])  # surface displacement under the apex
        F.append(-fc[2])
    u, F = np.array(u), np.array(F)
    ratio = F / hertz_force(u, 3e-3)
    assert np.all(ratio[-2:] > 0.95) and np.all(ratio[-2:] < 1.45), ratio
    # the u^(3/2) law between the last two loads
    expo = math.log(F[-1] / F[-2]) / math.log(u[-1] / u[-2])
    assert 1.35 < expo < 1.65, expo


# ------------------------------------------------------------------ lagged friction
# IPC's lagged dissipative friction (Li et al. 2020, Sec. 5): D = mu lambda f0(|u|), u the
# tangential relative displacement of the closest points over the step, lambda the pair's normal
# force at the step start.  f1 = f0' is 1 above eps_v h (Coulomb) and -y^2/(eps_v h)^2 + 2y/(eps_v h)
# below it (static friction as a stiff spring).
def _friction_pair_points(kind, rng, d0):
    """Lagged points of a pair at distance d0 with face-interior (PT) or edge-interior (EE)
    closest points, randomly rotated and shifted."""
    R = rand_rot(rng)
    if kind == 0:
        P = np.array([[0.05, 0.02, 0.0], [-1.0, -0.8, 0.0], [1.2, -0.6, 0.0], [0.1, 1.1, 0.0]]) * 1e-3
        P[0, 2] = d0
    else:
        P = np.array([[-1.0, 0.1, 0.0], [1.1, -0.2, 0.0], [0.2, -1.0, 0.0], [-0.1, 1.2, 0.0]]) * 1e-3
        P[2:, 2] = d0
    return P @ R.T + rng.normal(size=3) * 1e-3


def test_friction_force_is_coulomb_when_sliding_and_a_spring_when_sticking():
    dhat, kappa, mu, eh = 1e-4, 30.0, 0.4, 1e-5
    P = np.array([[0.05e-3, 0.02e-3, 0.3 * dhat], [-1e-3, -0.8e-3, 0.0], [1.2e-3, -0.6e-3, 0.0],
                  [0.1e-3, 1.1e-3, 0.0]])
    # the lagged normal force is the barrier's: kappa |db/dx| on the point (unit distance gradient)
    _, _, gb, _ = O.pair_barrier(0, P, dhat)
    lam_barrier = kappa * np.linalg.norm(gb[:3])
    for du in (np.array([3e-5, -2e-5, 0.0]), np.array([1e-8, 2e-8, 0.0]), np.array([4e-6, 3e-6, 0.0])):
        Pn = P.copy()
        Pn[0] += du
        a, e, g, H, lam = O.friction_pair(0, P, Pn, dhat, kappa, 0.0, mu, eh)
        assert a == 1 and abs(lam - lam_barrier) <= 1e-10 * lam_barrier
        f = -g[:3]
        y = np.linalg.norm(du)
        f1 = 1.0 if y >= eh else 2 * y / eh - (y / eh) ** 2
        assert abs(np.linalg.norm(f) - mu * lam * f1) <= 1e-10 * mu * lam * f1
        # opposite to the slip, in the tangent plane
        assert abs(np.dot(f, du) + np.linalg.norm(f) * y) <= 1e-10 * np.linalg.norm(f) * y
        assert abs(f[2]) <= 1e-12 * np.linalg.norm(f)
        # the triangle takes the reaction
        assert np.abs(g.reshape(4, 3).sum(0)).max() <= 1e-12 * np.abs(g).max()
    # no contact at the step start: no friction
    Pfar = P.copy()
    Pfar[0, 2] = 1.5 * dhat
    assert O.friction_pair(0, Pfar, Pfar + 1e-6, dhat, kappa, 0.0, mu, eh)[0] == 0


@pytest.mark.parametrize("kind", [0, 1])
def test_friction_central_differences(kind):
    rng = np.random.default_rng(11 + kind)
    dhat, kappa, mu, eh = 1e-4, 30.0, 0.3, 2e-5
    for trial in range(4):
        P = _friction_pair_points(kind, rng, rng.uniform(0.2, 0.8) * dhat)
        for scale in (0.2 * eh, 5 * eh):  # sticking and sliding
            Pn = P + rng.normal(size=P.shape) * scale
            a, e, g, H, lam = O.friction_pair(kind, P, Pn, dhat, kappa, 0.0, mu, eh)
            assert a == 1
            h = 1e-9
            gfd = np.zeros(12)
            Hfd = np.zeros((12, 12))
            for i in range(12):
                dp = np.zeros(12)
                dp[i] = h
                ep = O.friction_pair(kind, P, Pn + dp.reshape(4, 3), dhat, kappa, 0.0, mu, eh)
                em = O.friction_pair(kind, P, Pn - dp.reshape(4, 3), dhat, kappa, 0.0, mu, eh)
                gfd[i] = (ep[1] - em[1]) / (2 * h)
                Hfd[:, i] = (ep[2] - em[2]) / (2 * h)
            assert np.abs(g - gfd).max() <= 1e-6 * np.abs(g).max()
            assert np.abs(H - Hfd).max() <= 1e-6 * np.abs(H).max()
            # convex: the Hessian of the lagged friction needs no projection
            assert np.linalg.eigvalsh(0.5 * (H + H.T)).min() >= -1e-9 * np.abs(H).max()


def test_flat_plate_slides_with_coulomb_force():
    """A rigid flat plate pressed on the gel top and slid along +x faster than eps_v: once the gel
    top has sheared up to the friction limit, the tangential contact force is mu times the normal
    force (every contact normal is vertical); without friction the tangential force vanishes."""
    gel = W.gel_grid(6, 6, 3, (0.01, 0.01, 0.003))
    L = 0.03
    plate = W.Indenter(np.array([[-L, -L, 0.0], [L, -L, 0.0], [L, L, 0.0], [-L, L, 0.0]]),
                       np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32), "plate")
    p0, poses = W.press_slide_poses(plate, gel, (0.005, 0.005), 0.15e-3, 6, slide=0.9e-3, n_slide=18)
    wl = W.Workload("plate", gel, plate, p0, poses, W.DT)
    ratios = {}
    for mu in (0.0, 0.5):
        og = O.OracleGel.from_workload(wl, newton_tol=1e-7, friction=mu, eps_v=1e-3)
        for s in range(len(poses)):
            assert og.step(poses[s], wl.dt)["status"] == 0
        _, _, fc, _ = og.state()
        assert fc[2] < 0
        ratios[mu] = (fc[0] / -fc[2], fc[1] / -fc[2])
    # frictionless: only the plate diagonal's edge-edge pairs tilt with the gel top (1e-5 here)
    assert abs(ratios[0.0][0]) <= 1e-4 and abs(ratios[0.0][1]) <= 1e-4
    # with friction (0.5014 / -0.0012 here: the normal forces are lagged by a step and the gel
    # top still creeps sideways a little as it shears)
    assert abs(ratios[0.5][0] - 0.5) <= 0.01 and abs(ratios[0.5][1]) <= 5e-3


# ------------------------------------------------------------------ attachment-driven gel
# The paper's GIPC step sets the attachment points' targets (from the sensor case pose), then
# solves: the Dirichlet vertices move kinematically with their frame.
def test_attachment_rigid_translation_is_exact():
    """Gel moving with its case at constant velocity, no contact: the step is a rigid translation
    (inertia and elasticity both at rest; the Newton solve starts from the moved attachments and
    the old free positions, so it is met to the Newton tolerance, 2.4e-9 m here)."""
    wl = small_scene()
    og = O.OracleGel.from_workload(wl)
    far = W.pose((0.005, 0.005, 0.05))
    v0 = np.array([2e-3, -1e-3, 3e-3])
    X = wl.gel.verts
    og.set_state(X, np.tile(v0, (len(X), 1)), far)
    for s in range(1, 6):
        t = v0 * wl.dt * s
        info = og.step_attached(far, W.pose(t), wl.dt)
        assert info["status"] == 0
        x, v, fc, _ = og.state()
        assert np.abs(x - (X + t)).max() <= 1e-10
        assert np.abs(v - v0).max() <= 1e-10 / wl.dt
        assert np.all(fc == 0)


def test_attachment_motion_is_relative():
    """Pressing the indenter down onto a resting gel equals carrying the gel up (case and all, at
    the indenter's speed) against the resting indenter: the same motion in a frame moving at
    constant velocity (Galilean invariance of the incremental potential).  The indenter sits off
    the gel's mirror planes (a symmetric press is a bifurcation whose branch rounding picks) and
    moves slowly enough that neither run splits its steps."""
    gel = W.gel_grid(6, 6, 3, (0.01, 0.01, 0.003))
    ind = W.icosphere(0.004, 1)
    p0, poses = W.press_slide_poses(ind, gel, (0.0063, 0.0057), 0.15e-3, 20)
    wl = W.Workload("tiny_offset", gel, ind, p0, poses, W.DT)
    a = O.OracleGel.from_workload(wl, newton_tol=1e-7)
    b = O.OracleGel.from_workload(wl, newton_tol=1e-7)
    X = wl.gel.verts
    z0 = wl.pose0[6]
    vz = (wl.poses[0][6] - z0) / wl.dt  # indenter velocity (downwards)
    b.set_state(X, np.tile([0.0, 0.0, -vz], (len(X), 1)), wl.pose0)
    for s in range(len(wl.poses)):
        lift = z0 - wl.poses[s][6]
        ia = a.step(wl.poses[s], wl.dt)
        assert ia["status"] == 0 and ia["substeps"] == 1
        assert b.step_attached(wl.pose0, W.pose((0.0, 0.0, lift)), wl.dt)["status"] == 0
        xa, _, fa, _ = a.state()
        xb, _, fb, _ = b.state()
        assert np.abs(xb - np.array([0.0, 0.0, lift]) - xa).max() <= 1e-9
        assert np.abs(fb - fa).max() <= 1e-6 * np.abs(fa).max()
    assert fa[2] < 0


# ------------------------------------------------------------------ gel-surface readout
def _readout_gel():
    wl = W.small_gel_sphere(0)
    return wl, O.OracleGel.from_workload(wl)


def test_readout_at_rest():
    wl, og = _readout_gel()
    X = wl.gel.verts
    top = X[:, 2].max()
    rng = np.random.default_rng(5)
    m = np.column_stack([rng.uniform(0.0, 0.018, 50), rng.uniform(0.0, 0.024, 50)])
    pos, found = og.markers(X, m)
    assert found.all()
    assert np.abs(pos[:, :2] - m).max() <= 1e-15 and np.abs(pos[:, 2] - top).max() <= 1e-15
    _, f_off = og.markers(X, np.array([[0.019, 0.01], [-0.001, 0.01]]))
    assert not f_off.any()
    # pixel centres from -0.5 mm in 1 mm steps: rows (y) 1..24 and columns (x) 1..18 lie on the gel
    hm = og.height_map(X, 20, 26, -0.001, -0.001, 0.001, 0.001)
    assert np.abs(hm[1:25, 1:19] - top).max() <= 1e-15
    assert np.isnan(hm[0, :]).all() and np.isnan(hm[:, 0]).all()
    assert np.isnan(hm[25, :]).all() and np.isnan(hm[:, 19]).all()


def test_readout_follows_an_affine_deformation_exactly():
    wl, og = _readout_gel()
    X = wl.gel.verts
    top = X[:, 2].max()
    rng = np.random.default_rng(6)
    A = np.eye(3) + rng.uniform(-0.05, 0.05, size=(3, 3))
    b = rng.uniform(-1e-3, 1e-3, size=3)
    x = X @ A.T + b
    m = np.column_stack([rng.uniform(0.001, 0.017, 40), rng.uniform(0.001, 0.023, 40)])
    pos, found = og.markers(x, m)
    assert found.all()
    want = np.column_stack([m, np.full(len(m), top)]) @ A.T + b
    assert np.abs(pos - want).max() <= 1e-15 * 1e3 * 0.03
    # height of the mapped top plane at pixel centres well inside its image
    nx, ny, x0, y0, dx, dy = 30, 40, 0.002, 0.003, 0.0004, 0.0004
    hm = og.height_map(x, nx, ny, x0, y0, dx, dy)
    Axy, Axz = A[:2, :2], A[:2, 2]
    for j in range(ny):
        for i in range(nx):
            p = np.array([x0 + (i + 0.5) * dx, y0 + (j + 0.5) * dy])
            Xxy = np.linalg.solve(Axy, p - b[:2] - Axz * top)
            z = A[2, :2] @ Xxy + A[2, 2] * top + b[2]
            assert abs(hm[j, i] - z) <= 1e-15 * 1e3 * 0.01


def test_height_map_at_vertices_is_the_vertex_height():
    """Top vertices displaced vertically by a smooth bump: a pixel centred on a vertex reads the
    vertex's height (every covering triangle interpolates to it)."""
    wl, og = _readout_gel()
    X = wl.gel.verts.copy()
    top = X[:, 2].max()
    x = X.copy()
    t = np.abs(X[:, 2] - top) < 1e-12
    x[t, 2] -= 3e-4 * np.exp(-((X[t, 0] - 0.009) ** 2 + (X[t, 1] - 0.012) ** 2) / (4e-3) ** 2)
    hm = og.height_map(x, 10, 13, -0.001, -0.001, 0.002, 0.002)  # pixel centres on the 2 mm grid
    for k in np.nonzero(t)[0]:
        i, j = int(round(X[k, 0] / 0.002)), int(round(X[k, 1] / 0.002))
        assert abs(hm[j, i] - x[k, 2]) <= 1e-15


def test_oracle_threads_do_not_change_results():
    """The oracle's parallel loops only write per-element results and every sum is taken serially
    in index order: one thread and all threads give bitwise the same trajectory."""
    wl = W.small_gel_sphere(4)
    runs = []
    for threads in (1, 0):
        O.set_threads(threads)
        og = O.OracleGel.from_workload(wl, newton_tol=1e-7)
        xs = []
        for s in range(6):  # the sphere starts d_hat above the gel: contact from the first step
            info = og.step(wl.poses[s], wl.dt)
            assert info["status"] == 0
            xs.append(og.state()[0].copy())
        runs.append((np.array(xs), info["active_pairs"]))
    O.set_threads(0)
    assert runs[0][1] > 0
    assert np.array_equal(runs[0][0], runs[1][0])


# ---- pins of the barrier value, the candidate rule and the stationarity rule -------------------

def north_star_barrier(d, dhat):
    """b(d) = -(d - dhat)^2 ln(d / dhat) for 0 < d < dhat, 0 beyond (the task's barrier)."""
    return -(d - dhat) ** 2 * math.log(d / dhat) if d < dhat else 0.0


def barrier_geometries(d):
    """Hand-built point-triangle and edge-edge configurations whose distance is d by construction,
    one per closest-feature kind: point-face, point-edge, point-vertex, edge-edge (interior
    points of both) and edge-edge (an endpoint against the other edge's interior)."""
    tri = np.array([[0.0, 0.0, 0.0], [1e-3, 0.0, 0.0], [0.0, 1e-3, 0.0]])
    u = np.array([1.0, 1.0, 0.0]) / math.sqrt(2.0)  # in-plane outward normal of the edge t1-t2
    mid = 0.5 * (tri[1] + tri[2])
    out = {
        "PT face": (0, np.vstack([[2e-4, 2e-4, d], tri])),
        "PT edge": (0, np.vstack([mid + 0.6 * d * u + 0.8 * d * np.array([0.0, 0.0, 1.0]), tri])),
        "PT vertex": (0, np.vstack([[-0.5 * d, -0.5 * d, -d / math.sqrt(2.0)], tri])),
        "EE interior": (1, np.array([[-5e-4, 0.0, 0.0], [5e-4, 0.0, 0.0], [0.0, -5e-4, d], [0.0, 5e-4, d]])),
        "EE endpoint": (1, np.array([[-5e-4, 0.0, 0.0], [5e-4, 0.0, 0.0], [0.0, 0.6 * d, 0.8 * d],
                                     [0.0, 0.6 * d + 1e-3, 0.8 * d]])),
    }
    return out


@pytest.mark.parametrize("d", [1e-7, 3e-6, 2e-5, 6e-5, 9.5e-5, 1.2e-4])
def test_barrier_value_at_known_distances(d):
    dhat = 1e-4
    for name, (kind, P) in barrier_geometries(d).items():
        d2, _ = O.distance2(kind, P)
        assert abs(math.sqrt(d2) - d) <= 1e-12 * d, name
        eps_x = 1e-3 * np.sum((P[1] - P[0]) ** 2) * np.sum((P[3] - P[2]) ** 2) if kind == 1 else 0.0
        s, b, _, _ = O.pair_barrier(kind, P, dhat, eps_x)
        want = north_star_barrier(d, dhat)
        assert abs(b - want) <= 1e-9 * abs(want) + 1e-300, (name, b, want)
        assert (s == 1) == (d >= dhat), name


def _quat_R(q):
    w, x, y, z = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _boundary(tets):
    """Boundary triangles (faces of exactly one tet), their vertices and edges."""
    f = np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]], tets[:, [0, 1, 3]], tets[:, [0, 1, 2]]])
    key = np.sort(f, axis=1)
    uniq, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    tris = uniq[cnt == 1]
    e = np.sort(np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [0, 2]]]), axis=1)
    return np.unique(tris.ravel()), tris, np.unique(e, axis=0)


def _point_segment(p, a, b):
    ab = b - a
    t = np.clip(np.einsum("...i,...i", p - a, ab) / np.einsum("...i,...i", ab, ab), 0.0, 1.0)
    return np.linalg.norm(p - (a + t[..., None] * ab), axis=-1)


def _point_triangle(p, a, b, c):
    """Distance point-triangle: plane distance when the projection falls inside the triangle,
    otherwise the nearest of the three edges."""
    n = np.cross(b - a, c - a)
    nn = np.einsum("...i,...i", n, n)
    w = p - a
    dist = np.einsum("...i,...i", w, n)
    q = p - (dist / nn)[..., None] * n
    inside = np.ones(q.shape[:-1], dtype=bool)
    for u, v in ((a, b), (b, c), (c, a)):
        inside &= np.einsum("...i,...i", np.cross(v - u, q - u), n) >= 0.0
    plane = np.abs(dist) / np.sqrt(nn)
    edges = np.minimum(np.minimum(_point_segment(p, a, b), _point_segment(p, b, c)), _point_segment(p, c, a))
    return np.where(inside, plane, edges)


def _segment_segment(a0, a1, b0, b1):
    """Distance between segments: the line-line closest points when both fall inside the
    segments, otherwise the nearest endpoint-to-segment distance."""
    u, v, w0 = a1 - a0, b1 - b0, a0 - b0
    A, B, C = (np.einsum("...i,...i", u, u), np.einsum("...i,...i", u, v), np.einsum("...i,...i", v, v))
    D, E = np.einsum("...i,...i", u, w0), np.einsum("...i,...i", v, w0)
    den = A * C - B * B
    with np.errstate(divide="ignore", invalid="ignore"):
        s = (B * E - C * D) / den
        t = (A * E - B * D) / den
    ok = (den > 1e-14 * A * C) & (s > 0) & (s < 1) & (t > 0) & (t < 1)
    s, t = np.where(ok, s, 0.0), np.where(ok, t, 0.0)
    pl = np.linalg.norm(w0 + s[..., None] * u - t[..., None] * v, axis=-1)
    ends = np.minimum.reduce([_point_segment(a0, b0, b1), _point_segment(a1, b0, b1),
                              _point_segment(b0, a0, a1), _point_segment(b1, a0, a1)])
    return np.where(ok, np.minimum(pl, ends), ends)


def _near(alo, ahi, blo, bhi, pad):
    return np.all((alo - pad <= bhi) & (blo - pad <= ahi), axis=-1)


@pytest.mark.parametrize("case", ["sphere", "prism"])
def test_candidate_rule_and_active_set_against_all_pairs(case):
    """Every primitive pair (gel surface vertex / indenter triangle, indenter vertex / gel surface
    triangle, gel surface edge / indenter edge) is scanned with plain numpy: the pairs whose
    bounding boxes come within d_hat on every axis (R20) must be exactly the oracle's candidates,
    and the pairs closer than d_hat exactly its active pairs."""
    if case == "sphere":
        wl, steps = W.small_gel_sphere(0), 12
    else:
        wl, steps = W.mini_gel(3, grid=W.GRID_SMALL, kind="prism", depth=0.6e-3, n_press=8, slide=0.0,
                               n_slide=0), 6
    og = O.OracleGel.from_workload(wl)
    for s in range(steps):
        assert og.step(wl.poses[s], wl.dt)["status"] == 0
    x, _, _, pose = og.state()
    oc = og.pair_counts(x, pose)
    IW = wl.indenter.verts @ _quat_R(pose[:4]).T + pose[4:]
    sv, st, se = _boundary(wl.gel.tets)
    itris = wl.indenter.tris
    ie = np.unique(np.sort(np.concatenate([itris[:, [0, 1]], itris[:, [1, 2]], itris[:, [0, 2]]]), axis=1), axis=0)
    dhat = wl.dhat
    P = x[sv][:, None, :]
    T = IW[itris][None, :, :, :]
    cand_pt = _near(P, P, T.min(axis=2), T.max(axis=2), dhat)
    d_pt = _point_triangle(P, T[:, :, 0], T[:, :, 1], T[:, :, 2])
    Q = IW[:, None, :]
    G = x[st][None, :, :, :]
    cand_tp = _near(G.min(axis=2), G.max(axis=2), Q, Q, dhat)
    d_tp = _point_triangle(Q, G[:, :, 0], G[:, :, 1], G[:, :, 2])
    Ea = x[se][:, None, :, :]
    Eb = IW[ie][None, :, :, :]
    cand_ee = _near(Ea.min(axis=2), Ea.max(axis=2), Eb.min(axis=2), Eb.max(axis=2), dhat)
    d_ee = _segment_segment(Ea[:, :, 0], Ea[:, :, 1], Eb[:, :, 0], Eb[:, :, 1])
    mine = [int(cand_pt.sum()), int(cand_tp.sum()), int(cand_ee.sum()), 0, 0,
            int((d_pt < dhat).sum()), int((d_tp < dhat).sum()), int((d_ee < dhat).sum()), 0, 0]
    assert sum(mine[5:]) > 0 and (case == "sphere" or mine[7] > 0)
    assert list(oc) == mine, (list(oc), mine)


def test_soft_soft_candidates_and_active_set_against_all_pairs():
    """A soft ball squeezed between the gel and a plate (two mesh components): every surface
    vertex against every surface triangle of the other body, and every pair of surface edges of
    different bodies, scanned with plain numpy (components from scipy's graph routine, not the
    oracle's union-find): the box rule (R20) picks exactly the oracle's SPT and SEE candidates, the
    distance below d_hat exactly its active ones; the rigid pairs are still counted as before."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    wl = W.gel_ball(6, grid=W.GRID_SMALL, n_press=10, n_slide=0, depth=0.6e-3)
    og = O.OracleGel.from_workload(wl)
    for s in range(4):
        assert og.step(wl.poses[s], wl.dt)["status"] == 0
    x, _, _, pose = og.state()
    oc = og.pair_counts(x, pose)
    tets = wl.gel.tets
    n = len(x)
    rows = np.repeat(tets[:, :1], 3, axis=1).ravel()
    adj = sp.coo_matrix((np.ones(len(rows)), (rows, tets[:, 1:].ravel())), shape=(n, n))
    ncomp, comp = connected_components(adj, directed=False)
    assert ncomp == 2 and og.components()[0] == 2
    assert np.array_equal(og.components()[1] == og.components()[1][0], comp == comp[0])
    sv, st, se = _boundary(tets)
    dhat = wl.dhat
    P = x[sv][:, None, :]
    T = x[st][None, :, :, :]
    other = comp[sv][:, None] != comp[st[:, 0]][None, :]
    cand_spt = _near(P, P, T.min(axis=2), T.max(axis=2), dhat) & other
    i, k = np.nonzero(cand_spt)
    d_spt = _point_triangle(x[sv[i]], x[st[k, 0]], x[st[k, 1]], x[st[k, 2]])
    E = x[se]
    lo, hi = E.min(axis=1), E.max(axis=1)
    cand_see = _near(lo[:, None], hi[:, None], lo[None], hi[None], dhat)
    cand_see &= comp[se[:, 0]][:, None] != comp[se[:, 0]][None, :]
    cand_see = np.triu(cand_see, 1)
    a, b = np.nonzero(cand_see)
    d_see = _segment_segment(x[se[a, 0]], x[se[a, 1]], x[se[b, 0]], x[se[b, 1]])
    mine_ss = [len(i), len(a), int((d_spt < dhat).sum()), int((d_see < dhat).sum())]
    assert mine_ss[2] > 0 and mine_ss[3] > 0, mine_ss  # the ball touches the gel by step 4
    assert [oc[3], oc[4], oc[8], oc[9]] == mine_ss, (list(oc), mine_ss)
    assert oc[5] + oc[6] + oc[7] > 0  # and the plate touches the ball


def _ball_into(v0, steps, kappa, tol):
    """READING R25 pin: a soft ball falling (gravity, initial velocity v0) onto (a) the gel held
    fixed in the same mesh (soft-soft pairs) and (b) the ball alone onto a rigid indenter made of
    the gel's surface at rest (rigid pairs), both with the same absolute Newton tolerance; returns
    the ball's positions of each step in both and the most active pairs of each rigid type in (b)."""
    gel = W.gel_grid(*W.GRID_SMALL[0], W.GRID_SMALL[1])
    c = (0.009, 0.012, gel.top + 2 * W.DHAT + 3e-3)
    ball = W.ball_mesh(6, 3e-3, c)
    far = np.array([1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0])  # the plate of (a), out of reach
    plate = W.flat_plate(0.004, 3)
    nb = len(ball.verts)
    gel.dirichlet[:] = 1
    both = W.join_meshes(gel, ball)

    def diag(v):
        return float(np.linalg.norm(v.max(axis=0) - v.min(axis=0)))

    kw = dict(dhat=W.DHAT, kappa=kappa, gravity=(0.0, 0.0, -9.81), newton_max=2000)
    a = O.OracleGel(both.verts, both.tets, both.dirichlet, (E_, NU_, RHO_), plate.verts, plate.tris, far,
                    newton_tol=tol, **kw)
    sv, st, _ = _boundary(gel.tets)
    remap = np.full(len(gel.verts), -1)
    remap[sv] = np.arange(len(sv))
    ident = np.array([1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    b = O.OracleGel(ball.verts, ball.tets, ball.dirichlet, (E_, NU_, RHO_), gel.verts[sv], remap[st], ident,
                    newton_tol=tol * diag(both.verts) / diag(ball.verts), **kw)
    v = np.tile(v0, (nb, 1))
    a.set_state(both.verts, np.concatenate([np.zeros_like(gel.verts), v]), far)
    b.set_state(ball.verts, v, ident)
    xa, xb, most = [], [], np.zeros(3, dtype=int)
    for s in range(steps):
        ra, rb = a.step(far, W.DT), b.step(ident, W.DT)
        assert ra["status"] == 0 and rb["status"] == 0
        assert ra["active_pairs"] == rb["active_pairs"]
        most = np.maximum(most, b.pair_counts(b.state()[0], ident)[5:8])
        xa.append(a.state()[0][len(gel.verts):])
        xb.append(b.state()[0])
    return np.array(xa), np.array(xb), most


def test_soft_soft_contact_against_a_held_body_is_rigid_contact():
    """Contact between two deformable bodies uses the same barrier on the same primitive
    distances as contact with a rigid body (Sec. 2's GIPC pipeline, soft-to-soft): a ball dropped
    on a gel whose vertices are all held must move as the ball alone dropped on a rigid obstacle
    whose surface is the gel's surface, to the Newton tolerance.  Every rigid pair type is active
    in the second scene, so a missing soft-soft direction (gel vertex vs ball triangle, ball vertex
    vs gel triangle), a missing edge-edge type or another mollifier changes the trajectory."""
    xa, xb, most = _ball_into(np.array([0.01, 0.0, -0.05]), 6, 500.0, 1e-7)
    assert np.all(most > 0), most
    err = np.abs(xa - xb).max()
    assert err < 1e-9, err


def test_soft_soft_contact_conserves_momentum():
    """Two free balls (no held vertex, no gravity) thrown at each other: the elastic and the
    soft-soft barrier forces are internal (each pair's gradient sums to zero over its four points),
    so implicit Euler keeps the total momentum sum m_i v_i (to the Newton tolerance)."""
    b1 = W.ball_mesh(5, 3e-3, (0.0, 0.0, 0.0))
    b2 = W.ball_mesh(5, 3e-3, (0.0015, 0.0, 6e-3 + 3 * W.DHAT))
    both = W.join_meshes(b1, b2)
    far = np.array([1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0])
    plate = W.flat_plate(0.004, 3)
    og = O.OracleGel(both.verts, both.tets, both.dirichlet, (E_, NU_, RHO_), plate.verts, plate.tris, far,
                     dhat=W.DHAT, kappa=500.0, newton_tol=3e-7, newton_max=2000)
    n1 = len(b1.verts)
    v = np.zeros_like(both.verts)
    v[:n1] = (0.0, 0.0, 0.05)
    v[n1:] = (0.0, 0.0, -0.05)
    og.set_state(both.verts, v, far)
    m = og.mass()
    p0 = (m[:, None] * v).sum(axis=0)
    act, worst = 0, 0.0
    for s in range(5):
        r = og.step(far, W.DT)
        assert r["status"] == 0
        act = max(act, r["active_pairs"])
        vs = og.state()[1]
        dp = np.abs((m[:, None] * vs).sum(axis=0) - p0).max()
        worst = max(worst, dp / (0.5 * m.sum() * 0.05))  # against one ball's momentum
    print("soft-soft collision: relative momentum change %.2e, most active pairs %d" % (worst, act))
    assert act > 10, act
    assert worst < 1e-12, worst


def test_stationarity_rule_both_sides():
    """READING R8b: a line search that finds no decrease ends the solve as converged only when the
    model decrease -g.p is at most 1e-10 |E|; a larger one is a failed step."""
    for E in (3.7e-6, -2.0, 1.0):
        tol = 1e-10 * abs(E)
        assert O.stationary_rule(-0.5 * tol, E)
        assert O.stationary_rule(-tol, E)
        assert O.stationary_rule(0.0, E)
        assert not O.stationary_rule(-2.0 * tol, E)
        assert not O.stationary_rule(-1e3 * tol, E)


# ---------------- adaptive barrier stiffness (READING R5b) ----------------
def _weak_barrier_run(adapt, steps):
    """The sphere press of the 10x13x4 gel with kappa at 1 % of the fixed rule (the indenter's
    next placement eventually meets a gel surface the weak barrier let come too close)."""
    wl = W.small_gel_sphere(1)
    k0 = O.OracleGel.from_workload(wl).info()["kappa"] * 0.01
    og = O.OracleGel.from_workload(wl, kappa=k0, kappa_adapt_max=adapt, kappa_adapt_dmin=1e-5)
    infos = []
    for s in range(steps):
        infos.append(og.step(wl.poses[s], wl.dt))
        if infos[-1]["status"] != 0:
            break
    return og, k0, infos


def test_adaptive_kappa_carries_a_press_a_weak_fixed_barrier_cannot():
    O.set_threads(2)
    _, k0, fixed = _weak_barrier_run(0.0, 6)
    assert [i["status"] for i in fixed] == [0, 0, 0, 0, 4], fixed[-1]  # TX_ERR_INFEASIBLE at step 4
    assert all(i["kappa"] == k0 and i["kappa_doublings"] == 0 for i in fixed)
    og, k0, ad = _weak_barrier_run(100.0, 8)
    assert all(i["status"] == 0 for i in ad), ad[-1]
    # kappa = k0 2^n, at most 100 k0, and it doubled after a step exactly when that step ended nearer
    # than 10 um and nearer than the step before (the first step has no predecessor)
    prev_d, kap = math.inf, k0
    for i in ad:
        want = i["min_distance"] < 1e-5 and i["min_distance"] < prev_d and kap < 100.0 * k0
        assert i["kappa_doublings"] == int(want), i
        kap = min(2.0 * kap, 100.0 * k0) if want else kap
        assert abs(i["kappa"] - kap) <= 1e-12 * kap, (i["kappa"], kap)
        prev_d = i["min_distance"]
    assert sum(i["kappa_doublings"] for i in ad) >= 3
    og.reset()  # reset returns kappa to its initial value
    wl = W.small_gel_sphere(1)
    assert og.step(wl.poses[0], wl.dt)["kappa"] == k0


@pytest.mark.parametrize("n,nv,nt", [(10, 1000, 4374), (20, 8000, 41154), (23, 12167, 63888)])
def test_soft_ball_mesh_sizes_and_shape(n, nv, nt):
    """The soft-ball meshes of the Table 3 comparison: the documented vertex and tet counts, every
    tet positively oriented, and the cube's faces carried onto the sphere (every boundary vertex at
    the radius, every vertex inside it)."""
    r, c = 4e-3, np.array([0.01, 0.012, 0.006])
    b = W.ball_mesh(n, r, c)
    assert (len(b.verts), len(b.tets)) == (nv, nt)
    e = [b.verts[b.tets[:, k]] - b.verts[b.tets[:, 0]] for k in (1, 2, 3)]
    assert np.einsum("ij,ij->i", np.cross(e[0], e[1]), e[2]).min() > 0.0
    sv, _, _ = _boundary(b.tets)
    rad = np.linalg.norm(b.verts - c, axis=1)
    assert np.abs(rad[sv] - r).max() <= 1e-15 * 10 and rad.max() <= r * (1 + 1e-14)
    assert not b.dirichlet.any()


def test_body_numbering_and_a_vertex_in_no_tet():
    """Bodies are the tet mesh's connected components, numbered in the order of their first vertex
    in a tet; a vertex in no tet belongs to no body (it joins body 0 and is in no pair).  Here a
    stray vertex comes first, then two balls: two bodies, the first ball is body 0 (the gelpad
    slot of the readouts), and the stray vertex is counted in neither."""
    b1 = W.ball_mesh(4, 2e-3, (0.0, 0.0, 0.0))
    b2 = W.ball_mesh(4, 2e-3, (0.0, 0.0, 5e-3))
    both = W.join_meshes(b1, b2)
    verts = np.vstack([[[1.0, 1.0, 1.0]], both.verts])
    tets = (both.tets + 1).astype(np.int32)
    plate = W.flat_plate(0.004, 3)
    far = np.array([1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0])
    og = O.OracleGel(verts, tets, np.zeros(len(verts), dtype=np.uint8), (E_, NU_, RHO_), plate.verts, plate.tris,
                     far, dhat=W.DHAT, kappa=500.0)
    n, comp = og.components()
    assert n == 2
    assert comp[0] == 0 and np.all(comp[1:1 + len(b1.verts)] == 0) and np.all(comp[1 + len(b1.verts):] == 1)
