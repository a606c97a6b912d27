"""Kernel-level parity: per-tet elastic terms, per-pair barrier terms and ACCD on the GPU
(through the C ABI's unit entry points) against the FP64 oracle, element by element."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2411_04776_gb300 import binding as B  # noqa: E402
from paper_2411_04776_gb300 import workloads as W  # noqa: E402

MU = W.YOUNG / (2 * (1 + W.POISSON))
LAM = W.YOUNG * W.POISSON / ((1 + W.POISSON) * (1 - 2 * W.POISSON))


def random_tets(n, seed, strain):
    rng = np.random.default_rng(seed)
    Xs, xs = [], []
    while len(Xs) < n:
        X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * 1e-3 + rng.normal(scale=1e-4, size=(4, 3))
        if np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], 1)) <= 0:
            X[[2, 3]] = X[[3, 2]]
        F = np.eye(3) + strain * rng.normal(size=(3, 3))
        if np.linalg.det(F) < 0.2:
            continue
        Xs.append(X)
        xs.append(X @ F.T + rng.normal(scale=1e-3, size=3))
    return np.array(Xs), np.array(xs)


@pytest.mark.parametrize("strain", [0.0, 0.02, 0.3])
def test_tet_kernel_matches_oracle(strain):
    n = 300
    X, x = random_tets(n, 7, strain)
    Xd = torch.tensor(X.reshape(n, 12), device="cuda")
    xd = torch.tensor(x.reshape(n, 12), device="cuda")
    e, g, H = B.tx_eval_tets(Xd, xd, MU, LAM, project=True)
    torch.cuda.synchronize()
    e, g, H = e.cpu().numpy(), g.cpu().numpy(), H.cpu().numpy().reshape(n, 12, 12)
    for t in range(n):
        s, eo, go, Ho = O.tet(X[t], x[t], MU, LAM, project=True)
        assert s == 0
        # natural force scale of the element: V (mu + lambda) |grad N|; the GPU forms
        # P = mu F + (lambda ln J - mu) F^-T, whose terms cancel to O(eps) near rest
        vol = abs(np.linalg.det(np.stack([X[t][1] - X[t][0], X[t][2] - X[t][0], X[t][3] - X[t][0]], 1))) / 6
        fscale = vol * (MU + LAM) * np.abs(np.linalg.inv(np.stack([X[t][1] - X[t][0], X[t][2] - X[t][0],
                                                                    X[t][3] - X[t][0]], 1))).max()
        assert abs(e[t] - eo) <= 1e-12 * max(abs(eo), 1e-30) + 1e-25
        assert np.abs(g[t] - go).max() <= 1e-10 * np.abs(go).max() + 1e-13 * fscale
        assert np.abs(H[t] - Ho).max() <= 1e-9 * np.abs(Ho).max()


def random_pairs(n, seed):
    """Point-triangle and edge-edge pairs within dhat, covering every closest-feature type."""
    rng = np.random.default_rng(seed)
    dhat = W.DHAT
    kinds, Ps = [], []
    while len(Ps) < n:
        kind = len(Ps) % 2
        P = rng.normal(scale=0.5e-3, size=(4, 3))
        if kind == 0:
            nrm = np.cross(P[2] - P[1], P[3] - P[1])
            nrm /= np.linalg.norm(nrm)
            if len(Ps) % 6 == 0:
                # beyond a corner: the closest feature is the vertex P[1]
                out = -(P[2] - P[1]) - (P[3] - P[1])
                q = P[1] + 0.02 * out / np.linalg.norm(out) * dhat / 1e-4 * 1e-3
                P[0] = q + nrm * rng.uniform(-0.5, 0.5) * dhat
                P[0] = P[1] + (P[0] - P[1]) * (0.5 * dhat / np.linalg.norm(P[0] - P[1]))
            else:
                # near the triangle (face interior or beyond an edge)
                b = rng.dirichlet([1, 1, 1]) * rng.uniform(0.6, 1.3)
                q = P[1] + b[1] * (P[2] - P[1]) + b[2] * (P[3] - P[1])
                P[0] = q + nrm * rng.uniform(0.05, 0.95) * dhat + rng.normal(scale=2e-5, size=3)
        else:
            s, t = rng.uniform(-0.2, 1.2, size=2)
            pa = P[0] + s * (P[1] - P[0])
            pb = P[2] + t * (P[3] - P[2])
            shift = pa - pb + rng.normal(scale=1.0, size=3) * 0.5 * dhat / np.sqrt(3)
            P[2:] += shift
        d2, _ = O.distance2(kind, P)
        if 1e-14 < d2 < dhat * dhat:
            kinds.append(kind)
            Ps.append(P)
    return np.array(kinds, dtype=np.int32), np.array(Ps)


def test_pair_kernel_matches_oracle():
    n = 400
    kinds, P = random_pairs(n, 11)
    masks = np.where(kinds == 0, np.where(np.arange(n) % 4 == 0, 0b0001, 0b1110), 0b0011).astype(np.int32)
    eps = np.where(kinds == 1, 1e-3 * np.sum((P[:, 1] - P[:, 0]) ** 2, 1) * np.sum((P[:, 3] - P[:, 2]) ** 2, 1), 0.0)
    b, g, H, dt = B.tx_eval_pairs(torch.tensor(kinds, device="cuda"), torch.tensor(P.reshape(n, 12), device="cuda"),
                                  W.DHAT, torch.tensor(eps, device="cuda"), torch.tensor(masks, device="cuda"))
    torch.cuda.synchronize()
    b, g, H, dt = b.cpu().numpy(), g.cpu().numpy(), H.cpu().numpy().reshape(n, 12, 12), dt.cpu().numpy()
    seen = set()
    for i in range(n):
        s, bo, go, Ho = O.pair_barrier(int(kinds[i]), P[i], W.DHAT, eps[i], int(masks[i]))
        _, ty = O.distance2(int(kinds[i]), P[i])
        seen.add((int(kinds[i]), ty[0]))
        assert s == 0
        assert abs(b[i] - bo) <= 1e-10 * abs(bo) + 1e-30
        assert np.abs(g[i] - go).max() <= 1e-8 * np.abs(go).max()
        assert np.abs(H[i] - Ho).max() <= 1e-9 * np.abs(Ho).max(), (i, kinds[i], ty)
    assert {(0, 0), (0, 1), (0, 2), (1, 0), (1, 1), (1, 3)} <= seen


def test_accd_kernel_matches_oracle():
    rng = np.random.default_rng(12)
    n = 500
    kinds = (np.arange(n) % 2).astype(np.int32)
    P = rng.normal(scale=1e-3, size=(n, 4, 3))
    dP = rng.normal(scale=2e-3, size=(n, 4, 3))
    toi, hit = B.tx_eval_accd(torch.tensor(kinds, device="cuda"), torch.tensor(P.reshape(n, 12), device="cuda"),
                              torch.tensor(dP.reshape(n, 12), device="cuda"))
    torch.cuda.synchronize()
    toi, hit = toi.cpu().numpy(), hit.cpu().numpy()
    nh = 0
    for i in range(n):
        r, t = O.accd(int(kinds[i]), P[i], dP[i])
        assert hit[i] == r
        if r == 1:
            nh += 1
            assert abs(toi[i] - t) <= 1e-9 * max(t, 1e-3)
    assert nh > 20
