"""The standalone block-Jacobi PCG entry point against a dense direct solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_04776_gb300 import binding as B  # noqa: E402
from tests.bsr_util import random_bsr_spd  # noqa: E402


@pytest.mark.parametrize("n,seed", [(1, 0), (37, 1), (700, 2)])
def test_bsr_pcg_matches_dense_solve(n, seed):
    rp, ci, va, dense = random_bsr_spd(n, seed)
    b = np.random.default_rng(seed + 100).normal(size=3 * n)
    x, it, rr = B.tx_bsr_pcg(torch.tensor(rp, device="cuda"), torch.tensor(ci, device="cuda"),
                             torch.tensor(va, device="cuda"), torch.tensor(b, device="cuda"), rel_tol=1e-12)
    ref = np.linalg.solve(dense, b)
    assert rr <= 1e-12 and it >= 1
    np.testing.assert_allclose(x.cpu().numpy(), ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_bsr_pcg_zero_rhs_and_iteration_cap():
    rp, ci, va, dense = random_bsr_spd(50, 3)
    dv = lambda a: torch.tensor(a, device="cuda")  # noqa: E731
    x, it, rr = B.tx_bsr_pcg(dv(rp), dv(ci), dv(va), dv(np.zeros(150)), rel_tol=1e-12)
    assert it == 0 and rr == 0.0 and float(x.abs().max()) == 0.0
    b = np.ones(150)
    x, it, rr = B.tx_bsr_pcg(dv(rp), dv(ci), dv(va), dv(b), rel_tol=1e-30, max_iter=3)
    assert it == 3 and rr > 0.0
