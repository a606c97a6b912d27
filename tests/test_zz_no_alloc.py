"""The no-allocation PCG entry point (tx_bsr_pcg_noalloc) against the allocating one
(tx_bsr_pcg), called through the C ABI twice in a row on different systems so that contents
left in the shared scratch array by one call cannot leak into the next.

This file is named to be collected last: a run that stops at the first failure has run every
other test by the time it gets here.  It passes alone in a fresh process and after the others."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_04776_gb300 import binding as B  # noqa: E402
from tests.bsr_util import random_bsr_spd  # noqa: E402


def dv(a):
    return torch.tensor(a, device="cuda")


@pytest.mark.parametrize("calls", [[(700, 5), (41, 6)]])
def test_noalloc_matches_allocating_solver_twice(calls):
    for n, seed in calls:
        rp, ci, va, dense = random_bsr_spd(n, seed)
        b = np.random.default_rng(seed + 7).normal(size=3 * n)
        x_ref, it_ref, rr_ref = B.tx_bsr_pcg(dv(rp), dv(ci), dv(va), dv(b), rel_tol=1e-12)
        x_out = torch.full((3 * n,), float("nan"), dtype=torch.float64, device="cuda")
        x, it, rr = B.tx_bsr_pcg_noalloc(dv(rp), dv(ci), dv(va), dv(b), x=x_out, rel_tol=1e-12)
        torch.cuda.synchronize()
        assert it == it_ref and rr <= 1e-12
        np.testing.assert_allclose(x.cpu().numpy(), x_ref.cpu().numpy(), rtol=0,
                                   atol=1e-10 * float(x_ref.abs().max()))
        ref = np.linalg.solve(dense, b)
        np.testing.assert_allclose(x.cpu().numpy(), ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_noalloc_rejects_oversized_systems():
    L = B.load()
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    s = L.tx_bsr_pcg_noalloc(65537, ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                             ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                             ctypes.c_void_p(dummy.data_ptr()), 1e-8, 10, ctypes.byref(it), ctypes.byref(rr),
                             ctypes.c_void_p(0))
    assert s == 1 and b"65536" in L.tx_last_error()
