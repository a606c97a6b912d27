"""Failure paths of the library, made to run without faulting the device: a bounded device wait
that gives up (the group barriers of the PCG wait for an arrival that never comes, with a short
poll limit), an allocation that fails on the host side before it reaches the CUDA runtime, the
Newton iteration cap, and a reset after which the gel steps exactly like a fresh one.  Every
failed step must leave the state where it was (steps are transactional) and the handle usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_04776_gb300 import binding as B  # noqa: E402
from paper_2411_04776_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import PARITY_NEWTON_TOL, POS_TOL  # noqa: E402


def contact_state(wl, gel, steps):
    for s in range(steps):
        assert gel.step(wl.poses[s], wl.dt) == 0
    return gel.get_state()


@pytest.mark.parametrize("precision", [B.TX_PREC_FP64, B.TX_PREC_MIXED], ids=["fp64", "mixed"])
def test_device_wait_timeout_rolls_back(precision):
    wl = W.small_gel_sphere(0)
    gel = B.Gel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL, precision=precision)
    ref = B.Gel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL, precision=precision)
    x0, v0, p0 = contact_state(wl, gel, 12)
    contact_state(wl, ref, 12)
    B.tx_debug_inject(B.TX_INJECT_WAIT_TIMEOUT, 1)
    try:
        st = gel.step(wl.poses[12], wl.dt)
    finally:
        B.tx_debug_inject(B.TX_INJECT_WAIT_TIMEOUT, 0)
    assert st == 10, B.STATUS_NAMES.get(st, st)  # TX_ERR_DEVICE_TIMEOUT
    x1, v1, p1 = gel.get_state()
    assert np.array_equal(x1, x0) and np.array_equal(v1, v0) and np.array_equal(p1, p0)
    # the context and the handle stay usable: the retried step equals an undisturbed gel's
    assert gel.step(wl.poses[12], wl.dt) == 0
    assert ref.step(wl.poses[12], wl.dt) == 0
    d = np.abs(gel.state()[0] - ref.state()[0]).max()
    print("retried step vs undisturbed gel: %.3e m" % d)
    assert d <= POS_TOL
    gel.close()
    ref.close()


def test_injected_allocation_failure_at_create_frees_everything():
    wl = W.mini_gel(seed=7, grid=W.GRID_MID, depth=0.5e-3)
    desc = B.GelDesc.from_workload(wl)
    B.Gel(desc).close()  # module loaded, context up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (1, 2, 7, 20, 45, 60):
        B.tx_debug_inject(B.TX_INJECT_ALLOC_FAIL, k)
        try:
            with pytest.raises(B.TxError) as e:
                B.tx_gel_create(desc)
        finally:
            B.tx_debug_inject(B.TX_INJECT_ALLOC_FAIL, 0)
        assert e.value.status == 2, k  # TX_ERR_OOM
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, k  # nothing leaked
    g = B.Gel(desc)  # disarmed: creation works again
    assert g.step(wl.poses[0], wl.dt) == 0
    g.close()


def test_newton_cap_is_transactional():
    wl = W.small_gel_sphere(0)
    gel = B.Gel.from_workload(wl, newton_max_iter=1)
    x0, v0, p0 = gel.get_state()
    st = 0
    for s in range(30):  # the first step that needs more than one Newton update fails
        st = gel.step(wl.poses[s], wl.dt)
        if st != 0:
            break
        x0, v0, p0 = gel.get_state()
    assert st == 5, B.STATUS_NAMES.get(st, st)  # TX_ERR_NEWTON_MAXIT
    x1, v1, p1 = gel.get_state()
    assert np.array_equal(x1, x0) and np.array_equal(v1, v0) and np.array_equal(p1, p0)
    gel.close()


@pytest.mark.parametrize("precision", [B.TX_PREC_FP64, B.TX_PREC_MIXED], ids=["fp64", "mixed"])
def test_reset_gel_steps_like_a_fresh_one(precision):
    """After a reset no trace of the previous trajectory is left (positions, velocities and the
    previous Newton direction the next solve starts from)."""
    wl = W.small_gel_sphere(1)
    used = B.Gel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL, precision=precision)
    contact_state(wl, used, 20)
    used.reset()
    fresh = B.Gel.from_workload(wl, newton_tol=PARITY_NEWTON_TOL, precision=precision)
    for s in range(14):
        assert used.step(wl.poses[s], wl.dt) == 0
        assert fresh.step(wl.poses[s], wl.dt) == 0
    d = np.abs(used.state()[0] - fresh.state()[0]).max()
    print("reset gel vs fresh gel after 14 steps: %.3e m" % d)
    assert d <= POS_TOL
    used.close()
    fresh.close()
