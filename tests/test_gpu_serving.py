"""Continuous-batching server: requests admitted under an HBM budget while others are in flight,
and each environment's result is the same as stepping its gel alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_04776_gb300 import binding as B  # noqa: E402
from paper_2411_04776_gb300 import serving as S  # noqa: E402
from paper_2411_04776_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import PARITY_NEWTON_TOL, POS_TOL  # noqa: E402


@pytest.mark.parametrize("precision", [B.TX_PREC_FP64, B.TX_PREC_MIXED], ids=["fp64", "mixed"])
def test_serving_results_equal_alone_under_budget(precision):
    wls = [W.small_gel_sphere(s) for s in range(4)] + [W.mini_gel(7, grid=W.GRID_MID, depth=0.5e-3)]
    fp = [B.tx_gel_footprint_bytes(B.GelDesc.from_workload(w, precision=precision)) for w in wls]
    budget = sorted(fp)[-1] + sorted(fp)[-2] + 1  # at most the two largest gels in flight
    srv = S.GelServer(wls, budget, precision=precision, newton_tol=PARITY_NEWTON_TOL)
    # staggered arrivals: new requests join while others are mid-Newton
    schedule = [[0, 1, 2, 3, 4], [], [0], [1], [], [2, 4], [3], [0], [], [1, 2], [4], [3], [0, 1]]
    done = srv.run_schedule(schedule)
    n_req = sum(len(s) for s in schedule)
    assert len(done) == n_req and all(r.status == 0 for r in done)
    assert srv.max_inflight_bytes <= budget and srv.max_inflight >= 2
    # some request was admitted while another one was still in flight (continuous batching)
    overlaps = sum(1 for a in done for b in done if a is not b and a.admitted < b.admitted < a.done)
    assert overlaps > 0
    for e, w in enumerate(wls):
        n_steps = int(srv.cursor[e])
        alone = B.Gel.from_workload(w, newton_tol=PARITY_NEWTON_TOL, precision=precision)
        for s in range(n_steps):
            assert alone.step(w.poses[s], w.dt) == 0
        xa = alone.state()[0]
        xs = B.tx_batch_state(srv.handle, e, len(w.gel.verts))[0]
        assert np.abs(xa - xs).max() <= POS_TOL, (e, np.abs(xa - xs).max())
    srv.close()


def test_poisson_arrivals_rate():
    arr = S.poisson_arrivals(100, 2000.0, 2.0, seed=3)
    assert abs(len(arr) - 4000) < 4 * np.sqrt(4000)
    assert all(0 <= e < 100 for _, e in arr)
