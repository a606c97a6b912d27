"""Hertz indentation through the CUDA library: contact force against Hertz's closed form under
mesh refinement, and against the FP64 oracle on the coarse mesh."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2411_04776_gb300 import binding as B  # noqa: E402
from paper_2411_04776_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import FORCE_PARITY_NEWTON_TOL, PARITY_NEWTON_TOL  # noqa: E402

HALF = 8e-3
RADIUS = 3e-3


def hertz_force(uc):
    """Rigid frictionless sphere on an elastic half-space (Johnson, Contact Mechanics, 1985,
    Sec. 4.2): F = 4/3 E* sqrt(R) uc^(3/2), E* = E / (1 - nu^2)."""
    return 4.0 / 3.0 * W.YOUNG / (1.0 - W.POISSON ** 2) * math.sqrt(RADIUS) * uc ** 1.5


def centre(X):
    c = np.where((np.abs(X[:, 0] - HALF) < 1e-9) & (np.abs(X[:, 1] - HALF) < 1e-9) & (X[:, 2] > HALF - 1e-9))[0]
    assert len(c) == 1
    return int(c[0])


def run_gpu(h0, ratio, tol=PARITY_NEWTON_TOL):
    wl = W.hertz_block(h0=h0, ratio=ratio, half=HALF, thick=HALF, dhat=15e-6, step=12e-6)
    c = centre(wl.gel.verts)
    g = B.Gel(B.GelDesc.from_workload(wl, newton_tol=tol), stream=torch.cuda.current_stream())
    out = []
    for p in wl.poses:
        assert g.step(p, wl.dt) == 0
        x, _, fc, _ = g.state()
        out.append((wl.gel.verts[c, 2] - x[c, 2], -fc[2]))
    g.close()
    return wl, np.array(out)


def test_hertz_force_converges_under_refinement():
    errs = []
    for h0, ratio in [(80e-6, 1.5), (60e-6, 1.3), (30e-6, 1.2)]:
        _, r = run_gpu(h0, ratio)
        ratio_last = r[-1, 1] / hertz_force(r[-1, 0])
        errs.append(abs(ratio_last - 1.0))
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 0.15, errs


def test_hertz_coarse_matches_oracle():
    wl, r = run_gpu(80e-6, 1.5, FORCE_PARITY_NEWTON_TOL)
    og = O.OracleGel.from_workload(wl, newton_tol=FORCE_PARITY_NEWTON_TOL)
    c = centre(wl.gel.verts)
    for s, p in enumerate(wl.poses):
        assert og.step(p, wl.dt)["status"] == 0
        x, _, fc, _ = og.state()
        assert abs((wl.gel.verts[c, 2] - x[c, 2]) - r[s, 0]) <= 4e-9
        assert abs(-fc[2] - r[s, 1]) <= 1e-4 * abs(r[s, 1])
