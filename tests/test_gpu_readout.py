"""Gel-surface readout on the GPU (markers carried by their rest top-surface triangle, and the CUDA
rasterised top-surface height map) against the oracle's readout of the same state: at rest, and
at the oracle's own state after a contact trajectory (the GPU gel takes that state as input)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2411_04776_gb300 import binding as B  # noqa: E402
from paper_2411_04776_gb300 import workloads as W  # noqa: E402

# pixel grid over the 18 x 24 mm gel whose centres never fall on the gel's boundary
GRID = dict(nx=64, ny=80, x0=-0.5e-3, y0=-0.6e-3, dx=0.3e-3, dy=0.315e-3)


def test_readout_at_rest():
    wl = W.small_gel_sphere(0)
    gel = B.Gel.from_workload(wl)
    X = wl.gel.verts
    top = X[:, 2].max()
    rng = np.random.default_rng(8)
    m = np.column_stack([rng.uniform(0.0, 0.018, 60), rng.uniform(0.0, 0.024, 60)])
    pos, found = gel.markers(np.vstack([m, [[0.019, 0.01], [-0.001, 0.01]]]))
    assert found[:60].all() and not found[60:].any()
    assert np.abs(pos[:60, :2] - m).max() <= 1e-15 and np.abs(pos[:60, 2] - top).max() <= 1e-15
    hm = gel.height_map(**GRID)
    px = GRID["x0"] + (np.arange(GRID["nx"]) + 0.5) * GRID["dx"]
    py = GRID["y0"] + (np.arange(GRID["ny"]) + 0.5) * GRID["dy"]
    inside = (py[:, None] > 0) & (py[:, None] < 0.024) & (px[None, :] > 0) & (px[None, :] < 0.018)
    assert np.all(np.isnan(hm[~inside])) and np.abs(hm[inside] - top).max() <= 1e-15
    gel.close()


def test_readout_matches_oracle_after_contact():
    wl = W.small_gel_sphere(2)
    og = O.OracleGel.from_workload(wl, newton_tol=1e-7)
    for s in range(20):
        assert og.step(wl.poses[s], wl.dt)["status"] == 0
    xo, vo, _, pose = og.state()
    assert xo[:, 2].min() >= 0.0 and (xo[:, 2] < wl.gel.top - 1e-4).any()  # an indentation
    gel = B.Gel.from_workload(wl)
    gel.set_state(xo, vo, pose)
    rng = np.random.default_rng(9)
    m = np.column_stack([rng.uniform(0.0, 0.018, 100), rng.uniform(0.0, 0.024, 100)])
    pg, fg = gel.markers(m)
    po, fo = og.markers(xo, m)
    assert np.array_equal(fg, fo) and fg.all()
    assert np.abs(pg - po).max() <= 1e-15
    hg = gel.height_map(**GRID)
    ho = og.height_map(xo, GRID["nx"], GRID["ny"], GRID["x0"], GRID["y0"], GRID["dx"], GRID["dy"])
    assert np.array_equal(np.isnan(hg), np.isnan(ho))
    ok = ~np.isnan(ho)
    assert np.abs(hg[ok] - ho[ok]).max() <= 1e-15
    assert np.nanmin(ho) < wl.gel.top - 1e-4  # the indentation shows in the map
    # a camera-sized map (480 x 640) of the same surface
    big = gel.height_map(640, 480, 0.0, 0.0, 0.018 / 640, 0.024 / 480)
    assert np.isfinite(big).mean() > 0.99
    gel.close()
