"""Shared helpers of the GPU tests (synthetic states and tolerances)."""
import numpy as np

# parity gate on positions: 1e-6 of the 4 mm gel thickness
POS_TOL = 4e-9


def smooth_state(wl, seed, amp=2e-5):
    """Seeded smooth displacement of the free vertices (no inversion), predictor and h."""
    rng = np.random.default_rng(seed)
    X = wl.gel.verts
    k = rng.normal(size=(3, 3)) * 300.0
    ph = rng.uniform(0, 2 * np.pi, size=3)
    disp = amp * np.sin(X @ k.T + ph)
    disp[wl.gel.dirichlet == 1] = 0.0
    x = X + disp
    xt = X + 0.5 * disp
    return x, xt, wl.dt
