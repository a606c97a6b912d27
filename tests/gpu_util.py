"""Shared helpers of the GPU tests (synthetic states and tolerances)."""
import numpy as np

# parity gate on positions: 1e-6 of the 4 mm gel thickness
POS_TOL = 4e-9

# Newton tolerance of the parity runs.  The projected Newton iteration converges linearly (rate
# about 1/2), so a run stopped at ||p||_inf / h < tol * bbox sits about that far from the
# minimiser.  At 1e-7 the oracle's own positions move by up to 2.3 nm when the tolerance is
# tightened to 1e-9 (coarse Hertz block), inside the 4 nm gate; tighter tolerances run into the
# FP64 resolution of the energy on the 10x13x4 gel (the line search stalls).
PARITY_NEWTON_TOL = 1e-7
# The contact force is far more sensitive: at 1e-7 the oracle's own force moves by up to 7e-4
# (relative) under the same tightening, at 1e-8 by 2e-6, so force parity at 1e-4 runs at 1e-8.
FORCE_PARITY_NEWTON_TOL = 1e-8


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


GOLDEN = {"window": "c1_prism_window_oracle.npz", "fastpress": "c1_prism_fastpress_oracle.npz"}


def load_golden(case):
    """FP64 oracle snapshots of the GelSight-Mini gel (tests/golden/make_oracle_snapshots.py):
    displacements and contact forces at the snapshot steps, substeps, Newton iterations and
    active pairs per step.  "window": the benchmark trajectory, steps 0..24; "fastpress": the
    same prism pressed 1.0 mm over 12 steps, steps 0 and 1 (each split in two)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", GOLDEN[case])
    z = np.load(path)
    return {k: z[k] for k in z.files}


def golden_workload(case):
    from paper_2411_04776_gb300 import workloads as W
    if case == "window":
        return W.mini_gel(seed=0)
    return W.mini_gel(seed=0, depth=1.0e-3, n_press=12, slide=0.0, n_slide=0)
