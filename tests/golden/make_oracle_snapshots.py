"""Writes FP64 oracle snapshots of the GelSight-Mini gel (41x51x9 grid, 18,819 vertices, 96,000
tets) for the GPU parity tests:

* c1_prism_window_oracle.npz -- the benchmark's own trajectory (workloads.mini_gel(seed=0): the
  seeded triangular prism pressed 1.0 mm over 60 steps), steps 0..24: the benchmark's timed
  window (steps 5..24) is deep-press contact with ~300-900 active pairs;
* c1_prism_fastpress_oracle.npz -- the same gel and prism pressed 1.0 mm over 12 steps (92 um per
  step), steps 0 and 1: the indenter move of each has to be split (R7), ~300 active pairs.

Only the CPU oracle (oracle/) computes these values; the CUDA library is never involved.  The
oracle runs at the parity Newton tolerance and stores, at the listed steps, the displacement of
every vertex from its rest position (float32: the rounding, below 1e-10 m for displacements under
1.5 mm, is far inside the 4 nm parity gate) and the contact force, and for every step the number
of substeps, Newton iterations and active contact pairs.  Each file is rewritten after every
stored step, so an interrupted run keeps what it has.  Run from the repository root:

    python tests/golden/make_oracle_snapshots.py [window|fastpress]

(the window takes about an hour on 8 cores -- the Newton iteration converges linearly, 7 to 60
iterations per step at this tolerance; the oracle's parallel loops give bitwise the same result for
any thread count)."""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2411_04776_gb300 import workloads as W  # noqa: E402

NEWTON_TOL = 1e-7   # the parity tolerance of the GPU tests (tests/gpu_util.PARITY_NEWTON_TOL)
NEWTON_MAX = 400    # deep contact at this tolerance takes up to ~130 iterations per step

CASES = {
    "window": dict(file="c1_prism_window_oracle.npz", make=lambda: W.mini_gel(seed=0), steps=25,
                   snap=(4, 9, 14, 19, 24)),
    "fastpress": dict(file="c1_prism_fastpress_oracle.npz",
                      make=lambda: W.mini_gel(seed=0, depth=1.0e-3, n_press=12, slide=0.0, n_slide=0),
                      steps=2, snap=(0, 1)),
}


def run(name):
    case = CASES[name]
    out = os.path.join(HERE, case["file"])
    wl = case["make"]()
    og = O.OracleGel.from_workload(wl, newton_tol=NEWTON_TOL, newton_max=NEWTON_MAX)
    X = wl.gel.verts
    disp, force, snaps, substeps, active, newton = [], [], [], [], [], []
    t0 = time.perf_counter()
    for s in range(case["steps"]):
        info = og.step(wl.poses[s], wl.dt)
        assert info["status"] == 0, (s, info)
        substeps.append(info["substeps"])
        active.append(info["active_pairs"])
        newton.append(info["newton_iters"])
        x, _, fc, _ = og.state()
        if s in case["snap"]:
            disp.append((x - X).astype(np.float32))
            force.append(fc.copy())
            snaps.append(s)
            np.savez_compressed(out, workload=np.array(wl.name), newton_tol=NEWTON_TOL, newton_max=NEWTON_MAX,
                                snap_steps=np.array(snaps), disp=np.stack(disp), contact_force=np.stack(force),
                                substeps=np.array(substeps), active_pairs=np.array(active),
                                newton_iters=np.array(newton))
        print(f"{name} step {s}: {info}  ({time.perf_counter() - t0:.0f} s)", flush=True)
    print("wrote", out)


if __name__ == "__main__":
    for n in (sys.argv[1:] or list(CASES)):
        run(n)
