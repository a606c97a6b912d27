"""Writes tests/golden/c1_prism_oracle.npz: FP64 oracle snapshots of the GelSight-Mini gel
(41x51x9 grid, 18,819 vertices, 96,000 tets) pressed by the seeded triangular prism of the
benchmark workload (workloads.mini_gel(seed=0): 1.0 mm over 60 steps, then a 2 mm slide).

Only the CPU oracle (oracle/) computes these values; the CUDA library is never involved.  The
oracle runs the first STEPS steps of that trajectory at the parity Newton tolerance and stores,
at the steps listed in SNAP, the displacement of every vertex from its rest position (float32:
the rounding, below 1e-10 m for displacements under 1.5 mm, is far inside the 4 nm parity
gate), the contact force, and for every step the number of substeps (step splitting of the
kinematic indenter) and of active contact pairs.  Run from the repository root:

    python tests/golden/make_oracle_snapshots.py

(about half an hour on 8 cores; the oracle's parallel loops give bitwise the same result for
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
STEPS = 30          # covers the benchmark's timed window (steps 5..24) and the split steps after it
SNAP = (4, 9, 14, 19, 24, 27, 28, 29)
OUT = os.path.join(HERE, "c1_prism_oracle.npz")


def main():
    O.set_threads(0)
    wl = W.mini_gel(seed=0)
    og = O.OracleGel.from_workload(wl, newton_tol=NEWTON_TOL)
    X = wl.gel.verts
    disp, force, substeps, active, newton = [], [], [], [], []
    t0 = time.perf_counter()
    for s in range(STEPS):
        info = og.step(wl.poses[s], wl.dt)
        assert info["status"] == 0, (s, info)
        substeps.append(info["substeps"])
        active.append(info["active_pairs"])
        newton.append(info["newton_iters"])
        x, _, fc, _ = og.state()
        if s in SNAP:
            disp.append((x - X).astype(np.float32))
            force.append(fc.copy())
        print(f"step {s}: {info}  ({time.perf_counter() - t0:.0f} s)", flush=True)
    np.savez_compressed(OUT, workload=np.array(wl.name), newton_tol=NEWTON_TOL, snap_steps=np.array(SNAP),
                        disp=np.stack(disp), contact_force=np.stack(force), substeps=np.array(substeps),
                        active_pairs=np.array(active), newton_iters=np.array(newton))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
