"""Parity of the streaming PCG kernels (the matrix streamed from HBM every iteration, the kernels
the large batched configurations run) in both forms: per-gel CTA groups (k_pcg64 in FP64,
k_pcg_mixed in mixed precision; tx_params.pcg_plan = 1) and the pool of one CTA per SM
(k_pcg64_pool, k_pcg_mixed_pool; pcg_plan = 2), on a batch of gels of uneven size, one from each of
the three grids, so that the small gels finish their solves while the large one still iterates
(the pool re-splits the remaining slices): every gel against the FP64 oracle and against the same
gel stepped alone (which takes the resident kernels).  The profile counters show that only the
asked-for form ran."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2411_04776_gb300 import binding as B  # noqa: E402
from paper_2411_04776_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import PARITY_NEWTON_TOL, POS_TOL, load_golden  # noqa: E402

STEPS = 10


def batch_workloads():
    return [W.small_gel_sphere(2),
            W.mini_gel(seed=7, grid=W.GRID_MID, depth=0.5e-3, n_press=20, slide=0.0, n_slide=0),
            W.mini_gel(seed=0)]  # the benchmark's GelSight-Mini trajectory (oracle snapshots stored)


@pytest.fixture(scope="module")
def reference():
    """Oracle positions of the two smaller gels at every step; stored oracle snapshots of the
    GelSight-Mini gel (steps 4 and 9 are inside this window)."""
    O.set_threads(0)
    wls = batch_workloads()
    ref = {}
    for g in (0, 1):
        og = O.OracleGel.from_workload(wls[g], newton_tol=PARITY_NEWTON_TOL)
        xs = []
        for s in range(STEPS):
            assert og.step(wls[g].poses[s], wls[g].dt)["status"] == 0
            xs.append(og.state()[0].copy())
        ref[g] = xs
    gold = load_golden("window")
    assert str(gold["workload"]) == wls[2].name
    ref[2] = {int(s): wls[2].gel.verts + gold["disp"][k].astype(np.float64)
              for k, s in enumerate(gold["snap_steps"]) if s < STEPS}
    assert len(ref[2]) >= 2
    return wls, ref


def run_batch(wls, precision, plan):
    descs = [B.GelDesc.from_workload(w, newton_tol=PARITY_NEWTON_TOL, precision=precision, pcg_plan=plan,
                                     newton_max_iter=400) for w in wls]
    b = B.tx_batch_create(descs, stream=torch.cuda.current_stream())
    B.tx_batch_profile(b, True)
    out = []
    try:
        for s in range(STEPS):
            st, sts = B.tx_batch_step(b, np.stack([w.poses[s] for w in wls]), np.array([w.dt for w in wls]))
            assert st == 0 and np.all(sts == 0), sts
            out.append([B.tx_batch_state(b, g, len(w.gel.verts))[0] for g, w in enumerate(wls)])
        prof = B.tx_batch_profile(b, False)
    finally:
        B.tx_batch_destroy(b)
    return out, prof


def run_alone(w, precision, steps=STEPS):
    gel = B.Gel.from_workload(w, newton_tol=PARITY_NEWTON_TOL, precision=precision, newton_max_iter=400,
                              stream=torch.cuda.current_stream())
    out = []
    for s in range(steps):
        assert gel.step(w.poses[s], w.dt) == 0
        out.append(gel.state()[0])
    gel.close()
    return out


@pytest.mark.parametrize("plan", [1, 2], ids=["groups", "pool"])
@pytest.mark.parametrize("precision", [B.TX_PREC_FP64, B.TX_PREC_MIXED], ids=["fp64", "mixed"])
def test_streaming_batch_matches_oracle_and_alone(reference, precision, plan):
    wls, ref = reference
    out, prof = run_batch(wls, precision, plan=plan)
    assert prof["pcg_streaming_launches"] > 0 and prof["pcg_resident_launches"] == 0, prof
    # plan 1: the per-gel CTA groups only; plan 2: the pool only
    assert prof["pcg_pool_launches"] == (prof["pcg_streaming_launches"] if plan == 2 else 0), prof
    worst = np.zeros(3)
    for s in range(STEPS):
        for g in (0, 1):
            worst[g] = max(worst[g], np.abs(out[s][g] - ref[g][s]).max())
        if s in ref[2]:
            worst[2] = max(worst[2], np.abs(out[s][2] - ref[2][s]).max())
    print("streaming PCG (%s, %s) vs oracle, max vertex error per gel [m]: %s"
          % ("fp64" if precision == B.TX_PREC_FP64 else "mixed", "pool" if plan == 2 else "groups", worst))
    assert np.all(worst <= POS_TOL), worst
    for g, w in enumerate(wls):
        alone = run_alone(w, precision)
        d = max(np.abs(alone[s] - out[s][g]).max() for s in range(STEPS))
        assert d <= POS_TOL, (g, d)


def test_automatic_plan_pools_a_large_batch_and_each_gel_matches_alone():
    """32 gels of the 21x26x5 grid, each with its own seeded indenter: too many slices for the
    resident kernels and enough gels for the automatic plan to take the pool; every gel of the
    batch against the same gel stepped alone (resident kernels)."""
    wls = [W.mini_gel(seed=s, grid=W.GRID_MID, depth=0.5e-3, n_press=20, slide=0.0, n_slide=0) for s in range(32)]
    steps = 8
    descs = [B.GelDesc.from_workload(w, newton_tol=PARITY_NEWTON_TOL, newton_max_iter=400) for w in wls]
    b = B.tx_batch_create(descs, stream=torch.cuda.current_stream())
    B.tx_batch_profile(b, True)
    out = []
    try:
        for s in range(steps):
            st, sts = B.tx_batch_step(b, np.stack([w.poses[s] for w in wls]), np.array([w.dt for w in wls]))
            assert st == 0 and np.all(sts == 0), sts
        out = [B.tx_batch_state(b, g, len(w.gel.verts))[0] for g, w in enumerate(wls)]
        contact = [B.tx_batch_state(b, g, len(w.gel.verts))[3].active_pairs for g, w in enumerate(wls)]
        prof = B.tx_batch_profile(b, False)
    finally:
        B.tx_batch_destroy(b)
    # the pool while 32 gels iterate; Newton rounds of fewer gels (the others converged) may take the
    # per-gel groups or the resident kernels
    assert prof["pcg_pool_launches"] > 0 and prof["pcg_pool_launches"] <= prof["pcg_streaming_launches"], prof
    assert sum(c > 0 for c in contact) >= 8, contact  # the gels are in contact by then
    worst = 0.0
    for g in range(0, 32, 4):  # every fourth gel alone (the others ran in the same launches)
        alone = run_alone(wls[g], B.TX_PREC_FP64, steps)
        worst = max(worst, float(np.abs(alone[steps - 1] - out[g]).max()))
    print("pooled batch of 32 gels vs alone: max vertex difference %.3e m" % worst)
    assert worst <= POS_TOL, worst
