"""Seeded symmetric positive definite 3x3-block sparse systems for the linear-solver tests."""
import numpy as np


def random_bsr_spd(n, seed, nnz_per_row=6):
    """Block-CSR arrays (row_ptr, col_idx, vals (nnzb, 9)) and the dense matrix of a random SPD
    system: a sparse random block pattern G, A = G^T G + diag shift (symmetric pattern)."""
    rng = np.random.default_rng(seed)
    pattern = set()
    for i in range(n):
        pattern.add((i, i))
        for j in rng.integers(0, n, size=nnz_per_row // 2):
            pattern.add((i, int(j)))
            pattern.add((int(j), i))
    dense = np.zeros((3 * n, 3 * n))
    for (i, j) in pattern:
        if i <= j:
            blk = rng.normal(size=(3, 3)) * 0.3
            dense[3 * i:3 * i + 3, 3 * j:3 * j + 3] += blk
            if i != j:
                dense[3 * j:3 * j + 3, 3 * i:3 * i + 3] += blk.T
    dense = 0.5 * (dense + dense.T)
    shift = np.abs(dense).sum(1).max() + 1.0
    dense += shift * np.eye(3 * n)
    rows = sorted(pattern)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    col_idx, vals = [], []
    for i in range(n):
        cols = sorted(j for (r, j) in rows if r == i)
        row_ptr[i + 1] = row_ptr[i] + len(cols)
        for j in cols:
            col_idx.append(j)
            vals.append(dense[3 * i:3 * i + 3, 3 * j:3 * j + 3].ravel())
    return row_ptr, np.array(col_idx, dtype=np.int32), np.array(vals), dense
