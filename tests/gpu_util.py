"""Helpers for the GPU parity tests (comparison only; no arithmetic of the method)."""
import numpy as np


def match_row(a, b):
    """Nearest-neighbour pairing of two root sets (a: GPU, b: oracle).  Returns
    (index into b for each a, max pairing distance, smallest separation within b)."""
    a = np.asarray(a)
    b = np.asarray(b)
    d = np.abs(a[:, None] - b[None, :])
    idx = d.argmin(axis=1)
    dist = d[np.arange(len(a)), idx]
    sep = np.abs(b[:, None] - b[None, :])
    np.fill_diagonal(sep, np.inf)
    return idx, float(dist.max()), float(sep.min()) if len(b) > 1 else np.inf


def compare_chain(zg, zo, tol=1e-9):
    """Row-by-row multiset comparison; asserts a 1:1, unambiguous pairing within tol.
    Returns (worst distance, list of pairings)."""
    assert zg.shape == zo.shape
    worst = 0.0
    pairs = []
    for j in range(zg.shape[0]):
        idx, dist, sep = match_row(zg[j], zo[j])
        assert len(set(idx.tolist())) == len(idx), f"row {j}: pairing is not 1:1"
        assert dist < tol, f"row {j}: max |dz| = {dist}"
        assert dist < 1e-3 * sep, f"row {j}: pairing ambiguous (sep {sep})"
        worst = max(worst, dist)
        pairs.append(idx)
    return worst, pairs
