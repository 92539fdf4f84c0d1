"""Merging of superparticles (Sec. 2.3.2, the merging passage; test infrastructure only).

Two SPs of one species become one: w = w1 + w2, and with the effective weight
mu = w1 w2 / (w1 + w2) the position and velocity are r_m = r1 mu/w2 + r2 mu/w1 and
v_m = v1 mu/w2 + v2 mu/w1 (the centre of mass; momentum is conserved, kinetic energy drops by
(1/2) m mu |v1 - v2|^2 in real-particle units).

Readings (the paper gives the formulas, not when or which SPs merge):
  * Merging runs right after the cell sort, before the collisions, on the sorted SPs of every
    species, and only when the step asks for it (parameter merge_max > 0).
  * In a cell holding N > M = merge_max SPs of a species, the SPs at cell-sorted places 2m and
    2m + 1 merge for m < min(N - M, floor(N/2)); a pair whose weights sum above w_max_units,
    or that holds a zero weight, is left alone.
  * The merged SP takes the first place and keeps its id; the second keeps its place with
    weight 0 (no charge, no collisions) and leaves at the next sort.
  * Arithmetic in float64 in the order written above, rounded once to float32; the merged
    position stays in the cell (a convex combination of two points of it).
"""
import numpy as np

F32 = np.float32


def merge_pair(w1, w2, a1, a2):
    """a1 mu/w2 + a2 mu/w1 in float64 (one component), mu = w1 w2 / (w1 + w2)."""
    w1, w2 = float(w1), float(w2)
    mu = w1 * w2 / (w1 + w2)
    return float(a1) * (mu / w2) + float(a2) * (mu / w1)


def merge_species(sp_, off, merge_max, w_max_units):
    """Merge in place over the cells of one cell-sorted species; returns the merges done."""
    cnt = np.diff(off)
    done = 0
    for c in np.nonzero(cnt > merge_max)[0]:
        N = int(cnt[c])
        for m in range(min(N - merge_max, N // 2)):
            a, b = off[c] + 2 * m, off[c] + 2 * m + 1
            w1, w2 = int(sp_["w"][a]), int(sp_["w"][b])
            if w1 <= 0 or w2 <= 0 or w1 + w2 > w_max_units:
                continue
            for f in ("x", "y", "z", "vx", "vy", "vz"):
                sp_[f][a] = F32(merge_pair(w1, w2, sp_[f][a], sp_[f][b]))
            sp_["w"][a] = w1 + w2
            sp_["w"][b] = 0
            done += 1
    return done
