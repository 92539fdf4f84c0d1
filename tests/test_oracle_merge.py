"""Pins of the oracle's SP merging (Sec. 2.3.2): the merged SP is the centre of mass (weight,
momentum and position moments conserved), the kinetic energy drops by exactly
(1/2) m mu |v1 - v2|^2, the count per cell falls to the cap, and the cap on weights holds."""
import numpy as np
import pytest

from oracle import merge as M, particles as P
from oracle.grid import Grid


def _cell_pop(g, n_per, seed, wmax=9):
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, n_per + 1, g.ncell)
    cells = np.repeat(np.arange(g.ncell), counts)
    n = len(cells)
    i, j, k = cells % g.nx, (cells // g.nx) % g.ny, cells // (g.nx * g.ny)
    f = rng.random((n, 3))
    sp_ = {"x": (i + f[:, 0]).astype(np.float32), "y": (j + f[:, 1]).astype(np.float32),
           "z": (k + f[:, 2]).astype(np.float32)}
    for c in ("vx", "vy", "vz"):
        sp_[c] = (rng.normal(size=n) * 1e5).astype(np.float32)
    sp_["w"] = rng.integers(1, wmax + 1, n).astype(np.int32)
    sp_["id"] = np.arange(n, dtype=np.uint64)
    return P.stable_sort(g, sp_)


def test_merge_pair_is_centre_of_mass():
    rng = np.random.default_rng(0)
    for _ in range(500):
        w1, w2 = (int(x) for x in rng.integers(1, 1000, 2))
        a1, a2 = rng.normal(size=2) * 1e3
        assert M.merge_pair(w1, w2, a1, a2) == pytest.approx((w1 * a1 + w2 * a2) / (w1 + w2), rel=1e-14, abs=1e-12)
        assert min(a1, a2) - 1e-9 <= M.merge_pair(w1, w2, a1, a2) <= max(a1, a2) + 1e-9


def test_merging_conserves_moments_and_loses_the_relative_energy():
    g = Grid(4, 3, 3, 1e-9, 0.0, 0.0)
    sp_, off = _cell_pop(g, 12, 1)
    m_cu = 1.0
    before = {f: sp_[f].astype(np.float64).copy() for f in P.FIELDS}
    w0 = sp_["w"].astype(np.int64).copy()
    done = M.merge_species(sp_, off, 4, 1 << 20)
    assert done > 20
    w1 = sp_["w"].astype(np.int64)
    assert w1.sum() == w0.sum()
    loss = 0.0
    for c in range(g.ncell):
        s = slice(off[c], off[c + 1])
        N = off[c + 1] - off[c]
        assert int(np.sum(w1[s] > 0)) == (N if N <= 4 else max(4, N - N // 2))
        for f in ("x", "y", "z", "vx", "vy", "vz"):
            m0 = (w0[s] * before[f][s]).sum()
            m1 = (w1[s] * sp_[f][s].astype(np.float64)).sum()
            assert m1 == pytest.approx(m0, rel=1e-6, abs=1e-6 * np.abs(w0[s] * before[f][s]).sum() + 1e-9)
        # energy drops by (1/2) mu |v1 - v2|^2 per merged pair (mu the effective weight)
        for mm in range(min(N - 4, N // 2) if N > 4 else 0):
            a, b = off[c] + 2 * mm, off[c] + 2 * mm + 1
            mu = w0[a] * w0[b] / (w0[a] + w0[b])
            loss += 0.5 * m_cu * mu * sum((before[f][a] - before[f][b]) ** 2 for f in ("vx", "vy", "vz"))
    K0 = 0.5 * m_cu * (w0 * sum(before[f] ** 2 for f in ("vx", "vy", "vz"))).sum()
    K1 = 0.5 * m_cu * (w1 * sum(sp_[f].astype(np.float64) ** 2 for f in ("vx", "vy", "vz"))).sum()
    assert K0 - K1 == pytest.approx(loss, rel=1e-5)
    # merged positions stay in their cells, so the sort order and offsets remain valid
    assert np.array_equal(P.cell_keys(g, sp_), np.repeat(np.arange(g.ncell), np.diff(off)))


def test_weight_cap_and_small_cells():
    g = Grid(2, 2, 2, 1e-9, 0.0, 0.0)
    sp_, off = _cell_pop(g, 10, 2, wmax=6)
    w0 = sp_["w"].copy()
    M.merge_species(sp_, off, 2, 7)
    assert sp_["w"].max() <= 7 and int(sp_["w"].astype(np.int64).sum()) == int(w0.astype(np.int64).sum())
    sp2, off2 = _cell_pop(g, 3, 3)
    before = {f: sp2[f].copy() for f in P.FIELDS}
    assert M.merge_species(sp2, off2, 3, 1 << 20) == 0          # no cell above the cap
    for f in P.FIELDS:
        assert np.array_equal(sp2[f], before[f])
