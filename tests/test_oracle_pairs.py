"""Pins for the oracle's neighbour search (CPU only).

The neighbour graph is the paper's input graph: atoms share an edge when closer than the
cutoff (Methods, semi-local energy equation), built with a skin so it need not be rebuilt every
step (Results "Distributed potential computation", pruning paragraph).  Pins, none of which
re-use the oracle's own formulas:
  * brute force vs linked cells (two different algorithms, exact set equality);
  * perfect-fcc coordination shells 12/18/42/54 (crystallography, tests/golden/fcc_shells.txt),
    also in a single conventional cell where every neighbour is a periodic image;
  * lattice-point counts for one atom in a small cubic / triclinic cell (integer-point
    enumeration of |n H| < R written independently below);
  * edge symmetry (i, j, n) <-> (j, i, -n).
"""
import os

import numpy as np
import pytest

import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _set(p):
    i, j, s = p
    return set(zip(i.tolist(), j.tolist(), map(tuple, s.tolist())))


@pytest.mark.parametrize("R", [3.0, 5.0, 6.0])
def test_brute_equals_cells_water(orc, R):
    sy = syn.water_box(64, seed=1)
    xw, _ = orc.wrap(sy.positions, sy.cell)
    a = orc.pairs_brute(xw, sy.cell, R)
    b = orc.pairs_cells(xw, sy.cell, R)
    assert len(a[0]) == len(b[0]) > 0
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_brute_is_sorted_and_symmetric(orc):
    sy = syn.water_box(27, seed=3)
    xw, _ = orc.wrap(sy.positions, sy.cell)
    i, j, s = orc.pairs_brute(xw, sy.cell, 5.0)
    key = np.stack([i, j, s[:, 0], s[:, 1], s[:, 2]], 1)
    assert (np.diff(np.lexsort(key.T[::-1])) > 0).all()
    S = _set((i, j, s))
    for (a, b, n) in S:
        assert (b, a, (-n[0], -n[1], -n[2])) in S


@pytest.mark.parametrize("tilt_seed", [0, 1, 2])
def test_brute_equals_cells_triclinic_small(orc, tilt_seed):
    rng = np.random.default_rng(tilt_seed)
    L = 7.0
    H = np.array([[L, 0, 0], [rng.uniform(-0.1, 0.1) * L, L, 0],
                  [rng.uniform(-0.1, 0.1) * L, rng.uniform(-0.1, 0.1) * L, L]])
    f = rng.uniform(0, 1, size=(20, 3))
    x = f @ H + rng.normal(0, 3.0, size=(20, 3))     # some atoms outside the cell
    xw, m = orc.wrap(x, H)
    # wrapped positions lie in the cell: fractional coordinates in [0, 1]
    fr = xw @ np.linalg.inv(H)
    assert (fr > -1e-12).all() and (fr < 1 + 1e-12).all()
    np.testing.assert_allclose(xw, x - m @ H, atol=1e-12)
    for R in (3.0, 6.0, 9.5):     # 9.5 > L: several images per pair
        a = orc.pairs_brute(xw, H, R)
        b = orc.pairs_cells(xw, H, R)
        for u, v in zip(a, b):
            np.testing.assert_array_equal(u, v)


def _golden_shells():
    rows = []
    with open(os.path.join(GOLDEN, "fcc_shells.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                c, k = line.split()
                rows.append((float(c), int(k)))
    return rows


@pytest.mark.parametrize("cells", [(1, 1, 1), (2, 2, 2), (3, 3, 3)])
def test_fcc_coordination_shells(orc, cells):
    a = 4.05
    sy = syn.fcc(*cells, a=a, jitter=0.0)
    xw, _ = orc.wrap(sy.positions, sy.cell)
    for frac, expect in _golden_shells():
        i, j, s = orc.pairs_cells(xw, sy.cell, frac * a)
        counts = np.bincount(i, minlength=sy.n)
        assert (counts == expect).all(), (cells, frac, np.unique(counts))
        if cells == (1, 1, 1):
            ib, jb, sb = orc.pairs_brute(xw, sy.cell, frac * a)
            assert len(ib) == len(i)


def _lattice_points(H, R):
    """Number of lattice vectors n H (n integer, n != 0) with |n H| < R, by plain enumeration."""
    m = int(np.ceil(R / min(np.linalg.svd(H, compute_uv=False)))) + 2
    r = np.arange(-m, m + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    d = np.linalg.norm(n @ H, axis=1)
    return int(((d < R) & (np.abs(n).sum(1) > 0)).sum())


@pytest.mark.parametrize("R,expect", [(2.5, 6), (3.0, 18), (3.5, 26), (4.1, 32)])
def test_single_atom_cubic_images(orc, R, expect):
    H = np.eye(3) * 2.0
    x = np.array([[0.3, 1.1, 1.7]])
    xw, _ = orc.wrap(x, H)
    for fn in (orc.pairs_brute, orc.pairs_cells):
        i, j, s = fn(xw, H, R)
        assert len(i) == expect == _lattice_points(H, R)


def test_single_atom_triclinic_images(orc):
    H = np.array([[3.0, 0.0, 0.0], [0.4, 2.8, 0.0], [-0.3, 0.5, 3.3]])
    x = np.array([[1.0, 1.0, 1.0]])
    xw, _ = orc.wrap(x, H)
    for R in (2.0, 4.0, 6.5):
        expect = _lattice_points(H, R)
        for fn in (orc.pairs_brute, orc.pairs_cells):
            assert len(fn(xw, H, R)[0]) == expect


def test_pair_distances_within_cutoff(orc):
    sy = syn.fcc(3, 3, 3, jitter=0.05, seed=2)
    xw, _ = orc.wrap(sy.positions, sy.cell)
    R = 5.0
    i, j, s = orc.pairs_cells(xw, sy.cell, R)
    d = np.linalg.norm(xw[j] - xw[i] + s.astype(float) @ sy.cell, axis=1)
    assert (d < R + 1e-12).all()
    # nothing within R - 1e-9 is missing: compare counts with a dense numpy minimum-image check
    diff = xw[None, :, :] - xw[:, None, :]
    fr = diff @ np.linalg.inv(sy.cell)
    fr -= np.round(fr)
    dm = np.linalg.norm(fr @ sy.cell, axis=2)
    np.fill_diagonal(dm, np.inf)
    assert int((dm < R - 1e-9).sum()) <= len(i) <= int((dm < R + 1e-9).sum())
