"""GPU neighbour build vs the FP64 oracle: the sorted pair set must match bit for bit.

The neighbour graph with skin is the paper's input graph (Results "Distributed potential
computation"); the test and its rounding are fixed in include/painn.h, so any difference in a
single (i, j, n) is a failure.
"""
import numpy as np
import pytest

import synthetic as syn
from gpu_common import engine

pytestmark = pytest.mark.gpu


def _gpu_pairs(eng, sy, cutoff, skin):
    pot = eng.Potential(64, T=1, n_species=4)
    n = pot.build_neighbors(sy.positions, sy.cell, cutoff=cutoff, skin=skin)
    i, j, s = pot.get_pairs(n)
    pot.close()
    return i, j, s


def _oracle_pairs(orc, sy, R):
    xw, _ = orc.wrap(sy.positions, sy.cell)
    return orc.pairs_cells(xw, sy.cell, R)


def _assert_same(a, b):
    assert len(a[0]) == len(b[0]), (len(a[0]), len(b[0]))
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("cutoff,skin", [(5.0, 0.0), (5.0, 1.0), (3.0, 0.5)])
def test_water192_pairs_exact(orc, cutoff, skin):
    eng = engine()
    sy = syn.water_box(64, seed=0)
    _assert_same(_gpu_pairs(eng, sy, cutoff, skin), _oracle_pairs(orc, sy, cutoff + skin))


def test_water96k_pairs_exact_first_frame(orc):
    """Water box of 32,000 molecules (96,000 atoms, L = 98.6 A), cutoff 5 + skin 1."""
    eng = engine()
    sy = syn.water_box(32000, seed=0)
    _assert_same(_gpu_pairs(eng, sy, 5.0, 1.0), _oracle_pairs(orc, sy, 6.0))


@pytest.mark.parametrize("cells", [(1, 1, 1), (2, 2, 2), (3, 2, 5)])
def test_fcc_pairs_exact_small_cells(orc, cells):
    """Cells thinner than 2 (rc + skin): every neighbour may be a periodic image."""
    eng = engine()
    sy = syn.fcc(*cells, jitter=0.05, seed=1)
    _assert_same(_gpu_pairs(eng, sy, 5.0, 1.0), _oracle_pairs(orc, sy, 6.0))


def test_fcc_perfect_shell_counts(orc):
    eng = engine()
    sy = syn.fcc(3, 3, 3, a=4.05, jitter=0.0)
    for frac, expect in ((0.8, 12), (1.05, 18), (1.3, 42), (1.5, 54)):
        i, j, s = _gpu_pairs(eng, sy, frac * 4.05, 0.0)
        assert (np.bincount(i, minlength=sy.n) == expect).all()


def test_triclinic_mixture_pairs_exact(orc):
    eng = engine()
    sy = syn.mixture(n_chain=40, n_water=400, seed=2)
    _assert_same(_gpu_pairs(eng, sy, 5.0, 1.0), _oracle_pairs(orc, sy, 6.0))


def test_unwrapped_and_single_atom(orc):
    eng = engine()
    rng = np.random.default_rng(5)
    H = np.array([[6.5, 0, 0], [0.7, 6.0, 0], [-0.5, 0.9, 7.2]])
    x = rng.uniform(-20, 20, size=(30, 3))          # far outside the cell
    sy = syn.System(x, np.zeros(30, np.int32), np.ones(30), H)
    _assert_same(_gpu_pairs(eng, sy, 5.0, 1.0), _oracle_pairs(orc, sy, 6.0))
    one = syn.System(np.array([[0.3, 0.2, 0.1]]), np.zeros(1, np.int32), np.ones(1), np.eye(3) * 2.0)
    i, j, s = _gpu_pairs(eng, one, 3.0, 0.5)
    assert len(i) == 26        # 2 |n| < 3.5  <=>  |n|^2 in {1, 2, 3}: 6 + 12 + 8 lattice points
    _assert_same((i, j, s), _oracle_pairs(orc, one, 3.5))


def test_fcc_million_sampled_rows(orc):
    """Full-size 63^3-cell fcc (1,000,188 atoms): the whole GPU pair set equals the oracle's
    linked-cell set (the oracle's cell search is pinned to brute force on small systems)."""
    eng = engine()
    sy = syn.fcc(63, 63, 63, a=4.05, jitter=0.05, seed=0)
    g = _gpu_pairs(eng, sy, 5.0, 1.0)
    o = _oracle_pairs(orc, sy, 6.0)
    _assert_same(g, o)
