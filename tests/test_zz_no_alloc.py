"""The neighbour-list entry point that allocates nothing (ctd_neighbors_noalloc).

It is for callers that cannot let the library allocate device memory (an MD code with its own
fixed memory pool, or one that must not allocate between set-up and teardown).  Its pair set
must equal the one the allocating entry point (ctd_build_neighbors + ctd_get_pairs) produces,
exactly, on consecutive calls that reuse the same static scratch array, and the oracle's
brute-force pair set; its image shifts are relative to the positions the caller passed, so
unwrapped positions give the same pair vectors.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synthetic as syn
from gpu_common import engine

pytestmark = pytest.mark.gpu


def _sorted(i, j, s):
    order = np.lexsort((s[:, 2], s[:, 1], s[:, 0], j, i))
    return i[order], j[order], s[order]


def _reference(eng, sy, cutoff, skin):
    pot = eng.Potential(32, T=1, n_species=4)
    n = pot.build_neighbors(sy.positions, sy.cell, cutoff=cutoff, skin=skin)
    out = pot.get_pairs(n)
    pot.close()
    return out


def _noalloc(sy, cutoff, skin, cap=None):
    import torch
    from paper_2506_04055_gb300 import _lib
    x = torch.tensor(sy.positions, dtype=torch.float64, device="cuda")
    H = np.ascontiguousarray(sy.cell, np.float64)
    cap = cap if cap is not None else 200 * sy.n
    pi = torch.full((max(cap, 1),), -1, dtype=torch.int32, device="cuda")
    pj = torch.full((max(cap, 1),), -1, dtype=torch.int32, device="cuda")
    ps = torch.zeros((max(cap, 1), 3), dtype=torch.int8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    code, n = _lib.ctd_neighbors_noalloc(sy.n, P(x), H.ctypes.data_as(ctypes.c_void_p), cutoff, skin,
                                         P(pi), P(pj), P(ps), cap, stream)
    torch.cuda.synchronize()
    return code, n, pi[:n].cpu().numpy(), pj[:n].cpu().numpy(), ps[:n].cpu().numpy()


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(orc):
    """ctd_get_pairs reports shifts relative to the wrapped positions; with the wrap counts m
    (x~ = x - m H) they become shifts relative to the caller's positions, n - m_j + m_i."""
    eng = engine()
    from paper_2506_04055_gb300 import _lib
    systems = [(syn.water_box(500, seed=3), 5.0, 1.0),      # 1,500 atoms
               (syn.fcc(6, 6, 6, jitter=0.05, seed=1), 5.0, 1.0),   # 864 atoms, fewer cells
               (syn.water_box(64, seed=0), 5.0, 0.0)]       # 192 atoms, multi-image cells
    for sy, rc, skin in systems:
        ri, rj, rs = _reference(eng, sy, rc, skin)
        _, m = orc.wrap(sy.positions, sy.cell)
        ref = _sorted(ri, rj, (rs.astype(np.int32) - m[rj] + m[ri]).astype(np.int8))
        code, n, i, j, s = _noalloc(sy, rc, skin)
        assert code == _lib.CTD_OK
        assert n == len(ref[0])
        got = _sorted(i, j, s)
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b)


def test_noalloc_limits():
    engine()
    from paper_2506_04055_gb300 import _lib
    sy = syn.water_box(64, seed=0)
    code, n, *_ = _noalloc(sy, 5.0, 1.0, cap=10)
    assert code == _lib.CTD_ERR_CAPACITY and n > 10
    big = syn.fcc(13, 13, 13, jitter=0.0)      # 8,788 atoms: within the atom limit
    code, n, *_ = _noalloc(big, 5.0, 1.0, cap=0)
    assert code == _lib.CTD_ERR_CAPACITY and n == 54 * big.n
    too_many = syn.fcc(21, 21, 21, jitter=0.0)  # 37,044 atoms > 32,768
    code, n, *_ = _noalloc(too_many, 5.0, 1.0, cap=0)
    assert code == _lib.CTD_ERR_INVALID_ARG and n == 0


def _caller_shifts_from_oracle(orc, positions, cell, R):
    """The oracle's brute-force pairs, with shifts made relative to the unwrapped positions:
    xw = x - m H, so xw_j - xw_i + n H = x_j - x_i + (n - m_j + m_i) H."""
    xw, m = orc.wrap(positions, cell)
    i, j, n = orc.pairs_brute(xw, cell, R)
    s = (n.astype(np.int32) - m[j] + m[i]).astype(np.int8)
    return _sorted(i, j, s)


def test_noalloc_matches_the_oracle_brute_force(orc):
    engine()
    from paper_2506_04055_gb300 import _lib
    for sy, rc, skin in ((syn.water_box(21, seed=2), 5.0, 1.0),     # 63 atoms, L = 8.6 A: many images
                         (syn.water_box(64, seed=0), 5.0, 1.0)):    # 192 atoms
        code, n, i, j, s = _noalloc(sy, rc, skin)
        assert code == _lib.CTD_OK
        ref = _caller_shifts_from_oracle(orc, sy.positions, sy.cell, rc + skin)
        assert n == len(ref[0])
        for a, b in zip(_sorted(i, j, s), ref):
            np.testing.assert_array_equal(a, b)


def test_noalloc_shifts_are_relative_to_unwrapped_positions(orc):
    """Atoms moved by whole lattice vectors (k in {-2..2}^3) keep every pair: the shifts change
    by k_i - k_j and the pair vectors x_j - x_i + shift . H computed from the caller's own
    positions are those of the wrapped input."""
    engine()
    from paper_2506_04055_gb300 import _lib
    sy = syn.water_box(21, seed=2)
    rng = np.random.default_rng(7)
    k = rng.integers(-2, 3, size=(sy.n, 3))
    moved = syn.System(sy.positions + k @ sy.cell, sy.species, sy.masses, sy.cell)
    code0, n0, i0, j0, s0 = _noalloc(sy, 5.0, 1.0)
    code1, n1, i1, j1, s1 = _noalloc(moved, 5.0, 1.0)
    assert code0 == code1 == _lib.CTD_OK and n0 == n1
    a, b = _sorted(i0, j0, s0), _sorted(i1, j1, (s1.astype(np.int32) + k[j1] - k[i1]).astype(np.int8))
    for u, w in zip(a, b):
        np.testing.assert_array_equal(u, w)
    ib, jb, sb = _sorted(i1, j1, s1)
    r_moved = moved.positions[jb] - moved.positions[ib] + sb.astype(np.float64) @ sy.cell
    r_plain = sy.positions[a[1]] - sy.positions[a[0]] + a[2].astype(np.float64) @ sy.cell
    np.testing.assert_allclose(np.sort(np.linalg.norm(r_moved, axis=1)), np.sort(np.linalg.norm(r_plain, axis=1)),
                               rtol=0, atol=1e-9)
    assert np.linalg.norm(r_moved, axis=1).max() < 6.0
    # and they agree with the oracle's brute force on the moved positions
    ref = _caller_shifts_from_oracle(orc, moved.positions, sy.cell, 6.0)
    for u, w in zip(_sorted(i1, j1, s1), ref):
        np.testing.assert_array_equal(u, w)


def test_noalloc_rejects_nonfinite_positions():
    engine()
    from paper_2506_04055_gb300 import _lib
    sy = syn.water_box(21, seed=2)
    x = sy.positions.copy()
    x[5, 2] = np.nan
    bad = syn.System(x, sy.species, sy.masses, sy.cell)
    code, n, *_ = _noalloc(bad, 5.0, 1.0)
    assert code == _lib.CTD_ERR_NONFINITE
    code, n, *_ = _noalloc(sy, 5.0, 1.0)      # the next call is unaffected
    assert code == _lib.CTD_OK and n > 0
