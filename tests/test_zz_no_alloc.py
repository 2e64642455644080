"""The neighbour-list entry point that allocates nothing (ctd_neighbors_noalloc).

It is for callers that cannot let the library allocate device memory (an MD code with its own
fixed memory pool, or one that must not allocate between set-up and teardown).  Its pair set
must equal the one the allocating entry point (ctd_build_neighbors + ctd_get_pairs) produces,
exactly, on consecutive calls that reuse the same static scratch array.  This file is
collected last on purpose.
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


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    eng = engine()
    from paper_2506_04055_gb300 import _lib
    systems = [(syn.water_box(500, seed=3), 5.0, 1.0),      # 1,500 atoms
               (syn.fcc(6, 6, 6, jitter=0.05, seed=1), 5.0, 1.0),   # 864 atoms, fewer cells
               (syn.water_box(64, seed=0), 5.0, 0.0)]       # 192 atoms, multi-image cells
    for sy, rc, skin in systems:
        ref = _reference(eng, sy, rc, skin)
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
