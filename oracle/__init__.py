"""FP64 CPU oracle for the PaiNN-form energy / force / virial path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
this package.  The product path (``paper_2506_04055_gb300``) never imports, links or runs it.
It shares no code with the CUDA library; both read the same inputs from ``synthetic``.

``oracle.c`` holds the arithmetic (plain loops, double precision, compiled with
``-ffp-contract=off``); this module compiles it with gcc and marshals numpy arrays.

What pins each function (tests/test_oracle_*.py):
  * pairs_brute / pairs_cells -- pinned (brute force vs cells, fcc shell counts, image counts)
  * painn                     -- pinned (closed forms, invariances, finite differences,
                                 strain finite differences, supercell extensivity)
  * nve                       -- pinned (time reversibility, dt^2 energy-error scaling)
  * nvt                       -- pinned (NVE limit, conserved extended energy and its dt^2
                                 scaling, time reversibility, mean temperature of free particles)
  * local.local_model         -- the strictly local edge model in PyTorch CPU float64 (module
                                 local.py); pinned (scalar dimer and trimer evaluations, finite
                                 differences, invariances, strict locality, cutoff continuity)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-D_DEFAULT_SOURCE"]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, no contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Model(ctypes.Structure):
    _fields_ = [("F", ctypes.c_int32), ("K", ctypes.c_int32), ("T", ctypes.c_int32),
                ("S", ctypes.c_int32), ("rc", ctypes.c_double), ("eps", ctypes.c_double),
                ("e_scale", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_inv_transpose.argtypes = [P, P]
            lib.orc_wrap.argtypes = [ctypes.c_int64, P, P, P, P]
            for f in (lib.orc_pairs_brute, lib.orc_pairs_cells):
                f.argtypes = [ctypes.c_int64, P, P, ctypes.c_double, P, P, P, ctypes.c_int64]
                f.restype = ctypes.c_int64
            lib.orc_param_count.argtypes = [ctypes.c_int32] * 4
            lib.orc_param_count.restype = ctypes.c_int64
            lib.orc_painn.argtypes = [P, P, ctypes.c_int64, P, P, P, ctypes.c_int64, P, P, P, P, P, P,
                                      P, P]
            lib.orc_painn.restype = ctypes.c_int
            lib.orc_nve.argtypes = [P, P, ctypes.c_int64, P, P, P, P, P, ctypes.c_double,
                                    ctypes.c_int32, P, P]
            lib.orc_nvt.argtypes = [P, P, ctypes.c_int64, P, P, P, P, P, ctypes.c_double,
                                    ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                    P, P, P, P, P]
            lib.orc_nvt.restype = ctypes.c_int
            lib.orc_nve.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def inv_transpose(cell) -> np.ndarray:
    """G = H^{-T} by the cofactor formula (the form the canonical pair test uses)."""
    H = _f64(cell, (3, 3))
    G = np.empty((3, 3))
    _load().orc_inv_transpose(_p(H), _p(G))
    return G


def wrap(positions, cell):
    """Wrapped positions xw and integer translations m with xw = x - m @ H (up to rounding)."""
    x = _f64(positions, (-1, 3))
    H = _f64(cell, (3, 3))
    xw = np.empty_like(x)
    m = np.empty(x.shape, np.int32)
    _load().orc_wrap(x.shape[0], _p(x), _p(H), _p(xw), _p(m))
    return xw, m


def _pairs(fn, xw, cell, R):
    xw = _f64(xw, (-1, 3))
    H = _f64(cell, (3, 3))
    n = xw.shape[0]
    cnt = fn(n, _p(xw), _p(H), float(R), None, None, None, 0)
    if cnt < 0:
        raise MemoryError("oracle pair search failed")
    i = np.empty(cnt, np.int32)
    j = np.empty(cnt, np.int32)
    s = np.empty((cnt, 3), np.int8)
    fn(n, _p(xw), _p(H), float(R), _p(i), _p(j), _p(s), cnt)
    return i, j, s


def sort_pairs(i, j, s):
    """Order pairs by (i, j, n1, n2, n3)."""
    order = np.lexsort((s[:, 2], s[:, 1], s[:, 0], j, i))
    return i[order], j[order], s[order]


def pairs_brute(xw, cell, R):
    """All (i, j, n) with |xw_j - xw_i + n H| < R by exhaustive search; sorted.  Pinned."""
    return _pairs(_load().orc_pairs_brute, xw, cell, R)


def pairs_cells(xw, cell, R, sort=True):
    """Same set by a linked-cell search (checked against pairs_brute); sorted if asked."""
    i, j, s = _pairs(_load().orc_pairs_cells, xw, cell, R)
    return sort_pairs(i, j, s) if sort else (i, j, s)


def param_count(F, K, T, S) -> int:
    return int(_load().orc_param_count(F, K, T, S))


def painn(params, F, K, T, S, species, positions, cell, pairs=None, rc=5.0, eps=1e-8,
          e_scale=1.0, forces=True, virial=True, weights=None):
    """Energy, per-atom energies, forces and virial in FP64.

    ``pairs`` = (i, j, n) over the given positions (edges beyond rc are ignored); when None
    they are found with the oracle's own cell search on wrapped positions.  ``weights`` [n]
    (default all ones): the energy is sum_i w_i U_i and forces / virial are its derivatives
    (one processor's share of a spatial decomposition when w marks the owned atoms).
    Returns dict(energy, energies (unweighted U_i), forces [n,3] or None, virial [3,3] or None).
    """
    lib = _load()
    params = _f64(params)
    if params.size != param_count(F, K, T, S):
        raise ValueError("parameter vector has the wrong length")
    x = _f64(positions, (-1, 3))
    H = _f64(cell, (3, 3))
    Z = np.ascontiguousarray(species, np.int32)
    n = x.shape[0]
    if pairs is None:
        x, _ = wrap(x, H)
        pairs = pairs_cells(x, H, rc, sort=False)
    pi, pj, pn = (np.ascontiguousarray(pairs[0], np.int32), np.ascontiguousarray(pairs[1], np.int32),
                  np.ascontiguousarray(pairs[2], np.int8))
    md = Model(F, K, T, S, rc, eps, e_scale)
    E = np.zeros(1)
    Ei = np.empty(n)
    Fo = np.empty((n, 3)) if forces else None
    Wv = np.empty((3, 3)) if virial else None
    w = None if weights is None else _f64(weights)
    if w is not None and w.shape != (n,):
        raise ValueError("weights must have one entry per atom")
    rcode = lib.orc_painn(ctypes.byref(md), _p(params), n, _p(Z), _p(x), _p(H), pi.size, _p(pi),
                          _p(pj), _p(pn), _p(w), _p(E), _p(Ei), _p(Fo), _p(Wv))
    if rcode != 0:
        raise RuntimeError(f"orc_painn failed with {rcode}")
    return {"energy": float(E[0]), "energies": Ei, "forces": Fo, "virial": Wv}


def nve(params, F, K, T, S, species, masses, positions, velocities, cell, dt, nsteps, rc=5.0,
        eps=1e-8, e_scale=1.0):
    """Velocity-Verlet NVE trajectory.  Returns (x, v, epot[nsteps+1], ekin[nsteps+1])."""
    lib = _load()
    x = _f64(positions, (-1, 3)).copy()
    v = _f64(velocities, (-1, 3)).copy()
    H = _f64(cell, (3, 3))
    Z = np.ascontiguousarray(species, np.int32)
    m = _f64(masses)
    ep = np.empty(nsteps + 1)
    ek = np.empty(nsteps + 1)
    md = Model(F, K, T, S, rc, eps, e_scale)
    rcode = lib.orc_nve(ctypes.byref(md), _p(_f64(params)), x.shape[0], _p(Z), _p(m), _p(H),
                        _p(x), _p(v), float(dt), int(nsteps), _p(ep), _p(ek))
    if rcode != 0:
        raise RuntimeError(f"orc_nve failed with {rcode}")
    return x, v, ep, ek


def nvt(params, F, K, T, S, species, masses, positions, velocities, cell, dt, nsteps, temperature, tau,
        chain=3, xi=None, vxi=None, rc=5.0, eps=1e-8, e_scale=1.0):
    """Nose-Hoover chain NVT trajectory (temperature in K, tau and dt in fs).  Returns
    (x, v, epot, ekin, ethermo, xi, vxi): ethermo is the chain's energy, epot + ekin + ethermo
    the conserved quantity; xi / vxi the chain state after the run (pass them back to continue)."""
    lib = _load()
    x = _f64(positions, (-1, 3)).copy()
    v = _f64(velocities, (-1, 3)).copy()
    H = _f64(cell, (3, 3))
    Z = np.ascontiguousarray(species, np.int32)
    m = _f64(masses)
    xi = np.zeros(chain) if xi is None else _f64(xi).copy()
    vxi = np.zeros(chain) if vxi is None else _f64(vxi).copy()
    ep, ek, eth = np.empty(nsteps + 1), np.empty(nsteps + 1), np.empty(nsteps + 1)
    md = Model(F, K, T, S, rc, eps, e_scale)
    rcode = lib.orc_nvt(ctypes.byref(md), _p(_f64(params)), x.shape[0], _p(Z), _p(m), _p(H), _p(x), _p(v),
                        float(dt), int(nsteps), float(temperature), float(tau), int(chain), _p(xi), _p(vxi),
                        _p(ep), _p(ek), _p(eth))
    if rcode != 0:
        raise RuntimeError(f"orc_nvt failed with {rcode}")
    return x, v, ep, ek, eth, xi, vxi

