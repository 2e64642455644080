"""Full-size parity on sampled atoms: the 1,000,188-atom fcc workload (BF16, as benchmarked) and a
1,492,992-atom fcc system on the FP32 path (beyond 1.4M atoms, where the FP32 GEMM's row count
once exceeded a grid limit), against the FP64 oracle atom by atom.

U_i depends only on the atoms within T rc of atom i (T message-passing steps of range rc), and the
force on atom i only on the U_j of atoms within T rc of it (Results, "Distributed potential
computation": energy sum and sum rule).  So the oracle evaluates, for a sampled atom, an open
cluster of the periodic system: for U_i the atoms within T rc + 1 A with weight 1 on atom i; for
F_i the atoms within 2 T rc + 1 A with weight 1 on every atom within T rc + 0.5 A of atom i."""
import numpy as np
import pytest

import synthetic as syn
from gpu_common import engine, model

pytestmark = pytest.mark.gpu

RC = 5.0


def cluster(sy, i, radius):
    """Atoms (and periodic images) within `radius` of atom i, centred on it, in an open box."""
    H = sy.cell
    d = sy.positions - sy.positions[i]
    G = np.linalg.inv(H)
    d -= np.round(d @ G) @ H                  # minimum image (the box is far wider than 2 radius)
    r = np.linalg.norm(d, axis=1)
    idx = np.nonzero(r < radius)[0]
    pos = d[idx] + radius + RC + 1.0
    box = np.eye(3) * (2 * radius + 2 * RC + 2.0)
    return idx, pos, box, r[idx]


def oracle_energy_of(orc, vals, F, T, S, sy, i):
    idx, pos, box, _ = cluster(sy, i, T * RC + 1.0)
    w = (idx == i).astype(float)
    return orc.painn(vals, F, 20, T, S, sy.species[idx], pos, box, weights=w, forces=False, virial=False)["energy"]


def oracle_force_on(orc, vals, F, T, S, sy, i):
    idx, pos, box, r = cluster(sy, i, 2 * T * RC + 1.0)
    w = (r < T * RC + 0.5).astype(float)
    out = orc.painn(vals, F, 20, T, S, sy.species[idx], pos, box, weights=w, virial=False)
    return out["forces"][np.nonzero(idx == i)[0][0]]


def _check(orc, sy, F, T, precision, e_tol, f_tol, samples):
    eng = engine()
    vals, blob = model(F, T, 1, seed=0)
    with eng.Potential(F, T=T, n_species=1, precision=precision, params=blob) as pot:
        out = pot.compute(sy.species, sy.positions, sy.cell, energies=True)
    f, e = out["forces"], out["energies"]
    assert np.isfinite(f).all() and np.isfinite(e).all()
    e_scale = float(np.sqrt(np.mean(e ** 2)))
    f_scale = float(np.sqrt(np.mean(f ** 2)))
    for i in samples:
        ue = oracle_energy_of(orc, vals, F, T, 1, sy, i)
        assert abs(e[i] - ue) <= e_tol * e_scale, (i, e[i], ue)
    fo = oracle_force_on(orc, vals, F, T, 1, sy, samples[0])
    assert np.abs(f[samples[0]] - fo).max() <= f_tol * f_scale, (f[samples[0]], fo)
    return out


def test_bf16_1M_sampled_atoms(orc):
    """The benchmarked configuration: 1,000,188 atoms, F = 128, T = 3, BF16 (tensor-core kernels)."""
    sy = syn.fcc(63, 63, 63, jitter=0.05, seed=0)
    rng = np.random.default_rng(1)
    samples = [int(k) for k in rng.integers(0, sy.n, 3)]
    # BF16 operands: per-atom errors of a few 1e-2 of the scales (RMS force error 9.5e-3)
    _check(orc, sy, 128, 3, "bf16", e_tol=5e-2, f_tol=6e-2, samples=samples)


def test_fp32_1p49M_sampled_atoms(orc):
    """1,492,992 atoms on the FP32 path (3n = 4.48M rows in the U/V GEMM)."""
    sy = syn.fcc(72, 72, 72, jitter=0.05, seed=2)
    rng = np.random.default_rng(2)
    samples = [int(k) for k in rng.integers(0, sy.n, 3)]
    out = _check(orc, sy, 128, 3, "fp32", e_tol=2e-5, f_tol=2e-5, samples=samples)
    assert np.abs(out["forces"].sum(0)).max() < 1e-5 * np.abs(out["forces"]).sum(0).max()
