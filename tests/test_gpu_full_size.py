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


def _energy_job(args):
    vals, F, T, S, species, pos, box, w = args
    import oracle
    return oracle.painn(vals, F, 20, T, S, species, pos, box, weights=w, forces=False, virial=False)["energy"]


def _force_job(args):
    vals, F, T, S, species, pos, box, w, k = args
    import oracle
    return oracle.painn(vals, F, 20, T, S, species, pos, box, weights=w, virial=False)["forces"][k]


def _pool_map(fn, jobs):
    """The oracle's open clusters in a spawned process pool (one per host core)."""
    import multiprocessing
    import os
    from concurrent.futures import ProcessPoolExecutor
    n = max(1, min(len(jobs), os.cpu_count() or 1))
    with ProcessPoolExecutor(max_workers=n, mp_context=multiprocessing.get_context("spawn")) as ex:
        return list(ex.map(fn, jobs))


def _check(orc, sy, F, T, precision, e_rms, e_max, f_rms, f_max, e_samples, f_samples):
    """Per-atom energies of e_samples and forces on f_samples against the oracle's open clusters:
    RMS and largest error over the samples, relative to the RMS per-atom energy and force."""
    eng = engine()
    vals, blob = model(F, T, 1, seed=0)
    with eng.Potential(F, T=T, n_species=1, precision=precision, params=blob) as pot:
        out = pot.compute(sy.species, sy.positions, sy.cell, energies=True)
    f, e = out["forces"], out["energies"]
    assert np.isfinite(f).all() and np.isfinite(e).all()
    e_scale = float(np.sqrt(np.mean(e ** 2)))
    f_scale = float(np.sqrt(np.mean(f ** 2)))
    ejobs, fjobs = [], []
    for i in e_samples:
        idx, pos, box, _ = cluster(sy, i, T * RC + 1.0)
        ejobs.append((vals, F, T, 1, sy.species[idx], pos, box, (idx == i).astype(float)))
    for i in f_samples:
        idx, pos, box, r = cluster(sy, i, 2 * T * RC + 1.0)
        fjobs.append((vals, F, T, 1, sy.species[idx], pos, box, (r < T * RC + 0.5).astype(float),
                      int(np.nonzero(idx == i)[0][0])))
    ue = np.array(_pool_map(_energy_job, ejobs))
    fo = np.array(_pool_map(_force_job, fjobs))
    de = (e[e_samples] - ue) / e_scale
    df = (f[f_samples] - fo) / f_scale
    print(f"{precision}: energy error RMS {np.sqrt(np.mean(de ** 2)):.2e} max {np.abs(de).max():.2e} "
          f"({len(e_samples)} atoms); force error RMS {np.sqrt(np.mean(df ** 2)):.2e} max {np.abs(df).max():.2e} "
          f"({len(f_samples)} atoms)")
    assert np.sqrt(np.mean(de ** 2)) <= e_rms and np.abs(de).max() <= e_max, de
    assert np.sqrt(np.mean(df ** 2)) <= f_rms and np.abs(df).max() <= f_max, df
    return out


def test_bf16_1M_sampled_atoms(orc):
    """The benchmarked configuration: 1,000,188 atoms, F = 128, T = 3, BF16 (tensor-core kernels):
    32 per-atom energies and 8 forces.  BF16 operands: the sub-run's relative force RMSE is 9.1e-3;
    estimated from 24 force components its RMS can read up to ~1.3x that, so the sample's RMS is
    held to 1.5e-2 of the RMS force and single components to 5e-2."""
    sy = syn.fcc(63, 63, 63, jitter=0.05, seed=0)
    rng = np.random.default_rng(1)
    samples = [int(k) for k in rng.choice(sy.n, 32, replace=False)]
    _check(orc, sy, 128, 3, "bf16", e_rms=2e-2, e_max=6e-2, f_rms=1.5e-2, f_max=5e-2,
           e_samples=samples, f_samples=samples[:8])


def test_fp32_1p49M_sampled_atoms(orc):
    """1,492,992 atoms on the FP32 path (3n = 4.48M rows in the U/V GEMM): 16 energies, 4 forces."""
    sy = syn.fcc(72, 72, 72, jitter=0.05, seed=2)
    rng = np.random.default_rng(2)
    samples = [int(k) for k in rng.choice(sy.n, 16, replace=False)]
    out = _check(orc, sy, 128, 3, "fp32", e_rms=1e-5, e_max=2e-5, f_rms=1e-5, f_max=2e-5,
                 e_samples=samples, f_samples=samples[:4])
    assert np.abs(out["forces"].sum(0)).max() < 1e-5 * np.abs(out["forces"]).sum(0).max()
