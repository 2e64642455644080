"""Resident NVE loop (ctd_md_run) vs the oracle's FP64 velocity Verlet.

192-atom water box, F = 64, 3 layers, Xavier weights from seed 0, 300 K Maxwell-Boltzmann
velocities, dt = 0.5 fs, 100 steps.  The GPU path is FP32 (forces agree with the oracle to
~1e-6 relative), so trajectories agree closely over 100 steps; the total-energy drift is
reported.  A hotter, longer run checks that Verlet-list rebuilds (skin/2 rule) keep the
dynamics on the rebuild-every-step oracle trajectory."""
import numpy as np
import pytest

import synthetic as syn
from gpu_common import engine, model

pytestmark = pytest.mark.gpu


def _nve_pair(orc, eng, sy, v0, F, T, S, dt, nsteps, skin, seed=0, bias=0.0):
    vals, blob = model(F, T, S, seed=seed, bias=bias)
    x_o, v_o, ep_o, ek_o = orc.nve(vals, F, 20, T, S, sy.species, sy.masses, sy.positions, v0, sy.cell, dt, nsteps)
    with eng.Potential(F, T=T, n_species=S, params=blob) as pot:
        pot.md_set_state(sy.species, sy.masses, sy.positions, v0, sy.cell, skin=skin)
        ep, ek, nreb = pot.md_run(nsteps, dt)
        x, v = pot.md_get_state()
    return (x, v, ep, ek, nreb), (x_o, v_o, ep_o, ek_o)


def test_water192_nve_100_steps(orc):
    eng = engine()
    sy = syn.water_box(64, seed=0)
    v0 = syn.maxwell_boltzmann(sy.masses, 300.0, seed=0)
    (x, v, ep, ek, nreb), (xo, vo, epo, eko) = _nve_pair(orc, eng, sy, v0, 64, 3, 2, 0.5, 100, 1.0)
    assert np.abs(x - xo).max() < 1e-4
    assert np.abs(v - vo).max() < 1e-5
    np.testing.assert_allclose(ep, epo, rtol=0, atol=1e-4)
    etot, etot_o = ep + ek, epo + eko
    drift = (etot[-1] - etot[0]) / sy.n
    drift_o = (etot_o[-1] - etot_o[0]) / sy.n
    print(f"water192 NVE 100 x 0.5 fs: drift {drift:.3e} eV/atom (oracle {drift_o:.3e}), rebuilds {nreb}")
    assert abs(drift - drift_o) < 1e-6


def test_hot_run_rebuilds_track_oracle(orc):
    """3000 K fcc cell, dt 1 fs, skin 0.4 A: several rebuilds within 60 steps."""
    eng = engine()
    sy = syn.fcc(3, 3, 3, jitter=0.05, seed=2)
    v0 = syn.maxwell_boltzmann(sy.masses, 3000.0, seed=3)
    (x, v, ep, ek, nreb), (xo, vo, epo, eko) = _nve_pair(orc, eng, sy, v0, 64, 2, 1, 1.0, 60, 0.4, seed=1)
    assert nreb >= 2
    assert np.abs(x - xo).max() < 1e-4
    np.testing.assert_allclose(ep + ek, epo + eko, rtol=0, atol=1e-4)
    print(f"fcc108 3000 K: rebuilds {nreb}, drift {(ep[-1] + ek[-1] - ep[0] - ek[0]) / sy.n:.3e} eV/atom")


def test_md_resume_equals_single_run():
    """Two calls of 20 steps give the same state as one call of 40 (state stays resident)."""
    eng = engine()
    sy = syn.water_box(30, seed=4)
    v0 = syn.maxwell_boltzmann(sy.masses, 300.0, seed=5)
    _, blob = model(64, 2, 2, seed=6)
    with eng.Potential(64, T=2, n_species=2, params=blob) as pot:
        pot.md_set_state(sy.species, sy.masses, sy.positions, v0, sy.cell, skin=1.0)
        pot.md_run(20, 0.5)
        pot.md_run(20, 0.5)
        xa, va = pot.md_get_state()
    with eng.Potential(64, T=2, n_species=2, params=blob) as pot:
        pot.md_set_state(sy.species, sy.masses, sy.positions, v0, sy.cell, skin=1.0)
        pot.md_run(40, 0.5)
        xb, vb = pot.md_get_state()
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)
