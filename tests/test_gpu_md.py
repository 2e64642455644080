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


def _run_nvt_pair(orc, temperature, tau, chain, nsteps, dt, v_temp=300.0, skin=1.0):
    eng = engine()
    F, T, S = 64, 3, 2
    sy = syn.water_box(64, seed=0)
    vals, blob = model(F, T, S, seed=0)
    v0 = syn.maxwell_boltzmann(sy.masses, v_temp, seed=0)
    o = orc.nvt(vals, F, 20, T, S, sy.species, sy.masses, sy.positions, v0, sy.cell, dt, nsteps,
                temperature=temperature, tau=tau, chain=chain)
    with eng.Potential(F, T=T, n_species=S, params=blob) as pot:
        pot.md_set_state(sy.species, sy.masses, sy.positions, v0, sy.cell, skin=skin)
        pot.md_set_thermostat(temperature, tau, chain)
        ep, ek, _ = pot.md_run(nsteps, dt)
        xi, vxi, eth = pot.md_get_thermostat(nsteps)
        x, v = pot.md_get_state()
    return (x, v, ep, ek, eth, xi, vxi), o


@pytest.mark.parametrize("chain", [1, 3])
def test_water192_nvt_tracks_oracle(orc, chain):
    """Nose-Hoover chain NVT, 100 steps of 0.5 fs with a strong thermostat (tau = 20 fs, target
    600 K from 300 K): positions, energies, chain state and the conserved extended energy
    follow the oracle's FP64 trajectory."""
    g, o = _run_nvt_pair(orc, 600.0, 20.0, chain, 100, 0.5)
    x, v, ep, ek, eth, xi, vxi = g
    xo, vo, epo, eko, etho, xio, vxio = o
    assert np.abs(x - xo).max() < 1e-4
    assert np.abs(v - vo).max() < 1e-5
    np.testing.assert_allclose(ep, epo, rtol=0, atol=1e-4)
    np.testing.assert_allclose(ek, eko, rtol=0, atol=1e-4)
    np.testing.assert_allclose(eth, etho, rtol=0, atol=1e-4)
    np.testing.assert_allclose(vxi, vxio, rtol=1e-4, atol=1e-9)
    np.testing.assert_allclose(xi, xio, rtol=1e-4, atol=1e-9)
    # the thermostat did work, and the extended energy is conserved as in the oracle
    assert np.abs(eth - eth[0]).max() > 0.1
    h, ho = ep + ek + eth, epo + eko + etho
    assert np.abs(h - h[0]).max() < 2 * np.abs(ho - ho[0]).max() + 1e-4


def test_nvt_heavy_thermostat_equals_nve():
    """tau = 1e12 fs: the chain never moves and the trajectory is the NVE one."""
    eng = engine()
    F, T, S = 64, 3, 2
    sy = syn.water_box(64, seed=1)
    _, blob = model(F, T, S, seed=1)
    v0 = syn.maxwell_boltzmann(sy.masses, 300.0, seed=1)
    out = []
    for chain in (0, 3):
        with eng.Potential(F, T=T, n_species=S, params=blob) as pot:
            pot.md_set_state(sy.species, sy.masses, sy.positions, v0, sy.cell, skin=1.0)
            if chain:
                pot.md_set_thermostat(300.0, 1e12, chain)
            ep, ek, _ = pot.md_run(40, 0.5)
            out.append((ep, ek) + pot.md_get_state())
    for a, b in zip(out[0], out[1]):
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-10 * max(1.0, np.abs(a).max()))


def test_thermostat_arguments_are_checked():
    eng = engine()
    _, blob = model(64, 3, 2, seed=0)
    with eng.Potential(64, T=3, n_species=2, params=blob) as pot:
        for bad in ((300.0, 100.0, 17), (0.0, 100.0, 3), (300.0, -1.0, 3), (float("nan"), 100.0, 3)):
            with pytest.raises(eng.CtdError):
                pot.md_set_thermostat(*bad)
        with pytest.raises(eng.CtdError):
            pot.md_get_thermostat()


def test_nvt_checkpoint_restart():
    """State and chain state saved mid-run and restored into a new context continue the NVT
    trajectory (new neighbour list: agreement to FP32 summation order)."""
    eng = engine()
    F, T, S = 64, 3, 2
    sy = syn.water_box(64, seed=2)
    _, blob = model(F, T, S, seed=2)
    v0 = syn.maxwell_boltzmann(sy.masses, 300.0, seed=2)
    with eng.Potential(F, T=T, n_species=S, params=blob) as pot:
        pot.md_set_state(sy.species, sy.masses, sy.positions, v0, sy.cell, skin=1.0)
        pot.md_set_thermostat(500.0, 25.0, 3)
        pot.md_run(30, 0.5)
        x_ref, v_ref = pot.md_get_state()
        xi_ref, vxi_ref, _ = pot.md_get_thermostat()
    with eng.Potential(F, T=T, n_species=S, params=blob) as pot:
        pot.md_set_state(sy.species, sy.masses, sy.positions, v0, sy.cell, skin=1.0)
        pot.md_set_thermostat(500.0, 25.0, 3)
        pot.md_run(12, 0.5)
        x12, v12 = pot.md_get_state()
        xi12, vxi12, _ = pot.md_get_thermostat()
    with eng.Potential(F, T=T, n_species=S, params=blob) as pot:
        pot.md_set_state(sy.species, sy.masses, x12, v12, sy.cell, skin=1.0)
        pot.md_set_thermostat(500.0, 25.0, 3)
        pot.md_set_thermostat_state(xi12, vxi12)
        pot.md_run(18, 0.5)
        x, v = pot.md_get_state()
        xi, vxi, _ = pot.md_get_thermostat()
    assert np.abs(vxi12).max() > 1e-4
    np.testing.assert_allclose(x, x_ref, rtol=0, atol=1e-6)
    np.testing.assert_allclose(v, v_ref, rtol=0, atol=1e-7)
    np.testing.assert_allclose(vxi, vxi_ref, rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(xi, xi_ref, rtol=1e-6, atol=1e-12)
