"""Pins for the oracle's NVE velocity-Verlet loop (CPU only).

Forces from the potential drive every MD step (Results "Distributed potential computation";
the paper's runs use LAMMPS integrators, Methods "Molecular Dynamics Simulations").  Pins:
free flight with no forces (closed form x = x0 + v t), time reversibility of velocity Verlet,
and the second-order (dt^2) scaling of the energy error.
"""
import numpy as np
import pytest

import synthetic as syn


def test_free_flight_without_interaction_layers(orc):
    F, K, T, S = 4, 3, 0, 2           # T = 0: energy independent of positions, zero forces
    vals = syn.xavier_params(F, K, T, S, seed=0)
    sy = syn.water_box(8, seed=0)
    v0 = syn.maxwell_boltzmann(sy.masses, 300.0, seed=1)
    x, v, ep, ek = orc.nve(vals, F, K, T, S, sy.species, sy.masses, sy.positions, v0, sy.cell,
                           dt=0.5, nsteps=10)
    np.testing.assert_allclose(x, sy.positions + 10 * 0.5 * v0, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(v, v0)
    # kinetic energy of 300 K Maxwell-Boltzmann velocities: 3/2 N kB T within sampling noise
    assert ek[0] == pytest.approx(1.5 * sy.n * syn.KB_EV * 300.0, rel=0.35)


def _system():
    F, K, T, S = 8, 20, 2, 2
    vals = syn.xavier_params(F, K, T, S, seed=2)
    sy = syn.water_box(8, seed=3)
    v0 = syn.maxwell_boltzmann(sy.masses, 300.0, seed=4)
    return vals, (F, K, T, S), sy, v0


def test_time_reversibility(orc):
    vals, dims, sy, v0 = _system()
    x1, v1, _, _ = orc.nve(vals, *dims, sy.species, sy.masses, sy.positions, v0, sy.cell, 0.5, 20)
    x2, v2, _, _ = orc.nve(vals, *dims, sy.species, sy.masses, x1, -v1, sy.cell, 0.5, 20)
    np.testing.assert_allclose(x2, sy.positions, atol=1e-9)
    np.testing.assert_allclose(-v2, v0, atol=1e-9)


def test_energy_error_scales_as_dt_squared(orc):
    vals, dims, sy, v0 = _system()
    errs = []
    for dt, n in ((0.5, 20), (0.25, 40)):
        _, _, ep, ek = orc.nve(vals, *dims, sy.species, sy.masses, sy.positions, v0, sy.cell, dt, n)
        etot = ep + ek
        errs.append(np.abs(etot - etot[0]).max())
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.0, (errs, ratio)
