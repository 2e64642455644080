"""Pins for the oracle's Nose-Hoover chain NVT loop (CPU only).

The paper's production and timing runs are NVT with a Nose-Hoover thermostat of damping
parameter tau (Methods, "MD simulations").  The oracle integrates a chain of M thermostats with
the symmetric Trotter splitting (chain half step, velocity Verlet, chain half step).  Pins:
  * tau -> infinity (infinitely heavy thermostats) reproduces the NVE trajectory;
  * the extended energy H = U + K + sum_j Q_j vxi_j^2 / 2 + Nf kT xi_1 + kT sum_{j>1} xi_j is
    conserved, with an error that scales as dt^2 (second-order integrator);
  * time reversibility: reversing the velocities and the thermostat velocities retraces the path;
  * for free particles and one thermostat, dvxi/dt = (2K - Nf kT)/Q makes the time average of
    2K / (Nf kB) equal the target temperature up to Q (vxi(t) - vxi(0)) / (t Nf kB);
  * the chain length matters (M = 1 and M = 3 give different trajectories, both conserving H).
"""
import numpy as np
import pytest

import synthetic as syn

KB = 8.617333262e-5


def _system(T=2, seed=3):
    F, K, S = 8, 20, 2
    vals = syn.xavier_params(F, K, T, S, seed=2)
    sy = syn.water_box(8, seed=seed)
    v0 = syn.maxwell_boltzmann(sy.masses, 300.0, seed=4)
    return vals, (F, K, T, S), sy, v0


def test_boltzmann_constant_matches_generators():
    assert KB == pytest.approx(syn.KB_EV, rel=1e-9)


def test_heavy_thermostat_is_nve(orc):
    vals, dims, sy, v0 = _system()
    x1, v1, ep1, ek1 = orc.nve(vals, *dims, sy.species, sy.masses, sy.positions, v0, sy.cell, 0.5, 20)
    x2, v2, ep2, ek2, eth, xi, vxi = orc.nvt(vals, *dims, sy.species, sy.masses, sy.positions, v0, sy.cell, 0.5,
                                             20, temperature=300.0, tau=1e12, chain=3)
    np.testing.assert_allclose(x2, x1, rtol=0, atol=1e-10)
    np.testing.assert_allclose(v2, v1, rtol=0, atol=1e-12)
    np.testing.assert_allclose(ep2, ep1, rtol=1e-12, atol=1e-12)
    assert np.abs(vxi).max() < 1e-20


@pytest.mark.parametrize("chain", [1, 3])
def test_extended_energy_conserved_dt_squared(orc, chain):
    vals, dims, sy, v0 = _system()
    errs, drifts = [], []
    for dt, n in ((0.5, 40), (0.25, 80)):
        _, _, ep, ek, eth, _, vxi = orc.nvt(vals, *dims, sy.species, sy.masses, sy.positions, v0, sy.cell, dt, n,
                                            temperature=600.0, tau=10.0, chain=chain)
        h = ep + ek + eth
        errs.append(np.abs(h - h[0]).max())
        # the thermostat is active: the chain energy moves by much more than the error of H
        drifts.append(np.abs(eth - eth[0]).max())
        assert np.abs(vxi).max() > 1e-4
    assert drifts[0] > 20 * errs[0]
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.0, (errs, ratio)


def test_time_reversibility(orc):
    vals, dims, sy, v0 = _system()
    x1, v1, _, _, _, xi1, vxi1 = orc.nvt(vals, *dims, sy.species, sy.masses, sy.positions, v0, sy.cell, 0.5, 30,
                                         temperature=500.0, tau=15.0, chain=3)
    x2, v2, _, _, _, xi2, vxi2 = orc.nvt(vals, *dims, sy.species, sy.masses, x1, -v1, sy.cell, 0.5, 30,
                                         temperature=500.0, tau=15.0, chain=3, xi=xi1, vxi=-vxi1)
    np.testing.assert_allclose(x2, sy.positions, rtol=0, atol=1e-9)
    np.testing.assert_allclose(-v2, v0, rtol=0, atol=1e-9)
    np.testing.assert_allclose(-vxi2, np.zeros(3), rtol=0, atol=1e-11)
    np.testing.assert_allclose(xi2, np.zeros(3), rtol=0, atol=1e-9)


def test_free_particles_mean_temperature(orc):
    """No interaction layers (zero forces), one thermostat: the time average of the kinetic
    temperature converges to the target, with the bound set by the final thermostat velocity."""
    F, K, T, S = 4, 3, 0, 2
    vals = syn.xavier_params(F, K, T, S, seed=0)
    sy = syn.water_box(8, seed=0)
    v0 = syn.maxwell_boltzmann(sy.masses, 100.0, seed=5)
    n = sy.n
    Nf = 3 * n - 3
    target, tau, dt, steps = 300.0, 20.0, 1.0, 4000
    _, _, ep, ek, eth, _, vxi = orc.nvt(vals, F, K, T, S, sy.species, sy.masses, sy.positions, v0, sy.cell, dt,
                                        steps, temperature=target, tau=tau, chain=1)
    Tk = 2.0 * ek / (Nf * KB)
    # trapezoid average over the run
    mean = (0.5 * (Tk[0] + Tk[-1]) + Tk[1:-1].sum()) / steps
    Q = Nf * KB * target * tau * tau
    bound = Q * abs(vxi[0]) / (steps * dt * Nf * KB)   # vxi starts at 0
    assert abs(mean - target) <= 1.1 * bound + 2e-3 * target, (mean, bound)
    assert abs(Tk[0] - 100.0) < 60.0 and Tk.max() > 1.5 * target * 0.8   # it was heated
    h = ep + ek + eth
    assert np.abs(h - h[0]).max() < 1e-4 * abs(ek).max()


def test_chain_length_changes_the_path(orc):
    vals, dims, sy, v0 = _system()
    a = orc.nvt(vals, *dims, sy.species, sy.masses, sy.positions, v0, sy.cell, 0.5, 40, temperature=600.0,
                tau=10.0, chain=1)
    b = orc.nvt(vals, *dims, sy.species, sy.masses, sy.positions, v0, sy.cell, 0.5, 40, temperature=600.0,
                tau=10.0, chain=3)
    assert np.abs(a[0] - b[0]).max() > 1e-6
