"""Served replicas against the FP64 oracle (continuous batching of independent MD replicas).

Each replica in a mixed batch -- admitted at different steps, NVE and Nose-Hoover NVT side by
side, one of them a 63-atom water box thinner than twice the cutoff plus skin (multi-image
neighbour search) -- is compared element by element with the oracle's own velocity-Verlet
(orc_nve) or Nose-Hoover chain (orc_nvt) trajectory from the same initial state, and its final
virial with the oracle's virial at the replica's final positions.

Tolerances follow from the FP32 force and energy bars (relative force RMSE 1e-5, |dE|/N 1e-6 of
the RMS per-atom energy): with |F| ~ 1 eV/A and hydrogen masses, a 1e-5 relative force error
moves a velocity by < 1e-6 A/fs and a position by < 1e-5 A over 15 steps of 0.5 fs.  The served
potential energy must add nothing to the FP32 path's own static error: after subtracting the
offset of a direct (unserved) evaluation at the initial positions from the oracle, the served
energy along the trajectory is held to the energy bar.  The offset itself is held to the bar by the
direct-evaluation tests; here it is only bounded by 2e-6 of the RMS per-atom energy, because on
the fcc replica of this model the per-atom energy (0.030 eV) is what is left of readout terms of
RMS 0.26 eV, so FP32 rounding of those terms (about 5e-8 eV per atom) is 1.6e-6 of it.  The BF16 replicas (tensor-core path, F = 128) are held to the BF16 force bar through their displacements."""
import numpy as np
import pytest

import synthetic as syn
from gpu_common import (BF16_FORCE_RMSE, FP32_ENERGY_PER_ATOM, FP32_VIRIAL_REL, engine, model,
                        virial_rel)

pytestmark = pytest.mark.gpu

T, S, DT, NSTEPS = 2, 3, 0.5, 15


def _systems():
    small = syn.water_box(21, seed=2)            # 63 atoms, L = 8.6 A < 2 (rc + skin)
    f = syn.fcc(3, 3, 3, jitter=0.05, seed=1)    # 108 atoms
    f.species[:] = 2
    w = syn.water_box(64, seed=0)                # 192 atoms
    out = []
    for k, sy in enumerate((small, f, w)):
        out.append((sy, syn.maxwell_boltzmann(sy.masses, 300.0, seed=20 + k)))
    return out


def _serve(eng, blob, F, items, thermos, precision, late):
    """items[k] submitted at step late[k]; thermos[k] = (T, tau, M) or None."""
    srv = eng.Server(F, blob, T=T, n_species=S, precision=precision, dt=DT)
    ids = [None] * len(items)
    for step in range(NSTEPS + max(late) + 10):
        for k, (sy, v) in enumerate(items):
            if late[k] == step:
                ids[k] = srv.submit(sy.species, sy.masses, sy.positions, v, sy.cell, NSTEPS, skin=1.0)
                if thermos[k] is not None:
                    srv.set_thermostat(ids[k], *thermos[k])
        srv.step()
        if all(i is not None and srv.poll(i)["state"] == 2 for i in ids):
            break
    out = []
    for k, i in enumerate(ids):
        r = srv.poll(i)
        assert r["state"] == 2 and r["steps_done"] == NSTEPS
        if thermos[k] is not None:
            r.update(srv.thermostat(i))
        out.append(r)
    srv.close()
    return out


def test_served_fp32_replicas_follow_the_oracle(orc):
    eng = engine()
    F = 64
    vals, blob = model(F, T, S, seed=31, bias=0.1)
    items = _systems()
    nvt = (500.0, 25.0, 3)
    thermos = [None, nvt, None]
    res = _serve(eng, blob, F, items, thermos, "fp32", late=[0, 2, 5])
    for (sy, v0), th, r in zip(items, thermos, res):
        if th is None:
            xo, vo, epo, eko = orc.nve(vals, F, 20, T, S, sy.species, sy.masses, sy.positions, v0, sy.cell,
                                       DT, NSTEPS)
        else:
            xo, vo, epo, eko, etho, xio, vxio = orc.nvt(vals, F, 20, T, S, sy.species, sy.masses, sy.positions,
                                                        v0, sy.cell, DT, NSTEPS, th[0], th[1], chain=th[2])
            np.testing.assert_allclose(r["ethermo"], etho, rtol=0, atol=1e-6 * sy.n)
            np.testing.assert_allclose(r["xi"], xio, rtol=1e-5, atol=1e-9)
            np.testing.assert_allclose(r["vxi"], vxio, rtol=1e-5, atol=1e-9)
        ref0 = orc.painn(vals, F, 20, T, S, sy.species, sy.positions, sy.cell)
        escale = float(np.sqrt(np.mean(ref0["energies"] ** 2)))
        np.testing.assert_allclose(r["positions"], xo, rtol=0, atol=2e-5)
        np.testing.assert_allclose(r["velocities"], vo, rtol=0, atol=5e-6)
        with eng.Potential(F, K=20, T=T, n_species=S, precision="fp32", params=blob) as pot:
            e_direct = pot.compute(sy.species, sy.positions, sy.cell, forces=False, virial=False)["energy"]
        bar = FP32_ENERGY_PER_ATOM * escale * sy.n
        offset = e_direct - epo[0]
        assert abs(offset) <= 2 * bar, (offset, bar)
        np.testing.assert_allclose(r["epot"] - offset, epo, rtol=0, atol=bar)
        np.testing.assert_allclose(r["ekin"], eko, rtol=1e-5, atol=1e-9)
        # the virial of the last force evaluation, at the replica's final positions
        refw = orc.painn(vals, F, 20, T, S, sy.species, r["positions"], sy.cell)["virial"]
        assert virial_rel(r["virial"], refw) <= FP32_VIRIAL_REL


def test_served_bf16_tensor_core_replicas_follow_the_oracle(orc):
    eng = engine()
    F = 128
    vals = syn.xavier_params(F, 20, T, S, seed=32, bias_scale=0.1)
    blob = syn.params_blob(F, 20, T, S, values=vals)
    items = _systems()
    res = _serve(eng, blob, F, items, [None] * 3, "bf16", late=[0, 1, 3])
    for (sy, v0), r in zip(items, res):
        xo, vo, epo, eko = orc.nve(vals, F, 20, T, S, sy.species, sy.masses, sy.positions, v0, sy.cell,
                                   DT, NSTEPS)
        ref0 = orc.painn(vals, F, 20, T, S, sy.species, sy.positions, sy.cell)
        escale = float(np.sqrt(np.mean(ref0["energies"] ** 2)))
        assert abs(r["epot"][0] - epo[0]) / sy.n <= 1e-2 * escale
        # displacements over the run, against the oracle's, at the BF16 force bar
        d, do = r["positions"] - sy.positions, xo - sy.positions
        rel = float(np.sqrt(((d - do) ** 2).sum() / (do ** 2).sum()))
        assert rel <= 3 * BF16_FORCE_RMSE, rel
        refw = orc.painn(vals, F, 20, T, S, sy.species, r["positions"], sy.cell)["virial"]
        assert virial_rel(r["virial"], refw) <= 2e-2
