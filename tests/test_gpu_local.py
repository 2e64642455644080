"""Strictly local equivariant edge model (CTD_FAMILY_LOCAL) on the GPU against the FP64 oracle.

Methods, "(Semi-)Local Potential Models" and "Chosen Architectures": the Allegro-type model
passes messages only between edges leaving the same atom.  Parity with oracle/local.py at the
FP32 tolerances (force RMSE 1e-5 relative, |dE|/N 1e-6 of the per-atom energy scale) on water,
a crystal and a triclinic four-species mixture; per-atom energies; strict locality holds bit
for bit; the resident MD loop follows the oracle's velocity-Verlet trajectory; served replicas
are bit-identical alone and mixed; the spatial decomposition with one-hop copies; degenerate
systems and invalid descriptions."""
import numpy as np
import pytest

import synthetic as syn
from gpu_common import compare, engine

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::UserWarning")]

K = 20


@pytest.fixture(scope="module")
def loc():
    import oracle.local as ol
    return ol


def _model(F, L, S, C, seed, bias=0.2, e_scale=1.0):
    vals = syn.local_xavier_params(F, K, L, S, C, seed=seed, bias_scale=bias)
    return vals, syn.local_params_blob(F, K, L, S, C, e_scale=e_scale, values=vals)


def _pot(eng, F, L, S, C, blob):
    return eng.Potential(F, K=K, T=L, n_species=S, params=blob, family="local", channels=C)


CASES = {
    "water192": (lambda: syn.water_box(64, seed=0), 64, 2, 2, 16),
    "fcc256": (lambda: syn.fcc(4, 4, 4, seed=1), 32, 3, 1, 8),
    "mixture": (lambda: syn.mixture(n_chain=30, n_water=150, seed=2), 16, 1, 4, 4),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_matches_oracle(loc, case):
    make, F, L, S, C = CASES[case]
    sy = make()
    eng = engine()
    vals, blob = _model(F, L, S, C, seed=len(case))
    ref = loc.local_model(vals, F, K, L, S, C, sy.species, sy.positions, sy.cell)
    with _pot(eng, F, L, S, C, blob) as pot:
        out = pot.compute(sy.species, sy.positions, sy.cell, energies=True, stats=True)
    compare(out, ref)
    scale = float(np.sqrt(np.mean(ref["energies"] ** 2)))
    np.testing.assert_allclose(out["energies"], ref["energies"], rtol=0, atol=2e-5 * scale)
    assert out["stats"]["n_active_edges"] == ref["n_edges"]


def test_energy_scale_and_tiny_cell(loc):
    """e_scale in the blob, and a cell thinner than twice the cutoff (many images per pair)."""
    F, L, S, C = 16, 2, 2, 4
    sy = syn.water_box(8, seed=3)          # L ~ 6.2 A < 2 rc
    eng = engine()
    vals, blob = _model(F, L, S, C, seed=4, e_scale=0.37)
    ref = loc.local_model(vals, F, K, L, S, C, sy.species, sy.positions, sy.cell, e_scale=0.37)
    with _pot(eng, F, L, S, C, blob) as pot:
        out = pot.compute(sy.species, sy.positions, sy.cell, energies=True)
    compare(out, ref)


def test_strict_locality_bit_for_bit():
    """A - B - C on a line (|AB| = |BC| = 3 A, |AC| = 6 A > rc), three layers: moving C leaves
    A's energy unchanged bit for bit (nothing beyond A's cutoff sphere enters its arithmetic)."""
    F, L, S, C = 16, 3, 2, 4
    eng = engine()
    _, blob = _model(F, L, S, C, seed=5)
    base = np.array([[5.0, 10.0, 10.0], [8.0, 10.0, 10.0], [11.0, 10.0, 10.0]])
    moved = base.copy()
    moved[2] += [0.2, 0.3, -0.1]
    z = np.array([0, 1, 0], np.int32)
    with _pot(eng, F, L, S, C, blob) as pot:
        a = pot.compute(z, base, np.eye(3) * 40.0, energies=True)
        b = pot.compute(z, moved, np.eye(3) * 40.0, energies=True)
    assert a["energies"][0] == b["energies"][0]
    assert a["energies"][1] != b["energies"][1]


def test_md_follows_oracle_trajectory(loc):
    """20 velocity-Verlet steps of 0.5 fs (water, 192 atoms): positions, velocities and energies
    follow the same integrator driven by the oracle's FP64 forces."""
    F, L, S, C = 32, 2, 2, 8
    sy = syn.water_box(64, seed=6)
    eng = engine()
    vals, blob = _model(F, L, S, C, seed=6, bias=0.0)   # forces below 1 eV/A: a gentle trajectory
    v0 = syn.maxwell_boltzmann(sy.masses, 300.0, seed=6)
    dt, nsteps = 0.5, 20
    acc = 9.648533212331002e-3   # (eV / A) / amu in A / fs^2
    x, v = sy.positions.copy(), v0.copy()
    f = loc.local_model(vals, F, K, L, S, C, sy.species, x, sy.cell)["forces"]
    ep_ref = [loc.local_model(vals, F, K, L, S, C, sy.species, x, sy.cell, need_grad=False)["energy"]]
    for _ in range(nsteps):
        v = v + 0.5 * dt * acc * f / sy.masses[:, None]
        x = x + dt * v
        o = loc.local_model(vals, F, K, L, S, C, sy.species, x, sy.cell)
        f = o["forces"]
        v = v + 0.5 * dt * acc * f / sy.masses[:, None]
        ep_ref.append(o["energy"])
    with _pot(eng, F, L, S, C, blob) as pot:
        pot.md_set_state(sy.species, sy.masses, sy.positions, v0, sy.cell, skin=1.0)
        ep, ek, _ = pot.md_run(nsteps, dt)
        xg, vg = pot.md_get_state()
    assert np.abs(xg - x).max() < 1e-5
    assert np.abs(vg - v).max() < 1e-6
    scale = np.abs(np.asarray(ep_ref)).max() / len(sy.species)
    np.testing.assert_allclose(ep, ep_ref, rtol=0, atol=1e-5 * scale * len(sy.species))


def test_served_replicas_alone_equal_mixed():
    F, L, S, C = 32, 2, 2, 8
    eng = engine()
    _, blob = _model(F, L, S, C, seed=7)
    items = []
    for k, sy in enumerate((syn.water_box(40, seed=7), syn.water_box(21, seed=8), syn.water_box(30, seed=9))):
        items.append((sy, syn.maxwell_boltzmann(sy.masses, 300.0, seed=20 + k)))

    def run(subset):
        srv = eng.Server(F, blob, K=K, T=L, n_species=S, dt=0.5, family="local", channels=C)
        ids = [srv.submit(sy.species, sy.masses, sy.positions, v, sy.cell, 8, skin=1.0) for sy, v in subset]
        for _ in range(40):
            srv.step()
            if all(srv.poll(i)["state"] == 2 for i in ids):
                break
        out = srv.poll(ids[0])
        srv.close()
        return out

    alone = run(items[:1])
    mixed = run(items)
    assert alone["state"] == 2 and mixed["state"] == 2
    np.testing.assert_array_equal(alone["epot"], mixed["epot"])
    np.testing.assert_array_equal(alone["positions"], mixed["positions"])
    np.testing.assert_array_equal(alone["velocities"], mixed["velocities"])


def test_degenerate_systems():
    F, L, S, C = 16, 2, 2, 4
    eng = engine()
    _, blob = _model(F, L, S, C, seed=8)
    with _pot(eng, F, L, S, C, blob) as pot:
        out = pot.compute(np.zeros(0, np.int32), np.zeros((0, 3)), np.eye(3) * 20.0)
        assert out["energy"] == 0.0 and out["forces"].shape == (0, 3)
        # isolated atoms: no edges, zero energy, forces and virial
        x = np.array([[1.0, 1.0, 1.0], [12.0, 12.0, 12.0]])
        out = pot.compute(np.array([0, 1], np.int32), x, np.eye(3) * 24.0, energies=True)
        assert out["energy"] == 0.0
        assert np.all(out["forces"] == 0.0) and np.all(out["virial"] == 0.0)


def test_invalid_descriptions_rejected():
    eng = engine()
    _, blob = _model(16, 2, 2, 4, seed=9)
    for kw in ({"channels": 6}, {"channels": 0}, {"precision": "bf16", "channels": 4}):
        F = 16
        with pytest.raises(eng.CtdError):
            eng.Potential(F, K=K, T=2, n_species=2, family="local", **kw)
    with pytest.raises(eng.CtdError):
        eng.Potential(12, K=K, T=2, n_species=2, family="local", channels=4)
    # a PaiNN blob does not load into a local context, nor the other way round
    painn = syn.params_blob(32, K, 2, 2)
    with pytest.raises(eng.CtdError):
        eng.Potential(32, K=K, T=2, n_species=2, family="local", channels=4, params=painn)
    _, blob32 = _model(32, 2, 2, 4, seed=9)
    with pytest.raises(eng.CtdError):
        eng.Potential(32, K=K, T=2, n_species=2, params=blob32)


@pytest.mark.parametrize("grid", [(2, 1, 1), (2, 2, 1)])
def test_spatial_decomposition_one_hop(loc, orc, grid):
    """The decomposition of a strictly local model: copies within rc + skin of each domain (one
    hop, whatever the layer count), owned energies summed over domains, copy forces summed onto
    their atoms: the oracle's periodic result at the FP32 tolerances."""
    from test_gpu_domains import expected_counts
    F, L, S, C = 16, 3, 1, 4
    sy = syn.fcc(5, 5, 5, seed=10)
    eng = engine()
    vals, blob = _model(F, L, S, C, seed=10)
    ref = loc.local_model(vals, F, K, L, S, C, sy.species, sy.positions, sy.cell)
    with eng.Domains(F, blob, grid=grid, K=K, T=L, n_species=S, family="local", channels=C, skin=1.0) as dom:
        out = dom.compute(sy.species, sy.positions, sy.cell, energies=True)
        info = dom.info()
    compare(out, ref)
    owned, cands = expected_counts(orc, sy.positions, sy.cell, grid, 5.0 + 1.0)
    assert [d["n_owned"] for d in info] == owned
    assert [d["n_candidates"] for d in info] == cands


@pytest.mark.parametrize("case", ["water192_F64", "fcc256_F128"])
def test_bf16_tensor_core_path_matches_oracle(loc, case):
    """BF16 path: the dense edge GEMMs (two-body MLP, latent update, channel projections, readout
    and their adjoints) on the tcgen05 GEMM with BF16 operands and FP32 accumulation, the rest
    FP32.  Against the FP64 oracle at the BF16 force bar (relative force RMSE <= 1e-2)."""
    from gpu_common import rel_force_rmse, virial_rel
    if case == "water192_F64":
        sy, F, L, S, C = syn.water_box(64, seed=0), 64, 2, 2, 16
    else:
        sy, F, L, S, C = syn.fcc(4, 4, 4, jitter=0.05, seed=1), 128, 2, 1, 32
    eng = engine()
    vals, blob = _model(F, L, S, C, seed=11, bias=0.1)
    ref = loc.local_model(vals, F, K, L, S, C, sy.species, sy.positions, sy.cell)
    with eng.Potential(F, K=K, T=L, n_species=S, params=blob, family="local", channels=C, precision="bf16") as pot:
        out = pot.compute(sy.species, sy.positions, sy.cell, energies=True)
    fr = rel_force_rmse(out["forces"], ref["forces"])
    scale = float(np.sqrt(np.mean(ref["energies"] ** 2)))
    er = abs(out["energy"] - ref["energy"]) / sy.n / scale
    wr = virial_rel(out["virial"], ref["virial"])
    print(f"local bf16 {case}: force rmse {fr:.2e}, energy {er:.2e}, virial {wr:.2e}")
    assert fr <= 1e-2 and er <= 1e-2 and wr <= 2e-2, (fr, er, wr)


def test_bf16_rejects_channel_counts_off_the_tensor_core_tiles():
    eng = engine()
    with pytest.raises(eng.CtdError):
        eng.Potential(64, K=K, T=2, n_species=2, family="local", channels=8, precision="bf16")
