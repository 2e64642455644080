"""GPU energy / forces / virial vs the FP64 oracle (FP32 path).

Tolerances (FP32 path): relative force RMSE <= 1e-5, |dE|/N <= 1e-6 of the RMS per-atom energy,
relative virial error <= 1e-5.  The oracle evaluates U = sum_i U_i and f = -dU/dx (arXiv
2506.04055, Methods energy-sum equation; Results sum-rule equation) with its own pair search.
"""
import numpy as np
import pytest

import synthetic as syn
from gpu_common import compare, engine, model, rel_force_rmse

pytestmark = pytest.mark.gpu


def _run(eng, orc, sy, F, T, S, bias=0.2, seed=0, precision="fp32", K=20, e_scale=1.0):
    vals, blob = model(F, T, S, seed=seed, bias=bias, K=K, e_scale=e_scale)
    with eng.Potential(F, K=K, T=T, n_species=S, precision=precision, params=blob) as pot:
        out = pot.compute(sy.species, sy.positions, sy.cell, energies=True)
    ref = orc.painn(vals, F, K, T, S, sy.species, sy.positions, sy.cell, e_scale=e_scale)
    return out, ref


def test_water192_F64_T3(orc):
    """192-atom water box (64 H2O, L = 12.42 A), F = 64, 3 layers, 20 Gaussians, rc = 5 A."""
    eng = engine()
    sy = syn.water_box(64, seed=0)
    out, ref = _run(eng, orc, sy, 64, 3, 2)
    compare(out, ref)
    np.testing.assert_allclose(out["energies"], ref["energies"], rtol=0,
                               atol=1e-5 * np.abs(ref["energies"]).max())


def test_water192_xavier_zero_bias(orc):
    """The benchmark's weights: Xavier-uniform from seed 0, zero biases."""
    eng = engine()
    sy = syn.water_box(64, seed=0)
    out, ref = _run(eng, orc, sy, 64, 3, 2, bias=0.0)
    compare(out, ref)


def test_water1500_several_tiles(orc):
    eng = engine()
    sy = syn.water_box(500, seed=3)
    out, ref = _run(eng, orc, sy, 64, 2, 2, seed=4)
    compare(out, ref)


def test_fcc_F128(orc):
    """fcc a = 4.05 A, 6x6x6 cells (864 atoms), F = 128, 3 layers."""
    eng = engine()
    sy = syn.fcc(6, 6, 6, jitter=0.05, seed=0)
    out, ref = _run(eng, orc, sy, 128, 3, 1, seed=1)
    compare(out, ref)


def test_triclinic_mixture_T2(orc):
    """4-species triclinic mixture (cut-down of the 90,300-atom system), F = 64, 2 layers."""
    eng = engine()
    sy = syn.mixture(n_chain=30, n_water=150, seed=1)
    out, ref = _run(eng, orc, sy, 64, 2, 4, seed=2)
    compare(out, ref)


def test_small_cells_multi_image(orc):
    """64-atom-class boxes thinner than 2 (rc + skin): forces through periodic self-images."""
    eng = engine()
    for sy in (syn.water_box(21, seed=2), syn.fcc(1, 1, 1, jitter=0.1, seed=3), syn.fcc(2, 2, 1, seed=4)):
        out, ref = _run(eng, orc, sy, 32, 2, 2, seed=5)
        compare(out, ref)


def test_other_widths_and_basis(orc):
    eng = engine()
    sy = syn.water_box(40, seed=6)
    for F, K in ((32, 8), (256, 20), (64, 32), (64, 7)):
        out, ref = _run(eng, orc, sy, F, 1, 2, K=K, seed=F + K)
        compare(out, ref)


def test_T0_and_single_atom(orc):
    eng = engine()
    sy = syn.water_box(8, seed=0)
    out, ref = _run(eng, orc, sy, 64, 0, 2)
    assert abs(out["energy"] - ref["energy"]) < 1e-5 * abs(ref["energy"])
    assert np.abs(out["forces"]).max() == 0.0
    one = syn.System(np.array([[0.3, 0.2, 0.1]]), np.zeros(1, np.int32), np.ones(1), np.eye(3) * 4.0)
    out, ref = _run(eng, orc, one, 32, 2, 1)
    assert out["energy"] == pytest.approx(ref["energy"], rel=1e-5)
    assert np.abs(out["forces"]).max() < 1e-5
    np.testing.assert_allclose(out["virial"], ref["virial"], atol=1e-5 * np.abs(ref["virial"]).max())


def test_empty_system():
    eng = engine()
    _, blob = model(32, 2, 1)
    with eng.Potential(32, T=2, n_species=1, params=blob) as pot:
        out = pot.compute(np.zeros(0, np.int32), np.zeros((0, 3)), np.eye(3) * 10.0)
    assert out["energy"] == 0.0 and out["forces"].shape == (0, 3)
    assert np.abs(out["virial"]).max() == 0.0


def test_deterministic_and_device_pointers():
    import torch
    eng = engine()
    sy = syn.water_box(200, seed=7)
    _, blob = model(64, 3, 2, bias=0.1)
    with eng.Potential(64, T=3, n_species=2, params=blob) as pot:
        a = pot.compute(sy.species, sy.positions, sy.cell)
        b = pot.compute(sy.species, sy.positions, sy.cell, rebuild=True)
        x = torch.tensor(sy.positions, device="cuda")
        z = torch.tensor(sy.species, device="cuda")
        c = pot.compute(z, x, sy.cell)
        torch.cuda.synchronize()
    assert a["energy"] == b["energy"]
    np.testing.assert_array_equal(a["forces"], b["forces"])
    np.testing.assert_array_equal(a["virial"], b["virial"])
    assert float(c["energy"][0]) == a["energy"]
    np.testing.assert_array_equal(c["forces"].cpu().numpy(), a["forces"])


def test_skin_reuse_and_rebuild(orc):
    """Within skin/2 the Verlet list is reused (no rebuild) and results track the oracle at the
    new positions; beyond it the list is rebuilt."""
    eng = engine()
    sy = syn.water_box(100, seed=8)
    vals, blob = model(64, 2, 2, seed=9, bias=0.1)
    rng = np.random.default_rng(0)
    with eng.Potential(64, T=2, n_species=2, params=blob) as pot:
        pot.build_neighbors(sy.positions, sy.cell, skin=1.0)
        x1 = sy.positions + rng.uniform(-0.25, 0.25, size=sy.positions.shape)
        o1 = pot.compute(sy.species, x1, sy.cell, stats=True)
        assert o1["stats"]["rebuilt"] == 0
        r1 = orc.painn(vals, 64, 20, 2, 2, sy.species, x1, sy.cell)
        compare(o1, r1)
        x2 = sy.positions + rng.uniform(-0.7, 0.7, size=sy.positions.shape)
        o2 = pot.compute(sy.species, x2, sy.cell, stats=True)
        assert o2["stats"]["rebuilt"] == 1
        compare(o2, orc.painn(vals, 64, 20, 2, 2, sy.species, x2, sy.cell))


def test_force_sum_and_virial_symmetry_at_1M():
    """Properties that hold at any size, at the 1,000,188-atom fcc workload (F = 128, T = 3):
    sum of forces ~ 0 and a symmetric virial."""
    eng = engine()
    sy = syn.fcc(63, 63, 63, jitter=0.05, seed=0)
    _, blob = model(128, 3, 1, seed=0)
    with eng.Potential(128, T=3, n_species=1, params=blob) as pot:
        out = pot.compute(sy.species, sy.positions, sy.cell)
    f = out["forces"]
    assert np.isfinite(f).all()
    assert np.abs(f.sum(0)).max() < 1e-5 * np.abs(f).sum(0).max()
    W = out["virial"]
    assert np.abs(W - W.T).max() < 1e-5 * np.abs(W).max()


def test_fcc_4000_subcell_force_rmse(orc):
    """The 10x10x10-cell (4,000-atom) fcc sub-run of the 1M-atom configuration vs the oracle."""
    eng = engine()
    sy = syn.fcc(10, 10, 10, jitter=0.05, seed=0)
    out, ref = _run(eng, orc, sy, 128, 3, 1, bias=0.0, seed=0)
    compare(out, ref)


def test_autograd_function_matches_forces_and_differences():
    import torch
    eng = engine()
    sy = syn.water_box(30, seed=11)
    _, blob = model(64, 2, 2, seed=12, bias=0.1)
    with eng.Potential(64, T=2, n_species=2, params=blob) as pot:
        x = torch.tensor(sy.positions, device="cuda", requires_grad=True)
        z = torch.tensor(sy.species, device="cuda")
        E, W = eng.PaiNNEnergy.apply(x, z, sy.cell, pot)
        E.backward()
        ref = pot.compute(sy.species, sy.positions, sy.cell)
        np.testing.assert_allclose(x.grad.cpu().numpy(), -ref["forces"], rtol=0, atol=1e-12)
        # directional central difference in FP64 positions (FP32 arithmetic inside)
        d = torch.randn_like(x)
        d /= d.norm()
        h = 1e-2
        with torch.no_grad():
            ep = pot.compute(sy.species, (x + h * d).cpu().numpy(), sy.cell, forces=False, virial=False)["energy"]
            em = pot.compute(sy.species, (x - h * d).cpu().numpy(), sy.cell, forces=False, virial=False)["energy"]
        fd = (ep - em) / (2 * h)
        an = float((x.grad * d).sum())
        assert fd == pytest.approx(an, rel=2e-3, abs=2e-4)


def test_bounded_wait_gives_up_and_context_stays_usable():
    """Failure detection without a fault: a device wait on an mbarrier that nothing arrives on
    gives up after its limit, frees its tensor memory and reports CTD_ERR_TIMEOUT; the same
    context then computes exactly what it computed before."""
    from paper_2506_04055_gb300 import _lib
    eng = engine()
    sy = syn.fcc(4, 4, 4, seed=1)
    _, blob = model(128, 2, 1, seed=1)
    with eng.Potential(128, T=2, n_species=1, precision="bf16", params=blob) as pot:
        before = pot.compute(sy.species, sy.positions, sy.cell)
        code, waited = _lib.ctd_selftest_wait(pot.ctx, 50.0)
        assert code == _lib.CTD_ERR_TIMEOUT
        assert "wait gave up" in _lib.ctd_last_error(pot.ctx)
        assert 50.0 <= waited < 1000.0
        code, _ = _lib.ctd_selftest_wait(pot.ctx, 5.0)      # repeatable
        assert code == _lib.CTD_ERR_TIMEOUT
        after = pot.compute(sy.species, sy.positions, sy.cell)
        assert after["energy"] == before["energy"]
        np.testing.assert_array_equal(after["forces"], before["forces"])
        assert _lib.ctd_selftest_wait(pot.ctx, 0.0)[0] == _lib.CTD_ERR_INVALID_ARG
