"""Stored versus recomputed edge filters in the adjoint (CTD_OPT_EDGE_STORE).

The adjoint needs, per edge, the cutoff-scaled radial filter and its distance derivative.  By
default it recomputes them from the basis; with the option on, the forward message kernel
stores them and the adjoint reads them back.  Both must agree with the FP64 oracle at the FP32
tolerances, the option must fall back to recomputation when the store does not fit the HBM
budget, and a fallback call must be bit-identical to a recompute call."""
import numpy as np
import pytest

import synthetic as syn
from gpu_common import BF16_FORCE_RMSE, compare, engine, model

pytestmark = pytest.mark.gpu


def _compute(eng, blob, sy, F, T, S, store, precision="fp32", budget=0):
    from paper_2506_04055_gb300 import _lib
    with eng.Potential(F, T=T, n_species=S, precision=precision, params=blob, hbm_budget_bytes=budget) as pot:
        pot.set_option(_lib.CTD_OPT_EDGE_STORE, 1 if store else 0)
        return pot.compute(sy.species, sy.positions, sy.cell, energies=True, stats=True)


def test_store_matches_oracle_and_recompute(orc):
    """4-species triclinic mixture (cut-down of the 90,300-atom system), F = 64, 2 layers."""
    eng = engine()
    sy = syn.mixture(n_chain=30, n_water=150, seed=1)
    vals, blob = model(64, 2, 4, seed=2, bias=0.2)
    ref = orc.painn(vals, 64, 20, 2, 4, sy.species, sy.positions, sy.cell)
    rec = _compute(eng, blob, sy, 64, 2, 4, store=False)
    sto = _compute(eng, blob, sy, 64, 2, 4, store=True)
    assert rec["stats"]["edges_stored"] == 0 and sto["stats"]["edges_stored"] == 1
    compare(sto, ref)
    compare(rec, ref)
    # the forward pass is the same arithmetic either way
    assert sto["energy"] == rec["energy"]
    np.testing.assert_allclose(sto["forces"], rec["forces"], rtol=0, atol=1e-5 * np.abs(rec["forces"]).max())


def test_store_several_row_chunks(orc):
    """Water with F = 32: receiver rows longer than F edges span several staging chunks."""
    eng = engine()
    sy = syn.water_box(200, seed=7)
    vals, blob = model(32, 3, 2, seed=8, bias=0.1)
    ref = orc.painn(vals, 32, 20, 3, 2, sy.species, sy.positions, sy.cell)
    sto = _compute(eng, blob, sy, 32, 3, 2, store=True)
    assert sto["stats"]["edges_stored"] == 1
    compare(sto, ref)


def test_store_falls_back_over_budget():
    """A budget that holds the model's buffers but not the edge store: recompute, bit-identical."""
    eng = engine()
    sy = syn.water_box(300, seed=3)
    F, T, S = 64, 2, 2
    _, blob = model(F, T, S, seed=4, bias=0.1)
    rec = _compute(eng, blob, sy, F, T, S, store=False)
    held = rec["stats"]["bytes_allocated"]
    store_bytes = T * rec["stats"]["n_verlet_edges"] * 6 * F * 4
    budget = held + store_bytes // 2
    fb = _compute(eng, blob, sy, F, T, S, store=True, budget=budget)
    assert fb["stats"]["edges_stored"] == 0
    assert fb["energy"] == rec["energy"]
    np.testing.assert_array_equal(fb["forces"], rec["forces"])
    np.testing.assert_array_equal(fb["virial"], rec["virial"])
    # with room for it the same call stores
    ok = _compute(eng, blob, sy, F, T, S, store=True, budget=held + 2 * store_bytes)
    assert ok["stats"]["edges_stored"] == 1


def test_store_bf16_F64(orc):
    """BF16 path with F = 64 (CUDA-core edge kernels): stored filters, oracle at BF16 tolerance."""
    eng = engine()
    sy = syn.water_box(64, seed=0)
    vals, blob = model(64, 3, 2, seed=0, bias=0.1)
    ref = orc.painn(vals, 64, 20, 3, 2, sy.species, sy.positions, sy.cell)
    sto = _compute(eng, blob, sy, 64, 3, 2, store=True, precision="bf16")
    rec = _compute(eng, blob, sy, 64, 3, 2, store=False, precision="bf16")
    assert sto["stats"]["edges_stored"] == 1
    compare(sto, ref, force_tol=BF16_FORCE_RMSE, e_tol=1e-2, w_tol=2e-2)
    np.testing.assert_allclose(sto["forces"], rec["forces"], rtol=0, atol=1e-5 * np.abs(rec["forces"]).max())
