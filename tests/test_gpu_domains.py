"""Spatial domain decomposition on one GPU (ctd_domains_*), against the FP64 oracle.

arXiv 2506.04055, Results "Distributed potential computation": the sum of the owned atoms'
energies over all domains is the total energy, and the summed partial forces of an atom's
copies are its force; pruning copies beyond T hops changes nothing.  Each case compares the
decomposed GPU result with the oracle's periodic result at the FP32 (or BF16) tolerances and
with the library's own single-system result, and checks the per-domain counts against the
halo rule evaluated here in FP64 with the library's expression order.
"""
import itertools

import numpy as np
import pytest

import synthetic as syn
from gpu_common import BF16_FORCE_RMSE, compare, engine, model

pytestmark = pytest.mark.gpu

RC = 5.0


def expected_counts(orc, x, H, grid, rcomm):
    """Owned atoms and halo copies per domain (before hop pruning), in the order of
    ctd_domains_info: the owner is the domain whose box holds f = s - floor(s) with
    s = (G0 x0 + G1 x1) + G2 x2, and a copy is every image f + n with
    q/p - h <= f + n < (q+1)/p + h per direction, h = rcomm |G_a|."""
    G = orc.inv_transpose(H)
    s = (G[None, :, 0] * x[:, None, 0] + G[None, :, 1] * x[:, None, 1]) + G[None, :, 2] * x[:, None, 2]
    f = s - np.floor(s)
    p = np.asarray(grid)
    owner = np.minimum(np.floor(f * p).astype(int), p - 1)
    gn = np.sqrt((G[:, 0] * G[:, 0] + G[:, 1] * G[:, 1]) + G[:, 2] * G[:, 2])
    h = rcomm * gn
    m = np.ceil(h).astype(int) + 1
    owned, cands = [], []
    for q in itertools.product(*(range(g) for g in grid)):
        per_axis = []
        for a in range(3):
            lo = q[a] / grid[a] - h[a]
            hi = (q[a] + 1) / grid[a] + h[a]
            cnt = np.zeros(len(x), int)
            for k in range(-m[a], m[a] + 1):
                u = f[:, a] + float(k)
                cnt += (u >= lo) & (u < hi)
            per_axis.append(cnt)
        total = int((per_axis[0] * per_axis[1] * per_axis[2]).sum())
        own = int(np.all(owner == np.asarray(q), axis=1).sum())
        owned.append(own)
        cands.append(total - own)
    return owned, cands


def single(eng, blob, sy, F, T, S, precision="fp32"):
    with eng.Potential(F, T=T, n_species=S, precision=precision, params=blob) as pot:
        return pot.compute(sy.species, sy.positions, sy.cell, energies=True)


def decomposed(eng, blob, sy, F, T, S, grid, hop=True, precision="fp32", skin=1.0, **kw):
    with eng.Domains(F, blob, grid=grid, T=T, n_species=S, precision=precision, hop_prune=hop, skin=skin) as dom:
        out = dom.compute(sy.species, sy.positions, sy.cell, energies=True, stats=True, **kw)
        out["info"] = dom.info()
        return out


@pytest.mark.parametrize("grid", [(1, 1, 1), (2, 1, 1), (2, 2, 2), (3, 1, 2)])
def test_fcc_matches_oracle_and_single_system(orc, grid):
    eng = engine()
    F, T, S = 32, 2, 1
    sy = syn.fcc(5, 5, 5, seed=3)
    vals, blob = model(F, T, S, seed=11, bias=0.2)
    ref = orc.painn(vals, F, 20, T, S, sy.species, sy.positions, sy.cell)
    one = single(eng, blob, sy, F, T, S)
    out = decomposed(eng, blob, sy, F, T, S, grid)
    compare(out, ref)
    compare(one, ref)
    # the decomposition sums the same per-atom terms in another order: FP32 rounding apart
    assert abs(out["energy"] - one["energy"]) <= 1e-6 * np.abs(one["energies"]).sum()
    np.testing.assert_allclose(out["forces"], one["forces"], rtol=0, atol=2e-5 * np.abs(one["forces"]).max())
    np.testing.assert_allclose(out["energies"], one["energies"], rtol=0, atol=1e-5 * np.abs(one["energies"]).max())
    owned, cands = expected_counts(orc, sy.positions, sy.cell, grid, T * RC + 1.0)
    info = out["info"]
    assert [d["n_owned"] for d in info] == owned
    assert [d["n_candidates"] for d in info] == cands
    assert sum(owned) == len(sy.species)
    assert all(d["n_copies"] <= d["n_candidates"] for d in info)
    assert out["stats"]["n_atoms"] == sum(d["n_owned"] + d["n_copies"] for d in info)


def test_hop_pruning_changes_nothing_but_the_work():
    eng = engine()
    F, T, S = 32, 3, 1
    sy = syn.fcc(6, 6, 6, seed=4)
    _, blob = model(F, T, S, seed=12, bias=0.2)
    a = decomposed(eng, blob, sy, F, T, S, (2, 2, 1), hop=False)
    b = decomposed(eng, blob, sy, F, T, S, (2, 2, 1), hop=True)
    assert sum(d["n_copies"] for d in b["info"]) < sum(d["n_copies"] for d in a["info"])
    assert sum(d["n_active_edges"] for d in b["info"]) < sum(d["n_active_edges"] for d in a["info"])
    assert [d["n_owned"] for d in a["info"]] == [d["n_owned"] for d in b["info"]]
    assert abs(a["energy"] - b["energy"]) <= 1e-6 * np.abs(a["energies"]).sum()
    np.testing.assert_allclose(b["forces"], a["forces"], rtol=0, atol=2e-5 * np.abs(a["forces"]).max())
    np.testing.assert_allclose(b["virial"], a["virial"], rtol=0, atol=2e-5 * np.abs(a["virial"]).max())


def test_triclinic_mixture_four_species(orc):
    eng = engine()
    F, T, S = 32, 2, 4
    sy = syn.mixture(n_chain=30, n_water=150, seed=5)
    vals, blob = model(F, T, S, seed=13, bias=0.2)
    ref = orc.painn(vals, F, 20, T, S, sy.species, sy.positions, sy.cell)
    out = decomposed(eng, blob, sy, F, T, S, (2, 1, 2))
    compare(out, ref)
    owned, cands = expected_counts(orc, sy.positions, sy.cell, (2, 1, 2), T * RC + 1.0)
    assert [d["n_owned"] for d in out["info"]] == owned
    assert [d["n_candidates"] for d in out["info"]] == cands


def test_unwrapped_positions_and_reuse_until_skin(orc):
    """Positions outside the cell (several images away) give the same result; the
    decomposition is reused while displacements stay below skin/2 and rebuilt after."""
    eng = engine()
    F, T, S = 32, 2, 2
    sy = syn.water_box(100, seed=6)
    vals, blob = model(F, T, S, seed=14, bias=0.2)
    rng = np.random.default_rng(0)
    shifts = rng.integers(-2, 3, size=(len(sy.species), 3)).astype(float)
    x_unwrapped = sy.positions + shifts @ sy.cell
    with eng.Domains(F, blob, grid=(2, 2, 1), T=T, n_species=S, skin=1.0) as dom:
        o1 = dom.compute(sy.species, x_unwrapped, sy.cell, stats=True)
        assert o1["stats"]["rebuilt"] == 1
        compare(o1, orc.painn(vals, F, 20, T, S, sy.species, sy.positions, sy.cell))
        x2 = x_unwrapped + rng.normal(0, 0.1, x_unwrapped.shape).clip(-0.28, 0.28)
        o2 = dom.compute(sy.species, x2, sy.cell, stats=True)
        assert o2["stats"]["rebuilt"] == 0
        compare(o2, orc.painn(vals, F, 20, T, S, sy.species, x2, sy.cell))
        x3 = x2.copy()
        x3[7] += np.array([0.8, 0.0, 0.0])
        o3 = dom.compute(sy.species, x3, sy.cell, stats=True)
        assert o3["stats"]["rebuilt"] == 1
        compare(o3, orc.painn(vals, F, 20, T, S, sy.species, x3, sy.cell))


def test_device_pointers_match_host():
    import torch
    eng = engine()
    F, T, S = 32, 2, 1
    sy = syn.fcc(4, 4, 4, seed=7)
    _, blob = model(F, T, S, seed=15, bias=0.2)
    with eng.Domains(F, blob, grid=(2, 1, 1), T=T, n_species=S) as dom:
        h = dom.compute(sy.species, sy.positions, sy.cell)
        d = dom.compute(torch.tensor(sy.species, device="cuda"), torch.tensor(sy.positions, device="cuda"),
                        sy.cell)
        assert float(d["energy"].cpu()[0]) == h["energy"]
        np.testing.assert_array_equal(d["forces"].cpu().numpy(), h["forces"])
        np.testing.assert_array_equal(d["virial"].cpu().numpy(), h["virial"])


def test_bf16_tensor_core_path(orc):
    """F = 128: the tensor-core message and adjoint kernels run over the batched domains."""
    eng = engine()
    F, T, S = 128, 3, 1
    sy = syn.fcc(6, 6, 6, seed=8)
    vals, blob = model(F, T, S, seed=16, bias=0.1)
    ref = orc.painn(vals, F, 20, T, S, sy.species, sy.positions, sy.cell)
    out = decomposed(eng, blob, sy, F, T, S, (2, 2, 1), precision="bf16")
    compare(out, ref, force_tol=BF16_FORCE_RMSE, e_tol=1e-2, w_tol=2e-2)


def test_empty_system():
    eng = engine()
    _, blob = model(32, 2, 1, seed=0)
    with eng.Domains(32, blob, grid=(2, 1, 1), T=2, n_species=1) as dom:
        out = dom.compute(np.zeros(0, np.int32), np.zeros((0, 3)), np.eye(3) * 20.0)
        assert out["energy"] == 0.0
        assert out["forces"].shape == (0, 3)
        assert np.all(out["virial"] == 0.0)


def test_slab_with_empty_domains(orc):
    """An fcc slab in a box four times its thickness (vacuum along x), 8 domains along x: the
    domains in the vacuum hold neither owned atoms nor copies, and the result still matches."""
    eng = engine()
    F, T, S = 32, 2, 1
    sy = syn.fcc(4, 4, 4, seed=9)
    cell = sy.cell.copy()
    cell[0, 0] *= 4.0
    sy = syn.System(sy.positions, sy.species, sy.masses, cell, "slab")
    vals, blob = model(F, T, S, seed=17, bias=0.2)
    ref = orc.painn(vals, F, 20, T, S, sy.species, sy.positions, sy.cell)
    out = decomposed(eng, blob, sy, F, T, S, (8, 1, 1))
    compare(out, ref)
    empty = [d for d in out["info"] if d["n_owned"] == 0 and d["n_copies"] == 0]
    assert len(empty) >= 2
    assert sum(d["n_owned"] for d in out["info"]) == len(sy.species)
