"""Pins for the oracle's per-atom energy weights and the spatial-decomposition sum rule (CPU).

What the paper fixes (arXiv 2506.04055, Results "Distributed potential computation"): the energy
is a sum of per-atom energies U_i that depend only on atoms within T hops of i (T message-passing
steps, hop length at most R), so a domain that holds its owned atoms plus copies of every atom
within T*R of its boundary computes each owned U_i exactly; the total energy is the sum of the
owned U_i over all domains, and the total force on an atom is the sum of the partial forces on
its copies (sum-rule equation).  The copied atoms that are not within T hops of an owned atom
can be dropped (the pseudo-message pruning) without changing anything.

The decomposition here is built independently of the library, with numpy: for each domain of a
p0 x p1 x p2 grid over the fractional coordinates, every periodic image of every atom inside the
domain's box widened by the halo becomes an atom of an open (non-periodic) subsystem; owned
atoms get weight 1, copies weight 0.  The oracle's weighted energy of each subsystem must add up
to the periodic oracle's energy, and the copies' forces must add up to its forces.
"""
import itertools

import numpy as np
import pytest

import synthetic as syn

RC = 5.0


def decompose(x, H, grid, halo):
    """Subsystems of a spatial decomposition: list of (positions, global index, weight, cell)."""
    G = np.linalg.inv(H).T
    s = x @ G.T
    f = s - np.floor(s)
    xw = f @ H
    owner = np.minimum((f * np.asarray(grid)).astype(int), np.asarray(grid) - 1)
    h = halo * np.linalg.norm(G, axis=1)            # halo in fractional units per axis
    m = np.ceil(h).astype(int) + 1
    subs = []
    for q in itertools.product(*(range(p) for p in grid)):
        lo = np.array([q[a] / grid[a] - h[a] for a in range(3)])
        hi = np.array([(q[a] + 1) / grid[a] + h[a] for a in range(3)])
        pos, src, w = [], [], []
        for n in itertools.product(*(range(-m[a], m[a] + 1) for a in range(3))):
            u = f + np.asarray(n, float)
            inside = np.all((u >= lo) & (u < hi), axis=1)
            for i in np.nonzero(inside)[0]:
                pos.append(xw[i] + np.asarray(n, float) @ H)
                src.append(i)
                w.append(1.0 if (tuple(owner[i]) == q and n == (0, 0, 0)) else 0.0)
        pos = np.array(pos)
        # open subsystem: a box wider than the copies' extent by more than the cutoff
        lo_x = pos.min(axis=0) - RC - 1.0
        ext = pos.max(axis=0) - pos.min(axis=0) + 2 * RC + 2.0
        subs.append((pos - lo_x, np.array(src), np.array(w), np.diag(ext)))
    return subs


def hop_levels(n, pairs, seeds, T):
    """Hop distance (capped at T + 1) from the seed atoms over the given directed pairs."""
    lev = np.full(n, T + 1)
    lev[seeds] = 0
    i, j = pairs[0], pairs[1]
    for t in range(1, T + 1):
        reached = lev[j] == t - 1
        cand = np.zeros(n, bool)
        cand[i[reached]] = True
        lev[cand & (lev > t)] = t
    return lev


def run_decomposed(orc, vals, F, K, T, S, sy, grid, halo, prune_hops=False):
    n = len(sy.species)
    E, Fo, W = 0.0, np.zeros((n, 3)), np.zeros((3, 3))
    counts = []
    for pos, src, w, cell in decompose(sy.positions, sy.cell, grid, halo):
        Z = sy.species[src]
        pairs = None
        if prune_hops:
            xw, _ = orc.wrap(pos, cell)
            pi, pj, pn = orc.pairs_cells(xw, cell, RC)
            lev = hop_levels(len(src), (pi, pj), np.nonzero(w)[0], T)
            keep_atom = lev <= T
            keep_edge = (lev[pi] <= T - 1) | (lev[pj] <= T - 1)
            new = -np.ones(len(src), int)
            new[keep_atom] = np.arange(keep_atom.sum())
            keep_edge &= keep_atom[pi] & keep_atom[pj]
            pairs = (new[pi[keep_edge]], new[pj[keep_edge]], pn[keep_edge])
            pos, src, w, Z = xw[keep_atom], src[keep_atom], w[keep_atom], Z[keep_atom]
        r = orc.painn(vals, F, K, T, S, Z, pos, cell, pairs=pairs, weights=w)
        E += r["energy"]
        np.add.at(Fo, src, r["forces"])
        W += r["virial"]
        counts.append((int(w.sum()), len(src)))
    return E, Fo, W, counts


def test_weights_one_equals_unweighted(orc):
    F, K, T, S = 8, 20, 2, 2
    vals = syn.xavier_params(F, K, T, S, seed=1, bias_scale=0.2)
    sy = syn.water_box(12, seed=3)
    a = orc.painn(vals, F, K, T, S, sy.species, sy.positions, sy.cell)
    b = orc.painn(vals, F, K, T, S, sy.species, sy.positions, sy.cell, weights=np.ones(len(sy.species)))
    assert a["energy"] == b["energy"]
    np.testing.assert_array_equal(a["forces"], b["forces"])
    np.testing.assert_array_equal(a["virial"], b["virial"])


def test_unit_weight_selects_one_atom_energy_and_its_gradient(orc):
    """w = e_k: E = U_k (the unweighted per-atom energy) and the forces are -dU_k/dx by central
    finite differences; the virial is -dU_k/d(strain)."""
    F, K, T, S = 8, 20, 2, 2
    vals = syn.xavier_params(F, K, T, S, seed=2, bias_scale=0.2)
    sy = syn.water_box(10, seed=4)
    n = len(sy.species)
    k = 7
    w = np.zeros(n)
    w[k] = 1.0
    base = orc.painn(vals, F, K, T, S, sy.species, sy.positions, sy.cell)
    r = orc.painn(vals, F, K, T, S, sy.species, sy.positions, sy.cell, weights=w)
    assert r["energy"] == pytest.approx(base["energies"][k], rel=1e-14, abs=1e-15)
    np.testing.assert_array_equal(r["energies"], base["energies"])   # U_i themselves are unweighted

    def Uk(x, cell=sy.cell):
        return orc.painn(vals, F, K, T, S, sy.species, x, cell, forces=False, virial=False)["energies"][k]

    h = 1e-4
    fd = np.zeros((n, 3))
    for i in range(n):
        for c in range(3):
            xp, xm = sy.positions.copy(), sy.positions.copy()
            xp[i, c] += h
            xm[i, c] -= h
            fd[i, c] = -(Uk(xp) - Uk(xm)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 1e-6
    np.testing.assert_allclose(r["forces"], fd, rtol=0, atol=1e-7 * max(scale, 1.0))
    # virial = -dU_k/d(eps) under x -> (1 + eps) x, H -> H (1 + eps)^T
    hs = 1e-6
    Wfd = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            e = np.zeros((3, 3))
            e[a, b] = hs
            up = Uk(sy.positions @ (np.eye(3) + e).T, sy.cell @ (np.eye(3) + e).T)
            dn = Uk(sy.positions @ (np.eye(3) - e).T, sy.cell @ (np.eye(3) - e).T)
            Wfd[a, b] = -(up - dn) / (2 * hs)
    np.testing.assert_allclose(r["virial"], Wfd, rtol=0, atol=1e-6 * max(np.abs(Wfd).max(), 1.0))


def test_weights_are_linear(orc):
    """E(w) = sum_i w_i U_i for arbitrary weights; forces and virial are linear in w."""
    F, K, T, S = 8, 20, 2, 2
    vals = syn.xavier_params(F, K, T, S, seed=5, bias_scale=0.2)
    sy = syn.water_box(12, seed=6)
    n = len(sy.species)
    rng = np.random.default_rng(0)
    w1, w2 = rng.uniform(-1, 2, n), rng.uniform(-1, 2, n)
    r1 = orc.painn(vals, F, K, T, S, sy.species, sy.positions, sy.cell, weights=w1)
    r2 = orc.painn(vals, F, K, T, S, sy.species, sy.positions, sy.cell, weights=w2)
    r12 = orc.painn(vals, F, K, T, S, sy.species, sy.positions, sy.cell, weights=0.5 * w1 + 2.0 * w2)
    assert r1["energy"] == pytest.approx(float(w1 @ r1["energies"]), rel=1e-13)
    assert r12["energy"] == pytest.approx(0.5 * r1["energy"] + 2.0 * r2["energy"], rel=1e-12)
    np.testing.assert_allclose(r12["forces"], 0.5 * r1["forces"] + 2.0 * r2["forces"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r12["virial"], 0.5 * r1["virial"] + 2.0 * r2["virial"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("grid", [(2, 1, 1), (2, 2, 1), (1, 1, 1)])
def test_sum_rule_over_domains(orc, grid):
    """Owned energies summed over the domains = the periodic energy; copies' forces summed to
    their atoms = the periodic forces; subsystem virials summed = the periodic virial.  The
    (1, 1, 1) grid is the single-processor case: one domain whose copies are the periodic
    images within the halo."""
    F, K, T, S = 8, 20, 2, 1
    vals = syn.xavier_params(F, K, T, S, seed=7, bias_scale=0.2)
    sy = syn.fcc(3, 3, 3, seed=1)
    ref = orc.painn(vals, F, K, T, S, sy.species, sy.positions, sy.cell)
    E, Fo, W, counts = run_decomposed(orc, vals, F, K, T, S, sy, grid, halo=T * RC)
    assert sum(c[0] for c in counts) == len(sy.species)     # every atom owned exactly once
    assert E == pytest.approx(ref["energy"], rel=1e-12)
    fs = np.abs(ref["forces"]).max()
    np.testing.assert_allclose(Fo, ref["forces"], rtol=0, atol=1e-10 * fs)
    np.testing.assert_allclose(W, ref["virial"], rtol=0, atol=1e-10 * np.abs(ref["virial"]).max())


def test_sum_rule_triclinic_mixture(orc):
    """Triclinic cell with four species (a cut-down of the mixture generator)."""
    F, K, T, S = 8, 20, 2, 4
    vals = syn.xavier_params(F, K, T, S, seed=8, bias_scale=0.2)
    sy = syn.mixture(n_chain=12, n_water=60, seed=2)
    ref = orc.painn(vals, F, K, T, S, sy.species, sy.positions, sy.cell)
    E, Fo, W, _ = run_decomposed(orc, vals, F, K, T, S, sy, (2, 1, 2), halo=T * RC)
    assert E == pytest.approx(ref["energy"], rel=1e-12)
    np.testing.assert_allclose(Fo, ref["forces"], rtol=0, atol=1e-10 * np.abs(ref["forces"]).max())
    np.testing.assert_allclose(W, ref["virial"], rtol=0, atol=1e-10 * np.abs(ref["virial"]).max())


def test_hop_pruning_changes_nothing(orc):
    """Dropping copies more than T hops from every owned atom, and the edges not incident to an
    atom within T - 1 hops, leaves energy, forces and virial unchanged and removes atoms."""
    F, K, T, S = 8, 20, 2, 1
    vals = syn.xavier_params(F, K, T, S, seed=9, bias_scale=0.2)
    sy = syn.fcc(3, 3, 3, seed=2)
    E0, F0, W0, c0 = run_decomposed(orc, vals, F, K, T, S, sy, (2, 2, 1), halo=T * RC)
    E1, F1, W1, c1 = run_decomposed(orc, vals, F, K, T, S, sy, (2, 2, 1), halo=T * RC, prune_hops=True)
    assert sum(c[1] for c in c1) < sum(c[1] for c in c0)
    assert E1 == pytest.approx(E0, rel=1e-13)
    np.testing.assert_allclose(F1, F0, rtol=0, atol=1e-12 * np.abs(F0).max())
    np.testing.assert_allclose(W1, W0, rtol=0, atol=1e-12 * np.abs(W0).max())


def test_thin_halo_breaks_the_sum_rule(orc):
    """A halo of (T - 1) R misses part of the owned atoms' environments: the sum rule fails."""
    F, K, T, S = 8, 20, 2, 1
    vals = syn.xavier_params(F, K, T, S, seed=7, bias_scale=0.2)
    sy = syn.fcc(3, 3, 3, seed=1)
    ref = orc.painn(vals, F, K, T, S, sy.species, sy.positions, sy.cell)
    E, Fo, _, _ = run_decomposed(orc, vals, F, K, T, S, sy, (2, 1, 1), halo=(T - 1) * RC)
    assert abs(E - ref["energy"]) > 1e-8 * abs(ref["energy"])
    assert np.abs(Fo - ref["forces"]).max() > 1e-6 * np.abs(ref["forces"]).max()
