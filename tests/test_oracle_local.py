"""Pins of the FP64 oracle of the strictly local edge model (oracle/local.py), on the CPU.

Methods, "(Semi-)Local Potential Models" and "Chosen Architectures": the Allegro-type model
exchanges information only between edges leaving the same atom, so an atom's energy is a
function of its own cutoff sphere alone.  Pins: a dimer and a trimer evaluated with scalar
arithmetic along the bond (all vectors of a dimer are parallel to it), central differences of
the energy in positions and in strain, invariance under rotations, reflections, translations
and permutations, strict locality through three layers, continuity at the cutoff, energy
weights and supercell extensivity.
"""
import math

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.filterwarnings("ignore::UserWarning")

RC = 5.0
K = 20


@pytest.fixture(scope="module")
def loc():
    torch = pytest.importorskip("torch")
    del torch
    import oracle.local as ol
    return ol


def _silu(x):
    return x / (1.0 + math.exp(-x))


def _vals(F, L, S, C, seed, bias=0.2):
    return syn.local_xavier_params(F, K, L, S, C, seed=seed, bias_scale=bias)


def _named(vals, F, L, S, C):
    out, off = {}, 0
    for name, shape in syn.local_param_shapes(F, K, L, S, C):
        cnt = int(np.prod(shape))
        out[name] = vals[off:off + cnt].reshape(shape)
        off += cnt
    return out


def _scalar_edge_energy(p, F, L, S, C, zi, zj, d, cos_other=None, d_other=None, z_other=None):
    """Energy of the edge i -> j for a centre whose only other edge (if any) goes to an atom at
    distance d_other, at angle arccos(cos_other) from the first: plain Python floats.  Every
    vector feature of an edge is a multiple of that edge's direction, so vectors are carried as
    their coefficients and dot products of two directions give 1 or cos_other."""
    def fc(r):
        return 0.5 * (math.cos(math.pi * r / RC) + 1.0)

    def x0(r, a, b):
        sig = RC / (K - 1)
        beta = [math.exp(-((r - k * sig) ** 2) / (2 * sig * sig)) * fc(r) for k in range(K)]
        out = []
        for f in range(F):
            z = sum(beta[k] * p["A0"][k, f] for k in range(K)) + p["A0"][K + a, f] + p["A0"][K + S + b, f] + p["c0"][f]
            out.append(_silu(z))
        return out

    def matvec(x, M):   # row vector times matrix
        return [sum(x[q] * M[q, c] for q in range(len(x))) for c in range(M.shape[1])]

    edges = [(d, zj, 1.0)]
    if d_other is not None:
        edges.append((d_other, z_other, cos_other))
    # per edge: latent x, scalars s, vector coefficients v (along the edge's own direction)
    xs = [x0(r, zi, b) for r, b, _ in edges]
    ws = [matvec(x, p["P0"]) for x in xs]
    ss = [w[:C] for w in ws]
    vs = [w[C:] for w in ws]
    for layer in range(1, L + 1):
        oms = [matvec(x, p[f"Q{layer}"]) for x in xs]
        Gs = [sum(fc(edges[e][0]) * oms[e][c] for e in range(len(edges))) for c in range(C)]
        # Gv as coefficients of each edge direction: Gv = sum_e fc_e om_e[C+c] u_e
        gv_coef = [[fc(edges[e][0]) * oms[e][C + c] for c in range(C)] for e in range(len(edges))]

        def dot_with_gv(e, c):   # u_e . Gv[c]
            tot = 0.0
            for q in range(len(edges)):
                cosq = 1.0 if q == e else edges[1][2]
                tot += gv_coef[q][c] * cosq
            return tot

        new_x, new_s, new_v = [], [], []
        for e in range(len(edges)):
            ts = [ss[e][c] * Gs[c] for c in range(C)] + [vs[e][c] * dot_with_gv(e, c) for c in range(C)]
            new_x.append([_silu(z) for z in
                          [a + b for a, b in zip(matvec(xs[e] + ts, p[f"M{layer}"]), p[f"m{layer}"])]])
            if layer < L:
                new_s.append(matvec(ts, p[f"Gs{layer}"]))
                # tv = [s Gv | v Gs]; only the component along u_e matters for the next layer's
                # dot products when every other direction enters through cosines -- true when
                # the centre has one edge (Gv is then parallel to u_e)
                assert len(edges) == 1
                tv = [ss[e][c] * gv_coef[e][c] for c in range(C)] + [vs[e][c] * Gs[c] for c in range(C)]
                new_v.append(matvec(tv, p[f"Gv{layer}"]))
        xs, ss, vs = new_x, new_s, new_v
    h = [_silu(a + b) for a, b in zip(matvec(xs[0], p["R1"]), p["d1"])]
    return fc(d) * (sum(h[k] * p["R2"][k] for k in range(F // 2)) + p["d2"][0])


@pytest.mark.parametrize("d", [1.1, 2.7, 4.6])
def test_dimer_scalar_evaluation(loc, d):
    """Two atoms of different species, two layers: each atom's energy equals the scalar
    evaluation along the bond (centre and neighbour species in their own slots)."""
    F, L, S, C = 8, 2, 2, 2
    vals = _vals(F, L, S, C, seed=1)
    p = _named(vals, F, L, S, C)
    u = np.array([0.3, -0.5, 0.81])
    u /= np.linalg.norm(u)
    x = np.array([[10.0, 10.0, 10.0], [10.0, 10.0, 10.0]]) + np.outer([0.0, d], u)
    out = loc.local_model(vals, F, K, L, S, C, np.array([0, 1]), x, np.eye(3) * 30.0, need_grad=False)
    e0 = _scalar_edge_energy(p, F, L, S, C, 0, 1, d)
    e1 = _scalar_edge_energy(p, F, L, S, C, 1, 0, d)
    assert out["energies"][0] == pytest.approx(e0, rel=1e-12, abs=1e-14)
    assert out["energies"][1] == pytest.approx(e1, rel=1e-12, abs=1e-14)
    assert abs(e0 - e1) > 1e-6   # the species slots matter


@pytest.mark.parametrize("theta", [40.0, 95.0, 150.0])
def test_trimer_angle_enters_through_vector_path(loc, theta):
    """A centre with two neighbours, one layer: its energy equals the scalar evaluation in
    which the angle enters only through u_1 . u_2 = cos(theta) (the 1 x 1 -> 0 path), and it
    changes with the angle."""
    F, L, S, C = 8, 1, 2, 2
    vals = _vals(F, L, S, C, seed=2)
    p = _named(vals, F, L, S, C)
    d1, d2 = 2.2, 3.1
    t = math.radians(theta)
    x = np.array([[0.0, 0.0, 0.0], [d1, 0.0, 0.0], [d2 * math.cos(t), d2 * math.sin(t), 0.0]]) + 10.0
    z = np.array([0, 1, 1])
    out = loc.local_model(vals, F, K, L, S, C, z, x, np.eye(3) * 30.0, need_grad=False)
    e_01 = _scalar_edge_energy(p, F, L, S, C, 0, 1, d1, math.cos(t), d2, 1)
    e_02 = _scalar_edge_energy(p, F, L, S, C, 0, 1, d2, math.cos(t), d1, 1)
    assert out["energies"][0] == pytest.approx(e_01 + e_02, rel=1e-12, abs=1e-14)
    other = loc.local_model(vals, F, K, L, S, C, z,
                            np.array([[0.0, 0.0, 0.0], [d1, 0.0, 0.0], [0.0, d2, 0.0]]) + 10.0,
                            np.eye(3) * 30.0, need_grad=False)
    if abs(theta - 90.0) > 1.0:
        assert abs(other["energies"][0] - out["energies"][0]) > 1e-8


def _water(nmol, seed):
    return syn.water_box(nmol, seed=seed)


def test_forces_match_central_differences(loc):
    F, L, S, C = 8, 2, 2, 4
    vals = _vals(F, L, S, C, seed=3)
    sy = _water(16, seed=1)
    ref = loc.local_model(vals, F, K, L, S, C, sy.species, sy.positions, sy.cell)
    h = 1e-5
    rng = np.random.default_rng(0)
    for a in rng.choice(len(sy.species), 5, replace=False):
        for c in range(3):
            e = []
            for sgn in (1, -1):
                x = sy.positions.copy()
                x[a, c] += sgn * h
                e.append(loc.local_model(vals, F, K, L, S, C, sy.species, x, sy.cell, need_grad=False)["energy"])
            fd = -(e[0] - e[1]) / (2 * h)
            assert ref["forces"][a, c] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    np.testing.assert_allclose(ref["forces"].sum(0), 0.0, atol=1e-12)


def test_virial_matches_strain_differences(loc):
    """W_ab = -sum_e r_e,a dE/dr_e,b equals -dE/d eps_ba under x -> (1+eps) x, H -> H (1+eps)^T."""
    F, L, S, C = 8, 2, 2, 4
    vals = _vals(F, L, S, C, seed=4)
    sy = _water(16, seed=2)
    H = sy.cell.copy()
    H[1, 0] = 0.6; H[2, 0] = -0.4; H[2, 1] = 0.3
    W = loc.local_model(vals, F, K, L, S, C, sy.species, sy.positions, H)["virial"]
    h = 1e-6
    for a in range(3):
        for b in range(3):
            e = []
            for sgn in (1, -1):
                eps = np.zeros((3, 3)); eps[a, b] = sgn * h
                M = np.eye(3) + eps
                e.append(loc.local_model(vals, F, K, L, S, C, sy.species, sy.positions @ M.T, H @ M.T,
                                         need_grad=False)["energy"])
            assert W[b, a] == pytest.approx(-(e[0] - e[1]) / (2 * h), rel=1e-6, abs=1e-7)
    np.testing.assert_allclose(W, W.T, atol=1e-12 * np.abs(W).max())


@pytest.mark.parametrize("reflect", [False, True])
def test_rotation_reflection_invariance(loc, reflect):
    F, L, S, C = 8, 2, 2, 4
    vals = _vals(F, L, S, C, seed=5)
    sy = _water(12, seed=3)
    q, _ = np.linalg.qr(np.random.default_rng(1).normal(size=(3, 3)))
    if (np.linalg.det(q) < 0) != reflect:
        q[:, 0] *= -1
    a = loc.local_model(vals, F, K, L, S, C, sy.species, sy.positions, sy.cell)
    b = loc.local_model(vals, F, K, L, S, C, sy.species, sy.positions @ q.T, sy.cell @ q.T)
    assert b["energy"] == pytest.approx(a["energy"], rel=1e-12)
    np.testing.assert_allclose(b["forces"], a["forces"] @ q.T, atol=1e-11)
    np.testing.assert_allclose(b["virial"], q @ a["virial"] @ q.T, atol=1e-10)


def test_translation_and_permutation_invariance(loc):
    F, L, S, C = 8, 2, 2, 4
    vals = _vals(F, L, S, C, seed=6)
    sy = _water(12, seed=4)
    a = loc.local_model(vals, F, K, L, S, C, sy.species, sy.positions, sy.cell)
    t = loc.local_model(vals, F, K, L, S, C, sy.species, sy.positions + np.array([1.3, -7.1, 22.0]), sy.cell)
    assert t["energy"] == pytest.approx(a["energy"], rel=1e-12)
    np.testing.assert_allclose(t["forces"], a["forces"], atol=1e-11)
    perm = np.random.default_rng(2).permutation(len(sy.species))
    p = loc.local_model(vals, F, K, L, S, C, sy.species[perm], sy.positions[perm], sy.cell)
    assert p["energy"] == pytest.approx(a["energy"], rel=1e-12)
    np.testing.assert_allclose(p["forces"], a["forces"][perm], atol=1e-11)
    np.testing.assert_allclose(p["energies"], a["energies"][perm], atol=1e-12)


def test_strict_locality_through_three_layers(loc):
    """A - B - C on a line, |AB| = |BC| = 3 A, |AC| = 6 A > rc: moving C (still within rc of B)
    leaves A's energy exactly unchanged with three layers, while B's changes."""
    F, L, S, C = 8, 3, 2, 2
    vals = _vals(F, L, S, C, seed=7)
    base = np.array([[5.0, 10.0, 10.0], [8.0, 10.0, 10.0], [11.0, 10.0, 10.0]])
    moved = base.copy()
    moved[2] += [0.2, 0.3, -0.1]
    z = np.array([0, 1, 0])
    a = loc.local_model(vals, F, K, L, S, C, z, base, np.eye(3) * 40.0, need_grad=False)
    b = loc.local_model(vals, F, K, L, S, C, z, moved, np.eye(3) * 40.0, need_grad=False)
    assert a["energies"][0] == b["energies"][0]
    assert abs(a["energies"][1] - b["energies"][1]) > 1e-8


def test_continuity_at_the_cutoff(loc):
    """A dimer just inside and just outside rc: energies and forces go to zero continuously
    (the cosine cutoff and its derivative vanish at rc)."""
    F, L, S, C = 8, 2, 2, 2
    vals = _vals(F, L, S, C, seed=8)
    z = np.array([0, 1])
    for delta, tol_e, tol_f in ((1e-3, 1e-4, 1e-2), (1e-4, 1e-6, 1e-3)):
        inside = loc.local_model(vals, F, K, L, S, C, z, np.array([[5.0, 5, 5], [5.0 + RC - delta, 5, 5]]),
                                 np.eye(3) * 40.0)
        outside = loc.local_model(vals, F, K, L, S, C, z, np.array([[5.0, 5, 5], [5.0 + RC + delta, 5, 5]]),
                                  np.eye(3) * 40.0)
        assert outside["energy"] == 0.0 and np.all(outside["forces"] == 0.0)
        assert abs(inside["energy"]) < tol_e
        assert np.abs(inside["forces"]).max() < tol_f


def test_energy_weights_scale_per_atom_energies(loc):
    F, L, S, C = 8, 2, 2, 4
    vals = _vals(F, L, S, C, seed=9)
    sy = _water(8, seed=5)
    w = np.random.default_rng(3).uniform(0.0, 1.0, len(sy.species))
    a = loc.local_model(vals, F, K, L, S, C, sy.species, sy.positions, sy.cell)
    b = loc.local_model(vals, F, K, L, S, C, sy.species, sy.positions, sy.cell, weights=w)
    np.testing.assert_allclose(b["energies"], a["energies"] * w, rtol=1e-14, atol=1e-15)
    # w = 1 on one atom, 0 elsewhere: its forces are minus the gradient of that atom's energy
    one = np.zeros(len(sy.species)); one[4] = 1.0
    c = loc.local_model(vals, F, K, L, S, C, sy.species, sy.positions, sy.cell, weights=one)
    h = 1e-5
    for comp in range(3):
        e = []
        for sgn in (1, -1):
            x = sy.positions.copy(); x[7, comp] += sgn * h
            e.append(loc.local_model(vals, F, K, L, S, C, sy.species, x, sy.cell, need_grad=False)["energies"][4])
        assert c["forces"][7, comp] == pytest.approx(-(e[0] - e[1]) / (2 * h), rel=1e-6, abs=1e-9)


def test_supercell_extensivity(loc):
    """A 2x1x2 replica of a periodic cell has 4x the energy and virial, and each copy of an atom
    carries its forces and energy (periodic images are handled like any other neighbour)."""
    F, L, S, C = 8, 2, 2, 4
    vals = _vals(F, L, S, C, seed=11)
    sy = _water(8, seed=6)
    a = loc.local_model(vals, F, K, L, S, C, sy.species, sy.positions, sy.cell)
    reps = [(i, 0, k) for i in range(2) for k in range(2)]
    x = np.concatenate([sy.positions + np.array(r) @ sy.cell for r in reps])
    z = np.concatenate([sy.species] * len(reps))
    H = sy.cell * np.array([[2.0], [1.0], [2.0]])
    b = loc.local_model(vals, F, K, L, S, C, z, x, H)
    assert b["energy"] == pytest.approx(4 * a["energy"], rel=1e-12)
    np.testing.assert_allclose(b["virial"], 4 * a["virial"], rtol=1e-11, atol=1e-11)
    n = len(sy.species)
    for q in range(len(reps)):
        np.testing.assert_allclose(b["forces"][q * n:(q + 1) * n], a["forces"], atol=1e-11)
        np.testing.assert_allclose(b["energies"][q * n:(q + 1) * n], a["energies"], atol=1e-12)
