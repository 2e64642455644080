"""Pins for the oracle's PaiNN-form energy, forces and virial (CPU only).

What the paper fixes (arXiv 2506.04055): U = sum_i U_i over a cutoff graph (Methods, semi-local
energy equation); f_i = -dU/dr_i (Results "Distributed potential computation", sum-rule
equation); invariance of U to permutation, translation, rotation and reflection (Methods
"Descriptors"); locality with receptive field T*R (Methods "Graph Neural Networks").  The PaiNN
layer itself is not printed in the paper; the closed forms below evaluate hand-chosen special
cases of it with scalar algebra so that a dropped term, a swapped split block, a transposed
weight or a wrong radial/cutoff constant changes the value.
"""
import math

import numpy as np
import pytest

import synthetic as syn

RC = 5.0


def silu(x):
    return x / (1.0 + math.exp(-x))


def zero_params(F, K, T, S):
    vals = np.zeros(sum(int(np.prod(s)) for _, s in syn.param_shapes(F, K, T, S)))
    return vals, syn.unpack_params(vals, F, K, T, S)


def dimer(d, L=40.0, direction=(1.0, 0.0, 0.0)):
    u = np.asarray(direction, float)
    u /= np.linalg.norm(u)
    x = np.array([[10.0, 11.0, 12.0], [10.0, 11.0, 12.0]]) + np.array([[0, 0, 0], d * u])
    return x, np.eye(3) * L


def fc(d):
    return 0.5 * (math.cos(math.pi * d / RC) + 1.0) if d < RC else 0.0


# ----------------------------------------------------------------------------- closed forms
def test_T0_energy_is_readout_of_embedding(orc):
    """With no interaction layer U_i = e_scale (R2 . silu(R1 emb[Z_i] + d1) + d2); F = 0, W = 0."""
    F, K, T, S = 4, 3, 0, 2
    vals = syn.xavier_params(F, K, T, S, seed=5, bias_scale=0.3)
    P = syn.unpack_params(vals, F, K, T, S)
    sy = syn.water_box(8, seed=0)
    r = orc.painn(vals, F, K, T, S, sy.species, sy.positions, sy.cell, e_scale=1.7)
    expect = 0.0
    for z in sy.species:
        h = P["R1"] @ P["emb"][z] + P["d1"]
        expect += 1.7 * (sum(P["R2"][k] * silu(h[k]) for k in range(F // 2)) + P["d2"][0])
    assert r["energy"] == pytest.approx(expect, rel=1e-13)
    assert np.abs(r["forces"]).max() == 0.0 and np.abs(r["virial"]).max() == 0.0


def _const_layer(P, t, F, phi, beta, c2, U=None, V=None):
    """phi-MLP -> constant b2 = phi; filter -> constant bf = beta (times f_c); update MLP ->
    constant c2; U, V given (default identity)."""
    P[f"b2_{t}"][:] = phi
    P[f"bf_{t}"][:] = beta
    P[f"c2_{t}"][:] = c2
    P[f"U_{t}"][:] = np.eye(F) if U is None else U
    P[f"V_{t}"][:] = np.eye(F) if V is None else V


@pytest.mark.parametrize("d", [1.3, 2.7, 4.2, 4.999])
def test_dimer_one_layer_closed_form(orc, d):
    """T = 1 dimer with constant message / filter / update blocks.

    With phi = (ps, pvv, pvs), W_e = beta f_c(d), a = (avv, asv, ass) constants and U = V = I:
      s^m = e + ps*bs*fc ;  v^m_i = u_i * q, q = pvs*bvs*fc ;  <Uv, Vv> = q^2
      s'  = s^m + ass + asv q^2 ;  U_i = R2 . silu(R1 s' + d1) + d2 ; U = 2 U_i.
    """
    F, K, T, S = 2, 3, 1, 1
    vals, P = zero_params(F, K, T, S)
    e = np.array([0.3, -0.7])
    P["emb"][0] = e
    ps, pvv, pvs = np.array([0.9, -0.4]), np.array([0.25, 0.6]), np.array([-1.1, 0.8])
    bs, bvv, bvs = np.array([0.5, 1.3]), np.array([-0.2, 0.7]), np.array([0.45, -0.9])
    avv, asv, ass = np.array([0.1, -0.3]), np.array([0.65, 0.2]), np.array([-0.15, 0.35])
    _const_layer(P, 0, F, np.r_[ps, pvv, pvs], np.r_[bs, bvv, bvs], np.r_[avv, asv, ass])
    P["R1"][:] = [[1.2, -0.8]]
    P["d1"][:] = [0.05]
    P["R2"][:] = [1.5]
    P["d2"][:] = [-0.2]
    x, H = dimer(d, direction=(0.3, -0.5, 0.8))
    r = orc.painn(vals, F, K, T, S, [0, 0], x, H)
    c = fc(d)
    q = pvs * bvs * c
    sp = e + ps * bs * c + ass + asv * q * q
    Ui = 1.5 * silu(float(P["R1"][0] @ sp) + 0.05) - 0.2
    assert r["energy"] == pytest.approx(2 * Ui, rel=1e-12, abs=1e-14)
    np.testing.assert_allclose(r["energies"], [Ui, Ui], rtol=1e-12)


def test_dimer_beyond_cutoff_is_two_free_atoms(orc):
    F, K, T, S = 2, 3, 1, 1
    vals = syn.xavier_params(F, K, T, S, seed=3, bias_scale=0.4)
    for d in (5.0, 5.5):
        x, H = dimer(d)
        r = orc.painn(vals, F, K, T, S, [0, 0], x, H)
        x2, _ = dimer(20.0)
        r2 = orc.painn(vals, F, K, T, S, [0, 0], x2, H)
        assert r["energy"] == r2["energy"]
        assert np.abs(r["forces"]).max() == 0.0
    # continuity as the pair enters the cutoff: f_c and f_c' vanish at rc
    x, H = dimer(RC - 1e-6)
    near = orc.painn(vals, F, K, T, S, [0, 0], x, H)
    assert abs(near["energy"] - r2["energy"]) < 1e-9
    assert np.abs(near["forces"]).max() < 1e-5


@pytest.mark.parametrize("k0", [0, 7, 19])
def test_dimer_radial_basis_closed_form(orc, k0):
    """One filter channel reads one Gaussian: W_s0 = rbf_k0(d) f_c(d) with mu_k = k rc/(K-1),
    sigma = rc/(K-1); U_i = silu(e0 + ps0 * W_s0) (everything else zero)."""
    F, K, T, S = 2, 20, 1, 1
    vals, P = zero_params(F, K, T, S)
    P["emb"][0] = [0.4, 0.0]
    P["b2_0"][0] = 1.7                     # phi_s0
    P["Wf_0"][0, k0] = 1.0                 # W_s0 = rbf_k0 f_c
    P["R1"][:] = [[1.0, 0.0]]
    P["R2"][:] = [1.0]
    sig = RC / (K - 1)
    for d in (0.9, 2.1, 3.6, 4.8):
        x, H = dimer(d)
        r = orc.painn(vals, F, K, T, S, [0, 0], x, H)
        rb = math.exp(-(d - k0 * RC / (K - 1)) ** 2 / (2 * sig * sig))
        expect = 2 * silu(0.4 + 1.7 * rb * fc(d))
        assert r["energy"] == pytest.approx(expect, rel=1e-12)


def test_dimer_phi_mlp_closed_form(orc):
    """phi = W2 silu(W1 s + b1) + b2 with asymmetric 2x2 W1 and a 6x2 W2 (order [s|vv|vs])."""
    F, K, T, S = 2, 3, 1, 1
    vals, P = zero_params(F, K, T, S)
    e = np.array([0.6, -0.2])
    P["emb"][0] = e
    W1 = np.array([[0.5, -1.2], [0.9, 0.3]])
    b1 = np.array([0.1, -0.4])
    W2 = np.array([[0.7, 0.2], [-0.5, 1.1], [0.3, 0.3], [0.0, -0.6], [1.4, -0.2], [0.8, 0.5]])
    b2 = np.array([0.05, -0.1, 0.2, 0.0, -0.3, 0.15])
    P["W1_0"][:] = W1
    P["b1_0"][:] = b1
    P["W2_0"][:] = W2
    P["b2_0"][:] = b2
    beta = np.array([0.4, -0.9, 0.3, 0.8, 0.6, -0.5])
    c2 = np.array([0.2, -0.1, 0.7, 0.4, -0.3, 0.25])
    _const_layer(P, 0, F, b2, beta, c2)
    P["W1_0"][:] = W1     # _const_layer only touched b2/bf/c2/U/V
    P["R1"][:] = [[0.9, 1.3]]
    P["R2"][:] = [1.0]
    d = 3.1
    x, H = dimer(d, direction=(1, 1, 0))
    r = orc.painn(vals, F, K, T, S, [0, 0], x, H)
    a1 = np.array([silu(v) for v in W1 @ e + b1])
    phi = W2 @ a1 + b2
    c = fc(d)
    q = phi[4:6] * beta[4:6] * c
    sp = e + phi[0:2] * beta[0:2] * c + c2[4:6] + c2[2:4] * q * q
    expect = 2 * silu(float(np.array([0.9, 1.3]) @ sp))
    assert r["energy"] == pytest.approx(expect, rel=1e-12)


def test_dimer_two_layers_vector_channel(orc):
    """T = 2 exercises v_j phi_vv W_vv (zero in layer 1 since v^0 = 0) and a_vv U v.

    Layer 1 (constants, U = V = I):  v1_i = u_i q1 (1 + avv1),  s1 = e + ps1 bs1 fc + ass1 + asv1 q1^2
    Layer 2: v_j = -v_i for a dimer, so v^m_i = u_i w with
             w = q1 (1 + avv1) (1 - pvv2 bvv2 fc) + pvs2 bvs2 fc;  s2 = s1 + ps2 bs2 fc + ass2 + asv2 (U w).(V w)
    with non-identity U, V in layer 2 so the <Uv, Vv> term sees both matrices."""
    F, K, T, S = 2, 3, 2, 1
    vals, P = zero_params(F, K, T, S)
    e = np.array([0.2, 0.5])
    P["emb"][0] = e
    phi1, beta1, c21 = (np.array([0.3, -0.6, 0.9, 0.4, 1.2, -0.7]),
                        np.array([0.8, 0.2, -0.5, 0.6, 0.5, 0.9]),
                        np.array([0.3, -0.4, 0.1, 0.2, -0.2, 0.6]))
    phi2, beta2, c22 = (np.array([-0.4, 0.7, 0.55, -0.35, 0.6, 0.9]),
                        np.array([0.3, -0.8, 0.75, 0.45, -0.6, 0.2]),
                        np.array([-0.25, 0.5, 0.4, -0.3, 0.15, -0.45]))
    U2 = np.array([[1.1, -0.4], [0.3, 0.8]])
    V2 = np.array([[0.6, 0.9], [-0.7, 0.2]])
    _const_layer(P, 0, F, phi1, beta1, c21)
    _const_layer(P, 1, F, phi2, beta2, c22, U=U2, V=V2)
    P["R1"][:] = [[0.7, -1.1]]
    P["R2"][:] = [1.3]
    d = 2.4
    x, H = dimer(d, direction=(0.2, 0.9, -0.4))
    r = orc.painn(vals, F, K, T, S, [0, 0], x, H, eps=1e-8)
    c = fc(d)
    q1 = phi1[4:6] * beta1[4:6] * c
    s1 = e + phi1[0:2] * beta1[0:2] * c + c21[4:6] + c21[2:4] * q1 * q1
    w1 = q1 * (1 + c21[0:2])
    w = w1 - w1 * phi2[2:4] * beta2[2:4] * c + phi2[4:6] * beta2[4:6] * c
    Uw, Vw = U2 @ w, V2 @ w
    s2 = s1 + phi2[0:2] * beta2[0:2] * c + c22[4:6] + c22[2:4] * Uw * Vw
    expect = 2 * 1.3 * silu(float(np.array([0.7, -1.1]) @ s2))
    assert r["energy"] == pytest.approx(expect, rel=1e-12)


def test_update_mlp_sees_norm_of_Vv(orc):
    """a = A2 silu(A1 [s ; sqrt(|Vv|^2 + eps)] + c1) + c2: the second half of A1 reads nV."""
    F, K, T, S = 2, 3, 1, 1
    vals, P = zero_params(F, K, T, S)
    e = np.array([0.1, 0.3])
    P["emb"][0] = e
    phi = np.array([0.0, 0.0, 0.0, 0.0, 0.8, -1.2])
    beta = np.array([0.0, 0.0, 0.0, 0.0, 0.7, 0.4])
    _const_layer(P, 0, F, phi, beta, np.zeros(6))
    A1 = np.array([[0.2, -0.5, 1.1, 0.4], [0.6, 0.3, -0.8, 0.9]])
    c1 = np.array([0.05, -0.1])
    A2 = np.array([[0.3, 0.1], [0.2, -0.4], [0.5, 0.6], [-0.3, 0.2], [0.9, -0.7], [0.4, 0.8]])
    P["A1_0"][:] = A1
    P["c1_0"][:] = c1
    P["A2_0"][:] = A2
    P["R1"][:] = [[1.0, 0.5]]
    P["R2"][:] = [1.0]
    d = 3.3
    x, H = dimer(d)
    eps = 1e-8
    r = orc.painn(vals, F, K, T, S, [0, 0], x, H, eps=eps)
    c = fc(d)
    q = phi[4:6] * beta[4:6] * c
    nV = np.sqrt(q * q + eps)
    a2 = np.array([silu(t) for t in A1 @ np.r_[e, nV] + c1])
    a = A2 @ a2
    s1 = e + a[4:6] + a[2:4] * q * q
    expect = 2 * silu(float(np.array([1.0, 0.5]) @ s1))
    assert r["energy"] == pytest.approx(expect, rel=1e-12)


# ----------------------------------------------------------------------------- derivatives
def _model(seed=0, F=8, K=20, T=2, S=2, bias=0.2):
    return syn.xavier_params(F, K, T, S, seed=seed, bias_scale=bias), (F, K, T, S)


def _small_water(nmol=12, seed=0):
    sy = syn.water_box(nmol, seed=seed)
    return sy


def test_forces_match_central_differences(orc):
    vals, dims = _model(seed=1, F=8, T=3)
    sy = _small_water(27, seed=2)
    xw, _ = orc.wrap(sy.positions, sy.cell)
    pairs = orc.pairs_cells(xw, sy.cell, RC + 1.5)     # skin list: stays valid under +-h
    r = orc.painn(vals, *dims, sy.species, xw, sy.cell, pairs=pairs)
    h = 1e-4
    rng = np.random.default_rng(0)
    for i in rng.choice(sy.n, 6, replace=False):
        for c in range(3):
            xp = xw.copy(); xp[i, c] += h
            xm = xw.copy(); xm[i, c] -= h
            ep = orc.painn(vals, *dims, sy.species, xp, sy.cell, pairs=pairs, forces=False, virial=False)["energy"]
            em = orc.painn(vals, *dims, sy.species, xm, sy.cell, pairs=pairs, forces=False, virial=False)["energy"]
            fd = -(ep - em) / (2 * h)
            assert r["forces"][i, c] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_virial_matches_strain_differences(orc):
    """W_ab = -sum_e r_e,a dU/dr_e,b equals -dU/d eps_ba under x -> (1+eps) x, H -> H (1+eps)^T."""
    vals, dims = _model(seed=2, F=8, T=2)
    sy = _small_water(16, seed=4)
    H = sy.cell.copy()
    H[1, 0] = 0.6; H[2, 0] = -0.4; H[2, 1] = 0.3         # triclinic
    xw, _ = orc.wrap(sy.positions, H)
    pairs = orc.pairs_cells(xw, H, RC + 1.5)
    r = orc.painn(vals, *dims, sy.species, xw, H, pairs=pairs)
    W = r["virial"]
    h = 1e-6
    for a in range(3):
        for b in range(3):
            E = []
            for sgn in (1, -1):
                eps = np.zeros((3, 3)); eps[a, b] = sgn * h
                M = np.eye(3) + eps
                E.append(orc.painn(vals, *dims, sy.species, xw @ M.T, H @ M.T, pairs=pairs,
                                   forces=False, virial=False)["energy"])
            dEde = (E[0] - E[1]) / (2 * h)
            assert W[b, a] == pytest.approx(-dEde, rel=1e-6, abs=1e-7)
    np.testing.assert_allclose(W, W.T, atol=1e-12 * np.abs(W).max())


def test_force_sum_zero_and_energy_sum(orc):
    vals, dims = _model(seed=3, F=16, T=3)
    sy = syn.water_box(40, seed=5)
    r = orc.painn(vals, *dims, sy.species, sy.positions, sy.cell)
    assert np.abs(r["forces"].sum(0)).max() < 1e-12 * max(1.0, np.abs(r["forces"]).max()) * sy.n
    assert r["energy"] == pytest.approx(r["energies"].sum(), rel=1e-14)


# ----------------------------------------------------------------------------- invariances
def _random_rotation(rng, reflect=False):
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    if reflect:
        q = q @ np.diag([1, 1, -1])
    return q


@pytest.mark.parametrize("reflect", [False, True])
def test_rotation_reflection_invariance(orc, reflect):
    vals, dims = _model(seed=4, F=8, T=3)
    sy = _small_water(20, seed=6)
    H = sy.cell.copy(); H[2, 0] = 0.5; H[1, 0] = -0.3
    r0 = orc.painn(vals, *dims, sy.species, sy.positions, H)
    Q = _random_rotation(np.random.default_rng(7), reflect)
    r1 = orc.painn(vals, *dims, sy.species, sy.positions @ Q.T, H @ Q.T)
    assert r1["energy"] == pytest.approx(r0["energy"], rel=1e-12)
    np.testing.assert_allclose(r1["forces"], r0["forces"] @ Q.T, atol=1e-11)
    np.testing.assert_allclose(r1["virial"], Q @ r0["virial"] @ Q.T, atol=1e-10)


def test_translation_and_permutation_invariance(orc):
    vals, dims = _model(seed=5, F=8, T=2)
    sy = _small_water(20, seed=8)
    r0 = orc.painn(vals, *dims, sy.species, sy.positions, sy.cell)
    r1 = orc.painn(vals, *dims, sy.species, sy.positions + np.array([3.3, -17.2, 40.1]), sy.cell)
    assert r1["energy"] == pytest.approx(r0["energy"], rel=1e-12)
    np.testing.assert_allclose(r1["forces"], r0["forces"], atol=1e-11)
    perm = np.random.default_rng(1).permutation(sy.n)
    r2 = orc.painn(vals, *dims, sy.species[perm], sy.positions[perm], sy.cell)
    assert r2["energy"] == pytest.approx(r0["energy"], rel=1e-12)
    np.testing.assert_allclose(r2["forces"], r0["forces"][perm], atol=1e-11)
    np.testing.assert_allclose(r2["energies"], r0["energies"][perm], rtol=1e-11)


def test_species_matter(orc):
    """Swapping the species of one O/H pair changes the energy (embedding is read by Z)."""
    vals, dims = _model(seed=6, F=8, T=2)
    sy = _small_water(8, seed=1)
    r0 = orc.painn(vals, *dims, sy.species, sy.positions, sy.cell)
    Z = sy.species.copy(); Z[0], Z[1] = Z[1], Z[0]
    r1 = orc.painn(vals, *dims, Z, sy.positions, sy.cell)
    assert abs(r1["energy"] - r0["energy"]) > 1e-6


def test_pruned_edges_change_nothing(orc):
    """Edges longer than rc contribute exactly nothing (the per-step pruning is exact)."""
    vals, dims = _model(seed=7, F=8, T=3)
    sy = _small_water(27, seed=3)
    xw, _ = orc.wrap(sy.positions, sy.cell)
    a = orc.painn(vals, *dims, sy.species, xw, sy.cell, pairs=orc.pairs_cells(xw, sy.cell, RC))
    b = orc.painn(vals, *dims, sy.species, xw, sy.cell, pairs=orc.pairs_cells(xw, sy.cell, RC + 2.0))
    assert a["energy"] == b["energy"]
    np.testing.assert_array_equal(a["forces"], b["forces"])
    np.testing.assert_allclose(a["virial"], b["virial"], rtol=1e-13, atol=1e-13)


def test_supercell_extensivity(orc):
    """A 2x1x2 replica of a periodic box has 4x the energy and the same per-atom forces."""
    vals, dims = _model(seed=8, F=8, T=2)
    sy = syn.fcc(2, 2, 2, jitter=0.1, seed=9)
    r = orc.painn(vals, *dims, sy.species, sy.positions, sy.cell)
    reps = [np.array([a, 0, c]) @ sy.cell for a in range(2) for c in range(2)]
    X = np.concatenate([sy.positions + t for t in reps])
    H2 = sy.cell * np.array([2, 1, 2])[:, None]
    r2 = orc.painn(vals, *dims, np.tile(sy.species, 4), X, H2)
    assert r2["energy"] == pytest.approx(4 * r["energy"], rel=1e-12)
    np.testing.assert_allclose(r2["forces"], np.tile(r["forces"], (4, 1)), atol=1e-11)
    np.testing.assert_allclose(r2["virial"], 4 * r["virial"], rtol=1e-10, atol=1e-10)


def test_locality_receptive_field(orc):
    """U_i depends only on atoms within T*rc (a path of at most T edges, Methods "Graph Neural
    Networks"): in a chain along x, moving the last atom changes U_0 only if it is within T hops."""
    F, K, T, S = 8, 20, 2, 1
    vals = syn.xavier_params(F, K, T, S, seed=9, bias_scale=0.2)
    H = np.diag([200.0, 30.0, 30.0])
    xs = [0.0, 4.0, 8.0, 12.0]
    base = np.array([[x, 5.0, 5.0] for x in xs])
    r0 = orc.painn(vals, F, K, T, S, [0] * 4, base, H)
    moved = base.copy(); moved[3, 1] += 0.3          # atom 3 is 3 hops from atom 0
    r1 = orc.painn(vals, F, K, T, S, [0] * 4, moved, H)
    assert r1["energies"][0] == r0["energies"][0]
    assert r1["energies"][1] != r0["energies"][1]    # atom 1 is 2 hops away: within T = 2
