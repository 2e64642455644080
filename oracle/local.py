"""FP64 oracle for the strictly local equivariant edge model (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
this module; the product path never does.  It shares no code with the CUDA library.

Methods, "(Semi-)Local Potential Models" and "Chosen Architectures": the Allegro model passes
messages only between directed edges that leave the same atom, so an atom's energy depends on
nothing beyond its cutoff sphere however many layers the model has.  The paper gives no
equations for it; the form below is this project's restatement of an Allegro-type model
restricted to rotation orders l <= 1 and even parity:

  edge e = (i -> j, image n), r_e = x_j - x_i + n H, d_e = |r_e|, u_e = r_e / d_e,
  f_c(d) = (cos(pi d / rc) + 1) / 2, beta_e[k] = rbf_k(d_e) f_c(d_e) (the Gaussians of the
  PaiNN path: mu_k = k rc/(K-1), sigma = rc/(K-1)).
  two-body latent   x0_e = silu([beta_e | onehot(Z_i) | onehot(Z_j)] A0 + c0)          (F)
  initial features  w_e = x0_e P0;  s_e[c] = w_e[c],  v_e[c] = w_e[C+c] u_e            (C scalars, C vectors)
  layer l = 1..L:   om_e = x_e Q_l                                                      (2C)
                    Gs_i[c] = sum_{e from i} f_c(d_e) om_e[c]
                    Gv_i[c] = sum_{e from i} f_c(d_e) om_e[C+c] u_e
                    for e from i:  ts_e = [s_e * Gs_i | sum_a v_e[.,a] Gv_i[.,a]]      (paths 0x0->0, 1x1->0)
                                   tv_e = [s_e * Gv_i | v_e * Gs_i]                    (paths 0x1->1, 1x0->1)
                    x_e <- silu([x_e | ts_e] M_l + m_l)
                    (l < L)  s_e <- ts_e Gs_l,  v_e[.,a] <- tv_e[.,a] Gv_l             (channel mixing)
  readout           E_e = f_c(d_e) (silu(x_e R1 + d1) . R2 + d2),  E_i = e_scale w_i sum_{e from i} E_e

Forces are -dE/dx by automatic differentiation of the FP64 expression (PyTorch CPU), virial
W = -sum_e r_e (x) dE/dr_e.  What pins it (tests/test_oracle_local.py): central differences of
energy in positions and strain, rotation / translation / permutation invariance, strict locality
(an atom's energy ignores atoms beyond its cutoff, through any number of layers), continuity
of energy and forces when a pair crosses the cutoff, and a dimer evaluated with scalar
arithmetic.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import pairs_brute, wrap


def local_param_count(F: int, K: int, L: int, S: int, C: int) -> int:
    """Number of float64 values in the parameter list, in the order _unpack reads them."""
    KA = K + 2 * S
    n = KA * F + F + F * 2 * C
    for layer in range(1, L + 1):
        n += F * 2 * C + (F + 2 * C) * F + F
        if layer < L:
            n += 2 * (2 * C * C)
    Fh = F // 2
    return n + F * Fh + Fh + Fh + 1


def _unpack(params, F, K, L, S, C):
    p = torch.as_tensor(np.asarray(params, np.float64))
    assert p.numel() == local_param_count(F, K, L, S, C)
    off = 0

    def take(*shape):
        nonlocal off
        cnt = int(np.prod(shape))
        t = p[off:off + cnt].reshape(shape)
        off += cnt
        return t

    KA = K + 2 * S
    w = {"A0": take(KA, F), "c0": take(F), "P0": take(F, 2 * C), "layers": []}
    for layer in range(1, L + 1):
        lw = {"Q": take(F, 2 * C), "M": take(F + 2 * C, F), "m": take(F)}
        if layer < L:
            lw["Gs"] = take(2 * C, C)
            lw["Gv"] = take(2 * C, C)
        w["layers"].append(lw)
    Fh = F // 2
    w["R1"], w["d1"], w["R2"], w["d2"] = take(F, Fh), take(Fh), take(Fh), take(1)
    return w


def edges(positions, cell, rc):
    """Directed edges (i, j, r_e) with |r_e| < rc over all periodic images, r_e = x_j - x_i + n H
    from the wrapped positions (the oracle's brute-force pair set)."""
    H = np.asarray(cell, np.float64)
    xw, _ = wrap(np.asarray(positions, np.float64), H)
    i, j, s = pairs_brute(xw, H, rc)
    r = xw[j] - xw[i] + s.astype(np.float64) @ H
    return i, j, r


def silu(x):
    return x * torch.sigmoid(x)


def edge_energy_terms(w, F, K, L, S, C, species, i, j, r, n, rc):
    """Per-edge energies E_e (before e_scale and weights) as a function of the edge vectors r
    (torch, [E][3]); i, j: edge endpoints."""
    Z = torch.as_tensor(np.asarray(species, np.int64))
    it, jt = torch.as_tensor(i, dtype=torch.int64), torch.as_tensor(j, dtype=torch.int64)
    d = torch.sqrt((r * r).sum(1))
    u = r / d[:, None]
    fc = 0.5 * (torch.cos(math.pi * d / rc) + 1.0)
    k = torch.arange(K, dtype=torch.float64)
    mu, sig = k * rc / (K - 1), rc / (K - 1)
    beta = torch.exp(-((d[:, None] - mu) ** 2) / (2.0 * sig * sig)) * fc[:, None]
    oh = torch.eye(S, dtype=torch.float64)
    inp = torch.cat([beta, oh[Z[it]], oh[Z[jt]]], 1)
    x = silu(inp @ w["A0"] + w["c0"])
    w0 = x @ w["P0"]
    s = w0[:, :C]
    v = w0[:, None, C:] * u[:, :, None]                      # [E][3][C]
    for layer, lw in enumerate(w["layers"], start=1):
        om = x @ lw["Q"]
        Gs = torch.zeros(n, C, dtype=torch.float64).index_add(0, it, fc[:, None] * om[:, :C])
        Gv = torch.zeros(n, 3, C, dtype=torch.float64).index_add(
            0, it, (fc[:, None] * om[:, C:])[:, None, :] * u[:, :, None])
        gs, gv = Gs[it], Gv[it]
        ts = torch.cat([s * gs, (v * gv).sum(1)], 1)         # [E][2C]
        tv = torch.cat([s[:, None, :] * gv, v * gs[:, None, :]], 2)   # [E][3][2C]
        x = silu(torch.cat([x, ts], 1) @ lw["M"] + lw["m"])
        if layer < L:
            s = ts @ lw["Gs"]
            v = tv @ lw["Gv"]
    h = silu(x @ w["R1"] + w["d1"])
    return fc * (h @ w["R2"] + w["d2"][0])


def local_model(params, F, K, L, S, C, species, positions, cell, rc=5.0, e_scale=1.0, weights=None,
                need_grad=True):
    """Energy, per-atom energies, forces and virial (FP64) of the strictly local edge model.
    weights (per atom, optional): E = sum_i w_i E_i, the gradients seeded with w_i."""
    n = len(species)
    w = _unpack(params, F, K, L, S, C)
    i, j, r_np = edges(positions, cell, rc)
    r = torch.tensor(r_np, dtype=torch.float64, requires_grad=need_grad)
    ee = edge_energy_terms(w, F, K, L, S, C, species, i, j, r, n, rc)
    it = torch.as_tensor(i, dtype=torch.int64)
    Ei = torch.zeros(n, dtype=torch.float64).index_add(0, it, ee) * e_scale
    if weights is not None:
        Ei = Ei * torch.as_tensor(np.asarray(weights, np.float64))
    E = Ei.sum()
    out = {"energy": float(E.detach()), "energies": Ei.detach().numpy().copy(), "n_edges": len(i)}
    if not need_grad:
        return out
    (g,) = torch.autograd.grad(E, r) if len(i) else (torch.zeros((0, 3), dtype=torch.float64),)
    g = g.numpy()
    f = np.zeros((n, 3))
    np.add.at(f, i, g)      # r_e = x_j - x_i: -dE/dx_i collects +dE/dr_e of the edges leaving i
    np.add.at(f, j, -g)
    out["forces"] = f
    out["virial"] = -(r_np.T @ g)
    return out
