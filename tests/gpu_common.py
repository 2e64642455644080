"""Helpers shared by the GPU tests: build/load the engine, tolerances, oracle comparison."""
import numpy as np

import synthetic as syn

# Tolerances (stated for the FP32 path): relative force RMSE and per-atom energy error as a
# fraction of the RMS per-atom energy; virial relative Frobenius error.
FP32_FORCE_RMSE = 1e-5
FP32_ENERGY_PER_ATOM = 1e-6
FP32_VIRIAL_REL = 1e-5
BF16_FORCE_RMSE = 1e-2


def engine():
    import paper_2506_04055_gb300 as eng
    eng.build()
    eng.load()
    return eng


def rel_force_rmse(f, fref):
    return float(np.sqrt(((f - fref) ** 2).sum()) / np.sqrt((fref ** 2).sum()))


def energy_err_per_atom(e, eref, eatoms_ref):
    n = len(eatoms_ref)
    scale = float(np.sqrt(np.mean(eatoms_ref ** 2)))
    return abs(e - eref) / n / scale


def virial_rel(w, wref):
    return float(np.linalg.norm(w - wref) / np.linalg.norm(wref))


def compare(out, ref, force_tol=FP32_FORCE_RMSE, e_tol=FP32_ENERGY_PER_ATOM, w_tol=FP32_VIRIAL_REL):
    fr = rel_force_rmse(out["forces"], ref["forces"])
    er = energy_err_per_atom(out["energy"], ref["energy"], ref["energies"])
    wr = virial_rel(out["virial"], ref["virial"])
    assert fr <= force_tol, f"relative force RMSE {fr:.3e} > {force_tol}"
    assert er <= e_tol, f"|dE|/N / rms(E_i) {er:.3e} > {e_tol}"
    assert wr <= w_tol, f"relative virial error {wr:.3e} > {w_tol}"
    return fr, er, wr


def model(F, T, S, seed=0, bias=0.0, K=20, rc=5.0, e_scale=1.0):
    vals = syn.xavier_params(F, K, T, S, seed=seed, bias_scale=bias)
    blob = syn.params_blob(F, K, T, S, rc=rc, e_scale=e_scale, values=vals)
    return vals, blob
