"""BF16 path (tcgen05 MLPs, FP32 accumulation and elementwise, FP64 reductions) vs the FP64 oracle.

Stated tolerance: relative force RMSE <= 1e-2.  Energy: |dE|/N <= 1e-2 of the RMS per-atom
energy (the energy error is reported alongside; BF16 operands carry 2^-9 relative rounding)."""
import numpy as np
import pytest

import synthetic as syn
from gpu_common import BF16_FORCE_RMSE, compare, engine, model, rel_force_rmse

pytestmark = pytest.mark.gpu


def _run(eng, orc, sy, F, T, S, bias=0.1, seed=0, tc_adjoint=None):
    vals, blob = model(F, T, S, seed=seed, bias=bias)
    with eng.Potential(F, T=T, n_species=S, precision="bf16", params=blob) as pot:
        if tc_adjoint is not None:
            from paper_2506_04055_gb300 import _lib
            pot.set_option(_lib.CTD_OPT_TC_ADJOINT, tc_adjoint)
        out = pot.compute(sy.species, sy.positions, sy.cell, energies=True)
    ref = orc.painn(vals, F, 20, T, S, sy.species, sy.positions, sy.cell)
    return out, ref


def test_bf16_water192_F64(orc):
    eng = engine()
    out, ref = _run(eng, orc, syn.water_box(64, seed=0), 64, 3, 2, bias=0.0)
    fr, er, wr = compare(out, ref, force_tol=BF16_FORCE_RMSE, e_tol=1e-2, w_tol=2e-2)
    print(f"bf16 water192: force rmse {fr:.2e}, energy {er:.2e}, virial {wr:.2e}")


def test_bf16_fcc4000_F128(orc):
    """The 10x10x10-cell (4,000-atom) fcc sub-run of the 1M-atom configuration."""
    eng = engine()
    out, ref = _run(eng, orc, syn.fcc(10, 10, 10, jitter=0.05, seed=0), 128, 3, 1, bias=0.0)
    fr, er, wr = compare(out, ref, force_tol=BF16_FORCE_RMSE, e_tol=1e-2, w_tol=2e-2)
    print(f"bf16 fcc4000: force rmse {fr:.2e}, energy {er:.2e}, virial {wr:.2e}")


@pytest.mark.parametrize("variant", [0, 1])
def test_bf16_tensor_core_adjoint(orc, variant):
    """Each edge-adjoint variant (CUDA cores with FP32 weights; tcgen05 filter with FP16 weights and
    basis) on the fcc sub-cell and a small cell; the removed option value 2 is rejected."""
    eng = engine()
    for sy in (syn.fcc(10, 10, 10, jitter=0.05, seed=0), syn.water_box(21, seed=2)):
        out, ref = _run(eng, orc, sy, 128, 3, 2, bias=0.1, tc_adjoint=variant)
        fr, er, wr = compare(out, ref, force_tol=BF16_FORCE_RMSE, e_tol=1e-2, w_tol=2e-2)
        print(f"bf16 tc-adjoint{variant} {sy.name}: force rmse {fr:.2e}, energy {er:.2e}, virial {wr:.2e}")
    from paper_2506_04055_gb300 import _lib
    with eng.Potential(128, T=1, n_species=1, precision="bf16") as pot:
        with pytest.raises(eng.CtdError):
            pot.set_option(_lib.CTD_OPT_TC_ADJOINT, 2)


def test_bf16_mixture_biases(orc):
    eng = engine()
    out, ref = _run(eng, orc, syn.mixture(n_chain=30, n_water=150, seed=1), 64, 2, 4, bias=0.2, seed=3)
    fr, er, wr = compare(out, ref, force_tol=BF16_FORCE_RMSE, e_tol=1e-2, w_tol=2e-2)
    print(f"bf16 mixture: force rmse {fr:.2e}, energy {er:.2e}, virial {wr:.2e}")


def test_bf16_small_cell_and_tails(orc):
    eng = engine()
    for sy in (syn.water_box(21, seed=2), syn.fcc(3, 3, 2, jitter=0.1, seed=3)):
        out, ref = _run(eng, orc, sy, 128, 2, 2, seed=4)
        fr, er, wr = compare(out, ref, force_tol=BF16_FORCE_RMSE, e_tol=1e-2, w_tol=2e-2)
        print(f"bf16 {sy.name}: force rmse {fr:.2e}, energy {er:.2e}, virial {wr:.2e}")


def test_bf16_vs_fp32_at_1M():
    """Full 1,000,188-atom fcc workload: BF16 forces within 1e-2 relative RMSE of the FP32 path
    (which matches the oracle to 1e-5 at every size it is checked)."""
    eng = engine()
    sy = syn.fcc(63, 63, 63, jitter=0.05, seed=0)
    _, blob = model(128, 3, 1, seed=0)
    outs = {}
    for prec in ("fp32", "bf16"):
        with eng.Potential(128, T=3, n_species=1, precision=prec, params=blob) as pot:
            outs[prec] = pot.compute(sy.species, sy.positions, sy.cell)
    fr = rel_force_rmse(outs["bf16"]["forces"], outs["fp32"]["forces"])
    assert fr <= BF16_FORCE_RMSE, fr
    print(f"bf16 vs fp32 at 1M: force rmse {fr:.2e}")


def test_bf16_rejects_unsupported_width():
    eng = engine()
    with pytest.raises(eng.CtdError):
        eng.Potential(32, T=1, n_species=1, precision="bf16")


def _sparse_system():
    """A 30 A cubic cell with a dense water cluster (rows of 40-70 edges: several 16-edge steps)
    and three isolated atoms (rows without edges)."""
    w = syn.water_box(40, seed=6)
    x = np.concatenate([w.positions, [[25.0, 25.0, 25.0], [25.0, 12.0, 25.0], [12.0, 25.0, 25.0]]])
    z = np.concatenate([w.species, [0, 1, 0]]).astype(np.int32)
    m = np.concatenate([w.masses, [16.0, 1.0, 16.0]])
    return syn.System(x, z, m, np.eye(3) * 30.0, name="sparse")


@pytest.mark.parametrize("message", [0, 1])
def test_bf16_message_variants(orc, message):
    """Message step on CUDA cores with the FP32 filter (0) or as the tensor-core contraction over
    each receiver's edges (1: FP16 message rows x basis, FP32 filter weights per receiver), on
    the fcc sub-cell, a small water cell, a 4-species mixture with filter biases, and a sparse
    cell with isolated atoms and rows spanning several 16-edge steps."""
    from paper_2506_04055_gb300 import _lib
    eng = engine()
    cases = ((syn.fcc(10, 10, 10, jitter=0.05, seed=0), 1, 0.1), (syn.water_box(21, seed=2), 2, 0.1),
             (syn.mixture(n_chain=30, n_water=150, seed=1), 4, 0.2), (_sparse_system(), 2, 0.1))
    for sy, S, bias in cases:
        vals, blob = model(128, 2, S, seed=5, bias=bias)
        with eng.Potential(128, T=2, n_species=S, precision="bf16", params=blob) as pot:
            pot.set_option(_lib.CTD_OPT_TC_MESSAGE, message)
            out = pot.compute(sy.species, sy.positions, sy.cell, energies=True)
        ref = orc.painn(vals, 128, 20, 2, S, sy.species, sy.positions, sy.cell)
        fr, er, wr = compare(out, ref, force_tol=BF16_FORCE_RMSE, e_tol=1e-2, w_tol=2e-2)
        print(f"bf16 message{message} {sy.name}: force rmse {fr:.2e}, energy {er:.2e}, virial {wr:.2e}")
