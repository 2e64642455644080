"""Failure detection of the buffering contract (Results, "Runtime optimizations and buffering":
inputs are buffered to capacities that only grow, and a computation that cannot be served is
reported, not silently wrong).

Every failure here is made on the host: non-finite input coordinates, a corrupt or truncated
parameter blob, an HBM budget too small for the buffers, a cell too thin for the image search.
None of them reaches a kernel in a state that could fault: non-finite positions are binned with
a clamped cell index (checked by reading the binning kernel) and then reported.  After each
failure the same context must still give the results a fresh context gives, bit for bit; a
context that computes a small, then a large, then the small system again (its buffers grown in
between) must too."""
import struct

import numpy as np
import pytest

import synthetic as syn
from gpu_common import engine, model

pytestmark = pytest.mark.gpu

F, T, S = 64, 2, 2


def _same(a, b):
    assert a["energy"] == b["energy"]
    np.testing.assert_array_equal(a["forces"], b["forces"])
    np.testing.assert_array_equal(a["virial"], b["virial"])


def _fresh(eng, blob, sy, **kw):
    with eng.Potential(F, T=T, n_species=S, params=blob, **kw) as pot:
        return pot.compute(sy.species, sy.positions, sy.cell)


@pytest.mark.parametrize("where", ["first_call", "after_a_list"])
def test_nonfinite_positions_are_reported_and_the_context_recovers(where):
    eng = engine()
    from paper_2506_04055_gb300 import _lib
    _, blob = model(F, T, S, seed=1, bias=0.1)
    sy = syn.water_box(64, seed=0)
    ref = _fresh(eng, blob, sy)
    with eng.Potential(F, T=T, n_species=S, params=blob) as pot:
        if where == "after_a_list":
            _same(pot.compute(sy.species, sy.positions, sy.cell), ref)
        for bad in (np.nan, np.inf, -np.inf):
            x = sy.positions.copy()
            x[17, 1] = bad
            with pytest.raises(eng.CtdError) as err:
                pot.compute(sy.species, x, sy.cell)
            assert err.value.code == _lib.CTD_ERR_NONFINITE
            _same(pot.compute(sy.species, sy.positions, sy.cell), ref)
        # the neighbour build and the MD state reject them too
        x = sy.positions.copy()
        x[3, 0] = np.nan
        with pytest.raises(eng.CtdError) as err:
            pot.build_neighbors(x, sy.cell)
        assert err.value.code == _lib.CTD_ERR_NONFINITE
        with pytest.raises(eng.CtdError) as err:
            pot.md_set_state(sy.species, sy.masses, x, np.zeros_like(x), sy.cell)
        assert err.value.code == _lib.CTD_ERR_NONFINITE
        _same(pot.compute(sy.species, sy.positions, sy.cell), ref)


def test_corrupt_or_truncated_parameter_blob_is_rejected():
    eng = engine()
    from paper_2506_04055_gb300 import _lib
    _, blob = model(F, T, S, seed=2)
    sy = syn.water_box(30, seed=1)
    ref = _fresh(eng, blob, sy)
    n_values = struct.unpack_from("<q", blob, 56)[0]
    bad_blobs = {
        "truncated header": blob[:40],
        "truncated values": blob[:-8],
        "bad magic": b"CTDPAINX" + blob[8:],
        "wrong value count": blob[:56] + struct.pack("<q", n_values + 1) + blob[64:],
        "header F differs from the description": blob[:12] + struct.pack("<i", 2 * F) + blob[16:],
        "non-finite weight": blob[:64] + struct.pack("<d", float("nan")) + blob[72:],
        "empty": b"",
    }
    with eng.Potential(F, T=T, n_species=S) as pot:
        with pytest.raises(eng.CtdError) as err:   # no parameters yet
            pot.compute(sy.species, sy.positions, sy.cell)
        assert err.value.code == _lib.CTD_ERR_STATE
        for what, b in bad_blobs.items():
            with pytest.raises(eng.CtdError) as err:
                pot.load_params(b)
            assert err.value.code == _lib.CTD_ERR_INVALID_ARG, what
        pot.load_params(blob)
        _same(pot.compute(sy.species, sy.positions, sy.cell), ref)
        # a bad blob after a good one leaves the good parameters in place
        with pytest.raises(eng.CtdError):
            pot.load_params(bad_blobs["wrong value count"])
        _same(pot.compute(sy.species, sy.positions, sy.cell), ref)


def test_hbm_budget_is_enforced():
    eng = engine()
    from paper_2506_04055_gb300 import _lib
    _, blob = model(F, T, S, seed=3)
    sy = syn.water_box(500, seed=2)   # 1,500 atoms: tens of MB of buffers
    with eng.Potential(F, T=T, n_species=S, params=blob, hbm_budget_bytes=2 * 1024 * 1024) as pot:
        with pytest.raises(eng.CtdError) as err:
            pot.compute(sy.species, sy.positions, sy.cell, stats=True)
        assert err.value.code == _lib.CTD_ERR_OUT_OF_BUDGET
    ref = _fresh(eng, blob, sy)
    with eng.Potential(F, T=T, n_species=S, params=blob, hbm_budget_bytes=2 * 1024 ** 3) as pot:
        out = pot.compute(sy.species, sy.positions, sy.cell, stats=True)
        assert 0 < out["stats"]["bytes_allocated"] <= 2 * 1024 ** 3
        _same(out, ref)


def test_cell_too_thin_for_the_image_search():
    eng = engine()
    from paper_2506_04055_gb300 import _lib
    _, blob = model(F, T, S, seed=4)
    sy = syn.water_box(8, seed=3)
    thin = np.diag([20.0, 20.0, 0.05])      # 0.05 A along c: the search would need 120 images
    x = sy.positions.copy()
    x[:, 2] = 0.01
    with eng.Potential(F, T=T, n_species=S, params=blob) as pot:
        with pytest.raises(eng.CtdError) as err:
            pot.compute(sy.species, x, thin)
        assert err.value.code == _lib.CTD_ERR_CELL_TOO_SMALL
        with pytest.raises(eng.CtdError) as err:
            pot.compute(sy.species, sy.positions, np.diag([20.0, 20.0, 0.0]))   # singular
        assert err.value.code == _lib.CTD_ERR_INVALID_ARG
        _same(pot.compute(sy.species, sy.positions, sy.cell), _fresh(eng, blob, sy))


@pytest.mark.parametrize("precision,width", [("fp32", 64), ("bf16", 128)])
def test_small_large_small_equals_fresh_contexts(precision, width):
    """Grow-only buffers: a context that computed a much larger system gives the small system's
    results bit for bit as a fresh context does (F = 128 BF16 runs the tensor-core kernels), and
    its statistics separate the bytes the current shapes need from the bytes held."""
    eng = engine()
    vals = syn.xavier_params(width, 20, T, S, seed=5, bias_scale=0.1)
    blob = syn.params_blob(width, 20, T, S, values=vals)
    small = syn.water_box(40, seed=4)
    large = syn.water_box(3000, seed=5)

    def fresh(sy):
        with eng.Potential(width, T=T, n_species=S, params=blob, precision=precision) as pot:
            return pot.compute(sy.species, sy.positions, sy.cell, stats=True)

    ref_small, ref_large = fresh(small), fresh(large)
    with eng.Potential(width, T=T, n_species=S, params=blob, precision=precision) as pot:
        a = pot.compute(small.species, small.positions, small.cell, stats=True)
        held_small = a["stats"]["bytes_allocated"]
        b = pot.compute(large.species, large.positions, large.cell, stats=True)
        assert b["stats"]["bytes_allocated"] > 4 * held_small     # the buffers grew
        c = pot.compute(small.species, small.positions, small.cell, stats=True)
        assert c["stats"]["bytes_allocated"] == b["stats"]["bytes_allocated"]   # and never shrink
    # bytes in use follow the current shapes; what is held above them is the growth headroom
    # (a quarter of each buffer grown, plus 256-byte rounding) and, after the large system, the
    # capacity the small one leaves unused
    for r in (a, b):
        use, held = r["stats"]["bytes_in_use"], r["stats"]["bytes_allocated"]
        assert 0 < use <= held <= 1.25 * use + (1 << 17)
    assert 0 < c["stats"]["bytes_in_use"] * 4 < b["stats"]["bytes_in_use"]
    for got, ref in ((a, ref_small), (b, ref_large), (c, ref_small)):
        _same(got, ref)


def _offset(name, F, K, S):
    off = 0
    for nm, shape in syn.param_shapes(F, K, 1, S):
        if nm == name:
            return off
        off += int(np.prod(shape))
    raise KeyError(name)


def test_fp16_storage_beyond_range_is_reported():
    """The BF16 path stores the message table (F = 128 contraction), the U/V products, the
    update coefficients and the SiLU arguments in FP16; a value beyond FP16's largest finite value
    (65504) is reported instead of turning into an Inf.  Update coefficients beyond it are reported
    on either message step; so is a message table beyond it, through the table itself where the
    contraction stores it in FP16 and through the update's SiLU argument h2 (fed by the message)
    where the CUDA-core message step keeps the FP32 table; the FP32 path computes both systems."""
    eng = engine()
    from paper_2506_04055_gb300 import _lib
    Fb, Tb, Sb, K = 128, 1, 1, 20
    sy = syn.fcc(3, 3, 3, jitter=0.05, seed=2)
    base = syn.xavier_params(Fb, K, Tb, Sb, seed=5, bias_scale=0.1)
    phi = base.copy()
    o = _offset("b2_0", Fb, K, Sb)
    phi[o:o + 3 * Fb] = 7.0e4                        # every phi channel beyond the FP16 range
    coef = base.copy()
    o = _offset("c2_0", Fb, K, Sb)
    coef[o:o + 3 * Fb] = 7.0e4                       # every update coefficient beyond it
    for vals, raises in ((phi, {1: True, 0: True}), (coef, {1: True, 0: True})):
        blob = syn.params_blob(Fb, K, Tb, Sb, values=vals)
        for msg in (1, 0):
            with eng.Potential(Fb, K=K, T=Tb, n_species=Sb, precision="bf16", params=blob) as pot:
                pot.set_option(_lib.CTD_OPT_TC_MESSAGE, msg)
                if raises[msg]:
                    with pytest.raises(eng.CtdError) as err:
                        pot.compute(sy.species, sy.positions, sy.cell)
                    assert err.value.code == _lib.CTD_ERR_NONFINITE and "FP16" in str(err.value)
                else:
                    out = pot.compute(sy.species, sy.positions, sy.cell)
                    assert np.isfinite(out["energy"]) and np.isfinite(out["forces"]).all()
        with eng.Potential(Fb, K=K, T=Tb, n_species=Sb, precision="fp32", params=blob) as pot:
            out = pot.compute(sy.species, sy.positions, sy.cell)
            assert np.isfinite(out["energy"]) and np.isfinite(out["forces"]).all()
