"""Serving loop: continuous batching of independent MD replicas (ctd_serve_*).

Checks: a replica's trajectory is bit-identical alone and in a mix of other replicas admitted
at other times; it agrees with the single-system resident MD loop (ctd_md_run); admission
respects the HBM budget; finished replicas return their final state in the caller's order."""
import numpy as np
import pytest

import synthetic as syn
from gpu_common import engine, model

pytestmark = pytest.mark.gpu

F, T, S = 64, 2, 3
DT = 0.5


def _replicas():
    w = syn.water_box(64, seed=0)
    f = syn.fcc(3, 3, 3, jitter=0.05, seed=1)
    f.species[:] = 2
    small = syn.water_box(21, seed=2)
    g = syn.fcc(2, 2, 2, jitter=0.05, seed=3)
    g.species[:] = 2
    out = []
    for k, sy in enumerate((w, f, small, g)):
        v = syn.maxwell_boltzmann(sy.masses, 300.0, seed=10 + k)
        out.append((sy, v))
    return out


def _run_server(eng, blob, items, nsteps, precision, stagger=0, budget=0, max_replicas=64):
    srv = eng.Server(F, blob, T=T, n_species=S, precision=precision, dt=DT, hbm_budget_bytes=budget,
                     max_replicas=max_replicas)
    ids = []
    late = items[:stagger] if stagger else []
    first = items[stagger:] if stagger else items
    for sy, v in first:
        ids.append(srv.submit(sy.species, sy.masses, sy.positions, v, sy.cell, nsteps, skin=1.0))
    steps = 0
    max_res = 0
    while True:
        if stagger and steps == 3:
            for sy, v in late:
                ids.append(srv.submit(sy.species, sy.masses, sy.positions, v, sy.cell, nsteps, skin=1.0))
        res, adm, fin = srv.step()
        max_res = max(max_res, res)
        steps += 1
        if all(srv.poll(i)["state"] == 2 for i in ids) and (not stagger or steps > 3):
            break
        assert steps < 10 * nsteps + 50
    results = {i: srv.poll(i) for i in ids}
    srv.close()
    return ids, results, max_res


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_alone_equals_mixed(precision):
    eng = engine()
    _, blob = model(F, T, S, seed=4, bias=0.1)
    items = _replicas()
    a = items[0]
    ids1, r1, _ = _run_server(eng, blob, [a], 12, precision)
    # the same replica submitted late, into a batch that already runs three others
    ids2, r2, _ = _run_server(eng, blob, [a] + items[1:], 12, precision, stagger=1)
    alone, mixed = r1[ids1[0]], r2[ids2[-1]]
    np.testing.assert_array_equal(alone["epot"], mixed["epot"])
    np.testing.assert_array_equal(alone["positions"], mixed["positions"])
    np.testing.assert_array_equal(alone["velocities"], mixed["velocities"])
    assert np.isfinite(alone["epot"]).all() and alone["steps_done"] == 12


def test_matches_single_system_md():
    eng = engine()
    _, blob = model(F, T, S, seed=5, bias=0.1)
    sy, v = _replicas()[1]
    ids, res, _ = _run_server(eng, blob, [(sy, v)], 15, "fp32")
    r = res[ids[0]]
    with eng.Potential(F, T=T, n_species=S, params=blob) as pot:
        pot.md_set_state(sy.species, sy.masses, sy.positions, v, sy.cell, skin=1.0)
        ep, ek, _ = pot.md_run(15, DT)
        x, vv = pot.md_get_state()
    np.testing.assert_allclose(r["positions"], x, rtol=0, atol=1e-9)
    np.testing.assert_allclose(r["velocities"], vv, rtol=0, atol=1e-9)
    np.testing.assert_allclose(r["epot"], ep, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(r["ekin"], ek, rtol=1e-9, atol=1e-12)


def test_budget_limits_residency():
    eng = engine()
    _, blob = model(F, T, S, seed=6)
    items = _replicas() * 3
    # budget for roughly two of the larger replicas at a time
    ids, res, max_res = _run_server(eng, blob, items, 4, "fp32", budget=200 * 1024 * 1024, max_replicas=3)
    assert max_res <= 3
    assert all(res[i]["state"] == 2 and res[i]["steps_done"] == 4 for i in ids)


def test_alone_equals_mixed_tensor_core_F128():
    """F = 128 on the BF16 path runs the tensor-core edge kernels, whose row chunks span replica
    boundaries in the batched system: a replica's trajectory must still not depend on its
    neighbours in the batch."""
    eng = engine()
    Fw, Tw, Sw = 128, 2, 3
    vals = syn.xavier_params(Fw, 20, Tw, Sw, seed=7, bias_scale=0.1)
    blob = syn.params_blob(Fw, 20, Tw, Sw, values=vals)
    items = _replicas()

    def run(subset, stagger):
        srv = eng.Server(Fw, blob, T=Tw, n_species=Sw, precision="bf16", dt=DT)
        ids = []
        for k, (sy, v) in enumerate(subset):
            if k < len(subset) - stagger:
                ids.append(srv.submit(sy.species, sy.masses, sy.positions, v, sy.cell, 6, skin=1.0))
        for step in range(40):
            if stagger and step == 2:
                sy, v = subset[-1]
                ids.append(srv.submit(sy.species, sy.masses, sy.positions, v, sy.cell, 6, skin=1.0))
            srv.step()
            if all(srv.poll(i)["state"] == 2 for i in ids) and (not stagger or step >= 2):
                break
        out = srv.poll(ids[-1])
        srv.close()
        return out

    alone = run([items[0]], 0)
    mixed = run(items[1:] + [items[0]], 1)
    assert alone["state"] == 2 and mixed["state"] == 2
    np.testing.assert_array_equal(alone["epot"], mixed["epot"])
    np.testing.assert_array_equal(alone["positions"], mixed["positions"])


def test_snapshot_restart_continues_trajectory():
    """A checkpoint of a resident replica, resubmitted with the remaining steps to a new server,
    continues the trajectory (the new server builds its own neighbour list, so agreement is to
    FP32 summation order, not bit for bit)."""
    eng = engine()
    _, blob = model(F, T, S, seed=8, bias=0.1)
    sy, v = _replicas()[0]
    N, K = 20, 8
    ids, res, _ = _run_server(eng, blob, [(sy, v)], N, "fp32")
    ref = res[ids[0]]
    srv = eng.Server(F, blob, T=T, n_species=S, precision="fp32", dt=DT)
    rid = srv.submit(sy.species, sy.masses, sy.positions, v, sy.cell, N, skin=1.0)
    with pytest.raises(eng.CtdError):
        srv.snapshot(rid)   # still queued
    for _ in range(K + 1):  # the first step evaluates the initial forces without moving
        srv.step()
    snap = srv.snapshot(rid)
    assert snap["steps_done"] == K
    srv.step()              # the replica keeps running after a snapshot
    assert srv.poll(rid)["steps_done"] == K + 1
    srv.close()
    srv2 = eng.Server(F, blob, T=T, n_species=S, precision="fp32", dt=DT)
    rid2 = srv2.submit(sy.species, sy.masses, snap["positions"], snap["velocities"], sy.cell, N - K, skin=1.0)
    for _ in range(N - K + 5):
        if srv2.poll(rid2)["state"] == 2:
            break
        srv2.step()
    out = srv2.poll(rid2)
    assert out["state"] == 2
    with pytest.raises(eng.CtdError):
        srv2.snapshot(rid2)  # finished: poll has the final state
    srv2.close()
    np.testing.assert_allclose(out["positions"], ref["positions"], rtol=0, atol=1e-6)
    np.testing.assert_allclose(out["velocities"], ref["velocities"], rtol=0, atol=1e-7)
    np.testing.assert_allclose(out["epot"][: N - K + 1], ref["epot"][K : N + 1], rtol=0, atol=1e-5)


# ---- Nose-Hoover chain thermostat on served replicas (NVT) ----------------------------------

NVT = (500.0, 25.0, 3)   # target temperature (K), tau (fs), chain length


def _run_nvt_server(eng, blob, items, thermos, nsteps, late=0):
    """Serve items (the last `late` of them submitted after three steps), each with its
    thermostat (None: NVE); returns poll() and thermostat() results in submission order."""
    srv = eng.Server(F, blob, T=T, n_species=S, precision="fp32", dt=DT)
    ids = []

    def submit(k):
        sy, v = items[k]
        rid = srv.submit(sy.species, sy.masses, sy.positions, v, sy.cell, nsteps, skin=1.0)
        if thermos[k] is not None:
            srv.set_thermostat(rid, *thermos[k])
        ids.append(rid)

    for k in range(len(items) - late):
        submit(k)
    for step in range(10 * nsteps + 50):
        if late and step == 3:
            for k in range(len(items) - late, len(items)):
                submit(k)
        srv.step()
        if all(srv.poll(i)["state"] == 2 for i in ids) and (not late or step >= 3):
            break
    out = []
    for k, i in enumerate(ids):
        r = srv.poll(i)
        if thermos[k] is not None:
            r.update(srv.thermostat(i))
        out.append(r)
    srv.close()
    return out


def test_nvt_replica_matches_single_system_md():
    """A served replica with a Nose-Hoover chain follows ctd_md_run's NVT trajectory (the two
    reduce the kinetic energy in different orders: agreement to rounding)."""
    eng = engine()
    _, blob = model(F, T, S, seed=9, bias=0.1)
    sy, v = _replicas()[0]
    r = _run_nvt_server(eng, blob, [(sy, v)], [NVT], 30)[0]
    with eng.Potential(F, T=T, n_species=S, params=blob) as pot:
        pot.md_set_state(sy.species, sy.masses, sy.positions, v, sy.cell, skin=1.0)
        pot.md_set_thermostat(*NVT)
        ep, ek, _ = pot.md_run(30, DT)
        xi, vxi, eth = pot.md_get_thermostat(30)
        x, vv = pot.md_get_state()
    assert r["state"] == 2 and r["steps_done"] == 30
    assert np.abs(vxi).max() > 1e-4          # the chain moved
    np.testing.assert_allclose(r["positions"], x, rtol=0, atol=1e-9)
    np.testing.assert_allclose(r["velocities"], vv, rtol=0, atol=1e-9)
    np.testing.assert_allclose(r["epot"], ep, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(r["ekin"], ek, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(r["ethermo"], eth, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(r["xi"], xi, rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(r["vxi"], vxi, rtol=1e-9, atol=1e-15)


def test_nvt_alone_equals_mixed():
    """Thermostatted and plain replicas share the batch: each one's trajectory (and chain) is
    bit-identical to its run alone, whatever the mix and admission time."""
    eng = engine()
    _, blob = model(F, T, S, seed=10, bias=0.1)
    items = _replicas()
    hot = (800.0, 15.0, 2)
    alone_nvt = _run_nvt_server(eng, blob, [items[0]], [NVT], 12)[0]
    alone_nve = _run_nvt_server(eng, blob, [items[1]], [None], 12)[0]
    mixed = _run_nvt_server(eng, blob, [items[1], items[2], items[3], items[0]], [None, hot, None, NVT], 12, late=1)
    for a, b in ((alone_nvt, mixed[3]), (alone_nve, mixed[0])):
        for key in ("epot", "ekin", "positions", "velocities"):
            np.testing.assert_array_equal(a[key], b[key])
    for key in ("ethermo", "xi", "vxi"):
        np.testing.assert_array_equal(alone_nvt[key], mixed[3][key])
    assert np.isfinite(mixed[1]["ethermo"]).all() and np.abs(mixed[1]["vxi"]).max() > 0.0


def test_nvt_checkpoint_restart():
    """Snapshot and chain state of a resident NVT replica, resubmitted with the remaining steps
    and the saved chain, continue its trajectory (new neighbour list: agreement to FP32
    summation order)."""
    eng = engine()
    _, blob = model(F, T, S, seed=11, bias=0.1)
    sy, v = _replicas()[0]
    N, K = 20, 8
    ref = _run_nvt_server(eng, blob, [(sy, v)], [NVT], N)[0]
    srv = eng.Server(F, blob, T=T, n_species=S, precision="fp32", dt=DT)
    rid = srv.submit(sy.species, sy.masses, sy.positions, v, sy.cell, N, skin=1.0)
    srv.set_thermostat(rid, *NVT)
    for _ in range(K + 1):
        srv.step()
    snap = srv.snapshot(rid)
    chain = srv.thermostat(rid)
    with pytest.raises(eng.CtdError):
        srv.set_thermostat(rid, *NVT)   # resident: the thermostat is fixed
    srv.close()
    assert snap["steps_done"] == K and np.abs(chain["vxi"]).max() > 1e-5
    srv2 = eng.Server(F, blob, T=T, n_species=S, precision="fp32", dt=DT)
    rid2 = srv2.submit(sy.species, sy.masses, snap["positions"], snap["velocities"], sy.cell, N - K, skin=1.0)
    srv2.set_thermostat(rid2, *NVT, xi=chain["xi"], vxi=chain["vxi"])
    for _ in range(N - K + 5):
        if srv2.poll(rid2)["state"] == 2:
            break
        srv2.step()
    out = srv2.poll(rid2)
    out.update(srv2.thermostat(rid2))
    srv2.close()
    assert out["state"] == 2
    np.testing.assert_allclose(out["positions"], ref["positions"], rtol=0, atol=1e-6)
    np.testing.assert_allclose(out["velocities"], ref["velocities"], rtol=0, atol=1e-7)
    np.testing.assert_allclose(out["xi"], ref["xi"], rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(out["vxi"], ref["vxi"], rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(out["ethermo"][: N - K + 1], ref["ethermo"][K : N + 1], rtol=0, atol=1e-6)


def test_serve_thermostat_arguments_are_checked():
    eng = engine()
    _, blob = model(F, T, S, seed=12)
    sy, v = _replicas()[2]
    with eng.Server(F, blob, T=T, n_species=S, dt=DT) as srv:
        rid = srv.submit(sy.species, sy.masses, sy.positions, v, sy.cell, 2, skin=1.0)
        for bad in ((300.0, 100.0, 17), (0.0, 100.0, 3), (300.0, -1.0, 3), (float("nan"), 100.0, 3)):
            with pytest.raises(eng.CtdError):
                srv.set_thermostat(rid, *bad)
        with pytest.raises(eng.CtdError):
            srv.set_thermostat(rid, 300.0, 100.0, 2, xi=[0.0, float("inf")], vxi=[0.0, 0.0])
        with pytest.raises(eng.CtdError):
            srv.thermostat(rid)             # no thermostat
        one = srv.submit(sy.species[:1], sy.masses[:1], sy.positions[:1], v[:1], sy.cell, 2, skin=1.0)
        with pytest.raises(eng.CtdError):
            srv.set_thermostat(one, 300.0, 100.0, 3)   # a single atom has no thermal degrees of freedom
        srv.set_thermostat(rid, 300.0, 100.0, 3)
        srv.set_thermostat(rid, 300.0, 100.0, 0)       # back to NVE while queued
        with pytest.raises(eng.CtdError):
            srv.thermostat(rid)


def test_buffer_regrowth_mid_run_leaves_trajectories_unchanged():
    """Grow-only buffers shared by the batch (Results, "Runtime optimizations and buffering":
    nearly full buffers grow together).  A 6,000-atom replica admitted after three steps makes
    every batch buffer of the server grow; the two small replicas resident before and after the
    growth keep trajectories bit-identical to a server that never grew."""
    eng = engine()
    _, blob = model(F, T, S, seed=13, bias=0.1)
    items = _replicas()
    small = [items[2], items[1]]
    big = syn.water_box(2000, seed=14)
    vbig = syn.maxwell_boltzmann(big.masses, 300.0, seed=15)

    def run(with_big):
        srv = eng.Server(F, blob, T=T, n_species=S, precision="fp32", dt=DT)
        ids = [srv.submit(sy.species, sy.masses, sy.positions, v, sy.cell, 12, skin=1.0) for sy, v in small]
        held = []
        for step in range(40):
            if with_big and step == 3:
                held.append(srv.stats()["bytes_held"])
                srv.submit(big.species, big.masses, big.positions, vbig, big.cell, 4, skin=1.0)
            srv.step()
            if with_big and step == 3:
                held.append(srv.stats()["bytes_held"])
            if all(srv.poll(i)["state"] == 2 for i in ids) and step > 4:
                break
        out = [srv.poll(i) for i in ids]
        srv.close()
        return out, held

    grown, held = run(True)
    plain, _ = run(False)
    assert held[1] > 2 * held[0], held          # the admission regrew the batch buffers
    for a, b in zip(grown, plain):
        assert a["state"] == 2 and a["steps_done"] == 12
        for key in ("epot", "ekin", "positions", "velocities", "virial"):
            np.testing.assert_array_equal(a[key], b[key])


@pytest.mark.parametrize("precision,Fw", [("fp32", 64), ("bf16", 128)])
def test_graph_replay_equals_eager(precision, Fw):
    """A step's device work replayed as a CUDA graph gives the trajectories of eager steps bit
    for bit, across an admission, retirements and a Nose-Hoover replica; replays happen (the
    layout holds between those events) and launch the whole model per replay."""
    eng = engine()
    vals = syn.xavier_params(Fw, 20, T, S, seed=9, bias_scale=0.1)
    blob = syn.params_blob(Fw, 20, T, S, values=vals)
    items = _replicas()

    def run(graph):
        srv = eng.Server(Fw, blob, T=T, n_species=S, precision=precision, dt=DT)
        srv.use_graph(graph)
        ids = [srv.submit(sy.species, sy.masses, sy.positions, v, sy.cell, 20 if k != 1 else 12, skin=1.0)
               for k, (sy, v) in enumerate(items[:3])]
        srv.set_thermostat(ids[1], 400.0, 20.0, 2)
        for step in range(80):
            if step == 6:
                sy, v = items[3]
                ids.append(srv.submit(sy.species, sy.masses, sy.positions, v, sy.cell, 10, skin=1.0))
            srv.step()
            if len(ids) == 4 and all(srv.poll(i)["state"] == 2 for i in ids):
                break
        res = [srv.poll(i) for i in ids]
        gs = srv.graph_stats()
        srv.close()
        return res, gs

    ra, ga = run(True)
    rb, gb = run(False)
    assert gb["graph_steps"] == 0 and ga["graph_steps"] >= 10 and ga["kernels_per_replay"] > 20, ga
    for a, b in zip(ra, rb):
        assert a["state"] == 2 and b["state"] == 2
        np.testing.assert_array_equal(a["epot"], b["epot"])
        np.testing.assert_array_equal(a["positions"], b["positions"])
        np.testing.assert_array_equal(a["velocities"], b["velocities"])
