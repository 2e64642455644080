"""ctypes binding of the C ABI in include/painn.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  No arithmetic of the method
happens in Python: neighbour search, model, adjoint, reductions and integration all run in the
CUDA kernels of ``libctd_painn.so``.  If the library cannot be loaded, ``load()`` raises; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libctd_painn.so")

CTD_OK = 0
CTD_ERR_INVALID_ARG = -1
CTD_ERR_CAPACITY = -2
CTD_ERR_OUT_OF_BUDGET = -3
CTD_ERR_CELL_TOO_SMALL = -4
CTD_ERR_CUDA = -5
CTD_ERR_TIMEOUT = -6
CTD_ERR_NONFINITE = -7
CTD_ERR_STATE = -8
CTD_PREC_FP32 = 0
CTD_PREC_BF16 = 1
CTD_FAMILY_PAINN = 0
CTD_FAMILY_LOCAL = 1
CTD_NEED_FORCES = 1
CTD_NEED_VIRIAL = 2
CTD_REBUILD = 4
CTD_DEVICE_PTRS = 8

ERROR_NAMES = {
    CTD_ERR_INVALID_ARG: "CTD_ERR_INVALID_ARG", CTD_ERR_CAPACITY: "CTD_ERR_CAPACITY",
    CTD_ERR_OUT_OF_BUDGET: "CTD_ERR_OUT_OF_BUDGET", CTD_ERR_CELL_TOO_SMALL: "CTD_ERR_CELL_TOO_SMALL",
    CTD_ERR_CUDA: "CTD_ERR_CUDA", CTD_ERR_TIMEOUT: "CTD_ERR_TIMEOUT",
    CTD_ERR_NONFINITE: "CTD_ERR_NONFINITE", CTD_ERR_STATE: "CTD_ERR_STATE",
}

# Every symbol include/painn.h declares (checked by the CPU test suite).
EXPORTS = [
    "ctd_create", "ctd_load_params", "ctd_build_neighbors", "ctd_get_pairs", "ctd_compute",
    "ctd_set_energy_out", "ctd_md_set_state", "ctd_md_run", "ctd_md_get_state",
    "ctd_md_set_thermostat", "ctd_md_get_thermostat", "ctd_md_set_thermostat_state", "ctd_serve_snapshot",
    "ctd_serve_set_thermostat", "ctd_serve_thermostat",
    "ctd_set_option", "ctd_profile_enable", "ctd_profile_read", "ctd_gemm_bf16",
    "ctd_serve_create", "ctd_serve_submit", "ctd_serve_step", "ctd_serve_poll", "ctd_serve_stats",
    "ctd_serve_use_graph", "ctd_serve_graph_stats",
    "ctd_serve_last_error", "ctd_serve_destroy", "ctd_domains_create", "ctd_domains_compute",
    "ctd_domains_info", "ctd_domains_context", "ctd_domains_last_error", "ctd_domains_destroy",
    "ctd_neighbors_noalloc", "ctd_selftest_wait",
    "ctd_last_error",
    "ctd_destroy",
]
CTD_NOALLOC_MAX_ATOMS = 32768
CTD_NOALLOC_MAX_CELLS = 32768
CTD_NSTAGES = 8
STAGES = ["build", "prune", "node", "edge_fwd", "edge_bwd", "forces", "md", "other"]


class ctd_model_desc(ctypes.Structure):
    _fields_ = [("F", ctypes.c_int32), ("K", ctypes.c_int32), ("T", ctypes.c_int32),
                ("n_species", ctypes.c_int32), ("rc", ctypes.c_double), ("precision", ctypes.c_int32),
                ("family", ctypes.c_int32), ("channels", ctypes.c_int32)]


class ctd_stats(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int64), ("n_verlet_edges", ctypes.c_int64),
                ("n_active_edges", ctypes.c_int64), ("rebuilt", ctypes.c_int32),
                ("retries", ctypes.c_int32), ("max_displacement", ctypes.c_double),
                ("bytes_allocated", ctypes.c_int64), ("ms_neighbors", ctypes.c_float),
                ("ms_model", ctypes.c_float), ("edges_stored", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("bytes_in_use", ctypes.c_int64)]


class ctd_domain_info(ctypes.Structure):
    _fields_ = [("n_owned", ctypes.c_int64), ("n_copies", ctypes.c_int64), ("n_candidates", ctypes.c_int64),
                ("n_verlet_edges", ctypes.c_int64), ("n_active_edges", ctypes.c_int64),
                ("grid_index", ctypes.c_int32 * 3), ("reserved", ctypes.c_int32)]


class CtdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libctd_painn.so (build it first with ``paper_2506_04055_gb300.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: run paper_2506_04055_gb300.build() first")
    lib = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "ctd_create": ([P, P, ctypes.c_size_t, P], ctypes.c_int),
        "ctd_load_params": ([P, P, ctypes.c_size_t], ctypes.c_int),
        "ctd_build_neighbors": ([P, I64, P, P, D, D, I32, P], ctypes.c_int),
        "ctd_get_pairs": ([P, P, P, P, I64], ctypes.c_int),
        "ctd_compute": ([P, I64, P, P, P, I32, P, P, P, P], ctypes.c_int),
        "ctd_set_energy_out": ([P, P], ctypes.c_int),
        "ctd_md_set_state": ([P, I64, P, P, P, P, P, D], ctypes.c_int),
        "ctd_md_run": ([P, I32, D, P, P, P], ctypes.c_int),
        "ctd_md_get_state": ([P, P, P], ctypes.c_int),
        "ctd_md_set_thermostat": ([P, D, D, I32], ctypes.c_int),
        "ctd_md_get_thermostat": ([P, P, P, P], ctypes.c_int),
        "ctd_md_set_thermostat_state": ([P, P, P], ctypes.c_int),
        "ctd_serve_snapshot": ([P, I64, P, P, P], ctypes.c_int),
        "ctd_serve_set_thermostat": ([P, I64, D, D, I32, P, P], ctypes.c_int),
        "ctd_serve_thermostat": ([P, I64, P, P, P], ctypes.c_int),
        "ctd_set_option": ([P, I32, I64], ctypes.c_int),
        "ctd_profile_enable": ([P, I32], ctypes.c_int),
        "ctd_profile_read": ([P, P, P, I32], ctypes.c_int),
        "ctd_gemm_bf16": ([P, I64, I32, I32, P, I64, P, P, I64], ctypes.c_int),
        "ctd_neighbors_noalloc": ([I64, P, P, D, D, P, P, P, I64, P, P], ctypes.c_int),
        "ctd_serve_create": ([P, P, P, ctypes.c_size_t, ctypes.c_size_t, I32, D, P], ctypes.c_int),
        "ctd_serve_submit": ([P, I64, P, P, P, P, P, D, I32, P], ctypes.c_int),
        "ctd_serve_step": ([P, P, P, P], ctypes.c_int),
        "ctd_serve_poll": ([P, I64, P, P, P, P, P, P, P], ctypes.c_int),
        "ctd_serve_stats": ([P, P, P, P, P], ctypes.c_int),
        "ctd_serve_use_graph": ([P, I32], ctypes.c_int),
        "ctd_serve_graph_stats": ([P, P, P, P, P], ctypes.c_int),
        "ctd_serve_last_error": ([P], ctypes.c_char_p),
        "ctd_serve_destroy": ([P], None),
        "ctd_domains_create": ([P, P, P, ctypes.c_size_t, ctypes.c_size_t, P, I32, D, P], ctypes.c_int),
        "ctd_domains_compute": ([P, I64, P, P, P, I32, P, P, P, P], ctypes.c_int),
        "ctd_domains_info": ([P, I32, P], ctypes.c_int),
        "ctd_domains_context": ([P], P),
        "ctd_domains_last_error": ([P], ctypes.c_char_p),
        "ctd_domains_destroy": ([P], None),
        "ctd_selftest_wait": ([P, D, P], ctypes.c_int),
        "ctd_last_error": ([P], ctypes.c_char_p),
        "ctd_destroy": ([P], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(ctx, code):
    if code != CTD_OK:
        msg = load().ctd_last_error(ctx)
        raise CtdError(code, msg.decode() if msg else "")
    return code


# ---- same-name wrappers (pointers are ints or ctypes pointers) ---------------------------
def ctd_create(desc: ctd_model_desc, hbm_budget_bytes: int = 0, cuda_stream: int | None = None):
    ctx = ctypes.c_void_p()
    code = load().ctd_create(ctypes.byref(ctx), ctypes.byref(desc), hbm_budget_bytes, cuda_stream)
    if code != CTD_OK:
        raise CtdError(code, "ctd_create failed (no CUDA device or invalid model description)")
    return ctx


def ctd_load_params(ctx, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    return check(ctx, load().ctd_load_params(ctx, buf, len(blob)))


def ctd_build_neighbors(ctx, n, positions_ptr, cell_ptr, cutoff, skin, flags=0):
    out = ctypes.c_int64()
    check(ctx, load().ctd_build_neighbors(ctx, n, positions_ptr, cell_ptr, cutoff, skin, flags,
                                          ctypes.byref(out)))
    return out.value


def ctd_get_pairs(ctx, i_ptr, j_ptr, shift_ptr, cap):
    return check(ctx, load().ctd_get_pairs(ctx, i_ptr, j_ptr, shift_ptr, cap))


def ctd_compute(ctx, n, species_ptr, positions_ptr, cell_ptr, flags, energy_ptr, forces_ptr,
                virial_ptr, stats=None):
    return check(ctx, load().ctd_compute(ctx, n, species_ptr, positions_ptr, cell_ptr, flags,
                                         energy_ptr, forces_ptr, virial_ptr,
                                         ctypes.byref(stats) if stats is not None else None))


def ctd_set_energy_out(ctx, ptr):
    return check(ctx, load().ctd_set_energy_out(ctx, ptr))


def ctd_md_set_state(ctx, n, species_ptr, masses_ptr, positions_ptr, velocities_ptr, cell_ptr, skin):
    return check(ctx, load().ctd_md_set_state(ctx, n, species_ptr, masses_ptr, positions_ptr,
                                              velocities_ptr, cell_ptr, skin))


def ctd_md_run(ctx, nsteps, dt, epot_ptr, ekin_ptr):
    nreb = ctypes.c_int32()
    check(ctx, load().ctd_md_run(ctx, nsteps, dt, epot_ptr, ekin_ptr, ctypes.byref(nreb)))
    return nreb.value


def ctd_md_get_state(ctx, positions_ptr, velocities_ptr):
    return check(ctx, load().ctd_md_get_state(ctx, positions_ptr, velocities_ptr))


def ctd_md_set_thermostat(ctx, temperature, tau, chain):
    return check(ctx, load().ctd_md_set_thermostat(ctx, float(temperature), float(tau), int(chain)))


def ctd_md_get_thermostat(ctx, xi_ptr, vxi_ptr, ethermo_ptr):
    return check(ctx, load().ctd_md_get_thermostat(ctx, xi_ptr, vxi_ptr, ethermo_ptr))


def ctd_md_set_thermostat_state(ctx, xi_ptr, vxi_ptr):
    return check(ctx, load().ctd_md_set_thermostat_state(ctx, xi_ptr, vxi_ptr))


CTD_OPT_TC_ADJOINT = 1
CTD_OPT_EDGE_STORE = 2
CTD_OPT_TC_MESSAGE = 3
CTD_OPT_EDGE_CHUNK_ROWS = 4


def ctd_set_option(ctx, option, value):
    return check(ctx, load().ctd_set_option(ctx, option, value))


def ctd_profile_enable(ctx, enable: bool):
    return check(ctx, load().ctd_profile_enable(ctx, 1 if enable else 0))


def ctd_profile_read(ctx, reset: bool = True):
    ms = (ctypes.c_double * CTD_NSTAGES)()
    ln = (ctypes.c_int64 * CTD_NSTAGES)()
    check(ctx, load().ctd_profile_read(ctx, ms, ln, 1 if reset else 0))
    return {s: (ms[k], ln[k]) for k, s in enumerate(STAGES)}


def ctd_gemm_bf16(ctx, M, N, K, a_ptr, lda, b_ptr, c_ptr, ldc):
    return check(ctx, load().ctd_gemm_bf16(ctx, M, N, K, a_ptr, lda, b_ptr, c_ptr, ldc))


def ctd_neighbors_noalloc(n, positions_ptr, cell_ptr, cutoff, skin, i_ptr, j_ptr, shift_ptr, cap,
                          cuda_stream=None):
    """Returns (status code, number of pairs); never raises on CTD_ERR_CAPACITY so callers can
    size their arrays from the count."""
    npairs = ctypes.c_int64()
    code = load().ctd_neighbors_noalloc(n, positions_ptr, cell_ptr, cutoff, skin, i_ptr, j_ptr,
                                        shift_ptr, cap, ctypes.byref(npairs), cuda_stream)
    return code, npairs.value


def serve_check(srv, code):
    if code != CTD_OK:
        msg = load().ctd_serve_last_error(srv)
        raise CtdError(code, msg.decode() if msg else "")
    return code


def ctd_serve_create(desc, blob, hbm_budget_bytes=0, max_replicas=1024, dt=1.0, cuda_stream=None):
    srv = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    code = load().ctd_serve_create(ctypes.byref(srv), ctypes.byref(desc), buf, len(blob), hbm_budget_bytes,
                                   max_replicas, dt, cuda_stream)
    if code != CTD_OK:
        raise CtdError(code, "ctd_serve_create failed")
    return srv


def ctd_serve_submit(srv, n, species_ptr, masses_ptr, positions_ptr, velocities_ptr, cell_ptr, skin, nsteps):
    rid = ctypes.c_int64()
    serve_check(srv, load().ctd_serve_submit(srv, n, species_ptr, masses_ptr, positions_ptr, velocities_ptr,
                                             cell_ptr, skin, nsteps, ctypes.byref(rid)))
    return rid.value


def ctd_serve_step(srv):
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    serve_check(srv, load().ctd_serve_step(srv, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def ctd_serve_poll(srv, rid, positions_ptr=None, velocities_ptr=None, epot_ptr=None, ekin_ptr=None,
                   virial_ptr=None):
    st, done = ctypes.c_int32(), ctypes.c_int32()
    serve_check(srv, load().ctd_serve_poll(srv, rid, ctypes.byref(st), ctypes.byref(done), positions_ptr,
                                           velocities_ptr, epot_ptr, ekin_ptr, virial_ptr))
    return st.value, done.value


def ctd_serve_snapshot(srv, rid, positions_ptr, velocities_ptr):
    done = ctypes.c_int32()
    serve_check(srv, load().ctd_serve_snapshot(srv, rid, positions_ptr, velocities_ptr, ctypes.byref(done)))
    return done.value


def ctd_serve_set_thermostat(srv, rid, temperature, tau, chain, xi_ptr=None, vxi_ptr=None):
    serve_check(srv, load().ctd_serve_set_thermostat(srv, rid, temperature, tau, chain, xi_ptr, vxi_ptr))


def ctd_serve_thermostat(srv, rid, xi_ptr=None, vxi_ptr=None, eth_ptr=None):
    serve_check(srv, load().ctd_serve_thermostat(srv, rid, xi_ptr, vxi_ptr, eth_ptr))


def ctd_serve_graph_stats(srv):
    g, e, k, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    serve_check(srv, load().ctd_serve_graph_stats(srv, ctypes.byref(g), ctypes.byref(e), ctypes.byref(k),
                                                  ctypes.byref(c)))
    return {"graph_steps": g.value, "eager_steps": e.value, "kernels_per_replay": k.value, "captures": c.value}


def ctd_serve_stats(srv):
    atoms, reps, q, held = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    serve_check(srv, load().ctd_serve_stats(srv, ctypes.byref(atoms), ctypes.byref(reps), ctypes.byref(q),
                                            ctypes.byref(held)))
    return {"resident_atoms": atoms.value, "resident_replicas": reps.value, "queued": q.value,
            "bytes_held": held.value}


def ctd_serve_destroy(srv):
    load().ctd_serve_destroy(srv)


def domains_check(dom, code):
    if code != CTD_OK:
        msg = load().ctd_domains_last_error(dom)
        raise CtdError(code, msg.decode() if msg else "")
    return code


def ctd_domains_create(desc, blob, grid, hop_prune=True, skin=1.0, hbm_budget_bytes=0, cuda_stream=None):
    dom = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    g = (ctypes.c_int32 * 3)(*[int(v) for v in grid])
    code = load().ctd_domains_create(ctypes.byref(dom), ctypes.byref(desc), buf, len(blob), hbm_budget_bytes,
                                     g, 1 if hop_prune else 0, float(skin), cuda_stream)
    if code != CTD_OK:
        raise CtdError(code, "ctd_domains_create failed")
    return dom


def ctd_domains_compute(dom, n, species_ptr, positions_ptr, cell_ptr, flags, energy_ptr, forces_ptr,
                        virial_ptr, stats=None):
    return domains_check(dom, load().ctd_domains_compute(dom, n, species_ptr, positions_ptr, cell_ptr, flags,
                                                         energy_ptr, forces_ptr, virial_ptr,
                                                         ctypes.byref(stats) if stats is not None else None))


def ctd_domains_info(dom, domain):
    info = ctd_domain_info()
    domains_check(dom, load().ctd_domains_info(dom, domain, ctypes.byref(info)))
    out = {k: getattr(info, k) for k, _ in ctd_domain_info._fields_ if k not in ("grid_index", "reserved")}
    out["grid_index"] = tuple(info.grid_index)
    return out


def ctd_domains_context(dom):
    return ctypes.c_void_p(load().ctd_domains_context(dom))


def ctd_domains_destroy(dom):
    load().ctd_domains_destroy(dom)


def ctd_selftest_wait(ctx, limit_ms):
    """Returns (status code, milliseconds waited); CTD_ERR_TIMEOUT is the expected code."""
    waited = ctypes.c_double()
    code = load().ctd_selftest_wait(ctx, float(limit_ms), ctypes.byref(waited))
    return code, waited.value


def ctd_last_error(ctx) -> str:
    msg = load().ctd_last_error(ctx)
    return msg.decode() if msg else ""


def ctd_destroy(ctx):
    load().ctd_destroy(ctx)
