"""GB300 engine for a PaiNN-form semi-local potential (arXiv 2506.04055, chemtrain-deploy):
energy, forces and virial over a periodic neighbour graph, plus a resident NVE loop.

The compute path is the CUDA library ``libctd_painn.so`` (sm_103a) behind the C ABI in
``include/painn.h``; this package only marshals arguments.  ``Potential`` wraps one context;
``PaiNNEnergy`` is the ``torch.autograd.Function`` whose backward returns -grad_E * forces
from the library's hand-written adjoint.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (CTD_DEVICE_PTRS, CTD_FAMILY_LOCAL, CTD_FAMILY_PAINN, CTD_NEED_FORCES,  # noqa: F401
                   CTD_NEED_VIRIAL, CTD_PREC_BF16, CTD_PREC_FP32, CTD_REBUILD, CtdError, ctd_model_desc,
                   ctd_stats)

_FAMILIES = {"painn": CTD_FAMILY_PAINN, "local": CTD_FAMILY_LOCAL}

__all__ = ["Potential", "Server", "Domains", "PaiNNEnergy", "CtdError", "build", "load"]


def build(force: bool = False) -> str:
    from .buildlib import build as _build
    return _build(force=force)


def load():
    return _lib.load()


def _is_torch_cuda(a) -> bool:
    try:
        import torch
    except ImportError:
        return False
    return isinstance(a, torch.Tensor) and a.is_cuda


def _host(a, dtype, shape=None):
    a = np.ascontiguousarray(a, dtype=dtype)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())


def _compute(call, ctx, species, positions, cell, forces, virial, rebuild, stats, energies):
    """Marshal one energy / forces / virial call: numpy -> host pointers, CUDA torch tensors ->
    device pointers; ``call(n, z, x, H, flags, E, F, W, stats)`` runs the C entry point and
    ``ctx`` is the context whose per-atom energy output is set around it."""
    H = _host(cell, np.float64, (3, 3))
    flags = (CTD_NEED_FORCES if forces else 0) | (CTD_NEED_VIRIAL if virial else 0)
    flags |= CTD_REBUILD if rebuild else 0
    st = ctd_stats() if stats else None
    if _is_torch_cuda(positions):
        import torch
        dev = positions.device
        x = positions.detach().to(torch.float64).contiguous()
        z = species.to(device=dev, dtype=torch.int32).contiguous()
        n = int(x.shape[0])
        E = torch.zeros(1, dtype=torch.float64, device=dev)
        Fo = torch.empty((n, 3), dtype=torch.float64, device=dev) if forces else None
        W = torch.empty((3, 3), dtype=torch.float64, device=dev) if virial else None
        Ea = torch.empty(n, dtype=torch.float64, device=dev) if energies else None
        flags |= CTD_DEVICE_PTRS
        # inputs were produced on torch's stream; the context runs on its own stream
        torch.cuda.current_stream(dev).synchronize()
    else:
        x = _host(positions, np.float64, (-1, 3))
        z = _host(species, np.int32)
        n = int(x.shape[0])
        E = np.zeros(1)
        Fo = np.empty((n, 3)) if forces else None
        W = np.empty((3, 3)) if virial else None
        Ea = np.empty(n) if energies else None
    _lib.ctd_set_energy_out(ctx, _ptr(Ea))
    try:
        call(n, _ptr(z), _ptr(x), _ptr(H), flags, _ptr(E), _ptr(Fo), _ptr(W), st)
    finally:
        _lib.ctd_set_energy_out(ctx, None)
    out = {"energy": E if flags & CTD_DEVICE_PTRS else float(E[0]), "forces": Fo, "virial": W}
    if energies:
        out["energies"] = Ea
    if stats:
        out["stats"] = {k: getattr(st, k) for k, _ in ctd_stats._fields_}
    return out


class Potential:
    """One engine context: model description, parameters, neighbour list, MD state.

    precision: "fp32" (all products in FP32) or "bf16" (tensor-core MLPs, FP32 accumulation).
    params: the blob of ``synthetic.params_blob`` (64-byte header + float64 weights).
    family: "painn" (message passing, T layers) or "local" (strictly local equivariant edge
    model, T layers, ``channels`` equivariant channels, FP32; blob of ``synthetic.local_params_blob``).
    stream: a CUDA stream handle (int) or None for a stream owned by the context.
    """

    def __init__(self, F: int, K: int = 20, T: int = 3, n_species: int = 2, rc: float = 5.0,
                 precision: str = "fp32", params: bytes | None = None, hbm_budget_bytes: int = 0,
                 stream: int | None = None, family: str = "painn", channels: int = 0):
        prec = {"fp32": CTD_PREC_FP32, "bf16": CTD_PREC_BF16}[precision]
        self.desc = ctd_model_desc(F, K, T, n_species, rc, prec, _FAMILIES[family], channels)
        self.F, self.K, self.T, self.S, self.rc, self.precision = F, K, T, n_species, rc, precision
        self.ctx = _lib.ctd_create(self.desc, hbm_budget_bytes, stream)
        if params is not None:
            self.load_params(params)

    # -- lifetime ------------------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            _lib.ctd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- parameters and neighbours ----------------------------------------------------------
    def load_params(self, blob: bytes):
        _lib.ctd_load_params(self.ctx, blob)

    def set_option(self, option: int, value: int):
        _lib.ctd_set_option(self.ctx, option, value)

    def build_neighbors(self, positions, cell, cutoff: float | None = None, skin: float = 1.0) -> int:
        cutoff = self.rc if cutoff is None else cutoff
        H = _host(cell, np.float64, (3, 3))
        if _is_torch_cuda(positions):
            x = positions.contiguous()
            flags = CTD_DEVICE_PTRS
        else:
            x = _host(positions, np.float64, (-1, 3))
            flags = 0
        return _lib.ctd_build_neighbors(self.ctx, int(x.shape[0]), _ptr(x), _ptr(H), float(cutoff),
                                        float(skin), flags)

    def get_pairs(self, n_pairs: int):
        i = np.empty(n_pairs, np.int32)
        j = np.empty(n_pairs, np.int32)
        s = np.empty((n_pairs, 3), np.int8)
        _lib.ctd_get_pairs(self.ctx, _ptr(i), _ptr(j), _ptr(s), n_pairs)
        return i, j, s

    # -- energy / forces / virial ----------------------------------------------------------
    def compute(self, species, positions, cell, forces: bool = True, virial: bool = True,
                rebuild: bool = False, stats: bool = False, energies: bool = False):
        """Energy (eV), forces [n,3] (eV/A), virial [3,3] (eV).  numpy inputs -> numpy outputs
        (host pointers through the ABI); CUDA torch tensors -> CUDA torch tensors (device
        pointers, the context's stream)."""
        def call(n, z, x, H, flags, E, Fo, W, st):
            _lib.ctd_compute(self.ctx, n, z, x, H, flags, E, Fo, W, st)
        return _compute(call, self.ctx, species, positions, cell, forces, virial, rebuild, stats, energies)

    # -- launch accounting ------------------------------------------------------------------
    def profile(self, enable: bool = True):
        _lib.ctd_profile_enable(self.ctx, enable)

    def profile_read(self, reset: bool = True):
        """{stage: (device ms, launches)} since the last reset."""
        return _lib.ctd_profile_read(self.ctx, reset)

    # -- molecular dynamics ----------------------------------------------------------------
    def md_set_state(self, species, masses, positions, velocities, cell, skin: float = 1.0):
        z = _host(species, np.int32)
        m = _host(masses, np.float64)
        x = _host(positions, np.float64, (-1, 3))
        v = _host(velocities, np.float64, (-1, 3))
        H = _host(cell, np.float64, (3, 3))
        self._md_n = x.shape[0]
        _lib.ctd_md_set_state(self.ctx, x.shape[0], _ptr(z), _ptr(m), _ptr(x), _ptr(v), _ptr(H),
                              float(skin))

    def md_run(self, nsteps: int, dt: float):
        """Run nsteps velocity-Verlet steps on the device.  Returns (epot, ekin, n_rebuilds)."""
        ep = np.empty(nsteps + 1)
        ek = np.empty(nsteps + 1)
        nreb = _lib.ctd_md_run(self.ctx, nsteps, float(dt), _ptr(ep), _ptr(ek))
        return ep, ek, nreb

    def md_get_state(self):
        x = np.empty((self._md_n, 3))
        v = np.empty((self._md_n, 3))
        _lib.ctd_md_get_state(self.ctx, _ptr(x), _ptr(v))
        return x, v

    def md_set_thermostat(self, temperature: float, tau: float, chain: int = 3):
        """Nose-Hoover chain NVT for md_run (temperature in K, tau in fs; chain=0: NVE)."""
        _lib.ctd_md_set_thermostat(self.ctx, temperature, tau, chain)
        self._chain = int(chain)

    def md_set_thermostat_state(self, xi, vxi):
        """Restore a chain state saved with md_get_thermostat (after md_set_state and
        md_set_thermostat), to continue a checkpointed NVT trajectory."""
        _lib.ctd_md_set_thermostat_state(self.ctx, _ptr(_host(xi, np.float64)), _ptr(_host(vxi, np.float64)))

    def md_get_thermostat(self, nsteps: int | None = None):
        """(xi, vxi, chain energy after each step of the last md_run of nsteps steps)."""
        M = getattr(self, "_chain", 0)
        xi, vxi = np.empty(M), np.empty(M)
        eth = np.empty(nsteps + 1) if nsteps is not None else None
        _lib.ctd_md_get_thermostat(self.ctx, _ptr(xi), _ptr(vxi), _ptr(eth))
        return xi, vxi, eth


class Server:
    """Continuous-batching MD server (see ctd_serve_* in include/painn.h).

    submit() queues a replica, step() advances every resident replica by one velocity-Verlet
    step (admitting and retiring between steps), poll() returns a request's state and results."""

    def __init__(self, F: int, params: bytes, K: int = 20, T: int = 3, n_species: int = 2, rc: float = 5.0,
                 precision: str = "fp32", hbm_budget_bytes: int = 0, max_replicas: int = 1024, dt: float = 1.0,
                 stream: int | None = None, family: str = "painn", channels: int = 0):
        prec = {"fp32": CTD_PREC_FP32, "bf16": CTD_PREC_BF16}[precision]
        self.desc = ctd_model_desc(F, K, T, n_species, rc, prec, _FAMILIES[family], channels)
        self.srv = _lib.ctd_serve_create(self.desc, params, hbm_budget_bytes, max_replicas, dt, stream)
        self._n = {}
        self._steps = {}
        self._chain = {}

    def close(self):
        if getattr(self, "srv", None):
            _lib.ctd_serve_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, species, masses, positions, velocities, cell, nsteps: int, skin: float = 1.0) -> int:
        z = _host(species, np.int32)
        m = _host(masses, np.float64)
        x = _host(positions, np.float64, (-1, 3))
        v = _host(velocities, np.float64, (-1, 3))
        H = _host(cell, np.float64, (3, 3))
        rid = _lib.ctd_serve_submit(self.srv, x.shape[0], _ptr(z), _ptr(m), _ptr(x), _ptr(v), _ptr(H),
                                    float(skin), int(nsteps))
        self._n[rid] = x.shape[0]
        self._steps[rid] = int(nsteps)
        return rid

    def step(self):
        """Returns (resident replicas, admitted, finished)."""
        return _lib.ctd_serve_step(self.srv)

    def poll(self, rid: int):
        n, ns = self._n[rid], self._steps[rid]
        x = np.empty((n, 3))
        v = np.empty((n, 3))
        ep = np.full(ns + 1, np.nan)
        ek = np.full(ns + 1, np.nan)
        w = np.empty((3, 3))
        state, done = _lib.ctd_serve_poll(self.srv, rid, _ptr(x), _ptr(v), _ptr(ep), _ptr(ek), _ptr(w))
        out = {"state": state, "steps_done": done, "epot": ep, "ekin": ek, "virial": w}
        if state == 2:
            out["positions"], out["velocities"] = x, v
        return out

    def snapshot(self, rid: int):
        """Current positions, velocities and steps done of a resident replica (a checkpoint);
        submitting them with the remaining steps continues its trajectory."""
        n = self._n[rid]
        x = np.empty((n, 3))
        v = np.empty((n, 3))
        done = _lib.ctd_serve_snapshot(self.srv, rid, _ptr(x), _ptr(v))
        return {"positions": x, "velocities": v, "steps_done": done}

    def set_thermostat(self, rid: int, temperature: float, tau: float, chain: int = 3, xi=None, vxi=None):
        """Nose-Hoover chain for a queued request (chain 0: NVE); xi / vxi restore a saved chain."""
        if (xi is None) != (vxi is None):
            raise ValueError("give both xi and vxi, or neither")
        a = b = None
        if xi is not None:
            a = _host(xi, np.float64)
            b = _host(vxi, np.float64)
            if a.shape != (chain,) or b.shape != (chain,):
                raise ValueError("xi and vxi need one value per thermostat")
        _lib.ctd_serve_set_thermostat(self.srv, rid, float(temperature), float(tau), int(chain),
                                      _ptr(a) if a is not None else None, _ptr(b) if b is not None else None)
        self._chain[rid] = int(chain)

    def thermostat(self, rid: int):
        """Chain state (xi, vxi) and the chain energy recorded with each step of a request."""
        M, ns = self._chain.get(rid, 0), self._steps[rid]
        xi = np.empty(max(M, 1))
        vxi = np.empty(max(M, 1))
        eth = np.full(ns + 1, np.nan)
        _lib.ctd_serve_thermostat(self.srv, rid, _ptr(xi), _ptr(vxi), _ptr(eth))
        return {"xi": xi[:M], "vxi": vxi[:M], "ethermo": eth}

    def stats(self):
        return _lib.ctd_serve_stats(self.srv)

    def use_graph(self, enable: bool = True):
        """Record and replay each step's device work as a CUDA graph (default on)."""
        _lib.serve_check(self.srv, _lib.load().ctd_serve_use_graph(self.srv, 1 if enable else 0))

    def graph_stats(self):
        """Steps run by graph replay and eagerly, kernels per replay, graphs recorded."""
        return _lib.ctd_serve_graph_stats(self.srv)


class Domains:
    """Spatial domain decomposition of one periodic system (see ctd_domains_* in
    include/painn.h): grid = (p0, p1, p2) domains, each with copies of the atoms within
    T rc + skin of its box; copies more than T hops from the domain's own atoms are dropped when
    hop_prune is set.  compute() returns what Potential.compute returns, from the summed domain
    energies and the summed partial forces of each atom's copies; info() the per-domain counts."""

    def __init__(self, F: int, params: bytes, grid=(2, 2, 2), K: int = 20, T: int = 3, n_species: int = 2,
                 rc: float = 5.0, precision: str = "fp32", hop_prune: bool = True, skin: float = 1.0,
                 hbm_budget_bytes: int = 0, stream: int | None = None, family: str = "painn", channels: int = 0):
        prec = {"fp32": CTD_PREC_FP32, "bf16": CTD_PREC_BF16}[precision]
        self.desc = ctd_model_desc(F, K, T, n_species, rc, prec, _FAMILIES[family], channels)
        self.grid = tuple(int(g) for g in grid)
        self.dom = _lib.ctd_domains_create(self.desc, params, self.grid, hop_prune, skin, hbm_budget_bytes, stream)
        self.ctx = _lib.ctd_domains_context(self.dom)

    def close(self):
        if getattr(self, "dom", None):
            _lib.ctd_domains_destroy(self.dom)
            self.dom = None
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_option(self, option: int, value: int):
        _lib.ctd_set_option(self.ctx, option, value)

    def compute(self, species, positions, cell, forces: bool = True, virial: bool = True,
                rebuild: bool = False, stats: bool = False, energies: bool = False):
        def call(n, z, x, H, flags, E, Fo, W, st):
            _lib.ctd_domains_compute(self.dom, n, z, x, H, flags, E, Fo, W, st)
        return _compute(call, self.ctx, species, positions, cell, forces, virial, rebuild, stats, energies)

    def info(self):
        """Per-domain counts (owned atoms, copies kept, copies before pruning, edges)."""
        n = self.grid[0] * self.grid[1] * self.grid[2]
        return [_lib.ctd_domains_info(self.dom, d) for d in range(n)]

    def profile(self, enable: bool = True):
        _lib.ctd_profile_enable(self.ctx, enable)

    def profile_read(self, reset: bool = True):
        return _lib.ctd_profile_read(self.ctx, reset)


def _make_autograd():
    import torch

    class PaiNNEnergy(torch.autograd.Function):
        """E = PaiNNEnergy.apply(positions, species, cell, potential) -> (energy, virial).

        positions: CUDA float64 [n,3].  The forward call runs the library's energy, forces and
        virial kernels; backward returns grad_E * (-forces) for the positions (the virial is a
        non-differentiable second output)."""

        @staticmethod
        def forward(ctx, positions, species, cell, potential):
            out = potential.compute(species, positions, cell, forces=True, virial=True)
            ctx.save_for_backward(out["forces"])
            ctx.mark_non_differentiable(out["virial"])
            return out["energy"][0], out["virial"]

        @staticmethod
        def backward(ctx, grad_e, grad_w):
            (forces,) = ctx.saved_tensors
            return -grad_e * forces, None, None, None

    return PaiNNEnergy


class _Lazy:
    _cls = None

    def __getattr__(self, item):
        if _Lazy._cls is None:
            _Lazy._cls = _make_autograd()
        return getattr(_Lazy._cls, item)


PaiNNEnergy = _Lazy()
