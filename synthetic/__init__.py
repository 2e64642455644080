"""Seeded synthetic inputs shared by the FP64 oracle tests, the GPU tests and the benchmark.

This module only *generates data*: atom positions, species, masses, cells, initial
velocities, request sizes and a parameter blob of random weights.  It contains none of
the arithmetic of the potential, of the neighbour search or of the integrator, so the
oracle (``oracle/``) and the CUDA path (``paper_2506_04055_gb300/``) can both consume
its output without sharing any of the method's code.

Systems are shaped like the paper's workloads (Sec. "Molecular Dynamics Simulations":
liquid water, fcc aluminium, a solvated mini-protein).  The paper's structures, datasets
and trained weights are not available, so these generators stand in for them:

* ``water_box``  -- rigid TIP3P-geometry molecules (O-H 0.9572 A, HOH 104.52 deg) with
  random orientations, oxygens on a seeded subset of a simple-cubic lattice, 1.0 g/cm^3.
* ``fcc``        -- single-species fcc crystal, n1 x n2 x n3 conventional cells,
  Gaussian jitter per coordinate.
* ``mixture``    -- 4-species solvated-chain system: a self-avoiding random-walk chain
  in water-like triatomics, triclinic cell with tilts up to 10 %.
* ``params_blob`` -- Xavier-uniform weights (PCG64 stream, fixed tensor order).

Units: Angstrom, amu, fs, K.  The cell ``H`` is a 3x3 array whose ROWS are the lattice
vectors a, b, c.
"""
from __future__ import annotations

import math
import struct

import numpy as np

# --------------------------------------------------------------------------- constants
AMU_PER_H2O = 15.999 + 2 * 1.008          # amu
AVOGADRO_CM3_PER_A3 = 1e-24                # 1 A^3 = 1e-24 cm^3
AMU_G = 1.66053906660e-24                  # g
MASS = {0: 15.999, 1: 1.008, 2: 12.011, 3: 14.007}   # O, H, C-like, N-like
MASS_AL = 26.98
OH_BOND = 0.9572
HOH_ANGLE_DEG = 104.52
KB_EV = 8.617333262e-5                     # eV / K
EV_PER_AMU_A2_FS2 = 103.6426965           # 1 amu A^2 / fs^2 in eV


def water_box_length(n_molecules: int, density_g_cm3: float = 1.0) -> float:
    """Edge of the cubic box holding ``n_molecules`` waters at the given density (A)."""
    mass_g = n_molecules * AMU_PER_H2O * AMU_G
    vol_a3 = mass_g / density_g_cm3 / AVOGADRO_CM3_PER_A3
    return vol_a3 ** (1.0 / 3.0)


def _random_rotations(rng: np.random.Generator, m: int) -> np.ndarray:
    """m uniformly distributed rotation matrices (unit quaternions from normals)."""
    q = rng.standard_normal((m, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    rot = np.empty((m, 3, 3))
    rot[:, 0, 0] = 1 - 2 * (y * y + z * z)
    rot[:, 0, 1] = 2 * (x * y - z * w)
    rot[:, 0, 2] = 2 * (x * z + y * w)
    rot[:, 1, 0] = 2 * (x * y + z * w)
    rot[:, 1, 1] = 1 - 2 * (x * x + z * z)
    rot[:, 1, 2] = 2 * (y * z - x * w)
    rot[:, 2, 0] = 2 * (x * z - y * w)
    rot[:, 2, 1] = 2 * (y * z + x * w)
    rot[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return rot


def _water_local_geometry() -> np.ndarray:
    """O, H1, H2 offsets of one rigid molecule in its own frame (A)."""
    half = math.radians(HOH_ANGLE_DEG) / 2
    return np.array([
        [0.0, 0.0, 0.0],
        [OH_BOND * math.sin(half), OH_BOND * math.cos(half), 0.0],
        [-OH_BOND * math.sin(half), OH_BOND * math.cos(half), 0.0],
    ])


class System:
    """A periodic configuration: positions [n,3], species [n] int32, masses [n], cell [3,3]."""

    def __init__(self, positions, species, masses, cell, name=""):
        self.positions = np.ascontiguousarray(positions, dtype=np.float64)
        self.species = np.ascontiguousarray(species, dtype=np.int32)
        self.masses = np.ascontiguousarray(masses, dtype=np.float64)
        self.cell = np.ascontiguousarray(cell, dtype=np.float64)
        self.name = name

    @property
    def n(self) -> int:
        return int(self.positions.shape[0])

    def __repr__(self):
        return f"System({self.name!r}, n={self.n})"


def water_box(n_molecules: int, seed: int = 0, density: float = 1.0) -> System:
    """Cubic water box: 3*n_molecules atoms, species O=0, H=1 (order O, H, H per molecule)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = water_box_length(n_molecules, density)
    side = int(math.ceil(n_molecules ** (1.0 / 3.0) - 1e-9))
    while side ** 3 < n_molecules:
        side += 1
    sites = np.stack(np.meshgrid(np.arange(side), np.arange(side), np.arange(side),
                                 indexing="ij"), axis=-1).reshape(-1, 3)
    chosen = np.sort(rng.permutation(side ** 3)[:n_molecules])
    o_pos = (sites[chosen] + 0.5) * (L / side)
    rot = _random_rotations(rng, n_molecules)
    local = _water_local_geometry()
    pos = o_pos[:, None, :] + np.einsum("mab,kb->mka", rot, local)
    species = np.tile(np.array([0, 1, 1], dtype=np.int32), n_molecules)
    masses = np.array([MASS[int(z)] for z in species])
    return System(pos.reshape(-1, 3), species, masses, np.eye(3) * L, f"water{3 * n_molecules}")


def fcc(n1: int, n2: int, n3: int, a: float = 4.05, jitter: float = 0.05, seed: int = 0,
        species: int = 0, mass: float = MASS_AL) -> System:
    """Single-species fcc crystal of n1*n2*n3 conventional cells (4 atoms each)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    cells = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3),
                                 indexing="ij"), axis=-1).reshape(-1, 3)
    pos = ((cells[:, None, :] + basis[None, :, :]) * a).reshape(-1, 3)
    if jitter > 0:
        pos = pos + rng.normal(0.0, jitter, size=pos.shape)
    n = pos.shape[0]
    cell = np.diag([n1 * a, n2 * a, n3 * a])
    return System(pos, np.full(n, species, np.int32), np.full(n, mass), cell,
                  f"fcc{n1}x{n2}x{n3}")


def mixture(n_chain: int = 300, n_water: int = 30000, tilt: float = 0.10, seed: int = 0,
            bond: float = 1.5, avoid: float = 1.2, clearance: float = 2.5) -> System:
    """Solvated-chain mixture: a self-avoiding random-walk chain (species 2,3 alternating,
    bond ``bond`` A) in ``n_water`` water-like triatomics, triclinic cell with tilts
    xy, xz, yz ~ U(-tilt*L, tilt*L).  Box volume chosen for ~1 g/cm^3 overall."""
    rng = np.random.Generator(np.random.PCG64(seed))
    chain_mass = sum(MASS[2 + (k % 2)] for k in range(n_chain))
    total_mass_g = (n_water * AMU_PER_H2O + chain_mass) * AMU_G
    L = (total_mass_g / 1.0 / AVOGADRO_CM3_PER_A3) ** (1.0 / 3.0)
    xy, xz, yz = rng.uniform(-tilt * L, tilt * L, size=3)
    H = np.array([[L, 0.0, 0.0], [xy, L, 0.0], [xz, yz, L]])
    # chain: self-avoiding random walk started at the box centre (Cartesian, unwrapped)
    chain = np.empty((n_chain, 3))
    chain[0] = H.sum(axis=0) / 2
    k = 1
    tries = 0
    while k < n_chain:
        step = rng.standard_normal(3)
        step *= bond / np.linalg.norm(step)
        cand = chain[k - 1] + step
        if k < 2 or np.min(np.linalg.norm(chain[:k - 1] - cand, axis=1)) >= avoid:
            chain[k] = cand
            k += 1
            tries = 0
        else:
            tries += 1
            if tries > 1000:
                raise RuntimeError("random walk trapped")
    # water on a fractional lattice, enlarged until n_water sites clear the chain
    Ginv = np.linalg.inv(H.T)
    chain_frac = (Ginv @ chain.T).T
    side = int(math.ceil(n_water ** (1 / 3)))
    while True:
        g = (np.stack(np.meshgrid(np.arange(side), np.arange(side), np.arange(side),
                                  indexing="ij"), axis=-1).reshape(-1, 3) + 0.5) / side
        cart = g @ H
        keep = np.ones(len(g), bool)
        for c in range(n_chain):   # minimum-image distance to every chain atom
            df = g - chain_frac[c]
            df -= np.round(df)
            d = np.linalg.norm(df @ H, axis=1)
            keep &= d >= clearance
        if keep.sum() >= n_water:
            break
        side += 1
    idx = np.flatnonzero(keep)
    idx = np.sort(rng.permutation(idx)[:n_water])
    o_pos = cart[idx]
    rot = _random_rotations(rng, n_water)
    wpos = (o_pos[:, None, :] + np.einsum("mab,kb->mka", rot, _water_local_geometry())).reshape(-1, 3)
    pos = np.concatenate([chain, wpos])
    species = np.concatenate([np.array([2 + (k % 2) for k in range(n_chain)], np.int32),
                              np.tile(np.array([0, 1, 1], np.int32), n_water)])
    masses = np.array([MASS[int(z)] for z in species])
    return System(pos, species, masses, H, f"mixture{len(pos)}")


def maxwell_boltzmann(masses: np.ndarray, temperature: float, seed: int = 0) -> np.ndarray:
    """Velocities (A/fs) drawn at ``temperature`` K, centre-of-mass momentum removed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = np.asarray(masses, np.float64)
    sigma = np.sqrt(KB_EV * temperature / (m * EV_PER_AMU_A2_FS2))
    v = rng.standard_normal((len(m), 3)) * sigma[:, None]
    p = (m[:, None] * v).sum(axis=0)
    v -= p / m.sum()
    return v


def request_sizes(n_requests: int, lo: int = 64, hi: int = 20000, seed: int = 0) -> np.ndarray:
    """Target atom counts drawn log-uniformly in [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_requests)).round().astype(np.int64)


def system_near(n_target: int, kind: str, seed: int = 0) -> System:
    """Water box (floor(n/3) molecules) or fcc (n1 n2 n3 cells, 4 n1 n2 n3 closest to n)."""
    if kind == "water":
        return water_box(max(1, n_target // 3), seed=seed)
    best = None
    for n1 in range(1, 20):
        for n2 in range(n1, 20):
            for n3 in range(n2, 20):
                n = 4 * n1 * n2 * n3
                score = (abs(n - n_target), n3 - n1)
                if best is None or score < best[0]:
                    best = (score, (n1, n2, n3))
    return fcc(*best[1], seed=seed)


# --------------------------------------------------------------------------- parameters
PARAM_MAGIC = b"CTDPAINN"
PARAM_VERSION = 1
PARAM_HEADER_BYTES = 64


def param_shapes(F: int, K: int, T: int, S: int):
    """(name, shape) of every weight tensor, in blob order.  Matrices are [out, in]."""
    shapes = [("emb", (S, F))]
    for t in range(T):
        shapes += [
            (f"W1_{t}", (F, F)), (f"b1_{t}", (F,)), (f"W2_{t}", (3 * F, F)), (f"b2_{t}", (3 * F,)),
            (f"Wf_{t}", (3 * F, K)), (f"bf_{t}", (3 * F,)),
            (f"U_{t}", (F, F)), (f"V_{t}", (F, F)),
            (f"A1_{t}", (F, 2 * F)), (f"c1_{t}", (F,)), (f"A2_{t}", (3 * F, F)), (f"c2_{t}", (3 * F,)),
        ]
    shapes += [("R1", (F // 2, F)), ("d1", (F // 2,)), ("R2", (F // 2,)), ("d2", (1,))]
    return shapes


def xavier_params(F: int, K: int, T: int, S: int, seed: int = 0, bias_scale: float = 0.0):
    """Flat float64 parameter vector.  Every matrix is Xavier-uniform
    U(+-sqrt(6/(fan_in+fan_out))); the embedding uses fan_in = S.  Biases are zero unless
    ``bias_scale`` > 0, in which case they are U(-bias_scale, bias_scale) (used by tests so
    that bias terms are exercised)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for name, shape in param_shapes(F, K, T, S):
        if name == "emb":
            fan_in, fan_out = S, F
            bound = math.sqrt(6.0 / (fan_in + fan_out))
            out.append(rng.uniform(-bound, bound, size=shape).ravel())
        elif name == "R2":
            bound = math.sqrt(6.0 / (shape[0] + 1))
            out.append(rng.uniform(-bound, bound, size=shape).ravel())
        elif len(shape) == 2:
            bound = math.sqrt(6.0 / (shape[0] + shape[1]))
            out.append(rng.uniform(-bound, bound, size=shape).ravel())
        else:
            if bias_scale > 0:
                out.append(rng.uniform(-bias_scale, bias_scale, size=shape).ravel())
            else:
                out.append(np.zeros(shape).ravel())
    return np.concatenate(out).astype(np.float64)


def params_blob(F: int, K: int = 20, T: int = 3, S: int = 2, rc: float = 5.0, eps: float = 1e-8,
                e_scale: float = 1.0, seed: int = 0, bias_scale: float = 0.0,
                values: np.ndarray | None = None) -> bytes:
    """Serialised parameters: 64-byte header followed by float64 values.

    header: magic[8]="CTDPAINN", int32 version, F, K, T, S, int32 reserved,
            float64 rc, eps, e_scale, int64 n_values   (little endian)
    """
    if values is None:
        values = xavier_params(F, K, T, S, seed, bias_scale)
    values = np.ascontiguousarray(values, np.float64)
    expect = sum(int(np.prod(s)) for _, s in param_shapes(F, K, T, S))
    if values.size != expect:
        raise ValueError(f"expected {expect} values, got {values.size}")
    head = PARAM_MAGIC + struct.pack("<iiiiii", PARAM_VERSION, F, K, T, S, 0)
    head += struct.pack("<dddq", rc, eps, e_scale, values.size)
    assert len(head) == PARAM_HEADER_BYTES
    return head + values.tobytes()


def unpack_params(values: np.ndarray, F: int, K: int, T: int, S: int) -> dict:
    """Name -> array views of a flat parameter vector (for building hand-set test weights)."""
    out, off = {}, 0
    for name, shape in param_shapes(F, K, T, S):
        n = int(np.prod(shape))
        out[name] = values[off:off + n].reshape(shape)
        off += n
    return out


# ---- parameters of the strictly local edge model ---------------------------------------------
LOCAL_MAGIC = b"CTDLOCAL"


def local_param_shapes(F: int, K: int, L: int, S: int, C: int):
    """(name, shape) of every parameter of the strictly local edge model in blob order: the
    two-body MLP A0 [K+2S][F] and c0, the initial-feature map P0 [F][2C]; per layer l the
    environment weights Q_l [F][2C], the latent update M_l [F+2C][F] and m_l, and for l < L the
    channel mixings Gs_l, Gv_l [2C][C]; the readout R1 [F][F/2], d1, R2 [F/2], d2."""
    shapes = [("A0", (K + 2 * S, F)), ("c0", (F,)), ("P0", (F, 2 * C))]
    for layer in range(1, L + 1):
        shapes += [(f"Q{layer}", (F, 2 * C)), (f"M{layer}", (F + 2 * C, F)), (f"m{layer}", (F,))]
        if layer < L:
            shapes += [(f"Gs{layer}", (2 * C, C)), (f"Gv{layer}", (2 * C, C))]
    Fh = F // 2
    return shapes + [("R1", (F, Fh)), ("d1", (Fh,)), ("R2", (Fh,)), ("d2", (1,))]


def local_xavier_params(F: int, K: int, L: int, S: int, C: int, seed: int = 0, bias_scale: float = 0.0):
    """Flat float64 parameters of the local model: matrices Xavier-uniform, R2 with fan_out 1,
    biases zero or U(-bias_scale, bias_scale)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for name, shape in local_param_shapes(F, K, L, S, C):
        if name == "R2":
            bound = math.sqrt(6.0 / (shape[0] + 1))
            out.append(rng.uniform(-bound, bound, size=shape).ravel())
        elif len(shape) == 2:
            bound = math.sqrt(6.0 / (shape[0] + shape[1]))
            out.append(rng.uniform(-bound, bound, size=shape).ravel())
        elif bias_scale > 0:
            out.append(rng.uniform(-bias_scale, bias_scale, size=shape).ravel())
        else:
            out.append(np.zeros(shape).ravel())
    return np.concatenate(out).astype(np.float64)


def local_params_blob(F: int, K: int = 20, L: int = 2, S: int = 2, C: int = 16, rc: float = 5.0,
                      e_scale: float = 1.0, seed: int = 0, bias_scale: float = 0.0,
                      values: np.ndarray | None = None) -> bytes:
    """Serialised local-model parameters: 64-byte header followed by float64 values.

    header: magic[8]="CTDLOCAL", int32 version, F, K, L, S, C,
            float64 rc, 0.0 (unused), e_scale, int64 n_values   (little endian)
    """
    if values is None:
        values = local_xavier_params(F, K, L, S, C, seed, bias_scale)
    values = np.ascontiguousarray(values, np.float64)
    expect = sum(int(np.prod(s)) for _, s in local_param_shapes(F, K, L, S, C))
    if values.size != expect:
        raise ValueError(f"expected {expect} values, got {values.size}")
    head = LOCAL_MAGIC + struct.pack("<iiiiii", PARAM_VERSION, F, K, L, S, C)
    head += struct.pack("<dddq", rc, 0.0, e_scale, values.size)
    assert len(head) == PARAM_HEADER_BYTES
    return head + values.tobytes()
