/*
 * painn.h -- C ABI of the GB300 engine for a PaiNN-form semi-local potential
 * (energy, forces, virial) over a periodic neighbour graph.
 *
 * Method: arXiv 2506.04055 ("chemtrain-deploy").  The total energy is a sum of semi-local
 * per-atom energies over a cutoff graph (Methods, "(Semi-)Local Potential Models", energy-sum
 * equation); forces are its negative gradient (Results, "Distributed potential computation",
 * sum-rule equation); the MD code hands the library positions and a neighbour graph built
 * with a skin, the library prunes edges longer than the cutoff every step, buffers data to
 * fixed capacities that only grow, checks for overflow after a run and repeats it with larger
 * buffers (Results, "Runtime optimizations and buffering").  The model is PaiNN (Methods,
 * "Chosen Architectures"), with cutoff 5 A (Methods, "Training Details").
 *
 * Conventions (all entry points):
 *   - Units: Angstrom, eV, amu, fs.  Arrays are row-major.  A cell is double[9] whose ROWS
 *     are the lattice vectors a, b, c; every system is periodic in all three directions.
 *   - Atom arrays are in the caller's order.  Positions/forces are [n][3] double.
 *   - Pointers are host pointers unless CTD_DEVICE_PTRS is set in `flags`, in which case
 *     species/positions/energy/forces/virial are device pointers valid on the context's
 *     stream.  The caller owns every pointer it passes; the library copies what it keeps.
 *   - The context owns its device buffers.  They grow (never shrink) up to the HBM budget
 *     given at creation; a call that would exceed it fails with CTD_ERR_OUT_OF_BUDGET.
 *   - Calls on one context are not thread-safe; distinct contexts are independent.
 *   - Every call returns CTD_OK (0) or a negative CTD_ERR_* code; ctd_last_error() then
 *     describes the failure.  Device kernels never trap: they raise status words that the
 *     host reads after the launch.
 */
#ifndef CTD_PAINN_H
#define CTD_PAINN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------------------------- */
#define CTD_OK 0
#define CTD_ERR_INVALID_ARG (-1)   /* bad pointer, size, flag, cell or parameter blob          */
#define CTD_ERR_CAPACITY (-2)      /* an internal buffer overflowed and could not be regrown    */
#define CTD_ERR_OUT_OF_BUDGET (-3) /* growing a buffer would exceed the HBM budget              */
#define CTD_ERR_CELL_TOO_SMALL (-4) /* cell thinner than the search needs (image limit, 127)    */
#define CTD_ERR_CUDA (-5)          /* a CUDA runtime call failed                                */
#define CTD_ERR_TIMEOUT (-6)       /* a bounded device wait gave up                             */
#define CTD_ERR_NONFINITE (-7)     /* NaN/Inf in positions or results                           */
#define CTD_ERR_STATE (-8)         /* call out of order (no parameters, no neighbour list, ...) */

/* ---- precision of the dense contractions ----------------------------------------------- */
#define CTD_PREC_FP32 0   /* every product in FP32 on CUDA cores                              */
#define CTD_PREC_BF16 1   /* node MLPs in BF16 on tcgen05 with FP32 accumulation; at F = 128
                             also the edge message (FP16 rows x basis, FP32 filter weights)
                             and the adjoint's radial filter; F must be 64 or 128           */

/* ---- flags for ctd_compute ---------------------------------------------------------------- */
#define CTD_NEED_FORCES 1      /* write forces[n][3]                                          */
#define CTD_NEED_VIRIAL 2      /* write virial[9] = -sum_e r_e (x) dU/dr_e (row-major, eV)     */
#define CTD_REBUILD 4          /* rebuild the neighbour list even if the skin still holds     */
#define CTD_DEVICE_PTRS 8      /* I/O pointers are device pointers on the context's stream    */

/* ---- model families ------------------------------------------------------------------------ */
#define CTD_FAMILY_PAINN 0  /* semi-local message passing (PaiNN form; Methods, "Chosen
                               Architectures"): T layers reach T cutoffs                        */
#define CTD_FAMILY_LOCAL 1  /* strictly local equivariant edge model (Allegro form, rotation
                               orders <= 1): messages only between edges leaving the same atom,
                               so an atom's energy depends on its own cutoff sphere alone        */

/* Model description.  F: feature width (even, multiple of 32, <= 256); K: radial basis size
 * (<= 32); T: interaction layers (<= 8); n_species: embedding rows; rc: cutoff (A);
 * precision: CTD_PREC_*.  Must equal the header of the parameter blob.
 * family: CTD_FAMILY_*.  For CTD_FAMILY_LOCAL: F = latent width (multiple of 8, 8..256),
 * channels = equivariant channels C (multiple of 4, 4..64), T = layers (1..8), precision
 * CTD_PREC_FP32; ctd_load_params then takes the "CTDLOCAL" blob.  channels is ignored for
 * CTD_FAMILY_PAINN (zero-initialise both fields for the PaiNN form). */
typedef struct {
  int32_t F, K, T, n_species;
  double rc;
  int32_t precision;
  int32_t family;
  int32_t channels;
} ctd_model_desc;

/* Per-call statistics (the library "returns statistics of the computation"). */
typedef struct {
  int64_t n_atoms;
  int64_t n_verlet_edges;   /* directed edges within rc + skin                                */
  int64_t n_active_edges;   /* directed edges within rc this step                             */
  int32_t rebuilt;          /* 1 if this call rebuilt the neighbour list                      */
  int32_t retries;          /* repeats after a capacity overflow                              */
  double max_displacement;  /* largest displacement since the last rebuild (A)                */
  int64_t bytes_allocated;  /* device bytes held by the context                               */
  float ms_neighbors, ms_model;   /* device time of the neighbour and model stages (ms)      */
  int32_t edges_stored;     /* 1 if the adjoint read per-edge filters stored by the forward   */
  int32_t reserved;
  int64_t bytes_in_use;     /* device bytes the current shapes need: bytes_allocated less the  */
                            /* growth headroom (25 % of each buffer grown)                     */
} ctd_stats;

typedef struct ctd_ctx ctd_ctx;

/* Create a context on the current CUDA device.  `hbm_budget_bytes` caps the device memory
 * the context may hold (0 = no cap).  `cuda_stream` is a cudaStream_t (NULL = a new stream
 * owned by the context).  On success *out receives the context. */
int ctd_create(ctd_ctx **out, const ctd_model_desc *desc, size_t hbm_budget_bytes,
               void *cuda_stream);

/* Copy model parameters from a host blob: 64-byte header (magic "CTDPAINN", int32 version=1,
 * F, K, T, S, reserved; float64 rc, eps, e_scale; int64 n_values) followed by n_values
 * float64 weights in this order (matrices [out][in]): emb[S][F]; per layer W1[F][F] b1[F]
 * W2[3F][F] b2[3F] Wf[3F][K] bf[3F] U[F][F] V[F][F] A1[F][2F] c1[F] A2[3F][F] c2[3F];
 * R1[F/2][F] d1[F/2] R2[F/2] d2[1].  The caller keeps the blob. */
/* CTD_FAMILY_LOCAL: magic "CTDLOCAL", int32 version=1, F, K, T (= layers L), S, C; float64
 * rc, unused, e_scale; int64 n_values; then the float64 weights, matrices [in][out]:
 * A0[K+2S][F] c0[F] P0[F][2C]; per layer l = 1..L: Q[F][2C] M[F+2C][F] m[F], and for l < L
 * Gs[2C][C] Gv[2C][C]; R1[F][F/2] d1[F/2] R2[F/2] d2[1].  The model, per directed edge
 * e = (i -> j) with r_e = x_j - x_i (+ image), d = |r_e|, u = r_e / d, cosine cutoff f_c and
 * the Gaussian basis b_k of the PaiNN form: x = silu([b f_c | onehot(Z_i) | onehot(Z_j)] A0 + c0);
 * s = (x P0)[0:C], v = (x P0)[C:2C] u; per layer: om = x Q, atom sums over i's edges
 * Gs_i = sum f_c om[0:C], Gv_i = sum f_c om[C:2C] u; ts = [s Gs_i | v . Gv_i],
 * tv = [s Gv_i | v Gs_i]; x = silu([x | ts] M + m); (l < L) s = ts Gs, v = tv Gv; energy
 * E_i = e_scale sum_{e from i} f_c (silu(x R1 + d1) . R2 + d2). */
int ctd_load_params(ctd_ctx *ctx, const void *blob, size_t nbytes);

/* Build the Verlet neighbour list of n atoms: every (i, j, n) with
 * |x~_j - x~_i + n1 a + n2 b + n3 c| < cutoff + skin, i != j or n != 0, where x~ are the
 * positions wrapped into the cell.  The test is evaluated in FP64 with every product and sum
 * rounded separately in a fixed order (bit-reproducible).  Positions are host doubles [n][3]
 * (device pointers if flags & CTD_DEVICE_PTRS).  *n_pairs_out receives the number of
 * directed pairs.  The list is kept in the context and reused by ctd_compute until an atom
 * moves more than skin/2. */
int ctd_build_neighbors(ctd_ctx *ctx, int64_t n, const double *positions, const double cell[9],
                        double cutoff, double skin, int32_t flags, int64_t *n_pairs_out);

/* Copy the current Verlet list to host arrays ordered by (i, j, n1, n2, n3), caller's atom
 * indices; shift holds n1, n2, n3 per pair relative to the wrapped positions.  cap = array
 * length; returns CTD_ERR_CAPACITY if the list is longer (nothing written). */
int ctd_get_pairs(ctd_ctx *ctx, int32_t *i, int32_t *j, int8_t *shift, int64_t cap);

/* Energy (and forces, virial) of n atoms.  Rebuilds the neighbour list when none exists, when
 * n or the cell changed, when an atom moved more than skin/2 since the last build, or when
 * CTD_REBUILD is set (the skin defaults to 1 A if ctd_build_neighbors was never called).
 * energy: double[1]; forces: double[n][3] (with CTD_NEED_FORCES); virial: double[9] (with
 * CTD_NEED_VIRIAL); stats may be NULL. */
int ctd_compute(ctd_ctx *ctx, int64_t n, const int32_t *species, const double *positions,
                const double cell[9], int32_t flags, double *energy, double *forces,
                double *virial, ctd_stats *stats);

/* Optional per-atom energy output (double[n], same pointer kind as the compute call); NULL
 * disables it. */
int ctd_set_energy_out(ctd_ctx *ctx, double *energies);

/* ---- molecular dynamics (NVE velocity Verlet, state resident on the device) --------------- */

/* Load an MD state: n atoms, species, masses (amu), positions (A), velocities (A/fs), cell,
 * neighbour skin (A).  Host arrays; copied to the device. */
int ctd_md_set_state(ctd_ctx *ctx, int64_t n, const int32_t *species, const double *masses,
                     const double *positions, const double *velocities, const double cell[9],
                     double skin);

/* Advance nsteps velocity-Verlet steps of dt fs entirely on the device, rebuilding the
 * neighbour list whenever an atom moved more than skin/2.  epot/ekin (host, may be NULL)
 * receive nsteps+1 potential / kinetic energies (eV).  n_rebuilds (may be NULL) receives the
 * number of rebuilds. */
int ctd_md_run(ctd_ctx *ctx, int32_t nsteps, double dt, double *epot, double *ekin,
               int32_t *n_rebuilds);

/* Copy the MD state back (host arrays [n][3], either may be NULL). */
int ctd_md_get_state(ctd_ctx *ctx, double *positions, double *velocities);

/* Nose-Hoover chain thermostat for ctd_md_run (NVT; Methods, "MD simulations": Nose-Hoover
 * thermostat with a temperature damping parameter).  chain = number of thermostats M (1..16;
 * 0 switches back to NVE); temperature in K; tau in fs.  Equations (Martyna, Tuckerman, Klein):
 * dv_i/dt = F_i/m_i - vxi_1 v_i, dvxi_1/dt = (2K - Nf kB T)/Q_1 - vxi_2 vxi_1,
 * dvxi_j/dt = (Q_{j-1} vxi_{j-1}^2 - kB T)/Q_j - vxi_{j+1} vxi_j, dxi_j/dt = vxi_j, with
 * Q_1 = Nf kB T tau^2, Q_j = kB T tau^2 and Nf = 3n - 3; each step is a chain half step, velocity
 * Verlet, a chain half step (symmetric Trotter splitting).  The chain starts at rest; this call
 * and ctd_md_set_state reset it.  The conserved quantity is epot + ekin + the chain energy that
 * ctd_md_get_thermostat returns. */
int ctd_md_set_thermostat(ctd_ctx *ctx, double temperature, double tau, int32_t chain);
/* Chain state (xi[M], vxi[M], host, may be NULL) and the chain energy after every step of the
 * last ctd_md_run (ethermo[nsteps+1], may be NULL): sum_j Q_j vxi_j^2/2 + Nf kB T xi_1
 * + kB T sum_{j>1} xi_j (eV).  CTD_ERR_STATE without a thermostat. */
int ctd_md_get_thermostat(ctd_ctx *ctx, double *xi, double *vxi, double *ethermo);
/* Restore a chain state (xi[M], vxi[M], host) saved by ctd_md_get_thermostat, after
 * ctd_md_set_state and ctd_md_set_thermostat, to continue a checkpointed NVT trajectory.
 * CTD_ERR_STATE without a thermostat; CTD_ERR_INVALID_ARG for non-finite values. */
int ctd_md_set_thermostat_state(ctd_ctx *ctx, const double *xi, const double *vxi);

/* ---- options -------------------------------------------------------------------------- */
/* CTD_OPT_TC_ADJOINT (value 0 or 1; default 1): on the BF16 path with F = 128, run the edge
 * adjoint with the radial filter and its distance derivative on tcgen05 with FP16 weights and
 * basis (1), or on CUDA cores with FP32 weights (0).  A model whose filter weights exceed the
 * FP16 range is loaded with 0. */
#define CTD_OPT_TC_ADJOINT 1
/* CTD_OPT_EDGE_STORE (value 0 or 1; default 0): the forward message kernel stores, per active
 * edge and layer, the cutoff-scaled radial filter and its distance derivative (6F floats), and
 * the adjoint reads them instead of recomputing basis and filter (the default).  Storage costs
 * T x E x 6F x 4 bytes; it is used only when that fits the HBM budget (if one is set) and 80 %
 * of the device's free memory, and otherwise the call recomputes (ctd_stats.edges_stored says
 * which).  It applies to the CUDA-core edge kernels: the FP32 path, and BF16 with F != 128 or
 * with both tensor-core edge kernels switched off (CTD_OPT_TC_MESSAGE 0, CTD_OPT_TC_ADJOINT 0). */
#define CTD_OPT_EDGE_STORE 2
/* CTD_OPT_TC_MESSAGE (value 0 or 1; default 1): on the BF16 path with F = 128, compute the
 * message step as a tensor-core contraction over each receiver's edges (1): the senders' message
 * rows [phi_s | v_a phi_vv | phi_vs] in FP16 times the per-edge basis f_c rbf_k (with u_a for
 * the vector term), accumulated in FP32, and the FP32 filter weights applied per receiver
 * (Wf rbf + bf = sum_k Wf'[c][k] b_k with the bias as column K); or on CUDA cores with the FP32
 * filter (0). */
#define CTD_OPT_TC_MESSAGE 3
/* CTD_OPT_EDGE_CHUNK_ROWS (value >= 0; default 32): the tensor-core adjoint hands out the
 * sorted rows in chunks of this many rows, block-cyclically over all row streams of the GPU;
 * 0 gives each stream one contiguous range. */
#define CTD_OPT_EDGE_CHUNK_ROWS 4
int ctd_set_option(ctd_ctx *ctx, int32_t option, int64_t value);

/* ---- launch accounting and stage timing (benchmarks, statistics) ------------------------- */
/* Stages: 0 neighbour build, 1 per-step prune, 2 node MLPs (message phi, update, readout),
 * 3 edge message, 4 edge adjoint, 5 forces / virial / energy reductions, 6 integrator,
 * 7 other (output scatter, checks). */
#define CTD_NSTAGES 8

/* enable != 0: bracket every kernel launch with CUDA events on the context's stream (adds a
 * small host cost per launch).  Launch counts are always kept. */
int ctd_profile_enable(ctd_ctx *ctx, int32_t enable);

/* Copy the accumulated device milliseconds and launch counts per stage (arrays of
 * CTD_NSTAGES, either may be NULL) since the last reset; reset != 0 zeroes them.  Waits for
 * the timed launches to finish. */
int ctd_profile_read(ctd_ctx *ctx, double *ms, int64_t *launches, int32_t reset);

/* ---- tensor-core building block ---------------------------------------------------------- */
/* C[M][N] = A[M][K] . B[N][K]^T with BF16 operands and FP32 accumulation on the tcgen05
 * tensor cores, operand tiles staged by TMA -- the contraction every MLP of the BF16 path
 * runs on.  Device pointers on the context's stream: A bf16 row-major with leading dimension
 * lda (elements, lda*2 a multiple of 16 bytes), B bf16 [N][K] row-major, C float row-major
 * with leading dimension ldc.  K: multiple of 32, >= 64; N: multiple of 32, <= 512.  Synchronises
 * the stream; CTD_ERR_TIMEOUT if a bounded device wait gave up. */
int ctd_gemm_bf16(ctd_ctx *ctx, int64_t M, int32_t N, int32_t K, const void *A, int64_t lda,
                  const void *B, float *C, int64_t ldc);

/* ---- serving: continuous batching of independent MD replicas --------------------------------- */
/* A server keeps many independent replicas (own atoms, cell, neighbour list) resident on one
 * GPU and advances all of them together: each ctd_serve_step is one velocity-Verlet step in
 * which every stage (integrator, prune, model, adjoint, force assembly) is one launch over the
 * concatenation of the resident replicas.  Requests queue FIFO and are admitted between steps
 * while the HBM budget (hbm_budget_bytes of ctd_serve_create; 0 = none) and max_replicas allow;
 * a replica leaves after its nsteps steps and its final state stays available to
 * ctd_serve_poll.  A replica's trajectory does not depend on which other replicas share the
 * batch (per-replica reductions run in a fixed order of its own atoms).  dt: time step (fs),
 * shared by all replicas; max_replicas 1..65535.  The params blob is the one ctd_load_params
 * takes. */
typedef struct ctd_server ctd_server;
int ctd_serve_create(ctd_server **out, const ctd_model_desc *desc, const void *params, size_t nbytes,
                     size_t hbm_budget_bytes, int32_t max_replicas, double dt, void *cuda_stream);
/* Queue one replica (host arrays, copied): n atoms, species, masses (amu), positions (A),
 * velocities (A/fs), cell, neighbour skin (A), number of steps.  *request_id identifies it. */
int ctd_serve_submit(ctd_server *s, int64_t n, const int32_t *species, const double *masses,
                     const double *positions, const double *velocities, const double cell[9],
                     double skin, int32_t nsteps, int64_t *request_id);
/* Retire finished replicas, admit queued ones, run one step of all resident replicas (a newly
 * admitted replica's first step evaluates its initial forces without moving it).  Outputs
 * (may be NULL): replicas resident during the step, admitted and retired by this call. */
int ctd_serve_step(ctd_server *s, int32_t *n_resident, int32_t *n_admitted, int32_t *n_finished);
/* State of a request: 0 queued, 1 resident, 2 finished; steps done.  When finished, positions
 * and velocities ([n][3], caller's atom order) receive the final state.  epot / ekin receive the
 * energies recorded so far (one per step, the first at the initial positions: up to nsteps+1
 * values); virial[9] the latest virial.  Any output pointer may be NULL. */
int ctd_serve_poll(ctd_server *s, int64_t request_id, int32_t *state, int32_t *steps_done,
                   double *positions, double *velocities, double *epot, double *ekin, double *virial);
/* Checkpoint of a resident replica: its current positions and velocities ([n][3], caller's atom
 * order, host) and the steps it has done; the replica stays resident.  Submitting the snapshot
 * with the remaining step count continues the trajectory (on this or another server).
 * CTD_ERR_STATE if the request is queued or finished (poll returns the final state). */
int ctd_serve_snapshot(ctd_server *s, int64_t request_id, double *positions, double *velocities,
                       int32_t *steps_done);
/* Nose-Hoover chain thermostat for one queued request (NVT; the chain and its parameters as in
 * ctd_md_set_thermostat: chain = M thermostats 0..16, 0 = NVE; temperature (K) and tau (fs)
 * positive and finite; n >= 2).  xi[M], vxi[M] (host, may both be NULL = zero) restore a chain
 * state saved by ctd_serve_thermostat, to continue a checkpointed NVT replica.  Each step of the
 * replica is then a chain half step, the velocity-Verlet step, and a chain half step, like
 * ctd_md_run's NVT step; the kinetic energies recorded for it are those after the chain's
 * velocity factor.  Replicas with and without thermostats share the batch, and a replica's
 * trajectory still does not depend on the others.  CTD_ERR_STATE unless the request is queued. */
int ctd_serve_set_thermostat(ctd_server *s, int64_t request_id, double temperature, double tau,
                             int32_t chain, const double *xi, const double *vxi);
/* Chain state of a request with a thermostat: xi[M], vxi[M] (host; the current state while
 * resident, the final one when finished) and ethermo, the chain energy recorded with each
 * energy of ctd_serve_poll (up to nsteps+1 values).  Any output may be NULL.  CTD_ERR_STATE
 * without a thermostat. */
int ctd_serve_thermostat(ctd_server *s, int64_t request_id, double *xi, double *vxi, double *ethermo);
int ctd_serve_stats(ctd_server *s, int64_t *resident_atoms, int32_t *resident_replicas,
                    int32_t *queued, int64_t *bytes_held);

/* A served step's device work after the per-replica rebuild decisions -- the prune, the model
 * (energy, forces, virial) over the whole batch, the second half kick, the per-replica sums and
 * thermostat half step -- is recorded once as a CUDA graph when the batch layout (resident
 * replicas, atom count, device buffers, options) has not changed over the previous step, and
 * replayed as one graph launch while it stays unchanged; a change (admission, retirement, a
 * buffer that grows) runs that step eagerly and records again on the next.  Replay and eager
 * steps launch the same kernels on the same data, so trajectories are identical either way.
 * Not used for the strictly local family, with stored edge filters, or while per-launch
 * profiling is on.  ctd_serve_use_graph(s, 0) turns it off (default on). */
int ctd_serve_use_graph(ctd_server *s, int32_t enable);
/* Steps run by graph replay and eagerly, kernel launches in one replay, graphs recorded.
 * Any output may be NULL. */
int ctd_serve_graph_stats(ctd_server *s, int64_t *graph_steps, int64_t *eager_steps,
                          int64_t *kernels_per_replay, int64_t *captures);
const char *ctd_serve_last_error(ctd_server *s);
void ctd_serve_destroy(ctd_server *s);

/* ---- spatial domain decomposition with copied atoms ---------------------------------------- */
/* Results, "Distributed potential computation" (energy-sum and sum-rule equations) and
 * "Parallelization cost": the periodic system is split into grid[0] x grid[1] x grid[2]
 * domains over its fractional coordinates; each atom is owned by the domain whose box holds its
 * wrapped position, and each domain also holds copies of every atom and periodic image within
 * R_comm = T rc + skin of its box (measured perpendicular to the box faces).  A domain's energy
 * is the sum of its owned atoms' U_i; the total energy is the sum over domains, and the force
 * on an atom the sum of the partial forces on its copies.  With hop_prune != 0, copies more
 * than T hops (over the neighbour graph with cutoff rc + skin) from every owned atom are
 * dropped, and edges with neither atom within T - 1 hops are not evaluated; the results do not
 * change (up to FP32 summation order).
 *
 * All domains run on this GPU as one batched system: this is the decomposition a run on
 * grid[0] grid[1] grid[2] processors would compute, with its two exchanges (copy positions
 * before the model, copy forces after it) as kernels.  ctd_domains_info reports the work the
 * copies add.  desc / params / nbytes / hbm_budget_bytes / cuda_stream: as ctd_create and
 * ctd_load_params.  grid[a] in 1..64 with at most 4096 domains; skin >= 0 (A).  Options
 * (ctd_set_option) and profiling go through the context ctd_domains_context returns.  T is the
 * model's reach in hops: desc->T for CTD_FAMILY_PAINN, 1 for CTD_FAMILY_LOCAL (strictly local:
 * R_comm = rc + skin and copies one hop deep, whatever the layer count). */
typedef struct ctd_domains ctd_domains;
typedef struct {
  int64_t n_owned;         /* atoms the domain owns                                           */
  int64_t n_copies;        /* copies of other atoms (and periodic images) it evaluates         */
  int64_t n_candidates;    /* copies within R_comm before hop pruning                          */
  int64_t n_verlet_edges;  /* its neighbour pairs (cutoff rc + skin)                            */
  int64_t n_active_edges;  /* its edges in the last evaluation (r < rc, hop test)               */
  int32_t grid_index[3];   /* the domain's position in the grid                                 */
  int32_t reserved;
} ctd_domain_info;
int ctd_domains_create(ctd_domains **out, const ctd_model_desc *desc, const void *params, size_t nbytes,
                       size_t hbm_budget_bytes, const int32_t grid[3], int32_t hop_prune, double skin,
                       void *cuda_stream);
/* Energy, forces and virial of the periodic system by the decomposition, with the conventions
 * and flags of ctd_compute (CTD_REBUILD forces a new decomposition).  The decomposition and
 * the domains' neighbour lists are reused while no atom has moved more than skin / 2 since
 * they were built; n or cell changing also rebuilds them.  forces[n][3] in the caller's order
 * are the summed partial forces of each atom's copies (FP64 sums in a fixed order); per-atom
 * energies (ctd_set_energy_out on the context) come from each atom's owned copy.  stats:
 * n_atoms counts owned atoms plus copies, the edge counts are summed over the domains. */
int ctd_domains_compute(ctd_domains *d, int64_t n, const int32_t *species, const double *positions,
                        const double cell[9], int32_t flags, double *energy, double *forces,
                        double *virial, ctd_stats *stats);
/* Counts of domain index `domain` (0 <= domain < grid[0] grid[1] grid[2], row-major over the
 * grid) from the last ctd_domains_compute; CTD_ERR_STATE before the first. */
int ctd_domains_info(ctd_domains *d, int32_t domain, ctd_domain_info *info);
/* The batched context behind the decomposition (model options, profiling, per-atom energies);
 * owned by the decomposition, do not destroy it. */
ctd_ctx *ctd_domains_context(ctd_domains *d);
const char *ctd_domains_last_error(ctd_domains *d);
void ctd_domains_destroy(ctd_domains *d);

/* ---- neighbour list without device allocation ------------------------------------------ */
/* The paper has no counterpart to this call; it exists for callers of this library that must
 * not allocate device memory: an MD code that manages a fixed device memory pool and cannot
 * let a library call cudaMalloc/cudaFree behind it, or a driver that must not allocate
 * between its own set-up and teardown.
 *
 * It finds the same pair set as ctd_build_neighbors (same wrap, same cell search, same FP64
 * pair test with cutoff + skin) without a context and without allocating: every scratch
 * array lives in one static device array of about 4 MB that each GPU loading this library
 * holds until the process exits.  Limits: n <= CTD_NOALLOC_MAX_ATOMS atoms and at most
 * CTD_NOALLOC_MAX_CELLS search cells (cell volume / (cutoff + skin)^3, roughly); beyond
 * either the call returns CTD_ERR_INVALID_ARG and does nothing.
 *
 * positions: device doubles [n][3] (any atom order, need not be wrapped); cell: host
 * double[9] (rows = lattice vectors).  pair_i, pair_j: device int32 [cap]; pair_shift: device
 * int8 [cap][3].  They receive the pairs in the caller's atom indices (grouped by atom, not
 * sorted) with the image shift relative to the positions passed in: the pair's vector is
 * x_j - x_i + shift[0] a + shift[1] b + shift[2] c for those positions, wrapped or not.  If a
 * shift does not fit int8 (positions more than ~127 cells outside the cell) the call returns
 * CTD_ERR_INVALID_ARG.  *n_pairs (host) receives the number of pairs; if it exceeds cap (or
 * INT32_MAX) nothing is written and CTD_ERR_CAPACITY is returned, so the caller can size its
 * arrays and call again.  Non-finite positions: CTD_ERR_NONFINITE.
 * cuda_stream: the cudaStream_t to run on (NULL = default stream); the call synchronises it and
 * copies counts to host memory, so it must not be called on a stream that is being captured
 * into a CUDA graph (it returns CTD_ERR_INVALID_ARG there).
 *
 * The first call on each device looks up the device address of the static array (with that
 * device current).  All calls share the one array, and each starts by clearing the parts that
 * must start at zero; calls that overlap on the GPU (different streams or threads at once)
 * race on it and must be serialised by the caller. */
#define CTD_NOALLOC_MAX_ATOMS 32768
#define CTD_NOALLOC_MAX_CELLS 32768
int ctd_neighbors_noalloc(int64_t n, const double *positions, const double cell[9], double cutoff,
                          double skin, int32_t *pair_i, int32_t *pair_j, int8_t *pair_shift,
                          int64_t cap, int64_t *n_pairs, void *cuda_stream);

/* ---- failure detection self-test ------------------------------------------------------------ */
/* Runs, on the context's stream, the path a tensor-core kernel takes when a bounded device wait
 * gives up: one CTA allocates tensor memory, waits on an mbarrier that nothing arrives on for
 * limit_ms (0 < limit_ms <= 2000), records the timeout, frees the tensor memory and returns.
 * Returns CTD_ERR_TIMEOUT (the expected outcome; the context stays usable) and, in *waited_ms
 * (may be NULL), how long the wait lasted.  Nothing faults or hangs. */
int ctd_selftest_wait(ctd_ctx *ctx, double limit_ms, double *waited_ms);

/* Text of the last failure on this context (never NULL). */
const char *ctd_last_error(ctd_ctx *ctx);

/* Release every device buffer and the context (and its stream if it created one). */
void ctd_destroy(ctd_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* CTD_PAINN_H */
