// serve.cu -- continuous-batching MD server: many independent replicas of uneven size resident
// on one GPU, advanced together one velocity-Verlet step at a time.
//
// Each admitted replica keeps its positions, velocities, masses, species, neighbour list and
// atom order on the device.  The resident replicas are packed into one batched system (atoms
// concatenated, per-replica neighbour lists concatenated with offsets; no edge crosses two
// replicas), so every stage of a step -- integrator, per-step prune, every model kernel, the
// force assembly -- runs as one launch over all of them.  Requests wait in a FIFO queue and are
// admitted between steps while the HBM budget and the replica cap allow; a replica leaves when
// its step count is reached and its final state is kept for polling.  Per-replica energies,
// virials and displacements come from segmented reductions whose order depends only on the
// replica itself, so a replica's trajectory is the same alone and in any mix.
//
// A queued request may carry a Nose-Hoover chain (Methods, "MD simulations": NVT).  Its chain
// state is one row of the batch's chain table; one thread per replica takes the chain half
// steps, and the velocity factors enter the masked kick and one scaling pass (factor 1 for
// replicas without a thermostat, so they are unaffected by the others).
//
// The paper's buffering rules (Results, "Runtime optimizations and buffering": capacities that
// only grow, repeat with larger buffers) apply to the batch arrays as to a single system.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <unordered_map>

#include "ctx.cuh"

namespace ctd {

struct RepDesc {
  const int32_t* vrow;
  const int32_t* vcol;
  const float4* vbase;
  const int32_t* vrev;
  int64_t atom_off, edge_off;
  int32_t n, nv;
};

// Concatenate per-replica Verlet lists (local indices) into the batch list (global indices).
__global__ void k_concat_verlet(const RepDesc* __restrict__ reps, int32_t* __restrict__ vrow,
                                int32_t* __restrict__ vcol, float4* __restrict__ vbase, int32_t* __restrict__ vrev) {
  const RepDesc d = reps[blockIdx.y];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= (int64_t)d.n || k < d.nv;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (k <= d.n) vrow[d.atom_off + k] = (int32_t)(d.edge_off + d.vrow[k]);
    if (k < d.nv) {
      vcol[d.edge_off + k] = (int32_t)(d.atom_off + d.vcol[k]);
      vbase[d.edge_off + k] = d.vbase[k];
      vrev[d.edge_off + k] = (int32_t)(d.edge_off + d.vrev[k]);
    }
  }
}

// Per-replica reductions, one block per replica, fixed order (independent of the batch).
// out[r*12 + 0] = sum of per-atom energies, [1] = kinetic energy (eV), [2] = max |d|^2,
// [3..11] = virial.
__global__ void k_rep_reduce(const int64_t* __restrict__ aoff, const int32_t* __restrict__ arow,
                             const float* __restrict__ eatom, const double* __restrict__ mass,
                             const double* __restrict__ vel, const float4* __restrict__ delta,
                             const float4* __restrict__ ar, const float4* __restrict__ hedge, int with_virial,
                             double* __restrict__ out) {
  __shared__ double sh[12][kThreads / 32];
  const int64_t a0 = aoff[blockIdx.x], a1 = aoff[blockIdx.x + 1];
  double acc[12];
  for (int q = 0; q < 12; ++q) acc[q] = 0.0;
  constexpr double kAccConv = 9.648533212331002e-3;
  for (int64_t i = a0 + threadIdx.x; i < a1; i += blockDim.x) {
    acc[0] += (double)eatom[i];
    acc[1] += 0.5 * mass[i] * (vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] + vel[3 * i + 2] * vel[3 * i + 2]) /
              kAccConv;
    const float4 d = delta[i];
    acc[2] = fmax(acc[2], (double)(d.x * d.x + d.y * d.y + d.z * d.z));
    if (with_virial)
      for (int e = arow[i]; e < arow[i + 1]; ++e) {
        const float4 r = ar[e], h = hedge[e];
        const float rr[3] = {r.x, r.y, r.z}, hh[3] = {h.x, h.y, h.z};
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) acc[3 + 3 * p + q] += (double)rr[p] * (double)hh[q];
      }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int q = 0; q < 12; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) {
      const double x = __shfl_xor_sync(0xffffffffu, v, o);
      v = q == 2 ? fmax(v, x) : v + x;
    }
    if (lane == 0) sh[q][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    const int q = threadIdx.x;
    double v = q == 2 ? 0.0 : 0.0;
    for (int k = 0; k < kThreads / 32; ++k) v = q == 2 ? fmax(v, sh[q][k]) : v + sh[q][k];
    out[(int64_t)blockIdx.x * 12 + q] = v;
  }
}

// Velocity-Verlet halves for replicas whose flag says "integrating" (a replica's first step
// only evaluates its forces).  g (may be null): per-replica factor of the thermostat's half step,
// applied to the velocities before the kick (1 for replicas without a thermostat).
__global__ void k_kick_drift_masked(int64_t n, double dt, const float* __restrict__ force, const double* __restrict__ mass,
                                    const int32_t* __restrict__ rep, const int32_t* __restrict__ flags,
                                    const double* __restrict__ g, double* __restrict__ x, double* __restrict__ v) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n || !(flags[rep[k]] & 1)) return;
  const double gk = g ? g[rep[k]] : 1.0;
  const double s = 0.5 * dt * 9.648533212331002e-3 / mass[k];
  for (int c = 0; c < 3; ++c) {
    const double vc = gk * v[3 * k + c] + s * (double)force[3 * k + c];
    v[3 * k + c] = vc;
    x[3 * k + c] += dt * vc;
  }
}
__global__ void k_kick_masked(int64_t n, double dt, const float* __restrict__ force, const double* __restrict__ mass,
                              const int32_t* __restrict__ rep, const int32_t* __restrict__ flags, double* __restrict__ v) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n || !(flags[rep[k]] & 1)) return;
  const double s = 0.5 * dt * 9.648533212331002e-3 / mass[k];
  for (int c = 0; c < 3; ++c) v[3 * k + c] += s * (double)force[3 * k + c];
}
__global__ void k_fill_i32(int64_t n, int32_t value, int32_t* __restrict__ out) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n) out[k] = value;
}
__global__ void k_iota(int64_t n, int32_t* __restrict__ out) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n) out[k] = (int32_t)k;
}

static inline unsigned blk(int64_t w) { return (unsigned)((w + kThreads - 1) / kThreads); }

constexpr int kChainStride = 40;   // doubles per replica: xi [M], vxi [M], last factor (M <= 16)

}  // namespace ctd

using namespace ctd;

namespace {

struct Replica {
  int64_t id = 0, n = 0;
  int32_t nsteps = 0, done = 0;
  int state = 0;          // 0 queued, 1 resident, 2 finished
  bool integrating = false;
  std::vector<int32_t> z;
  std::vector<double> m, x, v;
  double H[9];
  double skin = 1.0;
  std::vector<double> epot, ekin;
  double virial[9] = {0};
  int64_t off = 0;
  CellGeom geom{};
  int64_t ncell = 0;
  DBuf vrow, vcol, vbase, vrev, uperm;
  int64_t nv = 0;
  size_t est_bytes = 0;
  int32_t rebuilds = 0;
  std::vector<double> out_x, out_v;
  // Nose-Hoover chain (chain length 0: NVE); the chain state lives on the device while the
  // replica is resident and in `chain` otherwise
  int nhc_M = 0;
  double nhc_T = 0.0, nhc_tau = 0.0;
  std::vector<double> chain, eth;
};

}  // namespace

struct ctd_server {
  ctd_ctx* c = nullptr;
  double dt = 1.0;
  int32_t max_replicas = 1024;
  int64_t next_id = 1;
  std::deque<Replica*> queue;
  std::vector<Replica*> resident;
  std::unordered_map<int64_t, Replica*> reps;
  size_t resident_est = 0;
  // batch bookkeeping (device)
  DBuf rep_table, rep_off, rep_of_atom, rep_flags, rep_out;
  // thermostats of the resident replicas (when any has one): parameters, chain states,
  // kinetic energy after the last step, velocity factors, chain energies
  DBuf rep_np, rep_chain, rep_ke, rep_g, rep_eth;
  bool any_nvt = false;
  // staging for repacking the batch arrays
  DBuf st_x, st_xref, st_v, st_m, st_z, st_f;
  // build scratch (largest replica)
  DBuf b_xw, b_wrap, b_cell, b_ccount, b_cstart, b_cursor, b_tmp, b_perm, b_inv, b_xws, b_xnew, b_count, b_img,
      b_scan, b_i32, b_d3;
  bool lists_dirty = true;
  std::string err;
  // The step's device work after the rebuild decisions (prune, model, second kick, per-replica
  // sums) as a CUDA graph: captured once the batch layout has stayed the same over one eager
  // step, replayed while it stays the same (one graph launch instead of ~65 kernel launches).
  bool use_graph = true;
  cudaGraphExec_t gexec = nullptr;
  uint64_t gkey = 0, last_key = 0;
  int64_t graph_kernels = 0, steps_graph = 0, steps_eager = 0, captures = 0;
  std::vector<DBuf*> bufs() {
    return {&rep_table, &rep_off, &rep_of_atom, &rep_flags, &rep_out, &rep_np, &rep_chain, &rep_ke, &rep_g, &rep_eth, &st_x, &st_xref, &st_v, &st_m, &st_z, &st_f,
            &b_xw, &b_wrap, &b_cell, &b_ccount, &b_cstart, &b_cursor, &b_tmp, &b_perm, &b_inv, &b_xws, &b_xnew,
            &b_count, &b_img, &b_scan, &b_i32, &b_d3};
  }
};

namespace {

int sfail(ctd_server* s, int code, const std::string& msg) {
  s->err = msg;
  return code;
}

void free_buf(ctd_ctx* c, DBuf& b) {
  if (b.p) {
    ++c->alloc_gen;
    cudaFree(b.p);
    c->held -= b.bytes;
    c->used -= b.need;
    b.p = nullptr;
    b.bytes = 0;
    b.need = 0;
  }
}

// Device bytes a replica is expected to need (model buffers as evaluate() sizes them, edge
// lists, state), for admission.  Per Verlet edge: the replica's own list and the batch copy
// (vcol, vbase, vrev: 24 B each), the Verlet -> active map (4 B) and the active list (acol,
// ar, vidx, arev, aend, hedge: 48 B); 120 Verlet edges per atom bound the water and fcc
// densities at rc + skin = 6 A.  The batch buffers only grow and take 25 % headroom when they
// do (ensure()), so the estimate carries that factor too.
size_t estimate_bytes(const ctd_ctx* c, int64_t n) {
  const int64_t per_atom_state = 256;   // positions, references, velocities, masses, forces, ...
  const int64_t edges = 120 * n;
  const size_t raw = (size_t)n * (model_bytes_per_atom(c) + per_atom_state) + (size_t)edges * 100;
  return raw + raw / 4;
}

// Build the Verlet list of one resident replica from its current positions (segment of the
// batch arrays) and re-sort its segment by cell.
int build_replica(ctd_server* s, Replica& R) {
  ctd_ctx* c = s->c;
  cudaStream_t st = c->st;
  const int64_t n = R.n, off = R.off;
  int r = setup_geometry_into(c, R.geom, &R.ncell, R.H, c->desc.rc + R.skin);
  if (r) return r;
  const int64_t n1 = n > 0 ? n : 1;
  ENSURE(c, s->b_xw, sizeof(double) * 3 * n1);
  ENSURE(c, s->b_wrap, sizeof(int32_t) * 3 * n1);
  ENSURE(c, s->b_cell, sizeof(int32_t) * n1);
  ENSURE(c, s->b_ccount, sizeof(int32_t) * (R.ncell + 1));
  ENSURE(c, s->b_cstart, sizeof(int32_t) * (R.ncell + 1));
  ENSURE(c, s->b_cursor, sizeof(int32_t) * (R.ncell + 1));
  ENSURE(c, s->b_tmp, sizeof(int32_t) * n1);
  ENSURE(c, s->b_perm, sizeof(int32_t) * n1);
  ENSURE(c, s->b_inv, sizeof(int32_t) * n1);
  ENSURE(c, s->b_xws, sizeof(double) * 3 * n1);
  ENSURE(c, s->b_xnew, sizeof(double) * 3 * n1);
  ENSURE(c, s->b_count, sizeof(int32_t) * n1);
  ENSURE(c, s->b_scan, scan_temp_bytes(std::max<int64_t>(n1, R.ncell)) + 64);
  ENSURE(c, s->b_i32, sizeof(int32_t) * n1);
  ENSURE(c, s->b_d3, sizeof(double) * 3 * n1);
  ENSURE(c, R.vrow, sizeof(int32_t) * (n1 + 1));
  ENSURE(c, c->status, sizeof(int32_t) * 4);
  double* X = P<double>(c->x_s) + 3 * off;
  StageGuard sg(STG_BUILD);
  CUDA_OK(c, cudaMemsetAsync(c->status.p, 0, sizeof(int32_t), st));
  CUDA_OK(c, cudaMemsetAsync(s->b_ccount.p, 0, sizeof(int32_t) * R.ncell, st));
  CUDA_OK(c, cudaMemsetAsync(s->b_cursor.p, 0, sizeof(int32_t) * R.ncell, st));
  launch_wrap_bin(st, n, X, R.geom, P<double>(s->b_xw), P<int32_t>(s->b_wrap), P<int32_t>(s->b_cell),
                  P<int32_t>(s->b_ccount));
  launch_exclusive_scan(st, R.ncell, P<int32_t>(s->b_ccount), P<int32_t>(s->b_cstart), s->b_scan.p);
  launch_place(st, n, P<int32_t>(s->b_cell), P<int32_t>(s->b_cstart), P<int32_t>(s->b_cursor), P<int32_t>(s->b_tmp));
  launch_sort_cells(st, R.ncell, P<int32_t>(s->b_cstart), P<int32_t>(s->b_tmp), P<int32_t>(s->b_perm));
  launch_gather_sorted(st, n, P<int32_t>(s->b_perm), P<double>(s->b_xw), X, nullptr, P<double>(s->b_xws),
                       P<double>(s->b_xnew), nullptr, P<int32_t>(s->b_inv));
  launch_pair_search(st, false, n, P<double>(s->b_xws), P<int32_t>(s->b_cstart), R.geom, P<int32_t>(s->b_count),
                     nullptr, nullptr, nullptr, nullptr);
  launch_exclusive_scan(st, n, P<int32_t>(s->b_count), P<int32_t>(R.vrow), s->b_scan.p);
  int32_t total = 0;
  CUDA_OK(c, cudaMemcpyAsync(&total, P<int32_t>(R.vrow) + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CUDA_OK(c, cudaStreamSynchronize(st));
  if (total < 0) return fail(c, CTD_ERR_CAPACITY, "replica has more than 2^31 neighbour pairs");
  const int64_t e1 = total > 0 ? total : 1;
  ENSURE(c, R.vcol, sizeof(int32_t) * e1);
  ENSURE(c, R.vbase, sizeof(float4) * e1);
  ENSURE(c, R.vrev, sizeof(int32_t) * e1);
  ENSURE(c, s->b_img, sizeof(uint32_t) * e1);
  launch_pair_search(st, true, n, P<double>(s->b_xws), P<int32_t>(s->b_cstart), R.geom, P<int32_t>(s->b_count),
                     P<int32_t>(R.vrow), P<int32_t>(R.vcol), P<uint32_t>(s->b_img), P<float4>(R.vbase));
  launch_reverse(st, n, P<int32_t>(R.vrow), P<int32_t>(R.vcol), P<uint32_t>(s->b_img), P<int32_t>(R.vrev),
                 P<int>(c->status));
  R.nv = total;
  // re-sort the replica's segment: positions (= new reference), velocities, masses, species, order
  const int32_t* perm = P<int32_t>(s->b_perm);
  CUDA_OK(c, cudaMemcpyAsync(X, s->b_xnew.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
  CUDA_OK(c, cudaMemcpyAsync(P<double>(c->xref_s) + 3 * off, s->b_xnew.p, sizeof(double) * 3 * n,
                             cudaMemcpyDeviceToDevice, st));
  launch_gather_rows_d(st, n, 3, perm, P<double>(c->md_v) + 3 * off, P<double>(s->b_d3));
  CUDA_OK(c, cudaMemcpyAsync(P<double>(c->md_v) + 3 * off, s->b_d3.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
  launch_gather_rows_d(st, n, 1, perm, P<double>(c->md_m) + off, P<double>(s->b_d3));
  CUDA_OK(c, cudaMemcpyAsync(P<double>(c->md_m) + off, s->b_d3.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  launch_gather_i32(st, n, perm, P<int32_t>(c->z_s) + off, P<int32_t>(s->b_i32));
  CUDA_OK(c, cudaMemcpyAsync(P<int32_t>(c->z_s) + off, s->b_i32.p, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st));
  launch_gather_i32(st, n, perm, P<int32_t>(R.uperm), P<int32_t>(s->b_i32));
  CUDA_OK(c, cudaMemcpyAsync(R.uperm.p, s->b_i32.p, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st));
  r = check_status(c);
  if (r) return r;
  ++R.rebuilds;
  s->lists_dirty = true;
  return CTD_OK;
}

// Copy the final state of a resident replica (caller's atom order) to its host record.
int collect(ctd_server* s, Replica& R) {
  ctd_ctx* c = s->c;
  cudaStream_t st = c->st;
  const int64_t n = R.n;
  ENSURE(c, s->b_d3, sizeof(double) * 3 * (n > 0 ? n : 1));
  R.out_x.resize(3 * n);
  R.out_v.resize(3 * n);
  launch_scatter_rows_d(st, n, 3, P<int32_t>(R.uperm), P<double>(c->x_s) + 3 * R.off, P<double>(s->b_d3));
  CUDA_OK(c, cudaMemcpyAsync(R.out_x.data(), s->b_d3.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
  CUDA_OK(c, cudaStreamSynchronize(st));
  launch_scatter_rows_d(st, n, 3, P<int32_t>(R.uperm), P<double>(c->md_v) + 3 * R.off, P<double>(s->b_d3));
  CUDA_OK(c, cudaMemcpyAsync(R.out_v.data(), s->b_d3.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
  CUDA_OK(c, cudaStreamSynchronize(st));
  return CTD_OK;
}

// Repack the batch arrays for a new resident set: surviving replicas keep their (sorted)
// segments, new replicas are appended from their host data in the caller's order.
int repack(ctd_server* s, const std::vector<Replica*>& next) {
  ctd_ctx* c = s->c;
  cudaStream_t st = c->st;
  if (s->any_nvt && !s->resident.empty()) {   // chain states of the outgoing set back to the host
    const size_t R0 = s->resident.size();
    std::vector<double> h(kChainStride * R0);
    CUDA_OK(c, cudaMemcpyAsync(h.data(), s->rep_chain.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
    CUDA_OK(c, cudaStreamSynchronize(st));
    for (size_t k = 0; k < R0; ++k)
      if (s->resident[k]->nhc_M > 0)
        s->resident[k]->chain.assign(h.begin() + kChainStride * k, h.begin() + kChainStride * (k + 1));
  }
  int64_t N = 0;
  for (Replica* R : next) N += R->n;
  const int64_t N1 = N > 0 ? N : 1;
  ENSURE(c, s->st_x, sizeof(double) * 3 * N1);
  ENSURE(c, s->st_xref, sizeof(double) * 3 * N1);
  ENSURE(c, s->st_v, sizeof(double) * 3 * N1);
  ENSURE(c, s->st_m, sizeof(double) * N1);
  ENSURE(c, s->st_z, sizeof(int32_t) * N1);
  ENSURE(c, s->st_f, sizeof(float) * 3 * N1);   // forces carried into the next half kick
  int64_t off = 0;
  for (Replica* R : next) {
    const size_t n = (size_t)R->n;
    if (R->state == 1) {   // already resident: move its segment
      CUDA_OK(c, cudaMemcpyAsync(P<double>(s->st_x) + 3 * off, P<double>(c->x_s) + 3 * R->off, 24 * n, cudaMemcpyDeviceToDevice, st));
      CUDA_OK(c, cudaMemcpyAsync(P<double>(s->st_xref) + 3 * off, P<double>(c->xref_s) + 3 * R->off, 24 * n, cudaMemcpyDeviceToDevice, st));
      CUDA_OK(c, cudaMemcpyAsync(P<double>(s->st_v) + 3 * off, P<double>(c->md_v) + 3 * R->off, 24 * n, cudaMemcpyDeviceToDevice, st));
      CUDA_OK(c, cudaMemcpyAsync(P<double>(s->st_m) + off, P<double>(c->md_m) + R->off, 8 * n, cudaMemcpyDeviceToDevice, st));
      CUDA_OK(c, cudaMemcpyAsync(P<int32_t>(s->st_z) + off, P<int32_t>(c->z_s) + R->off, 4 * n, cudaMemcpyDeviceToDevice, st));
      CUDA_OK(c, cudaMemcpyAsync(P<float>(s->st_f) + 3 * off, P<float>(c->force_s) + 3 * R->off, 12 * n, cudaMemcpyDeviceToDevice, st));
    } else {               // new: host data, caller's order
      CUDA_OK(c, cudaMemcpyAsync(P<double>(s->st_x) + 3 * off, R->x.data(), 24 * n, cudaMemcpyHostToDevice, st));
      CUDA_OK(c, cudaMemcpyAsync(P<double>(s->st_xref) + 3 * off, R->x.data(), 24 * n, cudaMemcpyHostToDevice, st));
      CUDA_OK(c, cudaMemcpyAsync(P<double>(s->st_v) + 3 * off, R->v.data(), 24 * n, cudaMemcpyHostToDevice, st));
      CUDA_OK(c, cudaMemcpyAsync(P<double>(s->st_m) + off, R->m.data(), 8 * n, cudaMemcpyHostToDevice, st));
      CUDA_OK(c, cudaMemcpyAsync(P<int32_t>(s->st_z) + off, R->z.data(), 4 * n, cudaMemcpyHostToDevice, st));
    }
    R->off = off;
    off += R->n;
  }
  CUDA_OK(c, cudaStreamSynchronize(st));   // host vectors of new replicas are read before they change
  std::swap(c->x_s, s->st_x);
  std::swap(c->xref_s, s->st_xref);
  std::swap(c->md_v, s->st_v);
  std::swap(c->md_m, s->st_m);
  std::swap(c->z_s, s->st_z);
  std::swap(c->force_s, s->st_f);
  c->n = N;
  // per-replica tables
  const int64_t R = (int64_t)next.size();
  ENSURE(c, s->rep_off, sizeof(int64_t) * (R + 1));
  ENSURE(c, s->rep_of_atom, sizeof(int32_t) * N1);
  ENSURE(c, s->rep_flags, sizeof(int32_t) * (R > 0 ? R : 1));
  ENSURE(c, s->rep_out, sizeof(double) * 12 * (R > 0 ? R : 1));
  std::vector<int64_t> offs(R + 1, 0);
  for (int64_t k = 0; k < R; ++k) offs[k + 1] = offs[k] + next[k]->n;
  CUDA_OK(c, cudaMemcpyAsync(s->rep_off.p, offs.data(), sizeof(int64_t) * (R + 1), cudaMemcpyHostToDevice, st));
  for (int64_t k = 0; k < R; ++k)
    if (next[k]->n > 0) {
      LaunchScope ls_(st);
      k_fill_i32<<<blk(next[k]->n), kThreads, 0, st>>>(next[k]->n, (int32_t)k, P<int32_t>(s->rep_of_atom) + offs[k]);
    }
  // thermostat tables in the new order
  s->any_nvt = false;
  for (Replica* Rp : next) s->any_nvt = s->any_nvt || Rp->nhc_M > 0;
  if (s->any_nvt) {
    const int64_t R1 = R > 0 ? R : 1;
    ENSURE(c, s->rep_np, sizeof(NhcParams) * R1);
    ENSURE(c, s->rep_chain, sizeof(double) * kChainStride * R1);
    ENSURE(c, s->rep_ke, sizeof(double) * R1);
    ENSURE(c, s->rep_g, sizeof(double) * R1);
    ENSURE(c, s->rep_eth, sizeof(double) * R1);
    std::vector<NhcParams> np(R);
    std::vector<double> ch(kChainStride * R, 0.0), ke(R, 0.0);
    for (int64_t k = 0; k < R; ++k) {
      const Replica& Q = *next[k];
      NhcParams& p = np[k];
      memset(&p, 0, sizeof(p));
      p.M = Q.nhc_M;
      if (Q.nhc_M > 0) {   // Nf = 3n - 3: the centre of mass is at rest
        p.kT = 8.617333262e-5 * Q.nhc_T;
        p.Nf = 3.0 * (double)Q.n - 3.0;
        for (int j = 0; j < p.M; ++j) p.Q[j] = (j == 0 ? p.Nf : 1.0) * p.kT * Q.nhc_tau * Q.nhc_tau;
        std::copy(Q.chain.begin(), Q.chain.end(), ch.begin() + kChainStride * k);
      }
      if (!Q.ekin.empty()) ke[k] = Q.ekin.back();
    }
    CUDA_OK(c, cudaMemcpyAsync(s->rep_np.p, np.data(), sizeof(NhcParams) * R, cudaMemcpyHostToDevice, st));
    CUDA_OK(c, cudaMemcpyAsync(s->rep_chain.p, ch.data(), sizeof(double) * ch.size(), cudaMemcpyHostToDevice, st));
    CUDA_OK(c, cudaMemcpyAsync(s->rep_ke.p, ke.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st));
  }
  CUDA_OK(c, cudaStreamSynchronize(st));
  s->resident = next;
  s->lists_dirty = true;
  return CTD_OK;
}

int concat_lists(ctd_server* s) {
  ctd_ctx* c = s->c;
  cudaStream_t st = c->st;
  std::vector<RepDesc> d;
  int64_t E = 0, maxw = 1;
  for (Replica* R : s->resident) {
    RepDesc q;
    q.vrow = P<int32_t>(R->vrow);
    q.vcol = P<int32_t>(R->vcol);
    q.vbase = P<float4>(R->vbase);
    q.vrev = P<int32_t>(R->vrev);
    q.atom_off = R->off;
    q.edge_off = E;
    q.n = (int32_t)R->n;
    q.nv = (int32_t)R->nv;
    d.push_back(q);
    E += R->nv;
    maxw = std::max<int64_t>(maxw, std::max<int64_t>(R->n + 1, R->nv));
  }
  if (E > INT32_MAX) return fail(c, CTD_ERR_CAPACITY, "batch has more than 2^31 neighbour pairs");
  const int64_t N1 = c->n > 0 ? c->n : 1, E1 = E > 0 ? E : 1;
  ENSURE(c, c->vrow, sizeof(int32_t) * (N1 + 1));
  ENSURE(c, c->vcol, sizeof(int32_t) * E1);
  ENSURE(c, c->vbase, sizeof(float4) * E1);
  ENSURE(c, c->vrev, sizeof(int32_t) * E1);
  ENSURE(c, c->v2a, sizeof(int32_t) * E1);
  ENSURE(c, s->rep_table, sizeof(RepDesc) * (d.size() > 0 ? d.size() : 1));
  ENSURE(c, c->scan_tmp, scan_temp_bytes(N1) + 64);
  if (!d.empty()) {
    CUDA_OK(c, cudaMemcpyAsync(s->rep_table.p, d.data(), sizeof(RepDesc) * d.size(), cudaMemcpyHostToDevice, st));
    dim3 grid((unsigned)std::min<int64_t>((maxw + kThreads - 1) / kThreads, 4096), (unsigned)d.size());
    LaunchScope ls_(st);
    k_concat_verlet<<<grid, kThreads, 0, st>>>(P<RepDesc>(s->rep_table), P<int32_t>(c->vrow), P<int32_t>(c->vcol),
                                               P<float4>(c->vbase), P<int32_t>(c->vrev));
  } else {
    CUDA_OK(c, cudaMemsetAsync(c->vrow.p, 0, sizeof(int32_t), st));
  }
  CUDA_OK(c, cudaStreamSynchronize(st));   // the descriptor table is host memory until here
  c->n_verlet = E;
  s->lists_dirty = false;
  return CTD_OK;
}

void release(ctd_server* s, Replica* R) {
  free_buf(s->c, R->vrow);
  free_buf(s->c, R->vcol);
  free_buf(s->c, R->vbase);
  free_buf(s->c, R->vrev);
  free_buf(s->c, R->uperm);
}

}  // namespace

extern "C" {

namespace {

void drop_graph(ctd_server* s) {
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  s->gexec = nullptr;
  s->gkey = 0;
  s->graph_kernels = 0;
}

// Everything a captured step depends on besides device memory contents: the buffers (by their
// allocation generation), the batch size and layout, the thermostat mode and the model options.
uint64_t layout_key(const ctd_server* s, int64_t nres) {
  const ctd_ctx* c = s->c;
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
  mix(c->alloc_gen); mix((uint64_t)c->n); mix((uint64_t)nres); mix(s->any_nvt ? 1 : 0);
  mix(c->mw.tc_adjoint); mix(c->mw.tc_message); mix((uint64_t)c->mw.edge_chunk_rows);
  mix((uint64_t)c->desc.precision); mix(c->use_ew); mix(c->use_near);
  // a model without layers clears the per-edge gradients with a memset sized by the Verlet list
  if (c->desc.T == 0) mix((uint64_t)c->n_verlet);
  return h == 0 ? 1 : h;
}

// Step part 5-6: prune, forces of the whole batch, second half kick, per-replica energies and
// virial, thermostat half step.  No host synchronisation, so that it can be captured.
int step_device(ctd_server* s, int64_t nres) {
  ctd_ctx* c = s->c;
  cudaStream_t st = c->st;
  const int64_t N = c->n;
  int r = prune(c, nullptr);
  if (r) return r;
  r = evaluate(c, true);
  if (r) return r;
  StageGuard sg(STG_MD);
  {
    LaunchScope ls_(st);
    k_kick_masked<<<blk(N), kThreads, 0, st>>>(N, s->dt, P<float>(c->force_s), P<double>(c->md_m),
                                               P<int32_t>(s->rep_of_atom), P<int32_t>(s->rep_flags),
                                               P<double>(c->md_v));
  }
  {
    LaunchScope ls_(st);
    k_rep_reduce<<<(unsigned)nres, kThreads, 0, st>>>(P<int64_t>(s->rep_off), P<int32_t>(c->arow),
                                                     P<float>(c->eatom), P<double>(c->md_m), P<double>(c->md_v),
                                                     P<float4>(c->delta), P<float4>(c->ar), P<float4>(c->hedge), 1,
                                                     P<double>(s->rep_out));
  }
  if (s->any_nvt) {
    launch_rep_nhc_half(st, (int)nres, P<NhcParams>(s->rep_np), 0.5 * s->dt, P<double>(s->rep_out) + 1, 12,
                        P<int32_t>(s->rep_flags), P<double>(s->rep_chain), kChainStride, P<double>(s->rep_g),
                        P<double>(s->rep_ke), P<double>(s->rep_eth));
    launch_scale_v_rep(st, N, P<int32_t>(s->rep_of_atom), P<double>(s->rep_g), P<double>(c->md_v));
  }
  return CTD_OK;
}

// Captures step_device into s->gexec; false (nothing launched, capture state cleared) if the
// capture does not complete (a buffer would have had to grow, or a call is not capturable).
bool capture_step(ctd_server* s, int64_t nres, uint64_t key) {
  ctd_ctx* c = s->c;
  drop_graph(s);
  cudaGraph_t g = nullptr;
  c->capturing = true;
  int r = CTD_ERR_CUDA;
  if (cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    r = step_device(s, nres);
    if (cudaStreamEndCapture(c->st, &g) != cudaSuccess) r = CTD_ERR_CUDA;
  }
  c->capturing = false;
  bool ok = r == CTD_OK && g && layout_key(s, nres) == key && cudaGraphInstantiate(&s->gexec, g, 0) == cudaSuccess;
  if (ok) {
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    int64_t kern = 0;
    for (size_t k = 0; k < nn; ++k) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[k], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kern;
    }
    s->graph_kernels = kern;
    s->gkey = key;
    ++s->captures;
  } else {
    s->gexec = nullptr;
    cudaGetLastError();
    c->err.clear();
  }
  if (g) cudaGraphDestroy(g);
  return ok;
}

}  // namespace

int ctd_serve_create(ctd_server** out, const ctd_model_desc* desc, const void* params, size_t nbytes,
                     size_t hbm_budget_bytes, int32_t max_replicas, double dt, void* cuda_stream) {
  // replicas index the y dimension of the list concatenation grid (at most 65,535)
  if (!out || !desc || !(dt > 0.0) || max_replicas < 1 || max_replicas > 65535) return CTD_ERR_INVALID_ARG;
  *out = nullptr;
  ctd_ctx* c = nullptr;
  int r = ctd_create(&c, desc, hbm_budget_bytes, cuda_stream);
  if (r) return r;
  r = ctd_load_params(c, params, nbytes);
  if (r) {
    ctd_destroy(c);
    return r;
  }
  ctd_server* s = new ctd_server();
  s->c = c;
  s->dt = dt;
  s->max_replicas = max_replicas;
  *out = s;
  return CTD_OK;
}

void ctd_serve_destroy(ctd_server* s) {
  if (!s) return;
  if (s->c) cudaStreamSynchronize(s->c->st);
  drop_graph(s);
  for (auto& kv : s->reps) {
    release(s, kv.second);
    delete kv.second;
  }
  for (DBuf* b : s->bufs()) free_buf(s->c, *b);
  ctd_destroy(s->c);
  delete s;
}

const char* ctd_serve_last_error(ctd_server* s) {
  if (!s) return "null server";
  return s->err.empty() ? ctd_last_error(s->c) : s->err.c_str();
}

int ctd_serve_submit(ctd_server* s, int64_t n, const int32_t* species, const double* masses, const double* positions,
                     const double* velocities, const double cell[9], double skin, int32_t nsteps, int64_t* request_id) {
  if (!s) return CTD_ERR_INVALID_ARG;
  if (n <= 0 || !species || !masses || !positions || !velocities || !cell || !(skin >= 0.0) || nsteps < 0 ||
      !request_id)
    return sfail(s, CTD_ERR_INVALID_ARG, "bad request");
  if (!finite_cell(cell)) return sfail(s, CTD_ERR_INVALID_ARG, "cell is singular or not finite");
  for (int64_t k = 0; k < n; ++k)
    if (!(masses[k] > 0.0) || species[k] < 0 || species[k] >= s->c->desc.n_species)
      return sfail(s, CTD_ERR_INVALID_ARG, "bad mass or species");
  Replica* R = new Replica();
  R->id = s->next_id++;
  R->n = n;
  R->nsteps = nsteps;
  R->z.assign(species, species + n);
  R->m.assign(masses, masses + n);
  R->x.assign(positions, positions + 3 * n);
  R->v.assign(velocities, velocities + 3 * n);
  memcpy(R->H, cell, sizeof(R->H));
  R->skin = skin;
  R->est_bytes = estimate_bytes(s->c, n);
  if (s->c->budget && R->est_bytes > s->c->budget) {
    delete R;
    return sfail(s, CTD_ERR_OUT_OF_BUDGET, "request can never fit the HBM budget");
  }
  s->reps[R->id] = R;
  s->queue.push_back(R);
  *request_id = R->id;
  return CTD_OK;
}

int ctd_serve_step(ctd_server* s, int32_t* n_resident, int32_t* n_admitted, int32_t* n_finished) {
  if (!s) return CTD_ERR_INVALID_ARG;
  ctd_ctx* c = s->c;
  Bind bind_(c);
  cudaStream_t st = c->st;
  s->err.clear();
  int32_t admitted = 0, finished = 0;
  // 1. retire replicas that reached their step count
  std::vector<Replica*> next;
  bool changed = false;
  for (Replica* R : s->resident) {
    if (R->integrating && R->done >= R->nsteps) {
      int r = collect(s, *R);
      if (r) return r;
      R->state = 2;
      release(s, R);
      s->resident_est -= R->est_bytes;
      ++finished;
      changed = true;
    } else {
      next.push_back(R);
    }
  }
  // 2. admit from the queue (FIFO) while the budget and the replica cap allow
  std::vector<Replica*> fresh;
  while (!s->queue.empty() && (int32_t)next.size() < s->max_replicas) {
    Replica* R = s->queue.front();
    if (c->budget && s->resident_est + R->est_bytes > c->budget) break;
    s->queue.pop_front();
    s->resident_est += R->est_bytes;
    next.push_back(R);
    fresh.push_back(R);
    ++admitted;
    changed = true;
  }
  if (changed) {
    int r = repack(s, next);
    if (r) return r;
    for (Replica* R : fresh) {
      R->state = 1;
      ENSURE(c, R->uperm, sizeof(int32_t) * (size_t)R->n);
      { LaunchScope ls_(st); k_iota<<<blk(R->n), kThreads, 0, st>>>(R->n, P<int32_t>(R->uperm)); }
      r = build_replica(s, *R);
      if (r) return r;
      R->x.clear(); R->x.shrink_to_fit();
      R->v.clear(); R->v.shrink_to_fit();
    }
  }
  const int64_t nres = (int64_t)s->resident.size();
  if (n_resident) *n_resident = (int32_t)nres;
  if (n_admitted) *n_admitted = admitted;
  if (n_finished) *n_finished = finished;
  if (nres == 0) return CTD_OK;
  // per-replica integration flags
  std::vector<int32_t> flags(nres);
  for (int64_t k = 0; k < nres; ++k) flags[k] = s->resident[k]->integrating ? 1 : 0;
  CUDA_OK(c, cudaMemcpyAsync(s->rep_flags.p, flags.data(), sizeof(int32_t) * nres, cudaMemcpyHostToDevice, st));
  const int64_t N = c->n;
  ENSURE(c, c->force_s, sizeof(float) * 3 * (N > 0 ? N : 1));
  ENSURE(c, c->delta, sizeof(float4) * (N > 0 ? N : 1));
  ENSURE(c, c->maxd, sizeof(unsigned int) * 4);
  // 3. thermostat half step (replicas with one), first half kick + drift
  {
    StageGuard sg(STG_MD);
    if (s->any_nvt)
      launch_rep_nhc_half(st, (int)nres, P<NhcParams>(s->rep_np), 0.5 * s->dt, P<double>(s->rep_ke), 1,
                          P<int32_t>(s->rep_flags), P<double>(s->rep_chain), kChainStride, P<double>(s->rep_g),
                          nullptr, nullptr);
    LaunchScope ls_(st);
    k_kick_drift_masked<<<blk(N), kThreads, 0, st>>>(N, s->dt, P<float>(c->force_s), P<double>(c->md_m),
                                                     P<int32_t>(s->rep_of_atom), P<int32_t>(s->rep_flags),
                                                     s->any_nvt ? P<double>(s->rep_g) : nullptr, P<double>(c->x_s),
                                                     P<double>(c->md_v));
  }
  // 4. per-replica displacement since its last build; rebuild the replicas past skin/2
  {
    StageGuard sg(STG_PRUNE);
    launch_delta(st, N, P<double>(c->x_s), P<double>(c->xref_s), P<float4>(c->delta), P<unsigned int>(c->maxd));
    LaunchScope ls_(st);
    k_rep_reduce<<<(unsigned)nres, kThreads, 0, st>>>(P<int64_t>(s->rep_off), nullptr, P<float>(c->force_s),
                                                     P<double>(c->md_m), P<double>(c->md_v), P<float4>(c->delta),
                                                     nullptr, nullptr, 0, P<double>(s->rep_out));
  }
  std::vector<double> ro(12 * nres);
  CUDA_OK(c, cudaMemcpyAsync(ro.data(), s->rep_out.p, sizeof(double) * 12 * nres, cudaMemcpyDeviceToHost, st));
  CUDA_OK(c, cudaStreamSynchronize(st));
  for (int64_t k = 0; k < nres; ++k) {
    Replica* R = s->resident[k];
    const double md = std::sqrt(ro[12 * k + 2]);
    if (!std::isfinite(md)) return sfail(s, CTD_ERR_NONFINITE, "non-finite positions in replica " + std::to_string(R->id));
    if (R->integrating && md > 0.5 * R->skin) {
      int r = build_replica(s, *R);
      if (r) return r;
    }
  }
  if (s->lists_dirty) {
    int r = concat_lists(s);
    if (r) return r;
  }
  // 5. forces of the whole batch; 6. second half kick, per-replica energies and virial,
  // thermostat half step from the kinetic energy after the kick and the velocity factor it
  // gives (kinetic energy recorded after it).  Replayed as a CUDA graph while the layout holds.
  ENSURE(c, c->status, sizeof(int32_t) * 4);
  CUDA_OK(c, cudaMemsetAsync(c->status.p, 0, sizeof(int32_t), st));
  const bool graphable = s->use_graph && !c->local() && !prof_recording() &&
                         !model_stores_edges(c->mw, c->desc.precision);
  const uint64_t key = layout_key(s, nres);
  bool launched = false;
  if (graphable && s->gexec && s->gkey == key) {
    CUDA_OK(c, cudaGraphLaunch(s->gexec, st));
    launched = true;
  } else if (graphable && key == s->last_key && capture_step(s, nres, key)) {
    CUDA_OK(c, cudaGraphLaunch(s->gexec, st));
    launched = true;
  }
  if (launched) {
    ++s->steps_graph;
    prof_count_launches(s->graph_kernels);
  } else {
    int r = step_device(s, nres);
    if (r) return r;
    ++s->steps_eager;
  }
  s->last_key = layout_key(s, nres);
  CUDA_OK(c, cudaMemcpyAsync(ro.data(), s->rep_out.p, sizeof(double) * 12 * nres, cudaMemcpyDeviceToHost, st));
  std::vector<double> ke(s->any_nvt ? nres : 0), eth(s->any_nvt ? nres : 0);
  if (s->any_nvt) {
    CUDA_OK(c, cudaMemcpyAsync(ke.data(), s->rep_ke.p, sizeof(double) * nres, cudaMemcpyDeviceToHost, st));
    CUDA_OK(c, cudaMemcpyAsync(eth.data(), s->rep_eth.p, sizeof(double) * nres, cudaMemcpyDeviceToHost, st));
  }
  int r = check_status(c);
  if (r) return r;
  for (int64_t k = 0; k < nres; ++k) {
    Replica* R = s->resident[k];
    R->epot.push_back(ro[12 * k + 0]);
    R->ekin.push_back(s->any_nvt ? ke[k] : ro[12 * k + 1]);
    if (R->nhc_M > 0) R->eth.push_back(eth[k]);
    for (int q = 0; q < 9; ++q) R->virial[q] = ro[12 * k + 3 + q];
    if (R->integrating) ++R->done;
    R->integrating = true;
  }
  return CTD_OK;
}

int ctd_serve_poll(ctd_server* s, int64_t request_id, int32_t* state, int32_t* steps_done, double* positions,
                   double* velocities, double* epot, double* ekin, double* virial) {
  if (!s) return CTD_ERR_INVALID_ARG;
  auto it = s->reps.find(request_id);
  if (it == s->reps.end()) return sfail(s, CTD_ERR_INVALID_ARG, "unknown request");
  Replica* R = it->second;
  if (state) *state = R->state;
  if (steps_done) *steps_done = R->done;
  if (R->state == 2) {
    if (positions) memcpy(positions, R->out_x.data(), sizeof(double) * R->out_x.size());
    if (velocities) memcpy(velocities, R->out_v.data(), sizeof(double) * R->out_v.size());
  }
  const size_t ne = R->epot.size();
  if (epot && ne) memcpy(epot, R->epot.data(), sizeof(double) * ne);
  if (ekin && ne) memcpy(ekin, R->ekin.data(), sizeof(double) * ne);
  if (virial) memcpy(virial, R->virial, sizeof(double) * 9);
  return CTD_OK;
}

int ctd_serve_snapshot(ctd_server* s, int64_t request_id, double* positions, double* velocities, int32_t* steps_done) {
  if (!s) return CTD_ERR_INVALID_ARG;
  Bind bind_(s->c);
  auto it = s->reps.find(request_id);
  if (it == s->reps.end()) return sfail(s, CTD_ERR_INVALID_ARG, "unknown request");
  Replica* R = it->second;
  if (R->state != 1) return sfail(s, CTD_ERR_STATE, "request is not resident");
  int r = collect(s, *R);   // current state in the caller's order, the replica stays resident
  if (r) return r;
  if (positions) memcpy(positions, R->out_x.data(), sizeof(double) * R->out_x.size());
  if (velocities) memcpy(velocities, R->out_v.data(), sizeof(double) * R->out_v.size());
  if (steps_done) *steps_done = R->done;
  return CTD_OK;
}

int ctd_serve_set_thermostat(ctd_server* s, int64_t request_id, double temperature, double tau, int32_t chain,
                             const double* xi, const double* vxi) {
  if (!s) return CTD_ERR_INVALID_ARG;
  auto it = s->reps.find(request_id);
  if (it == s->reps.end()) return sfail(s, CTD_ERR_INVALID_ARG, "unknown request");
  Replica* R = it->second;
  if (R->state != 0) return sfail(s, CTD_ERR_STATE, "the thermostat is set while the request is queued");
  if (chain < 0 || chain > 16) return sfail(s, CTD_ERR_INVALID_ARG, "chain length must be 0..16");
  if (chain > 0) {
    if (!(temperature > 0.0 && std::isfinite(temperature) && tau > 0.0 && std::isfinite(tau)))
      return sfail(s, CTD_ERR_INVALID_ARG, "temperature and tau must be positive and finite");
    if (R->n < 2) return sfail(s, CTD_ERR_INVALID_ARG, "a thermostat needs at least two atoms");
    if (!xi != !vxi) return sfail(s, CTD_ERR_INVALID_ARG, "give both xi and vxi, or neither");
    if (xi)
      for (int j = 0; j < chain; ++j)
        if (!std::isfinite(xi[j]) || !std::isfinite(vxi[j]))
          return sfail(s, CTD_ERR_INVALID_ARG, "non-finite chain state");
  }
  R->nhc_M = chain;
  R->nhc_T = chain > 0 ? temperature : 0.0;
  R->nhc_tau = chain > 0 ? tau : 0.0;
  R->chain.assign(kChainStride, 0.0);
  if (chain > 0 && xi)
    for (int j = 0; j < chain; ++j) {
      R->chain[j] = xi[j];
      R->chain[chain + j] = vxi[j];
    }
  R->eth.clear();
  return CTD_OK;
}

int ctd_serve_thermostat(ctd_server* s, int64_t request_id, double* xi, double* vxi, double* ethermo) {
  if (!s) return CTD_ERR_INVALID_ARG;
  Bind bind_(s->c);
  auto it = s->reps.find(request_id);
  if (it == s->reps.end()) return sfail(s, CTD_ERR_INVALID_ARG, "unknown request");
  Replica* R = it->second;
  if (R->nhc_M == 0) return sfail(s, CTD_ERR_STATE, "request has no thermostat");
  const int M = R->nhc_M;
  std::vector<double> ch = R->chain;
  if (R->state == 1) {   // resident: the chain state is on the device
    const auto pos = std::find(s->resident.begin(), s->resident.end(), R);
    const size_t k = (size_t)(pos - s->resident.begin());
    ch.assign(kChainStride, 0.0);
    ctd_ctx* c = s->c;
    CUDA_OK(c, cudaMemcpyAsync(ch.data(), P<double>(s->rep_chain) + kChainStride * k, sizeof(double) * kChainStride,
                               cudaMemcpyDeviceToHost, c->st));
    CUDA_OK(c, cudaStreamSynchronize(c->st));
  }
  if (xi) memcpy(xi, ch.data(), sizeof(double) * M);
  if (vxi) memcpy(vxi, ch.data() + M, sizeof(double) * M);
  if (ethermo && !R->eth.empty()) memcpy(ethermo, R->eth.data(), sizeof(double) * R->eth.size());
  return CTD_OK;
}

int ctd_serve_stats(ctd_server* s, int64_t* resident_atoms, int32_t* resident_replicas, int32_t* queued,
                    int64_t* bytes_held) {
  if (!s) return CTD_ERR_INVALID_ARG;
  if (resident_atoms) *resident_atoms = s->c->n;
  if (resident_replicas) *resident_replicas = (int32_t)s->resident.size();
  if (queued) *queued = (int32_t)s->queue.size();
  if (bytes_held) *bytes_held = (int64_t)s->c->held;
  return CTD_OK;
}

int ctd_serve_use_graph(ctd_server* s, int32_t enable) {
  if (!s) return CTD_ERR_INVALID_ARG;
  Bind bind_(s->c);
  cudaStreamSynchronize(s->c->st);
  s->use_graph = enable != 0;
  drop_graph(s);
  s->last_key = 0;
  return CTD_OK;
}

int ctd_serve_graph_stats(ctd_server* s, int64_t* graph_steps, int64_t* eager_steps, int64_t* kernels_per_replay,
                          int64_t* captures) {
  if (!s) return CTD_ERR_INVALID_ARG;
  if (graph_steps) *graph_steps = s->steps_graph;
  if (eager_steps) *eager_steps = s->steps_eager;
  if (kernels_per_replay) *kernels_per_replay = s->graph_kernels;
  if (captures) *captures = s->captures;
  return CTD_OK;
}

}  // extern "C"
