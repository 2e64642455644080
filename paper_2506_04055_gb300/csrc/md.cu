// md.cu -- velocity-Verlet NVE kernels, output scatter to the caller's atom order and the
// deterministic FP64 reductions of energy / virial partials.
//
// Forces drive every MD step (arXiv 2506.04055, Results "Distributed potential computation");
// the integrator is velocity Verlet in FP64 on cell-sorted arrays.  Units: A, fs, amu, eV;
// acceleration (A/fs^2) = 9.648533212331002e-3 * F (eV/A) / m (amu).
#include "ctd_internal.cuh"

namespace ctd {

constexpr double kAcc = 9.648533212331002e-3;

// v = g v + dt/2 a(F);  x += dt v   (first half of velocity Verlet; g = *vscale, the thermostat's
// velocity factor of the preceding chain half step, or 1 without a thermostat)
__global__ void k_kick_drift(int64_t n, double dt, const float* __restrict__ force, const double* __restrict__ mass,
                             const double* __restrict__ vscale, double* __restrict__ x, double* __restrict__ v) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double g = vscale ? *vscale : 1.0;
  double s = 0.5 * dt * kAcc / mass[k];
  for (int c = 0; c < 3; ++c) {
    double vc = g * v[3 * k + c] + s * (double)force[3 * k + c];
    v[3 * k + c] = vc;
    x[3 * k + c] += dt * vc;
  }
}

// ---- Nose-Hoover chain (NVT; Methods "MD simulations": Nose-Hoover thermostat, damping tau) ----
// Chain of M thermostats (Martyna, Tuckerman, Klein 1996): dv_i/dt = F_i/m_i - vxi_1 v_i,
// dvxi_1/dt = (2K - Nf kT)/Q_1 - vxi_2 vxi_1, dvxi_j/dt = (Q_{j-1} vxi_{j-1}^2 - kT)/Q_j
// - vxi_{j+1} vxi_j, dxi_j/dt = vxi_j; Q_1 = Nf kT tau^2, Q_j = kT tau^2.  A chain half step of
// length h: vxi_M, then vxi_{M-1} .. vxi_1 each between two factors exp(-h vxi_{j+1} / 4), the
// velocity factor exp(-h vxi_1), xi_j += h vxi_j, and the mirrored sweep back up.  The chain is
// a handful of scalars: one thread advances it; the velocity factor is applied by the next kick.
// state: xi [M], vxi [M], the factor of the last half step [1].
__device__ double nhc_force(int j, double ke, const NhcParams& p, const double* vxi) {
  if (j == 0) return (2.0 * ke - p.Nf * p.kT) / p.Q[0];
  return (p.Q[j - 1] * vxi[j - 1] * vxi[j - 1] - p.kT) / p.Q[j];
}

// One chain half step of length h from the kinetic energy ke; returns the velocity factor and
// stores it in state[2M].
__device__ double nhc_half_step(const NhcParams& p, double h, double ke, double* state) {
  const int M = p.M;
  double* xi = state;
  double* vxi = state + M;
  vxi[M - 1] += 0.5 * h * nhc_force(M - 1, ke, p, vxi);
  for (int j = M - 2; j >= 0; --j) {
    const double e = exp(-0.25 * h * vxi[j + 1]);
    vxi[j] *= e;
    vxi[j] += 0.5 * h * nhc_force(j, ke, p, vxi);
    vxi[j] *= e;
  }
  const double g = exp(-h * vxi[0]);
  ke *= g * g;
  for (int j = 0; j < M; ++j) xi[j] += h * vxi[j];
  for (int j = 0; j < M - 1; ++j) {
    const double e = exp(-0.25 * h * vxi[j + 1]);
    vxi[j] *= e;
    vxi[j] += 0.5 * h * nhc_force(j, ke, p, vxi);
    vxi[j] *= e;
  }
  vxi[M - 1] += 0.5 * h * nhc_force(M - 1, ke, p, vxi);
  state[2 * M] = g;
  return g;
}

__global__ void k_nhc_half(NhcParams p, double h, const double* __restrict__ ke_in, double* __restrict__ state) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  nhc_half_step(p, h, *ke_in, state);
}

// Chain energy of one replica's state.
__device__ double nhc_chain_energy(const NhcParams& p, const double* state) {
  double e = 0.0;
  for (int j = 0; j < p.M; ++j)
    e += 0.5 * p.Q[j] * state[p.M + j] * state[p.M + j] + (j == 0 ? p.Nf * p.kT : p.kT) * state[j];
  return e;
}

// Served replicas, one thread each: replicas with a thermostat (M > 0) that integrate this step
// (flags bit 0) advance their chain from their kinetic energy ke[r * ke_stride]; the velocity
// factor goes to g[r] (1 for the others).  ke_after[r] receives the kinetic energy after the
// factor and eth[r] the chain energy (both may be null).
__global__ void k_rep_nhc_half(int R, const NhcParams* __restrict__ params, double h, const double* __restrict__ ke,
                               int ke_stride, const int32_t* __restrict__ flags, double* __restrict__ states,
                               int state_stride, double* __restrict__ g, double* __restrict__ ke_after,
                               double* __restrict__ eth) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const NhcParams p = params[r];
  const double k = ke[(int64_t)r * ke_stride];
  double* st = states + (int64_t)r * state_stride;
  double gr = 1.0;
  if (p.M > 0 && (flags[r] & 1)) gr = nhc_half_step(p, h, k, st);
  g[r] = gr;
  if (ke_after) ke_after[r] = k * gr * gr;
  if (eth) eth[r] = p.M > 0 ? nhc_chain_energy(p, st) : 0.0;
}

// v *= g[replica of the atom]
__global__ void k_scale_v_rep(int64_t n, const int32_t* __restrict__ rep, const double* __restrict__ g,
                              double* __restrict__ v) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double gk = g[rep[k]];
  for (int c = 0; c < 3; ++c) v[3 * k + c] *= gk;
}

// Energy of the chain: sum_j Q_j vxi_j^2 / 2 + Nf kT xi_1 + kT sum_{j>1} xi_j.
__global__ void k_nhc_energy(NhcParams p, const double* __restrict__ state, double* __restrict__ out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  *out = nhc_chain_energy(p, state);
}

__global__ void k_scale_v(int64_t n3, const double* __restrict__ g, double* __restrict__ v) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n3) v[k] *= *g;
}

// v += dt/2 a(F)   (second half)
__global__ void k_kick(int64_t n, double dt, const float* __restrict__ force, const double* __restrict__ mass,
                       double* __restrict__ v) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s = 0.5 * dt * kAcc / mass[k];
  for (int c = 0; c < 3; ++c) v[3 * k + c] += s * (double)force[3 * k + c];
}

// per-block partial sums of m v^2 / 2 (eV)
__global__ void k_kinetic(int64_t n, const double* __restrict__ mass, const double* __restrict__ v,
                          double* __restrict__ partials) {
  __shared__ double sb[kThreads / 32];
  double acc = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    acc += 0.5 * mass[k] * (v[3 * k] * v[3 * k] + v[3 * k + 1] * v[3 * k + 1] + v[3 * k + 2] * v[3 * k + 2]) / kAcc;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sb[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += sb[w];
    partials[blockIdx.x] = s;
  }
}

// out[c] = scale * sum_b partials[b * width + c], compensated (Neumaier) and in a fixed order:
// one block per column; thread t sums partials t, t + 256, ... then a pairwise tree over the
// threads carries the sums and their compensation terms.  The order depends only on nb, so the
// result is deterministic.  (A single warp walking the partials one by one spent ~170 us on
// GB300's FP64 latency chain for 608 partials.)
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads) k_sum_partials(int nb, int width, const double* __restrict__ partials,
                                                              double* __restrict__ out, double scale) {
  __shared__ double ss[kSumThreads], sc[kSumThreads];
  const int c = blockIdx.x, tid = threadIdx.x;
  double s = 0.0, comp = 0.0;
  for (int b = tid; b < nb; b += kSumThreads) {
    const double x = partials[(int64_t)b * width + c], t = s + x;
    comp += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  ss[tid] = s;
  sc[tid] = comp;
  __syncthreads();
  for (int h = kSumThreads / 2; h > 0; h >>= 1) {
    if (tid < h) {
      const double a = ss[tid], b = ss[tid + h], t = a + b;
      const double e = fabs(a) >= fabs(b) ? (a - t) + b : (b - t) + a;
      ss[tid] = t;
      sc[tid] = sc[tid] + sc[tid + h] + e;
    }
    __syncthreads();
  }
  if (tid == 0) out[c] = (ss[0] + sc[0]) * scale;
}

// out[perm[k]] = (double) in[k]  for [n][w] rows
__global__ void k_scatter_rows(int64_t n, int w, const int32_t* __restrict__ perm, const float* __restrict__ in,
                               double* __restrict__ out) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * w) return;
  int64_t k = idx / w;
  int c = (int)(idx % w);
  out[(int64_t)perm[k] * w + c] = (double)in[idx];
}

// out[perm[k]] = in[k]  (double rows) and the inverse gather
__global__ void k_scatter_rows_d(int64_t n, int w, const int32_t* __restrict__ perm, const double* __restrict__ in,
                                 double* __restrict__ out) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * w) return;
  int64_t k = idx / w;
  int c = (int)(idx % w);
  out[(int64_t)perm[k] * w + c] = in[idx];
}

__global__ void k_gather_rows_d(int64_t n, int w, const int32_t* __restrict__ perm, const double* __restrict__ in,
                                double* __restrict__ out) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * w) return;
  int64_t k = idx / w;
  int c = (int)(idx % w);
  out[idx] = in[(int64_t)perm[k] * w + c];
}

__global__ void k_gather_i32(int64_t n, const int32_t* __restrict__ perm, const int32_t* __restrict__ in,
                             int32_t* __restrict__ out) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  out[k] = in[perm[k]];
}

// flag non-finite entries of a double array
__global__ void k_check_finite(int64_t n, const double* __restrict__ a, int* status) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  if (!isfinite(a[k])) atomicOr(status, (int)ST_NONFINITE);
}

static inline unsigned nblk(int64_t w) { return (unsigned)((w + kThreads - 1) / kThreads); }

void launch_kick_drift(cudaStream_t st, int64_t n, double dt, const float* f, const double* m, const double* vscale,
                       double* x, double* v) {
  if (n) { LaunchScope ls_(st); k_kick_drift<<<nblk(n), kThreads, 0, st>>>(n, dt, f, m, vscale, x, v); }
}
void launch_nhc_half(cudaStream_t st, const NhcParams& p, double h, const double* ke, double* state) {
  LaunchScope ls_(st);
  k_nhc_half<<<1, 32, 0, st>>>(p, h, ke, state);
}
void launch_nhc_energy(cudaStream_t st, const NhcParams& p, const double* state, double* out) {
  LaunchScope ls_(st);
  k_nhc_energy<<<1, 32, 0, st>>>(p, state, out);
}
void launch_rep_nhc_half(cudaStream_t st, int R, const NhcParams* params, double h, const double* ke, int ke_stride,
                         const int32_t* flags, double* states, int state_stride, double* g, double* ke_after,
                         double* eth) {
  if (R > 0) {
    LaunchScope ls_(st);
    k_rep_nhc_half<<<(R + 127) / 128, 128, 0, st>>>(R, params, h, ke, ke_stride, flags, states, state_stride, g,
                                                   ke_after, eth);
  }
}
void launch_scale_v_rep(cudaStream_t st, int64_t n, const int32_t* rep, const double* g, double* v) {
  if (n) { LaunchScope ls_(st); k_scale_v_rep<<<nblk(n), kThreads, 0, st>>>(n, rep, g, v); }
}
void launch_scale_v(cudaStream_t st, int64_t n, const double* g, double* v) {
  if (n) { LaunchScope ls_(st); k_scale_v<<<nblk(3 * n), kThreads, 0, st>>>(3 * n, g, v); }
}
void launch_kick(cudaStream_t st, int64_t n, double dt, const float* f, const double* m, double* v) {
  if (n) { LaunchScope ls_(st); k_kick<<<nblk(n), kThreads, 0, st>>>(n, dt, f, m, v); }
}
void launch_kinetic(cudaStream_t st, int64_t n, const double* m, const double* v, double* partials, int nb) {
  { LaunchScope ls_(st); k_kinetic<<<nb, kThreads, 0, st>>>(n, m, v, partials); }
}
void launch_sum_partials(cudaStream_t st, int nb, int width, const double* partials, double* out, double scale) {
  if (width < 1) return;
  { LaunchScope ls_(st); k_sum_partials<<<width, kSumThreads, 0, st>>>(nb, width, partials, out, scale); }
}
void launch_scatter_rows(cudaStream_t st, int64_t n, int w, const int32_t* perm, const float* in, double* out) {
  if (n) { LaunchScope ls_(st); k_scatter_rows<<<nblk(n * w), kThreads, 0, st>>>(n, w, perm, in, out); }
}
void launch_scatter_rows_d(cudaStream_t st, int64_t n, int w, const int32_t* perm, const double* in, double* out) {
  if (n) { LaunchScope ls_(st); k_scatter_rows_d<<<nblk(n * w), kThreads, 0, st>>>(n, w, perm, in, out); }
}
void launch_gather_rows_d(cudaStream_t st, int64_t n, int w, const int32_t* perm, const double* in, double* out) {
  if (n) { LaunchScope ls_(st); k_gather_rows_d<<<nblk(n * w), kThreads, 0, st>>>(n, w, perm, in, out); }
}
void launch_gather_i32(cudaStream_t st, int64_t n, const int32_t* perm, const int32_t* in, int32_t* out) {
  if (n) { LaunchScope ls_(st); k_gather_i32<<<nblk(n), kThreads, 0, st>>>(n, perm, in, out); }
}
void launch_check_finite(cudaStream_t st, int64_t n, const double* a, int* status) {
  if (n) { LaunchScope ls_(st); k_check_finite<<<nblk(n), kThreads, 0, st>>>(n, a, status); }
}

}  // namespace ctd
