// neighbors.cu -- cell-list Verlet neighbour build and per-step pruning (sm_103a).
//
// The MD side builds neighbour lists with edges longer than the model cutoff so that they need
// not be rebuilt every step, and the model prunes edges longer than the cutoff every step
// (arXiv 2506.04055, Results "Distributed potential computation", pruning paragraph).
//
// Build (on rebuild only):
//   wrap_bin      s = G x, f = s - floor(s), x~ = f H (FP64, every op rounded separately),
//                 slab index per direction, atom counts per cell
//   scan + place  counting sort by cell; sort_cells makes the order within a cell ascending
//                 in the caller's index, so the whole build is deterministic
//   pair_search   one warp per atom, lanes over the atoms of each neighbour cell, the pair
//                 test in FP64 with __dmul_rn/__dadd_rn in the canonical order, warp-ballot
//                 compaction; run twice (count, then fill at scanned offsets)
//   reverse       rev[e] = index of (j <- i, -n) for e = (i <- j, n)
// Per step:
//   delta         d_i = x_i - x_ref,i (FP64 -> FP32) and the largest |d_i|^2 (skin trigger)
//   prune         r_e = b_e + (d_j - d_i) in FP32 with b_e the FP32 edge vector at build; keep
//                 |r_e| < rc (warp ballot, count then fill); rev of the active list via the
//                 Verlet -> active map.  r_rev = -r_e exactly, so both directions survive
//                 together.
#include <cmath>

#include "ctd_internal.cuh"

namespace ctd {

// ------------------------------------------------------------------------------- wrap + bin
__global__ void k_wrap_bin(int64_t n, const double* __restrict__ x, CellGeom g,
                           double* __restrict__ xw, int32_t* __restrict__ wrapm,
                           int32_t* __restrict__ cell, int32_t* __restrict__ cell_count) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  double f[3];
  int c[3];
  for (int a = 0; a < 3; ++a) {
    double s = __dadd_rn(__dadd_rn(__dmul_rn(g.G[3 * a], xi[0]), __dmul_rn(g.G[3 * a + 1], xi[1])),
                         __dmul_rn(g.G[3 * a + 2], xi[2]));
    double fl = floor(s);
    f[a] = __dsub_rn(s, fl);
    wrapm[3 * i + a] = (int32_t)fl;
    int ci = (int)floor(f[a] * (double)g.nc[a]);
    c[a] = ci < 0 ? 0 : (ci >= g.nc[a] ? g.nc[a] - 1 : ci);
  }
  for (int k = 0; k < 3; ++k)
    xw[3 * i + k] = __dadd_rn(__dadd_rn(__dmul_rn(f[0], g.H[k]), __dmul_rn(f[1], g.H[3 + k])),
                              __dmul_rn(f[2], g.H[6 + k]));
  int lin = cell_linear(g, c[0], c[1], c[2]);
  cell[i] = lin;
  atomicAdd(&cell_count[lin], 1);
}

void launch_wrap_bin(cudaStream_t st, int64_t n, const double* x_user, const CellGeom& g,
                     double* xw, int32_t* wrapm, int32_t* cell, int32_t* cell_count) {
  if (n == 0) return;
  { LaunchScope ls_(st); k_wrap_bin<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(n, x_user, g, xw, wrapm,
                                                                             cell, cell_count); }
}

// ------------------------------------------------------------------------------- counting sort
__global__ void k_place(int64_t n, const int32_t* __restrict__ cell, const int32_t* __restrict__ start,
                        int32_t* __restrict__ cursor, int32_t* __restrict__ tmp_idx) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = cell[i];
  int pos = start[c] + atomicAdd(&cursor[c], 1);
  tmp_idx[pos] = (int32_t)i;
}

void launch_place(cudaStream_t st, int64_t n, const int32_t* cell, const int32_t* cell_start,
                  int32_t* cursor, int32_t* tmp_idx) {
  if (n == 0) return;
  { LaunchScope ls_(st); k_place<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(n, cell, cell_start, cursor,
                                                                         tmp_idx); }
}

// One warp per cell: rank of each member = number of members with a smaller caller index.
__global__ void k_sort_cells(int64_t ncell, const int32_t* __restrict__ start,
                             const int32_t* __restrict__ tmp_idx, int32_t* __restrict__ perm) {
  int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (c >= ncell) return;
  int b = start[c], e = start[c + 1];
  for (int k = b + lane; k < e; k += 32) {
    int v = tmp_idx[k];
    int rank = 0;
    for (int l = b; l < e; ++l) rank += (tmp_idx[l] < v);
    perm[b + rank] = v;
  }
}

void launch_sort_cells(cudaStream_t st, int64_t ncell, const int32_t* cell_start,
                       const int32_t* tmp_idx, int32_t* perm) {
  if (ncell == 0) return;
  int64_t threads = ncell * 32;
  { LaunchScope ls_(st); k_sort_cells<<<(unsigned)((threads + kThreads - 1) / kThreads), kThreads, 0, st>>>(ncell, cell_start,
                                                                                    tmp_idx, perm); }
}

__global__ void k_gather_sorted(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ xw,
                                const double* __restrict__ xu, const int32_t* __restrict__ zu,
                                double* __restrict__ xw_s, double* __restrict__ xref_s,
                                int32_t* __restrict__ z_s, int32_t* __restrict__ inv) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  int i = perm[k];
  for (int c = 0; c < 3; ++c) {
    xw_s[3 * k + c] = xw[3 * (int64_t)i + c];
    xref_s[3 * k + c] = xu[3 * (int64_t)i + c];
  }
  if (zu) z_s[k] = zu[i];
  inv[i] = (int32_t)k;
}

void launch_gather_sorted(cudaStream_t st, int64_t n, const int32_t* perm, const double* xw,
                          const double* x_user, const int32_t* species_user, double* xw_s,
                          double* xref_s, int32_t* species_s, int32_t* inv_perm) {
  if (n == 0) return;
  { LaunchScope ls_(st); k_gather_sorted<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(
      n, perm, xw, x_user, species_user, xw_s, xref_s, species_s, inv_perm); }
}

// ------------------------------------------------------------------------------- pair search
__device__ __forceinline__ uint32_t pack_img(int a, int b, int c) {
  return (uint32_t)(uint8_t)(int8_t)a | ((uint32_t)(uint8_t)(int8_t)b << 8) |
         ((uint32_t)(uint8_t)(int8_t)c << 16);
}

// One warp per cell of the grid: the cell's atoms (in groups of up to 32, the "home" atoms)
// against the atoms of every neighbour cell, visited in a fixed order of slab offsets; within a
// neighbour cell the candidates are in sorted order.  Each neighbour cell is staged in shared
// memory (in pieces of up to kPsPiece atoms, image shift applied) and the lanes run over the
// (home atom, candidate) pairs, so all 32 lanes work whatever the cell occupancy.
//
// Every pair first takes an FP32 distance test against R2f, a threshold above R^2 by a bound on
// the FP32 rounding of the positions, the image shift and the squared distance (computed on the
// host from the cell and the search range): it only drops pairs whose exact distance is beyond
// the cutoff.  The survivors (about one in seven) queue up per warp in the order they were found
// and take the canonical FP64 test in batches of 32.  The pairs kept are those of the FP64 test
// alone; each home atom's row lists them by neighbour cell, then candidate, and is written
// through a per-atom cursor, so the fill is deterministic.
constexpr int kPsQueue = 64;   // per-warp survivor queue (a batch of 32 plus one chunk)
constexpr int kPsPiece = 64;   // neighbour atoms staged at a time
constexpr int kPsWarps = kThreads / 32;

template <bool FILL>
__global__ void k_pair_search(int64_t ncells, const double* __restrict__ xs, const int32_t* __restrict__ cstart,
                              CellGeom g, float r2f, int32_t* __restrict__ count, const int32_t* __restrict__ row_ptr,
                              int32_t* __restrict__ col, uint32_t* __restrict__ img,
                              float4* __restrict__ base) {
  __shared__ float4 hx[kPsWarps][32];          // home atoms (FP32)
  __shared__ float4 nx[kPsWarps][kPsPiece];    // neighbour piece (FP32, image shift applied)
  __shared__ int32_t cur[kPsWarps][32];        // per home atom: pairs kept so far
  __shared__ int32_t qj[kPsWarps][kPsQueue];
  __shared__ uint32_t qi[kPsWarps][kPsQueue];
  __shared__ int32_t qa[kPsWarps][kPsQueue];
  const int64_t cw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  if (cw >= ncells) return;
  const unsigned lt = (1u << lane) - 1u;
  const int c0 = (int)(cw / ((int64_t)g.nc[1] * g.nc[2])), c1 = (int)((cw / g.nc[2]) % g.nc[1]),
            c2 = (int)(cw % g.nc[2]);
  const int hlin = cell_linear(g, c0, c1, c2);
  const int hs = cstart[hlin], he = cstart[hlin + 1];
  const float hf[9] = {(float)g.H[0], (float)g.H[1], (float)g.H[2], (float)g.H[3], (float)g.H[4],
                       (float)g.H[5], (float)g.H[6], (float)g.H[7], (float)g.H[8]};
  for (int h0 = hs; h0 < he; h0 += 32) {
    const int ga = he - h0 < 32 ? he - h0 : 32;
    if (lane < ga) {
      const int64_t i = h0 + lane;
      hx[wq][lane] = make_float4((float)xs[3 * i], (float)xs[3 * i + 1], (float)xs[3 * i + 2], 0.f);
      cur[wq][lane] = 0;
    }
    __syncwarp();
    int qn = 0;
    // canonical FP64 test of the first nb queued survivors (in queue order); kept pairs go to
    // their home atom's row at its cursor, ranked among this batch's lanes of the same atom
    auto batch = [&](int nb) {
      bool keep = false;
      double dv0 = 0, dv1 = 0, dv2 = 0;
      int j = 0, a = 32 + lane;   // lanes without an entry get keys no home atom has
      uint32_t pim = 0;
      if (lane < nb) {
        j = qj[wq][lane];
        pim = qi[wq][lane];
        a = qa[wq][lane];
        const int64_t i = h0 + a;
        const int im0 = (int8_t)(pim & 0xff), im1 = (int8_t)((pim >> 8) & 0xff), im2 = (int8_t)((pim >> 16) & 0xff);
        double sh[3];
        for (int c = 0; c < 3; ++c)
          sh[c] = __dadd_rn(__dadd_rn(__dmul_rn((double)im0, g.H[c]), __dmul_rn((double)im1, g.H[3 + c])),
                            __dmul_rn((double)im2, g.H[6 + c]));
        dv0 = __dadd_rn(__dsub_rn(xs[3 * (int64_t)j], xs[3 * i]), sh[0]);
        dv1 = __dadd_rn(__dsub_rn(xs[3 * (int64_t)j + 1], xs[3 * i + 1]), sh[1]);
        dv2 = __dadd_rn(__dsub_rn(xs[3 * (int64_t)j + 2], xs[3 * i + 2]), sh[2]);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dv0, dv0), __dmul_rn(dv1, dv1)), __dmul_rn(dv2, dv2));
        keep = d2 < g.R2;
      }
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      const unsigned peers = __match_any_sync(0xffffffffu, a);
      const int before = __popc(m & peers & lt);
      if (FILL && keep) {
        const int pos = row_ptr[h0 + a] + cur[wq][a] + before;
        col[pos] = j;
        img[pos] = pim;
        base[pos] = make_float4((float)dv0, (float)dv1, (float)dv2, 0.0f);
      }
      __syncwarp();
      if (lane < nb && (peers & lt) == 0) cur[wq][a] += __popc(m & peers);   // one lane per home atom
      __syncwarp();
    };
    for (int d0 = -g.M[0]; d0 <= g.M[0]; ++d0)
      for (int d1 = -g.M[1]; d1 <= g.M[1]; ++d1)
        for (int d2 = -g.M[2]; d2 <= g.M[2]; ++d2) {
          int cc[3] = {c0 + d0, c1 + d1, c2 + d2};
          int im[3], w[3];
          for (int a = 0; a < 3; ++a) {
            int q = cc[a] >= 0 ? cc[a] / g.nc[a] : -((-cc[a] + g.nc[a] - 1) / g.nc[a]);
            im[a] = q;
            w[a] = cc[a] - q * g.nc[a];
          }
          float shf[3];
          for (int c = 0; c < 3; ++c)
            shf[c] = fmaf((float)im[0], hf[c], fmaf((float)im[1], hf[3 + c], (float)im[2] * hf[6 + c]));
          const bool zero_img = (im[0] == 0) && (im[1] == 0) && (im[2] == 0);
          const uint32_t pim = pack_img(im[0], im[1], im[2]);
          const int nlin = cell_linear(g, w[0], w[1], w[2]);
          const int bs = cstart[nlin], be = cstart[nlin + 1];
          for (int b0 = bs; b0 < be; b0 += kPsPiece) {
            const int nb = be - b0 < kPsPiece ? be - b0 : kPsPiece;
            for (int t = lane; t < nb; t += 32) {
              const int64_t jj = b0 + t;
              nx[wq][t] = make_float4((float)xs[3 * jj] + shf[0], (float)xs[3 * jj + 1] + shf[1],
                                      (float)xs[3 * jj + 2] + shf[2], 0.f);
            }
            __syncwarp();
            const int total = ga * nb;
            for (int p0 = 0; p0 < total; p0 += 32) {
              const int p = p0 + lane;
              bool pass = false;
              int a = 0, bb = 0;
              if (p < total) {
                a = p / nb;
                bb = p - a * nb;
                const float4 y = nx[wq][bb], x = hx[wq][a];
                const float e0 = y.x - x.x, e1 = y.y - x.y, e2 = y.z - x.z;
                pass = fmaf(e2, e2, fmaf(e1, e1, e0 * e0)) < r2f && !(zero_img && b0 + bb == h0 + a);
              }
              const unsigned m = __ballot_sync(0xffffffffu, pass);
              if (pass) {
                const int slot = qn + __popc(m & lt);
                qj[wq][slot] = b0 + bb;
                qi[wq][slot] = pim;
                qa[wq][slot] = a;
              }
              qn += __popc(m);
              __syncwarp();
              if (qn >= 32) {
                batch(32);
                // move the overflow (at most 31 entries) to the front of the queue
                int32_t mj = 0, ma = 0;
                uint32_t mi = 0;
                if (lane + 32 < qn) { mj = qj[wq][lane + 32]; mi = qi[wq][lane + 32]; ma = qa[wq][lane + 32]; }
                __syncwarp();
                if (lane + 32 < qn) { qj[wq][lane] = mj; qi[wq][lane] = mi; qa[wq][lane] = ma; }
                qn -= 32;
                __syncwarp();
              }
            }
            __syncwarp();   // the piece is read before the next one overwrites it
          }
        }
    if (qn > 0) batch(qn);
    if (!FILL && lane < ga) count[h0 + lane] = cur[wq][lane];
    __syncwarp();
  }
}

// FP32 threshold of the prefilter: R^2 plus a bound on the FP32 error of the squared distance.
// The wrapped positions lie in the cell and the image shifts span at most M cells per direction,
// so every coordinate entering a difference is bounded by A = sum_a (M_a + 2) |h_a|_1; each of
// the position and shift conversions, the difference and the sum adds at most 2^-24 A per
// component (16 2^-24 A is taken), and the squared distance near R adds 2 sqrt(3) R e + 3 e^2
// plus its own rounding (8 2^-24 R^2 taken).  The result is rounded up to a float.
static float prefilter_r2(const CellGeom& g) {
  double A = 0.0;
  for (int a = 0; a < 3; ++a)
    A += (g.M[a] + 2) * (std::fabs(g.H[3 * a]) + std::fabs(g.H[3 * a + 1]) + std::fabs(g.H[3 * a + 2]));
  const double u = 5.9604644775390625e-08;   // 2^-24
  const double e = 16.0 * u * A, R = std::sqrt(g.R2);
  const double t = g.R2 + 2.0 * std::sqrt(3.0) * R * e + 3.0 * e * e + 8.0 * u * g.R2;
  return std::nextafter((float)t, INFINITY);
}

void launch_pair_search(cudaStream_t st, bool fill, int64_t n, const double* xw_s,
                        const int32_t* cell_start, const CellGeom& g, int32_t* count,
                        const int32_t* row_ptr, int32_t* col, uint32_t* img, float4* base) {
  if (n == 0) return;
  const int64_t ncells = (int64_t)g.nc[0] * g.nc[1] * g.nc[2];   // one warp per grid cell
  const int64_t threads = ncells * 32;
  const unsigned blocks = (unsigned)((threads + kThreads - 1) / kThreads);
  const float r2f = prefilter_r2(g);
  if (fill)
    { LaunchScope ls_(st); k_pair_search<true><<<blocks, kThreads, 0, st>>>(ncells, xw_s, cell_start, g, r2f, count, row_ptr, col, img, base); }
  else
    { LaunchScope ls_(st); k_pair_search<false><<<blocks, kThreads, 0, st>>>(ncells, xw_s, cell_start, g, r2f, count, row_ptr, col, img, base); }
}

// ------------------------------------------------------------------------------- reverse edges
__device__ __forceinline__ uint32_t neg_img(uint32_t v) {
  int a = (int8_t)(v & 0xff), b = (int8_t)((v >> 8) & 0xff), c = (int8_t)((v >> 16) & 0xff);
  return pack_img(-a, -b, -c);
}

// One warp per row i; for each edge e = (i <- j, n) the warp scans row j for (j <- i, -n).
__global__ void k_reverse(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const uint32_t* __restrict__ img, int32_t* __restrict__ rev, int* status) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    int j = col[e];
    uint32_t want = neg_img(img[e]);
    int found = -1;
    for (int b = rp[j]; b < rp[j + 1] && found < 0; b += 32) {
      int k = b + lane;
      bool hit = (k < rp[j + 1]) && col[k] == (int)i && img[k] == want;
      unsigned m = __ballot_sync(0xffffffffu, hit);
      if (m) found = b + __ffs(m) - 1;
    }
    if (lane == 0) {
      rev[e] = found;
      if (found < 0) atomicOr(status, (int)ST_REV_MISSING);
    }
  }
}

void launch_reverse(cudaStream_t st, int64_t n, const int32_t* row_ptr, const int32_t* col,
                    const uint32_t* img, int32_t* rev, int* status) {
  if (n == 0) return;
  int64_t threads = n * 32;
  { LaunchScope ls_(st); k_reverse<<<(unsigned)((threads + kThreads - 1) / kThreads), kThreads, 0, st>>>(n, row_ptr, col, img,
                                                                                 rev, status); }
}

// ------------------------------------------------------------------------------- per step
__global__ void k_gather_positions(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ xu,
                                   double* __restrict__ xs) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  int64_t i = perm[k];
  xs[3 * k] = xu[3 * i];
  xs[3 * k + 1] = xu[3 * i + 1];
  xs[3 * k + 2] = xu[3 * i + 2];
}

void launch_gather_positions(cudaStream_t st, int64_t n, const int32_t* perm, const double* x_user,
                             double* x_s) {
  if (n == 0) return;
  { LaunchScope ls_(st); k_gather_positions<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(n, perm, x_user, x_s); }
}

__global__ void k_delta(int64_t n, const double* __restrict__ xs, const double* __restrict__ xref,
                        float4* __restrict__ delta, unsigned int* maxd2) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float d2 = 0.0f;
  if (k < n) {
    float dx = (float)(xs[3 * k] - xref[3 * k]);
    float dy = (float)(xs[3 * k + 1] - xref[3 * k + 1]);
    float dz = (float)(xs[3 * k + 2] - xref[3 * k + 2]);
    delta[k] = make_float4(dx, dy, dz, 0.0f);
    d2 = dx * dx + dy * dy + dz * dz;
    if (!(d2 == d2) || d2 > 3.0e38f) d2 = 3.0e38f;   // NaN / Inf: force the trigger
  }
  for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
  if ((threadIdx.x & 31) == 0 && d2 > 0.0f) atomicMax(maxd2, __float_as_uint(d2));
}

void launch_delta(cudaStream_t st, int64_t n, const double* x_s, const double* xref_s, float4* delta,
                  unsigned int* maxdisp2_bits) {
  if (n == 0) return;
  { LaunchScope ls_(st); k_delta<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(n, x_s, xref_s, delta,
                                                                         maxdisp2_bits); }
}

template <bool FILL>
__global__ void k_prune(int64_t n, const int32_t* __restrict__ vrow, const int32_t* __restrict__ vcol,
                        const float4* __restrict__ vbase, const float4* __restrict__ delta, float rc2,
                        const uint8_t* __restrict__ near, int32_t* __restrict__ acount,
                        const int32_t* __restrict__ arow, int32_t* __restrict__ acol, float4* __restrict__ ar,
                        int32_t* __restrict__ vidx, int32_t* __restrict__ v2a) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  const float4 di = delta[i];
  // near (null: keep all): an edge is kept only if one of its atoms is within T - 1 hops of an
  // owned atom of its domain; the test is symmetric, so every kept edge keeps its reverse.
  const bool near_i = near == nullptr || near[i] != 0;
  int out = FILL ? arow[i] : 0, cnt = 0;
  const int b = vrow[i], e = vrow[i + 1];
  for (int e0 = b; e0 < e; e0 += 32) {
    int ev = e0 + lane;
    bool keep = false;
    float rx = 0, ry = 0, rz = 0, r2 = 0;
    int j = 0;
    if (ev < e) {
      j = vcol[ev];
      float4 bb = vbase[ev], dj = delta[j];
      rx = bb.x + (dj.x - di.x);
      ry = bb.y + (dj.y - di.y);
      rz = bb.z + (dj.z - di.z);
      r2 = rx * rx + ry * ry + rz * rz;
      keep = r2 < rc2 && (near_i || near[j] != 0);
    }
    unsigned m = __ballot_sync(0xffffffffu, keep);
    if (FILL) {
      int pos = out + cnt + __popc(m & ((1u << lane) - 1u));
      if (keep) {
        acol[pos] = j;
        ar[pos] = make_float4(rx, ry, rz, sqrtf(r2));
        vidx[pos] = ev;
      }
      if (ev < e) v2a[ev] = keep ? pos : -1;
    }
    cnt += __popc(m);
  }
  if (!FILL && lane == 0) acount[i] = cnt;
}

void launch_prune(cudaStream_t st, bool fill, int64_t n, const int32_t* vrow, const int32_t* vcol,
                  const float4* vbase, const float4* delta, float rc2, const uint8_t* near, int32_t* acount,
                  const int32_t* arow, int32_t* acol, float4* ar, int32_t* vidx, int32_t* v2a) {
  if (n == 0) return;
  int64_t threads = n * 32;
  unsigned blocks = (unsigned)((threads + kThreads - 1) / kThreads);
  if (fill)
    { LaunchScope ls_(st); k_prune<true><<<blocks, kThreads, 0, st>>>(n, vrow, vcol, vbase, delta, rc2, near, acount, arow, acol, ar, vidx, v2a); }
  else
    { LaunchScope ls_(st); k_prune<false><<<blocks, kThreads, 0, st>>>(n, vrow, vcol, vbase, delta, rc2, near, acount, arow, acol, ar, vidx, v2a); }
}

__global__ void k_prune_rev(int64_t n_active, const int32_t* __restrict__ vidx,
                            const int32_t* __restrict__ vrev, const int32_t* __restrict__ v2a,
                            int32_t* __restrict__ arev) {
  int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= n_active) return;
  arev[a] = v2a[vrev[vidx[a]]];
}

// The active edge count lives on the device (arow[n]); launch over the Verlet capacity bound
// given by the caller through arow's last entry is not known on the host, so the kernel is
// launched per row instead: one warp per row walks its active edges.
// Also writes aend[a]: 0 except on the last active edge of a non-empty row, where it is 1 plus
// the number of empty rows that follow (the rows an edge walker completes at that edge).
__global__ void k_prune_rev_rows(int64_t n, const int32_t* __restrict__ arow, const int32_t* __restrict__ vidx,
                                 const int32_t* __restrict__ vrev, const int32_t* __restrict__ v2a,
                                 int32_t* __restrict__ arev, int32_t* __restrict__ aend) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int a1 = arow[i + 1];
  for (int a = arow[i] + lane; a < a1; a += 32) {
    const int rv = vrev[vidx[a]];
    arev[a] = rv >= 0 ? v2a[rv] : -1;   // -1 is flagged by the force kernel
    if (aend) {
      int cnt = 0;
      if (a == a1 - 1) {
        cnt = 1;
        for (int64_t r = i + 1; r < n && arow[r + 1] == a1; ++r) ++cnt;
      }
      aend[a] = cnt;
    }
  }
}

void launch_prune_rev(cudaStream_t st, int64_t n, const int32_t* arow, const int32_t* vidx,
                      const int32_t* vrev, const int32_t* v2a, int32_t* arev, int32_t* aend) {
  if (n == 0) return;
  int64_t threads = n * 32;
  { LaunchScope ls_(st); k_prune_rev_rows<<<(unsigned)((threads + kThreads - 1) / kThreads), kThreads, 0, st>>>(n, arow, vidx, vrev,
                                                                                        v2a, arev, aend); }
}

}  // namespace ctd
