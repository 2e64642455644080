// noalloc.cu -- neighbour-list build that allocates no device memory.
//
// Some callers cannot call cudaMalloc: an MD code that owns a fixed device memory pool and
// forbids other allocators, or code that must not allocate between its own set-up and
// teardown.  ctd_neighbors_noalloc serves them: the caller passes device positions and device
// output arrays, and every scratch array of the build (wrapped and cell-sorted positions,
// cell counts and starts, the sort permutation, per-atom pair counts, row offsets and scan
// partial sums) lives in one file-scope static device array of fixed size.  Every GPU that
// loads the library holds that array until the process exits.
//
// The pairs are the same set ctd_build_neighbors finds (same wrap, same cell search, same
// FP64 pair test); they are written in the caller's atom indices, grouped by atom in cell
// order, not sorted, with each image shift taken relative to the caller's own positions (the
// wrap counts of both atoms folded in), so that r_ij = x_j - x_i + shift . H holds for the
// positions the caller passed, wrapped or not.
#include <cmath>
#include <cstring>
#include <mutex>

#include "ctd_internal.cuh"
#include "../../include/painn.h"

namespace ctd {
namespace {

constexpr int64_t kNAMaxAtoms = CTD_NOALLOC_MAX_ATOMS;
constexpr int64_t kNAMaxCells = CTD_NOALLOC_MAX_CELLS;
constexpr int64_t kNAScanSums = (kNAMaxAtoms > kNAMaxCells ? kNAMaxAtoms : kNAMaxCells) / 2048 + 2;

// Layout of the scratch array (byte offsets, each 256-byte aligned).
constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffXw = 0;                                                  // double [3N]
constexpr size_t kOffXwS = al(kOffXw + sizeof(double) * 3 * kNAMaxAtoms);     // double [3N]
constexpr size_t kOffXref = al(kOffXwS + sizeof(double) * 3 * kNAMaxAtoms);   // double [3N]
constexpr size_t kOffWrap = al(kOffXref + sizeof(double) * 3 * kNAMaxAtoms);  // int [3N]
constexpr size_t kOffCell = al(kOffWrap + sizeof(int32_t) * 3 * kNAMaxAtoms); // int [N]
constexpr size_t kOffTmp = al(kOffCell + sizeof(int32_t) * kNAMaxAtoms);      // int [N]
constexpr size_t kOffPerm = al(kOffTmp + sizeof(int32_t) * kNAMaxAtoms);      // int [N]
constexpr size_t kOffInv = al(kOffPerm + sizeof(int32_t) * kNAMaxAtoms);      // int [N]
constexpr size_t kOffCount = al(kOffInv + sizeof(int32_t) * kNAMaxAtoms);     // int [N]
constexpr size_t kOffRow = al(kOffCount + sizeof(int32_t) * kNAMaxAtoms);     // int [N+1]
constexpr size_t kOffCCount = al(kOffRow + sizeof(int32_t) * (kNAMaxAtoms + 1));   // int [C+1]
constexpr size_t kOffCStart = al(kOffCCount + sizeof(int32_t) * (kNAMaxCells + 1)); // int [C+1]
constexpr size_t kOffCursor = al(kOffCStart + sizeof(int32_t) * (kNAMaxCells + 1)); // int [C+1]
constexpr size_t kOffSums = al(kOffCursor + sizeof(int32_t) * (kNAMaxCells + 1));   // int [sums]
constexpr size_t kOffStatus = al(kOffSums + sizeof(int32_t) * kNAScanSums);         // int [4]
constexpr size_t kScratchBytes = al(kOffStatus + sizeof(int32_t) * 4);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array, looked up once per device (host code may not take the
// address of a __device__ variable directly: that would be a host-side shadow).
std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned char* g_addr[kMaxDevices] = {};
int32_t g_host_counts[kNAMaxAtoms];   // per-atom pair counts, for the int64 total (guarded by g_mu)

int scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return CTD_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return CTD_ERR_CUDA;
    }
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return CTD_OK;
}

// Fill pass writing caller indices.  Same enumeration and FP64 pair test as the count pass,
// from the home cell the binning assigned (cell[perm[i]]), so both passes visit the same
// neighbour cells.  Writes are bounded by the row's counted slots and by cap.  Status bits:
// 2 a pair beyond its row or cap, 4 a row with fewer pairs than counted (its tail would be
// stale), 8 a shift relative to the caller's positions outside the int8 range.
__global__ void k_na_fill(int64_t n, const double* __restrict__ xs, const int32_t* __restrict__ cstart, CellGeom g,
                          const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ perm,
                          const int32_t* __restrict__ cell, const int32_t* __restrict__ wrapm, int64_t cap,
                          int32_t* __restrict__ pi, int32_t* __restrict__ pj, int8_t* __restrict__ shift,
                          int* status) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  const double xi0 = xs[3 * i], xi1 = xs[3 * i + 1], xi2 = xs[3 * i + 2];
  const int self = perm[i];
  const int hl = cell[self];   // lexicographic: (c0 nc1 + c1) nc2 + c2
  const int ci[3] = {hl / (g.nc[1] * g.nc[2]), (hl / g.nc[2]) % g.nc[1], hl % g.nc[2]};
  const int wi[3] = {wrapm[3 * self], wrapm[3 * self + 1], wrapm[3 * self + 2]};
  const int out = row_ptr[i], end = row_ptr[i + 1];
  int cnt = 0;
  for (int d0 = -g.M[0]; d0 <= g.M[0]; ++d0)
    for (int d1 = -g.M[1]; d1 <= g.M[1]; ++d1)
      for (int d2 = -g.M[2]; d2 <= g.M[2]; ++d2) {
        int cc[3] = {ci[0] + d0, ci[1] + d1, ci[2] + d2};
        int im[3], w[3];
        for (int a = 0; a < 3; ++a) {
          int q = cc[a] >= 0 ? cc[a] / g.nc[a] : -((-cc[a] + g.nc[a] - 1) / g.nc[a]);
          im[a] = q;
          w[a] = cc[a] - q * g.nc[a];
        }
        double sh[3];
        for (int c = 0; c < 3; ++c)
          sh[c] = __dadd_rn(__dadd_rn(__dmul_rn((double)im[0], g.H[c]), __dmul_rn((double)im[1], g.H[3 + c])),
                            __dmul_rn((double)im[2], g.H[6 + c]));
        bool zero_img = (im[0] == 0) && (im[1] == 0) && (im[2] == 0);
        int lin = (w[0] * g.nc[1] + w[1]) * g.nc[2] + w[2];
        int b = cstart[lin], e = cstart[lin + 1];
        for (int j0 = b; j0 < e; j0 += 32) {
          int j = j0 + lane;
          bool keep = false;
          if (j < e) {
            double dv0 = __dadd_rn(__dsub_rn(xs[3 * (int64_t)j], xi0), sh[0]);
            double dv1 = __dadd_rn(__dsub_rn(xs[3 * (int64_t)j + 1], xi1), sh[1]);
            double dv2 = __dadd_rn(__dsub_rn(xs[3 * (int64_t)j + 2], xi2), sh[2]);
            double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dv0, dv0), __dmul_rn(dv1, dv1)), __dmul_rn(dv2, dv2));
            keep = (d2 < g.R2) && !(zero_img && j == (int)i);
          }
          unsigned m = __ballot_sync(0xffffffffu, keep);
          if (keep) {
            int pos = out + cnt + __popc(m & ((1u << lane) - 1u));
            const int other = perm[j];
            // x~ = x - wrap . H for both atoms, so the caller's shift is im - wrap_j + wrap_i
            int sc[3];
            bool fits = true;
            for (int a = 0; a < 3; ++a) {
              sc[a] = im[a] - wrapm[3 * other + a] + wi[a];
              fits = fits && sc[a] >= -128 && sc[a] <= 127;
            }
            if (!fits) atomicOr(status, 8);
            if (pos < end && pos < cap) {
              pi[pos] = self;
              pj[pos] = other;
              shift[3 * (int64_t)pos] = (int8_t)sc[0];
              shift[3 * (int64_t)pos + 1] = (int8_t)sc[1];
              shift[3 * (int64_t)pos + 2] = (int8_t)sc[2];
            } else {
              atomicOr(status, 2);
            }
          }
          cnt += __popc(m);
        }
      }
  if (lane == 0 && cnt != end - out) atomicOr(status, 4);
}

}  // namespace
}  // namespace ctd

using namespace ctd;

extern "C" int ctd_neighbors_noalloc(int64_t n, const double* positions, const double cell[9], double cutoff,
                                     double skin, int32_t* pair_i, int32_t* pair_j, int8_t* pair_shift,
                                     int64_t cap, int64_t* n_pairs, void* cuda_stream) {
  if (n_pairs) *n_pairs = 0;
  if (n < 0 || n > kNAMaxAtoms || (n > 0 && !positions) || !cell || !n_pairs || cap < 0 ||
      (cap > 0 && (!pair_i || !pair_j || !pair_shift)))
    return CTD_ERR_INVALID_ARG;
  if (!(cutoff > 0.0) || !(skin >= 0.0)) return CTD_ERR_INVALID_ARG;
  for (int k = 0; k < 9; ++k)
    if (!std::isfinite(cell[k])) return CTD_ERR_INVALID_ARG;
  // cell geometry: G = H^{-T} by cofactors in the canonical order (no contraction in this file)
  CellGeom g{};
  memcpy(g.H, cell, sizeof(g.H));
  {
    const double* H = cell;
    volatile double c[9];
    c[0] = H[4] * H[8] - H[5] * H[7];
    c[1] = H[5] * H[6] - H[3] * H[8];
    c[2] = H[3] * H[7] - H[4] * H[6];
    c[3] = H[2] * H[7] - H[1] * H[8];
    c[4] = H[0] * H[8] - H[2] * H[6];
    c[5] = H[1] * H[6] - H[0] * H[7];
    c[6] = H[1] * H[5] - H[2] * H[4];
    c[7] = H[2] * H[3] - H[0] * H[5];
    c[8] = H[0] * H[4] - H[1] * H[3];
    double det = (H[0] * c[0] + H[1] * c[1]) + H[2] * c[2];
    if (!(std::fabs(det) > 1e-9)) return CTD_ERR_INVALID_ARG;
    for (int k = 0; k < 9; ++k) g.G[k] = c[k] / det;
  }
  const double R = cutoff + skin;
  int64_t ncell = 1;
  for (int a = 0; a < 3; ++a) {
    double w = 1.0 / std::sqrt(g.G[3 * a] * g.G[3 * a] + g.G[3 * a + 1] * g.G[3 * a + 1] + g.G[3 * a + 2] * g.G[3 * a + 2]);
    int nc = (int)std::floor(w / (R * (1.0 + 1e-6)));
    if (nc < 1) nc = 1;
    if (nc > 1024) nc = 1024;
    g.nc[a] = nc;
    g.M[a] = (int)std::ceil(R * nc * (1.0 + 1e-6) / w);
    if (g.M[a] > 100) return CTD_ERR_CELL_TOO_SMALL;
    ncell *= nc;
  }
  if (ncell > kNAMaxCells) return CTD_ERR_INVALID_ARG;
  g.R2 = R * R;
  // Bounds on the int32 counts: a home atom's search visits each cell at most
  // visits = prod_a ceil((2 M_a + 1) / nc_a) times (once per image), so it counts at most
  // n * visits pairs, and all atoms together at most n^2 * visits.
  int64_t visits = 1;
  for (int a = 0; a < 3; ++a) visits *= (2 * (int64_t)g.M[a] + 1 + g.nc[a] - 1) / g.nc[a];
  if (n * visits > (int64_t)INT32_MAX) return CTD_ERR_INVALID_ARG;   // one atom's count could overflow
  const bool total_may_overflow = n * n * visits > (int64_t)INT32_MAX;

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  {
    // the call synchronises its stream and reads results into host memory: not capturable
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
      cudaGetLastError();
      return CTD_ERR_CUDA;
    }
    if (cs != cudaStreamCaptureStatusNone) return CTD_ERR_INVALID_ARG;
  }
  unsigned char* base = nullptr;
  int r = scratch_address(&base);
  if (r) return r;
  double* xw = reinterpret_cast<double*>(base + kOffXw);
  double* xw_s = reinterpret_cast<double*>(base + kOffXwS);
  double* xref = reinterpret_cast<double*>(base + kOffXref);
  int32_t* wrapm = reinterpret_cast<int32_t*>(base + kOffWrap);
  int32_t* cellid = reinterpret_cast<int32_t*>(base + kOffCell);
  int32_t* tmp = reinterpret_cast<int32_t*>(base + kOffTmp);
  int32_t* perm = reinterpret_cast<int32_t*>(base + kOffPerm);
  int32_t* inv = reinterpret_cast<int32_t*>(base + kOffInv);
  int32_t* count = reinterpret_cast<int32_t*>(base + kOffCount);
  int32_t* row = reinterpret_cast<int32_t*>(base + kOffRow);
  int32_t* ccount = reinterpret_cast<int32_t*>(base + kOffCCount);
  int32_t* cstart = reinterpret_cast<int32_t*>(base + kOffCStart);
  int32_t* cursor = reinterpret_cast<int32_t*>(base + kOffCursor);
  int32_t* sums = reinterpret_cast<int32_t*>(base + kOffSums);
  int* status = reinterpret_cast<int*>(base + kOffStatus);

  // The array keeps the previous call's contents: clear everything that must start at zero.
  if (cudaMemsetAsync(ccount, 0, sizeof(int32_t) * (ncell + 1), st) != cudaSuccess ||
      cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (ncell + 1), st) != cudaSuccess ||
      cudaMemsetAsync(status, 0, sizeof(int32_t) * 4, st) != cudaSuccess) {
    cudaGetLastError();
    return CTD_ERR_CUDA;
  }
  launch_check_finite(st, 3 * n, positions, status + 1);
  launch_wrap_bin(st, n, positions, g, xw, wrapm, cellid, ccount);
  launch_exclusive_scan(st, ncell, ccount, cstart, sums);
  launch_place(st, n, cellid, cstart, cursor, tmp);
  launch_sort_cells(st, ncell, cstart, tmp, perm);
  launch_gather_sorted(st, n, perm, xw, positions, nullptr, xw_s, xref, nullptr, inv);
  launch_pair_search(st, false, n, xw_s, cstart, g, count, nullptr, nullptr, nullptr, nullptr);
  int stv[2] = {0, 0};
  if (total_may_overflow) {
    // the row offsets are an int32 scan: total the per-atom counts in int64 first
    std::lock_guard<std::mutex> lock(g_mu);
    if (cudaMemcpyAsync(g_host_counts, count, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(stv, status, sizeof(stv), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return CTD_ERR_CUDA;
    }
    if (stv[1]) return CTD_ERR_NONFINITE;
    int64_t total64 = 0;
    for (int64_t k = 0; k < n; ++k) total64 += g_host_counts[k];
    if (total64 > (int64_t)INT32_MAX) {
      *n_pairs = total64;
      return CTD_ERR_CAPACITY;
    }
  }
  launch_exclusive_scan(st, n, count, row, sums);
  int32_t total = 0;
  if (cudaMemcpyAsync(&total, row + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(stv, status, sizeof(stv), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return CTD_ERR_CUDA;
  }
  if (stv[1]) return CTD_ERR_NONFINITE;
  *n_pairs = total;
  if (total > cap) return CTD_ERR_CAPACITY;
  if (n > 0) {
    int64_t threads = n * 32;
    LaunchScope ls_(st);
    k_na_fill<<<(unsigned)((threads + kThreads - 1) / kThreads), kThreads, 0, st>>>(
        n, xw_s, cstart, g, row, perm, cellid, wrapm, cap, pair_i, pair_j, pair_shift, status);
  }
  if (cudaMemcpyAsync(stv, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return CTD_ERR_CUDA;
  }
  if (cudaGetLastError() != cudaSuccess) return CTD_ERR_CUDA;
  if (stv[0] & 8) return CTD_ERR_INVALID_ARG;   // a shift does not fit int8: positions too far out
  return stv[0] ? CTD_ERR_CAPACITY : CTD_OK;
}
