// scan.cu -- exclusive prefix sum of int32 counts (CSR row pointers, cell starts).
// Three launches: per-block totals, a scan of the totals, a per-block rescan with the offset.
// Deterministic (no atomics); out[n] receives the total.
#include "ctd_internal.cuh"

namespace ctd {

constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;   // 2048 elements per block

__device__ __forceinline__ int block_exclusive_scan(int v, int* smem_warp, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < (kThreads / 32) ? smem_warp[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < (kThreads / 32)) smem_warp[lane] = w;
  }
  __syncthreads();
  int warp_off = warp ? smem_warp[warp - 1] : 0;
  total = smem_warp[kThreads / 32 - 1];
  __syncthreads();
  return warp_off + x - v;
}

__global__ void k_scan_totals(int64_t n, const int32_t* __restrict__ in, int32_t* __restrict__ sums) {
  __shared__ int sw[kThreads / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int acc = 0;
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) acc += in[base + k];
  int total;
  block_exclusive_scan(acc, sw, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_sums(int nb, int32_t* __restrict__ sums) {
  __shared__ int sw[kThreads / 32];
  int carry = 0;
  for (int b0 = 0; b0 < nb; b0 += kThreads) {
    int idx = b0 + threadIdx.x;
    int v = idx < nb ? sums[idx] : 0;
    int total;
    int ex = block_exclusive_scan(v, sw, total);
    if (idx < nb) sums[idx] = ex + carry;
    carry += total;
  }
}

__global__ void k_scan_apply(int64_t n, const int32_t* __restrict__ in, const int32_t* __restrict__ sums,
                             int32_t* __restrict__ out) {
  __shared__ int sw[kThreads / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int vals[kScanItems];
  int acc = 0;
  for (int k = 0; k < kScanItems; ++k) {
    vals[k] = base + k < n ? in[base + k] : 0;
    acc += vals[k];
  }
  int total;
  int ex = block_exclusive_scan(acc, sw, total) + sums[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = ex;
    ex += vals[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kThreads - 1) out[n] = ex;
}

size_t scan_temp_bytes(int64_t n) {
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  return (size_t)(nb + 1) * sizeof(int32_t);
}

void launch_exclusive_scan(cudaStream_t st, int64_t n, const int32_t* in, int32_t* out, void* temp) {
  int32_t* sums = static_cast<int32_t*>(temp);
  if (n == 0) {
    cudaMemsetAsync(out, 0, sizeof(int32_t), st);
    return;
  }
  int nb = (int)((n + kScanTile - 1) / kScanTile);
  { LaunchScope ls_(st); k_scan_totals<<<nb, kThreads, 0, st>>>(n, in, sums); }
  { LaunchScope ls_(st); k_scan_sums<<<1, kThreads, 0, st>>>(nb, sums); }
  { LaunchScope ls_(st); k_scan_apply<<<nb, kThreads, 0, st>>>(n, in, sums, out); }
}

}  // namespace ctd
