// gemm_bf16.cu -- persistent tcgen05 GEMM for the node MLPs of the BF16 path:
//   C[M][N] = A[M][K] . W[N][K]^T   (BF16 operands, FP32 accumulation in TMEM)
// with the same fused epilogues as the FP32 SIMT GEMM (bias, bias + SiLU, residual add,
// multiply by SiLU').  A rows are atoms (or atom x spatial component), W is a weight matrix
// stored [out][in], i.e. K-major, so both operands are K-major 128B-swizzled tiles.
//
// One CTA per SM (persistent over 128-row tiles).  Warp 0: TMA producer (the weight tile W is
// loaded once per CTA and stays in shared memory; A tiles stream through one or two stages).
// Warp 1: TMEM allocation and the single-thread MMA issue (M = 128, N up to 256 per
// instruction, K = 16 per instruction).  Warps 2-5: epilogue, one thread per tile row
// (TMEM lane), 32 columns per tcgen05.ld.  Every wait is bounded; on a timeout the kernel
// records ST_TIMEOUT in the status word and winds down.
#include <cstdio>

#include "ctd_internal.cuh"
#include "umma.cuh"

namespace ctd {

using bf16 = __nv_bfloat16;

struct GemmBf16Args {
  int64_t M;
  int N, K;
  const float* bias;
  const float* aux;
  int ldaux;
  float* out;
  int ldo;
  bf16* outb;
  int ldob;
  int* status;
  int a_stages, n_acc, b_box_rows, n_chunk;
  uint32_t tmem_cols;
};

constexpr int kTileM = 128;
constexpr int kBlockK = 64;
constexpr int kATileBytes = kTileM * kBlockK * 2;   // 16 KB per 64-column block

template <int EPI>
__global__ void __launch_bounds__(192, 1) k_gemm_bf16(const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB, GemmBf16Args p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int KB = p.K / kBlockK;
  const int N = p.N;
  unsigned char* sB = smem;                                        // KB x N x 128 B
  unsigned char* sA = sB + (size_t)KB * N * 128;                   // a_stages x KB x 16 KB
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + (size_t)p.a_stages * KB * kATileBytes);
  uint64_t* full = bars;          // [2]
  uint64_t* empty = bars + 2;     // [2]
  uint64_t* tfull = bars + 4;     // [2]
  uint64_t* tempty = bars + 6;    // [2]
  uint64_t* bbar = bars + 8;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 9);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (p.M + kTileM - 1) / kTileM;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      umma::mbar_init(&full[i], 1);
      umma::mbar_init(&empty[i], 1);
      umma::mbar_init(&tfull[i], 1);
      umma::mbar_init(&tempty[i], 4);
    }
    umma::mbar_init(bbar, 1);
    umma::mbar_fence_init();
  }
  if (warp == 1) umma::tmem_alloc(tmem_slot, p.tmem_cols);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  int issued = 0, last_acc = 0;

  if (warp == 0) {
    if (lane == 0) {
      umma::mbar_expect_tx(bbar, (uint32_t)(N * p.K * 2));
      for (int kb = 0; kb < KB; ++kb)
        for (int r0 = 0; r0 < N; r0 += p.b_box_rows)
          umma::tma_load_2d(sB + (size_t)kb * N * 128 + (size_t)r0 * 128, &tmB, kb * kBlockK, r0, bbar);
      int it = 0;
      for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int s = it % p.a_stages, u = it / p.a_stages;
        if (it >= p.a_stages && !umma::mbar_wait(&empty[s], (u - 1) & 1)) { ok = false; break; }
        umma::mbar_expect_tx(&full[s], (uint32_t)(KB * kATileBytes));
        for (int kb = 0; kb < KB; ++kb)
          umma::tma_load_2d(sA + ((size_t)s * KB + kb) * kATileBytes, &tmA, kb * kBlockK, (int)(tile * kTileM),
                            &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      if (!umma::mbar_wait(bbar, 0)) ok = false;
      int it = 0;
      for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++it) {
        const int s = it % p.a_stages, a = it % p.n_acc;
        if (!umma::mbar_wait(&full[s], (it / p.a_stages) & 1)) { ok = false; break; }
        if (it >= p.n_acc && !umma::mbar_wait(&tempty[a], ((it / p.n_acc) - 1) & 1)) { ok = false; break; }
        umma::fence_after();
        const uint32_t idesc = umma::idesc_bf16_m128(p.n_chunk);
        for (int kb = 0; kb < KB; ++kb) {
          const uint32_t a_base = umma::smem_u32(sA + ((size_t)s * KB + kb) * kATileBytes);
          const uint32_t b_base = umma::smem_u32(sB + (size_t)kb * N * 128);
          for (int j = 0; j < kBlockK / 16; ++j) {
            const uint64_t ad = umma::desc_sw128(a_base + 32u * j);
            for (int nc = 0; nc < N; nc += p.n_chunk) {
              const uint64_t bd = umma::desc_sw128(b_base + (uint32_t)nc * 128u + 32u * j);
              umma::mma_bf16(tmem + (uint32_t)(a * N + nc), ad, bd, idesc, (kb | j) != 0);
            }
          }
        }
        umma::mma_commit(&empty[s]);
        umma::mma_commit(&tfull[a]);
        last_acc = a;
        ++issued;
      }
      // the MMAs of the last issued tile have completed before TMEM is released
      if (issued > 0) umma::mbar_wait(&tfull[last_acc], ((issued - 1) / p.n_acc) & 1, 200000000ull);
    }
  } else {
    // epilogue warps 2..5: TMEM lane quarter = warp % 4
    const int q = warp & 3;
    const int row = q * 32 + lane;
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      const int a = it % p.n_acc;
      if (!umma::mbar_wait(&tfull[a], (it / p.n_acc) & 1)) { ok = false; break; }
      umma::fence_after();
      const int64_t m = tile * kTileM + row;
      for (int c0 = 0; c0 < N; c0 += 32) {
        float v[32];
        umma::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * N + c0), v);
        if (m < p.M) {
          float o[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            float x = v[i];
            if (EPI == 0 || EPI == 1) x += p.bias ? p.bias[c0 + i] : 0.0f;
            if (EPI == 2) x += p.aux[m * p.ldaux + c0 + i];
            if (EPI == 3) x *= dsilu_f(p.aux[m * p.ldaux + c0 + i]);
            o[i] = x;
          }
          if (p.out) {
            float4* dst = reinterpret_cast<float4*>(p.out + m * p.ldo + c0);
#pragma unroll
            for (int i = 0; i < 8; ++i) dst[i] = make_float4(o[4 * i], o[4 * i + 1], o[4 * i + 2], o[4 * i + 3]);
          }
          if (p.outb) {
            uint4* dst = reinterpret_cast<uint4*>(p.outb + m * p.ldob + c0);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              uint32_t w[4];
#pragma unroll
              for (int h = 0; h < 4; ++h) {
                float x0 = o[8 * i + 2 * h], x1 = o[8 * i + 2 * h + 1];
                if (EPI == 1) { x0 = silu_f(x0); x1 = silu_f(x1); }
                __nv_bfloat162 b2 = __floats2bfloat162_rn(x0, x1);
                w[h] = *reinterpret_cast<uint32_t*>(&b2);
              }
              dst[i] = make_uint4(w[0], w[1], w[2], w[3]);
            }
          }
        }
      }
      umma::fence_before();
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&tempty[a]);
    }
  }
  if (!ok) atomicOr(p.status, (int)ST_TIMEOUT);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  if (warp == 1) umma::tmem_dealloc(tmem, p.tmem_cols);
}

// ------------------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2D bf16 tensor map over rows x cols (row pitch ld elements), box rows x 64 columns, 128B swizzle.
bool make_tmap_bf16(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)(rows > 0 ? rows : 1)};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

bool gemm_bf16_supported(int N, int K) { return K % 64 == 0 && K > 0 && N % 32 == 0 && N > 0 && N <= 512; }

template <int EPI>
int gemm_bf16(cudaStream_t st, int64_t M, int N, int K, const bf16* A, int64_t lda, const bf16* W,
              const float* bias, const float* aux, int ldaux, float* out, int ldo, bf16* outb, int ldob,
              int* status) {
  if (M == 0) return 0;
  if (!gemm_bf16_supported(N, K) || (lda * 2) % 16 != 0 || (reinterpret_cast<uintptr_t>(A) & 15) ||
      (reinterpret_cast<uintptr_t>(W) & 15))
    return -1;
  GemmBf16Args p{};
  p.M = M; p.N = N; p.K = K; p.bias = bias; p.aux = aux; p.ldaux = ldaux; p.out = out; p.ldo = ldo;
  p.outb = outb; p.ldob = ldob; p.status = status;
  p.b_box_rows = N % 64 == 0 ? 64 : 32;
  p.n_chunk = N <= 256 ? N : N / 2;
  if (p.n_chunk > 256 || p.n_chunk % 16) return -1;
  const int KB = K / kBlockK;
  const size_t b_bytes = (size_t)KB * N * 128, a_bytes = (size_t)KB * kATileBytes;
  const size_t limit = 227 * 1024 - 1024 - 256;
  p.a_stages = (b_bytes + 2 * a_bytes <= limit) ? 2 : 1;
  if (b_bytes + a_bytes > limit) return -1;
  p.n_acc = 2 * N <= 512 ? 2 : 1;
  uint32_t cols = 32;
  while (cols < (uint32_t)(p.n_acc * N)) cols <<= 1;
  p.tmem_cols = cols;
  CUtensorMap ta, tb;
  if (!make_tmap_bf16(&ta, A, M, K, lda, kTileM) || !make_tmap_bf16(&tb, W, N, K, K, p.b_box_rows)) return -2;
  size_t smem = 1024 + b_bytes + (size_t)p.a_stages * a_bytes + 256;
  // a CTA holding more than half of TMEM runs alone on its SM, so allocation never waits
  if (p.tmem_cols > 256 && smem < 120 * 1024) smem = 120 * 1024;
  static bool attr_set[4] = {false, false, false, false};
  if (!attr_set[EPI]) {
    cudaFuncSetAttribute(k_gemm_bf16<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr_set[EPI] = true;
  }
  const int64_t ntiles = (M + kTileM - 1) / kTileM;
  const int grid = (int)(ntiles < num_sms() ? ntiles : num_sms());
  {
    LaunchScope ls_(st);
    k_gemm_bf16<EPI><<<grid, 192, smem, st>>>(ta, tb, p);
  }
  return 0;
}

template int gemm_bf16<0>(cudaStream_t, int64_t, int, int, const bf16*, int64_t, const bf16*, const float*,
                          const float*, int, float*, int, bf16*, int, int*);
template int gemm_bf16<1>(cudaStream_t, int64_t, int, int, const bf16*, int64_t, const bf16*, const float*,
                          const float*, int, float*, int, bf16*, int, int*);
template int gemm_bf16<2>(cudaStream_t, int64_t, int, int, const bf16*, int64_t, const bf16*, const float*,
                          const float*, int, float*, int, bf16*, int, int*);
template int gemm_bf16<3>(cudaStream_t, int64_t, int, int, const bf16*, int64_t, const bf16*, const float*,
                          const float*, int, float*, int, bf16*, int, int*);

}  // namespace ctd
