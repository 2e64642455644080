// gemm_bf16.cu -- persistent tcgen05 GEMM for the node MLPs of the BF16 path:
//   C[M][N] = A[M][K] . W[N][K]^T   (BF16 operands, FP32 accumulation in TMEM)
// with the same fused epilogues as the FP32 SIMT GEMM (bias, bias + SiLU, residual add,
// multiply by SiLU') and one that packs the phi-MLP output into the message kernel's PHI rows.  A rows are atoms (or atom x spatial component), W is a weight matrix
// stored [out][in], i.e. K-major, so both operands are K-major 128B-swizzled tiles.
//
// One CTA per SM (persistent over 128-row tiles).  Warp 0: TMA producer (the weight tile W is
// loaded once per CTA and stays in shared memory; A streams through a ring of 64-column
// k-blocks, 16 KB each, as many stages as shared memory holds).  Warp 1: TMEM allocation and
// the single-thread MMA issue (M = 128, N up to 256 per instruction, K = 16 per instruction).
// Warps 2 and up: epilogue, epi_warps / 4 warps per TMEM lane quarter taking the quarter's
// 32-column chunks in turn.
// Every wait is bounded; on a timeout the kernel records ST_TIMEOUT in the status word and
// winds down.
#include <cstdio>

#include <cuda_fp16.h>

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
  const float* aux2;   // EPI 5: gsm [M/3][N], the first component of each interleaved quad
  const __half* auxh;  // EPI 6: the SiLU' argument in FP16 (stride ldaux)
  float* out;
  int ldo;
  bf16* outb;
  int ldob;
  __half* outh;   // EPI 0, 1 and 4: FP16 copy of out, same element stride ldo (optional; EPI 1: the
                  // SiLU argument; EPI 4: the message table)
  int* status;
  int a_stages, n_acc, b_box_rows, n_chunk;   // a_stages: k-block stages of the A ring
  uint32_t tmem_cols;
};

constexpr int kTileM = 128;
// Output rows per tile: EPI 5 takes 126 (42 whole atoms of three component rows; the MMA still
// covers 128 rows, the last two of which belong to the next tile and are ignored).
template <int EPI>
constexpr int tile_rows() { return EPI == 5 ? 126 : kTileM; }
constexpr int kBlockK = 64;
constexpr int kATileBytes = kTileM * kBlockK * 2;   // 16 KB per 64-column block
constexpr int kTP = 36;                              // row pitch (floats) of an epilogue transpose tile
// Epilogue warps, a multiple of 4 (epi_warps / 4 warps per TMEM lane quarter).  Sixteen hide the
// TMEM -> shared -> global latency of a chunk better than eight (U/V GEMM with FP16 output, 3M x
// 256 x 128: 0.47 against 0.69 ms); the PHI-packing epilogue holds three V quads per row in
// registers and stays at eight, the register budget of sixteen warps would spill it.
template <int EPI>
constexpr int epi_warps() { return EPI == 4 ? 8 : 16; }
constexpr int kMaxAStages = 8;

template <int EPI>
__global__ void __launch_bounds__(64 + 32 * epi_warps<EPI>(), 1) k_gemm_bf16(const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB, GemmBf16Args p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr int kEpiWarps = epi_warps<EPI>(), kEpiGroups = kEpiWarps / 4;
  const int KB = (p.K + kBlockK - 1) / kBlockK;   // a ragged last block is zero-filled by the TMA
  const int N = p.N;
  unsigned char* sB = smem;                                        // KB x N x 128 B
  unsigned char* sA = sB + (size_t)KB * N * 128;                   // a_stages x 16 KB
  float* sT = reinterpret_cast<float*>(sA + (size_t)p.a_stages * kATileBytes);   // kEpiWarps x 32 x kTP
  uint64_t* bars = reinterpret_cast<uint64_t*>(sT + kEpiWarps * 32 * kTP);
  uint64_t* full = bars;                    // [kMaxAStages]
  uint64_t* empty = bars + kMaxAStages;     // [kMaxAStages]
  uint64_t* tfull = bars + 2 * kMaxAStages; // [2]
  uint64_t* tempty = tfull + 2;             // [2]
  uint64_t* bbar = tempty + 2;
  uint64_t* gbar = bbar + 1;                // [4] EPI 5: one per epilogue group (its four quarter warps)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbar + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kRT = tile_rows<EPI>();
  const int64_t ntiles = (p.M + kRT - 1) / kRT;

  if (threadIdx.x == 0) {
    for (int i = 0; i < p.a_stages; ++i) {
      umma::mbar_init(&full[i], 1);
      umma::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      umma::mbar_init(&tfull[i], 1);
      umma::mbar_init(&tempty[i], kEpiWarps);
    }
    umma::mbar_init(bbar, 1);
    for (int i = 0; i < 4; ++i) umma::mbar_init(&gbar[i], 4);
    umma::mbar_fence_init();
  }
  if (warp == 1) umma::tmem_alloc(tmem_slot, p.tmem_cols);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  int64_t issued = 0;   // MMA thread: k-blocks issued

  if (warp == 0) {
    if (lane == 0) {
      umma::mbar_expect_tx(bbar, (uint32_t)(N * KB * kBlockK * 2));   // whole boxes, fill included
      for (int kb = 0; kb < KB; ++kb)
        for (int r0 = 0; r0 < N; r0 += p.b_box_rows)
          umma::tma_load_2d(sB + (size_t)kb * N * 128 + (size_t)r0 * 128, &tmB, kb * kBlockK, r0, bbar);
      int64_t g = 0;   // k-blocks loaded so far
      for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int s = (int)(g % p.a_stages);
          const int64_t u = g / p.a_stages;
          if (g >= p.a_stages && !umma::mbar_wait(&empty[s], (uint32_t)((u - 1) & 1))) { ok = false; break; }
          umma::mbar_expect_tx(&full[s], (uint32_t)kATileBytes);
          umma::tma_load_2d(sA + (size_t)s * kATileBytes, &tmA, kb * kBlockK, (int)(tile * kRT), &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      if (!umma::mbar_wait(bbar, 0)) ok = false;
      int it = 0;
      int64_t g = 0;   // k-blocks consumed so far
      const uint32_t idesc = umma::idesc_bf16_m128(p.n_chunk);
      for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++it) {
        const int a = it % p.n_acc;
        if (it >= p.n_acc && !umma::mbar_wait(&tempty[a], ((it / p.n_acc) - 1) & 1)) { ok = false; break; }
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int s = (int)(g % p.a_stages);
          if (!umma::mbar_wait(&full[s], (uint32_t)((g / p.a_stages) & 1))) { ok = false; break; }
          umma::fence_after();
          const uint32_t a_base = umma::smem_u32(sA + (size_t)s * kATileBytes);
          const uint32_t b_base = umma::smem_u32(sB + (size_t)kb * N * 128);
          for (int j = 0; j < kBlockK / 16; ++j) {
            const uint64_t ad = umma::desc_sw128(a_base + 32u * j);
            for (int nc = 0; nc < N; nc += p.n_chunk) {
              const uint64_t bd = umma::desc_sw128(b_base + (uint32_t)nc * 128u + 32u * j);
              umma::mma_bf16(tmem + (uint32_t)(a * N + nc), ad, bd, idesc, (kb | j) != 0);
            }
          }
          umma::mma_commit(&empty[s]);
          ++issued;
        }
        if (!ok) break;
        umma::mma_commit(&tfull[a]);
      }
      // every MMA issued has completed before TMEM is released (the commits of a thread
      // complete in order, so the last k-block's empty barrier covers all of them)
      if (issued > 0) {
        const int64_t last = issued - 1;
        umma::mbar_wait(&empty[last % p.a_stages], (uint32_t)((last / p.a_stages) & 1), 200000000ull);
      }
    }
  } else {
    // epilogue warps: TMEM lane quarter = warp % 4, group grp takes the quarter's chunks grp,
    // grp + kEpiGroups, ...  Each 32-row x 32-column chunk goes
    // TMEM -> registers (thread = row) -> padded shared tile -> registers (8 lanes per row,
    // 16 bytes each), so that global loads and stores move whole 128-byte row segments.
    const int q = warp & 3, grp = (warp - 2) >> 2;
    float* T = sT + (warp - 2) * 32 * kTP;
    const int cr = lane >> 3, cc = 4 * (lane & 7);   // row within a group of 4, column quad
    const int nchunks = N / 32;
    uint32_t gph = 0;   // EPI 5: phases of this group's barrier passed
    auto gsync = [&]() -> bool {
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&gbar[grp]);
      return umma::mbar_wait(&gbar[grp], (gph++) & 1);
    };
    int it = 0;
    for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++it) {
      const int a = it % p.n_acc;
      if (!umma::mbar_wait(&tfull[a], (it / p.n_acc) & 1)) { ok = false; break; }
      umma::fence_after();
      const int64_t m0 = tile * kRT + q * 32;   // first row of this warp's quarter
      if (grp >= nchunks) {
        umma::fence_before();
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&tempty[a]);
      }
      for (int ch = grp; ch < nchunks; ch += kEpiGroups) {
        const int c0 = 32 * ch;
        float v[32];
        umma::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * N + c0), v);
        if (ch + kEpiGroups >= nchunks) {
          // the accumulator has been read: the MMA of a later tile may reuse it
          umma::fence_before();
          __syncwarp();
          if (lane == 0) umma::mbar_arrive(&tempty[a]);
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 8; ++i)
          *reinterpret_cast<float4*>(T + lane * kTP + 4 * i) = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        __syncwarp();
        float4 bq = make_float4(0.f, 0.f, 0.f, 0.f);
        if ((EPI == 0 || EPI == 1 || EPI == 4) && p.bias) bq = *reinterpret_cast<const float4*>(p.bias + c0 + cc);
        // EPI 4 (phi packing, N = 3F): columns [phi_s | phi_vv | phi_vs]; row m of PHI (6F) gets
        // [phi_s | v_0 phi_vv | v_1 phi_vv | v_2 phi_vv | phi_vs | phi_vv], v from aux ([n][3F])
        const int Fb = N / 3, blk = EPI == 4 ? c0 / Fb : 0, f0 = c0 - blk * Fb + cc;
        float4 gv[EPI == 4 ? 8 : 1][3];
        if (EPI == 4 && blk == 1) {
          // aux null: v = 0 (first layer), psi = 0
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int64_t m = m0 + cr + 4 * j;
#pragma unroll
            for (int c = 0; c < 3; ++c)
              gv[j][c] = m < p.M && p.aux ? __ldg(reinterpret_cast<const float4*>(p.aux + m * p.ldaux + c * Fb + f0))
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
        // the chunk's aux values, all loads in flight before any store
        float4 g[8];
        if (EPI == 5) {
          // the group's four warps hold the four row quarters of this chunk in their shared tiles:
          // once all are written, the group's 128 threads assemble G4 quads of whole atoms,
          // 8 threads per atom (32 features, 512 contiguous bytes)
          if (!gsync()) { ok = false; break; }
          const int tg = ((warp - 2) & 3) * 32 + lane;
          const int64_t a0 = tile * (kRT / 3);
          for (int item = tg; item < (kRT / 3) * 8; item += 128) {
            const int al = item >> 3, fq = 4 * (item & 7);
            const int64_t ai = a0 + al;
            if (3 * ai >= p.M) break;
            float4 x[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              const int r = 3 * al + k, qq = r >> 5;
              const float* Tq = sT + (4 * grp + ((qq + 2) & 3)) * 32 * kTP;
              const float4 t = *reinterpret_cast<const float4*>(Tq + (r & 31) * kTP + fq);
              const float4 gk = __ldg(reinterpret_cast<const float4*>(p.aux + (3 * ai + k) * p.ldaux + c0 + fq));
              x[k] = make_float4(t.x + gk.x, t.y + gk.y, t.z + gk.z, t.w + gk.w);
            }
            const float4 gs = __ldg(reinterpret_cast<const float4*>(p.aux2 + ai * N + c0 + fq));
            float4* o = reinterpret_cast<float4*>(p.out + (ai * N + c0 + fq) * 4);
            o[0] = make_float4(gs.x, x[0].x, x[1].x, x[2].x);
            o[1] = make_float4(gs.y, x[0].y, x[1].y, x[2].y);
            o[2] = make_float4(gs.z, x[0].z, x[1].z, x[2].z);
            o[3] = make_float4(gs.w, x[0].w, x[1].w, x[2].w);
          }
          if (!gsync()) { ok = false; break; }   // the tiles are free for the next chunk
          continue;
        }
        if (EPI == 2 || EPI == 3) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int64_t m = m0 + cr + 4 * j;
            g[j] = m < p.M ? __ldg(reinterpret_cast<const float4*>(p.aux + m * p.ldaux + c0 + cc))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
        uint2 gh[EPI == 6 ? 8 : 1];   // EPI 6: four FP16 SiLU' arguments per row
        if (EPI == 6) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int64_t m = m0 + cr + 4 * j;
            gh[j] = m < p.M ? __ldg(reinterpret_cast<const uint2*>(p.auxh + m * p.ldaux + c0 + cc)) : make_uint2(0u, 0u);
          }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int r = cr + 4 * j;
          const int64_t m = m0 + r;
          float4 x = *reinterpret_cast<const float4*>(T + r * kTP + cc);
          if (m < p.M) {
            if (EPI == 0 || EPI == 1 || EPI == 4) { x.x += bq.x; x.y += bq.y; x.z += bq.z; x.w += bq.w; }
            if (EPI == 4) {
              // FP32 table (if out) and FP16 copy (if outh), both [phi_s | psi_0..2 | phi_vs | phi_vv]
              float* o = p.out ? p.out + m * p.ldo : nullptr;
              __half* oh = p.outh ? p.outh + m * p.ldo : nullptr;
              auto put = [&](int col, float4 y) {
                if (o) *reinterpret_cast<float4*>(o + col) = y;
              };
              auto put_h = [&](int col, float4 y) {
                if (oh) {
                  // FP16's largest finite value is 65504: a larger value is reported (it would round
                  // to Inf and reach the results as a non-finite value without its cause)
                  const float ym = fmaxf(fmaxf(fabsf(y.x), fabsf(y.y)), fmaxf(fabsf(y.z), fabsf(y.w)));
                  if (ym > 65504.f) atomicOr(p.status, (int)ST_FP16_RANGE);
                  const __half2 a = __floats2half2_rn(y.x, y.y), b = __floats2half2_rn(y.z, y.w);
                  *reinterpret_cast<uint2*>(oh + col) =
                      make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
                }
              };
              if (blk == 0) {
                put(f0, x);
                put_h(f0, x);
              } else if (blk == 2) {
                put(4 * Fb + f0, x);
                put_h(4 * Fb + f0, x);
              } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  const float4 y = make_float4(gv[j][c].x * x.x, gv[j][c].y * x.y, gv[j][c].z * x.z, gv[j][c].w * x.w);
                  put((1 + c) * Fb + f0, y);
                  put_h((1 + c) * Fb + f0, y);
                }
                put(5 * Fb + f0, x);
                put_h(5 * Fb + f0, x);
              }
              continue;
            }
            if (EPI == 2) { x.x += g[j].x; x.y += g[j].y; x.z += g[j].z; x.w += g[j].w; }
            if (EPI == 3) {
              x.x *= dsilu_fast(g[j].x); x.y *= dsilu_fast(g[j].y); x.z *= dsilu_fast(g[j].z); x.w *= dsilu_fast(g[j].w);
            }
            if (EPI == 6) {
              const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&gh[j].x));
              const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&gh[j].y));
              x.x *= dsilu_fast(a.x); x.y *= dsilu_fast(a.y); x.z *= dsilu_fast(b.x); x.w *= dsilu_fast(b.y);
            }
            if (p.out) *reinterpret_cast<float4*>(p.out + m * p.ldo + c0 + cc) = x;
            if ((EPI == 0 || EPI == 1) && p.outh) {
              const float ym = fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w)));
              if (ym > 65504.f) atomicOr(p.status, (int)ST_FP16_RANGE);
              const __half2 h01 = __floats2half2_rn(x.x, x.y), h23 = __floats2half2_rn(x.z, x.w);
              *reinterpret_cast<uint2*>(p.outh + m * p.ldo + c0 + cc) =
                  make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
            }
            if (p.outb) {
              float y0 = x.x, y1 = x.y, y2 = x.z, y3 = x.w;
              if (EPI == 1) { y0 = silu_fast(y0); y1 = silu_fast(y1); y2 = silu_fast(y2); y3 = silu_fast(y3); }
              __nv_bfloat162 b01 = __floats2bfloat162_rn(y0, y1), b23 = __floats2bfloat162_rn(y2, y3);
              *reinterpret_cast<uint2*>(p.outb + m * p.ldob + c0 + cc) =
                  make_uint2(*reinterpret_cast<uint32_t*>(&b01), *reinterpret_cast<uint32_t*>(&b23));
            }
          }
        }
      }
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

// K: a multiple of 32, at least one 64-column block (the tensor map's box is never wider than the
// tensor); a last half block reads zeros past column K, which add nothing to the product.
bool gemm_bf16_supported(int N, int K) { return K % 32 == 0 && K >= 64 && N % 32 == 0 && N > 0 && N <= 512; }

template <int EPI>
int gemm_bf16(cudaStream_t st, int64_t M, int N, int K, const bf16* A, int64_t lda, const bf16* W,
              const float* bias, const float* aux, int ldaux, float* out, int ldo, bf16* outb, int ldob,
              int* status, __half* outh, const float* aux2, const __half* auxh) {
  if (M == 0) return 0;
  // EPI 5: rows (atom, component) of whole atoms, 32-bit row arithmetic in the epilogue
  if (EPI == 5 && (M % 3 != 0 || M >= ((int64_t)1 << 31) || !out || !aux || !aux2 ||
                   (reinterpret_cast<uintptr_t>(aux2) & 15)))
    return -1;
  // the epilogue moves 16-byte quads of FP32 (8-byte quads of BF16) per row
  if (!gemm_bf16_supported(N, K) || (lda * 2) % 16 != 0 || (reinterpret_cast<uintptr_t>(A) & 15) ||
      (reinterpret_cast<uintptr_t>(W) & 15) || (out && (ldo % 4 || (reinterpret_cast<uintptr_t>(out) & 15))) ||
      (outh && ldo % 4) ||
      (outb && (ldob % 4 || (reinterpret_cast<uintptr_t>(outb) & 7))) ||
      (aux && (ldaux % 4 || (reinterpret_cast<uintptr_t>(aux) & 15))) || (bias && (reinterpret_cast<uintptr_t>(bias) & 15)))
    return -1;
  GemmBf16Args p{};
  p.M = M; p.N = N; p.K = K; p.bias = bias; p.aux = aux; p.ldaux = ldaux; p.aux2 = aux2; p.out = out; p.ldo = ldo;
  p.outb = outb; p.ldob = ldob; p.status = status; p.outh = (EPI == 0 || EPI == 1 || EPI == 4) ? outh : nullptr;
  if (p.outh && (reinterpret_cast<uintptr_t>(outh) & 7)) return -1;
  p.auxh = EPI == 6 ? auxh : nullptr;
  if (EPI == 6 && (!auxh || ldaux % 4 || (reinterpret_cast<uintptr_t>(auxh) & 7))) return -1;
  if ((EPI == 2 || EPI == 3) && !aux) return -1;
  p.b_box_rows = N % 64 == 0 ? 64 : 32;
  p.n_chunk = N <= 256 ? N : N / 2;
  if (p.n_chunk > 256 || p.n_chunk % 16) return -1;
  const int KB = (K + kBlockK - 1) / kBlockK;
  const size_t b_bytes = (size_t)KB * N * 128;
  constexpr int kEpiWarps = epi_warps<EPI>();
  const size_t t_bytes = (size_t)kEpiWarps * 32 * kTP * sizeof(float);
  const size_t limit = 227 * 1024 - 1024 - 256 - t_bytes;
  if (b_bytes + 2 * (size_t)kATileBytes > limit) return -1;
  p.a_stages = (int)((limit - b_bytes) / kATileBytes);
  if (p.a_stages > kMaxAStages) p.a_stages = kMaxAStages;
  p.n_acc = 2 * N <= 512 ? 2 : 1;
  uint32_t cols = 32;
  while (cols < (uint32_t)(p.n_acc * N)) cols <<= 1;
  p.tmem_cols = cols;
  CUtensorMap ta, tb;
  if (!make_tmap_bf16(&ta, A, M, K, lda, kTileM) || !make_tmap_bf16(&tb, W, N, K, K, p.b_box_rows)) return -2;
  size_t smem = 1024 + b_bytes + (size_t)p.a_stages * kATileBytes + t_bytes + 256;
  // a CTA holding more than half of TMEM runs alone on its SM, so allocation never waits
  if (p.tmem_cols > 256 && smem < 120 * 1024) smem = 120 * 1024;
  static bool attr_set[7] = {false, false, false, false, false, false, false};
  if (!attr_set[EPI]) {
    cudaFuncSetAttribute(k_gemm_bf16<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr_set[EPI] = true;
  }
  const int64_t ntiles = (M + tile_rows<EPI>() - 1) / tile_rows<EPI>();
  const int grid = (int)(ntiles < num_sms() ? ntiles : num_sms());
  {
    LaunchScope ls_(st);
    k_gemm_bf16<EPI><<<grid, 64 + 32 * kEpiWarps, smem, st>>>(ta, tb, p);
  }
  return 0;
}

template int gemm_bf16<0>(cudaStream_t, int64_t, int, int, const bf16*, int64_t, const bf16*, const float*,
                          const float*, int, float*, int, bf16*, int, int*, __half*, const float*,
                          const __half*);
template int gemm_bf16<1>(cudaStream_t, int64_t, int, int, const bf16*, int64_t, const bf16*, const float*,
                          const float*, int, float*, int, bf16*, int, int*, __half*, const float*,
                          const __half*);
template int gemm_bf16<2>(cudaStream_t, int64_t, int, int, const bf16*, int64_t, const bf16*, const float*,
                          const float*, int, float*, int, bf16*, int, int*, __half*, const float*,
                          const __half*);
template int gemm_bf16<3>(cudaStream_t, int64_t, int, int, const bf16*, int64_t, const bf16*, const float*,
                          const float*, int, float*, int, bf16*, int, int*, __half*, const float*,
                          const __half*);
template int gemm_bf16<4>(cudaStream_t, int64_t, int, int, const bf16*, int64_t, const bf16*, const float*,
                          const float*, int, float*, int, bf16*, int, int*, __half*, const float*,
                          const __half*);
template int gemm_bf16<5>(cudaStream_t, int64_t, int, int, const bf16*, int64_t, const bf16*, const float*,
                          const float*, int, float*, int, bf16*, int, int*, __half*, const float*,
                          const __half*);
template int gemm_bf16<6>(cudaStream_t, int64_t, int, int, const bf16*, int64_t, const bf16*, const float*,
                          const float*, int, float*, int, bf16*, int, int*, __half*, const float*,
                          const __half*);

}  // namespace ctd
