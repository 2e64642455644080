// edge_mma.cu -- the edge message step as a contraction on tcgen05 (BF16 path, F = 128).
//
// The PaiNN message (arXiv 2506.04055, Methods "Graph Neural Networks" / "Chosen
// Architectures"; equations in model_fp32.cu) sums, over the edges e = (i <- j) of receiver i,
//   s_i += phi_s,j W_s,e      v_i += psi_j W_vv,e + u_e phi_vs,j W_vs,e
// with the filter W_c,e = f_c(d_e) (sum_k Wf[c][k] rbf_k(d_e) + bf[c]).  Writing
// b_k(e) = f_c rbf_k (k < K) and b_K(e) = f_c (the bias column), the filter is
// W_c,e = sum_{k <= K} Wf'[c][k] b_k(e) with Wf'[c][K] = bf[c], and the sums reassociate into
//   D_blk[c][k] = sum_e x_blk,j(e)[c] b_k(e)          (x = phi_s, psi_0..2, phi_vs; for phi_vs
//                                                      the basis also carries u_e,a: 3 (K+1) columns)
//   s_i[c] += sum_k Wf'_s[c][k] D_s[c][k],  v_i,a[c] += sum_k Wf'_vv[c][k] D_psi_a[c][k]
//                                                     + sum_k Wf'_vs[c][k] D_vs,a[c][k].
// The first line is a dense contraction over the row's edges, run on the tensor cores: A is the
// senders' message rows (FP16, gathered by TMA tile::gather4 straight into a 128B-swizzled
// MN-major tile: M = 128 channels, K = 16 edges per step), B the per-edge basis (FP16, MN-major,
// N = 32 or 96), D accumulates in TMEM over the row's K-steps.  The second line runs per
// receiver on CUDA cores with the FP32 filter weights.  Both are exact rearrangements of the
// sum; the rounding is that of the FP16 operands (phi to 2^-11 relative, the basis likewise)
// with FP32 accumulation, and the filter weights stay FP32.
//
// CTA (one per SM, persistent over block-cyclic chunks of receiver rows):
//   warps 0..2  producers: per 16-edge unit of a row, the basis tiles and the gathers (ring of
//               kUnits units in shared memory)
//   warp 3      TMEM owner and single-thread MMA issue; per unit 5 MMAs (2 in the first layer,
//               whose psi channels are zero), accumulated into the row's TMEM buffer
//   warps 4..11 two epilogue warpgroups (thread = channel = TMEM lane), taking alternate rows
//               (TMEM buffers 0 / 1): read D, apply the FP32 filter weights, add the residual
// Rows without edges get the residual alone.  All waits are bounded (ST_TIMEOUT on expiry).
#include <cuda_fp16.h>

#include "ctd_internal.cuh"
#include "umma.cuh"

namespace ctd {
namespace {

constexpr int kF = 128;
constexpr int kKS = 16;                              // edges per unit (one MMA K-step)
constexpr int kNBlk = 5;                             // phi_s, psi_0, psi_1, psi_2, phi_vs
constexpr int kABlockBytes = kKS * kF * 2;           // 4096: one block of one unit
constexpr int kBPlainOff = kNBlk * kABlockBytes;     // basis b_k: 16 edges x 32 columns FP16
constexpr int kBUOff = kBPlainOff + kKS * 32 * 2;    // u_a b_k: 16 edges x 96 columns FP16
constexpr int kUnitBytes = kBUOff + kKS * 96 * 2;    // 24576
constexpr int kUnits = 9;
constexpr int kNProd = 3;
constexpr int kMmaWarp = 3;
constexpr int kEpiWarp0 = 4;
constexpr int kThreads_ = 32 * 12;
constexpr int kBufCols = 256;                        // TMEM columns per row buffer (224 used)
constexpr uint32_t kColS = 0, kColPsi = 32, kColVs = 128;

__host__ __device__ constexpr uint32_t idesc_f16_mn(int N) {
  // kind::f16: D F32, A = B = F16, both MN-major, M = 128
  return (1u << 4) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t swz) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)swz << 61;
  return d;
}
// A block of a unit, MN-major 128B swizzle: channel c = c0 + 8 c1 + 64 c2, edge k = k0 + 8 k1 at
// byte c0*2 + (c1 ^ k0)*16 + c2*1024 + k0*128 + k1*2048 (LBO 1024 between channel halves,
// SBO 2048 between 8-edge groups), the layout TMA writes for four gathered rows of 128 B.
__device__ __forceinline__ uint64_t a_desc(uint32_t base) { return desc(base, 1024, 2048, 2); }
// Basis operands, MN-major without swizzle: column n = n0 + 8 n1, edge k = k0 + 8 k1 at byte
// n0*2 + n1*128 + k0*16 + k1*(128 * N/8) (core matrices of 8 edges x 8 columns).
__device__ __forceinline__ uint64_t b_desc(uint32_t base, int N) { return desc(base, 128 * (N / 8), 128, 0); }
__device__ __forceinline__ uint32_t b_off(int n, int k, int N) {
  return (uint32_t)((n >> 3) * 128 + (k & 7) * 16 + (k >> 3) * 128 * (N / 8));
}

__device__ __forceinline__ void gather4(uint32_t dst, const CUtensorMap* map, int col, int r0, int r1, int r2, int r3,
                                        uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(col), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ uint4 pack8(const float* v) {
  uint32_t w[4];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const __half2 x = __floats2half2_rn(v[2 * h], v[2 * h + 1]);
    w[h] = *reinterpret_cast<const uint32_t*>(&x);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

struct MsgArgs {
  int64_t n;
  int64_t chunk_rows;
  int K;
  float rc;
  const int32_t* __restrict__ arow;
  const int32_t* __restrict__ acol;
  const float4* __restrict__ ar;
  const float* __restrict__ S;     // [n][F]
  const float* __restrict__ V;     // [n][3F]
  const float* __restrict__ Wf;    // [3F][KP] FP32
  const float* __restrict__ bf;    // [3F]
  int KP;
  float* __restrict__ SM;
  float* __restrict__ VM;
  __nv_bfloat16* __restrict__ VMb;
  int* status;
};

// The rows of this CTA, in order: block-cyclic chunks of chunk_rows rows.
struct RowIter {
  int64_t chunk, r, r1, n, cr;
  __device__ void begin(const MsgArgs& a) {
    n = a.n;
    cr = a.chunk_rows;
    chunk = blockIdx.x;
    r = chunk * cr;
    r1 = r + cr < n ? r + cr : n;
  }
  __device__ bool valid() const { return r < n; }
  __device__ void next() {
    if (++r >= r1) {
      chunk += gridDim.x;
      r = chunk * cr;
      r1 = r + cr < n ? r + cr : n;
    }
  }
};

template <bool V0, int KC>
__global__ void __launch_bounds__(kThreads_, 1) k_edge_msg_mma(const __grid_constant__ CUtensorMap tmPhi, MsgArgs p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + kUnits * kUnitBytes);   // [kUnits]
  uint64_t* freeb = full + kUnits;                                           // [kUnits]
  uint64_t* tfull = freeb + kUnits;                                          // [2]
  uint64_t* tempty = tfull + 2;                                              // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int K = KC > 0 ? KC : p.K;

  // zero the ring once: padded edge slots then hold finite values whatever was gathered before
  for (int i = threadIdx.x; i < kUnits * kUnitBytes / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(ring)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) {
    for (int u = 0; u < kUnits; ++u) {
      umma::mbar_init(&full[u], 1);
      umma::mbar_init(&freeb[u], 1);
    }
    for (int b = 0; b < 2; ++b) {
      umma::mbar_init(&tfull[b], 1);
      umma::mbar_init(&tempty[b], 4);
    }
    umma::mbar_fence_init();
  }
  if (warp == kMmaWarp) umma::tmem_alloc(tmem_slot, 512);
  umma::fence_proxy_async_smem();
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp < kNProd) {
    // ---------------------------------------------------------------- producers
    const float sig = p.rc / (float)(p.K - 1), inv2s2 = 1.0f / (2.0f * sig * sig), inv_rc = 1.0f / p.rc;
    const int slot = lane & 15, h = lane >> 4;   // h = 0: basis columns 0..15, h = 1: 16..31 and the gathers
    int64_t g = 0;                               // units of this CTA so far (all producers)
    int64_t last_g = -1;                         // this warp's last unit
    RowIter it;
    for (it.begin(p); ok && it.valid(); it.next()) {
      const int e0 = p.arow[it.r], e1 = p.arow[it.r + 1];
      for (int ub = e0; ub < e1; ub += kKS, ++g) {
        if ((int)(g % kNProd) != warp) continue;
        const int u = (int)(g % kUnits);
        // warp-uniform bounded wait (a lane timing out alone would leave the warp divergent)
        if (g >= kUnits && !__all_sync(0xffffffffu, umma::mbar_wait(&freeb[u], (uint32_t)(((g / kUnits) - 1) & 1)))) {
          ok = false;
          break;
        }
        unsigned char* unit = ring + (size_t)u * kUnitBytes;
        const int e = ub + slot;
        const bool live = e < e1;
        float4 r = make_float4(1.f, 0.f, 0.f, 1.f);
        int j = p.acol[ub];   // padded slots gather a live sender's row (finite, times a zero basis)
        if (live) {
          r = p.ar[e];
          j = p.acol[e];
        }
        const float d = r.w, id = 1.0f / d;
        const float fc = live ? 0.5f * (cospif(d * inv_rc) + 1.0f) : 0.0f;
        const float ux = r.x * id, uy = r.y * id, uz = r.z * id;
        float b[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int k = 16 * h + q;
          const float tq = d - (float)k * sig;
          b[q] = k < K ? fc * __expf(-tq * tq * inv2s2) : (k == K ? fc : 0.0f);
        }
        // this lane's two 8-column chunks of the plain basis and of each u_a-weighted copy
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          *reinterpret_cast<uint4*>(unit + kBPlainOff + b_off(16 * h + 8 * c, slot, 32)) = pack8(b + 8 * c);
          float w[8];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const float ua = a == 0 ? ux : (a == 1 ? uy : uz);
#pragma unroll
            for (int x = 0; x < 8; ++x) w[x] = ua * b[8 * c + x];
            *reinterpret_cast<uint4*>(unit + kBUOff + b_off(32 * a + 16 * h + 8 * c, slot, 96)) = pack8(w);
          }
        }
        const int nlive = e1 - ub < kKS ? e1 - ub : kKS;
        const int ngroups = (nlive + 3) >> 2;
        constexpr int nblk = V0 ? 2 : kNBlk;
        umma::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) umma::mbar_expect_tx(&full[u], (uint32_t)(ngroups * nblk * 2 * 4 * 128));
        __syncwarp();
        // gathers: lane 16 + q serves edge group q (slots 4q .. 4q + 3)
        const int jq0 = __shfl_sync(0xffffffffu, j, (4 * (lane & 3)) & 15);
        const int jq1 = __shfl_sync(0xffffffffu, j, (4 * (lane & 3) + 1) & 15);
        const int jq2 = __shfl_sync(0xffffffffu, j, (4 * (lane & 3) + 2) & 15);
        const int jq3 = __shfl_sync(0xffffffffu, j, (4 * (lane & 3) + 3) & 15);
        if (h == 1 && slot < ngroups) {
          const int q = slot;
          const uint32_t dst0 = umma::smem_u32(unit) + (uint32_t)((q >> 1) * 2048 + (q & 1) * 512);
#pragma unroll
          for (int bi = 0; bi < nblk; ++bi) {
            const int blk = V0 ? (bi == 0 ? 0 : 4) : bi;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh)
              gather4(dst0 + (uint32_t)(blk * kABlockBytes + hh * 1024), &tmPhi, blk * kF + hh * 64, jq0, jq1, jq2, jq3,
                      umma::smem_u32(&full[u]));
          }
        }
        last_g = g;
      }
    }
    // every gather this warp issued has landed before the CTA may exit (normally the MMA thread
    // has waited for all of them; after a timeout it may not have): units whose ring slot no
    // later unit reused, the others completed before their slot was refilled
    if (lane == 0)
      for (int64_t q = last_g; q >= 0 && q >= g - kUnits; q -= kNProd)
        umma::mbar_wait(&full[q % kUnits], (uint32_t)((q / kUnits) & 1), 200000000ull);
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint32_t id32 = idesc_f16_mn(32), id96 = idesc_f16_mn(96);
      int64_t g = 0, rows = 0;
      uint64_t* last_bar = nullptr;   // the barrier of the last commit, and its phase parity
      uint32_t last_par = 0;
      RowIter it;
      for (it.begin(p); ok && it.valid(); it.next()) {
        const int e0 = p.arow[it.r], e1 = p.arow[it.r + 1];
        if (e1 == e0) continue;
        const int b = (int)(rows & 1);
        if (rows >= 2 && !umma::mbar_wait(&tempty[b], (uint32_t)(((rows >> 1) - 1) & 1))) { ok = false; break; }
        const uint32_t d0 = tmem + (uint32_t)(b * kBufCols);
        for (int ub = e0; ub < e1; ub += kKS, ++g) {
          const int u = (int)(g % kUnits);
          if (!umma::mbar_wait(&full[u], (uint32_t)((g / kUnits) & 1))) { ok = false; break; }
          umma::fence_after();
          const uint32_t base = umma::smem_u32(ring + (size_t)u * kUnitBytes);
          const uint64_t bp = b_desc(base + kBPlainOff, 32), bu = b_desc(base + kBUOff, 96);
          const uint32_t acc = ub > e0 ? 1u : 0u;
          umma::mma_bf16(d0 + kColS, a_desc(base), bp, id32, acc);
          if (!V0)
            for (int a = 0; a < 3; ++a)
              umma::mma_bf16(d0 + kColPsi + 32 * a, a_desc(base + (uint32_t)((1 + a) * kABlockBytes)), bp, id32, acc);
          umma::mma_bf16(d0 + kColVs, a_desc(base + 4 * kABlockBytes), bu, id96, acc);
          umma::mma_commit(&freeb[u]);
          last_bar = &freeb[u];
          last_par = (uint32_t)((g / kUnits) & 1);
        }
        if (!ok) break;
        umma::mma_commit(&tfull[b]);
        last_bar = &tfull[b];
        last_par = (uint32_t)((rows >> 1) & 1);
        ++rows;
      }
      // every MMA issued has completed before TMEM is released (commits complete in order)
      if (last_bar) umma::mbar_wait(last_bar, last_par, 200000000ull);
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int wg = (warp - kEpiWarp0) >> 2, q4 = warp & 3, c = q4 * 32 + lane;
    // filter weights of channel c with the bias in column K: in registers for the usual basis
    // size (KC = 20), read through L1 per row otherwise
    constexpr int NW = KC > 0 ? KC + 1 : 32;
    constexpr int NR = KC > 0 ? NW : 1;
    float ws[NR], wvv[NR], wvs[NR];
    auto wf = [&](int blk, int k) -> float {
      return k < K ? __ldg(p.Wf + (size_t)(blk * kF + c) * p.KP + k) : (k == K ? __ldg(p.bf + blk * kF + c) : 0.0f);
    };
    if (KC > 0) {
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        ws[k] = wf(0, k);
        wvv[k] = wf(1, k);
        wvs[k] = wf(2, k);
      }
    }
    auto W = [&](const float (&w)[NR], int blk, int k) -> float { return KC > 0 ? w[k < NR ? k : 0] : wf(blk, k); };
    const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16);
    int64_t rows = 0;
    RowIter it;
    for (it.begin(p); it.valid(); it.next()) {
      const int64_t i = it.r;
      const int e0 = p.arow[i], e1 = p.arow[i + 1];
      if (e1 > e0) {
        const int b = (int)(rows & 1);
        const int64_t q = rows++;
        if (b != wg) continue;
        if (!ok) continue;
        const float s_in = p.S[i * kF + c];
        const float v_in0 = p.V[i * 3 * kF + c], v_in1 = p.V[i * 3 * kF + kF + c], v_in2 = p.V[i * 3 * kF + 2 * kF + c];
        if (!__all_sync(0xffffffffu, umma::mbar_wait(&tfull[b], (uint32_t)((q >> 1) & 1)))) {
          ok = false;
          continue;
        }
        umma::fence_after();
        const uint32_t t0 = lane_base + (uint32_t)(b * kBufCols);
        float D[32];
        float ds = 0.f, dv[3];
        // each sum is finished before the next TMEM load (the empty asm consumes it), so that one
        // 32-column tile is live at a time
        umma::tmem_ld32(t0 + kColS, D);
#pragma unroll
        for (int k = 0; k < NW; ++k) ds = fmaf(W(ws, 0, k), D[k], ds);
        asm volatile("" ::"f"(ds));
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          float acc = 0.f;
          if (!V0) {
            umma::tmem_ld32(t0 + kColPsi + 32 * a, D);
#pragma unroll
            for (int k = 0; k < NW; ++k) acc = fmaf(W(wvv, 1, k), D[k], acc);
            asm volatile("" ::"f"(acc));
          }
          umma::tmem_ld32(t0 + kColVs + 32 * a, D);
#pragma unroll
          for (int k = 0; k < NW; ++k) acc = fmaf(W(wvs, 2, k), D[k], acc);
          asm volatile("" ::"f"(acc));
          dv[a] = acc;
        }
        umma::fence_before();
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&tempty[b]);
        const float sm = s_in + ds, vm0 = v_in0 + dv[0], vm1 = v_in1 + dv[1], vm2 = v_in2 + dv[2];
        p.SM[i * kF + c] = sm;
        p.VM[i * 3 * kF + c] = vm0;
        p.VM[i * 3 * kF + kF + c] = vm1;
        p.VM[i * 3 * kF + 2 * kF + c] = vm2;
        if (p.VMb) {
          p.VMb[i * 3 * kF + c] = __float2bfloat16_rn(vm0);
          p.VMb[i * 3 * kF + kF + c] = __float2bfloat16_rn(vm1);
          p.VMb[i * 3 * kF + 2 * kF + c] = __float2bfloat16_rn(vm2);
        }
      } else if (wg == 0) {
        // a row without edges: the residual alone
        const float sm = p.S[i * kF + c];
        const float vm0 = p.V[i * 3 * kF + c], vm1 = p.V[i * 3 * kF + kF + c], vm2 = p.V[i * 3 * kF + 2 * kF + c];
        p.SM[i * kF + c] = sm;
        p.VM[i * 3 * kF + c] = vm0;
        p.VM[i * 3 * kF + kF + c] = vm1;
        p.VM[i * 3 * kF + 2 * kF + c] = vm2;
        if (p.VMb) {
          p.VMb[i * 3 * kF + c] = __float2bfloat16_rn(vm0);
          p.VMb[i * 3 * kF + kF + c] = __float2bfloat16_rn(vm1);
          p.VMb[i * 3 * kF + 2 * kF + c] = __float2bfloat16_rn(vm2);
        }
      }
    }
  }
  if (!ok) atomicOr(p.status, (int)ST_TIMEOUT);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  if (warp == kMmaWarp) umma::tmem_dealloc(tmem, 512);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* q = nullptr;
    cudaDriverEntryPointQueryResult r;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &q, cudaEnableDefault, &r) == cudaSuccess &&
        r == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(q);
  }
  return fn;
}

// Rows of the FP16 message table [n][5F] as gather4 sources: boxes of 64 columns x 1 row, 128B swizzle.
bool make_tmap_rows_f16(CUtensorMap* m, const __half* base, int64_t rows, int cols) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)(rows > 0 ? rows : 1)};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {64, 1};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t msg_smem() { return 1024 + (size_t)kUnits * kUnitBytes + 8 * (2 * kUnits + 4) + 16; }

}  // namespace

bool edge_mma_supported(int F, int K) { return F == kF && K >= 2 && K < 32; }

int edge_fwd_mma(cudaStream_t st, const ModelW& m, int t, int64_t n, const int32_t* arow, const int32_t* acol,
                 const float4* ar, const __half* PHIh, const float* S, const float* V, float* SM, float* VM,
                 __nv_bfloat16* VMb, int* status) {
  if (n == 0) return 0;
  if (!edge_mma_supported(m.F, m.K) || (reinterpret_cast<uintptr_t>(PHIh) & 15)) return -1;
  CUtensorMap tm;
  if (!make_tmap_rows_f16(&tm, PHIh, n, 5 * kF)) return -2;
  MsgArgs a{};
  a.n = n; a.K = m.K; a.rc = m.rc; a.arow = arow; a.acol = acol; a.ar = ar; a.S = S; a.V = V;
  a.Wf = m.L[t].Wf; a.bf = m.L[t].bf; a.KP = m.KP; a.SM = SM; a.VM = VM; a.VMb = VMb; a.status = status;
  a.chunk_rows = m.edge_chunk_rows > 0 ? m.edge_chunk_rows : 32;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t chunks = (n + a.chunk_rows - 1) / a.chunk_rows;
  const int grid = (int)(chunks < sms ? chunks : sms);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_edge_msg_mma<false, 20>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msg_smem());
    cudaFuncSetAttribute(k_edge_msg_mma<true, 20>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msg_smem());
    cudaFuncSetAttribute(k_edge_msg_mma<false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msg_smem());
    cudaFuncSetAttribute(k_edge_msg_mma<true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msg_smem());
    attr = true;
  }
  LaunchScope ls_(st);
  // the first layer's v = 0 (embedding): its psi channels are zero and not gathered
  if (t == 0 && m.K == 20) k_edge_msg_mma<true, 20><<<grid, kThreads_, msg_smem(), st>>>(tm, a);
  else if (t == 0) k_edge_msg_mma<true, 0><<<grid, kThreads_, msg_smem(), st>>>(tm, a);
  else if (m.K == 20) k_edge_msg_mma<false, 20><<<grid, kThreads_, msg_smem(), st>>>(tm, a);
  else k_edge_msg_mma<false, 0><<<grid, kThreads_, msg_smem(), st>>>(tm, a);
  return 0;
}

}  // namespace ctd
