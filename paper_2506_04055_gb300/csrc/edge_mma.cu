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
// senders' message rows (FP16, gathered by per-lane 16-byte asynchronous copies straight into a
// 128B-swizzled MN-major tile: M = 128 channels, K = 16 edges per step), B the per-edge basis
// (FP16, MN-major, N = 32 or 96), D accumulates in TMEM over the row's K-steps.  The second line runs per
// receiver on CUDA cores with the FP32 filter weights.  Both are exact rearrangements of the
// sum; the rounding is that of the FP16 operands (phi to 2^-11 relative, the basis likewise)
// with FP32 accumulation, and the filter weights stay FP32.
//
// CTA (one per SM, persistent over block-cyclic chunks of receiver rows):
//   warps 0..2  producers: per 16-edge unit of a row, the basis tiles and the gathers (ring of
//               kUnits units in shared memory); a unit is full once lane 0 has arrived after the
//               basis stores and every lane's copies have landed (cp.async.mbarrier.arrive)
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
constexpr int kNProd = 6;                            // producer warps
constexpr int kEpiWG = 1;                            // epilogue warpgroups (rows alternate between them)
constexpr int kNMma = 2;                             // MMA-issuing warps (rows alternate between them)
constexpr bool kTmaGather = true;                    // gathers by TMA tile::gather4 (else per-lane cp.async)
constexpr int kMmaWarp = kNProd;
constexpr int kEpiWarp0 = kNProd + kNMma;
constexpr int kThreads_ = 32 * (kNProd + kNMma + 4 * kEpiWG);
// A producer takes every kNProd-th unit and waits for the ring slot's previous unit (kUnits
// back) to be consumed.  Its own previous unit (kNProd back) was admitted only after the unit
// kUnits before that one was consumed, and the MMA consumes in order, so with kNProd <= kUnits
// no producer can run a whole ring ahead, which would alias the slot barriers' phase parity.
static_assert(kNProd <= kUnits, "more producer warps than ring units breaks the slot barrier protocol");
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

// 16-byte asynchronous global -> shared copy (L2 only), and the arrival on an mbarrier once all
// of this thread's earlier copies have landed (counted in the barrier's expected arrivals).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(umma::smem_u32(bar)) : "memory");
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
  const __half* __restrict__ PHIh;   // [n][6F] FP16 message table; columns 0..5F-1 are gathered
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

// The rows of this CTA, in order: block-cyclic chunks of chunk_rows (<= 31) rows.  A warp walks
// them together: lane l holds the row offset arow[r0 + l] of the current chunk (one load per
// chunk), and a row's edge range comes from two shuffles.
struct RowGen {
  int32_t chunk, r0, nrows, off, k, e0, e1, n, cr;
  bool valid;
  __device__ void load(const int32_t* __restrict__ arow, int lane) {
    r0 = chunk * cr;
    nrows = n - r0 < cr ? n - r0 : cr;
    off = lane <= nrows ? arow[r0 + lane] : 0;
    k = 0;
    e0 = __shfl_sync(0xffffffffu, off, 0);
    e1 = __shfl_sync(0xffffffffu, off, 1);
  }
  __device__ void begin(const MsgArgs& a, int lane) {
    n = (int32_t)a.n;
    cr = (int32_t)a.chunk_rows;
    chunk = blockIdx.x;
    valid = chunk * cr < n;
    if (valid) load(a.arow, lane);
  }
  __device__ void next(const int32_t* __restrict__ arow, int lane) {
    if (++k >= nrows) {
      chunk += gridDim.x;
      valid = chunk * cr < n;
      if (valid) load(arow, lane);
    } else {
      e0 = __shfl_sync(0xffffffffu, off, k);
      e1 = __shfl_sync(0xffffffffu, off, k + 1);
    }
  }
  __device__ int32_t row() const { return r0 + k; }
};

// The 16-edge units of this CTA in order (rows without edges have none).
struct UnitCursor {
  RowGen rg;
  int32_t ub;
  __device__ void skip_empty(const int32_t* __restrict__ arow, int lane) {
    while (rg.valid && rg.e0 == rg.e1) rg.next(arow, lane);
    ub = rg.e0;
  }
  __device__ void begin(const MsgArgs& a, int lane) {
    rg.begin(a, lane);
    skip_empty(a.arow, lane);
  }
  __device__ bool valid() const { return rg.valid; }
  __device__ void advance(const int32_t* __restrict__ arow, int lane) {
    ub += kKS;
    if (ub >= rg.e1) {
      rg.next(arow, lane);
      skip_empty(arow, lane);
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
      // TMA: lane 0's arrival with the byte count; copies: lane 0 after the basis, every lane's copies
      umma::mbar_init(&full[u], kTmaGather ? 1 : 1 + 32);
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
    // Warp w takes units w, w + kNProd, ...; the next unit's edge data is loaded while the
    // current one is processed.
    const float sig = p.rc / (float)(p.K - 1), inv2s2 = 1.0f / (2.0f * sig * sig), inv_rc = 1.0f / p.rc;
    const int slot = lane & 15, h = lane >> 4;   // h = 0: basis columns 0..15, h = 1: 16..31
    UnitCursor cur;
    cur.begin(p, lane);
    for (int s = 0; s < warp && cur.valid(); ++s) cur.advance(p.arow, lane);
    int64_t g = warp;        // this unit's index in the CTA's sequence
    int64_t last_g = -1;     // this warp's last unit
    auto fetch = [&](const UnitCursor& c, float4& r, int& j) {
      const int e = c.ub + slot;
      r = make_float4(1.f, 0.f, 0.f, 1.f);
      j = p.acol[c.ub];   // padded slots gather a live sender's row (finite, times a zero basis)
      if (e < c.rg.e1) {
        r = p.ar[e];
        j = p.acol[e];
      }
    };
    float4 r_cur;
    int j_cur = 0;
    if (cur.valid()) fetch(cur, r_cur, j_cur);
    while (ok && cur.valid()) {
      UnitCursor nxt = cur;
      for (int s = 0; s < kNProd && nxt.valid(); ++s) nxt.advance(p.arow, lane);
      float4 r_nxt;
      int j_nxt = 0;
      if (nxt.valid()) fetch(nxt, r_nxt, j_nxt);
      const int u = (int)(g % kUnits);
      // warp-uniform bounded wait (a lane timing out alone would leave the warp divergent)
      if (g >= kUnits && !__all_sync(0xffffffffu, umma::mbar_wait(&freeb[u], (uint32_t)(((g / kUnits) - 1) & 1)))) {
        ok = false;
        break;
      }
      unsigned char* unit = ring + (size_t)u * kUnitBytes;
      const bool live = cur.ub + slot < cur.rg.e1;
      const float4 r = r_cur;
      const int j = j_cur;
      const float d = r.w, id = 1.0f / d;
      const float fc = live ? 0.5f * (cospif(d * inv_rc) + 1.0f) : 0.0f;
      const float ux = r.x * id, uy = r.y * id, uz = r.z * id;
      // Basis columns k = 0 .. 23 of the edge (k < K Gaussians, k = K the cutoff alone, zero above;
      // columns 24 .. 31 stay zero from the ring's initialisation).  The lane pair splits them:
      // h = 0 evaluates k = 0 .. 11 and h = 1 k = 12 .. 23, so each evaluates at most 12
      // exponentials; 8-column chunk 1 (k = 8 .. 15) is assembled by h = 0 from both halves.
      float b[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        const int k = 12 * h + q;
        const float tq = d - (float)k * sig;
        b[q] = k < K ? fc * __expf(-tq * tq * inv2s2) : (k == K ? fc : 0.0f);
      }
      float o[4];   // the partner's k = 12 .. 15 (h = 0 needs them for chunk 1)
#pragma unroll
      for (int q = 0; q < 4; ++q) o[q] = __shfl_xor_sync(0xffffffffu, b[q], 16);
      float ch[2][8];   // this lane's chunks: h = 0: k 0..7 and 8..15; h = 1: k 16..23
      const int nch = h == 0 ? 2 : 1;
#pragma unroll
      for (int x = 0; x < 8; ++x) {
        ch[0][x] = h == 0 ? b[x] : b[4 + x];
        ch[1][x] = x < 4 ? b[8 + x] : o[x - 4];
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (c >= nch) break;
        const int col = h == 0 ? 8 * c : 16;
        *reinterpret_cast<uint4*>(unit + kBPlainOff + b_off(col, slot, 32)) = pack8(ch[c]);
        float w[8];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float ua = a == 0 ? ux : (a == 1 ? uy : uz);
#pragma unroll
          for (int x = 0; x < 8; ++x) w[x] = ua * ch[c][x];
          *reinterpret_cast<uint4*>(unit + kBUOff + b_off(32 * a + col, slot, 96)) = pack8(w);
        }
      }
      const int nlive = cur.rg.e1 - cur.ub < kKS ? cur.rg.e1 - cur.ub : kKS;
      umma::fence_proxy_async_smem();
      __syncwarp();
      if (kTmaGather) {
        // four rows x 128 B per gather4 (channel half hh of block blk of an edge group), spread
        // over the lanes; the barrier completes when lane 0 has arrived and the bytes landed
        constexpr int nbh = (V0 ? 2 : kNBlk) * 2;
        const int ngroups = (nlive + 3) >> 2;
        if (lane == 0) umma::mbar_expect_tx(&full[u], (uint32_t)(ngroups * nbh * 4 * 128));
        __syncwarp();
#pragma unroll
        for (int rep = 0; rep < 2; ++rep) {
          const int ci = lane + 32 * rep;
          const int q = ci % ngroups, bh = ci / ngroups;
          const int j0 = __shfl_sync(0xffffffffu, j, 4 * q), j1 = __shfl_sync(0xffffffffu, j, 4 * q + 1);
          const int j2 = __shfl_sync(0xffffffffu, j, 4 * q + 2), j3 = __shfl_sync(0xffffffffu, j, 4 * q + 3);
          if (bh < nbh) {
            const int bi = bh >> 1, hh = bh & 1;
            const int blk = V0 ? (bi == 0 ? 0 : 4) : bi;
            const uint32_t dst = umma::smem_u32(unit) +
                                 (uint32_t)(blk * kABlockBytes + (q >> 1) * 2048 + hh * 1024 + (q & 1) * 512);
            gather4(dst, &tmPhi, blk * kF + hh * 64, j0, j1, j2, j3, umma::smem_u32(&full[u]));
          }
        }
        last_g = g;
        g += kNProd;
        cur = nxt;
        r_cur = r_nxt;
        j_cur = j_nxt;
        continue;
      }
      if (lane == 0) umma::mbar_arrive(&full[u]);
      // gathers: the live slots' message rows, 16 bytes per copy; item = (slot, block, 16-byte
      // chunk of the 256-byte block), lanes take consecutive chunks of a row (coalesced reads),
      // each written to its 128B-swizzled place (chunk c of edge row k0 sits at chunk c ^ k0)
      constexpr int nbk = V0 ? 2 : kNBlk;   // gathered blocks (the first layer's psi are zero)
      const uint32_t ubase = umma::smem_u32(unit);
      const int items = nlive * nbk * 16;
      for (int base = 0; base < items; base += 32) {   // warp-uniform trip count (shuffles below)
        const int it = base + lane;
        const int sl = it / (nbk * 16), rem = it - sl * (nbk * 16), bi = rem >> 4, q = rem & 15;
        const int js = __shfl_sync(0xffffffffu, j, sl & 15);
        if (it < items) {
          const int blk = V0 ? (bi == 0 ? 0 : 4) : bi;
          const int k0 = sl & 7, hh = q >> 3, cc = q & 7;
          const uint32_t dst = ubase + (uint32_t)(blk * kABlockBytes + (sl >> 3) * 2048 + hh * 1024 + k0 * 128 +
                                                  ((cc ^ k0) << 4));
          cp_async16(dst, p.PHIh + (size_t)js * (6 * kF) + blk * kF + q * 8);
        }
      }
      cp_async_arrive(&full[u]);
      last_g = g;
      g += kNProd;
      cur = nxt;
      r_cur = r_nxt;
      j_cur = j_nxt;
    }
    // the gathers of this warp's last unit have landed before the CTA may exit (normally the MMA
    // thread has waited for all of them; after a timeout it may not have).  No later unit reuses
    // that ring slot (the CTA's last unit is at most kNProd - 1 further); earlier units were
    // issued at least one full unit earlier.
    if (lane == 0 && last_g >= 0)
      umma::mbar_wait(&full[last_g % kUnits], (uint32_t)((last_g / kUnits) & 1), 200000000ull);
  } else if (warp < kMmaWarp + kNMma) {
    // ---------------------------------------------------------------- MMA issue
    // the warp walks the units together (row offsets by chunk); lane 0 issues.  With two MMA
    // warps, warp m issues the rows whose TMEM buffer is m (every other row with edges).
    const int mw = warp - kMmaWarp;
    const uint32_t id32 = idesc_f16_mn(32), id96 = idesc_f16_mn(96);
    int64_t g = 0, rows = 0;
    uint64_t* last_bar = nullptr;   // the barrier of the last commit, and its phase parity
    uint32_t last_par = 0;
    UnitCursor cur;
    for (cur.begin(p, lane); ok && cur.valid(); cur.advance(p.arow, lane), ++g) {
      const bool first = cur.ub == cur.rg.e0, last = cur.ub + kKS >= cur.rg.e1;
      const int b = (int)(rows & 1);
      if (kNMma == 2 && b != mw) {   // the other MMA warp's row
        if (last) ++rows;
        continue;
      }
      if (first && rows >= 2 &&
          !__all_sync(0xffffffffu, umma::mbar_wait(&tempty[b], (uint32_t)(((rows >> 1) - 1) & 1)))) {
        ok = false;
        break;
      }
      const int u = (int)(g % kUnits);
      if (!__all_sync(0xffffffffu, umma::mbar_wait(&full[u], (uint32_t)((g / kUnits) & 1)))) {
        ok = false;
        break;
      }
      // the unit's copies and basis stores (generic proxy) before the MMAs read it (async proxy)
      umma::fence_proxy_async_smem();
      umma::fence_after();
      if (lane == 0) {
        const uint32_t d0 = tmem + (uint32_t)(b * kBufCols);
        const uint32_t base = umma::smem_u32(ring + (size_t)u * kUnitBytes);
        const uint64_t bp = b_desc(base + kBPlainOff, 32), bu = b_desc(base + kBUOff, 96);
        const uint32_t acc = first ? 0u : 1u;
        umma::mma_bf16(d0 + kColS, a_desc(base), bp, id32, acc);
        if (!V0)
          for (int a = 0; a < 3; ++a)
            umma::mma_bf16(d0 + kColPsi + 32 * a, a_desc(base + (uint32_t)((1 + a) * kABlockBytes)), bp, id32, acc);
        umma::mma_bf16(d0 + kColVs, a_desc(base + 4 * kABlockBytes), bu, id96, acc);
        umma::mma_commit(&freeb[u]);
        if (last) umma::mma_commit(&tfull[b]);
      }
      __syncwarp();
      last_bar = last ? &tfull[b] : &freeb[u];
      last_par = last ? (uint32_t)((rows >> 1) & 1) : (uint32_t)((g / kUnits) & 1);
      if (last) ++rows;
    }
    // every MMA issued has completed before TMEM is released (commits complete in order)
    if (lane == 0 && last_bar) umma::mbar_wait(last_bar, last_par, 200000000ull);
  } else {
    // ---------------------------------------------------------------- epilogue
    const int wg = (warp - kEpiWarp0) >> 2, q4 = warp & 3, c = q4 * 32 + lane;
    // filter weights of channel c with the bias in column K.  For the usual basis size (KC = 20)
    // the vs row stays in registers and the s and vv rows are reloaded (L1) before each use, so
    // that two rows of weights are live at a time; for other sizes every weight is read through
    // L1 where it is used.
    constexpr int NW = KC > 0 ? KC + 1 : 32;
    constexpr int NR = KC > 0 ? NW : 1;
    float ws[NR], wvv[NR], wvs[NR];
    auto wf = [&](int blk, int k) -> float {
      return k < K ? __ldg(p.Wf + (size_t)(blk * kF + c) * p.KP + k) : (k == K ? __ldg(p.bf + blk * kF + c) : 0.0f);
    };
    // a load the compiler does not hoist out of the row loop
    auto wf_row = [&](int blk, int k) -> float {
      const float* q = k < K ? p.Wf + (size_t)(blk * kF + c) * p.KP + k : p.bf + blk * kF + c;
      float v;
      asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(q));
      return k <= K ? v : 0.0f;
    };
    if (KC > 0) {
#pragma unroll
      for (int k = 0; k < NR; ++k) wvs[k] = wf(2, k);
    }
    auto W = [&](const float (&w)[NR], int blk, int k) -> float { return KC > 0 ? w[k < NR ? k : 0] : wf(blk, k); };
    const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16);
    int64_t rows = 0;
    RowGen it;
    for (it.begin(p, lane); it.valid; it.next(p.arow, lane)) {
      const int64_t i = it.row();
      const int e0 = it.e0, e1 = it.e1;
      if (e1 > e0) {
        const int b = (int)(rows & 1);
        const int64_t q = rows++;
        if (kEpiWG == 2 && b != wg) continue;
        if (!ok) continue;
        const float s_in = p.S[i * kF + c];
        // V null: the first layer, whose input vector features are zero
        const float v_in0 = p.V ? p.V[i * 3 * kF + c] : 0.f, v_in1 = p.V ? p.V[i * 3 * kF + kF + c] : 0.f,
                    v_in2 = p.V ? p.V[i * 3 * kF + 2 * kF + c] : 0.f;
        if (!__all_sync(0xffffffffu, umma::mbar_wait(&tfull[b], (uint32_t)((q >> 1) & 1)))) {
          ok = false;
          continue;
        }
        umma::fence_after();
        const uint32_t t0 = lane_base + (uint32_t)(b * kBufCols);
        float D[32];
        float ds = 0.f, dv[3];
        // each sum is finished before the next TMEM load (the empty asm consumes it), so that one
        // group of accumulator columns is live at a time; with KC = 20 the 21 used columns of a
        // group are read as 16 + 8
        auto group = [&](uint32_t col, const float (&w)[NR], int blk, float acc) -> float {
          if (KC > 0 && NW <= 24) {
            float lo[16], hi[8];
            umma::tmem_ld16(col, lo);
#pragma unroll
            for (int k = 0; k < 16; ++k) acc = fmaf(W(w, blk, k), lo[k], acc);
            asm volatile("" ::"f"(acc));
            umma::tmem_ld8(col + 16, hi);
#pragma unroll
            for (int k = 16; k < NW; ++k) acc = fmaf(W(w, blk, k), hi[k - 16], acc);
          } else {
            umma::tmem_ld32(col, D);
#pragma unroll
            for (int k = 0; k < NW; ++k) acc = fmaf(W(w, blk, k), D[k], acc);
          }
          asm volatile("" ::"f"(acc));
          return acc;
        };
        if (KC > 0) {
#pragma unroll
          for (int k = 0; k < NR; ++k) ws[k] = wf_row(0, k);
        }
        ds = group(t0 + kColS, ws, 0, 0.f);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          float acc = 0.f;
          if (!V0) {
            if (KC > 0) {
#pragma unroll
              for (int k = 0; k < NR; ++k) wvv[k] = wf_row(1, k);
            }
            acc = group(t0 + kColPsi + 32 * a, wvv, 1, acc);
          }
          dv[a] = group(t0 + kColVs + 32 * a, wvs, 2, acc);
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
        const float vm0 = p.V ? p.V[i * 3 * kF + c] : 0.f, vm1 = p.V ? p.V[i * 3 * kF + kF + c] : 0.f,
                    vm2 = p.V ? p.V[i * 3 * kF + 2 * kF + c] : 0.f;
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

// The first `cols` columns of the rows of an FP16 table with `ld` columns per row as gather4
// sources: boxes of 64 columns x 1 row, 128B swizzle.
bool make_tmap_rows_f16(CUtensorMap* m, const __half* base, int64_t rows, int cols, int ld) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)(rows > 0 ? rows : 1)};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
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
  CUtensorMap tm{};
  if (kTmaGather && !make_tmap_rows_f16(&tm, PHIh, n, 5 * kF, 6 * kF)) return -2;
  MsgArgs a{};
  a.PHIh = PHIh;
  a.n = n; a.K = m.K; a.rc = m.rc; a.arow = arow; a.acol = acol; a.ar = ar; a.S = S; a.V = V;
  a.Wf = m.L[t].Wf; a.bf = m.L[t].bf; a.KP = m.KP; a.SM = SM; a.VM = VM; a.VMb = VMb; a.status = status;
  // rows per block-cyclic chunk: at most 31 (a warp holds a chunk's row offsets, one per lane)
  a.chunk_rows = m.edge_chunk_rows > 0 && m.edge_chunk_rows < 31 ? m.edge_chunk_rows : 16;
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
