// edge_tc.cu -- edge message and its adjoint with the radial filter contraction on tcgen05
// (BF16 path, F = 128, radial basis K <= 32).
//
// The filter W_e = (Wf rbf(d_e) + bf) f_c(d_e) (PaiNN message function, arXiv 2506.04055
// Methods "Graph Neural Networks" / "Chosen Architectures") is a [3F x K] x [K x edges]
// contraction per tile of edges: D[c][e] = sum_k Wf[c][k] rbf_k(d_e).  It runs as UMMA with
// M = 128 filter channels (three M tiles: the s, vv and vs blocks), N = edges of the tile,
// K = 32 (the basis zero-padded), BF16 operands and FP32 accumulation in TMEM.  Everything
// after the contraction (bias, cutoff, message gathers, the segmented receiver sums, the
// adjoint terms) stays FP32 on CUDA cores.
//
// CTA layout (192 threads, two CTAs per SM):
//   warp 0   producer: per edge of the next tile, geometry, f_c and the basis (and its radial
//            derivative for the adjoint), written as a 128B-swizzled BF16 tile; Wf arrives
//            once per CTA by TMA
//   warp 1   TMEM owner and single-thread MMA issue
//   warps 2-5 epilogue: thread = feature channel f (TMEM lane), walks the tile's edges in CSR
//            order; a receiver's sums stay in registers until its row ends (no atomics)
// Each CTA owns a contiguous range of receiver rows, so no row is split between CTAs.  All
// waits are bounded and record ST_TIMEOUT on expiry.
#include "ctd_internal.cuh"
#include "umma.cuh"

namespace ctd {

using bf16 = __nv_bfloat16;

namespace {

constexpr int kF = 128;
constexpr int kKPad = 32;
constexpr int kWfTileBytes = 128 * 128;      // one M tile: 128 rows x 128 B
constexpr int kWfBytes = 3 * kWfTileBytes;   // s, vv, vs blocks

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

// Write 32 basis values (k = 0..31) of one edge as row `r` of a 128B-swizzled BF16 tile.
__device__ __forceinline__ void store_basis_row(unsigned char* tile, int r, const float (&v)[kKPad]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      __nv_bfloat162 b2 = __floats2bfloat162_rn(v[8 * c + 2 * h], v[8 * c + 2 * h + 1]);
      w[h] = *reinterpret_cast<uint32_t*>(&b2);
    }
    *reinterpret_cast<uint4*>(tile + umma::sw128_offset(r, 8 * c)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

struct EdgeTcArgs {
  int64_t n;
  int64_t rows_per_cta;
  int K;
  float rc;
  int accumulate;
  const int32_t* __restrict__ arow;
  const int32_t* __restrict__ acol;
  const float4* __restrict__ ar;
  const float* __restrict__ PHI;   // [n][6F]
  const float* __restrict__ S;     // [n][F]
  const float* __restrict__ V;     // [n][3F]
  const float* __restrict__ Gsm;   // [n][F]   (adjoint)
  const float* __restrict__ Gvm;   // [n][3F]  (adjoint)
  const float* __restrict__ bf;    // [3F]
  float* __restrict__ SM;
  float* __restrict__ VM;
  bf16* __restrict__ VMb;
  float* __restrict__ GPHI;        // [n][5F]  (adjoint)
  float4* __restrict__ hedge;      // [E]      (adjoint)
  int* status;
};

}  // namespace

// ------------------------------------------------------------------------------ message
// Row bookkeeping shared by both kernels: the producer marks, for each edge slot of a tile,
// how many rows end at that edge (the row itself plus any empty rows right after it); rows
// without edges at the start of the CTA's range are flushed before the first tile.
__device__ __forceinline__ void mark_row_ends(int lane, int* sfl, int NE, int64_t tb, int64_t r1,
                                              const int32_t* __restrict__ arow, int64_t& rp) {
  for (int s = lane; s < NE; s += 32) sfl[s] = 0;
  __syncwarp();
  if (lane == 0) {
    while (rp < r1) {
      const int64_t v = arow[rp + 1];
      if (v > tb + NE) break;
      sfl[v - 1 - tb] += 1;
      ++rp;
    }
  }
  __syncwarp();
}

template <int NE>
__global__ void __launch_bounds__(192, 2) k_edge_fwd_tc(const __grid_constant__ CUtensorMap tmWf, EdgeTcArgs p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = align1024(smem_raw);
  unsigned char* sA = smem;                                  // Wf tiles
  unsigned char* sB = sA + kWfBytes;                         // [2][NE x 128 B] basis tiles
  int* sj = reinterpret_cast<int*>(sB + 2 * NE * 128);       // [2][NE] sender index
  int* sfl = sj + 2 * NE;                                    // [2][NE] rows ending at the slot
  float4* sgeo = reinterpret_cast<float4*>(sfl + 2 * NE);    // [2][NE] (u, f_c)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sgeo + 2 * NE);
  uint64_t* wbar = bars;
  uint64_t* bready = bars + 1;   // [2]
  uint64_t* bfree = bars + 3;    // [2]
  uint64_t* tfull = bars + 5;
  uint64_t* tempty = bars + 6;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 7);

  const int64_t r0 = (int64_t)blockIdx.x * p.rows_per_cta;
  if (r0 >= p.n) return;
  const int64_t r1 = (r0 + p.rows_per_cta < p.n) ? r0 + p.rows_per_cta : p.n;
  const int64_t e0 = p.arow[r0], e1 = p.arow[r1];
  const int ntiles = (int)((e1 - e0 + NE - 1) / NE);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    umma::mbar_init(wbar, 1);
    for (int i = 0; i < 2; ++i) {
      umma::mbar_init(&bready[i], 1);
      umma::mbar_init(&bfree[i], 4);
    }
    umma::mbar_init(tfull, 1);
    umma::mbar_init(tempty, 4);
    umma::mbar_fence_init();
  }
  if (warp == 1) umma::tmem_alloc(tmem_slot, 256);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  int issued = 0;

  if (warp == 0) {
    if (lane == 0) {
      umma::mbar_expect_tx(wbar, kWfBytes);
      for (int m = 0; m < 3; ++m) umma::tma_load_2d(sA + m * kWfTileBytes, &tmWf, 0, m * 128, wbar);
    }
    const float sig = p.rc / (float)(p.K - 1), inv2s2 = 1.0f / (2.0f * sig * sig), inv_rc = 1.0f / p.rc;
    int64_t rp = r0;
    while (rp < r1 && p.arow[rp + 1] == e0) ++rp;   // leading empty rows: flushed by the epilogue
    for (int it = 0; it < ntiles; ++it) {
      const int b = it & 1;
      if (it >= 2 && !umma::mbar_wait(&bfree[b], ((it >> 1) - 1) & 1)) { ok = false; break; }
      unsigned char* tile = sB + b * NE * 128;
      const int64_t tb = e0 + (int64_t)it * NE;
      for (int s = lane; s < NE; s += 32) {
        const int64_t e = tb + s;
        float rb[kKPad];
        int j = 0;
        float4 geo = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < e1) {
          const float4 r = p.ar[e];
          const float d = r.w, id = 1.0f / d;
          geo = make_float4(r.x * id, r.y * id, r.z * id, 0.5f * (cospif(d * inv_rc) + 1.0f));
          j = p.acol[e];
#pragma unroll
          for (int k = 0; k < kKPad; ++k) {
            const float t = d - (float)k * sig;
            rb[k] = k < p.K ? expf(-t * t * inv2s2) : 0.0f;
          }
        } else {
#pragma unroll
          for (int k = 0; k < kKPad; ++k) rb[k] = 0.0f;
        }
        store_basis_row(tile, s, rb);
        sj[b * NE + s] = j;
        sgeo[b * NE + s] = geo;
      }
      mark_row_ends(lane, sfl + b * NE, NE, tb, r1, p.arow, rp);
      umma::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&bready[b]);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      if (!umma::mbar_wait(wbar, 0)) ok = false;
      const uint32_t idesc = umma::idesc_bf16_m128(NE);
      for (int it = 0; ok && it < ntiles; ++it) {
        const int b = it & 1;
        if (!umma::mbar_wait(&bready[b], (it >> 1) & 1)) { ok = false; break; }
        if (it >= 1 && !umma::mbar_wait(tempty, (it - 1) & 1)) { ok = false; break; }
        umma::fence_after();
        const uint32_t bbase = umma::smem_u32(sB + b * NE * 128);
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
          for (int k = 0; k < 2; ++k)
            umma::mma_bf16(tmem + (uint32_t)(m * NE), umma::desc_sw128(umma::smem_u32(sA + m * kWfTileBytes) + 32u * k),
                           umma::desc_sw128(bbase + 32u * k), idesc, k > 0);
        umma::mma_commit(tfull);
        ++issued;
      }
    }
  } else {
    const int q = warp & 3, f = q * 32 + lane;
    const float bs = p.bf[f], bvv = p.bf[kF + f], bvs = p.bf[2 * kF + f];
    int64_t r = r0;
    float as = 0.f, a0 = 0.f, a1 = 0.f, a2 = 0.f;
    auto flush = [&]() {
      const int64_t i = r;
      const float sm = p.S[i * kF + f] + as;
      const float v0 = p.V[i * 3 * kF + f] + a0, v1 = p.V[i * 3 * kF + kF + f] + a1,
                  v2 = p.V[i * 3 * kF + 2 * kF + f] + a2;
      p.SM[i * kF + f] = sm;
      p.VM[i * 3 * kF + f] = v0;
      p.VM[i * 3 * kF + kF + f] = v1;
      p.VM[i * 3 * kF + 2 * kF + f] = v2;
      if (p.VMb) {
        p.VMb[i * 3 * kF + f] = __float2bfloat16_rn(v0);
        p.VMb[i * 3 * kF + kF + f] = __float2bfloat16_rn(v1);
        p.VMb[i * 3 * kF + 2 * kF + f] = __float2bfloat16_rn(v2);
      }
      as = a0 = a1 = a2 = 0.f;
      ++r;
    };
    while (r < r1 && p.arow[r + 1] == e0) flush();
    for (int it = 0; it < ntiles; ++it) {
      const int b = it & 1;
      if (!umma::mbar_wait(tfull, it & 1)) { ok = false; break; }
      umma::fence_after();
      const int64_t tb = e0 + (int64_t)it * NE;
      const int nlive = (int)((e1 - tb) < NE ? (e1 - tb) : NE);
      const int* tj = sj + b * NE;
      const int* tf = sfl + b * NE;
      const float4* tg = sgeo + b * NE;
      float ga[8][5], gb[8][5];
      // neighbour messages of 8 edges: phi_s, psi_0..2, phi_vs of sender j, channel f
      auto gather8 = [&](float (&G)[8][5], int s0) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const bool live = s0 + u < nlive;
          const float* pj = p.PHI + (int64_t)(live ? tj[s0 + u] : 0) * 6 * kF + f;
#pragma unroll
          for (int k = 0; k < 5; ++k) G[u][k] = live ? __ldg(pj + k * kF) : 0.f;
        }
      };
      auto compute8 = [&](const float (&G)[8][5], int s0, const float* ds, const float* dv, const float* dw) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (s0 + u < nlive) {
            const float4 geo = tg[s0 + u];
            const float fc = geo.w;
            const float ws = (ds[u] + bs) * fc, wvv = (dv[u] + bvv) * fc, wvs = (dw[u] + bvs) * fc;
            as = fmaf(G[u][0], ws, as);
            const float tvs = G[u][4] * wvs;
            a0 = fmaf(G[u][1], wvv, fmaf(geo.x, tvs, a0));
            a1 = fmaf(G[u][2], wvv, fmaf(geo.y, tvs, a1));
            a2 = fmaf(G[u][3], wvv, fmaf(geo.z, tvs, a2));
            for (int nf = tf[s0 + u]; nf > 0; --nf) flush();
          }
        }
      };
      gather8(ga, 0);
#pragma unroll
      for (int c = 0; c < NE / 16; ++c) {
        float ds[16], dv[16], dw[16];
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(c * 16);
        umma::tmem_ld16(ta, ds);
        umma::tmem_ld16(ta + NE, dv);
        umma::tmem_ld16(ta + 2 * NE, dw);
        if (c == NE / 16 - 1) {
          umma::fence_before();
          __syncwarp();
          if (lane == 0) umma::mbar_arrive(tempty);
        }
        gather8(gb, c * 16 + 8);
        compute8(ga, c * 16, ds, dv, dw);
        if (c + 1 < NE / 16) gather8(ga, (c + 1) * 16);
        compute8(gb, c * 16 + 8, ds + 8, dv + 8, dw + 8);
      }
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&bfree[b]);
    }
    if (ok)
      while (r < r1) flush();
  }
  if (!ok) atomicOr(p.status, (int)ST_TIMEOUT);
  // the MMAs of the last issued tile have completed before TMEM is released
  if (warp == 1 && lane == 0 && issued > 0) umma::mbar_wait(tfull, (issued - 1) & 1, 200000000ull);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  if (warp == 1) umma::tmem_dealloc(tmem, 256);
}

// ------------------------------------------------------------------------------ adjoint
// Sender-side: row j walks edges e' = (j <- i); the reverse edge (i <- j) carried phi_j, v_j
// into receiver i with direction -u_e'.  Per tile the MMA gives both the filter W~ (basis)
// and its radial derivative W~' (derivative basis).  Per edge the channel partials of dU/dd
// and dU/du_rev are reduced over the four epilogue warps and turned into hedge[e'].
template <int NE>
__global__ void __launch_bounds__(192, 2) k_edge_bwd_tc(const __grid_constant__ CUtensorMap tmWf, EdgeTcArgs p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = align1024(smem_raw);
  unsigned char* sA = smem;                                    // Wf tiles
  unsigned char* sB = sA + kWfBytes;                           // [2][2][NE x 128 B] basis, derivative
  int* sj = reinterpret_cast<int*>(sB + 4 * NE * 128);         // [2][NE]
  int* sfl = sj + 2 * NE;                                      // [2][NE]
  float4* sgeo = reinterpret_cast<float4*>(sfl + 2 * NE);      // [2][NE] (u, d)
  float2* sfc = reinterpret_cast<float2*>(sgeo + 2 * NE);      // [2][NE] (f_c, f_c')
  float* red = reinterpret_cast<float*>(sfc + 2 * NE);         // [NE][4 warps][4]
  uint64_t* bars = reinterpret_cast<uint64_t*>(red + NE * 16);
  uint64_t* wbar = bars;
  uint64_t* bready = bars + 1;   // [2]
  uint64_t* bfree = bars + 3;    // [2]
  uint64_t* tfull = bars + 5;
  uint64_t* tempty = bars + 6;
  uint64_t* esync = bars + 7;    // [2] epilogue warps: partials written / edge gradients written
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 9);

  const int64_t r0 = (int64_t)blockIdx.x * p.rows_per_cta;
  if (r0 >= p.n) return;
  const int64_t r1 = (r0 + p.rows_per_cta < p.n) ? r0 + p.rows_per_cta : p.n;
  const int64_t e0 = p.arow[r0], e1 = p.arow[r1];
  const int ntiles = (int)((e1 - e0 + NE - 1) / NE);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    umma::mbar_init(wbar, 1);
    for (int i = 0; i < 2; ++i) {
      umma::mbar_init(&bready[i], 1);
      umma::mbar_init(&bfree[i], 4);
    }
    umma::mbar_init(tfull, 1);
    umma::mbar_init(tempty, 4);
    umma::mbar_init(&esync[0], 4);
    umma::mbar_init(&esync[1], 4);
    umma::mbar_fence_init();
  }
  if (warp == 1) umma::tmem_alloc(tmem_slot, 256);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  int issued = 0;

  if (warp == 0) {
    if (lane == 0) {
      umma::mbar_expect_tx(wbar, kWfBytes);
      for (int m = 0; m < 3; ++m) umma::tma_load_2d(sA + m * kWfTileBytes, &tmWf, 0, m * 128, wbar);
    }
    const float sig = p.rc / (float)(p.K - 1), inv2s2 = 1.0f / (2.0f * sig * sig), inv_s2 = 1.0f / (sig * sig);
    const float inv_rc = 1.0f / p.rc;
    int64_t rp = r0;
    while (rp < r1 && p.arow[rp + 1] == e0) ++rp;
    for (int it = 0; it < ntiles; ++it) {
      const int b = it & 1;
      if (it >= 2 && !umma::mbar_wait(&bfree[b], ((it >> 1) - 1) & 1)) { ok = false; break; }
      unsigned char* tile = sB + (2 * b) * NE * 128;
      unsigned char* dtile = sB + (2 * b + 1) * NE * 128;
      const int64_t tb = e0 + (int64_t)it * NE;
      for (int s = lane; s < NE; s += 32) {
        const int64_t e = tb + s;
        float rb[kKPad], drb[kKPad];
        int i = 0;
        float4 geo = make_float4(0.f, 0.f, 0.f, 1.f);
        float2 fcv = make_float2(0.f, 0.f);
        if (e < e1) {
          const float4 r = p.ar[e];
          const float d = r.w, id = 1.0f / d;
          geo = make_float4(r.x * id, r.y * id, r.z * id, d);
          fcv = make_float2(0.5f * (cospif(d * inv_rc) + 1.0f), -0.5f * 3.14159265358979f * inv_rc * sinpif(d * inv_rc));
          i = p.acol[e];
#pragma unroll
          for (int k = 0; k < kKPad; ++k) {
            const float t = d - (float)k * sig;
            const float v = k < p.K ? expf(-t * t * inv2s2) : 0.0f;
            rb[k] = v;
            drb[k] = -v * t * inv_s2;
          }
        } else {
#pragma unroll
          for (int k = 0; k < kKPad; ++k) rb[k] = drb[k] = 0.0f;
        }
        store_basis_row(tile, s, rb);
        store_basis_row(dtile, s, drb);
        sj[b * NE + s] = i;
        sgeo[b * NE + s] = geo;
        sfc[b * NE + s] = fcv;
      }
      mark_row_ends(lane, sfl + b * NE, NE, tb, r1, p.arow, rp);
      umma::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&bready[b]);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      if (!umma::mbar_wait(wbar, 0)) ok = false;
      const uint32_t idesc = umma::idesc_bf16_m128(NE);
      for (int it = 0; ok && it < ntiles; ++it) {
        const int b = it & 1;
        if (!umma::mbar_wait(&bready[b], (it >> 1) & 1)) { ok = false; break; }
        if (it >= 1 && !umma::mbar_wait(tempty, (it - 1) & 1)) { ok = false; break; }
        umma::fence_after();
#pragma unroll
        for (int h = 0; h < 2; ++h) {          // h = 0: basis -> W~, h = 1: derivative -> W~'
          const uint32_t bbase = umma::smem_u32(sB + (2 * b + h) * NE * 128);
#pragma unroll
          for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int k = 0; k < 2; ++k)
              umma::mma_bf16(tmem + (uint32_t)((3 * h + m) * NE),
                             umma::desc_sw128(umma::smem_u32(sA + m * kWfTileBytes) + 32u * k),
                             umma::desc_sw128(bbase + 32u * k), idesc, k > 0);
        }
        umma::mma_commit(tfull);
        ++issued;
      }
    }
  } else {
    const int q = warp & 3, f = q * 32 + lane;
    const float bs = p.bf[f], bvv = p.bf[kF + f], bvs = p.bf[2 * kF + f];
    int64_t r = r0;
    // this row's own messages phi_s, psi_0..2, phi_vs (channel f), and the next row's, prefetched
    float cur[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, nxt[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    auto fetch = [&](int64_t row, float (&o)[5]) {
      if (row < r1) {
        const float* pj = p.PHI + row * 6 * kF + f;
#pragma unroll
        for (int k = 0; k < 5; ++k) o[k] = __ldg(pj + k * kF);
      }
    };
    float gps = 0.f, gy0 = 0.f, gy1 = 0.f, gy2 = 0.f, gpvs = 0.f;
    auto flush = [&]() {
      float* o = p.GPHI + r * 5 * kF;
      o[f] = gps; o[kF + f] = gy0; o[2 * kF + f] = gy1; o[3 * kF + f] = gy2; o[4 * kF + f] = gpvs;
      gps = gy0 = gy1 = gy2 = gpvs = 0.f;
      ++r;
#pragma unroll
      for (int k = 0; k < 5; ++k) cur[k] = nxt[k];
      fetch(r + 1, nxt);
    };
    fetch(r, cur);
    fetch(r + 1, nxt);
    while (r < r1 && p.arow[r + 1] == e0) flush();
    for (int it = 0; it < ntiles; ++it) {
      const int b = it & 1;
      if (!umma::mbar_wait(tfull, it & 1)) { ok = false; break; }
      umma::fence_after();
      const int64_t tb = e0 + (int64_t)it * NE;
      const int nlive = (int)((e1 - tb) < NE ? (e1 - tb) : NE);
      const int* ti = sj + b * NE;
      const int* tf = sfl + b * NE;
      const float4* tg = sgeo + b * NE;
      const float2* tc = sfc + b * NE;
      float ga[8][4], gb[8][4];
      // receivers' gradients (gsm_i, gvm_i) of 8 edges, channel f
      auto gather8 = [&](float (&G)[8][4], int s0) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const bool live = s0 + u < nlive;
          const int64_t i = live ? ti[s0 + u] : 0;
          G[u][0] = live ? __ldg(p.Gsm + i * kF + f) : 0.f;
          G[u][1] = live ? __ldg(p.Gvm + i * 3 * kF + f) : 0.f;
          G[u][2] = live ? __ldg(p.Gvm + i * 3 * kF + kF + f) : 0.f;
          G[u][3] = live ? __ldg(p.Gvm + i * 3 * kF + 2 * kF + f) : 0.f;
        }
      };
      auto compute8 = [&](const float (&G)[8][4], int s0, const float (&W)[6][8]) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int slot = s0 + u;
          float pd = 0.f, pu0 = 0.f, pu1 = 0.f, pu2 = 0.f;
          const bool live = slot < nlive;
          if (live) {
            const float4 geo = tg[slot];
            const float2 fcv = tc[slot];
            const float ws = W[0][u] + bs, wvv = W[1][u] + bvv, wvs = W[2][u] + bvs;
            const float fc = fcv.x, dfc = fcv.y;
            const float Ws = ws * fc, Wvv = wvv * fc, Wvs = wvs * fc;
            const float gs = G[u][0], gv0 = G[u][1], gv1 = G[u][2], gv2 = G[u][3];
            gps = fmaf(gs, Ws, gps);
            gy0 = fmaf(gv0, Wvv, gy0);
            gy1 = fmaf(gv1, Wvv, gy1);
            gy2 = fmaf(gv2, Wvv, gy2);
            const float qv = -(gv0 * geo.x + gv1 * geo.y + gv2 * geo.z);
            gpvs = fmaf(qv, Wvs, gpvs);
            const float gWs = gs * cur[0], gWvv = gv0 * cur[1] + gv1 * cur[2] + gv2 * cur[3], gWvs = qv * cur[4];
            pd = fc * (gWs * W[3][u] + gWvv * W[4][u] + gWvs * W[5][u]) + dfc * (gWs * ws + gWvv * wvv + gWvs * wvs);
            const float tv = cur[4] * Wvs;
            pu0 = gv0 * tv; pu1 = gv1 * tv; pu2 = gv2 * tv;
          }
          // sum over the 32 channels of this warp: lane 8v ends with value v
          const bool hi = lane & 16;
          float s0v = hi ? pd : pu1, s1v = hi ? pu0 : pu2;
          float k0 = hi ? pu1 : pd, k1 = hi ? pu2 : pu0;
          k0 += __shfl_xor_sync(0xffffffffu, s0v, 16);
          k1 += __shfl_xor_sync(0xffffffffu, s1v, 16);
          const bool b8 = lane & 8;
          float sv = b8 ? k0 : k1, kk = b8 ? k1 : k0;
          kk += __shfl_xor_sync(0xffffffffu, sv, 8);
          kk += __shfl_xor_sync(0xffffffffu, kk, 4);
          kk += __shfl_xor_sync(0xffffffffu, kk, 2);
          kk += __shfl_xor_sync(0xffffffffu, kk, 1);
          if ((lane & 7) == 0) red[(slot * 4 + q) * 4 + (lane >> 3)] = kk;
          if (live)
            for (int nf = tf[slot]; nf > 0; --nf) flush();
        }
      };
      gather8(ga, 0);
#pragma unroll
      for (int c = 0; c < NE / 8; ++c) {
        float W[6][8];
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(c * 8);
#pragma unroll
        for (int h = 0; h < 6; ++h) umma::tmem_ld8(ta + h * NE, W[h]);
        if (c == NE / 8 - 1) {
          umma::fence_before();
          __syncwarp();
          if (lane == 0) umma::mbar_arrive(tempty);
        }
        if (c % 2 == 0) {
          if (c + 1 < NE / 8) gather8(gb, (c + 1) * 8);
          compute8(ga, c * 8, W);
        } else {
          if (c + 1 < NE / 8) gather8(ga, (c + 1) * 8);
          compute8(gb, c * 8, W);
        }
      }
      // all four epilogue warps have written their partials for this tile
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&esync[0]);
      if (!umma::mbar_wait(&esync[0], it & 1)) { ok = false; break; }
      const int t = f;   // 128 threads, NE <= 128 slots
      if (t < nlive) {
        float pd = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const float* rr = red + (t * 4 + w) * 4;
          pd += rr[0]; g0 += rr[1]; g1 += rr[2]; g2 += rr[3];
        }
        const float4 geo = tg[t];
        const float ux = -geo.x, uy = -geo.y, uz = -geo.z, id = 1.0f / geo.w;
        const float gdu = g0 * ux + g1 * uy + g2 * uz;
        float4 h = make_float4(pd * ux + (g0 - gdu * ux) * id, pd * uy + (g1 - gdu * uy) * id,
                               pd * uz + (g2 - gdu * uz) * id, 0.f);
        const int64_t e = tb + t;
        if (p.accumulate) {
          const float4 o = p.hedge[e];
          h.x += o.x; h.y += o.y; h.z += o.z;
        }
        p.hedge[e] = h;
      }
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&esync[1]);
      if (!umma::mbar_wait(&esync[1], it & 1)) { ok = false; break; }
      if (lane == 0) umma::mbar_arrive(&bfree[b]);
    }
    if (ok)
      while (r < r1) flush();
  }
  if (!ok) atomicOr(p.status, (int)ST_TIMEOUT);
  // the MMAs of the last issued tile have completed before TMEM is released
  if (warp == 1 && lane == 0 && issued > 0) umma::mbar_wait(tfull, (issued - 1) & 1, 200000000ull);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  if (warp == 1) umma::tmem_dealloc(tmem, 256);
}

// ------------------------------------------------------------------------------ host side
constexpr int kFwdNE = 64, kBwdNE = 32;

static size_t fwd_smem() {
  size_t s = 1024 + kWfBytes + 2 * kFwdNE * 128 + 4 * kFwdNE * 4 + 2 * kFwdNE * 16 + 128;
  return s < 80 * 1024 ? 80 * 1024 : s;   // at most two CTAs per SM: 2 x 256 TMEM columns
}
static size_t bwd_smem() {
  size_t s = 1024 + kWfBytes + 4 * kBwdNE * 128 + 4 * kBwdNE * 4 + 2 * kBwdNE * 16 + 2 * kBwdNE * 8 +
             kBwdNE * 16 * 4 + 256;
  return s < 80 * 1024 ? 80 * 1024 : s;
}

bool edge_tc_supported(int F, int K) { return F == kF && K <= kKPad && K >= 2; }

static int grid_for(int64_t n, int64_t* rows_per_cta) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t ctas = 2LL * sms;
  int64_t rpc = (n + ctas - 1) / ctas;
  if (rpc < 1) rpc = 1;
  *rows_per_cta = rpc;
  return (int)((n + rpc - 1) / rpc);
}

int edge_fwd_tc(cudaStream_t st, const ModelW& m, int t, int64_t n, const int32_t* arow, const int32_t* acol,
                const float4* ar, const float* PHI, const float* S, const float* V, float* SM, float* VM,
                bf16* VMb, int* status) {
  if (n == 0) return 0;
  CUtensorMap tm;
  if (!make_tmap_bf16(&tm, m.L[t].Wfb, 3 * kF, 64, 64, 128)) return -2;
  EdgeTcArgs a{};
  a.n = n; a.K = m.K; a.rc = m.rc; a.arow = arow; a.acol = acol; a.ar = ar; a.PHI = PHI; a.S = S; a.V = V;
  a.bf = m.L[t].bf; a.SM = SM; a.VM = VM; a.VMb = VMb; a.status = status;
  const int grid = grid_for(n, &a.rows_per_cta);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_edge_fwd_tc<kFwdNE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem());
    attr = true;
  }
  LaunchScope ls_(st);
  k_edge_fwd_tc<kFwdNE><<<grid, 192, fwd_smem(), st>>>(tm, a);
  return 0;
}

int edge_bwd_tc(cudaStream_t st, const ModelW& m, int t, int accumulate, int64_t n, const int32_t* arow,
                const int32_t* acol, const float4* ar, const float* PHI, const float* Gsm, const float* Gvm,
                float* GPHI, float4* hedge, int* status) {
  if (n == 0) return 0;
  CUtensorMap tm;
  if (!make_tmap_bf16(&tm, m.L[t].Wfb, 3 * kF, 64, 64, 128)) return -2;
  EdgeTcArgs a{};
  a.n = n; a.K = m.K; a.rc = m.rc; a.accumulate = accumulate; a.arow = arow; a.acol = acol; a.ar = ar;
  a.PHI = PHI; a.Gsm = Gsm; a.Gvm = Gvm; a.bf = m.L[t].bf; a.GPHI = GPHI; a.hedge = hedge; a.status = status;
  const int grid = grid_for(n, &a.rows_per_cta);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_edge_bwd_tc<kBwdNE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem());
    attr = true;
  }
  LaunchScope ls_(st);
  k_edge_bwd_tc<kBwdNE><<<grid, 192, bwd_smem(), st>>>(tm, a);
  return 0;
}

}  // namespace ctd
