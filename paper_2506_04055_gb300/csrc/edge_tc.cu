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

// Row r of a hi and a lo tile: hi = bf16(v), lo = bf16(v - hi).  The MMA adds Wf . hi and
// Wf . lo in FP32, so the basis enters with about 16 significant bits instead of 8 (the
// tensor pipe has ample headroom for the second product).
__device__ __forceinline__ void store_basis_row_split(unsigned char* hi, unsigned char* lo, int r,
                                                      const float (&v)[kKPad]) {
  float h[kKPad], l[kKPad];
#pragma unroll
  for (int k = 0; k < kKPad; ++k) {
    h[k] = __bfloat162float(__float2bfloat16_rn(v[k]));
    l[k] = v[k] - h[k];
  }
  store_basis_row(hi, r, h);
  store_basis_row(lo, r, l);
}

// Columns 16h .. 16h+15 of row r of a 128B-swizzled BF16 tile (two 16-byte chunks).
__device__ __forceinline__ void store_basis_half(unsigned char* tile, int r, int h, const float (&v)[16]) {
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    uint32_t w[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      __nv_bfloat162 b2 = __floats2bfloat162_rn(v[8 * c + 2 * x], v[8 * c + 2 * x + 1]);
      w[x] = *reinterpret_cast<uint32_t*>(&b2);
    }
    *reinterpret_cast<uint4*>(tile + umma::sw128_offset(r, 16 * h + 8 * c)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}
__device__ __forceinline__ void store_basis_half_split(unsigned char* hi, unsigned char* lo, int r, int h,
                                                       const float (&v)[16]) {
  float a[16], b[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    a[k] = __bfloat162float(__float2bfloat16_rn(v[k]));
    b[k] = v[k] - a[k];
  }
  store_basis_half(hi, r, h, a);
  store_basis_half(lo, r, h, b);
}

struct EdgeTcArgs {
  int64_t n;
  int64_t rows_per_cta;
  int64_t chunk_rows;              // block-cyclic kernels: rows per chunk
  int K;
  float rc;
  int accumulate;
  const int32_t* __restrict__ arow;
  const int32_t* __restrict__ acol;
  const int32_t* __restrict__ aend;  // rows completed at each edge (1 + following empty rows; 0 inside a row)
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
  const float* __restrict__ G4;    // [n][F][4] = (gsm, gvm_0..2) per feature (adjoint, interleaved)
  int* status;
};

}  // namespace

// ------------------------------------------------------------------------------ message
// Row bookkeeping shared by both kernels: the producer marks, for each edge slot of a tile,
// how many rows end at that edge (the row itself plus any empty rows right after it); rows
// without edges at the start of a stream's range are flushed before its first tile.
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

// Same flags as mark_row_ends, with the warp reading 32 row ends per step: row ends are
// non-decreasing, so the ends inside the tile are a prefix of the lanes.
__device__ __forceinline__ void mark_row_ends_warp(int lane, int* sfl, int NE, int64_t tb, int64_t r1,
                                                   const int32_t* __restrict__ arow, int64_t& rp) {
  for (int s = lane; s < NE; s += 32) sfl[s] = 0;
  __syncwarp();
  for (;;) {
    const int64_t row = rp + lane;
    const int64_t v = row < r1 ? (int64_t)arow[row + 1] : INT64_MAX;
    const bool in = v <= tb + NE;
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if (in) atomicAdd(&sfl[v - 1 - tb], 1);
    const int cnt = __popc(m);
    rp += cnt;
    if (cnt < 32) break;
  }
  __syncwarp();
}

// Streams: a CTA splits its rows into NS contiguous sub-ranges ("streams"), each with its own
// tiles, TMEM region and barriers and its own epilogue warpgroup, so one SM keeps 4 * NS
// epilogue warps busy on independent rows while sharing one copy of Wf.
struct StreamRange {
  int64_t r0, r1, e0, e1;
  int ntiles;
};
template <int NE, int NS>
__device__ __forceinline__ StreamRange stream_range(const EdgeTcArgs& p, int s) {
  StreamRange R;
  const int64_t c0 = (int64_t)blockIdx.x * p.rows_per_cta;
  const int64_t c1 = (c0 + p.rows_per_cta < p.n) ? c0 + p.rows_per_cta : p.n;
  const int64_t q = (c1 - c0 + NS - 1) / NS;
  R.r0 = c0 + s * q < c1 ? c0 + s * q : c1;
  R.r1 = R.r0 + q < c1 ? R.r0 + q : c1;
  R.e0 = p.arow[R.r0];
  R.e1 = p.arow[R.r1];
  R.ntiles = (int)((R.e1 - R.e0 + NE - 1) / NE);
  return R;
}

// Block-cyclic work for the bulk-gathered kernels: the sorted rows are cut into chunks of
// p.chunk_rows rows, and chunk k goes to stream k mod (gridDim.x * NS), the stream id being
// blockIdx.x * NS + s.  All streams of the GPU then sweep the (cell-ordered) atoms together,
// so the neighbour rows they gather at any moment stay within a window that fits in L2.
struct Chunk {
  int64_t r0, r1, e0, e1;
  int ntiles;
};
template <int NE>
__device__ __forceinline__ bool chunk_at(const EdgeTcArgs& p, int64_t k, Chunk& c) {
  const int64_t r0 = k * p.chunk_rows;
  if (r0 >= p.n) return false;
  c.r0 = r0;
  c.r1 = r0 + p.chunk_rows < p.n ? r0 + p.chunk_rows : p.n;
  c.e0 = p.arow[c.r0];
  c.e1 = p.arow[c.r1];
  c.ntiles = (int)((c.e1 - c.e0 + NE - 1) / NE);
  return true;
}

// Folded radial basis (k < K): b_k = f_c rbf_k, b_K = f_c, so that the filter's bias sits in
// column K of the BF16 filter matrix and the MMA yields W = f_c (Wf rbf + bf) itself; with
// DERIV also the distance derivative db_k = f_c rbf'_k + f_c' rbf_k, db_K = f_c'.
template <bool DERIV>
__device__ __forceinline__ void folded_basis(float d, int K, float sig, float inv2s2, float inv_s2, float inv_rc,
                                             float (&b)[kKPad], float (&db)[kKPad]) {
  const float fc = 0.5f * (cospif(d * inv_rc) + 1.0f);
  const float dfc = -0.5f * 3.14159265358979f * inv_rc * sinpif(d * inv_rc);
#pragma unroll
  for (int k = 0; k < kKPad; ++k) {
    const float t = d - (float)k * sig;
    const float v = k < K ? expf(-t * t * inv2s2) : 0.0f;
    b[k] = k < K ? fc * v : (k == K ? fc : 0.0f);
    if (DERIV) db[k] = k < K ? fc * (-v * t * inv_s2) + dfc * v : (k == K ? dfc : 0.0f);
  }
}

// warps 0..1 producers, warp 2 MMA / TMEM owner, warps 3 .. 3 + 4 NS - 1 epilogue
template <int NE, int NS, bool SPLIT, int TB, bool AEND = false, bool CHUNKED = false, bool V0 = false, int KC = 0>
__global__ void __launch_bounds__(32 * (3 + 4 * NS), 1) k_edge_fwd_tc(const __grid_constant__ CUtensorMap tmWf, EdgeTcArgs p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = align1024(smem_raw);
  unsigned char* sA = smem;                                        // Wf tiles
  constexpr int NB = SPLIT ? 2 : 1;                                // basis tiles per buffer (hi[, lo])
  static_assert(NS * TB * 3 * NE <= 512, "TMEM columns");
  unsigned char* sB = sA + kWfBytes;                               // [NS][2][NB][NE x 128 B] basis
  int* sj = reinterpret_cast<int*>(sB + NS * 2 * NB * NE * 128);   // [NS][2][NE] sender index
  int* sfl = sj + NS * 2 * NE;                                     // [NS][2][NE] rows ending at the slot
  float4* sgeo = reinterpret_cast<float4*>(sfl + NS * 2 * NE);     // [NS][2][NE] (u, f_c)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sgeo + NS * 2 * NE);
  uint64_t* wbar = bars;                 // Wf loaded
  uint64_t* sbar = bars + 1;             // per stream: bready[2], bfree[2], tfull[2], tempty[2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 1 + 8 * NS);

  if (!CHUNKED && (int64_t)blockIdx.x * p.rows_per_cta >= p.n) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nstreams = (int64_t)gridDim.x * NS;

  if (threadIdx.x == 0) {
    umma::mbar_init(wbar, 1);
    for (int s = 0; s < NS; ++s) {
      uint64_t* b = sbar + 8 * s;
      umma::mbar_init(&b[0], 1);
      umma::mbar_init(&b[1], 1);
      umma::mbar_init(&b[2], 4);
      umma::mbar_init(&b[3], 4);
      umma::mbar_init(&b[4], 1);
      umma::mbar_init(&b[5], 1);
      umma::mbar_init(&b[6], 4);
      umma::mbar_init(&b[7], 4);
    }
    umma::mbar_fence_init();
  }
  if (warp == 2) umma::tmem_alloc(tmem_slot, 512);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  int issued[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) issued[s] = 0;

  if (warp < 2) {
    if (warp == 0 && lane == 0) {
      umma::mbar_expect_tx(wbar, kWfBytes);
      for (int m = 0; m < 3; ++m) umma::tma_load_2d(sA + m * kWfTileBytes, &tmWf, 0, m * 128, wbar);
    }
    const float sig = p.rc / (float)(p.K - 1), inv2s2 = 1.0f / (2.0f * sig * sig), inv_rc = 1.0f / p.rc;
    // producer warp w serves streams w, w + 2, ...; tiles are produced round-robin.  Each stream
    // walks either one contiguous row range or (CHUNKED) its block-cyclic row chunks.
    constexpr int NO = (NS + 1) / 2;
    int64_t ck[NO], rp[NO];
    Chunk C[NO];
    bool have[NO];
    int t[NO], it[NO];
    auto first = [&](int o, int s) -> bool {
      if (CHUNKED) {
        ck[o] = (int64_t)blockIdx.x * NS + s;
        return chunk_at<NE>(p, ck[o], C[o]);
      }
      const StreamRange R = stream_range<NE, NS>(p, s);
      C[o].r0 = R.r0; C[o].r1 = R.r1; C[o].e0 = R.e0; C[o].e1 = R.e1; C[o].ntiles = R.ntiles;
      return true;
    };
    auto enter = [&](int o) {   // at a range's first tile: skip its leading empty rows
      rp[o] = C[o].r0;
      if (!AEND)
        while (rp[o] < C[o].r1 && p.arow[rp[o] + 1] == C[o].e0) ++rp[o];
    };
    auto norm = [&](int o) {
      while (have[o] && t[o] >= C[o].ntiles) {
        t[o] = 0;
        if (CHUNKED) {
          ck[o] += nstreams;
          have[o] = chunk_at<NE>(p, ck[o], C[o]);
        } else {
          have[o] = false;
        }
        if (have[o]) enter(o);
      }
    };
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const int s = warp + 2 * o;
      have[o] = s < NS && first(o, s);
      t[o] = 0;
      it[o] = 0;
      if (have[o]) enter(o);
    }
    bool any = true;
    while (ok && any) {
      any = false;
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        const int s = warp + 2 * o;
        if (s >= NS) continue;
        norm(o);
        if (!have[o]) continue;
        any = true;
        uint64_t* b = sbar + 8 * s;
        const int bb = it[o] & 1;
        if (it[o] >= 2 && !umma::mbar_wait(&b[2 + bb], ((it[o] >> 1) - 1) & 1)) { ok = false; break; }
        unsigned char* tile = sB + (s * 2 + bb) * NB * NE * 128;
        const int64_t tb = C[o].e0 + (int64_t)t[o] * NE;
        const int so = (s * 2 + bb) * NE;
        for (int k0 = lane; k0 < NE; k0 += 32) {
          const int64_t e = tb + k0;
          float rb[kKPad];
          int j = 0, ecnt = 0;
          float4 geo = make_float4(0.f, 0.f, 0.f, 0.f);
          if (e < C[o].e1) {
            const float4 r = p.ar[e];
            if (AEND) ecnt = p.aend[e];
            const float d = r.w, id = 1.0f / d;
            geo = make_float4(r.x * id, r.y * id, r.z * id, 0.5f * (cospif(d * inv_rc) + 1.0f));
            j = p.acol[e];
#pragma unroll
            for (int kk = 0; kk < kKPad; ++kk) {
              const float tq = d - (float)kk * sig;
              rb[kk] = kk < (KC > 0 ? KC : p.K) ? expf(-tq * tq * inv2s2) : 0.0f;
            }
          } else {
#pragma unroll
            for (int kk = 0; kk < kKPad; ++kk) rb[kk] = 0.0f;
          }
          if (SPLIT)
            store_basis_row_split(tile, tile + NE * 128, k0, rb);
          else
            store_basis_row(tile, k0, rb);
          sj[so + k0] = j;
          sgeo[so + k0] = geo;
          if (AEND) sfl[so + k0] = ecnt;
        }
        if (!AEND) mark_row_ends(lane, sfl + so, NE, tb, C[o].r1, p.arow, rp[o]);
        umma::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&b[bb]);
        ++t[o];
        ++it[o];
      }
    }
  } else if (warp == 2) {
    if (lane == 0) {
      if (!umma::mbar_wait(wbar, 0)) ok = false;
      const uint32_t idesc = umma::idesc_bf16_m128(NE);
      int64_t kc[NS];
      int t[NS], it[NS];
      bool have[NS];
      Chunk C[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        t[s] = 0;
        it[s] = 0;
        if (CHUNKED) {
          kc[s] = (int64_t)blockIdx.x * NS + s;
          have[s] = chunk_at<NE>(p, kc[s], C[s]);
        } else {
          const StreamRange R = stream_range<NE, NS>(p, s);
          C[s].r0 = R.r0; C[s].r1 = R.r1; C[s].e0 = R.e0; C[s].e1 = R.e1; C[s].ntiles = R.ntiles;
          have[s] = true;
        }
      }
      // one tile per stream in turn, blocking on each stream's barriers
      bool any = true;
      while (ok && any) {
        any = false;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          while (have[s] && t[s] >= C[s].ntiles) {
            t[s] = 0;
            if (CHUNKED) {
              kc[s] += nstreams;
              have[s] = chunk_at<NE>(p, kc[s], C[s]);
            } else {
              have[s] = false;
            }
          }
          if (!have[s]) continue;
          any = true;
          uint64_t* b = sbar + 8 * s;
          const int bb = it[s] & 1;
          if (!umma::mbar_wait(&b[bb], (it[s] >> 1) & 1)) { ok = false; break; }
          // TMEM buffer a was last read by the epilogue for tile it - TB
          const int a = it[s] % TB;
          if (it[s] >= TB && !umma::mbar_wait(&b[6 + a], ((it[s] / TB) - 1) & 1)) { ok = false; break; }
          umma::fence_after();
          const uint32_t bbase = umma::smem_u32(sB + (s * 2 + bb) * NB * NE * 128);
#pragma unroll
          for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int kk = 0; kk < 2 * NB; ++kk)   // k-halves of the hi tile[, then of the lo tile]
              umma::mma_bf16(tmem + (uint32_t)((s * TB + a) * 3 * NE + m * NE),
                             umma::desc_sw128(umma::smem_u32(sA + m * kWfTileBytes) + 32u * (kk & 1)),
                             umma::desc_sw128(bbase + (uint32_t)(kk >> 1) * NE * 128 + 32u * (kk & 1)), idesc, kk > 0);
          umma::mma_commit(&b[4 + a]);
          issued[s] = ++it[s];
          ++t[s];
        }
      }
    }
  } else {
    const int s = (warp - 3) >> 2;         // stream of this epilogue warpgroup
    const int q = warp & 3, f = q * 32 + lane;
    uint64_t* b = sbar + 8 * s;
    const float bs = p.bf[f], bvv = p.bf[kF + f], bvs = p.bf[2 * kF + f];
    int it = 0;
    Chunk C;
    int64_t kc = (int64_t)blockIdx.x * NS + s;
    bool have;
    if (CHUNKED) {
      have = chunk_at<NE>(p, kc, C);
    } else {
      const StreamRange R = stream_range<NE, NS>(p, s);
      C.r0 = R.r0; C.r1 = R.r1; C.e0 = R.e0; C.e1 = R.e1; C.ntiles = R.ntiles;
      have = true;
    }
    for (; ok && have; kc += nstreams, have = CHUNKED && chunk_at<NE>(p, kc, C)) {
    int64_t r = C.r0;
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
    while (r < C.r1 && p.arow[r + 1] == C.e0) flush();
    for (int t = 0; t < C.ntiles; ++t, ++it) {
      const int bb = it & 1, a = it % TB;
      if (!umma::mbar_wait(&b[4 + a], (it / TB) & 1)) { ok = false; break; }
      umma::fence_after();
      const int64_t tb = C.e0 + (int64_t)t * NE;
      const int nlive = (int)((C.e1 - tb) < NE ? (C.e1 - tb) : NE);
      const int so = (s * 2 + bb) * NE;
      const int* tj = sj + so;
      const int* tf = sfl + so;
      const float4* tg = sgeo + so;
#pragma unroll 1
      for (int c = 0; c < NE / 8; ++c) {
        // the senders' message rows first (they do not depend on the accumulator), so their
        // latency overlaps the TMEM loads below
        // V0 (first layer, v = 0): the psi channels v_a phi_vv are zero and not gathered
        float g[8][5];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const bool live = c * 8 + u < nlive;
          const float* pj = p.PHI + (int64_t)(live ? tj[c * 8 + u] : 0) * 6 * kF + f;
#pragma unroll
          for (int k = 0; k < 5; ++k) g[u][k] = live && (!V0 || k == 0 || k == 4) ? __ldg(pj + k * kF) : 0.f;
        }
        float ds[8], dv[8], dw[8];
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((s * TB + a) * 3 * NE + c * 8);
        umma::tmem_ld8x3(ta, NE, ds, dv, dw);
        if (c == NE / 8 - 1) {
          umma::fence_before();
          __syncwarp();
          if (lane == 0) umma::mbar_arrive(&b[6 + a]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int slot = c * 8 + u;
          if (slot < nlive) {
            const float4 geo = tg[slot];
            const float fc = geo.w;
            const float ws = (ds[u] + bs) * fc, wvv = (dv[u] + bvv) * fc, wvs = (dw[u] + bvs) * fc;
            as = fmaf(g[u][0], ws, as);
            const float tvs = g[u][4] * wvs;
            if (V0) {
              a0 = fmaf(geo.x, tvs, a0);
              a1 = fmaf(geo.y, tvs, a1);
              a2 = fmaf(geo.z, tvs, a2);
            } else {
              a0 = fmaf(g[u][1], wvv, fmaf(geo.x, tvs, a0));
              a1 = fmaf(g[u][2], wvv, fmaf(geo.y, tvs, a1));
              a2 = fmaf(g[u][3], wvv, fmaf(geo.z, tvs, a2));
            }
            for (int nf = tf[slot]; nf > 0 && r < C.r1; --nf) flush();
          }
        }
      }
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&b[2 + bb]);
    }
    if (!ok) break;
    while (r < C.r1) flush();
    }
  }
  if (!ok) atomicOr(p.status, (int)ST_TIMEOUT);
  // the MMAs of every stream's last issued tile have completed before TMEM is released
  if (warp == 2 && lane == 0)
    for (int s = 0; s < NS; ++s)
      if (issued[s] > 0)
        umma::mbar_wait(&sbar[8 * s + 4 + ((issued[s] - 1) % TB)], ((issued[s] - 1) / TB) & 1, 200000000ull);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  if (warp == 2) umma::tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------------------------ adjoint
// Sender-side: row j walks edges e' = (j <- i); the reverse edge (i <- j) carried phi_j, v_j
// into receiver i with direction -u_e'.  Per tile the MMA gives both the filter W~ (basis)
// and its radial derivative W~' (derivative basis).  Per edge the channel partials of dU/dd
// and dU/du_rev are reduced over the four warps of the stream's epilogue warpgroup and turned
// into hedge[e'].
template <int NE, int NS>
__global__ void __launch_bounds__(32 * (3 + 4 * NS), 1) k_edge_bwd_tc(const __grid_constant__ CUtensorMap tmWf, EdgeTcArgs p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = align1024(smem_raw);
  unsigned char* sA = smem;                                          // Wf tiles
  unsigned char* sB = sA + kWfBytes;                                 // [NS][2][2][NE x 128 B]
  int* sj = reinterpret_cast<int*>(sB + NS * 4 * NE * 128);          // [NS][2][NE]
  int* sfl = sj + NS * 2 * NE;                                       // [NS][2][NE]
  float4* sgeo = reinterpret_cast<float4*>(sfl + NS * 2 * NE);       // [NS][2][NE] (u, d)
  float2* sfc = reinterpret_cast<float2*>(sgeo + NS * 2 * NE);       // [NS][2][NE] (f_c, f_c')
  float* red = reinterpret_cast<float*>(sfc + NS * 2 * NE);          // [NS][NE][4 warps][4]
  uint64_t* bars = reinterpret_cast<uint64_t*>(red + NS * NE * 16);
  uint64_t* wbar = bars;
  uint64_t* sbar = bars + 1;    // per stream: bready[2], bfree[2], tfull, tempty, esync[2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 1 + 8 * NS);

  if ((int64_t)blockIdx.x * p.rows_per_cta >= p.n) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    umma::mbar_init(wbar, 1);
    for (int s = 0; s < NS; ++s) {
      uint64_t* b = sbar + 8 * s;
      umma::mbar_init(&b[0], 1);
      umma::mbar_init(&b[1], 1);
      umma::mbar_init(&b[2], 4);
      umma::mbar_init(&b[3], 4);
      umma::mbar_init(&b[4], 1);
      umma::mbar_init(&b[5], 4);
      umma::mbar_init(&b[6], 4);
      umma::mbar_init(&b[7], 4);
    }
    umma::mbar_fence_init();
  }
  if (warp == 2) umma::tmem_alloc(tmem_slot, 512);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  int issued[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) issued[s] = 0;

  if (warp < 2) {
    if (warp == 0 && lane == 0) {
      umma::mbar_expect_tx(wbar, kWfBytes);
      for (int m = 0; m < 3; ++m) umma::tma_load_2d(sA + m * kWfTileBytes, &tmWf, 0, m * 128, wbar);
    }
    const float sig = p.rc / (float)(p.K - 1), inv2s2 = 1.0f / (2.0f * sig * sig), inv_s2 = 1.0f / (sig * sig);
    const float inv_rc = 1.0f / p.rc;
    StreamRange R[NS];
    int64_t rp[NS];
    int maxt = 0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      R[s] = stream_range<NE, NS>(p, s);
      rp[s] = R[s].r0;
      while (rp[s] < R[s].r1 && p.arow[rp[s] + 1] == R[s].e0) ++rp[s];
      maxt = R[s].ntiles > maxt ? R[s].ntiles : maxt;
    }
    for (int it = 0; ok && it < maxt; ++it) {
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if ((s & 1) != warp || it >= R[s].ntiles) continue;
        uint64_t* b = sbar + 8 * s;
        const int bb = it & 1;
        if (it >= 2 && !umma::mbar_wait(&b[2 + bb], ((it >> 1) - 1) & 1)) { ok = false; break; }
        unsigned char* tile = sB + ((s * 2 + bb) * 2) * NE * 128;
        unsigned char* dtile = tile + NE * 128;
        const int64_t tb = R[s].e0 + (int64_t)it * NE;
        const int so = (s * 2 + bb) * NE;
        for (int k0 = lane; k0 < NE; k0 += 32) {
          const int64_t e = tb + k0;
          float rb[kKPad], drb[kKPad];
          int i = 0;
          float4 geo = make_float4(0.f, 0.f, 0.f, 1.f);
          float2 fcv = make_float2(0.f, 0.f);
          if (e < R[s].e1) {
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
          store_basis_row(tile, k0, rb);
          store_basis_row(dtile, k0, drb);
          sj[so + k0] = i;
          sgeo[so + k0] = geo;
          sfc[so + k0] = fcv;
        }
        mark_row_ends(lane, sfl + so, NE, tb, R[s].r1, p.arow, rp[s]);
        umma::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&b[bb]);
      }
    }
  } else if (warp == 2) {
    if (lane == 0) {
      if (!umma::mbar_wait(wbar, 0)) ok = false;
      const uint32_t idesc = umma::idesc_bf16_m128(NE);
      int nt[NS], maxt = 0;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        nt[s] = stream_range<NE, NS>(p, s).ntiles;
        maxt = nt[s] > maxt ? nt[s] : maxt;
      }
      for (int it = 0; ok && it < maxt; ++it) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          if (it >= nt[s]) continue;
          uint64_t* b = sbar + 8 * s;
          const int bb = it & 1;
          if (!umma::mbar_wait(&b[bb], (it >> 1) & 1)) { ok = false; break; }
          if (it >= 1 && !umma::mbar_wait(&b[5], (it - 1) & 1)) { ok = false; break; }
          umma::fence_after();
#pragma unroll
          for (int h = 0; h < 2; ++h) {          // h = 0: basis -> W~, h = 1: derivative -> W~'
            const uint32_t bbase = umma::smem_u32(sB + ((s * 2 + bb) * 2 + h) * NE * 128);
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
              for (int k = 0; k < 2; ++k)
                umma::mma_bf16(tmem + (uint32_t)(s * 6 * NE + (3 * h + m) * NE),
                               umma::desc_sw128(umma::smem_u32(sA + m * kWfTileBytes) + 32u * k),
                               umma::desc_sw128(bbase + 32u * k), idesc, k > 0);
          }
          umma::mma_commit(&b[4]);
          ++issued[s];
        }
      }
    }
  } else {
    const int s = (warp - 3) >> 2;
    const int q = warp & 3, f = q * 32 + lane;
    const StreamRange R = stream_range<NE, NS>(p, s);
    uint64_t* b = sbar + 8 * s;
    float* sred = red + s * NE * 16;
    const float bs = p.bf[f], bvv = p.bf[kF + f], bvs = p.bf[2 * kF + f];
    int64_t r = R.r0;
    float cur[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, nxt[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    auto fetch = [&](int64_t row, float (&o)[5]) {
      if (row < R.r1) {
        const float* pj = p.PHI + row * 6 * kF + f;
#pragma unroll
        for (int k = 0; k < 5; ++k) o[k] = __ldg(pj + k * kF);
      }
    };
    float gps = 0.f, gy0 = 0.f, gy1 = 0.f, gy2 = 0.f, gpvs = 0.f;
    auto flush = [&]() {
      if (p.GPHI) {
        float* o = p.GPHI + r * 5 * kF;
        o[f] = gps; o[kF + f] = gy0; o[2 * kF + f] = gy1; o[3 * kF + f] = gy2; o[4 * kF + f] = gpvs;
      }
      gps = gy0 = gy1 = gy2 = gpvs = 0.f;
      ++r;
#pragma unroll
      for (int k = 0; k < 5; ++k) cur[k] = nxt[k];
      fetch(r + 1, nxt);
    };
    fetch(r, cur);
    fetch(r + 1, nxt);
    while (r < R.r1 && p.arow[r + 1] == R.e0) flush();
    for (int it = 0; it < R.ntiles; ++it) {
      const int bb = it & 1;
      if (!umma::mbar_wait(&b[4], it & 1)) { ok = false; break; }
      umma::fence_after();
      const int64_t tb = R.e0 + (int64_t)it * NE;
      const int nlive = (int)((R.e1 - tb) < NE ? (R.e1 - tb) : NE);
      const int so = (s * 2 + bb) * NE;
      const int* ti = sj + so;
      const int* tf = sfl + so;
      const float4* tg = sgeo + so;
      const float2* tc = sfc + so;
#pragma unroll 1
      for (int c = 0; c < NE / 8; ++c) {
        float W[6][8];
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(s * 6 * NE + c * 8);
#pragma unroll
        for (int h = 0; h < 6; ++h) umma::tmem_ld8(ta + h * NE, W[h]);
        if (c == NE / 8 - 1) {
          umma::fence_before();
          __syncwarp();
          if (lane == 0) umma::mbar_arrive(&b[5]);
        }
        float G[8][4];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const bool live = c * 8 + u < nlive;
          const int64_t i = live ? ti[c * 8 + u] : 0;
          G[u][0] = live ? __ldg(p.Gsm + i * kF + f) : 0.f;
          G[u][1] = live ? __ldg(p.Gvm + i * 3 * kF + f) : 0.f;
          G[u][2] = live ? __ldg(p.Gvm + i * 3 * kF + kF + f) : 0.f;
          G[u][3] = live ? __ldg(p.Gvm + i * 3 * kF + 2 * kF + f) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int slot = c * 8 + u;
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
          if ((lane & 7) == 0) sred[(slot * 4 + q) * 4 + (lane >> 3)] = kk;
          if (live)
            for (int nf = tf[slot]; nf > 0; --nf) flush();
        }
      }
      // the four warps of this stream have written their partials for the tile
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&b[6]);
      if (!umma::mbar_wait(&b[6], it & 1)) { ok = false; break; }
      const int t = f;
      if (t < nlive) {
        float pd = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const float* rr = sred + (t * 4 + w) * 4;
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
      if (lane == 0) umma::mbar_arrive(&b[7]);
      if (!umma::mbar_wait(&b[7], it & 1)) { ok = false; break; }
      if (lane == 0) umma::mbar_arrive(&b[2 + bb]);
    }
    if (ok)
      while (r < R.r1) flush();
  }
  if (!ok) atomicOr(p.status, (int)ST_TIMEOUT);
  if (warp == 2 && lane == 0)
    for (int s = 0; s < NS; ++s)
      if (issued[s] > 0) umma::mbar_wait(&sbar[8 * s + 4], (issued[s] - 1) & 1, 200000000ull);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  if (warp == 2) umma::tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------------------------ bulk-gathered kernels
// Both kernels below: warps 0..NS-1 produce (one per stream: folded basis tiles, geometry,
// row-end flags, and cp.async.bulk copies of the gathered neighbour rows into shared memory,
// completing on the tile's mbarrier); warp 2 owns TMEM and issues the MMAs; 4 epilogue warps
// per stream, thread f of the stream handling feature f.  Tiles of NE edges, two buffers per
// stream, chunks of rows handed out block-cyclically (chunk_at).

// Message: W = f_c (Wf rbf + bf) for the tile's edges straight from the MMA (folded basis);
// per edge, thread f reads [phi_s | v_0 phi_vv | v_1 phi_vv | v_2 phi_vv | phi_vs] of the
// sender (gathered rows of PHI) and accumulates the receiver's messages over its row.
template <int NE, int NS>
__global__ void __launch_bounds__(32 * (3 + 4 * NS), 1) k_edge_fwd_tcg(const __grid_constant__ CUtensorMap tmWf, EdgeTcArgs p) {
  static_assert(NS <= 2, "one producer warp per stream");
  constexpr int kRow = 5 * kF;   // gathered floats per edge
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = align1024(smem_raw);
  unsigned char* sA = smem;                                          // Wf tiles (bias in column K)
  unsigned char* sB = sA + kWfBytes;                                 // [NS][2][hi, lo][NE x 128 B]
  float* sG = reinterpret_cast<float*>(sB + NS * 4 * NE * 128);      // [NS][2][NE][5F]
  int* sfl = reinterpret_cast<int*>(sG + (size_t)NS * 2 * NE * kRow);   // [NS][2][NE]
  float4* sgeo = reinterpret_cast<float4*>(sfl + NS * 2 * NE);       // [NS][2][NE] (u, d)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sgeo + NS * 2 * NE);
  uint64_t* wbar = bars;
  uint64_t* sbar = bars + 1;    // per stream: bready[2], bfree[2], tfull[2], tempty[2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 1 + 8 * NS);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nstreams = (int64_t)gridDim.x * NS;

  if (threadIdx.x == 0) {
    umma::mbar_init(wbar, 1);
    for (int s = 0; s < NS; ++s) {
      uint64_t* b = sbar + 8 * s;
      umma::mbar_init(&b[0], 1);
      umma::mbar_init(&b[1], 1);
      umma::mbar_init(&b[2], 4);
      umma::mbar_init(&b[3], 4);
      umma::mbar_init(&b[4], 1);
      umma::mbar_init(&b[5], 1);
      umma::mbar_init(&b[6], 4);
      umma::mbar_init(&b[7], 4);
    }
    umma::mbar_fence_init();
  }
  if (warp == 2) umma::tmem_alloc(tmem_slot, 256);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  int issued[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) issued[s] = 0;
  int gathered = 0;

  if (warp < 2) {
    if (warp == 0 && lane == 0) {
      umma::mbar_expect_tx(wbar, kWfBytes);
      for (int m = 0; m < 3; ++m) umma::tma_load_2d(sA + m * kWfTileBytes, &tmWf, 0, m * 128, wbar);
    }
    if (warp < NS) {
      const int s = warp;
      const float sig = p.rc / (float)(p.K - 1), inv2s2 = 1.0f / (2.0f * sig * sig), inv_s2 = 1.0f / (sig * sig);
      const float inv_rc = 1.0f / p.rc;
      uint64_t* b = sbar + 8 * s;
      // this stream's tiles in order: chunk k, tile t; the next tile's edge data is loaded one
      // tile ahead so that its latency overlaps the current tile
      int64_t k = (int64_t)blockIdx.x * NS + s;
      Chunk C;
      bool have = chunk_at<NE>(p, k, C);
      int t = 0;
      auto normalize = [&]() {
        while (have && t >= C.ntiles) {
          k += nstreams;
          t = 0;
          have = chunk_at<NE>(p, k, C);
        }
      };
      float4 rn = make_float4(0.f, 0.f, 0.f, 1.f);
      int jn = 0, en = 0, nln = 0;
      int64_t tbn = 0;
      auto fetch = [&]() {
        tbn = C.e0 + (int64_t)t * NE;
        nln = (int)((C.e1 - tbn) < NE ? (C.e1 - tbn) : NE);
        if (lane < nln) {
          rn = p.ar[tbn + lane];
          jn = p.acol[tbn + lane];
          en = p.aend[tbn + lane];
        }
      };
      normalize();
      bool cur = have;
      if (cur) fetch();
      for (int it = 0; cur && ok; ++it) {
        const float4 r = rn;
        const int jj = jn, ecnt = en, nlive = nln;
        const int64_t tb = tbn;
        ++t;
        normalize();
        cur = have;
        if (cur) fetch();
        const int bb = it & 1;
        float bv[kKPad], dummy[kKPad];
        float4 geo = make_float4(0.f, 0.f, 0.f, 1.f);
        if (lane < nlive) {
          const float d = r.w, id = 1.0f / d;
          geo = make_float4(r.x * id, r.y * id, r.z * id, d);
          folded_basis<false>(d, p.K, sig, inv2s2, inv_s2, inv_rc, bv, dummy);
        } else {
#pragma unroll
          for (int q = 0; q < kKPad; ++q) bv[q] = 0.0f;
        }
        if (it >= 2 && !umma::mbar_wait(&b[2 + bb], ((it >> 1) - 1) & 1)) { ok = false; break; }
        const int so = (s * 2 + bb) * NE;
        if (lane == 0) umma::mbar_expect_tx_only(&b[bb], (uint32_t)(nlive * kRow * 4));
        __syncwarp();
        if (lane < NE) {
          if (lane < nlive)
            umma::bulk_copy_g2s(sG + (size_t)(so + lane) * kRow, p.PHI + (int64_t)jj * 6 * kF, kRow * 4, &b[bb]);
          store_basis_row_split(sB + (s * 2 + bb) * 2 * NE * 128, sB + ((s * 2 + bb) * 2 + 1) * NE * 128, lane, bv);
          sgeo[so + lane] = geo;
          sfl[so + lane] = lane < nlive ? ecnt : 0;
        }
        gathered = it + 1;
        umma::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&b[bb]);
      }
    }
  } else if (warp == 2) {
    if (lane == 0) {
      if (!umma::mbar_wait(wbar, 0)) ok = false;
      const uint32_t idesc = umma::idesc_bf16_m128(NE);
      int64_t k[NS];
      int t[NS], it[NS];
      bool have[NS];
      Chunk C[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        k[s] = (int64_t)blockIdx.x * NS + s;
        t[s] = 0;
        it[s] = 0;
        have[s] = chunk_at<NE>(p, k[s], C[s]);
      }
      // issue for whichever stream has its next tile ready (non-blocking probes), so that a
      // late tile of one stream does not hold back the other; a stall of more than 2 s without
      // progress gives up with a timeout
      bool any = true;
      uint32_t idle = 0;
      uint64_t t_idle = 0;
      while (ok && any) {
        any = false;
        bool progressed = false;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          while (have[s] && t[s] >= C[s].ntiles) {
            k[s] += nstreams;
            t[s] = 0;
            have[s] = chunk_at<NE>(p, k[s], C[s]);
          }
          if (!have[s]) continue;
          any = true;
          uint64_t* b = sbar + 8 * s;
          const int bb = it[s] & 1;
          if (!umma::mbar_test(&b[bb], (it[s] / 2) & 1)) continue;
          if (it[s] >= 2 && !umma::mbar_test(&b[6 + bb], ((it[s] >> 1) - 1) & 1)) continue;
          progressed = true;
          umma::fence_after();
          const uint32_t bbase = umma::smem_u32(sB + (s * 2 + bb) * 2 * NE * 128);
#pragma unroll
          for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)   // k-halves of the hi tile, then of the lo tile
              umma::mma_bf16(tmem + (uint32_t)((s * 2 + bb) * 3 * NE + m * NE),
                             umma::desc_sw128(umma::smem_u32(sA + m * kWfTileBytes) + 32u * (kk & 1)),
                             umma::desc_sw128(bbase + (uint32_t)(kk >> 1) * NE * 128 + 32u * (kk & 1)), idesc, kk > 0);
          umma::mma_commit(&b[4 + bb]);
          issued[s] = ++it[s];
          ++t[s];
        }
        if (any && !progressed) {
          __nanosleep(64);
          if (idle++ == 0) t_idle = umma::globaltimer();
          else if ((idle & 255) == 0 && umma::globaltimer() - t_idle > 2000000000ull) ok = false;
        } else {
          idle = 0;
        }
      }
    }
  } else {
    const int s = (warp - 3) >> 2;
    const int q = warp & 3, f = q * 32 + lane;
    uint64_t* b = sbar + 8 * s;
    int it = 0;
    Chunk C;
    for (int64_t k = (int64_t)blockIdx.x * NS + s; ok && chunk_at<NE>(p, k, C); k += nstreams) {
      int64_t r = C.r0;
      float as = 0.f, a0 = 0.f, a1 = 0.f, a2 = 0.f;
      // residual stream of the current row, loaded one row ahead
      float rs = 0.f, rv0 = 0.f, rv1 = 0.f, rv2 = 0.f;
      auto fetch = [&](int64_t row) {
        if (row < C.r1) {
          rs = __ldg(p.S + row * kF + f);
          const float* v = p.V + row * 3 * kF + f;
          rv0 = __ldg(v); rv1 = __ldg(v + kF); rv2 = __ldg(v + 2 * kF);
        }
      };
      auto flush = [&]() {
        const int64_t i = r;
        const float v0 = rv0 + a0, v1 = rv1 + a1, v2 = rv2 + a2;
        p.SM[i * kF + f] = rs + as;
        float* vm = p.VM + i * 3 * kF + f;
        vm[0] = v0; vm[kF] = v1; vm[2 * kF] = v2;
        if (p.VMb) {
          bf16* vb = p.VMb + i * 3 * kF + f;
          vb[0] = __float2bfloat16_rn(v0); vb[kF] = __float2bfloat16_rn(v1); vb[2 * kF] = __float2bfloat16_rn(v2);
        }
        as = a0 = a1 = a2 = 0.f;
        ++r;
        fetch(r);
      };
      fetch(r);
      while (r < C.r1 && p.arow[r + 1] == C.e0) flush();
      for (int t = 0; t < C.ntiles; ++t, ++it) {
        const int bb = it & 1;
        if (!umma::mbar_wait(&b[4 + bb], (it >> 1) & 1)) { ok = false; break; }
        if (!umma::mbar_wait(&b[bb], (it >> 1) & 1)) { ok = false; break; }   // gathered rows visible
        umma::fence_after();
        const int64_t tb = C.e0 + (int64_t)t * NE;
        const int nlive = (int)((C.e1 - tb) < NE ? (C.e1 - tb) : NE);
        const int so = (s * 2 + bb) * NE;
        const int* tf = sfl + so;
        const float4* tg = sgeo + so;
        const float* tG = sG + (size_t)so * kRow + f;
#pragma unroll 1
        for (int c = 0; c < NE / 8; ++c) {
          float W[3][8];
          const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((s * 2 + bb) * 3 * NE + c * 8);
          umma::tmem_ld8(ta, W[0]);
          umma::tmem_ld8(ta + NE, W[1]);
          umma::tmem_ld8(ta + 2 * NE, W[2]);
          if (c == NE / 8 - 1) {
            umma::fence_before();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&b[6 + bb]);
          }
          auto edge = [&](int u, int slot) {
            const float* gg = tG + (size_t)slot * kRow;
            const float4 geo = tg[slot];
            as = fmaf(gg[0], W[0][u], as);
            const float tvs = gg[4 * kF] * W[2][u];
            a0 = fmaf(gg[kF], W[1][u], fmaf(geo.x, tvs, a0));
            a1 = fmaf(gg[2 * kF], W[1][u], fmaf(geo.y, tvs, a1));
            a2 = fmaf(gg[3 * kF], W[1][u], fmaf(geo.z, tvs, a2));
          };
          const int4 fa = *reinterpret_cast<const int4*>(tf + c * 8), fb = *reinterpret_cast<const int4*>(tf + c * 8 + 4);
          if ((fa.x | fa.y | fa.z | fa.w | fb.x | fb.y | fb.z | fb.w) == 0 && c * 8 + 8 <= nlive) {
#pragma unroll
            for (int u = 0; u < 8; ++u) edge(u, c * 8 + u);
          } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int slot = c * 8 + u;
              if (slot < nlive) {
                edge(u, slot);
                for (int nf = tf[slot]; nf > 0 && r < C.r1; --nf) flush();
              }
            }
          }
        }
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&b[2 + bb]);
      }
      if (!ok) break;
      while (r < C.r1) flush();
    }
  }
  if (!ok) atomicOr(p.status, (int)ST_TIMEOUT);
  if (warp < NS && lane == 0) {
    // the bulk copies of the last two tiles this producer issued have landed before exit
    for (int t = gathered - 2; t < gathered; ++t)
      if (t >= 0) umma::mbar_wait(&sbar[8 * warp + (t & 1)], (t >> 1) & 1, 200000000ull);
  }
  if (warp == 2 && lane == 0)
    for (int s = 0; s < NS; ++s)
      if (issued[s] > 0)
        umma::mbar_wait(&sbar[8 * s + 4 + ((issued[s] - 1) & 1)], ((issued[s] - 1) >> 1) & 1, 200000000ull);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  if (warp == 2) umma::tmem_dealloc(tmem, 256);
}

// Adjoint: the MMA yields the filter and its distance derivative per edge (FOLD: with f_c and
// the bias folded into the basis, W and dW/dd themselves; otherwise Wf rbf and Wf rbf', the
// bias and f_c applied in FP32 by the epilogue); the receivers' gradient rows (gsm_i: F floats, gvm_i: 3F floats) are gathered by bulk copies.
// Thread f accumulates the row's phi gradients and overwrites its own feature of the gathered
// row with its partials of (dU/dd, dU/du); after a stream barrier the partials are reduced over
// the F features from shared memory and turned into hedge[e].
// PIPE: the epilogue reads the accumulator in 4-edge halves, each half's TMEM loads in flight
// while the previous half is computed (only a tile's first load is waited on at once)
template <int NE, int NS, bool FOLD, bool SPLIT, int NBUF = 2, int KC = 0, bool G4L = false, bool L0 = false,
          bool PIPE = false>
__global__ void __launch_bounds__(32 * (3 + 4 * NS), 1) k_edge_bwd_tcg(const __grid_constant__ CUtensorMap tmWf, EdgeTcArgs p) {
  static_assert(NS <= 2, "one producer warp per stream");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = align1024(smem_raw);
  unsigned char* sA = smem;                                          // Wf tiles (bias in column K)
  // per buffer one (or, SPLIT, a hi and a lo) operand of 2 NE rows: the basis of the tile's
  // edges in rows 0..NE-1 and their derivative basis in rows NE..2NE-1, so that one MMA per
  // channel block yields [W | dW/dd] as 2 NE columns
  constexpr int NB = SPLIT ? 2 : 1;
  static_assert(NS * 2 * 6 * NE <= 512, "TMEM columns");
  static_assert(NE == 16 && NBUF >= 2 && NBUF <= 4, "tile shape: one lane pair per edge");
  unsigned char* sB = sA + kWfBytes;                                 // [NS][NBUF][NB][2 NE x 128 B]
  float* sG = reinterpret_cast<float*>(sB + NS * NBUF * NB * 2 * NE * 128);   // [NS][NBUF][NE][4F]
  int* sfl = reinterpret_cast<int*>(sG + (size_t)NS * NBUF * NE * 4 * kF);   // [NS][NBUF][NE]
  float4* sgeo = reinterpret_cast<float4*>(sfl + NS * NBUF * NE);    // [NS][NBUF][NE] (u, d)
  float2* sfc = reinterpret_cast<float2*>(sgeo + NS * NBUF * NE);    // [NS][NBUF][NE] (f_c, f_c'), !FOLD
  uint64_t* bars = reinterpret_cast<uint64_t*>(sfc + NS * NBUF * NE);
  uint64_t* wbar = bars;
  // per stream: bready[4], bfree[4] (NBUF used), tfull[2], tempty[2], esync
  constexpr int kBars = 13;
  uint64_t* sbar = bars + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 1 + kBars * NS);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nstreams = (int64_t)gridDim.x * NS;

  if (threadIdx.x == 0) {
    umma::mbar_init(wbar, 1);
    for (int s = 0; s < NS; ++s) {
      uint64_t* b = sbar + kBars * s;
      for (int x = 0; x < 4; ++x) {
        umma::mbar_init(&b[x], 1);       // bready
        umma::mbar_init(&b[4 + x], 4);   // bfree
      }
      umma::mbar_init(&b[8], 1);         // tfull
      umma::mbar_init(&b[9], 1);
      umma::mbar_init(&b[10], 4);        // tempty
      umma::mbar_init(&b[11], 4);
      umma::mbar_init(&b[12], 4);        // esync
    }
    umma::mbar_fence_init();
  }
  if (warp == 2) umma::tmem_alloc(tmem_slot, 512);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  int issued[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) issued[s] = 0;
  int gathered = 0;

  if (warp < 2) {
    if (warp == 0 && lane == 0) {
      umma::mbar_expect_tx(wbar, kWfBytes);
      for (int m = 0; m < 3; ++m) umma::tma_load_2d(sA + m * kWfTileBytes, &tmWf, 0, m * 128, wbar);
    }
    if (warp < NS) {
      const int s = warp;
      const float sig = p.rc / (float)(p.K - 1), inv2s2 = 1.0f / (2.0f * sig * sig), inv_s2 = 1.0f / (sig * sig);
      const float inv_rc = 1.0f / p.rc;
      uint64_t* b = sbar + kBars * s;
      // this stream's tiles in order: chunk k, tile t; the next tile's edge data is loaded one
      // tile ahead so that its latency overlaps the current tile
      int64_t k = (int64_t)blockIdx.x * NS + s;
      Chunk C;
      bool have = chunk_at<NE>(p, k, C);
      int t = 0;
      auto normalize = [&]() {
        while (have && t >= C.ntiles) {
          k += nstreams;
          t = 0;
          have = chunk_at<NE>(p, k, C);
        }
      };
      // lane pair (slot, h): slot = lane & 15 handles edge `slot` of the tile; its halves
      // h = lane >> 4 compute basis entries k = 2q + h and swap the ones the other half stores,
      // so that each lane writes 16 contiguous columns and issues one bulk copy
      const int slot = lane & (NE - 1), h = lane >> 4;
      const int KK = KC > 0 ? KC : p.K;
      float4 rn = make_float4(0.f, 0.f, 0.f, 1.f);
      int jn = 0, en = 0, nln = 0;
      int64_t tbn = 0;
      auto fetch = [&]() {
        tbn = C.e0 + (int64_t)t * NE;
        nln = (int)((C.e1 - tbn) < NE ? (C.e1 - tbn) : NE);
        if (slot < nln) {
          rn = p.ar[tbn + slot];
          jn = p.acol[tbn + slot];
          en = p.aend[tbn + slot];
        }
      };
      normalize();
      bool cur = have;
      if (cur) fetch();
      for (int it = 0; cur && ok; ++it) {
        const float4 r = rn;
        const int jj = jn, ecnt = en, nlive = nln;
        const int64_t tb = tbn;
        ++t;
        normalize();
        cur = have;
        if (cur) fetch();
        const int bb = it % NBUF;
        float bq[16], dq[16];
        float4 geo = make_float4(0.f, 0.f, 0.f, 1.f);
        float2 fcv = make_float2(0.f, 0.f);
        const bool live = slot < nlive;
        if (live) {
          const float d = r.w, id = 1.0f / d;
          geo = make_float4(r.x * id, r.y * id, r.z * id, d);
          const float fc = 0.5f * (cospif(d * inv_rc) + 1.0f);
          const float dfc = -0.5f * 3.14159265358979f * inv_rc * sinpif(d * inv_rc);
          fcv = make_float2(fc, dfc);
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int kk = 2 * q + h;
            const float tq = d - (float)kk * sig;
            const bool in = kk < KK;
            const float v = in ? expf(-tq * tq * inv2s2) : 0.0f;
            const float dv = -v * tq * inv_s2;
            if (FOLD) {
              // f_c and the bias column K folded in (see folded_basis)
              bq[q] = in ? fc * v : (kk == KK ? fc : 0.0f);
              dq[q] = in ? fc * dv + dfc * v : (kk == KK ? dfc : 0.0f);
            } else {
              bq[q] = v;
              dq[q] = dv;
            }
          }
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q) bq[q] = dq[q] = 0.0f;
        }
        // this lane's columns 16h .. 16h+15: its own parity and the partner's
        float bs[16], ds[16];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float yb = __shfl_xor_sync(0xffffffffu, h == 0 ? bq[8 + i] : bq[i], 16);
          const float yd = __shfl_xor_sync(0xffffffffu, h == 0 ? dq[8 + i] : dq[i], 16);
          bs[2 * i] = h == 0 ? bq[i] : yb;
          bs[2 * i + 1] = h == 0 ? yb : bq[8 + i];
          ds[2 * i] = h == 0 ? dq[i] : yd;
          ds[2 * i + 1] = h == 0 ? yd : dq[8 + i];
        }
        if (it >= NBUF && !umma::mbar_wait(&b[4 + bb], ((it / NBUF) - 1) & 1)) { ok = false; break; }
        const int so = (s * NBUF + bb) * NE;
        float* g = sG + (size_t)so * 4 * kF;
        if (lane == 0) umma::mbar_expect_tx_only(&b[bb], (uint32_t)(nlive * 4 * kF * 4));
        __syncwarp();
        unsigned char* tile = sB + (s * NBUF + bb) * NB * 2 * NE * 128;
        if (live) {
          if (G4L) {
            // G4L: the receiver's (gsm, gvm) interleaved per feature, one 2 KB row
            if (h == 0) umma::bulk_copy_g2s(g + (size_t)slot * 4 * kF, p.G4 + (int64_t)jj * 4 * kF, 4 * kF * 4, &b[bb]);
          } else if (h == 0) {
            umma::bulk_copy_g2s(g + (size_t)slot * 4 * kF, p.Gsm + (int64_t)jj * kF, kF * 4, &b[bb]);
          } else {
            umma::bulk_copy_g2s(g + (size_t)slot * 4 * kF + kF, p.Gvm + (int64_t)jj * 3 * kF, 3 * kF * 4, &b[bb]);
          }
        }
        if (SPLIT) {
          store_basis_half_split(tile, tile + 2 * NE * 128, slot, h, bs);
          store_basis_half_split(tile, tile + 2 * NE * 128, NE + slot, h, ds);
        } else {
          store_basis_half(tile, slot, h, bs);
          store_basis_half(tile, NE + slot, h, ds);
        }
        if (h == 0) {
          sgeo[so + slot] = geo;
          if (!FOLD) sfc[so + slot] = fcv;
          sfl[so + slot] = live ? ecnt : 0;
        }
        gathered = it + 1;
        umma::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&b[bb]);
      }
    }
  } else if (warp == 2) {
    if (lane == 0) {
      if (!umma::mbar_wait(wbar, 0)) ok = false;
      const uint32_t idesc = umma::idesc_bf16_m128(2 * NE);
      int64_t k[NS];
      int t[NS], it[NS];
      bool have[NS];
      Chunk C[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        k[s] = (int64_t)blockIdx.x * NS + s;
        t[s] = 0;
        it[s] = 0;
        have[s] = chunk_at<NE>(p, k[s], C[s]);
      }
      // issue for whichever stream has its next tile ready (non-blocking probes), so that a
      // late tile of one stream does not hold back the other; a stall of more than 2 s without
      // progress gives up with a timeout
      bool any = true;
      uint32_t idle = 0;
      uint64_t t_idle = 0;
      while (ok && any) {
        any = false;
        bool progressed = false;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          while (have[s] && t[s] >= C[s].ntiles) {
            k[s] += nstreams;
            t[s] = 0;
            have[s] = chunk_at<NE>(p, k[s], C[s]);
          }
          if (!have[s]) continue;
          any = true;
          uint64_t* b = sbar + kBars * s;
          const int bb = it[s] % NBUF, a = it[s] & 1;
          if (!umma::mbar_test(&b[bb], (it[s] / NBUF) & 1)) continue;
          if (it[s] >= 2 && !umma::mbar_test(&b[10 + a], ((it[s] >> 1) - 1) & 1)) continue;
          progressed = true;
          umma::fence_after();
          const uint32_t bbase = umma::smem_u32(sB + (s * NBUF + bb) * NB * 2 * NE * 128);
#pragma unroll
          for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int kk = 0; kk < 2 * NB; ++kk)   // k-halves of the hi operand[, then of the lo one]
              umma::mma_bf16(tmem + (uint32_t)((s * 2 + a) * 6 * NE + m * 2 * NE),
                             umma::desc_sw128(umma::smem_u32(sA + m * kWfTileBytes) + 32u * (kk & 1)),
                             umma::desc_sw128(bbase + (uint32_t)(kk >> 1) * 2 * NE * 128 + 32u * (kk & 1)), idesc, kk > 0);
          umma::mma_commit(&b[8 + a]);
          issued[s] = ++it[s];
          ++t[s];
        }
        if (any && !progressed) {
          __nanosleep(64);
          if (idle++ == 0) t_idle = umma::globaltimer();
          else if ((idle & 255) == 0 && umma::globaltimer() - t_idle > 2000000000ull) ok = false;
        } else {
          idle = 0;
        }
      }
    }
  } else {
    const int s = (warp - 3) >> 2;
    const int q = warp & 3, f = q * 32 + lane;
    uint64_t* b = sbar + kBars * s;
    const float bs = FOLD ? 0.f : p.bf[f], bvv = FOLD ? 0.f : p.bf[kF + f], bvs = FOLD ? 0.f : p.bf[2 * kF + f];
    int it = 0;
    Chunk C;
    for (int64_t k = (int64_t)blockIdx.x * NS + s; ok && chunk_at<NE>(p, k, C); k += nstreams) {
      int64_t r = C.r0;
      float cur[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, nxt[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      auto fetch = [&](int64_t row, float (&o)[5]) {
        if (row < C.r1) {
          const float* pj = p.PHI + row * 6 * kF + f;
#pragma unroll
          for (int kk = 0; kk < 5; ++kk)
            if (!L0 || kk == 0 || kk == 4) o[kk] = __ldg(pj + kk * kF);
        }
      };
      float gps = 0.f, gy0 = 0.f, gy1 = 0.f, gy2 = 0.f, gpvs = 0.f;
      auto flush = [&]() {
        if (p.GPHI) {
          float* o = p.GPHI + r * 5 * kF;
          o[f] = gps; o[kF + f] = gy0; o[2 * kF + f] = gy1; o[3 * kF + f] = gy2; o[4 * kF + f] = gpvs;
        }
        gps = gy0 = gy1 = gy2 = gpvs = 0.f;
        ++r;
#pragma unroll
        for (int kk = 0; kk < 5; ++kk) cur[kk] = nxt[kk];
        fetch(r + 1, nxt);
      };
      fetch(r, cur);
      fetch(r + 1, nxt);
      while (r < C.r1 && p.arow[r + 1] == C.e0) flush();
      for (int t = 0; t < C.ntiles; ++t, ++it) {
        const int bb = it % NBUF, a = it & 1;
        if (!umma::mbar_wait(&b[8 + a], (it >> 1) & 1)) { ok = false; break; }
        if (!umma::mbar_wait(&b[bb], (it / NBUF) & 1)) { ok = false; break; }   // gathered rows visible
        umma::fence_after();
        const int64_t tb = C.e0 + (int64_t)t * NE;
        const int nlive = (int)((C.e1 - tb) < NE ? (C.e1 - tb) : NE);
        const int so = (s * NBUF + bb) * NE;
        const int* tf = sfl + so;
        const float4* tg = sgeo + so;
        const float2* tc = sfc + so;
        float* tG = sG + (size_t)so * 4 * kF + f;   // this thread's feature in each gathered row
        // lane 8k of warp q writes edge 4q + k of the tile; its previous value is read now
        const int hslot = f >> 3;
        float4 hold = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p.accumulate && (lane & 7) == 0 && hslot < nlive) hold = p.hedge[tb + hslot];
        // this thread's gathered values of edge `slot`
        auto gat = [&](int slot) -> float4 {
          if (G4L) return *reinterpret_cast<const float4*>(sG + ((size_t)(so + slot) * kF + f) * 4);
          const float* gg = tG + (size_t)slot * 4 * kF;
          return make_float4(gg[0], gg[kF], gg[2 * kF], gg[3 * kF]);
        };
        // per edge (accumulator columns w0..w5 = W_s, dW_s, W_vv, dW_vv, W_vs, dW_vs): accumulate
        // the row's phi gradients; overwrite this thread's gathered gradients in place with its
        // partials of (dU/dd, dU/du)
        auto edge = [&](float w0, float w1, float w2, float w3, float w4, float w5, int slot, float gs, float gv0,
                        float gv1, float gv2) {
          float* gg = tG + (size_t)slot * 4 * kF;
          const float4 geo = tg[slot];
          float Ws, Wvv, Wvs, dWs, dWvv, dWvs;   // filter and its distance derivative, f_c included
          if (FOLD) {
            Ws = w0; Wvv = w2; Wvs = w4;
            dWs = w1; dWvv = w3; dWvs = w5;
          } else {
            const float2 fcv = tc[slot];
            const float ws = w0 + bs, wvv = w2 + bvv, wvs = w4 + bvs;
            Ws = ws * fcv.x; Wvv = wvv * fcv.x; Wvs = wvs * fcv.x;
            dWs = fcv.x * w1 + fcv.y * ws;
            dWvv = fcv.x * w3 + fcv.y * wvv;
            dWvs = fcv.x * w5 + fcv.y * wvs;
          }
          // L0 (first layer): v = 0 so psi = 0, and no phi gradients are written, so only the
          // per-edge partials are formed
          if (!L0) {
            gps = fmaf(gs, Ws, gps);
            gy0 = fmaf(gv0, Wvv, gy0);
            gy1 = fmaf(gv1, Wvv, gy1);
            gy2 = fmaf(gv2, Wvv, gy2);
          }
          const float qv = -(gv0 * geo.x + gv1 * geo.y + gv2 * geo.z);
          if (!L0) gpvs = fmaf(qv, Wvs, gpvs);
          const float gWs = gs * cur[0], gWvs = qv * cur[4];
          const float gWvv = L0 ? 0.0f : gv0 * cur[1] + gv1 * cur[2] + gv2 * cur[3];
          const float tv = cur[4] * Wvs;
          const float pd = gWs * dWs + gWvv * dWvv + gWvs * dWvs;
          if (G4L) {
            *reinterpret_cast<float4*>(sG + ((size_t)(so + slot) * kF + f) * 4) = make_float4(pd, gv0 * tv, gv1 * tv, gv2 * tv);
          } else {
            gg[0] = pd;
            gg[kF] = gv0 * tv;
            gg[2 * kF] = gv1 * tv;
            gg[3 * kF] = gv2 * tv;
          }
        };
        if (PIPE) {
          const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((s * 2 + a) * 6 * NE);
          uint32_t RA[6][4], RB[6][4];
          // four edges b .. b + 3 with their accumulator columns in R
          auto half = [&](const uint32_t (&R)[6][4], int b4) {
            const int4 fl = *reinterpret_cast<const int4*>(tf + b4);
            if ((fl.x | fl.y | fl.z | fl.w) == 0 && b4 + 4 <= nlive) {
              // no row ends in these four edges: their gathered values are read first
              float4 G[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) G[u] = gat(b4 + u);
#pragma unroll
              for (int u = 0; u < 4; ++u)
                edge(__uint_as_float(R[0][u]), __uint_as_float(R[1][u]), __uint_as_float(R[2][u]),
                     __uint_as_float(R[3][u]), __uint_as_float(R[4][u]), __uint_as_float(R[5][u]), b4 + u, G[u].x,
                     G[u].y, G[u].z, G[u].w);
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int slot = b4 + u;
                if (slot < nlive) {
                  const float4 gq = gat(slot);
                  edge(__uint_as_float(R[0][u]), __uint_as_float(R[1][u]), __uint_as_float(R[2][u]),
                       __uint_as_float(R[3][u]), __uint_as_float(R[4][u]), __uint_as_float(R[5][u]), slot, gq.x, gq.y,
                       gq.z, gq.w);
                  for (int nf = tf[slot]; nf > 0 && r < C.r1; --nf) flush();
                }
              }
            }
          };
          umma::tmem_ld4x6_issue(tbase, NE, RA);
          umma::tmem_wait4x6(RA);
#pragma unroll 1
          for (int c = 0; c < NE / 8; ++c) {
            umma::tmem_ld4x6_issue(tbase + c * 8 + 4, NE, RB);   // in flight during the first half
            half(RA, c * 8);
            umma::tmem_wait4x6(RB);
            if (c + 1 < NE / 8) {
              umma::tmem_ld4x6_issue(tbase + (c + 1) * 8, NE, RA);   // in flight during the second half
            } else {
              // every accumulator column of the tile has been read: the MMA may reuse the buffer
              umma::fence_before();
              __syncwarp();
              if (lane == 0) umma::mbar_arrive(&b[10 + a]);
            }
            half(RB, c * 8 + 4);
            if (c + 1 < NE / 8) umma::tmem_wait4x6(RA);
          }
        } else {
#pragma unroll 1
        for (int c = 0; c < NE / 8; ++c) {
          // column groups at stride NE: W_s, dW_s, W_vv, dW_vv, W_vs, dW_vs
          float W[6][8];
          umma::tmem_ld8x6(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((s * 2 + a) * 6 * NE + c * 8), NE, W);
          if (c == NE / 8 - 1) {
            umma::fence_before();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&b[10 + a]);
          }
          const int4 fa = *reinterpret_cast<const int4*>(tf + c * 8), fb = *reinterpret_cast<const int4*>(tf + c * 8 + 4);
          if ((fa.x | fa.y | fa.z | fa.w | fb.x | fb.y | fb.z | fb.w) == 0 && c * 8 + 8 <= nlive) {
            // no row ends in these eight edges: all their gathered values are read first, so
            // the 32 shared-memory loads overlap, then straight-line arithmetic
            float4 G[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) G[u] = gat(c * 8 + u);
#pragma unroll
            for (int u = 0; u < 8; ++u)
              edge(W[0][u], W[1][u], W[2][u], W[3][u], W[4][u], W[5][u], c * 8 + u, G[u].x, G[u].y, G[u].z, G[u].w);
          } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int slot = c * 8 + u;
              if (slot < nlive) {
                const float4 gq = gat(slot);
                edge(W[0][u], W[1][u], W[2][u], W[3][u], W[4][u], W[5][u], slot, gq.x, gq.y, gq.z, gq.w);
                for (int nf = tf[slot]; nf > 0 && r < C.r1; --nf) flush();
              }
            }
          }
        }
        }
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&b[12]);
        if (!umma::mbar_wait(&b[12], it & 1)) { ok = false; break; }
        {
          // Reduction over the F features: thread f sums half (h) of component `comp` of edge
          // `slot`, starting at a rotation 4 (2 comp + h) so that a quarter-warp's 16-byte reads
          // fall in distinct banks and the summation order depends on (comp, h) alone, not on
          // the edge's slot in the tile (results do not depend on where tiles start); the two
          // halves combine across lanes 2k, 2k+1, and lane 8k then holds the four components of
          // edge 4q + k.
          // G4L: thread f sums all four components of edge f >> 3 over 16 features
          // (part = f & 7, rotated by the part so that a quarter-warp's 16-byte reads fall in
          // distinct banks), then the eight parts combine across lanes 8k .. 8k+7
          const int o = f >> 1, slot = G4L ? (f >> 3) : (o >> 2), comp = o & 3, h = f & 1;
          float acc = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
          if (G4L) {
            const int part = f & 7;
            float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
            if (slot < nlive) {
              const float4* base = reinterpret_cast<const float4*>(sG) + (size_t)(so + slot) * kF + part * 16;
#pragma unroll
              for (int ii = 0; ii < 16; ++ii) {
                const float4 v = base[(ii + part) & 15];
                sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
              }
            }
#pragma unroll
            for (int off = 1; off < 8; off <<= 1) {
              sum.x += __shfl_xor_sync(0xffffffffu, sum.x, off);
              sum.y += __shfl_xor_sync(0xffffffffu, sum.y, off);
              sum.z += __shfl_xor_sync(0xffffffffu, sum.z, off);
              sum.w += __shfl_xor_sync(0xffffffffu, sum.w, off);
            }
            acc = sum.x; g0 = sum.y; g1 = sum.z; g2 = sum.w;
          } else {
          if (slot < nlive) {
            const float* base = sG + (size_t)so * 4 * kF + (size_t)slot * 4 * kF + comp * kF + h * 64;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
            for (int ii = 0; ii < 16; ++ii) {
              const float4 v = *reinterpret_cast<const float4*>(base + ((4 * ii + 4 * (lane & 7)) & 63));
              a0 += v.x; a1 += v.y; a2 += v.z; a3 += v.w;
            }
            acc = (a0 + a1) + (a2 + a3);
          }
          acc += __shfl_xor_sync(0xffffffffu, acc, 1);
          g0 = __shfl_down_sync(0xffffffffu, acc, 2);
          g1 = __shfl_down_sync(0xffffffffu, acc, 4);
          g2 = __shfl_down_sync(0xffffffffu, acc, 6);
          }
          if ((lane & 7) == 0 && slot < nlive) {
            const float pd = acc;
            const float4 geo = tg[slot];
            const float ux = -geo.x, uy = -geo.y, uz = -geo.z, id = 1.0f / geo.w;
            const float gdu = g0 * ux + g1 * uy + g2 * uz;
            float4 hv = make_float4(pd * ux + (g0 - gdu * ux) * id, pd * uy + (g1 - gdu * uy) * id,
                                    pd * uz + (g2 - gdu * uz) * id, 0.f);
            hv.x += hold.x; hv.y += hold.y; hv.z += hold.z;
            p.hedge[tb + slot] = hv;
          }
        }
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&b[4 + bb]);
      }
      if (!ok) break;
      while (r < C.r1) flush();
    }
  }
  if (!ok) atomicOr(p.status, (int)ST_TIMEOUT);
  if (warp < NS && lane == 0) {
    // the bulk copies of the last two tiles this producer issued have landed before exit
    for (int t = gathered - NBUF; t < gathered; ++t)
      if (t >= 0) umma::mbar_wait(&sbar[kBars * warp + (t % NBUF)], (t / NBUF) & 1, 200000000ull);
  }
  if (warp == 2 && lane == 0)
    for (int s = 0; s < NS; ++s)
      if (issued[s] > 0)
        umma::mbar_wait(&sbar[kBars * s + 8 + ((issued[s] - 1) & 1)], ((issued[s] - 1) >> 1) & 1, 200000000ull);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  if (warp == 2) umma::tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------------------------ host side
constexpr int kFwdNE = 32, kFwdNS = 4;   // 4 streams x 3 x 32 TMEM columns, 16 epilogue warps
constexpr bool kFwdSplit = false;        // basis as BF16 hi + lo (two MMAs) in the message kernel
constexpr int kFwdTB = 1;                // TMEM accumulator buffers per stream
constexpr bool kBwgSplit = false;        // basis as BF16 hi + lo in the bulk-gathered adjoint
constexpr int kBwdNE = 16, kBwdNS = 3;   // 3 streams x 6 x 16 TMEM columns, 12 epilogue warps
constexpr int kBwgNE = 16, kBwgNS = 2;   // bulk-gathered adjoint: 2 streams, double-buffered tiles
constexpr int kFwgNE = 16, kFwgNS = 2;   // bulk-gathered message kernel
constexpr int64_t kChunkRows = 32;       // default rows per block-cyclic chunk

static size_t fwd_smem(bool split = kFwdSplit) {
  return 1024 + kWfBytes + (size_t)kFwdNS * 2 * (split ? 2 : 1) * kFwdNE * 128 + (size_t)kFwdNS * 2 * kFwdNE * (4 + 4 + 16) +
         8 * (1 + 8 * kFwdNS) + 64;
}
static size_t bwd_smem() {
  return 1024 + kWfBytes + (size_t)kBwdNS * 4 * kBwdNE * 128 + (size_t)kBwdNS * 2 * kBwdNE * (4 + 4 + 16 + 8) +
         (size_t)kBwdNS * kBwdNE * 16 * 4 + 8 * (1 + 8 * kBwdNS) + 64;
}

static size_t bwg_smem(bool split = kBwgSplit, int ne = kBwgNE, int nbuf = 2) {
  return 1024 + kWfBytes + (size_t)kBwgNS * nbuf * (split ? 2 : 1) * 2 * ne * 128 + (size_t)kBwgNS * nbuf * ne * 4 * kF * 4 +
         (size_t)kBwgNS * nbuf * ne * (4 + 16 + 8) + 8 * (1 + 13 * kBwgNS) + 64;
}
static size_t fwg_smem() {
  return 1024 + kWfBytes + (size_t)kFwgNS * 4 * kFwgNE * 128 + (size_t)kFwgNS * 2 * kFwgNE * 5 * kF * 4 +
         (size_t)kFwgNS * 2 * kFwgNE * (4 + 16) + 8 * (1 + 8 * kFwgNS) + 64;
}

// K < kKPad leaves basis column K free for the folded filter bias
bool edge_tc_supported(int F, int K) { return F == kF && K < kKPad && K >= 2; }

// Rows per block-cyclic chunk: the context's setting, or one contiguous range per stream (0).
static int64_t chunk_rows_for(const ModelW& m, int64_t n, int ns) {
  if (m.edge_chunk_rows > 0) return m.edge_chunk_rows;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t streams = (int64_t)sms * ns;
  const int64_t r = (n + streams - 1) / streams;
  return r > 0 ? r : 1;
}

// One CTA per SM (512 TMEM columns each), rows split evenly over the CTAs.
static int grid_for(int64_t n, int64_t* rows_per_cta) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t ctas = sms;
  int64_t rpc = (n + ctas - 1) / ctas;
  if (rpc < 1) rpc = 1;
  *rows_per_cta = rpc;
  return (int)((n + rpc - 1) / rpc);
}

int edge_fwd_tc(cudaStream_t st, const ModelW& m, int t, int64_t n, const int32_t* arow, const int32_t* acol,
                const float4* ar, const float* PHI, const float* S, const float* V, float* SM, float* VM,
                bf16* VMb, int* status, const int32_t* aend) {
  if (n == 0) return 0;
  CUtensorMap tm;
  if (!make_tmap_bf16(&tm, m.L[t].Wfb, 3 * kF, 64, 64, 128)) return -2;
  EdgeTcArgs a{};
  a.n = n; a.K = m.K; a.rc = m.rc; a.arow = arow; a.acol = acol; a.ar = ar; a.PHI = PHI; a.S = S; a.V = V;
  a.bf = m.L[t].bf; a.SM = SM; a.VM = VM; a.VMb = VMb; a.status = status; a.aend = aend;
  const int grid = grid_for(n, &a.rows_per_cta);
  a.chunk_rows = chunk_rows_for(m, n, m.tc_message_variant == 4 ? kFwdNS : kFwgNS);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_edge_fwd_tc<kFwdNE, kFwdNS, kFwdSplit, kFwdTB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem());
    cudaFuncSetAttribute(k_edge_fwd_tc<kFwdNE, kFwdNS, kFwdSplit, kFwdTB, false, false, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem());
    cudaFuncSetAttribute(k_edge_fwd_tc<kFwdNE, kFwdNS, kFwdSplit, kFwdTB, false, false, true, 20>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem());
    cudaFuncSetAttribute(k_edge_fwd_tc<kFwdNE, kFwdNS, kFwdSplit, kFwdTB, false, false, false, 20>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem());
    cudaFuncSetAttribute(k_edge_fwd_tc<kFwdNE, kFwdNS, true, kFwdTB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(true));
    cudaFuncSetAttribute(k_edge_fwd_tc<kFwdNE, kFwdNS, kFwdSplit, kFwdTB, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem());
    cudaFuncSetAttribute(k_edge_fwd_tcg<kFwgNE, kFwgNS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwg_smem());
    attr = true;
  }
  LaunchScope ls_(st);
  if (m.tc_message_variant == 1) {
    // the first layer's v = 0 (embedding): its message kernel skips the psi channels
    // K = 20 (the usual basis) with a compile-time loop bound
    if (t == 0 && m.K == 20)
      k_edge_fwd_tc<kFwdNE, kFwdNS, kFwdSplit, kFwdTB, false, false, true, 20><<<grid, 32 * (3 + 4 * kFwdNS), fwd_smem(), st>>>(tm, a);
    else if (t == 0)
      k_edge_fwd_tc<kFwdNE, kFwdNS, kFwdSplit, kFwdTB, false, false, true><<<grid, 32 * (3 + 4 * kFwdNS), fwd_smem(), st>>>(tm, a);
    else if (m.K == 20)
      k_edge_fwd_tc<kFwdNE, kFwdNS, kFwdSplit, kFwdTB, false, false, false, 20><<<grid, 32 * (3 + 4 * kFwdNS), fwd_smem(), st>>>(tm, a);
    else
      k_edge_fwd_tc<kFwdNE, kFwdNS, kFwdSplit, kFwdTB><<<grid, 32 * (3 + 4 * kFwdNS), fwd_smem(), st>>>(tm, a);
  } else if (m.tc_message_variant == 4) {
    k_edge_fwd_tc<kFwdNE, kFwdNS, kFwdSplit, kFwdTB, false, true><<<grid, 32 * (3 + 4 * kFwdNS), fwd_smem(), st>>>(tm, a);
  } else if (m.tc_message_variant == 3) {
    k_edge_fwd_tc<kFwdNE, kFwdNS, true, kFwdTB><<<grid, 32 * (3 + 4 * kFwdNS), fwd_smem(true), st>>>(tm, a);
  } else {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_edge_fwd_tcg<kFwgNE, kFwgNS><<<sms, 32 * (3 + 4 * kFwgNS), fwg_smem(), st>>>(tm, a);
  }
  return 0;
}

int edge_bwd_tc(cudaStream_t st, const ModelW& m, int t, int accumulate, int64_t n, const int32_t* arow,
                const int32_t* acol, const float4* ar, const float* PHI, const float* Gsm, const float* Gvm,
                float* GPHI, float4* hedge, int* status, const int32_t* aend, const float* G4) {
  if (n == 0) return 0;
  CUtensorMap tm;
  if (!make_tmap_bf16(&tm, m.L[t].Wfb, 3 * kF, 64, 64, 128)) return -2;
  EdgeTcArgs a{};
  a.n = n; a.K = m.K; a.rc = m.rc; a.accumulate = accumulate; a.arow = arow; a.acol = acol; a.ar = ar;
  a.PHI = PHI; a.Gsm = Gsm; a.Gvm = Gvm; a.bf = m.L[t].bf; a.GPHI = GPHI; a.hedge = hedge; a.status = status;
  a.aend = aend;
  a.G4 = G4;
  const int grid = grid_for(n, &a.rows_per_cta);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_edge_bwd_tc<kBwdNE, kBwdNS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem());
    cudaFuncSetAttribute(k_edge_bwd_tcg<kBwgNE, kBwgNS, false, kBwgSplit>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwg_smem());
    cudaFuncSetAttribute(k_edge_bwd_tcg<kBwgNE, kBwgNS, true, kBwgSplit>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwg_smem());
    cudaFuncSetAttribute(k_edge_bwd_tcg<kBwgNE, kBwgNS, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwg_smem(true));
    cudaFuncSetAttribute(k_edge_bwd_tcg<kBwgNE, kBwgNS, false, kBwgSplit, 2, 20>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwg_smem());
    cudaFuncSetAttribute(k_edge_bwd_tcg<kBwgNE, kBwgNS, false, kBwgSplit, 2, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwg_smem());
    cudaFuncSetAttribute(k_edge_bwd_tcg<kBwgNE, kBwgNS, false, kBwgSplit, 2, 20, true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwg_smem());
    cudaFuncSetAttribute(k_edge_bwd_tcg<kBwgNE, kBwgNS, false, kBwgSplit, 2, 20, true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwg_smem());
    attr = true;
  }
  a.chunk_rows = chunk_rows_for(m, n, kBwgNS);
  LaunchScope ls_(st);
  if (m.tc_adjoint_variant >= 2) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (m.tc_adjoint_variant == 3)
      k_edge_bwd_tcg<kBwgNE, kBwgNS, true, kBwgSplit><<<sms, 32 * (3 + 4 * kBwgNS), bwg_smem(), st>>>(tm, a);
    else if (m.tc_adjoint_variant == 4)
      k_edge_bwd_tcg<kBwgNE, kBwgNS, false, true><<<sms, 32 * (3 + 4 * kBwgNS), bwg_smem(true), st>>>(tm, a);
    // the usual basis size (K = 20) with a compile-time loop bound; G4: gradients interleaved
    // (with the accumulator read in pipelined 4-edge halves)
    else if (m.K == 20 && G4 && t == 0 && !GPHI)   // first layer: v = 0, no phi gradients
      k_edge_bwd_tcg<kBwgNE, kBwgNS, false, kBwgSplit, 2, 20, true, true, true><<<sms, 32 * (3 + 4 * kBwgNS), bwg_smem(), st>>>(tm, a);
    else if (m.K == 20 && G4)
      k_edge_bwd_tcg<kBwgNE, kBwgNS, false, kBwgSplit, 2, 20, true, false, true><<<sms, 32 * (3 + 4 * kBwgNS), bwg_smem(), st>>>(tm, a);
    else if (G4)
      k_edge_bwd_tcg<kBwgNE, kBwgNS, false, kBwgSplit, 2, 0, true><<<sms, 32 * (3 + 4 * kBwgNS), bwg_smem(), st>>>(tm, a);
    else if (m.K == 20)
      k_edge_bwd_tcg<kBwgNE, kBwgNS, false, kBwgSplit, 2, 20><<<sms, 32 * (3 + 4 * kBwgNS), bwg_smem(), st>>>(tm, a);
    else
      k_edge_bwd_tcg<kBwgNE, kBwgNS, false, kBwgSplit><<<sms, 32 * (3 + 4 * kBwgNS), bwg_smem(), st>>>(tm, a);
  } else
    k_edge_bwd_tc<kBwdNE, kBwdNS><<<grid, 32 * (3 + 4 * kBwdNS), bwd_smem(), st>>>(tm, a);
  return 0;
}

}  // namespace ctd
