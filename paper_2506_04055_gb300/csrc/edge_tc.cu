// edge_tc.cu -- the edge adjoint with the radial filter contraction on tcgen05 (BF16 path,
// F = 128, radial basis K <= 31).
//
// The filter W_e = (Wf rbf(d_e) + bf) f_c(d_e) (PaiNN message function, arXiv 2506.04055
// Methods "Graph Neural Networks" / "Chosen Architectures") and its distance derivative are
// [3F x (K+1)] x [(K+1) x edges] contractions per tile of edges: with the weights [Wf | bf] and
// the basis columns (rbf_k f_c, f_c), D[c][e] = W_e[c], and with (rbf_k' f_c + rbf_k f_c', f_c')
// its distance derivative.  They run as UMMA with M = 128 filter channels (three M tiles: the
// s, vv and vs blocks), N = 2 x 16 edges (basis and derivative basis of a 16-edge tile),
// K = 32 (the basis zero-padded), FP16 operands (11 significant bits; the weights, the basis
// and its derivative lie far inside FP16's range) and FP32 accumulation in TMEM.  Everything
// after the contraction (the adjoint terms, the reductions over the features) stays FP32 on
// CUDA cores.
//
// CTA layout (one CTA per SM, 2 row streams):
//   warps 0..1 producers, one per stream: per edge of the next tile, geometry, f_c, f_c' and
//              the basis and its derivative (a lane pair per edge), written as a 128B-swizzled
//              FP16 tile; bulk copies of the receivers' interleaved gradient rows; Wf arrives
//              once per CTA by TMA
//   warp 2     TMEM owner and single-thread MMA issue
//   warps 3..  epilogue, four warps per stream: thread = feature channel f (TMEM lane); a
//              sender's phi gradients stay in registers until its row ends (no atomics)
// Rows are handed out in chunks block-cyclically over all streams of the GPU.  All waits are
// bounded and record ST_TIMEOUT on expiry.
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

// Columns 16h .. 16h+15 of row r of a 128B-swizzled FP16 tile (two 16-byte chunks).
__device__ __forceinline__ void store_basis_half(unsigned char* tile, int r, int h, const float (&v)[16]) {
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    uint32_t w[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      __half2 b2 = __floats2half2_rn(v[8 * c + 2 * x], v[8 * c + 2 * x + 1]);
      w[x] = *reinterpret_cast<uint32_t*>(&b2);
    }
    *reinterpret_cast<uint4*>(tile + umma::sw128_offset(r, 16 * h + 8 * c)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

struct EdgeTcArgs {
  int64_t n;
  int64_t chunk_rows;              // rows per block-cyclic chunk
  int K;
  float rc;
  int accumulate;                  // add to hedge (layers after the first processed)
  const int32_t* __restrict__ arow;
  const int32_t* __restrict__ acol;
  const int32_t* __restrict__ aend;  // rows completed at each edge (1 + following empty rows; 0 inside a row)
  const float4* __restrict__ ar;
  const float* __restrict__ PHI;   // [n][6F] FP32 message table, or
  const __half* __restrict__ PHIh; // [n][6F] its FP16 copy (the one the contracted message step used)
  float* __restrict__ GPHI;        // [n][3F]: the row's psi gradients (gpsi_0..2), or null (first layer)
  __nv_bfloat16* __restrict__ GP3b;  // [n][3F]: BF16 operand of the phi-MLP backward; blocks 0 and 2
                                     // (gphi_s, gphi_vs) written here, block 1 by the pass after
  float4* __restrict__ hedge;      // [E]
  const float* __restrict__ G4;    // [n][F][4] = (gsm, gvm_0..2) per feature, interleaved
  int* status;
};

}  // namespace


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

// Adjoint: the MMA yields the filter W = (Wf rbf + bf) f_c and its distance derivative per edge
// (f_c, f_c' and the bias folded into the basis tile); the receivers' gradient rows, (gsm_i, gvm_i) interleaved per feature (G4, 2 KB),
// are gathered by bulk copies.  Thread f accumulates the row's phi gradients and overwrites its
// own feature of the gathered row with its partials of (dU/dd, dU/du); after a stream barrier
// the partials are reduced over the F features from shared memory and turned into hedge[e].
// The epilogue reads the accumulator in 4-edge halves, each half's TMEM loads in flight while
// the previous half is computed.  KC: compile-time basis size (0: runtime).  L0: first layer
// (v = 0, no phi gradients).
template <int NE, int NS, int KC = 0, bool L0 = false>
__global__ void __launch_bounds__(32 * (3 + 4 * NS), 1) k_edge_bwd_tcg(const __grid_constant__ CUtensorMap tmWf, EdgeTcArgs p) {
  static_assert(NS <= 2, "one producer warp per stream");
  constexpr int NBUF = 2;   // tile buffers per stream
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = align1024(smem_raw);
  unsigned char* sA = smem;                                          // Wf tiles (bias in column K)
  // per buffer one operand of 2 NE rows: the basis of the tile's
  // edges in rows 0..NE-1 and their derivative basis in rows NE..2NE-1, so that one MMA per
  // channel block yields [W | dW/dd] as 2 NE columns
  static_assert(NS * 2 * 6 * NE <= 512, "TMEM columns");
  static_assert(NE == 16, "tile shape: one lane pair per edge");
  unsigned char* sB = sA + kWfBytes;                                 // [NS][NBUF][NB][2 NE x 128 B]
  float* sG = reinterpret_cast<float*>(sB + NS * NBUF * 2 * NE * 128);   // [NS][NBUF][NE][4F]
  int* sfl = reinterpret_cast<int*>(sG + (size_t)NS * NBUF * NE * 4 * kF);   // [NS][NBUF][NE]
  float4* sgeo = reinterpret_cast<float4*>(sfl + NS * NBUF * NE);    // [NS][NBUF][NE] (u, d)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sgeo + NS * NBUF * NE);
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
        const bool live = slot < nlive;
        if (live) {
          const float d = r.w, id = 1.0f / d;
          geo = make_float4(r.x * id, r.y * id, r.z * id, d);
          const float fc = 0.5f * (cospif(d * inv_rc) + 1.0f);
          const float dfc = -0.5f * 3.14159265358979f * inv_rc * sinpif(d * inv_rc);
          // the cutoff and the filter bias folded in: columns k < K hold b_k f_c and its distance
          // derivative b_k' f_c + b_k f_c', column K holds f_c and f_c' (it meets the bias bf in
          // the weights' column K), so the MMA yields W and dW/dd themselves
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int kk = 2 * q + h;
            const float tq = d - (float)kk * sig;
            const bool in = kk < KK;
            const float v = in ? expf(-tq * tq * inv2s2) : 0.0f;
            const float dv = -v * tq * inv_s2;
            bq[q] = in ? v * fc : (kk == KK ? fc : 0.0f);
            dq[q] = in ? fmaf(dv, fc, v * dfc) : (kk == KK ? dfc : 0.0f);
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
        unsigned char* tile = sB + (s * NBUF + bb) * 2 * NE * 128;
        // the receiver's (gsm, gvm) interleaved per feature, one 2 KB row
        if (live && h == 0)
          umma::bulk_copy_g2s(g + (size_t)slot * 4 * kF, p.G4 + (int64_t)jj * 4 * kF, 4 * kF * 4, &b[bb]);
        store_basis_half(tile, slot, h, bs);
        store_basis_half(tile, NE + slot, h, ds);
        if (h == 0) {
          sgeo[so + slot] = geo;
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
      const uint32_t idesc = umma::idesc_f16_m128(2 * NE);   // FP16 weights and basis
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
          const uint32_t bbase = umma::smem_u32(sB + (s * NBUF + bb) * 2 * NE * 128);
#pragma unroll
          for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)   // the two 16-column k-halves of the basis
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
    int it = 0;
    Chunk C;
    for (int64_t k = (int64_t)blockIdx.x * NS + s; ok && chunk_at<NE>(p, k, C); k += nstreams) {
      int64_t r = C.r0;
      // the row's table values (cur) and the next row's, prefetched as raw bits (nxt: FP32, or
      // FP16 in the low half) and converted only when that row begins, one row after the load
      const bool th = p.PHIh != nullptr;
      float cur[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      uint32_t nxt[5] = {0u, 0u, 0u, 0u, 0u};
      auto fetch = [&](int64_t row, uint32_t (&o)[5]) {
        if (row < C.r1) {
          if (th) {
            const __half* pj = p.PHIh + row * 6 * kF + f;
#pragma unroll
            for (int kk = 0; kk < 5; ++kk)
              if (!L0 || kk == 0 || kk == 4) o[kk] = __half_as_ushort(__ldg(pj + kk * kF));
          } else {
            const float* pj = p.PHI + row * 6 * kF + f;
#pragma unroll
            for (int kk = 0; kk < 5; ++kk)
              if (!L0 || kk == 0 || kk == 4) o[kk] = __float_as_uint(__ldg(pj + kk * kF));
          }
        }
      };
      auto take = [&]() {
#pragma unroll
        for (int kk = 0; kk < 5; ++kk)
          cur[kk] = th ? __half2float(__ushort_as_half((unsigned short)nxt[kk])) : __uint_as_float(nxt[kk]);
      };
      float gps = 0.f, gy0 = 0.f, gy1 = 0.f, gy2 = 0.f, gpvs = 0.f;
      auto flush = [&]() {
        if (p.GPHI) {
          float* o = p.GPHI + r * 3 * kF;
          o[f] = gy0; o[kF + f] = gy1; o[2 * kF + f] = gy2;
          // the phi-MLP backward reads gphi_s and gphi_vs only as BF16 operands
          __nv_bfloat16* ob = p.GP3b + r * 3 * kF;
          ob[f] = __float2bfloat16_rn(gps);
          ob[2 * kF + f] = __float2bfloat16_rn(gpvs);
        }
        gps = gy0 = gy1 = gy2 = gpvs = 0.f;
        ++r;
        take();
        fetch(r + 1, nxt);
      };
      fetch(r, nxt);
      take();
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
        // lane 8k of warp q writes edge 4q + k of the tile; its previous value is read now
        const int hslot = f >> 3;
        float4 hold = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p.accumulate && (lane & 7) == 0 && hslot < nlive) hold = p.hedge[tb + hslot];
        // this thread's gathered values of edge `slot`
        auto gat = [&](int slot) -> float4 {
          return *reinterpret_cast<const float4*>(sG + ((size_t)(so + slot) * kF + f) * 4);
        };
        // per edge (accumulator columns w0..w5 = W_s, dW_s, W_vv, dW_vv, W_vs, dW_vs): accumulate
        // the row's phi gradients; overwrite this thread's gathered gradients in place with its
        // partials of (dU/dd, dU/du)
        auto edge = [&](float w0, float w1, float w2, float w3, float w4, float w5, int slot, float gs, float gv0,
                        float gv1, float gv2) {
          const float4 geo = tg[slot];
          // the accumulator holds the filter and its distance derivative, cutoff and bias included
          const float Ws = w0, dWs = w1, Wvv = w2, dWvv = w3, Wvs = w4, dWvs = w5;
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
          *reinterpret_cast<float4*>(sG + ((size_t)(so + slot) * kF + f) * 4) = make_float4(pd, gv0 * tv, gv1 * tv, gv2 * tv);
        };
        {
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
        }
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&b[12]);
        if (!umma::mbar_wait(&b[12], it & 1)) { ok = false; break; }
        {
          // Reduction over the F features: thread f sums all four components of edge f >> 3
          // over 16 features (part = f & 7, rotated by the part so that a quarter-warp's 16-byte
          // reads fall in distinct banks, in an order that does not depend on the edge's slot in
          // the tile: results do not depend on where tiles start), then the eight parts combine
          // across lanes 8k .. 8k+7, and lane 8k holds the four components of edge 4q + k.
          const int slot = f >> 3, part = f & 7;
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
          const float acc = sum.x, g0 = sum.y, g1 = sum.z, g2 = sum.w;
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
constexpr int kBwgNE = 16, kBwgNS = 2;   // bulk-gathered adjoint: 2 streams, double-buffered tiles

static size_t bwg_smem() {
  return 1024 + kWfBytes + (size_t)kBwgNS * 2 * 2 * kBwgNE * 128 + (size_t)kBwgNS * 2 * kBwgNE * 4 * kF * 4 +
         (size_t)kBwgNS * 2 * kBwgNE * (4 + 16) + 8 * (1 + 13 * kBwgNS) + 64;
}

// K < kKPad leaves basis column K zero
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

int edge_bwd_tc(cudaStream_t st, const ModelW& m, int t, int accumulate, int64_t n, const int32_t* arow,
                const int32_t* acol, const float4* ar, const float* PHI, float* GPHI, __nv_bfloat16* GP3b,
                float4* hedge, int* status, const int32_t* aend, const float* G4, const __half* PHIh) {
  if (n == 0) return 0;
  if (!G4 || (!PHI && !PHIh) || (GPHI && !GP3b)) return -1;
  CUtensorMap tm;
  // the FP16 weights: 2-byte elements like BF16, which is all the TMA copy depends on
  if (!m.L[t].Wfh || !make_tmap_bf16(&tm, m.L[t].Wfh, 3 * kF, 64, 64, 128)) return -2;
  EdgeTcArgs a{};
  a.n = n; a.K = m.K; a.rc = m.rc; a.accumulate = accumulate; a.arow = arow; a.acol = acol; a.ar = ar;
  a.PHI = PHI; a.PHIh = PHIh; a.GPHI = GPHI; a.GP3b = GP3b; a.hedge = hedge; a.status = status; a.aend = aend; a.G4 = G4;
  a.chunk_rows = chunk_rows_for(m, n, kBwgNS);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_edge_bwd_tcg<kBwgNE, kBwgNS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwg_smem());
    cudaFuncSetAttribute(k_edge_bwd_tcg<kBwgNE, kBwgNS, 20>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwg_smem());
    cudaFuncSetAttribute(k_edge_bwd_tcg<kBwgNE, kBwgNS, 20, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwg_smem());
    attr = true;
  }
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 32 * (3 + 4 * kBwgNS);
  LaunchScope ls_(st);
  if (m.K == 20 && t == 0 && !GPHI)   // the usual basis size; first layer: v = 0, no phi gradients
    k_edge_bwd_tcg<kBwgNE, kBwgNS, 20, true><<<sms, threads, bwg_smem(), st>>>(tm, a);
  else if (m.K == 20)
    k_edge_bwd_tcg<kBwgNE, kBwgNS, 20><<<sms, threads, bwg_smem(), st>>>(tm, a);
  else
    k_edge_bwd_tcg<kBwgNE, kBwgNS><<<sms, threads, bwg_smem(), st>>>(tm, a);
  return 0;
}

}  // namespace ctd
