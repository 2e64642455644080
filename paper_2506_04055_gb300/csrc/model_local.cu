// model_local.cu -- the strictly local equivariant edge model (Allegro form, rotation orders
// <= 1), forward and hand-written adjoint, FP32 on CUDA cores.
//
// Methods, "(Semi-)Local Potential Models" and "Chosen Architectures": information moves only
// between directed edges that leave the same atom, so an atom's energy depends on its own
// cutoff sphere alone, whatever the number of layers.  Every quantity lives on an edge
// e = (i -> j) of the active CSR list (row i = the edges leaving atom i, r_e = x_j - x_i):
//   x = silu([b f_c | onehot Z_i | onehot Z_j] A0 + c0)             two-body latent   [E][F]
//   s = (x P0)[0:C], v = (x P0)[C:2C] u                             edge features     [E][C], [E][3][C]
//   layer l: om = x Q_l;  Gs_i = sum_{e from i} f_c om[0:C],  Gv_i = sum f_c om[C:2C] u
//            ts = [s Gs_i | v . Gv_i], tv = [s Gv_i | v Gs_i]        tensor-product paths
//            x = silu([x | ts] M_l + m_l);  (l < L) s = ts Gs_l, v = tv Gv_l
//   E_i = e_scale w_i sum_{e from i} f_c (silu(x R1 + d1) . R2 + d2)
// The dense contractions are GEMMs over edge rows (the FP32 SIMT GEMM of model_fp32.cu); the
// centre sums are one thread per (atom, channel) over its row in a fixed order; everything
// else is one thread per edge or per (edge, channel).  The adjoint reverses each step and ends
// in hedge = -dE/dr_e, from which the shared force kernel assembles forces and virial through
// the reverse-edge index (no atomics anywhere, so results do not depend on the batch).
#include "ctd_internal.cuh"

namespace ctd {
namespace {

constexpr float kPiF = 3.14159265358979323846f;

// Eight FP32 values as one 16-byte store of BF16 (a thread writing its own edge's row: one
// store per 8 columns instead of one per column)
__device__ __forceinline__ void st8_bf16(__nv_bfloat16* p, const float (&v)[8]) {
  uint32_t w[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    w[j] = *reinterpret_cast<const uint32_t*>(&b);
  }
  *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ float4 ld4f(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4_bf16(__nv_bfloat16* p, float4 v) {
  const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
  *reinterpret_cast<uint2*>(p) = make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
}

inline unsigned nblocks(int64_t w) { return (unsigned)((w + kThreads - 1) / kThreads); }

// Per-edge and per-atom arrays, carved from one allocation (128-byte aligned pieces).
struct LocalBufs {
  int32_t* erow;                      // [E] row (centre atom) of each edge
  float *geo, *in, *z0, *w0, *zh, *h;  // [E][8] (d, f_c, f_c', u, 0, 0), [E][KA], [E][F], [E][2C], [E][F/2] x2
  float* X[kMaxT + 1];                // [E][F+2C]: x^l in columns 0..F-1, ts of layer l+1 after it
  float *S[kMaxT], *V[kMaxT];         // s^l [E][C], v^l [E][3][C], l = 0..L-1
  float *OM[kMaxT + 1], *Z[kMaxT + 1];  // l = 1..L: [E][2C], [E][F]
  float* TV[kMaxT];                   // l = 1..L-1: [E][3][2C]
  float *gamS[kMaxT + 1], *gamV[kMaxT + 1];  // l = 1..L: [n][C], [n][3][C]
  // adjoint
  float *gzh, *gx, *gxc, *gts, *gtv, *gs[2], *gv[2], *gom, *gw0, *gin, *ggamS, *ggamV;
  float4* gg;                         // [E]: (dE/df_c, dE/du)
  // BF16 path: the tensor-core GEMMs' A operands, rows zero-padded to >= 64 columns
  __nv_bfloat16 *inb, *Xb[kMaxT + 1], *gzhb, *gomb, *gw0b, *gxb;   // [E][KAb], [E][F+2C], [E][Kh], [E][Kc] x2, [E][F]
};

inline int local_kc(const LocalW& w) { return 2 * w.C < 64 ? 64 : 2 * w.C; }   // padded K of 2C-wide gradients

struct Carver {
  float* base;
  int64_t off = 0;
  float* take(int64_t cnt) {
    off = (off + 31) / 32 * 32;
    float* p = base ? base + off : nullptr;
    off += cnt;
    return p;
  }
};

int64_t carve(const LocalW& w, int64_t n, int64_t E, float* base, LocalBufs* b) {
  const int64_t F = w.F, C = w.C, C2 = 2 * w.C, FX = F + C2, Fh = w.F / 2;
  Carver cv{base};
  b->erow = reinterpret_cast<int32_t*>(cv.take(E));
  b->geo = cv.take(E * 8);
  b->in = cv.take(E * w.KA);
  b->z0 = cv.take(E * F);
  b->w0 = cv.take(E * C2);
  for (int l = 0; l <= w.L; ++l) b->X[l] = cv.take(E * FX);
  for (int l = 0; l < w.L; ++l) {
    b->S[l] = cv.take(E * C);
    b->V[l] = cv.take(E * 3 * C);
  }
  for (int l = 1; l <= w.L; ++l) {
    b->OM[l] = cv.take(E * C2);
    b->Z[l] = cv.take(E * F);
    b->gamS[l] = cv.take(n * C);
    b->gamV[l] = cv.take(n * 3 * C);
    if (l < w.L) b->TV[l] = cv.take(E * 3 * C2);
  }
  b->zh = cv.take(E * Fh);
  b->h = cv.take(E * Fh);
  b->gzh = cv.take(E * Fh);
  b->gx = cv.take(E * F);
  b->gxc = cv.take(E * FX);
  b->gts = cv.take(E * C2);
  b->gtv = cv.take(E * 3 * C2);
  for (int q = 0; q < 2; ++q) {
    b->gs[q] = cv.take(E * C);
    b->gv[q] = cv.take(E * 3 * C);
  }
  b->gom = cv.take(E * C2);
  b->gw0 = cv.take(E * C2);
  b->gin = cv.take(E * w.KA);
  b->gg = reinterpret_cast<float4*>(cv.take(E * 4));
  b->ggamS = cv.take(n * C);
  b->ggamV = cv.take(n * 3 * C);
  auto tb = [&](int64_t cnt) { return reinterpret_cast<__nv_bfloat16*>(cv.take((cnt + 1) / 2)); };
  if (w.bf16) {
    const int64_t Kc = local_kc(w);
    b->inb = tb(E * w.KAb);
    for (int l = 0; l <= w.L; ++l) b->Xb[l] = tb(E * FX);
    b->gzhb = tb(E * w.Kh);
    b->gomb = tb(E * Kc);
    b->gw0b = tb(E * Kc);
    b->gxb = tb(E * F);
  } else {
    b->inb = b->gzhb = b->gomb = b->gw0b = b->gxb = nullptr;
    for (int l = 0; l <= w.L; ++l) b->Xb[l] = nullptr;
  }
  return cv.off;
}

// ---------------------------------------------------------------------------- forward kernels
__global__ void k_loc_erow(int64_t n, const int32_t* __restrict__ arow, int32_t* __restrict__ erow) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int32_t e = arow[i]; e < arow[i + 1]; ++e) erow[e] = (int32_t)i;
}

// geo[e] = (d, f_c, f_c', u_x, u_y, u_z, 0, 0); in[e] = [b_k(d) f_c (K) | onehot Z_i | onehot Z_j | 0].
// b_k = exp(-(d - k sigma)^2 / (2 sigma^2)), sigma = rc / (K - 1); f_c = (cos(pi d / rc) + 1) / 2.
// (inb: the same row in BF16, KAb >= KA columns (a multiple of 32), zeros after KA; may be null)
__global__ void k_loc_geom(int64_t E, int K, int S, int KA, float rc, const float4* __restrict__ ar,
                           const int32_t* __restrict__ acol, const int32_t* __restrict__ erow,
                           const int32_t* __restrict__ Z, float* __restrict__ geo, float* __restrict__ in,
                           __nv_bfloat16* __restrict__ inb, int KAb) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  const float4 r = ar[e];
  const float d = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
  const float inv = 1.0f / d;
  const float a = kPiF / rc;
  const float fc = 0.5f * (cosf(a * d) + 1.0f);
  const float dfc = -0.5f * a * sinf(a * d);
  float* g = geo + e * 8;
  g[0] = d; g[1] = fc; g[2] = dfc;
  g[3] = r.x * inv; g[4] = r.y * inv; g[5] = r.z * inv;
  g[6] = 0.0f; g[7] = 0.0f;
  const float sig = rc / (float)(K - 1);
  const float c = 1.0f / (2.0f * sig * sig);
  float* row = in + e * KA;
  for (int k = 0; k < K; ++k) {
    const float t = d - (float)k * sig;
    row[k] = expf(-t * t * c) * fc;
  }
  for (int k = K; k < KA; ++k) row[k] = 0.0f;
  const int zi = Z[erow[e]], zj = Z[acol[e]];
  const bool zi_ok = zi >= 0 && zi < S, zj_ok = zj >= 0 && zj < S;
  if (zi_ok) row[K + zi] = 1.0f;
  if (zj_ok) row[K + S + zj] = 1.0f;
  if (inb) {
    for (int k0 = 0; k0 < KAb; k0 += 8) {
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = k0 + j;
        const float t = d - (float)k * sig;
        v[j] = k < K ? expf(-t * t * c) * fc : (((zi_ok && k == K + zi) || (zj_ok && k == K + S + zj)) ? 1.0f : 0.0f);
      }
      st8_bf16(inb + e * KAb + k0, v);
    }
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// s[e][c] = w0[e][c], v[e][a][c] = w0[e][C+c] u_a
__global__ void k_loc_init(int64_t E, int C, const float* __restrict__ w0, const float* __restrict__ geo,
                           float* __restrict__ S0, float* __restrict__ V0) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= E * C) return;
  const int64_t e = idx / C;
  const int c = (int)(idx % C);
  const float* g = geo + e * 8;
  const float wv = w0[e * 2 * C + C + c];
  S0[e * C + c] = w0[e * 2 * C + c];
  for (int q = 0; q < 3; ++q) V0[(e * 3 + q) * C + c] = wv * g[3 + q];
}

// Gs[i][c] = sum_{e in row i} f_c om[e][c];  Gv[i][a][c] = sum_{e in row i} f_c om[e][C+c] u_a
__global__ void k_loc_env(int64_t n, int C, const int32_t* __restrict__ arow, const float* __restrict__ geo,
                          const float* __restrict__ om, float* __restrict__ gamS, float* __restrict__ gamV) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * C) return;
  const int64_t i = idx / C;
  const int c = (int)(idx % C);
  float gs = 0.0f, gv0 = 0.0f, gv1 = 0.0f, gv2 = 0.0f;
  for (int64_t e = arow[i]; e < arow[i + 1]; ++e) {
    const float* g = geo + e * 8;
    const float fc = g[1];
    gs = fmaf(fc, om[e * 2 * C + c], gs);
    const float t = fc * om[e * 2 * C + C + c];
    gv0 = fmaf(t, g[3], gv0);
    gv1 = fmaf(t, g[4], gv1);
    gv2 = fmaf(t, g[5], gv2);
  }
  gamS[i * C + c] = gs;
  gamV[(i * 3 + 0) * C + c] = gv0;
  gamV[(i * 3 + 1) * C + c] = gv1;
  gamV[(i * 3 + 2) * C + c] = gv2;
}

// ts[e] = [s Gs_i | v . Gv_i] (row stride ld), tv[e][a] = [s Gv_i[a] | v[a] Gs_i] (may be null)
__global__ void k_loc_tp(int64_t E, int C, const int32_t* __restrict__ erow, const float* __restrict__ S,
                         const float* __restrict__ V, const float* __restrict__ gamS, const float* __restrict__ gamV,
                         float* __restrict__ ts, int ld, float* __restrict__ tv, __nv_bfloat16* __restrict__ tsb) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= E * C) return;
  const int64_t e = idx / C;
  const int c = (int)(idx % C);
  const int64_t i = erow[e];
  const float s = S[e * C + c];
  const float v0 = V[(e * 3 + 0) * C + c], v1 = V[(e * 3 + 1) * C + c], v2 = V[(e * 3 + 2) * C + c];
  const float gs = gamS[i * C + c];
  const float g0 = gamV[(i * 3 + 0) * C + c], g1 = gamV[(i * 3 + 1) * C + c], g2 = gamV[(i * 3 + 2) * C + c];
  const float t0 = s * gs, t1 = fmaf(v2, g2, fmaf(v1, g1, v0 * g0));
  ts[e * ld + c] = t0;
  ts[e * ld + C + c] = t1;
  if (tsb) {   // BF16 copy, same row stride
    tsb[e * ld + c] = __float2bfloat16_rn(t0);
    tsb[e * ld + C + c] = __float2bfloat16_rn(t1);
  }
  if (tv) {
    float* t = tv + e * 6 * C;
    t[0 * 2 * C + c] = s * g0;
    t[1 * 2 * C + c] = s * g1;
    t[2 * 2 * C + c] = s * g2;
    t[0 * 2 * C + C + c] = v0 * gs;
    t[1 * 2 * C + C + c] = v1 * gs;
    t[2 * 2 * C + C + c] = v2 * gs;
  }
}

// E_i = e_scale w_i sum_{e in row i} f_c (h_e . R2 + d2); FP64 Neumaier sums per block.
// (H = silu(ZH) as stored, or computed here from ZH when H is null)
__global__ void k_loc_readout(int64_t n, int Fh, float e_scale, const int32_t* __restrict__ arow,
                              const float* __restrict__ geo, const float* __restrict__ H,
                              const float* __restrict__ ZH, const float* __restrict__ R2,
                              const float* __restrict__ d2, const float* __restrict__ ew, float* __restrict__ e_atom,
                              double* __restrict__ partials) {
  __shared__ double sbuf[kThreads / 32];
  double acc = 0.0, comp = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float e = 0.0f;
    for (int64_t q = arow[i]; q < arow[i + 1]; ++q) {
      float y = d2[0];
      for (int k = 0; k < Fh; ++k) y = fmaf(R2[k], H ? H[q * Fh + k] : silu_f(ZH[q * Fh + k]), y);
      e = fmaf(geo[q * 8 + 1], y, e);
    }
    e *= e_scale;
    if (ew) e *= ew[i];
    if (e_atom) e_atom[i] = e;
    const double x = (double)e, t = acc + x;
    comp += fabs(acc) >= fabs(x) ? (acc - t) + x : (x - t) + acc;
    acc = t;
  }
  double v = acc + comp;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sbuf[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += sbuf[w];
    partials[blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------- adjoint kernels
// Seed g = e_scale w_i per edge: dE/df_c = g (h . R2 + d2) starts gg; g_zh = g f_c R2 silu'(zh).
// One warp per edge (lanes over the F/2 columns; h . R2 summed by a shuffle tree).
__global__ void k_loc_readout_bwd(int64_t E, int Fh, float e_scale, const int32_t* __restrict__ erow,
                                  const float* __restrict__ geo, const float* __restrict__ H,
                                  const float* __restrict__ ZH, const float* __restrict__ R2,
                                  const float* __restrict__ d2, const float* __restrict__ ew, float* __restrict__ gzh,
                                  float4* __restrict__ gg, __nv_bfloat16* __restrict__ gzhb, int Kh) {
  const int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= E) return;
  const float g = ew ? e_scale * ew[erow[e]] : e_scale;
  const float fc = geo[e * 8 + 1];
  float y = 0.0f;
  for (int k = lane; k < Fh; k += 32) y = fmaf(R2[k], H ? H[e * Fh + k] : silu_f(ZH[e * Fh + k]), y);
  y = warp_sum(y) + d2[0];
  if (lane == 0) gg[e] = make_float4(g * y, 0.0f, 0.0f, 0.0f);
  const float a = g * fc;
  const int kend = gzhb ? Kh : Fh;
  for (int k = lane; k < kend; k += 32) {
    const float v = k < Fh ? a * R2[k] * dsilu_f(ZH[e * Fh + k]) : 0.0f;
    if (k < Fh) gzh[e * Fh + k] = v;
    if (gzhb) gzhb[e * Kh + k] = __float2bfloat16_rn(v);
  }
}

// dst[e][f] = src[e][f] (row stride lds) * silu'(Z[e][f]); dst may equal src when lds == F;
// dstb (may be null) receives a BF16 copy.  Four features per thread (F and lds multiples of 4).
__global__ void k_loc_mul_dsilu(int64_t E, int F, const float* src, int lds, const float* __restrict__ Z, float* dst,
                                __nv_bfloat16* __restrict__ dstb) {
  const int F4 = F >> 2;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= E * F4) return;
  const int64_t e = idx / F4;
  const int f = 4 * (int)(idx % F4);
  const float4 x = *reinterpret_cast<const float4*>(src + e * lds + f);
  const float4 z = *reinterpret_cast<const float4*>(Z + e * F + f);
  const float4 v = make_float4(x.x * dsilu_f(z.x), x.y * dsilu_f(z.y), x.z * dsilu_f(z.z), x.w * dsilu_f(z.w));
  *reinterpret_cast<float4*>(dst + e * F + f) = v;
  if (dstb) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    *reinterpret_cast<uint2*>(dstb + e * F + f) =
        make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
  }
}

// Edge side of the tensor-product adjoint: g_s = g_ts0 Gs + g_tv0 . Gv, g_v[a] = g_ts1 Gv[a] + g_tv1[a] Gs.
__global__ void k_loc_tp_bwd_edge(int64_t E, int C, const int32_t* __restrict__ erow, const float* __restrict__ gamS,
                                  const float* __restrict__ gamV, const float* __restrict__ gts, int ldg,
                                  const float* __restrict__ gtv, float* __restrict__ GS, float* __restrict__ GV) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= E * C) return;
  const int64_t e = idx / C;
  const int c = (int)(idx % C);
  const int64_t i = erow[e];
  const float a0 = gts[e * ldg + c], a1 = gts[e * ldg + C + c];
  const float gs = gamS[i * C + c];
  const float g0 = gamV[(i * 3 + 0) * C + c], g1 = gamV[(i * 3 + 1) * C + c], g2 = gamV[(i * 3 + 2) * C + c];
  float s = a0 * gs, v0 = a1 * g0, v1 = a1 * g1, v2 = a1 * g2;
  if (gtv) {
    const float* t = gtv + e * 6 * C;
    s = fmaf(t[0 * 2 * C + c], g0, s);
    s = fmaf(t[1 * 2 * C + c], g1, s);
    s = fmaf(t[2 * 2 * C + c], g2, s);
    v0 = fmaf(t[0 * 2 * C + C + c], gs, v0);
    v1 = fmaf(t[1 * 2 * C + C + c], gs, v1);
    v2 = fmaf(t[2 * 2 * C + C + c], gs, v2);
  }
  GS[e * C + c] = s;
  GV[(e * 3 + 0) * C + c] = v0;
  GV[(e * 3 + 1) * C + c] = v1;
  GV[(e * 3 + 2) * C + c] = v2;
}

// Centre side: g_Gs_i = sum_e (g_ts0 s + g_tv1 . v), g_Gv_i[a] = sum_e (g_ts1 v[a] + g_tv0[a] s).
__global__ void k_loc_tp_bwd_atom(int64_t n, int C, const int32_t* __restrict__ arow, const float* __restrict__ S,
                                  const float* __restrict__ V, const float* __restrict__ gts, int ldg,
                                  const float* __restrict__ gtv, float* __restrict__ ggamS, float* __restrict__ ggamV) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * C) return;
  const int64_t i = idx / C;
  const int c = (int)(idx % C);
  float gs = 0.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
  for (int64_t e = arow[i]; e < arow[i + 1]; ++e) {
    const float s = S[e * C + c];
    const float v0 = V[(e * 3 + 0) * C + c], v1 = V[(e * 3 + 1) * C + c], v2 = V[(e * 3 + 2) * C + c];
    const float a0 = gts[e * ldg + c], a1 = gts[e * ldg + C + c];
    gs = fmaf(a0, s, gs);
    g0 = fmaf(a1, v0, g0);
    g1 = fmaf(a1, v1, g1);
    g2 = fmaf(a1, v2, g2);
    if (gtv) {
      const float* t = gtv + e * 6 * C;
      gs = fmaf(t[0 * 2 * C + C + c], v0, gs);
      gs = fmaf(t[1 * 2 * C + C + c], v1, gs);
      gs = fmaf(t[2 * 2 * C + C + c], v2, gs);
      g0 = fmaf(t[0 * 2 * C + c], s, g0);
      g1 = fmaf(t[1 * 2 * C + c], s, g1);
      g2 = fmaf(t[2 * 2 * C + c], s, g2);
    }
  }
  ggamS[i * C + c] = gs;
  ggamV[(i * 3 + 0) * C + c] = g0;
  ggamV[(i * 3 + 1) * C + c] = g1;
  ggamV[(i * 3 + 2) * C + c] = g2;
}

// Environment sums, reversed: g_om[c] = f_c g_Gs[c], g_om[C+c] = f_c (g_Gv[c] . u);
// dE/df_c += om[c] g_Gs[c] + om[C+c] (g_Gv[c] . u);  dE/du += f_c om[C+c] g_Gv[c].
// Four lanes per edge, each over channel quads j, j + 4, ... (16-byte accesses; C a multiple of 4,
// of 16 when gomb is written), the sums over channels by two shuffle steps in a fixed order.
__global__ void k_loc_env_bwd(int64_t E, int C, const int32_t* __restrict__ erow, const float* __restrict__ geo,
                              const float* __restrict__ om, const float* __restrict__ ggamS,
                              const float* __restrict__ ggamV, float* __restrict__ gom, float4* __restrict__ gg,
                              __nv_bfloat16* __restrict__ gomb, int Kc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t e = t >> 2;
  const int j = (int)(t & 3);
  const bool live = e < E;
  const int64_t es = live ? e : 0;
  const int64_t i = erow[es];
  const float* g = geo + es * 8;
  const float fc = g[1], u0 = g[3], u1 = g[4], u2 = g[5];
  float gfc = 0.0f, gu0 = 0.0f, gu1 = 0.0f, gu2 = 0.0f;
  for (int c = 4 * j; live && c < C; c += 16) {
    const float4 gs = ld4f(ggamS + i * C + c);
    const float4 q0 = ld4f(ggamV + (i * 3 + 0) * C + c), q1 = ld4f(ggamV + (i * 3 + 1) * C + c),
                 q2 = ld4f(ggamV + (i * 3 + 2) * C + c);
    const float4 o0 = ld4f(om + es * 2 * C + c), o1 = ld4f(om + es * 2 * C + C + c);
    float4 va, vb;
    auto one = [&](float s_, float a0, float a1, float a2, float p0, float p1, float& ra, float& rb) {
      const float gd = fmaf(a2, u2, fmaf(a1, u1, a0 * u0));
      ra = fc * s_;
      rb = fc * gd;
      gfc = fmaf(p0, s_, fmaf(p1, gd, gfc));
      const float tt = fc * p1;
      gu0 = fmaf(tt, a0, gu0);
      gu1 = fmaf(tt, a1, gu1);
      gu2 = fmaf(tt, a2, gu2);
    };
    one(gs.x, q0.x, q1.x, q2.x, o0.x, o1.x, va.x, vb.x);
    one(gs.y, q0.y, q1.y, q2.y, o0.y, o1.y, va.y, vb.y);
    one(gs.z, q0.z, q1.z, q2.z, o0.z, o1.z, va.z, vb.z);
    one(gs.w, q0.w, q1.w, q2.w, o0.w, o1.w, va.w, vb.w);
    *reinterpret_cast<float4*>(gom + es * 2 * C + c) = va;
    *reinterpret_cast<float4*>(gom + es * 2 * C + C + c) = vb;
    if (gomb) {
      st4_bf16(gomb + es * Kc + c, va);
      st4_bf16(gomb + es * Kc + C + c, vb);
    }
  }
  if (live && gomb)
    for (int k = 2 * C + 4 * j; k < Kc; k += 16) st4_bf16(gomb + es * Kc + k, make_float4(0.f, 0.f, 0.f, 0.f));
  // the four lanes of an edge are consecutive lanes of one warp (t & 3)
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    gfc += __shfl_xor_sync(0xffffffffu, gfc, o);
    gu0 += __shfl_xor_sync(0xffffffffu, gu0, o);
    gu1 += __shfl_xor_sync(0xffffffffu, gu1, o);
    gu2 += __shfl_xor_sync(0xffffffffu, gu2, o);
  }
  if (live && j == 0) {
    float4 a = gg[e];
    a.x += gfc; a.y += gu0; a.z += gu1; a.w += gu2;
    gg[e] = a;
  }
}

// Initial features, reversed: g_w0[c] = g_s[c], g_w0[C+c] = g_v[c] . u;  dE/du += w0[C+c] g_v[c].
// Four lanes per edge over channel quads, as k_loc_env_bwd.
__global__ void k_loc_init_bwd(int64_t E, int C, const float* __restrict__ w0, const float* __restrict__ geo,
                               const float* __restrict__ GS, const float* __restrict__ GV, float* __restrict__ gw0,
                               float4* __restrict__ gg, __nv_bfloat16* __restrict__ gw0b, int Kc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t e = t >> 2;
  const int j = (int)(t & 3);
  const bool live = e < E;
  const int64_t es = live ? e : 0;
  const float* g = geo + es * 8;
  const float u0 = g[3], u1 = g[4], u2 = g[5];
  float gu0 = 0.0f, gu1 = 0.0f, gu2 = 0.0f;
  for (int c = 4 * j; live && c < C; c += 16) {
    const float4 q0 = ld4f(GV + (es * 3 + 0) * C + c), q1 = ld4f(GV + (es * 3 + 1) * C + c),
                 q2 = ld4f(GV + (es * 3 + 2) * C + c);
    const float4 va = ld4f(GS + es * C + c), wv = ld4f(w0 + es * 2 * C + C + c);
    const float4 vb = make_float4(fmaf(q2.x, u2, fmaf(q1.x, u1, q0.x * u0)), fmaf(q2.y, u2, fmaf(q1.y, u1, q0.y * u0)),
                                  fmaf(q2.z, u2, fmaf(q1.z, u1, q0.z * u0)), fmaf(q2.w, u2, fmaf(q1.w, u1, q0.w * u0)));
    *reinterpret_cast<float4*>(gw0 + es * 2 * C + c) = va;
    *reinterpret_cast<float4*>(gw0 + es * 2 * C + C + c) = vb;
    if (gw0b) {
      st4_bf16(gw0b + es * Kc + c, va);
      st4_bf16(gw0b + es * Kc + C + c, vb);
    }
    gu0 = fmaf(wv.w, q0.w, fmaf(wv.z, q0.z, fmaf(wv.y, q0.y, fmaf(wv.x, q0.x, gu0))));
    gu1 = fmaf(wv.w, q1.w, fmaf(wv.z, q1.z, fmaf(wv.y, q1.y, fmaf(wv.x, q1.x, gu1))));
    gu2 = fmaf(wv.w, q2.w, fmaf(wv.z, q2.z, fmaf(wv.y, q2.y, fmaf(wv.x, q2.x, gu2))));
  }
  if (live && gw0b)
    for (int k = 2 * C + 4 * j; k < Kc; k += 16) st4_bf16(gw0b + es * Kc + k, make_float4(0.f, 0.f, 0.f, 0.f));
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    gu0 += __shfl_xor_sync(0xffffffffu, gu0, o);
    gu1 += __shfl_xor_sync(0xffffffffu, gu1, o);
    gu2 += __shfl_xor_sync(0xffffffffu, gu2, o);
  }
  if (live && j == 0) {
    float4 a = gg[e];
    a.y += gu0; a.z += gu1; a.w += gu2;
    gg[e] = a;
  }
}

// Geometry, reversed: dE/dd = sum_k g_in[k] (b_k' f_c + b_k f_c') + (dE/df_c) f_c';
// dE/dr = dE/dd u + (dE/du - (dE/du . u) u) / d;  hedge = -dE/dr.
__global__ void k_loc_geom_bwd(int64_t E, int K, float rc, const float* __restrict__ geo, const float* __restrict__ gin,
                               int KA, const float4* __restrict__ gg, float4* __restrict__ hedge) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  const float* g = geo + e * 8;
  const float d = g[0], fc = g[1], dfc = g[2], u0 = g[3], u1 = g[4], u2 = g[5];
  const float sig = rc / (float)(K - 1);
  const float c = 1.0f / (2.0f * sig * sig);
  float gd = 0.0f;
  for (int k = 0; k < K; ++k) {
    const float t = d - (float)k * sig;
    const float b = expf(-t * t * c);
    const float db = b * (-2.0f * c * t);
    gd = fmaf(gin[e * KA + k], fmaf(db, fc, b * dfc), gd);
  }
  const float4 a = gg[e];
  gd = fmaf(a.x, dfc, gd);
  const float gu = fmaf(a.w, u2, fmaf(a.z, u1, a.y * u0));
  const float inv = 1.0f / d;
  hedge[e] = make_float4(-(gd * u0 + (a.y - gu * u0) * inv), -(gd * u1 + (a.z - gu * u1) * inv),
                         -(gd * u2 + (a.w - gu * u2) * inv), 0.0f);
}

}  // namespace

int64_t local_buffer_floats(const LocalW& w, int64_t n, int64_t E) {
  LocalBufs b;
  return carve(w, n, E, nullptr, &b) + 32;
}

int local_forward_backward(cudaStream_t st, const LocalW& w, int64_t n, int64_t E, const int32_t* species_s,
                            const int32_t* arow, const int32_t* acol, const float4* ar, float* buf,
                            bool need_grad, const float* ew, double* energy_partials, int n_energy_partials,
                            float* e_atom, float4* hedge, int* status) {
  const int F = w.F, C = w.C, C2 = 2 * w.C, FX = w.F + 2 * w.C, Fh = w.F / 2, L = w.L, KA = w.KA;
  const bool bf = w.bf16;   // BF16 path: the dense edge GEMMs on tcgen05 (BF16 operands, FP32 accumulation)
  const int Kc = local_kc(w), Kh = w.Kh, KAb = w.KAb;
  int bad = 0;   // a GEMM shape the tensor-core GEMM rejects (checked on the host)
  LocalBufs b;
  carve(w, n, E, buf, &b);
  StageGuard fwd_stage(STG_EDGE_FWD);   // the whole forward is edge work
  if (E > 0) {
    { LaunchScope ls_(st); k_loc_erow<<<nblocks(n), kThreads, 0, st>>>(n, arow, b.erow); }
    {
      LaunchScope ls_(st);
      k_loc_geom<<<nblocks(E), kThreads, 0, st>>>(E, w.K, w.S, KA, w.rc, ar, acol, b.erow, species_s, b.geo, b.in,
                                                  b.inb, KAb);
    }
    if (bf) {
      bad |= gemm_bf16<1>(st, E, F, KAb, b.inb, KAb, w.wb.A0t, w.c0, nullptr, 0, b.z0, F, b.Xb[0], FX, status);
      bad |= gemm_bf16<0>(st, E, C2, F, b.Xb[0], FX, w.wb.P0t, nullptr, nullptr, 0, b.w0, C2, nullptr, 0, status);
    } else {
      gemm_f32(st, 1, E, F, KA, b.in, KA, w.A0, w.c0, nullptr, 0, b.z0, F, b.X[0], FX);
      gemm_f32(st, 0, E, C2, F, b.X[0], FX, w.P0, nullptr, nullptr, 0, b.w0, C2, nullptr, 0);
    }
    { LaunchScope ls_(st); k_loc_init<<<nblocks(E * C), kThreads, 0, st>>>(E, C, b.w0, b.geo, b.S[0], b.V[0]); }
    for (int l = 1; l <= L; ++l) {
      const LocalLayerW& lw = w.Lw[l - 1];
      if (bf)
        bad |= gemm_bf16<0>(st, E, C2, F, b.Xb[l - 1], FX, w.wb.Qt[l - 1], nullptr, nullptr, 0, b.OM[l], C2, nullptr, 0, status);
      else
        gemm_f32(st, 0, E, C2, F, b.X[l - 1], FX, lw.Q, nullptr, nullptr, 0, b.OM[l], C2, nullptr, 0);
      { LaunchScope ls_(st); k_loc_env<<<nblocks(n * C), kThreads, 0, st>>>(n, C, arow, b.geo, b.OM[l], b.gamS[l], b.gamV[l]); }
      {
        LaunchScope ls_(st);
        k_loc_tp<<<nblocks(E * C), kThreads, 0, st>>>(E, C, b.erow, b.S[l - 1], b.V[l - 1], b.gamS[l], b.gamV[l],
                                                      b.X[l - 1] + F, FX, l < L ? b.TV[l] : nullptr,
                                                      bf ? b.Xb[l - 1] + F : nullptr);
      }
      if (bf)
        bad |= gemm_bf16<1>(st, E, F, FX, b.Xb[l - 1], FX, w.wb.Mt[l - 1], lw.m, nullptr, 0, b.Z[l], F, b.Xb[l], FX, status);
      else
        gemm_f32(st, 1, E, F, FX, b.X[l - 1], FX, lw.M, lw.m, nullptr, 0, b.Z[l], F, b.X[l], FX);
      if (l < L) {   // the 2C -> C channel mixings stay on the SIMT GEMM (N = C below a tensor-core tile)
        gemm_f32(st, 0, E, C, C2, b.X[l - 1] + F, FX, lw.Gs, nullptr, nullptr, 0, b.S[l], C, nullptr, 0);
        gemm_f32(st, 0, 3 * E, C, C2, b.TV[l], C2, lw.Gv, nullptr, nullptr, 0, b.V[l], C, nullptr, 0);
      }
    }
    if (bf)   // zh only; the readout applies silu itself
      bad |= gemm_bf16<0>(st, E, Fh, F, b.Xb[L], FX, w.wb.R1t, w.d1, nullptr, 0, b.zh, Fh, nullptr, 0, status);
    else
      gemm_f32(st, 1, E, Fh, F, b.X[L], FX, w.R1, w.d1, nullptr, 0, b.zh, Fh, b.h, Fh);
  }
  const float* H = bf ? nullptr : b.h;
  {
    LaunchScope ls_(st);
    k_loc_readout<<<n_energy_partials, kThreads, 0, st>>>(n, Fh, w.e_scale, arow, b.geo, H, b.zh, w.R2, w.d2, ew,
                                                          e_atom, energy_partials);
  }
  if (!need_grad || E == 0) return bad;
  StageGuard bwd_stage(STG_EDGE_BWD);
  {
    LaunchScope ls_(st);
    k_loc_readout_bwd<<<nblocks(E * 32), kThreads, 0, st>>>(E, Fh, w.e_scale, b.erow, b.geo, H, b.zh, w.R2, w.d2, ew,
                                                       b.gzh, b.gg, b.gzhb, Kh);
  }
  // g_z of layer L
  if (bf)
    bad |= gemm_bf16<3>(st, E, F, Kh, b.gzhb, Kh, w.wb.R1, nullptr, b.Z[L], F, b.gx, F, b.gxb, F, status);
  else
    gemm_f32(st, 3, E, F, Fh, b.gzh, Fh, w.R1t, nullptr, b.Z[L], F, b.gx, F, nullptr, 0);
  float *gs_in = b.gs[0], *gv_in = b.gv[0], *gs_out = b.gs[1], *gv_out = b.gv[1];
  for (int l = L; l >= 1; --l) {
    const LocalLayerW& lw = w.Lw[l - 1];
    // [g_x^{l-1} | g_ts] = g_z M_l^T
    if (bf)
      bad |= gemm_bf16<0>(st, E, FX, F, b.gxb, F, w.wb.M[l - 1], nullptr, nullptr, 0, b.gxc, FX, nullptr, 0, status);
    else
      gemm_f32(st, 0, E, FX, F, b.gx, F, lw.Mt, nullptr, nullptr, 0, b.gxc, FX, nullptr, 0);
    const float* gts = b.gxc + F;
    int ldg = FX;
    const float* gtv = nullptr;
    if (l < L) {   // the channel mixings of layer l feed layer l+1
      gemm_f32(st, 2, E, C2, C, gs_in, C, lw.Gst, nullptr, b.gxc + F, FX, b.gts, C2, nullptr, 0);
      gts = b.gts;
      ldg = C2;
      gemm_f32(st, 0, 3 * E, C2, C, gv_in, C, lw.Gvt, nullptr, nullptr, 0, b.gtv, C2, nullptr, 0);
      gtv = b.gtv;
    }
    {
      LaunchScope ls_(st);
      k_loc_tp_bwd_edge<<<nblocks(E * C), kThreads, 0, st>>>(E, C, b.erow, b.gamS[l], b.gamV[l], gts, ldg, gtv, gs_out,
                                                             gv_out);
    }
    {
      LaunchScope ls_(st);
      k_loc_tp_bwd_atom<<<nblocks(n * C), kThreads, 0, st>>>(n, C, arow, b.S[l - 1], b.V[l - 1], gts, ldg, gtv, b.ggamS,
                                                             b.ggamV);
    }
    {
      LaunchScope ls_(st);
      k_loc_env_bwd<<<nblocks(E * 4), kThreads, 0, st>>>(E, C, b.erow, b.geo, b.OM[l], b.ggamS, b.ggamV, b.gom, b.gg,
                                                     b.gomb, Kc);
    }
    // g_x^{l-1} = g_xc[:, 0:F] + g_om Q_l^T
    if (bf)
      bad |= gemm_bf16<2>(st, E, F, Kc, b.gomb, Kc, w.wb.Q[l - 1], nullptr, b.gxc, FX, b.gx, F, nullptr, 0, status);
    else
      gemm_f32(st, 2, E, F, C2, b.gom, C2, lw.Qt, nullptr, b.gxc, FX, b.gx, F, nullptr, 0);
    if (l > 1) {
      LaunchScope ls_(st);
      k_loc_mul_dsilu<<<nblocks(E * F / 4), kThreads, 0, st>>>(E, F, b.gx, F, b.Z[l - 1], b.gx, b.gxb);
    }
    std::swap(gs_in, gs_out);
    std::swap(gv_in, gv_out);
  }
  // gs_in, gv_in: gradients of the initial edge features
  { LaunchScope ls_(st); k_loc_init_bwd<<<nblocks(E * 4), kThreads, 0, st>>>(E, C, b.w0, b.geo, gs_in, gv_in, b.gw0, b.gg, b.gw0b, Kc); }
  if (bf)   // g_x0
    bad |= gemm_bf16<2>(st, E, F, Kc, b.gw0b, Kc, w.wb.P0, nullptr, b.gx, F, b.gxc, FX, nullptr, 0, status);
  else
    gemm_f32(st, 2, E, F, C2, b.gw0, C2, w.P0t, nullptr, b.gx, F, b.gxc, FX, nullptr, 0);
  { LaunchScope ls_(st); k_loc_mul_dsilu<<<nblocks(E * F / 4), kThreads, 0, st>>>(E, F, b.gxc, FX, b.z0, b.gx, b.gxb); }
  if (bf)
    bad |= gemm_bf16<0>(st, E, KA, F, b.gxb, F, w.wb.A0, nullptr, nullptr, 0, b.gin, KA, nullptr, 0, status);
  else
    gemm_f32(st, 0, E, KA, F, b.gx, F, w.A0t, nullptr, nullptr, 0, b.gin, KA, nullptr, 0);
  { LaunchScope ls_(st); k_loc_geom_bwd<<<nblocks(E), kThreads, 0, st>>>(E, w.K, w.rc, b.geo, b.gin, KA, b.gg, hedge); }
  return bad;
}

}  // namespace ctd
