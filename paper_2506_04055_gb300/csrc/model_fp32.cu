// model_fp32.cu -- PaiNN-form energy and its hand-written adjoint, all products in FP32 on
// CUDA cores (the FP32 reference precision of the engine).
//
// The potential is a sum of per-atom energies over a cutoff graph (arXiv 2506.04055, Methods,
// semi-local energy equation) computed by T message-passing layers (Methods, "Graph Neural
// Networks", message and update equations), instantiated as PaiNN (Methods, "Chosen
// Architectures"); forces are the negative gradient (Results, "Distributed potential
// computation", sum-rule equation).  Layer, with edge e = (i <- j), r_e = x_j - x_i + shift:
//   phi_j  = W2 silu(W1 s_j + b1) + b2                       = [phi_s | phi_vv | phi_vs]
//   W_e    = (Wf rbf(d_e) + bf) f_c(d_e)                      = [W_s | W_vv | W_vs]
//   s_i   += sum_e phi_s,j W_s,e
//   v_i   += sum_e (v_j phi_vv,j W_vv,e + u_e phi_vs,j W_vs,e)
//   Uv, Vv = U v, V v;  a = A2 silu(A1 [s ; sqrt(|Vv|^2 + eps)] + c1) + c2 = [a_vv | a_sv | a_ss]
//   v     += a_vv Uv;  s += a_ss + a_sv <Uv, Vv>
//   U_i    = e_scale (R2 . silu(R1 s_i + d1) + d2)
//
// GB300 layout: atoms are cell-sorted so neighbour gathers hit L2; per atom the gathered
// message table is PHI = [phi_s | psi_0 | psi_1 | psi_2 | phi_vs | phi_vv] with
// psi_a = v_a * phi_vv pre-multiplied once per atom (5F gathered floats per edge instead of 6F).
// Edge kernels run one group of F threads per receiver row (thread = feature channel), so the
// segmented sum over a receiver's CSR row stays in registers: no atomics.  The adjoint of the
// message step runs sender-side: the row of atom j visits every edge whose sender is j (the
// list holds both directions and the filter depends only on |r|), gathering the receivers'
// gradients; per-edge position gradients go to hedge[e] and the forces are assembled from
// hedge and the reverse-edge index, again without atomics.
#include "ctd_internal.cuh"
#include "../../include/painn.h"

namespace ctd {

// ================================================================================ SIMT GEMM
// out[m][n] = sum_k A[m][k] B[k][n], A [M][K] (lda), B [K][N] row-major; BM x BN tile
// (64 x 128, or 128 x 64 / 256 x 32 for narrow outputs), 256 threads, each 8 rows x 4 columns,
// K staged 32 at a time (A transposed in smem).  Every output is the same fmaf chain over k in
// increasing order whatever the tile, so the tile shapes give bit-identical results.
enum Epi { EPI_BIAS = 0, EPI_BIAS_SILU = 1, EPI_ADD = 2, EPI_DSILU = 3 };
constexpr int GBM = 64, GBN = 128, GBK = 32;

template <int EPI, int BN = GBN>
__global__ __launch_bounds__(256) void k_gemm(int64_t M, int N, int K, const float* __restrict__ A, int lda,
                                              const float* __restrict__ B, const float* __restrict__ bias,
                                              const float* aux, int ldaux, float* out, int ldo,
                                              float* __restrict__ out2, int ldo2) {
  constexpr int TX = BN / 4;          // column groups of 4
  constexpr int BM = 8 * (256 / TX);  // row groups of 8
  static_assert(BN == 32 || BN == 64 || BN == 128, "tile width");
  __shared__ __align__(16) float AsT[GBK][BM + 4];
  __shared__ __align__(16) float Bs[GBK][BN];
  const int tid = threadIdx.x, ty = tid / TX, tx = tid % TX;
  // 1-D grid, column tile fastest: consecutive blocks share their A rows (L2 reuse), and the row
  // tile count is not limited to the 65,535 of a grid's y dimension (M = 3n rows exceed it
  // beyond 1.4M atoms)
  const int ncol = (N + BN - 1) / BN;
  const int64_t m0 = (int64_t)(blockIdx.x / ncol) * BM;
  const int n0 = (int)(blockIdx.x % ncol) * BN;
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;

  for (int k0 = 0; k0 < K; k0 += GBK) {
    // A tile: BM rows x 32 k, BM/32 float4 per thread, stored transposed
#pragma unroll
    for (int q = 0; q < BM / 32; ++q) {
      int idx = tid + q * 256;
      int r = idx >> 3, c4 = (idx & 7) * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m0 + r < M && k0 + c4 < K) v = *reinterpret_cast<const float4*>(&A[(m0 + r) * lda + k0 + c4]);
      AsT[c4 + 0][r] = v.x;
      AsT[c4 + 1][r] = v.y;
      AsT[c4 + 2][r] = v.z;
      AsT[c4 + 3][r] = v.w;
    }
    // B tile: 32 k x BN n, BN/32 float4 per thread
#pragma unroll
    for (int q = 0; q < BN / 32; ++q) {
      int idx = tid + q * 256;
      int r = idx / TX, c4 = (idx % TX) * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k0 + r < K && n0 + c4 < N) v = *reinterpret_cast<const float4*>(&B[(int64_t)(k0 + r) * N + n0 + c4]);
      *reinterpret_cast<float4*>(&Bs[r][c4]) = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < GBK; ++k) {
      float4 a0 = *reinterpret_cast<const float4*>(&AsT[k][ty * 8]);
      float4 a1 = *reinterpret_cast<const float4*>(&AsT[k][ty * 8 + 4]);
      float4 b = *reinterpret_cast<const float4*>(&Bs[k][tx * 4]);
      float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  const int nb = n0 + tx * 4;
  if (nb >= N) return;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int64_t m = m0 + ty * 8 + i;
    if (m >= M) break;
    float r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float x = acc[i][j];
      if (EPI == EPI_BIAS || EPI == EPI_BIAS_SILU) x += bias ? bias[nb + j] : 0.0f;
      if (EPI == EPI_ADD) x += aux[m * ldaux + nb + j];
      if (EPI == EPI_DSILU) x *= dsilu_f(aux[m * ldaux + nb + j]);
      r[j] = x;
    }
    *reinterpret_cast<float4*>(&out[m * ldo + nb]) = make_float4(r[0], r[1], r[2], r[3]);
    if (EPI == EPI_BIAS_SILU)
      *reinterpret_cast<float4*>(&out2[m * ldo2 + nb]) =
          make_float4(silu_f(r[0]), silu_f(r[1]), silu_f(r[2]), silu_f(r[3]));
  }
}

// Small problems (fewer output tiles than one wave of the GPU): one thread per output element,
// the same fmaf chain over k in increasing order and the same epilogue as k_gemm, so results
// are bit for bit those of the tiled kernel, with more warps in flight than its few CTAs.
template <int EPI>
__global__ void k_gemm_small(int64_t M, int N, int K, const float* __restrict__ A, int lda,
                             const float* __restrict__ B, const float* __restrict__ bias,
                             const float* __restrict__ aux, int ldaux, float* __restrict__ out, int ldo,
                             float* __restrict__ out2, int ldo2) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  const int64_t m = idx / N;
  const int n = (int)(idx % N);
  const float* a = A + m * lda;
  float x = 0.0f;
  for (int k = 0; k < K; ++k) x = fmaf(__ldg(a + k), __ldg(B + (int64_t)k * N + n), x);
  if (EPI == EPI_BIAS || EPI == EPI_BIAS_SILU) x += bias ? bias[n] : 0.0f;
  if (EPI == EPI_ADD) x += aux[m * ldaux + n];
  if (EPI == EPI_DSILU) x *= dsilu_f(aux[m * ldaux + n]);
  out[m * ldo + n] = x;
  if (EPI == EPI_BIAS_SILU) out2[m * ldo2 + n] = silu_f(x);
}

template <int EPI, int BN = GBN>
static void gemm(cudaStream_t st, int64_t M, int N, int K, const float* A, int lda, const float* B,
                 const float* bias, const float* aux, int ldaux, float* out, int ldo, float* out2 = nullptr,
                 int ldo2 = 0) {
  if (M == 0) return;
  constexpr int BM = 8 * (256 / (BN / 4));
  const int64_t tiles = (int64_t)((N + BN - 1) / BN) * ((M + BM - 1) / BM);
  if (tiles < 152) {
    LaunchScope ls_(st);
    k_gemm_small<EPI><<<(unsigned)((M * N + 255) / 256), 256, 0, st>>>(M, N, K, A, lda, B, bias, aux, ldaux, out,
                                                                     ldo, out2, ldo2);
    return;
  }
  { LaunchScope ls_(st); k_gemm<EPI, BN><<<(unsigned)tiles, 256, 0, st>>>(M, N, K, A, lda, B, bias, aux, ldaux, out, ldo, out2, ldo2); }
}

// The tile width follows N (32, 64 or 128 columns), so narrow outputs do not compute idle
// columns; the results are those of the 128-column tile, bit for bit.
template <int BN>
static void gemm_epi(cudaStream_t st, int epi, int64_t M, int N, int K, const float* A, int lda, const float* B,
                     const float* bias, const float* aux, int ldaux, float* out, int ldo, float* out2, int ldo2) {
  switch (epi) {
    case EPI_BIAS: gemm<EPI_BIAS, BN>(st, M, N, K, A, lda, B, bias, aux, ldaux, out, ldo, out2, ldo2); break;
    case EPI_BIAS_SILU: gemm<EPI_BIAS_SILU, BN>(st, M, N, K, A, lda, B, bias, aux, ldaux, out, ldo, out2, ldo2); break;
    case EPI_ADD: gemm<EPI_ADD, BN>(st, M, N, K, A, lda, B, bias, aux, ldaux, out, ldo, out2, ldo2); break;
    default: gemm<EPI_DSILU, BN>(st, M, N, K, A, lda, B, bias, aux, ldaux, out, ldo, out2, ldo2); break;
  }
}
void gemm_f32(cudaStream_t st, int epi, int64_t M, int N, int K, const float* A, int lda, const float* B,
              const float* bias, const float* aux, int ldaux, float* out, int ldo, float* out2, int ldo2) {
  if (N <= 32) gemm_epi<32>(st, epi, M, N, K, A, lda, B, bias, aux, ldaux, out, ldo, out2, ldo2);
  else if (N <= 64) gemm_epi<64>(st, epi, M, N, K, A, lda, B, bias, aux, ldaux, out, ldo, out2, ldo2);
  else gemm_epi<128>(st, epi, M, N, K, A, lda, B, bias, aux, ldaux, out, ldo, out2, ldo2);
}

// ================================================================================ node kernels
__global__ void k_embed(int64_t n, int F, const int32_t* __restrict__ Z, const float* __restrict__ emb,
                        float* __restrict__ S, float* __restrict__ V, __nv_bfloat16* __restrict__ Sb) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * F) return;
  int64_t i = idx / F;
  int f = (int)(idx % F);
  S[idx] = emb[(int64_t)Z[i] * F + f];
  if (Sb) Sb[idx] = __float2bfloat16_rn(S[idx]);
  if (V) {   // null where the first layer's kernels take v = 0 without reading it
    V[i * 3 * F + f] = 0.0f;
    V[i * 3 * F + F + f] = 0.0f;
    V[i * 3 * F + 2 * F + f] = 0.0f;
  }
}

// PHI[i] = [phi_s | v_0 phi_vv | v_1 phi_vv | v_2 phi_vv | phi_vs | phi_vv]
__global__ void k_phi_pack(int64_t n, int F, const float* __restrict__ P3, const float* __restrict__ V,
                           float* __restrict__ PHI) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * F) return;
  int64_t i = idx / F;
  int f = (int)(idx % F);
  const float* p = P3 + i * 3 * F;
  const float* v = V + i * 3 * F;
  float* o = PHI + i * 6 * F;
  float pvv = p[F + f];
  o[f] = p[f];
  o[F + f] = v[f] * pvv;
  o[2 * F + f] = v[F + f] * pvv;
  o[3 * F + f] = v[2 * F + f] * pvv;
  o[4 * F + f] = p[2 * F + f];
  o[5 * F + f] = pvv;
}

// U/V products and update coefficients are read as FP32 (FP32 path) or from their FP16 copies
// (BF16 path)
__device__ __forceinline__ float ldx(const float* p) { return *p; }
__device__ __forceinline__ float ldx(const __half* p) { return __half2float(*p); }

// Four consecutive features per thread (F is a multiple of 4): 16-byte FP32 and 8-byte FP16 or
// BF16 accesses instead of one scalar per thread.
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 ld4(const __half* p) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ void st4(__nv_bfloat16* p, float4 v) {
  const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
  *reinterpret_cast<uint2*>(p) = make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
}

// Z = [s^m ; sqrt(sum_a Vv_a^2 + eps)], UV rows (i, a) = [Uv_a | Vv_a]; thread = 4 features
template <typename TX>
__global__ void k_update_pre(int64_t n, int F, float eps, const float* __restrict__ SM,
                             const TX* __restrict__ UV, float* __restrict__ Z, __nv_bfloat16* __restrict__ Zb) {
  const int F4 = F >> 2;
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * F4) return;
  const int64_t i = idx / F4;
  const int f = 4 * (int)(idx % F4);
  const TX* uv = UV + i * 3 * 2 * F;
  const float4 v0 = ld4(uv + F + f), v1 = ld4(uv + 3 * F + f), v2 = ld4(uv + 5 * F + f);
  const float4 sm = ld4(SM + i * F + f);
  const float4 nv = make_float4(sqrtf(v0.x * v0.x + v1.x * v1.x + v2.x * v2.x + eps),
                                sqrtf(v0.y * v0.y + v1.y * v1.y + v2.y * v2.y + eps),
                                sqrtf(v0.z * v0.z + v1.z * v1.z + v2.z * v2.z + eps),
                                sqrtf(v0.w * v0.w + v1.w * v1.w + v2.w * v2.w + eps));
  if (Z) {
    st4(Z + i * 2 * F + f, sm);
    st4(Z + i * 2 * F + F + f, nv);
  }
  if (Zb) {
    st4(Zb + i * 2 * F + f, sm);
    st4(Zb + i * 2 * F + F + f, nv);
  }
}

// s' = s^m + a_ss + a_sv <Uv, Vv>,  v'_a = v^m_a + a_vv Uv_a; WV false: s' only (the last
// layer's v and BF16 s reach neither the readout nor the backward).  Thread = 4 features.
template <typename TX, bool WV>
__global__ void k_update_post(int64_t n, int F, const float* __restrict__ SM, const float* __restrict__ VM,
                              const TX* __restrict__ UV, const TX* __restrict__ AV,
                              float* __restrict__ Sn, float* __restrict__ Vn, __nv_bfloat16* __restrict__ Snb) {
  const int F4 = F >> 2;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * F4) return;
  const int64_t i = idx / F4;
  const int f = 4 * (int)(idx % F4);
  const TX* uv = UV + i * 6 * F;
  const TX* a = AV + i * 3 * F;
  float4 sp = make_float4(0.f, 0.f, 0.f, 0.f), u[3];
#pragma unroll
  for (int al = 0; al < 3; ++al) {
    u[al] = ld4(uv + al * 2 * F + f);
    const float4 v = ld4(uv + al * 2 * F + F + f);
    sp.x += u[al].x * v.x; sp.y += u[al].y * v.y; sp.z += u[al].z * v.z; sp.w += u[al].w * v.w;
  }
  if (WV) {
    const float4 avv = ld4(a + f);
#pragma unroll
    for (int al = 0; al < 3; ++al) {
      const float4 vm = ld4(VM + i * 3 * F + al * F + f);
      st4(Vn + i * 3 * F + al * F + f, make_float4(vm.x + avv.x * u[al].x, vm.y + avv.y * u[al].y,
                                                   vm.z + avv.z * u[al].z, vm.w + avv.w * u[al].w));
    }
  }
  const float4 sm = ld4(SM + i * F + f), ass = ld4(a + 2 * F + f), asv = ld4(a + F + f);
  const float4 sn = make_float4(sm.x + ass.x + asv.x * sp.x, sm.y + ass.y + asv.y * sp.y,
                                sm.z + ass.z + asv.z * sp.z, sm.w + ass.w + asv.w * sp.w);
  st4(Sn + i * F + f, sn);
  if (Snb) st4(Snb + i * F + f, sn);
}

// Backward of the update elementwise part: given gs' (GS), gv' (GV):
//   g_a = [sum_a gv'_a Uv_a | gs' <Uv,Vv> | gs'],  gUv_a = gv'_a a_vv + gs' a_sv Vv_a,
//   gVv_a = gs' a_sv Uv_a (the |Vv| term is added after the A1 backward)
__global__ void k_update_bwd_pre(int64_t n, int F, const float* __restrict__ GS, const float* __restrict__ GV,
                                 const float* __restrict__ UV, const float* __restrict__ AV,
                                 float* __restrict__ GA, float* __restrict__ GUV, __nv_bfloat16* __restrict__ GAb) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * F) return;
  int64_t i = idx / F;
  int f = (int)(idx % F);
  const float* uv = UV + i * 6 * F;
  const float* a = AV + i * 3 * F;
  float gs = GS[idx], asv = a[F + f], avv = a[f];
  float gsp = gs * asv, sp = 0.0f, gavv = 0.0f;
#pragma unroll
  for (int al = 0; al < 3; ++al) {
    float u = uv[al * 2 * F + f], v = uv[al * 2 * F + F + f];
    float gv = GV[i * 3 * F + al * F + f];
    sp += u * v;
    gavv += gv * u;
    GUV[i * 6 * F + al * 2 * F + f] = gv * avv + gsp * v;
    GUV[i * 6 * F + al * 2 * F + F + f] = gsp * u;
  }
  if (GA) {
    GA[i * 3 * F + f] = gavv;
    GA[i * 3 * F + F + f] = gs * sp;
    GA[i * 3 * F + 2 * F + f] = gs;
  }
  if (GAb) {
    GAb[i * 3 * F + f] = __float2bfloat16_rn(gavv);
    GAb[i * 3 * F + F + f] = __float2bfloat16_rn(gs * sp);
    GAb[i * 3 * F + 2 * F + f] = __float2bfloat16_rn(gs);
  }
}

// gz = [gz_s | gz_n] (grad of [s^m ; |Vv|]):  gsm = gs' + gz_s;  gVv_a += gz_n Vv_a / |Vv|
__global__ void k_update_bwd_mid(int64_t n, int F, float eps, const float* __restrict__ GS,
                                 const float* __restrict__ GZ, const float* __restrict__ UV,
                                 float* __restrict__ Gsm, float* __restrict__ GUV, __nv_bfloat16* __restrict__ GUVb) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * F) return;
  int64_t i = idx / F;
  int f = (int)(idx % F);
  const float* uv = UV + i * 6 * F;
  float v0 = uv[F + f], v1 = uv[3 * F + f], v2 = uv[5 * F + f];
  float nv = sqrtf(v0 * v0 + v1 * v1 + v2 * v2 + eps);
  float g = GZ[i * 2 * F + F + f] / nv;
  Gsm[idx] = GS[idx] + GZ[i * 2 * F + f];
  GUV[i * 6 * F + F + f] += g * v0;
  GUV[i * 6 * F + 3 * F + f] += g * v1;
  GUV[i * 6 * F + 5 * F + f] += g * v2;
  if (GUVb) {
#pragma unroll
    for (int q = 0; q < 6; ++q) GUVb[i * 6 * F + q * F + f] = __float2bfloat16_rn(GUV[i * 6 * F + q * F + f]);
  }
}

// BF16 path: the same two steps writing the BF16 operand of the U/V backward GEMM directly.
//   pre: g_a (BF16) and the Uv half of each GUV row, gUv_a = gv'_a a_vv + gs' a_sv Vv_a;
//   mid: gsm = gs' + gz_s and the Vv half, gVv_a = gs' a_sv Uv_a + gz_n Vv_a / |Vv|.
__global__ void k_update_bwd_pre_bf16(int64_t n, int F, const float* __restrict__ GS, const float* __restrict__ GV,
                                      const __half* __restrict__ UV, const __half* __restrict__ AV,
                                      __nv_bfloat16* __restrict__ GAb, __nv_bfloat16* __restrict__ GUVb) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * F) return;
  int64_t i = idx / F;
  int f = (int)(idx % F);
  const __half* uv = UV + i * 6 * F;
  const __half* a = AV + i * 3 * F;
  const float gs = GS[idx], asv = ldx(a + F + f), avv = ldx(a + f);
  const float gsp = gs * asv;
  float sp = 0.0f, gavv = 0.0f;
#pragma unroll
  for (int al = 0; al < 3; ++al) {
    const float u = ldx(uv + al * 2 * F + f), v = ldx(uv + al * 2 * F + F + f);
    const float gv = GV[i * 3 * F + al * F + f];
    sp += u * v;
    gavv += gv * u;
    GUVb[i * 6 * F + al * 2 * F + f] = __float2bfloat16_rn(gv * avv + gsp * v);
  }
  GAb[i * 3 * F + f] = __float2bfloat16_rn(gavv);
  GAb[i * 3 * F + F + f] = __float2bfloat16_rn(gs * sp);
  GAb[i * 3 * F + 2 * F + f] = __float2bfloat16_rn(gs);
}

__global__ void k_update_bwd_mid_bf16(int64_t n, int F, float eps, const float* __restrict__ GS,
                                      const float* __restrict__ GZ, const __half* __restrict__ UV,
                                      const __half* __restrict__ AV, float* __restrict__ Gsm,
                                      __nv_bfloat16* __restrict__ GUVb) {
  const int F4 = F >> 2;   // thread = 4 features
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * F4) return;
  const int64_t i = idx / F4;
  const int f = 4 * (int)(idx % F4);
  const __half* uv = UV + i * 6 * F;
  const float4 v0 = ld4(uv + F + f), v1 = ld4(uv + 3 * F + f), v2 = ld4(uv + 5 * F + f);
  const float4 u0 = ld4(uv + f), u1 = ld4(uv + 2 * F + f), u2 = ld4(uv + 4 * F + f);
  const float4 gzs = ld4(GZ + i * 2 * F + f), gzn = ld4(GZ + i * 2 * F + F + f);
  const float4 gs = ld4(GS + i * F + f), asv = ld4(AV + i * 3 * F + F + f);
  float4 o0, o1, o2;
  auto one = [&](float x0, float x1, float x2, float y0, float y1, float y2, float gn, float g_s, float a_sv,
                 float& r0, float& r1, float& r2) {
    const float nv = sqrtf(x0 * x0 + x1 * x1 + x2 * x2 + eps);
    const float g = gn / nv, gsp = g_s * a_sv;
    r0 = gsp * y0 + g * x0;
    r1 = gsp * y1 + g * x1;
    r2 = gsp * y2 + g * x2;
  };
  one(v0.x, v1.x, v2.x, u0.x, u1.x, u2.x, gzn.x, gs.x, asv.x, o0.x, o1.x, o2.x);
  one(v0.y, v1.y, v2.y, u0.y, u1.y, u2.y, gzn.y, gs.y, asv.y, o0.y, o1.y, o2.y);
  one(v0.z, v1.z, v2.z, u0.z, u1.z, u2.z, gzn.z, gs.z, asv.z, o0.z, o1.z, o2.z);
  one(v0.w, v1.w, v2.w, u0.w, u1.w, u2.w, gzn.w, gs.w, asv.w, o0.w, o1.w, o2.w);
  st4(Gsm + i * F + f, make_float4(gs.x + gzs.x, gs.y + gzs.y, gs.z + gzs.z, gs.w + gzs.w));
  st4(GUVb + i * 6 * F + F + f, o0);
  st4(GUVb + i * 6 * F + 3 * F + f, o1);
  st4(GUVb + i * 6 * F + 5 * F + f, o2);
}

// Backward of PHI packing: gphi_vv = sum_a gpsi_a v_a, gv_a = gvm_a + gpsi_a phi_vv;
// GP3 = [gphi_s | gphi_vv | gphi_vs]
// (phi_vv from the FP32 table PHI, or from its FP16 copy PHIh when PHI is null)
__global__ void k_phi_bwd_pre(int64_t n, int F, const float* __restrict__ GPHI, const float* __restrict__ PHI,
                              const __half* __restrict__ PHIh, const float* __restrict__ V,
                              const float* __restrict__ Gvm, float* __restrict__ GP3, float* __restrict__ GVn,
                              __nv_bfloat16* __restrict__ GP3b) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * F) return;
  int64_t i = idx / F;
  int f = (int)(idx % F);
  const float* g = GPHI + i * 5 * F;
  const float pvv = PHI ? PHI[i * 6 * F + 5 * F + f] : __half2float(PHIh[i * 6 * F + 5 * F + f]);
  float gpvv = 0.0f;
#pragma unroll
  for (int al = 0; al < 3; ++al) {
    float gpsi = g[(1 + al) * F + f];
    gpvv += gpsi * V[i * 3 * F + al * F + f];
    GVn[i * 3 * F + al * F + f] = Gvm[i * 3 * F + al * F + f] + gpsi * pvv;
  }
  if (GP3) {
    GP3[i * 3 * F + f] = g[f];
    GP3[i * 3 * F + F + f] = gpvv;
    GP3[i * 3 * F + 2 * F + f] = g[4 * F + f];
  }
  if (GP3b) {
    GP3b[i * 3 * F + f] = __float2bfloat16_rn(g[f]);
    GP3b[i * 3 * F + F + f] = __float2bfloat16_rn(gpvv);
    GP3b[i * 3 * F + 2 * F + f] = __float2bfloat16_rn(g[4 * F + f]);
  }
}

// The same backward after the tensor-core adjoint, which wrote the psi gradients GPSI ([n][3F],
// FP32) and blocks 0 and 2 of GP3b itself: block 1 gets gphi_vv = sum_a gpsi_a v_a, and
// gv_a = gvm_a + gpsi_a phi_vv, gvm read from the interleaved G4 = (gsm, gvm_0..2) per feature.
// Thread = 4 features.
__global__ void k_phi_bwd_psi(int64_t n, int F, const float* __restrict__ GPSI, const float* __restrict__ PHI,
                              const __half* __restrict__ PHIh, const float* __restrict__ V,
                              const float4* __restrict__ G4, float* __restrict__ GVn,
                              __nv_bfloat16* __restrict__ GP3b) {
  const int F4 = F >> 2;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * F4) return;
  const int64_t i = idx / F4;
  const int f = 4 * (int)(idx % F4);
  const float4 pvv = PHI ? ld4(PHI + i * 6 * F + 5 * F + f) : ld4(PHIh + i * 6 * F + 5 * F + f);
  const float4* q = G4 + i * F + f;
  const float4 q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
  float4 gpvv = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int al = 0; al < 3; ++al) {
    const int64_t o = i * 3 * F + al * F + f;
    const float4 g = ld4(GPSI + o), v = ld4(V + o);
    const float4 gm = al == 0 ? make_float4(q0.y, q1.y, q2.y, q3.y)
                    : al == 1 ? make_float4(q0.z, q1.z, q2.z, q3.z) : make_float4(q0.w, q1.w, q2.w, q3.w);
    gpvv.x += g.x * v.x; gpvv.y += g.y * v.y; gpvv.z += g.z * v.z; gpvv.w += g.w * v.w;
    st4(GVn + o, make_float4(gm.x + g.x * pvv.x, gm.y + g.y * pvv.y, gm.z + g.z * pvv.z, gm.w + g.w * pvv.w));
  }
  st4(GP3b + i * 3 * F + F + f, gpvv);
}

// ================================================================================ edge kernels
__device__ __forceinline__ void group_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Forward message: one group of F threads per receiver row.  Edges of the row are staged
// F at a time (geometry, f_c, radial basis) in shared memory; thread f then accumulates
// channel f of s and of the three components of v over the staged edges.
//
// STORE: the kernel also writes, per edge e and channel c in (s, vv, vs), the cutoff-scaled
// filter W_c,e = f_c (Wf rbf + bf) and its distance derivative dW_c,e/dd, as
// wst[e][6F] = [W_s | W_vv | W_vs | dW_s | dW_vv | dW_vs], so that the adjoint reads them
// instead of recomputing the basis and the filter.
template <int KP, bool STORE>
__global__ __launch_bounds__(256) void k_edge_fwd(int64_t n, int F, int K, float rc,
                                                  const int32_t* __restrict__ arow, const int32_t* __restrict__ acol,
                                                  const float4* __restrict__ ar, const float* __restrict__ PHI,
                                                  const float* __restrict__ S, const float* __restrict__ V,
                                                  const float* __restrict__ Wf, const float* __restrict__ bf,
                                                  float* __restrict__ SM, float* __restrict__ VM,
                                                  __nv_bfloat16* __restrict__ VMb, float* __restrict__ wst,
                                                  int v_zero) {
  extern __shared__ __align__(16) float sm[];
  constexpr int KD = STORE ? KP : 0;            // derivative basis staged only when storing
  const int G = blockDim.x / F;                 // groups per block
  const int g = threadIdx.x / F, f = threadIdx.x % F;
  float* rbs = sm + (size_t)g * F * (KP + KD);                                   // [F edges][KP]
  float* drbs = rbs + (size_t)F * KP;                                            // [F edges][KD]
  float4* geo = reinterpret_cast<float4*>(sm + (size_t)G * F * (KP + KD)) + (size_t)g * F;  // (u, f_c)
  float* dfcs = reinterpret_cast<float*>(sm + (size_t)G * F * (KP + KD + 4)) + (size_t)g * F;
  int* js = reinterpret_cast<int*>(sm + (size_t)G * F * (KP + KD + 4 + (STORE ? 1 : 0))) + (size_t)g * F;

  float w_s[KP], w_vv[KP], w_vs[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    w_s[k] = Wf[(size_t)f * KP + k];
    w_vv[k] = Wf[(size_t)(F + f) * KP + k];
    w_vs[k] = Wf[(size_t)(2 * F + f) * KP + k];
  }
  const float b_s = bf[f], b_vv = bf[F + f], b_vs = bf[2 * F + f];
  const float inv_rc = 1.0f / rc, sig = rc / (float)(K - 1), inv2s2 = 1.0f / (2.0f * sig * sig);
  const float inv_s2 = 1.0f / (sig * sig);
  const int64_t ngroups = (int64_t)gridDim.x * G;

  for (int64_t i = (int64_t)blockIdx.x * G + g; i < n; i += ngroups) {
    const int a0 = arow[i], a1 = arow[i + 1];
    float as = 0.f, av0 = 0.f, av1 = 0.f, av2 = 0.f;
    for (int c0 = a0; c0 < a1; c0 += F) {
      const int cnt = min(F, a1 - c0);
      group_sync(1 + g, F);
      if (f < cnt) {
        float4 r = ar[c0 + f];
        float d = r.w, id = 1.0f / d;
        float fc = 0.5f * (cospif(d * inv_rc) + 1.0f);
        geo[f] = make_float4(r.x * id, r.y * id, r.z * id, fc);
        if (STORE) dfcs[f] = -0.5f * 3.14159265358979f * inv_rc * sinpif(d * inv_rc);
        js[f] = acol[c0 + f];
#pragma unroll
        for (int k = 0; k < KP; ++k) {
          float mu = (float)k * sig, t = d - mu;
          const float v = k < K ? expf(-t * t * inv2s2) : 0.0f;
          rbs[f * KP + k] = v;
          if (STORE) drbs[f * KP + k] = -v * t * inv_s2;
        }
      }
      group_sync(1 + g, F);
      for (int t = 0; t < cnt; ++t) {
        const float4 ge = geo[t];
        const float* rb = rbs + t * KP;
        float ws = b_s, wvv = b_vv, wvs = b_vs;
#pragma unroll
        for (int k = 0; k < KP; k += 4) {
          float4 q = *reinterpret_cast<const float4*>(rb + k);
          ws = fmaf(w_s[k], q.x, ws); ws = fmaf(w_s[k + 1], q.y, ws);
          ws = fmaf(w_s[k + 2], q.z, ws); ws = fmaf(w_s[k + 3], q.w, ws);
          wvv = fmaf(w_vv[k], q.x, wvv); wvv = fmaf(w_vv[k + 1], q.y, wvv);
          wvv = fmaf(w_vv[k + 2], q.z, wvv); wvv = fmaf(w_vv[k + 3], q.w, wvv);
          wvs = fmaf(w_vs[k], q.x, wvs); wvs = fmaf(w_vs[k + 1], q.y, wvs);
          wvs = fmaf(w_vs[k + 2], q.z, wvs); wvs = fmaf(w_vs[k + 3], q.w, wvs);
        }
        // v_zero (first layer, v = 0): the psi channels v_a phi_vv are zero and not gathered
        const float* p = PHI + (int64_t)js[t] * 6 * F;
        const float ps = p[f], pvs = p[4 * F + f];
        const float y0 = v_zero ? 0.f : p[F + f], y1 = v_zero ? 0.f : p[2 * F + f], y2 = v_zero ? 0.f : p[3 * F + f];
        if (STORE) {
          const float* drb = drbs + t * KP;
          float dws = 0.f, dwvv = 0.f, dwvs = 0.f;
#pragma unroll
          for (int k = 0; k < KP; ++k) {
            dws = fmaf(w_s[k], drb[k], dws);
            dwvv = fmaf(w_vv[k], drb[k], dwvv);
            dwvs = fmaf(w_vs[k], drb[k], dwvs);
          }
          const float fc = ge.w, dfc = dfcs[t];
          float* o = wst + (int64_t)(c0 + t) * 6 * F + f;
          o[0] = ws * fc;
          o[F] = wvv * fc;
          o[2 * F] = wvs * fc;
          o[3 * F] = fc * dws + dfc * ws;
          o[4 * F] = fc * dwvv + dfc * wvv;
          o[5 * F] = fc * dwvs + dfc * wvs;
        }
        ws *= ge.w; wvv *= ge.w; wvs *= ge.w;
        as = fmaf(ps, ws, as);
        const float tvs = pvs * wvs;
        av0 = fmaf(y0, wvv, fmaf(ge.x, tvs, av0));
        av1 = fmaf(y1, wvv, fmaf(ge.y, tvs, av1));
        av2 = fmaf(y2, wvv, fmaf(ge.z, tvs, av2));
      }
    }
    SM[i * F + f] = S[i * F + f] + as;
    VM[i * 3 * F + f] = V[i * 3 * F + f] + av0;
    VM[i * 3 * F + F + f] = V[i * 3 * F + F + f] + av1;
    VM[i * 3 * F + 2 * F + f] = V[i * 3 * F + 2 * F + f] + av2;
    if (VMb) {
      VMb[i * 3 * F + f] = __float2bfloat16_rn(VM[i * 3 * F + f]);
      VMb[i * 3 * F + F + f] = __float2bfloat16_rn(VM[i * 3 * F + F + f]);
      VMb[i * 3 * F + 2 * F + f] = __float2bfloat16_rn(VM[i * 3 * F + 2 * F + f]);
    }
  }
}

// Reduce four per-thread values over a warp; lane 8*q ends up with the sum of value q.
__device__ __forceinline__ float warp_reduce4(float v0, float v1, float v2, float v3, int lane) {
  // xor 16: lanes < 16 keep (v0, v1), lanes >= 16 keep (v2, v3)
  bool hi = lane & 16;
  float s0 = hi ? v0 : v2, s1 = hi ? v1 : v3;
  float k0 = hi ? v2 : v0, k1 = hi ? v3 : v1;
  k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
  k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
  // xor 8: lanes with bit 3 clear keep k0, set keep k1
  bool b8 = lane & 8;
  float s = b8 ? k0 : k1, k = b8 ? k1 : k0;
  k += __shfl_xor_sync(0xffffffffu, s, 8);
  k += __shfl_xor_sync(0xffffffffu, k, 4);
  k += __shfl_xor_sync(0xffffffffu, k, 2);
  k += __shfl_xor_sync(0xffffffffu, k, 1);
  return k;   // lane 0: v0, lane 8: v1, lane 16: v2, lane 24: v3
}

// Adjoint of the message step, sender-side.  Row j holds edges e' = (j <- i); its reverse
// (i <- j) carried phi_j, v_j into receiver i with direction u_rev = -u_e'.  Thread f gathers
// (gsm_i, gvm_i) and accumulates d/dphi_s,j, d/dpsi_j,a, d/dphi_vs,j over the row; per edge the
// partial d/dd and d/du_rev are reduced over the F channels and turned into
// hedge[e'] = dU/dr_(i<-j).
//
// STORED: the filter and its distance derivative come from wst (written by k_edge_fwd<.., true>
// for the same edge, whose distance equals its reverse's) instead of being recomputed.
template <int KP, bool STORED>
__global__ __launch_bounds__(256) void k_edge_bwd(int64_t n, int F, int K, float rc, int accumulate,
                                                  const int32_t* __restrict__ arow, const int32_t* __restrict__ acol,
                                                  const float4* __restrict__ ar, const float* __restrict__ PHI,
                                                  const float* __restrict__ Gsm, const float* __restrict__ Gvm,
                                                  const float* __restrict__ Wf, const float* __restrict__ bf,
                                                  float* __restrict__ GPHI, float4* __restrict__ hedge,
                                                  const float* __restrict__ wst) {
  extern __shared__ __align__(16) float sm[];
  constexpr int KB = STORED ? 0 : KP;   // basis staged only when recomputing
  const int G = blockDim.x / F;
  const int g = threadIdx.x / F, f = threadIdx.x % F, lane = threadIdx.x & 31, wig = f >> 5;
  const int NW = F / 32;
  float* rbs = sm + (size_t)g * F * (2 * KB + 8 + 4 * NW);     // [F][KB] rbf, [F][KB] drbf
  float* drbs = rbs + F * KB;
  float4* geo = reinterpret_cast<float4*>(drbs + F * KB);       // (u, d)
  float4* gfc = geo + F;                                        // (f_c, f_c', -, -)
  float* red = reinterpret_cast<float*>(gfc + F);               // [F edges][NW][4]
  int* js = reinterpret_cast<int*>(sm + (size_t)G * F * (2 * KB + 8 + 4 * NW)) + (size_t)g * F;

  float w_s[KB > 0 ? KB : 1], w_vv[KB > 0 ? KB : 1], w_vs[KB > 0 ? KB : 1];
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    w_s[k] = Wf[(size_t)f * KP + k];
    w_vv[k] = Wf[(size_t)(F + f) * KP + k];
    w_vs[k] = Wf[(size_t)(2 * F + f) * KP + k];
  }
  const float b_s = bf[f], b_vv = bf[F + f], b_vs = bf[2 * F + f];
  const float inv_rc = 1.0f / rc, sig = rc / (float)(K - 1), inv2s2 = 1.0f / (2.0f * sig * sig);
  const float inv_s2 = 1.0f / (sig * sig);
  const int64_t ngroups = (int64_t)gridDim.x * G;

  for (int64_t j = (int64_t)blockIdx.x * G + g; j < n; j += ngroups) {
    const float* pj = PHI + j * 6 * F;
    const float ps = pj[f], y0 = pj[F + f], y1 = pj[2 * F + f], y2 = pj[3 * F + f], pvs = pj[4 * F + f];
    float gps = 0.f, gy0 = 0.f, gy1 = 0.f, gy2 = 0.f, gpvs = 0.f;
    const int a0 = arow[j], a1 = arow[j + 1];
    for (int c0 = a0; c0 < a1; c0 += F) {
      const int cnt = min(F, a1 - c0);
      group_sync(1 + g, F);
      if (f < cnt) {
        float4 r = ar[c0 + f];
        float d = r.w, id = 1.0f / d;
        float fc = 0.5f * (cospif(d * inv_rc) + 1.0f);
        float dfc = -0.5f * 3.14159265358979f * inv_rc * sinpif(d * inv_rc);
        geo[f] = make_float4(r.x * id, r.y * id, r.z * id, d);
        gfc[f] = make_float4(fc, dfc, 0.f, 0.f);
        js[f] = acol[c0 + f];
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          float t = d - (float)k * sig;
          float rb = k < K ? expf(-t * t * inv2s2) : 0.0f;
          rbs[f * KP + k] = rb;
          drbs[f * KP + k] = -rb * t * inv_s2;
        }
      }
      group_sync(1 + g, F);
      for (int t = 0; t < cnt; ++t) {
        const float4 ge = geo[t];
        float Ws, Wvv, Wvs, pd_s, pd_vv, pd_vs;   // filter and dW/dd per channel (f_c folded in)
        if (STORED) {
          const float* w = wst + (int64_t)(c0 + t) * 6 * F + f;
          Ws = w[0]; Wvv = w[F]; Wvs = w[2 * F];
          pd_s = w[3 * F]; pd_vv = w[4 * F]; pd_vs = w[5 * F];
        } else {
          const float4 fcv = gfc[t];
          const float* rb = rbs + t * KP;
          const float* drb = drbs + t * KP;
          float ws = b_s, wvv = b_vv, wvs = b_vs, dws = 0.f, dwvv = 0.f, dwvs = 0.f;
#pragma unroll
          for (int k = 0; k < KB; k += 4) {
            float4 q = *reinterpret_cast<const float4*>(rb + k);
            float4 dq = *reinterpret_cast<const float4*>(drb + k);
            float qa[4] = {q.x, q.y, q.z, q.w}, da[4] = {dq.x, dq.y, dq.z, dq.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              ws = fmaf(w_s[k + u], qa[u], ws);
              wvv = fmaf(w_vv[k + u], qa[u], wvv);
              wvs = fmaf(w_vs[k + u], qa[u], wvs);
              dws = fmaf(w_s[k + u], da[u], dws);
              dwvv = fmaf(w_vv[k + u], da[u], dwvv);
              dwvs = fmaf(w_vs[k + u], da[u], dwvs);
            }
          }
          const float fc = fcv.x, dfc = fcv.y;
          Ws = ws * fc; Wvv = wvv * fc; Wvs = wvs * fc;
          pd_s = fc * dws + dfc * ws; pd_vv = fc * dwvv + dfc * wvv; pd_vs = fc * dwvs + dfc * wvs;
        }
        const int64_t i = js[t];
        const float gs = Gsm[i * F + f];
        const float gv0 = Gvm[i * 3 * F + f], gv1 = Gvm[i * 3 * F + F + f], gv2 = Gvm[i * 3 * F + 2 * F + f];
        gps = fmaf(gs, Ws, gps);
        gy0 = fmaf(gv0, Wvv, gy0);
        gy1 = fmaf(gv1, Wvv, gy1);
        gy2 = fmaf(gv2, Wvv, gy2);
        // u_rev = -u
        const float q = -(gv0 * ge.x + gv1 * ge.y + gv2 * ge.z);
        gpvs = fmaf(q, Wvs, gpvs);
        const float gWs = gs * ps, gWvv = gv0 * y0 + gv1 * y1 + gv2 * y2, gWvs = q * pvs;
        float pd = gWs * pd_s + gWvv * pd_vv + gWvs * pd_vs;
        const float tv = pvs * Wvs;
        float r = warp_reduce4(pd, gv0 * tv, gv1 * tv, gv2 * tv, lane);
        if ((lane & 7) == 0) red[(t * NW + wig) * 4 + (lane >> 3)] = r;
      }
      group_sync(1 + g, F);
      if (f < cnt) {
        float pd = 0.f, gu0 = 0.f, gu1 = 0.f, gu2 = 0.f;
        for (int w = 0; w < NW; ++w) {
          const float* rr = red + (f * NW + w) * 4;
          pd += rr[0]; gu0 += rr[1]; gu1 += rr[2]; gu2 += rr[3];
        }
        const float4 ge = geo[f];
        const float ux = -ge.x, uy = -ge.y, uz = -ge.z, id = 1.0f / ge.w;
        const float gdu = gu0 * ux + gu1 * uy + gu2 * uz;
        float4 h = make_float4(pd * ux + (gu0 - gdu * ux) * id, pd * uy + (gu1 - gdu * uy) * id,
                               pd * uz + (gu2 - gdu * uz) * id, 0.f);
        if (accumulate) {
          float4 o = hedge[c0 + f];
          h.x += o.x; h.y += o.y; h.z += o.z;
        }
        hedge[c0 + f] = h;
      }
    }
    if (GPHI) {
      float* o = GPHI + j * 5 * F;
      o[f] = gps;
      o[F + f] = gy0;
      o[2 * F + f] = gy1;
      o[3 * F + f] = gy2;
      o[4 * F + f] = gpvs;
    }
  }
}

// ================================================================================ readout, forces
// h3 = R1 s + d1 (done by the GEMM); U_i = e_scale (R2 . silu(h3) + d2);
// G3 = w_i e_scale R2 * silu'(h3) (seed of the backward pass); per-block FP64 partials of
// sum_i w_i U_i.  ew (null: all ones) weights each atom's energy: 1 for the atoms a domain owns,
// 0 for its copies of other domains' atoms (Results, "Distributed potential computation").
// e_atom receives w_i U_i.
__global__ void k_readout(int64_t n, int Fh, float e_scale, const float* __restrict__ H3,
                          const float* __restrict__ R2, const float* __restrict__ d2,
                          const float* __restrict__ ew, float* __restrict__ G3, __nv_bfloat16* __restrict__ G3b,
                          float* __restrict__ e_atom, double* __restrict__ partials) {
  __shared__ double sbuf[kThreads / 32];
  double acc = 0.0, comp = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float wi = ew ? ew[i] : 1.0f;
    // the readout's terms can largely cancel (U_i small next to them): they are summed in FP64
    // and rounded once to the FP32 per-atom energy; the total is the compensated sum of those
    // per-atom values, so that any grouping of atoms (a served replica) sums to the same total
    double e = (double)d2[0];
    for (int k = 0; k < Fh; ++k) {
      float h = H3[i * Fh + k];
      e = fma((double)R2[k], (double)silu_f(h), e);
      if (G3) {
        const float gk = wi * (e_scale * R2[k] * dsilu_f(h));
        G3[i * Fh + k] = gk;
        if (G3b) G3b[i * Fh + k] = __float2bfloat16_rn(gk);
      }
    }
    e *= (double)e_scale;
    e *= (double)wi;
    const float ef = (float)e;
    if (e_atom) e_atom[i] = ef;
    double x = (double)ef, t = acc + x;   // Neumaier
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

// Error-free transformations in FP32 (Knuth's TwoSum; the exact product split by one FMA):
// a + b = s + e and a * b = p + e exactly, with s, p the rounded results.
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// Add the pair (x, xe) to the float-float accumulator (s, c): c collects every rounding error.
__device__ __forceinline__ void ff_add(float& s, float& c, float x, float xe) {
  float t, e;
  two_sum_f(s, x, t, e);
  s = t;
  c = __fadd_rn(c, __fadd_rn(e, xe));
}

static bool readout_is_fused(int F) { return F == 64 || F == 128; }

// The readout MLP and its backward in one pass: per atom h = R1 s + d1 (F/2 units),
// E_i = e_scale w_i (R2 . silu(h) + d2) and, with gradients, g = w_i e_scale R2 * silu'(h) and
// gs = R1^T g, h and gs as FP32 fmaf chains over the inputs and over the hidden units in order
// (as the GEMMs they replace), the energy terms in FP64, summed over the 16 threads that hold an
// atom's units in a fixed tree (so independent of the launch).  A block of 512 threads stands for one
// 256-thread block of the grid-stride energy sum: it takes the 256-atom ranges starting at
// 256 (b + G k) (G = blocks), as two 128-atom tiles, and its thread t < 256 adds the energy of
// atom 256 (b + G k) + t, the same atoms in the same order.  s and R1 are staged transposed so
// that each thread's 4 atoms and 4 units come in 16-byte shared loads.
template <int F>
__global__ __launch_bounds__(512, 1) void k_readout_fused(int64_t n, float e_scale, const float* __restrict__ S,
                                                       const float* __restrict__ R1, const float* __restrict__ R1t,
                                                       const float* __restrict__ d1, const float* __restrict__ R2,
                                                       const float* __restrict__ d2, const float* __restrict__ ew,
                                                       float* __restrict__ GS, float* __restrict__ e_atom,
                                                       double* __restrict__ partials) {
  constexpr int FH = F / 2, TA = 128, F4 = F / 4, GP = FH + 4;
  constexpr int OPT = FH / 16, KPT = F / 16;   // units (forward) and inputs (backward) per thread
  extern __shared__ float4 rd_smem4[];
  float* sR1T = reinterpret_cast<float*>(rd_smem4);   // [F][FH]   R1^T (input, unit)
  float* sR1 = sR1T + F * FH;                         // [FH][F]   R1 (unit, input)
  float* sST = sR1 + FH * F;                          // [F][TA]   s^T of the tile
  float* sG = sST + F * TA;                           // [TA][GP]  g of the tile
  float* sE = sG + TA * GP;                           // [256]     per-atom energies of the range
  float* sR2 = sE + 256;                              // [FH]
  __shared__ double sbuf[8];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;   // ty: atoms 4 ty .. 4 ty + 3
  for (int idx = tid; idx < F * FH / 4; idx += 512) {
    reinterpret_cast<float4*>(sR1T)[idx] = reinterpret_cast<const float4*>(R1t)[idx];
    reinterpret_cast<float4*>(sR1)[idx] = reinterpret_cast<const float4*>(R1)[idx];
  }
  for (int k = tid; k < FH; k += 512) sR2[k] = R2[k];
  __syncthreads();
  double acc = 0.0, comp = 0.0;
  const int64_t G = (int64_t)gridDim.x * 256;
  for (int64_t base = (int64_t)blockIdx.x * 256; base < n; base += G) {
    for (int t2 = 0; t2 < 2; ++t2) {
      const int64_t a0 = base + t2 * TA;
      for (int idx = tid; idx < TA * F4; idx += 512) {
        const int a = idx % TA, k4 = idx / TA;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (a0 + a < n) v = reinterpret_cast<const float4*>(S + (a0 + a) * F)[k4];
        sST[(4 * k4 + 0) * TA + a] = v.x;
        sST[(4 * k4 + 1) * TA + a] = v.y;
        sST[(4 * k4 + 2) * TA + a] = v.z;
        sST[(4 * k4 + 3) * TA + a] = v.w;
      }
      __syncthreads();
      {
        float h[4][OPT];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < OPT; ++j) h[i][j] = 0.0f;
#pragma unroll 4
        for (int k = 0; k < F; ++k) {
          const float4 sa = *reinterpret_cast<const float4*>(sST + k * TA + 4 * ty);
          float r[OPT];
          if constexpr (OPT == 4) {
            const float4 q = *reinterpret_cast<const float4*>(sR1T + k * FH + 4 * tx);
            r[0] = q.x; r[1] = q.y; r[2] = q.z; r[3] = q.w;
          } else {
            const float2 q = *reinterpret_cast<const float2*>(sR1T + k * FH + 2 * tx);
            r[0] = q.x; r[1] = q.y;
          }
          const float sv[4] = {sa.x, sa.y, sa.z, sa.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < OPT; ++j) h[i][j] = fmaf(sv[i], r[j], h[i][j]);
        }
        // energy terms of this thread's units, each product split exactly (FMA) and added into a
        // float-float pair (TwoSum), the pairs of the 16 threads of an atom combined in a fixed
        // tree: the terms can largely cancel, and this keeps ~44 bits of their sum without the
        // FP64 pipe; g = w e_scale R2 silu'(h) goes to the g tile
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t ai = a0 + 4 * ty + i;
          const float wi = ai < n && ew ? ew[ai] : 1.0f;
          float es = 0.0f, ec = 0.0f;
#pragma unroll
          for (int j = 0; j < OPT; ++j) {
            const int o = OPT * tx + j;
            const float hk = h[i][j] + (d1 ? d1[o] : 0.0f);
            const float sl = silu_f(hk), pr = __fmul_rn(sR2[o], sl);
            ff_add(es, ec, pr, __fmaf_rn(sR2[o], sl, -pr));
            if (GS) sG[(4 * ty + i) * GP + o] = ai < n ? wi * (e_scale * sR2[o] * dsilu_f(hk)) : 0.0f;
          }
#pragma unroll
          for (int off = 1; off < 16; off <<= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, es, off), oc = __shfl_xor_sync(0xffffffffu, ec, off);
            ff_add(es, ec, os, oc);
          }
          if (tx == 0) {
            double e = ((double)es + (double)ec + (double)d2[0]) * (double)e_scale;
            e *= (double)wi;
            const float ef = ai < n ? (float)e : 0.0f;
            if (ai < n && e_atom) e_atom[ai] = ef;
            sE[t2 * TA + 4 * ty + i] = ef;
          }
        }
      }
      __syncthreads();
      if (GS) {
        // gs = R1^T g over the units in order: thread -> atoms 4 ty .. + 3, inputs KPT tx .. + KPT - 1
        float gq[4][KPT];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < KPT; ++j) gq[i][j] = 0.0f;
#pragma unroll 4
        for (int o = 0; o < FH; ++o) {
          const float gv[4] = {sG[(4 * ty) * GP + o], sG[(4 * ty + 1) * GP + o], sG[(4 * ty + 2) * GP + o],
                               sG[(4 * ty + 3) * GP + o]};
          float r[KPT];
#pragma unroll
          for (int j = 0; j < KPT; j += 4) {
            const float4 q = *reinterpret_cast<const float4*>(sR1 + o * F + KPT * tx + j);
            r[j] = q.x; r[j + 1] = q.y; r[j + 2] = q.z; r[j + 3] = q.w;
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < KPT; ++j) gq[i][j] = fmaf(gv[i], r[j], gq[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t ai = a0 + 4 * ty + i;
          if (ai < n)
#pragma unroll
            for (int j = 0; j < KPT; j += 4)
              *reinterpret_cast<float4*>(GS + ai * F + KPT * tx + j) =
                  make_float4(gq[i][j], gq[i][j + 1], gq[i][j + 2], gq[i][j + 3]);
        }
      }
      __syncthreads();   // the next tile overwrites s^T and g
    }
    if (tid < 256 && base + tid < n) {
      const double x = (double)sE[tid], t = acc + x;   // Neumaier
      comp += fabs(acc) >= fabs(x) ? (acc - t) + x : (x - t) + acc;
      acc = t;
    }
  }
  double v = acc + comp;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0 && tid < 256) sbuf[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    double sum = 0.0;
    for (int w = 0; w < 8; ++w) sum += sbuf[w];
    partials[blockIdx.x] = sum;
  }
}

template <int F>
static size_t readout_fused_smem() {
  return sizeof(float) * ((size_t)2 * F * (F / 2) + (size_t)F * 128 + (size_t)128 * (F / 2 + 4) + 256 + F / 2);
}

// F_i = sum_{e in row i} (hedge[rev e] - hedge[e]);  virial partials = sum_e r_e (x) hedge[e]
// (= -sum_e r_e (x) dU/dr_e over all edges).  One warp per row for the forces.  The virial is a
// compensated sum: every product r_p h_q is split exactly into a float pair (FMA) and added with
// TwoSum into float-float accumulators that each lane keeps over all its edges of all its rows
// (about 44 significant bits); the warp combines its lanes once at the end with TwoSum, and the
// warps of a block in FP64 Neumaier order, so the only roundings left are those of the
// float-float sums and of the final FP64 sums.
__global__ void k_forces(int64_t n, const int32_t* __restrict__ arow, const float4* __restrict__ ar,
                         const int32_t* __restrict__ arev, const float4* __restrict__ hedge,
                         float* __restrict__ force, double* __restrict__ vpart, int* status) {
  __shared__ double sv[kThreads / 32][18];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float v[9], ve[9];
#pragma unroll
  for (int p = 0; p < 9; ++p) v[p] = ve[p] = 0.f;
  const int64_t nw = (int64_t)gridDim.x * (kThreads / 32);
  for (int64_t i = (int64_t)blockIdx.x * (kThreads / 32) + w; i < n; i += nw) {
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int a = arow[i] + lane; a < arow[i + 1]; a += 32) {
      const int ra = arev[a];
      const float4 h = hedge[a], r = ar[a];
      float4 hr = make_float4(0.f, 0.f, 0.f, 0.f);
      if (ra >= 0) hr = hedge[ra];
      else atomicOr(status, (int)ST_REV_MISSING);
      fx += hr.x - h.x; fy += hr.y - h.y; fz += hr.z - h.z;
      const float rr[3] = {r.x, r.y, r.z}, hh[3] = {h.x, h.y, h.z};
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const float pr = __fmul_rn(rr[p], hh[q]);
          ff_add(v[3 * p + q], ve[3 * p + q], pr, __fmaf_rn(rr[p], hh[q], -pr));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
      fx += __shfl_xor_sync(0xffffffffu, fx, o);
      fy += __shfl_xor_sync(0xffffffffu, fy, o);
      fz += __shfl_xor_sync(0xffffffffu, fz, o);
    }
    if (lane == 0) {
      force[3 * i] = fx; force[3 * i + 1] = fy; force[3 * i + 2] = fz;
    }
  }
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      const float os = __shfl_xor_sync(0xffffffffu, v[p], o), oe = __shfl_xor_sync(0xffffffffu, ve[p], o);
      ff_add(v[p], ve[p], os, oe);
    }
  if (lane == 0)
    for (int p = 0; p < 9; ++p) {
      sv[w][p] = (double)v[p];
      sv[w][9 + p] = (double)ve[p];
    }
  __syncthreads();
  if (threadIdx.x < 9) {
    double s = 0.0, c = 0.0;
    for (int q = 0; q < kThreads / 32; ++q)
      for (int h = 0; h < 2; ++h) {
        const double x = sv[q][9 * h + threadIdx.x], t = s + x;
        c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
        s = t;
      }
    vpart[(int64_t)blockIdx.x * 9 + threadIdx.x] = s + c;
  }
}

// ================================================================================ driver
static inline unsigned blocks_for(int64_t work) { return (unsigned)((work + kThreads - 1) / kThreads); }

template <int KP>
static void edge_fwd_kp(cudaStream_t st, const ModelW& m, int t, int64_t n, const int32_t* arow,
                        const int32_t* acol, const float4* ar, const float* PHI, const float* S, const float* V,
                        float* SM, float* VM, __nv_bfloat16* VMb, float* wst) {
  const int v_zero = t == 0;   // the first layer's v is the embedding's zero
  const int F = m.F, G = kThreads / F;
  const int KD = wst ? KP : 0;
  size_t smem = (size_t)G * F * (KP + KD + 4 + (wst ? 1 : 0)) * sizeof(float) + (size_t)G * F * sizeof(int);
  int64_t blocks = (n + G - 1) / G;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  LaunchScope ls_(st);
  if (wst)
    k_edge_fwd<KP, true><<<(unsigned)blocks, kThreads, smem, st>>>(n, F, m.K, m.rc, arow, acol, ar, PHI, S, V,
                                                                   m.L[t].Wf, m.L[t].bf, SM, VM, VMb, wst, v_zero);
  else
    k_edge_fwd<KP, false><<<(unsigned)blocks, kThreads, smem, st>>>(n, F, m.K, m.rc, arow, acol, ar, PHI, S, V,
                                                                    m.L[t].Wf, m.L[t].bf, SM, VM, VMb, nullptr, v_zero);
}

template <int KP>
static void edge_bwd_kp(cudaStream_t st, const ModelW& m, int t, int accumulate, int64_t n, const int32_t* arow,
                        const int32_t* acol, const float4* ar, const float* PHI, const float* Gsm,
                        const float* Gvm, float* GPHI, float4* hedge, const float* wst) {
  const int F = m.F, G = kThreads / F, NW = F / 32;
  const int KB = wst ? 0 : KP;
  size_t smem = (size_t)G * F * (2 * KB + 8 + 4 * NW) * sizeof(float) + (size_t)G * F * sizeof(int);
  int64_t blocks = (n + G - 1) / G;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  LaunchScope ls_(st);
  if (wst)
    k_edge_bwd<KP, true><<<(unsigned)blocks, kThreads, smem, st>>>(n, F, m.K, m.rc, accumulate, arow, acol, ar, PHI,
                                                                   Gsm, Gvm, m.L[t].Wf, m.L[t].bf, GPHI, hedge, wst);
  else
    k_edge_bwd<KP, false><<<(unsigned)blocks, kThreads, smem, st>>>(n, F, m.K, m.rc, accumulate, arow, acol, ar, PHI,
                                                                    Gsm, Gvm, m.L[t].Wf, m.L[t].bf, GPHI, hedge, nullptr);
}

#define CTD_KP_DISPATCH(KPV, CALL) \
  switch (KPV) {                   \
    case 4: CALL(4); break;        \
    case 8: CALL(8); break;        \
    case 12: CALL(12); break;      \
    case 16: CALL(16); break;      \
    case 20: CALL(20); break;      \
    case 24: CALL(24); break;      \
    case 28: CALL(28); break;      \
    default: CALL(32); break;      \
  }

void edge_smem_setup() {
  static bool done = false;
  if (done) return;
  done = true;
#define CTD_SET_SMEM(K_)                                                                              \
  cudaFuncSetAttribute(k_edge_fwd<K_, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); \
  cudaFuncSetAttribute(k_edge_fwd<K_, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);  \
  cudaFuncSetAttribute(k_edge_bwd<K_, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); \
  cudaFuncSetAttribute(k_edge_bwd<K_, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  CTD_SET_SMEM(4) CTD_SET_SMEM(8) CTD_SET_SMEM(12) CTD_SET_SMEM(16) CTD_SET_SMEM(20) CTD_SET_SMEM(24)
  CTD_SET_SMEM(28) CTD_SET_SMEM(32)
#undef CTD_SET_SMEM
}

// Buffers (all float, sized by the caller; see api.cu for the list and shapes).
enum BufId {
  B_S0 = 0,                        // s, one buffer for every layer (ids B_S0 + t unused)
  B_V0 = B_S0 + kMaxT + 1,         // V[t] for t = 0..T
  B_PHI0 = B_V0 + kMaxT + 1,       // [n][6F] per layer
  B_H10 = B_PHI0 + kMaxT,          // [n][F]
  B_SM0 = B_H10 + kMaxT,           // [n][F]  s^m, v^m: read only within their layer's forward pass,
  B_VM0 = B_SM0 + kMaxT,           // [n][3F] so one buffer each (id + 0) serves every layer
  B_UV0 = B_VM0 + kMaxT,           // [3n][2F]
  B_H20 = B_UV0 + kMaxT,           // [n][F]
  B_AV0 = B_H20 + kMaxT,           // [n][3F]
  B_T1 = B_AV0 + kMaxT,            // [n][3F] scratch
  B_T2,                            // [n][3F] scratch
  B_T3,                            // [3n][2F] scratch
  B_GS, B_GV, B_GSM, B_GVM,        // [n][F], [n][3F], [n][F], [n][3F]
  B_GPHI,                          // [n][5F]
  B_G4,                            // [n][F][4] = (gsm, gvm_0..2) per feature (tensor-core adjoint)
  B_H3, B_G3,                      // [n][F/2]
  B_COUNT
};

int model_buffer_count() { return B_COUNT; }

// The readout and, with gradients, gs = dE/ds_T: one fused launch for F = 64 and 128, else the
// FP32 GEMM, readout and GEMM launches (H3 and G3 buffers).
static void readout_fwd_bwd(cudaStream_t st, const ModelW& m, int64_t n, const float* S_T, const float* ew,
                            bool need_grad, float* const* B, float* e_atom, double* partials, int n_partials) {
  const int F = m.F, Fh = F / 2;
  if (readout_is_fused(F)) {
    LaunchScope ls_(st);
    float* gs = need_grad ? B[B_GS] : nullptr;
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_readout_fused<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)readout_fused_smem<128>());
      cudaFuncSetAttribute(k_readout_fused<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)readout_fused_smem<64>());
      attr = true;
    }
    if (F == 128)
      k_readout_fused<128><<<n_partials, 512, readout_fused_smem<128>(), st>>>(n, m.e_scale, S_T, m.R1, m.R1t, m.d1,
                                                                               m.R2, m.d2, ew, gs, e_atom, partials);
    else
      k_readout_fused<64><<<n_partials, 512, readout_fused_smem<64>(), st>>>(n, m.e_scale, S_T, m.R1, m.R1t, m.d1,
                                                                             m.R2, m.d2, ew, gs, e_atom, partials);
    return;
  }
  gemm<EPI_BIAS>(st, n, Fh, F, S_T, F, m.R1t, m.d1, nullptr, 0, B[B_H3], Fh);
  {
    LaunchScope ls_(st);
    k_readout<<<n_partials, kThreads, 0, st>>>(n, Fh, m.e_scale, B[B_H3], m.R2, m.d2, ew,
                                               need_grad ? B[B_G3] : nullptr, nullptr, e_atom, partials);
  }
  if (need_grad) gemm<EPI_BIAS>(st, n, F, Fh, B[B_G3], Fh, m.R1, nullptr, nullptr, 0, B[B_GS], F);
}

// floats per atom of buffer id b (0 if unused for this T)
// The interleaved receiver gradients (G4) are read only by the bulk-gathered tensor-core
// adjoint of the BF16 path; no other path allocates them.
bool model_uses_g4(const ModelW& m, int precision) {
  return precision == CTD_PREC_BF16 && edge_tc_supported(m.F, m.K) && m.tc_adjoint;
}

// The BF16 path keeps the message table of each layer only as its FP16 copy when the contracted
// message step and the tensor-core adjoint both run: nothing else reads the FP32 table then.
bool model_phi_fp16_only(const ModelW& m, int precision) {
  return model_uses_g4(m, precision) && model_uses_msg_mma(m);
}

int64_t model_buffer_floats_per_atom(int b, const ModelW& m, int F, int T, int precision) {
  const bool g4 = model_uses_g4(m, precision), bf16 = precision == CTD_PREC_BF16;
  auto layer = [&](int base, int cnt) { return b >= base && b < base + cnt; };
  // s[t] is read only by layer t's forward (message residual; the backward never reads it), so
  // every layer's s lives in one buffer, overwritten by the next layer's update
  if (layer(B_S0, T + 1)) return b == B_S0 ? F : 0;
  if (layer(B_V0, T + 1)) {
    if (T > 0 && b == B_V0 + T) return 0;   // v[T] is never formed
    // v[0] = 0: the BF16 path with the contracted message step never stores it
    if (b == B_V0 && bf16 && model_uses_msg_mma(m)) return 0;
    return 3 * F;
  }
  if (layer(B_PHI0, T)) return model_phi_fp16_only(m, precision) ? 0 : 6 * F;
  if (layer(B_H10, T)) return bf16 ? 0 : F;   // the BF16 path keeps h1, h2 in FP16 (BB_H1H0, BB_H2H0)
  if (b == B_SM0 && T > 0) return F;
  if (b == B_VM0 && T > 0) return 3 * F;
  if (layer(B_UV0, T)) return bf16 ? 0 : 6 * F;   // the BF16 path keeps U/V products and
  if (layer(B_H20, T)) return bf16 ? 0 : F;
  if (layer(B_AV0, T)) return bf16 ? 0 : 3 * F;   // update coefficients in FP16 (BB_UVH0, BB_AVH0)
  switch (b) {
    case B_T1: return bf16 ? 2 * F : 3 * F;   // the BF16 path uses only T1, as [n][2F]
    case B_T2: return bf16 ? 0 : 3 * F;
    case B_T3: return bf16 ? 0 : 6 * F;
    case B_GS: case B_GSM: return F;
    case B_GV: return 3 * F;
    case B_GVM: return g4 ? 0 : 3 * F;   // with the tensor-core adjoint gvm lives only in G4
    case B_GPHI: return g4 ? 3 * F : 5 * F;   // the tensor-core adjoint writes only the psi gradients
    case B_G4: return g4 ? 4 * F : 0;
    case B_H3: case B_G3: return readout_is_fused(F) ? 0 : F / 2;   // the fused readout keeps h and g on chip
    default: return 0;
  }
}

void model_forward_backward_fp32(cudaStream_t st, const ModelW& m, int64_t n, const int32_t* species_s,
                                 const int32_t* arow, const int32_t* acol, const float4* ar,
                                 const int32_t* arev, float* const* B, bool need_grad,
                                 double* energy_partials, int n_energy_partials, float4* hedge,
                                 float* force_s, double* virial_partials, int n_virial_partials,
                                 float* e_atom, int* status, float* wstore, int64_t wstore_layer_floats,
                                 const float* ew) {
  edge_smem_setup();
  StageGuard node_stage(STG_NODE);
  const int F = m.F, T = m.T;
  const unsigned nb = blocks_for(n * F), nb4 = blocks_for(n * F / 4);   // nb4: four features per thread
  if (n > 0) { LaunchScope ls_(st); k_embed<<<nb, kThreads, 0, st>>>(n, F, species_s, m.emb, B[B_S0], B[B_V0], nullptr); }
  for (int t = 0; t < T; ++t) {
    const LayerW& L = m.L[t];
    float *S = B[B_S0], *V = B[B_V0 + t], *PHI = B[B_PHI0 + t], *H1 = B[B_H10 + t];
    float *SM = B[B_SM0], *VM = B[B_VM0], *UV = B[B_UV0 + t], *H2 = B[B_H20 + t], *AV = B[B_AV0 + t];
    float *T1 = B[B_T1], *T2 = B[B_T2];
    // phi = W2 silu(W1 s + b1) + b2
    gemm<EPI_BIAS_SILU>(st, n, F, F, S, F, L.W1t, L.b1, nullptr, 0, H1, F, T1, F);
    gemm<EPI_BIAS>(st, n, 3 * F, F, T1, F, L.W2t, L.b2, nullptr, 0, T2, 3 * F);
    if (n > 0) { LaunchScope ls_(st); k_phi_pack<<<nb, kThreads, 0, st>>>(n, F, T2, V, PHI); }
    // message
    float* wst = (wstore && need_grad) ? wstore + t * wstore_layer_floats : nullptr;
#define CTD_FWD(KPV) edge_fwd_kp<KPV>(st, m, t, n, arow, acol, ar, PHI, S, V, SM, VM, nullptr, wst)
    if (n > 0) {
      StageGuard sg(STG_EDGE_FWD);
      CTD_KP_DISPATCH(m.KP, CTD_FWD)
    }
#undef CTD_FWD
    // update
    gemm<EPI_BIAS>(st, 3 * n, 2 * F, F, VM, F, L.UVt, nullptr, nullptr, 0, UV, 2 * F);
    if (n > 0) { LaunchScope ls_(st); k_update_pre<float><<<nb4, kThreads, 0, st>>>(n, F, m.eps, SM, UV, T1, nullptr); }
    gemm<EPI_BIAS_SILU>(st, n, F, 2 * F, T1, 2 * F, L.A1t, L.c1, nullptr, 0, H2, F, T2, F);
    gemm<EPI_BIAS>(st, n, 3 * F, F, T2, F, L.A2t, L.c2, nullptr, 0, AV, 3 * F);
    if (n > 0) {
      LaunchScope ls_(st);
      if (t + 1 < T)
        k_update_post<float, true><<<nb4, kThreads, 0, st>>>(n, F, SM, VM, UV, AV, S, B[B_V0 + t + 1],
                                                             nullptr);
      else
        k_update_post<float, false><<<nb4, kThreads, 0, st>>>(n, F, SM, VM, UV, AV, S, nullptr, nullptr);
    }
  }
  // readout
  // readout, and dU/ds^T = G3 R1
  readout_fwd_bwd(st, m, n, B[B_S0], ew, need_grad, B, e_atom, energy_partials, n_energy_partials);
  if (!need_grad) return;
  if (n > 0) cudaMemsetAsync(B[B_GV], 0, sizeof(float) * (size_t)n * 3 * F, st);
  for (int t = T - 1; t >= 0; --t) {
    const LayerW& L = m.L[t];
    float *V = B[B_V0 + t], *PHI = B[B_PHI0 + t], *H1 = B[B_H10 + t];
    float *UV = B[B_UV0 + t], *H2 = B[B_H20 + t], *AV = B[B_AV0 + t];
    float *T1 = B[B_T1], *T2 = B[B_T2], *T3 = B[B_T3];
    float *GS = B[B_GS], *GV = B[B_GV], *GSM = B[B_GSM], *GVM = B[B_GVM], *GPHI = B[B_GPHI];
    // update backward
    if (n > 0) { LaunchScope ls_(st); k_update_bwd_pre<<<nb, kThreads, 0, st>>>(n, F, GS, GV, UV, AV, T1, T3, nullptr); }
    gemm<EPI_DSILU>(st, n, F, 3 * F, T1, 3 * F, L.A2, nullptr, H2, F, T2, F);          // gh2
    gemm<EPI_BIAS>(st, n, 2 * F, F, T2, F, L.A1, nullptr, nullptr, 0, T1, 2 * F);       // gz
    if (n > 0) { LaunchScope ls_(st); k_update_bwd_mid<<<nb, kThreads, 0, st>>>(n, F, m.eps, GS, T1, UV, GSM, T3, nullptr); }
    gemm<EPI_ADD>(st, 3 * n, F, 2 * F, T3, 2 * F, L.UV, nullptr, GV, F, GVM, F);         // gvm
    // message backward
    const float* wst = wstore ? wstore + t * wstore_layer_floats : nullptr;
    // the first layer's inputs (embedding, v = 0) do not depend on positions: its edge adjoint
    // writes no phi gradients and the phi backward below it is skipped
    float* gphi = t > 0 ? GPHI : nullptr;
#define CTD_BWD(KPV) edge_bwd_kp<KPV>(st, m, t, t != T - 1, n, arow, acol, ar, PHI, GSM, GVM, gphi, hedge, wst)
    if (n > 0) {
      StageGuard sg(STG_EDGE_BWD);
      CTD_KP_DISPATCH(m.KP, CTD_BWD)
    }
#undef CTD_BWD
    if (t == 0) break;
    // phi backward -> gradients w.r.t. the layer input (s_t, v_t)
    if (n > 0) { LaunchScope ls_(st); k_phi_bwd_pre<<<nb, kThreads, 0, st>>>(n, F, GPHI, PHI, nullptr, V, GVM, T2, GV, nullptr); }
    gemm<EPI_DSILU>(st, n, F, 3 * F, T2, 3 * F, L.W2, nullptr, H1, F, T1, F);          // gh1
    gemm<EPI_ADD>(st, n, F, F, T1, F, L.W1, nullptr, GSM, F, GS, F);                    // gs
  }
  StageGuard fstage(STG_FORCES);
  { LaunchScope ls_(st); k_forces<<<n_virial_partials, kThreads, 0, st>>>(n, arow, ar, arev, hedge, force_s, virial_partials, status); }
}


void launch_forces(cudaStream_t st, int64_t n, const int32_t* arow, const float4* ar, const int32_t* arev,
                   const float4* hedge, float* force, double* vpart, int n_vpart, int* status) {
  LaunchScope ls_(st);
  k_forces<<<n_vpart, kThreads, 0, st>>>(n, arow, ar, arev, hedge, force, vpart, status);
}

// ================================================================================ BF16 driver
// Same layer as above; every node MLP contraction runs on tcgen05 with BF16 operands and FP32
// accumulation (gemm_bf16.cu).  Producers write a BF16 shadow of each GEMM A operand; the
// elementwise work, the reductions and the residual streams s, v and their gradients stay FP32;
// the stored activations the backward reads as operands (message tables, U/V products, update
// coefficients, SiLU arguments) are kept in FP16, each write range-checked.
enum BufB {
  BB_S0 = 0,                 // bf16 s, one buffer     [n][F]
  BB_A1 = BB_S0 + kMaxT + 1, // silu(h1)               [n][F]
  BB_VM,                     // v^m                    [n][3F]
  BB_Z,                      // [s^m ; |Vv|]           [n][2F]
  BB_A2,                     // silu(h2)               [n][F]
  BB_GA,                     // g_a                    [n][3F]
  BB_GH2,                    // g_h2                   [n][F]
  BB_GUV,                    // [gUv | gVv]            [3n][2F]
  BB_GP3,                    // g_phi                  [n][3F]
  BB_GH1,                    // g_h1                   [n][F]
  BB_PHIH0,                  // FP16 message table of layer t, [n][6F] = [phi_s | psi_0..2 | phi_vs | phi_vv]
                             // (contracted message step; ids BB_PHIH0 + t)
  BB_UVH0 = BB_PHIH0 + kMaxT, // FP16 U/V products of layer t, rows (i, a) = [Uv_a | Vv_a]  [3n][2F]
  BB_AVH0 = BB_UVH0 + kMaxT,  // FP16 update coefficients of layer t, [a_vv | a_sv | a_ss]  [n][3F]
  BB_H1H0 = BB_AVH0 + kMaxT,  // FP16 SiLU arguments h1, h2 of layer t (read back only as SiLU'
  BB_H2H0 = BB_H1H0 + kMaxT,  // arguments of the BF16 backward GEMMs)  [n][F]
  BB_COUNT = BB_H2H0 + kMaxT
};

int model_bf16_buffer_count() { return BB_COUNT; }

bool model_uses_msg_mma(const ModelW& m) { return edge_mma_supported(m.F, m.K) && m.tc_message; }

// Stored edge filters are written by the CUDA-core message kernel and read by the CUDA-core
// adjoint, so they apply only when both run.
bool model_stores_edges(const ModelW& m, int precision) {
  if (!m.edge_store) return false;
  if (precision != CTD_PREC_BF16) return true;
  return !model_uses_msg_mma(m) && !(edge_tc_supported(m.F, m.K) && m.tc_adjoint);
}

int64_t model_bf16_buffer_elems_per_atom(int b, int F, int T, bool msg_mma) {
  if (b >= BB_S0 && b < BB_S0 + T + 1) return b == BB_S0 ? F : 0;   // read by the next W1 GEMM only
  if (b >= BB_PHIH0 && b < BB_PHIH0 + kMaxT) return msg_mma && b < BB_PHIH0 + T ? 6 * F : 0;
  if (b >= BB_UVH0 && b < BB_UVH0 + kMaxT) return b < BB_UVH0 + T ? 6 * F : 0;
  if (b >= BB_AVH0 && b < BB_AVH0 + kMaxT) return b < BB_AVH0 + T ? 3 * F : 0;
  if (b >= BB_H1H0 && b < BB_H1H0 + kMaxT) return b < BB_H1H0 + T ? F : 0;
  if (b >= BB_H2H0 && b < BB_H2H0 + kMaxT) return b < BB_H2H0 + T ? F : 0;
  switch (b) {
    case BB_A1: case BB_A2: case BB_GH2: case BB_GH1: return F;
    case BB_VM: case BB_GA: case BB_GP3: return 3 * F;
    case BB_Z: return 2 * F;
    case BB_GUV: return 6 * F;
    default: return 0;
  }
}

int model_forward_backward_bf16(cudaStream_t st, const ModelW& m, int64_t n, const int32_t* species_s,
                                const int32_t* arow, const int32_t* acol, const float4* ar, const int32_t* arev,
                                float* const* B, __nv_bfloat16* const* Bb, bool need_grad,
                                double* energy_partials, int n_energy_partials, float4* hedge, float* force_s,
                                double* virial_partials, int n_virial_partials, float* e_atom, int* status,
                                float* wstore, int64_t wstore_layer_floats, const int32_t* aend,
                                const float* ew) {
  edge_smem_setup();
  StageGuard node_stage(STG_NODE);
  const int F = m.F, T = m.T;
  const unsigned nb = blocks_for(n * F), nb4 = blocks_for(n * F / 4);   // nb4: four features per thread
  int bad = 0;
  // F = 128: the message step as the tensor-core contraction over each receiver's edges
  // (edge_mma.cu) and the adjoint with the radial filter on tcgen05 (edge_tc.cu), unless the
  // CUDA-core kernels are selected; other widths keep the CUDA-core edge kernels (FP32 filter).
  // The tensor-core kernels recompute the filter, so storing edge filters applies to the
  // CUDA-core kernels only.
  const bool use_tc = edge_tc_supported(F, m.K);
  const bool use_tc_bwd = use_tc && m.tc_adjoint;
  const bool msg_mma = model_uses_msg_mma(m);
  const bool g4 = model_uses_g4(m, CTD_PREC_BF16);
  // with the contracted message step each layer's table is kept in FP16 ([n][6F]); the FP32
  // table is written only for the CUDA-core adjoint, which reads it
  const bool phi32 = !model_phi_fp16_only(m, CTD_PREC_BF16);
  auto phih = [&](int t) { return msg_mma ? reinterpret_cast<__half*>(Bb[BB_PHIH0 + t]) : nullptr; };
  // with the contracted message step the first layer takes v = 0 without a stored v[0]
  if (n > 0) {
    LaunchScope ls_(st);
    k_embed<<<nb, kThreads, 0, st>>>(n, F, species_s, m.emb, B[B_S0], msg_mma ? nullptr : B[B_V0], Bb[BB_S0]);
  }
  for (int t = 0; t < T; ++t) {
    const LayerW& L = m.L[t];
    float *S = B[B_S0], *V = B[B_V0 + t], *PHI = phi32 ? B[B_PHI0 + t] : nullptr;
    float *SM = B[B_SM0], *VM = B[B_VM0];
    __half* H1 = reinterpret_cast<__half*>(Bb[BB_H1H0 + t]);   // SiLU arguments in FP16
    __half* H2 = reinterpret_cast<__half*>(Bb[BB_H2H0 + t]);
    __half* PHIh = phih(t);
    __half* UV = reinterpret_cast<__half*>(Bb[BB_UVH0 + t]);   // FP16 copies (range checked by the GEMMs)
    __half* AV = reinterpret_cast<__half*>(Bb[BB_AVH0 + t]);
    bad |= gemm_bf16<1>(st, n, F, F, Bb[BB_S0], F, L.W1b, L.b1, nullptr, 0, nullptr, F, Bb[BB_A1], F, status, H1);
    // phi = W2 silu(.) + b2, packed into PHI (and its FP16 copy) by the GEMM epilogue
    const float* Vin = (t == 0 && msg_mma) ? nullptr : V;   // null: v = 0, psi = 0
    bad |= gemm_bf16<4>(st, n, 3 * F, F, Bb[BB_A1], F, L.W2b, L.b2, Vin, 3 * F, PHI, 6 * F, nullptr, 0, status, PHIh);
    float* wst = (wstore && need_grad && !use_tc_bwd && !msg_mma) ? wstore + t * wstore_layer_floats : nullptr;
#define CTD_FWD(KPV) edge_fwd_kp<KPV>(st, m, t, n, arow, acol, ar, PHI, S, V, SM, VM, Bb[BB_VM], wst)
    if (n > 0) {
      StageGuard sg(STG_EDGE_FWD);
      if (msg_mma) {
        bad |= edge_fwd_mma(st, m, t, n, arow, acol, ar, PHIh, S, Vin, SM, VM, Bb[BB_VM], status);
      } else {
        CTD_KP_DISPATCH(m.KP, CTD_FWD)
      }
    }
#undef CTD_FWD
    bad |= gemm_bf16<0>(st, 3 * n, 2 * F, F, Bb[BB_VM], F, L.UVb, nullptr, nullptr, 0, nullptr, 2 * F, nullptr, 0,
                        status, UV);
    if (n > 0) { LaunchScope ls_(st); k_update_pre<__half><<<nb4, kThreads, 0, st>>>(n, F, m.eps, SM, UV, nullptr, Bb[BB_Z]); }
    bad |= gemm_bf16<1>(st, n, F, 2 * F, Bb[BB_Z], 2 * F, L.A1b, L.c1, nullptr, 0, nullptr, F, Bb[BB_A2], F, status,
                        H2);
    bad |= gemm_bf16<0>(st, n, 3 * F, F, Bb[BB_A2], F, L.A2b, L.c2, nullptr, 0, nullptr, 3 * F, nullptr, 0, status, AV);
    if (n > 0) {
      LaunchScope ls_(st);
      // the last layer's v and BF16 s feed nothing: only its FP32 s reaches the readout
      if (t + 1 < T)
        k_update_post<__half, true><<<nb4, kThreads, 0, st>>>(n, F, SM, VM, UV, AV, S, B[B_V0 + t + 1], Bb[BB_S0]);
      else
        k_update_post<__half, false><<<nb4, kThreads, 0, st>>>(n, F, SM, VM, UV, AV, S, nullptr, nullptr);
    }
  }
  // The readout MLP (F -> F/2 -> 1, ~1 % of the node FLOPs) stays in FP32: its output is the
  // per-atom energy itself, which BF16 operands would perturb by ~2^-9 of the readout terms.
  readout_fwd_bwd(st, m, n, B[B_S0], ew, need_grad, B, e_atom, energy_partials, n_energy_partials);
  if (!need_grad) return bad;
  if (n > 0) cudaMemsetAsync(B[B_GV], 0, sizeof(float) * (size_t)n * 3 * F, st);
  for (int t = T - 1; t >= 0; --t) {
    const LayerW& L = m.L[t];
    float *V = B[B_V0 + t], *PHI = phi32 ? B[B_PHI0 + t] : nullptr;
    const __half* H1 = reinterpret_cast<const __half*>(Bb[BB_H1H0 + t]);
    const __half* H2 = reinterpret_cast<const __half*>(Bb[BB_H2H0 + t]);
    const __half* UV = reinterpret_cast<const __half*>(Bb[BB_UVH0 + t]);
    const __half* AV = reinterpret_cast<const __half*>(Bb[BB_AVH0 + t]);
    float* T1 = B[B_T1];
    float *GS = B[B_GS], *GV = B[B_GV], *GSM = B[B_GSM], *GVM = B[B_GVM], *GPHI = B[B_GPHI];
    const __half* PHIh = phih(t);
    if (n > 0) { LaunchScope ls_(st); k_update_bwd_pre_bf16<<<nb, kThreads, 0, st>>>(n, F, GS, GV, UV, AV, Bb[BB_GA], Bb[BB_GUV]); }
    bad |= gemm_bf16<6>(st, n, F, 3 * F, Bb[BB_GA], 3 * F, L.A2tb, nullptr, nullptr, F, nullptr, 0, Bb[BB_GH2], F, status,
                        nullptr, nullptr, H2);
    bad |= gemm_bf16<0>(st, n, 2 * F, F, Bb[BB_GH2], F, L.A1tb, nullptr, nullptr, 0, T1, 2 * F, nullptr, 0, status);
    // the bulk-gathered tensor-core adjoint reads gsm and gvm interleaved per feature (G4)
    float* G4 = g4 ? B[B_G4] : nullptr;
    if (n > 0) { LaunchScope ls_(st); k_update_bwd_mid_bf16<<<nb4, kThreads, 0, st>>>(n, F, m.eps, GS, T1, UV, AV, GSM, Bb[BB_GUV]); }
    if (G4)   // gvm = gv + the U/V backward, written straight into G4 beside gsm
      bad |= gemm_bf16<5>(st, 3 * n, F, 2 * F, Bb[BB_GUV], 2 * F, L.UVtb, nullptr, GV, F, G4, F, nullptr, 0, status,
                          nullptr, GSM);
    else
      bad |= gemm_bf16<2>(st, 3 * n, F, 2 * F, Bb[BB_GUV], 2 * F, L.UVtb, nullptr, GV, F, GVM, F, nullptr, 0, status);
    const float* wst = (wstore && !use_tc_bwd && !msg_mma) ? wstore + t * wstore_layer_floats : nullptr;
    // first layer: no phi gradients, no phi backward (its inputs do not depend on positions)
    float* gphi = t > 0 ? GPHI : nullptr;
#define CTD_BWD(KPV) edge_bwd_kp<KPV>(st, m, t, t != T - 1, n, arow, acol, ar, PHI, GSM, GVM, gphi, hedge, wst)
    if (n > 0) {
      StageGuard sg(STG_EDGE_BWD);
      if (use_tc_bwd) {
        bad |= edge_bwd_tc(st, m, t, t != T - 1, n, arow, acol, ar, PHI, gphi, gphi ? Bb[BB_GP3] : nullptr, hedge,
                           status, aend, G4, phi32 ? nullptr : PHIh);
      } else {
        CTD_KP_DISPATCH(m.KP, CTD_BWD)
      }
    }
#undef CTD_BWD
    if (t == 0) break;
    if (n > 0) {
      LaunchScope ls_(st);
      if (use_tc_bwd)
        k_phi_bwd_psi<<<nb4, kThreads, 0, st>>>(n, F, GPHI, PHI, PHIh, V, reinterpret_cast<const float4*>(G4), GV,
                                                Bb[BB_GP3]);
      else
        k_phi_bwd_pre<<<nb, kThreads, 0, st>>>(n, F, GPHI, PHI, PHIh, V, GVM, nullptr, GV, Bb[BB_GP3]);
    }
    bad |= gemm_bf16<6>(st, n, F, 3 * F, Bb[BB_GP3], 3 * F, L.W2tb, nullptr, nullptr, F, nullptr, 0, Bb[BB_GH1], F,
                        status, nullptr, nullptr, H1);
    bad |= gemm_bf16<2>(st, n, F, F, Bb[BB_GH1], F, L.W1tb, nullptr, GSM, F, GS, F, nullptr, 0, status);
  }
  StageGuard fstage(STG_FORCES);
  { LaunchScope ls_(st); k_forces<<<n_virial_partials, kThreads, 0, st>>>(n, arow, ar, arev, hedge, force_s, virial_partials, status); }
  return bad;
}

}  // namespace ctd
