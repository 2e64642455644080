// ctd_internal.cuh -- internal declarations of the GB300 PaiNN engine (not part of the ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <cstddef>
#include <vector>

namespace ctd {

// ---------------------------------------------------------------- launch accounting / timing
// Every kernel launch is wrapped in a LaunchScope: it counts the launch under the current
// stage and, when profiling is on, brackets it with CUDA events on the launching stream.
enum Stage : int {
  STG_BUILD = 0, STG_PRUNE, STG_NODE, STG_EDGE_FWD, STG_EDGE_BWD, STG_FORCES, STG_MD, STG_MISC, STG_COUNT
};
struct ProfState {
  bool on = false;
  int stage = STG_MISC;
  double ms[STG_COUNT] = {};
  int64_t launches[STG_COUNT] = {};
  struct Rec { int stage; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  ~ProfState();
  void collect();            // waits for pending events and accumulates their times
};
void prof_bind(ProfState* p);   // bind the calling thread to a context's profiler (or null)
int prof_stage();
void prof_set_stage(int s);
bool prof_recording();                 // CUDA-event timing is on for the bound profiler
void prof_count_launches(int64_t k);   // add k launches (a graph replay) to the current stage
struct StageGuard {
  int prev;
  explicit StageGuard(int s) : prev(prof_stage()) { prof_set_stage(s); }
  ~StageGuard() { prof_set_stage(prev); }
};
struct LaunchScope {
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  explicit LaunchScope(cudaStream_t s);
  ~LaunchScope();
};

constexpr int kThreads = 256;
constexpr int kMaxT = 8;
constexpr int kMaxKP = 32;   // radial basis, padded to a multiple of 4

// Cell geometry for the neighbour build.  H rows are lattice vectors; G = H^{-T}.
struct CellGeom {
  double H[9];
  double G[9];
  int nc[3];      // cells (slabs) per lattice direction
  int M[3];       // neighbour slab half-range per direction
  double R2;      // (cutoff + skin)^2, rounded once in FP64
  int morton_bits;  // 0: cells numbered lexicographically; b > 0: Morton order on a 2^b grid
};

// Linear index of cell (c0, c1, c2).  Morton (Z-order) numbering keeps spatially close cells
// close in the cell-sorted atom order, so a block of consecutive rows is a compact region and
// its neighbours' features stay in L2.
__host__ __device__ __forceinline__ uint32_t morton_spread(uint32_t x) {
  x &= 0x3ffu;
  x = (x | (x << 16)) & 0x030000ffu;
  x = (x | (x << 8)) & 0x0300f00fu;
  x = (x | (x << 4)) & 0x030c30c3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}
__host__ __device__ __forceinline__ int cell_linear(const CellGeom& g, int c0, int c1, int c2) {
  if (g.morton_bits == 0) return (c0 * g.nc[1] + c1) * g.nc[2] + c2;
  return (int)(morton_spread((uint32_t)c0) | (morton_spread((uint32_t)c1) << 1) | (morton_spread((uint32_t)c2) << 2));
}

// Device-side status word, raised by kernels instead of trapping.
enum Status : int {
  ST_OK = 0,
  ST_REV_MISSING = 1,     // a reverse edge was not found
  ST_VERLET_OVERFLOW = 2, // more Verlet edges than capacity
  ST_NONFINITE = 4,
  ST_TIMEOUT = 8,         // a bounded device wait gave up
  ST_OWNERSHIP = 16,      // a spatial decomposition left an atom without exactly one owned copy
  ST_FP16_RANGE = 32,     // a value stored in FP16 (BF16 path) was outside the FP16 range
};

// FP32 weights of one interaction layer (device pointers).  "t" = transposed ([in][out]).
struct LayerW {
  const float *W1, *W1t, *b1;      // [F][F]
  const float *W2, *W2t, *b2;      // [3F][F], [F][3F]
  const float *Wf, *bf;            // [3F][KP] (zero padded), [3F]
  const float *UV, *UVt;           // [2F][F] = [U;V], [F][2F] = [U^T | V^T]
  const float *A1, *A1t, *c1;      // [F][2F], [2F][F]
  const float *A2, *A2t, *c2;      // [3F][F], [F][3F]
  // BF16 copies for the tensor-core path (same shapes as the FP32 arrays above)
  const __nv_bfloat16 *W1b, *W1tb, *W2b, *W2tb, *UVb, *UVtb, *A1b, *A1tb, *A2b, *A2tb;
  const __nv_bfloat16* Wfb;        // [3F][64] radial filter, zero padded (tensor-core edge kernels)
  const __half* Wfh;               // the same in FP16 (the tensor-core adjoint's filter operand)
};

struct ModelW {
  int F, K, KP, T, S;
  float rc, eps, e_scale;
  const float* emb;                // [S][F]
  LayerW L[kMaxT];
  const float *R1, *R1t, *d1, *R2, *d2;   // [F/2][F], [F][F/2]
  const __nv_bfloat16 *R1b, *R1tb;
  bool tc_adjoint;                 // BF16 path, F = 128: edge adjoint with the tensor-core filter
  bool edge_store;                 // store per-edge filters in the forward pass for the adjoint
  bool tc_message;                 // BF16 path, F = 128: message step as the tensor-core contraction (edge_mma.cu)
  int64_t edge_chunk_rows;         // tensor-core adjoint: rows per chunk (0: one range per stream)
};

// Strictly local equivariant edge model (model_local.cu): FP32 weights on the device, matrices
// [in][out] as the GEMMs' B operand and their transposes for the adjoint; A0 zero-padded to KA
// rows (K + 2S rounded up to a multiple of 4).
struct LocalLayerW {
  const float *Q, *Qt, *M, *Mt, *m;      // [F][2C], [2C][F], [F+2C][F], [F][F+2C], [F]
  const float *Gs, *Gst, *Gv, *Gvt;      // [2C][C], [C][2C] (layers l < L)
};
// BF16 copies of the local model's weights for the tensor-core GEMM (C = A W^T, W [N][K]):
// forward W = the [out][in] matrices, backward W = the [in][out] ones; K below 64 is zero-padded
// to 64 columns (KAb for the two-body input, 64 for the 2C- and F/2-wide gradients).
struct LocalWb {
  const __nv_bfloat16 *A0t, *P0t, *R1t, *A0, *P0, *R1;   // [F][KAb], [2C][F], [F/2][F], [KA][F], [F][64], [F][Kh]
  const __nv_bfloat16 *Qt[kMaxT], *Mt[kMaxT], *Q[kMaxT], *M[kMaxT];   // [2C][F], [F][F+2C], [F][64], [F+2C][F]
};
struct LocalW {
  int F, K, KA, L, S, C;
  float rc, e_scale;
  const float *A0, *A0t, *c0, *P0, *P0t;  // [KA][F], [F][KA], [F], [F][2C], [2C][F]
  LocalLayerW Lw[kMaxT];
  const float *R1, *R1t, *d1, *R2, *d2;   // [F][F/2], [F/2][F], [F/2], [F/2], [1]
  bool bf16 = false;                      // BF16 path: the edge GEMMs on tcgen05 (weights wb)
  int KAb = 0, Kh = 0;                    // padded K of the two-body input and of the F/2 gradient
  LocalWb wb{};
};
// Width of the two-body input rows: K + 2S rounded up to 4 (FP32) or to 32 (BF16, where it is a
// GEMM output width in the adjoint).
inline int local_ka(int K, int S, bool bf16) { return bf16 ? (K + 2 * S + 31) / 32 * 32 : (K + 2 * S + 3) / 4 * 4; }
// Device floats the local model needs for n atoms and E active edges.
int64_t local_buffer_floats(const LocalW& w, int64_t n, int64_t E);
// Energy partials, per-atom energies, and (need_grad) hedge = -dE/dr_e per active edge.  Nonzero
// if the BF16 path's GEMM rejected a shape (nothing is computed wrongly: the call fails).
int local_forward_backward(cudaStream_t st, const LocalW& w, int64_t n, int64_t E, const int32_t* species_s,
                           const int32_t* arow, const int32_t* acol, const float4* ar, float* buf,
                           bool need_grad, const float* ew, double* energy_partials, int n_energy_partials,
                           float* e_atom, float4* hedge, int* status);
// Forces F_i = sum_{e in row i} (hedge[rev e] - hedge[e]) and virial partials sum_e r_e (x) hedge[e].
void launch_forces(cudaStream_t st, int64_t n, const int32_t* arow, const float4* ar, const int32_t* arev,
                   const float4* hedge, float* force, double* vpart, int n_vpart, int* status);
// out = A B (+ epilogue) with the FP32 SIMT GEMM: epi 0 bias (may be null), 1 bias + silu into
// out2, 2 out = A B + aux (aux and out must not overlap), 3 out = (A B) * silu'(aux).
void gemm_f32(cudaStream_t st, int epi, int64_t M, int N, int K, const float* A, int lda, const float* B,
              const float* bias, const float* aux, int ldaux, float* out, int ldo, float* out2, int ldo2);

// ---------------------------------------------------------------- small device helpers
// SiLU and its derivative for FP32 results.  expf (not __expf): the fast exponential's error
// grows with |x| and is the same for the same input, so in a crystal, where every atom sees the
// same activations, it would add up coherently over the atoms' energies.
__device__ __forceinline__ float silu_f(float x) { return x / (1.0f + expf(-x)); }
__device__ __forceinline__ float dsilu_f(float x) {
  float s = 1.0f / (1.0f + expf(-x));
  return s * (1.0f + x * (1.0f - s));
}
// Approximate-division forms for epilogues whose result is rounded to BF16 (relative error of
// the division ~2 ulp of FP32, far below BF16's 2^-9; both tend to the right limits for large
// |x|: __fdividef returns 0 once the denominator exceeds 2^126).
__device__ __forceinline__ float silu_fast(float x) { return __fdividef(x, 1.0f + __expf(-x)); }
__device__ __forceinline__ float dsilu_fast(float x) {
  const float s = __fdividef(1.0f, 1.0f + __expf(-x));
  return s * (1.0f + x * (1.0f - s));
}

// ---------------------------------------------------------------- launchers (host side)
// neighbors.cu
void launch_wrap_bin(cudaStream_t st, int64_t n, const double* x_user, const CellGeom& g,
                     double* xw, int32_t* wrapm, int32_t* cell, int32_t* cell_count);
void launch_place(cudaStream_t st, int64_t n, const int32_t* cell, const int32_t* cell_start,
                  int32_t* cursor, int32_t* tmp_idx);
void launch_sort_cells(cudaStream_t st, int64_t ncell, const int32_t* cell_start,
                       const int32_t* tmp_idx, int32_t* perm);
void launch_gather_sorted(cudaStream_t st, int64_t n, const int32_t* perm, const double* xw,
                          const double* x_user, const int32_t* species_user, double* xw_s,
                          double* xref_s, int32_t* species_s, int32_t* inv_perm);
void launch_pair_search(cudaStream_t st, bool fill, int64_t n, const double* xw_s,
                        const int32_t* cell_start, const CellGeom& g, int32_t* count,
                        const int32_t* row_ptr, int32_t* col, uint32_t* img, float4* base);
void launch_reverse(cudaStream_t st, int64_t n, const int32_t* row_ptr, const int32_t* col,
                    const uint32_t* img, int32_t* rev, int* status);
void launch_delta(cudaStream_t st, int64_t n, const double* x_s, const double* xref_s,
                  float4* delta, unsigned int* maxdisp2_bits);
void launch_gather_positions(cudaStream_t st, int64_t n, const int32_t* perm, const double* x_user,
                             double* x_s);
void launch_prune(cudaStream_t st, bool fill, int64_t n, const int32_t* vrow, const int32_t* vcol,
                  const float4* vbase, const float4* delta, float rc2, const uint8_t* near, int32_t* acount,
                  const int32_t* arow, int32_t* acol, float4* ar, int32_t* vidx, int32_t* v2a);
void launch_prune_rev(cudaStream_t st, int64_t n, const int32_t* arow, const int32_t* vidx,
                      const int32_t* vrev, const int32_t* v2a, int32_t* arev,
                      int32_t* aend);
// scan.cu
size_t scan_temp_bytes(int64_t n);
void launch_exclusive_scan(cudaStream_t st, int64_t n, const int32_t* in, int32_t* out,
                           void* temp);   // out has n+1 entries; out[n] = total
// md.cu
void launch_kick_drift(cudaStream_t st, int64_t n, double dt, const float* f, const double* m, const double* vscale,
                       double* x, double* v);
// Nose-Hoover chain thermostat (md.cu)
struct NhcParams {
  int M;          // chain length (1..16)
  double kT, Nf;  // target kB T (eV), degrees of freedom
  double Q[16];   // thermostat masses (eV fs^2)
};
void launch_nhc_half(cudaStream_t st, const NhcParams& p, double h, const double* ke, double* state);
void launch_nhc_energy(cudaStream_t st, const NhcParams& p, const double* state, double* out);
void launch_scale_v(cudaStream_t st, int64_t n, const double* g, double* v);
void launch_rep_nhc_half(cudaStream_t st, int R, const NhcParams* params, double h, const double* ke, int ke_stride,
                         const int32_t* flags, double* states, int state_stride, double* g, double* ke_after,
                         double* eth);
void launch_scale_v_rep(cudaStream_t st, int64_t n, const int32_t* rep, const double* g, double* v);
void launch_kick(cudaStream_t st, int64_t n, double dt, const float* f, const double* m, double* v);
void launch_kinetic(cudaStream_t st, int64_t n, const double* m, const double* v, double* partials, int nb);
void launch_sum_partials(cudaStream_t st, int nb, int width, const double* partials, double* out, double scale);
void launch_scatter_rows(cudaStream_t st, int64_t n, int w, const int32_t* perm, const float* in, double* out);
void launch_scatter_rows_d(cudaStream_t st, int64_t n, int w, const int32_t* perm, const double* in, double* out);
void launch_gather_rows_d(cudaStream_t st, int64_t n, int w, const int32_t* perm, const double* in, double* out);
void launch_gather_i32(cudaStream_t st, int64_t n, const int32_t* perm, const int32_t* in, int32_t* out);
void launch_check_finite(cudaStream_t st, int64_t n, const double* a, int* status);
// gemm_bf16.cu: C[M][N] = A[M][K] . W[N][K]^T on tcgen05 (BF16 in, FP32 accumulate), epilogue
// EPI 0 bias, 1 bias + SiLU (bf16 copy gets the SiLU; outh: FP16 copy of the argument), 2 + aux,
// 3 * SiLU'(aux), 4 PHI packing,
// 5 + aux written as the interleaved (aux2, rows 3i..3i+2) quads of the adjoint's G4,
// 6 * SiLU'(auxh), the argument stored in FP16.
bool gemm_bf16_supported(int N, int K);
bool make_tmap_bf16(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows);
// edge_tc.cu: tensor-core edge adjoint (F = 128, K <= 31); G4 = the receivers' (gsm, gvm)
// interleaved per feature; GPHI [n][3F] gets the psi gradients and GP3b [n][3F] the BF16 phi_s
// and phi_vs gradients (blocks 0 and 2), both null on the first layer
bool edge_tc_supported(int F, int K);
int edge_bwd_tc(cudaStream_t st, const ModelW& m, int t, int accumulate, int64_t n, const int32_t* arow,
                const int32_t* acol, const float4* ar, const float* PHI, float* GPHI, __nv_bfloat16* GP3b,
                float4* hedge, int* status, const int32_t* aend, const float* G4, const __half* PHIh = nullptr);
// edge_mma.cu: the message step as a tensor-core contraction over each receiver's edges
// (F = 128, K < 32): gathered FP16 message rows x per-edge basis, FP32 filter weights after it.
bool edge_mma_supported(int F, int K);
int edge_fwd_mma(cudaStream_t st, const ModelW& m, int t, int64_t n, const int32_t* arow, const int32_t* acol,
                 const float4* ar, const __half* PHIh, const float* S, const float* V, float* SM, float* VM,
                 __nv_bfloat16* VMb, int* status);
template <int EPI>
int gemm_bf16(cudaStream_t st, int64_t M, int N, int K, const __nv_bfloat16* A, int64_t lda,
              const __nv_bfloat16* W, const float* bias, const float* aux, int ldaux, float* out, int ldo,
              __nv_bfloat16* outb, int ldob, int* status, __half* outh = nullptr, const float* aux2 = nullptr,
              const __half* auxh = nullptr);
// model_fp32.cu
int model_buffer_count();
bool model_uses_g4(const ModelW& m, int precision);
bool model_phi_fp16_only(const ModelW& m, int precision);
int64_t model_buffer_floats_per_atom(int b, const ModelW& m, int F, int T, int precision);
int model_bf16_buffer_count();
bool model_uses_msg_mma(const ModelW& m);
bool model_stores_edges(const ModelW& m, int precision);
int64_t model_bf16_buffer_elems_per_atom(int b, int F, int T, bool msg_mma);
int model_forward_backward_bf16(cudaStream_t st, const ModelW& m, int64_t n, const int32_t* species_s,
                                const int32_t* arow, const int32_t* acol, const float4* ar, const int32_t* arev,
                                float* const* bufs, __nv_bfloat16* const* bbufs, bool need_grad,
                                double* energy_partials, int n_energy_partials, float4* hedge, float* force_s,
                                double* virial_partials, int n_virial_partials, float* e_atom, int* status,
                                float* wstore, int64_t wstore_layer_floats, const int32_t* aend,
                                const float* ew);
void model_forward_backward_fp32(cudaStream_t st, const ModelW& m, int64_t n, const int32_t* species_s,
                                 const int32_t* arow, const int32_t* acol, const float4* ar,
                                 const int32_t* arev, float* const* bufs, bool need_grad,
                                 double* energy_partials, int n_energy_partials, float4* hedge,
                                 float* force_s, double* virial_partials, int n_virial_partials,
                                 float* e_atom, int* status, float* wstore, int64_t wstore_layer_floats,
                                 const float* ew);
}  // namespace ctd
