// api.cu -- the C ABI (include/painn.h): context, grow-only device buffers under an HBM budget,
// parameter loading, neighbour build / prune orchestration, energy-force-virial calls and
// the resident NVE loop.
//
// Buffering follows arXiv 2506.04055, Results "Runtime optimizations and buffering": inputs are
// held in device buffers with capacities that only grow, so shapes settle once a run reaches
// equilibrium; a call that needs more room grows the buffer (within the HBM budget) and
// proceeds, and the neighbour list is rebuilt only when an atom has moved more than half the
// skin since the last build.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.cuh"

using namespace ctd;

namespace ctd {

// The library always carries the tensor-core kernels (sm_103a), so the BF16 path is available.
bool bf16_available() { return true; }

// Host float -> bf16, round to nearest even (NaN kept quiet).
uint16_t to_bf16_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

}  // namespace ctd

namespace ctd {

int fail(ctd_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}



static void note_need(ctd_ctx* c, DBuf& b, size_t bytes) {
  c->used = c->used - b.need + bytes;
  b.need = bytes;
}

// Grow-only allocation with 25 % headroom, charged against the budget.
int ensure(ctd_ctx* c, DBuf& b, size_t bytes) {
  if (bytes <= b.bytes) {
    note_need(c, b, bytes);
    return CTD_OK;
  }
  if (c->capturing) return fail(c, CTD_ERR_STATE, "a buffer would grow during graph capture");
  ++c->alloc_gen;
  size_t want = bytes + bytes / 4 + 256;
  want = (want + 255) & ~(size_t)255;
  if (c->budget && c->held - b.bytes + want > c->budget) {
    want = bytes;
    if (c->held - b.bytes + want > c->budget)
      return fail(c, CTD_ERR_OUT_OF_BUDGET,
                  "device buffer of " + std::to_string(bytes) + " bytes exceeds the HBM budget (" +
                      std::to_string(c->budget) + " bytes, " + std::to_string(c->held) + " held)");
  }
  if (b.p) {
    cudaStreamSynchronize(c->st);
    cudaFree(b.p);
    c->held -= b.bytes;
    c->used -= b.need;
    b.p = nullptr;
    b.bytes = 0;
    b.need = 0;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? CTD_ERR_OUT_OF_BUDGET : CTD_ERR_CUDA,
                std::string("cudaMalloc(") + std::to_string(want) + ") -> " + cudaGetErrorString(e));
  }
  b.p = p;
  b.bytes = want;
  c->held += want;
  note_need(c, b, bytes);
  return CTD_OK;
}




// G = H^{-T} by cofactors, the expression order of the canonical pair test (every product and
// difference rounded on its own; this file is compiled without floating-point contraction).
void inv_transpose(const double H[9], double G[9]) {
  volatile double c[9];
  c[0] = H[4] * H[8] - H[5] * H[7];
  c[1] = H[5] * H[6] - H[3] * H[8];
  c[2] = H[3] * H[7] - H[4] * H[6];
  c[3] = H[2] * H[7] - H[1] * H[8];
  c[4] = H[0] * H[8] - H[2] * H[6];
  c[5] = H[1] * H[6] - H[0] * H[7];
  c[6] = H[1] * H[5] - H[2] * H[4];
  c[7] = H[2] * H[3] - H[0] * H[5];
  c[8] = H[0] * H[4] - H[1] * H[3];
  double det = (H[0] * c[0] + H[1] * c[1]) + H[2] * c[2];
  for (int k = 0; k < 9; ++k) G[k] = c[k] / det;
}

bool finite_cell(const double H[9]) {
  for (int k = 0; k < 9; ++k)
    if (!std::isfinite(H[k])) return false;
  double det = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
               H[2] * (H[3] * H[7] - H[4] * H[6]);
  return std::fabs(det) > 1e-9;
}

int setup_geometry_into(ctd_ctx* c, CellGeom& g, int64_t* ncell_out, const double H[9], double R) {
  memcpy(g.H, H, sizeof(double) * 9);
  inv_transpose(H, g.G);
  int64_t ncell = 1;
  for (int a = 0; a < 3; ++a) {
    double w = 1.0 / std::sqrt(g.G[3 * a] * g.G[3 * a] + g.G[3 * a + 1] * g.G[3 * a + 1] +
                               g.G[3 * a + 2] * g.G[3 * a + 2]);
    int nc = (int)std::floor(w / (R * (1.0 + 1e-6)));
    if (nc < 1) nc = 1;
    if (nc > 1024) nc = 1024;
    g.nc[a] = nc;
    g.M[a] = (int)std::ceil(R * nc * (1.0 + 1e-6) / w);
    if (g.M[a] > 100)
      return fail(c, CTD_ERR_CELL_TOO_SMALL, "cell thinner than cutoff/100 along a lattice direction");
    ncell *= nc;
  }
  g.R2 = R * R;
  // Morton numbering when the padded 2^b grid stays within 8x the cell count
  int mx = std::max(g.nc[0], std::max(g.nc[1], g.nc[2]));
  int bits = 0;
  while ((1 << bits) < mx) ++bits;
  const int64_t mcells = (int64_t)1 << (3 * bits);
  g.morton_bits = 0;
  if (bits > 0 && bits <= 9 && mcells <= std::max<int64_t>(8 * ncell, 4096)) {
    g.morton_bits = bits;
    ncell = mcells;
  }
  *ncell_out = ncell;
  return CTD_OK;
}

int setup_geometry(ctd_ctx* c, const double H[9], double R) {
  return setup_geometry_into(c, c->geom, &c->ncell, H, R);
}

int check_status(ctd_ctx* c) {
  int st = 0;
  CUDA_OK(c, cudaMemcpyAsync(&st, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  if (st & ST_REV_MISSING) return fail(c, CTD_ERR_CAPACITY, "reverse edge missing in the neighbour list");
  if (st & ST_FP16_RANGE)
    return fail(c, CTD_ERR_NONFINITE,
                "an activation stored in FP16 (message table, U/V products, update coefficients or SiLU arguments) "
                "is outside "
                "the FP16 range; the FP32 path keeps them in FP32");
  if (st & ST_NONFINITE) return fail(c, CTD_ERR_NONFINITE, "non-finite value in positions or results");
  if (st & ST_TIMEOUT) return fail(c, CTD_ERR_TIMEOUT, "a bounded device wait gave up");
  if (st & ST_OWNERSHIP) return fail(c, CTD_ERR_STATE, "domain decomposition: an atom is not owned exactly once");
  return CTD_OK;
}

// Build the Verlet list from positions already in c->x_user (device, caller order).
int build_from_device_positions(ctd_ctx* c, int64_t n, const double H[9], double cutoff, double skin) {
  if (!finite_cell(H)) return fail(c, CTD_ERR_INVALID_ARG, "cell is singular or not finite");
  if (!(cutoff > 0.0) || !(skin >= 0.0)) return fail(c, CTD_ERR_INVALID_ARG, "cutoff must be > 0, skin >= 0");
  // a build that fails below leaves no list behind, so the next call builds again
  c->have_list = false;
  int r = setup_geometry(c, H, cutoff + skin);
  if (r) return r;
  StageGuard sg(STG_BUILD);
  cudaStream_t st = c->st;
  const int64_t n1 = n > 0 ? n : 1;
  ENSURE(c, c->xw, sizeof(double) * 3 * n1);
  ENSURE(c, c->wrapm, sizeof(int32_t) * 3 * n1);
  ENSURE(c, c->cellid, sizeof(int32_t) * n1);
  ENSURE(c, c->cell_count, sizeof(int32_t) * (c->ncell + 1));
  ENSURE(c, c->cell_start, sizeof(int32_t) * (c->ncell + 1));
  ENSURE(c, c->cursor, sizeof(int32_t) * (c->ncell + 1));
  ENSURE(c, c->tmp_idx, sizeof(int32_t) * n1);
  ENSURE(c, c->perm, sizeof(int32_t) * n1);
  ENSURE(c, c->inv_perm, sizeof(int32_t) * n1);
  ENSURE(c, c->xw_s, sizeof(double) * 3 * n1);
  ENSURE(c, c->xref_s, sizeof(double) * 3 * n1);
  ENSURE(c, c->x_s, sizeof(double) * 3 * n1);
  ENSURE(c, c->z_s, sizeof(int32_t) * n1);
  ENSURE(c, c->count, sizeof(int32_t) * n1);
  ENSURE(c, c->vrow, sizeof(int32_t) * (n1 + 1));
  ENSURE(c, c->status, sizeof(int32_t) * 4);
  ENSURE(c, c->scan_tmp, scan_temp_bytes(std::max<int64_t>(n1, c->ncell)) + 64);
  CUDA_OK(c, cudaMemsetAsync(c->status.p, 0, sizeof(int32_t), st));
  // non-finite positions are reported (CTD_ERR_NONFINITE) instead of being binned: the binning
  // clamps their cell index, so they would silently find no neighbours
  launch_check_finite(st, 3 * n, P<double>(c->x_user), P<int>(c->status));
  CUDA_OK(c, cudaMemsetAsync(c->cell_count.p, 0, sizeof(int32_t) * c->ncell, st));
  CUDA_OK(c, cudaMemsetAsync(c->cursor.p, 0, sizeof(int32_t) * c->ncell, st));
  launch_wrap_bin(st, n, P<double>(c->x_user), c->geom, P<double>(c->xw), P<int32_t>(c->wrapm),
                  P<int32_t>(c->cellid), P<int32_t>(c->cell_count));
  launch_exclusive_scan(st, c->ncell, P<int32_t>(c->cell_count), P<int32_t>(c->cell_start), c->scan_tmp.p);
  launch_place(st, n, P<int32_t>(c->cellid), P<int32_t>(c->cell_start), P<int32_t>(c->cursor), P<int32_t>(c->tmp_idx));
  launch_sort_cells(st, c->ncell, P<int32_t>(c->cell_start), P<int32_t>(c->tmp_idx), P<int32_t>(c->perm));
  launch_gather_sorted(st, n, P<int32_t>(c->perm), P<double>(c->xw), P<double>(c->x_user), nullptr,
                       P<double>(c->xw_s), P<double>(c->xref_s), nullptr, P<int32_t>(c->inv_perm));
  launch_pair_search(st, false, n, P<double>(c->xw_s), P<int32_t>(c->cell_start), c->geom, P<int32_t>(c->count),
                     nullptr, nullptr, nullptr, nullptr);
  launch_exclusive_scan(st, n, P<int32_t>(c->count), P<int32_t>(c->vrow), c->scan_tmp.p);
  int32_t total = 0;
  CUDA_OK(c, cudaMemcpyAsync(&total, P<int32_t>(c->vrow) + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CUDA_OK(c, cudaStreamSynchronize(st));
  CUDA_OK(c, cudaGetLastError());
  if (total < 0) return fail(c, CTD_ERR_CAPACITY, "more than 2^31 neighbour pairs");
  const int64_t e1 = total > 0 ? total : 1;
  ENSURE(c, c->vcol, sizeof(int32_t) * e1);
  ENSURE(c, c->vimg, sizeof(uint32_t) * e1);
  ENSURE(c, c->vbase, sizeof(float4) * e1);
  ENSURE(c, c->vrev, sizeof(int32_t) * e1);
  ENSURE(c, c->v2a, sizeof(int32_t) * e1);
  launch_pair_search(st, true, n, P<double>(c->xw_s), P<int32_t>(c->cell_start), c->geom, P<int32_t>(c->count),
                     P<int32_t>(c->vrow), P<int32_t>(c->vcol), P<uint32_t>(c->vimg), P<float4>(c->vbase));
  launch_reverse(st, n, P<int32_t>(c->vrow), P<int32_t>(c->vcol), P<uint32_t>(c->vimg), P<int32_t>(c->vrev),
                 P<int>(c->status));
  CUDA_OK(c, cudaGetLastError());
  r = check_status(c);
  if (r) return r;
  c->n = n;
  c->n_verlet = total;
  memcpy(c->H, H, sizeof(double) * 9);
  c->cutoff = cutoff;
  c->skin = skin;
  c->have_list = true;
  c->last_maxdisp = 0.0;
  return CTD_OK;
}

int copy_in(ctd_ctx* c, void* dst, const void* src, size_t bytes, bool device) {
  if (bytes == 0) return CTD_OK;
  CUDA_OK(c, cudaMemcpyAsync(dst, src, bytes, device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st));
  return CTD_OK;
}

// Per-step prune of the Verlet list to the active list (positions already in c->x_s, sorted).
int prune(ctd_ctx* c, double* maxdisp_out) {
  StageGuard sg(STG_PRUNE);
  cudaStream_t st = c->st;
  const int64_t n = c->n, n1 = n > 0 ? n : 1, e1 = c->n_verlet > 0 ? c->n_verlet : 1;
  ENSURE(c, c->delta, sizeof(float4) * n1);
  ENSURE(c, c->maxd, sizeof(unsigned int) * 4);
  ENSURE(c, c->acount, sizeof(int32_t) * n1);
  ENSURE(c, c->arow, sizeof(int32_t) * (n1 + 1));
  ENSURE(c, c->acol, sizeof(int32_t) * e1);
  ENSURE(c, c->ar, sizeof(float4) * e1);
  ENSURE(c, c->vidx, sizeof(int32_t) * e1);
  ENSURE(c, c->arev, sizeof(int32_t) * e1);
  ENSURE(c, c->aend, sizeof(int32_t) * e1);
  CUDA_OK(c, cudaMemsetAsync(c->maxd.p, 0, sizeof(unsigned int), st));
  launch_delta(st, n, P<double>(c->x_s), P<double>(c->xref_s), P<float4>(c->delta), P<unsigned int>(c->maxd));
  if (maxdisp_out) {
    unsigned int bits = 0;
    CUDA_OK(c, cudaMemcpyAsync(&bits, c->maxd.p, sizeof(bits), cudaMemcpyDeviceToHost, st));
    CUDA_OK(c, cudaStreamSynchronize(st));
    float d2;
    memcpy(&d2, &bits, sizeof(d2));
    *maxdisp_out = std::sqrt((double)d2);
  }
  const float rc2 = (float)(c->desc.rc * c->desc.rc);
  const uint8_t* near = c->use_near ? P<uint8_t>(c->near) : nullptr;
  launch_prune(st, false, n, P<int32_t>(c->vrow), P<int32_t>(c->vcol), P<float4>(c->vbase), P<float4>(c->delta),
               rc2, near, P<int32_t>(c->acount), nullptr, nullptr, nullptr, nullptr, nullptr);
  launch_exclusive_scan(st, n, P<int32_t>(c->acount), P<int32_t>(c->arow), c->scan_tmp.p);
  launch_prune(st, true, n, P<int32_t>(c->vrow), P<int32_t>(c->vcol), P<float4>(c->vbase), P<float4>(c->delta),
               rc2, near, P<int32_t>(c->acount), P<int32_t>(c->arow), P<int32_t>(c->acol), P<float4>(c->ar),
               P<int32_t>(c->vidx), P<int32_t>(c->v2a));
  launch_prune_rev(st, n, P<int32_t>(c->arow), P<int32_t>(c->vidx), P<int32_t>(c->vrev), P<int32_t>(c->v2a),
                   P<int32_t>(c->arev), P<int32_t>(c->aend));
  CUDA_OK(c, cudaGetLastError());
  return CTD_OK;
}

// Device bytes per atom of the model's activation buffers (FP32 and, on the BF16 path, the
// BF16 operand copies), as evaluate() allocates them.
size_t model_bytes_per_atom(const ctd_ctx* c) {
  const int F = c->desc.F, T = c->desc.T;
  if (c->local()) {   // per-edge arrays at 64 active edges per atom (water and fcc at rc = 5 A: ~50)
    LocalW w = c->lw;
    w.F = F; w.L = T; w.C = c->desc.channels; w.S = c->desc.n_species;
    w.bf16 = c->desc.precision == CTD_PREC_BF16;
    w.KA = local_ka(c->desc.K, w.S, w.bf16);
    w.KAb = w.KA < 64 ? 64 : w.KA;
    w.Kh = F / 2 < 64 ? 64 : F / 2;
    return sizeof(float) * (size_t)local_buffer_floats(w, 1, 64);
  }
  size_t bytes = 0;
  for (int b = 0; b < model_buffer_count(); ++b)
    bytes += sizeof(float) * (size_t)model_buffer_floats_per_atom(b, c->mw, F, T, c->desc.precision);
  if (c->desc.precision == CTD_PREC_BF16)
    for (int b = 0; b < model_bf16_buffer_count(); ++b)
      bytes += sizeof(__nv_bfloat16) * (size_t)model_bf16_buffer_elems_per_atom(b, F, T, model_uses_msg_mma(c->mw));
  return bytes;
}

// Model evaluation on the current active list; forces (sorted, FP32) in c->force_s,
// energy in c->out_e[0], virial in c->out_w[0..8], per-atom energies (sorted) in c->eatom.
// The strictly local model: edge arrays sized by this step's active edge count.
int evaluate_local(ctd_ctx* c, bool need_grad) {
  cudaStream_t st = c->st;
  const int64_t n = c->n, n1 = n > 0 ? n : 1, e1 = c->n_verlet > 0 ? c->n_verlet : 1;
  int32_t act = 0;
  if (n > 0) {
    CUDA_OK(c, cudaMemcpyAsync(&act, P<int32_t>(c->arow) + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CUDA_OK(c, cudaStreamSynchronize(st));
  }
  const int64_t E = act;
  ENSURE(c, c->lbuf, sizeof(float) * (size_t)local_buffer_floats(c->lw, n1, E > 0 ? E : 1));
  ENSURE(c, c->hedge, sizeof(float4) * e1);
  ENSURE(c, c->force_s, sizeof(float) * 3 * n1);
  ENSURE(c, c->eatom, sizeof(float) * n1);
  ENSURE(c, c->epart, sizeof(double) * kPartials);
  ENSURE(c, c->vpart, sizeof(double) * 9 * kPartials);
  ENSURE(c, c->out_e, sizeof(double) * 4);
  ENSURE(c, c->out_w, sizeof(double) * 9);
  const float* ew = c->use_ew ? P<float>(c->ew) : nullptr;
  c->last_stored = false;
  ENSURE(c, c->status, sizeof(int32_t) * 4);
  const int bad = local_forward_backward(st, c->lw, n, E, P<int32_t>(c->z_s), P<int32_t>(c->arow),
                                         P<int32_t>(c->acol), P<float4>(c->ar), P<float>(c->lbuf), need_grad, ew,
                                         P<double>(c->epart), kPartials, P<float>(c->eatom), P<float4>(c->hedge),
                                         P<int>(c->status));
  if (bad) return fail(c, CTD_ERR_INVALID_ARG, "local model, BF16 path: unsupported GEMM shape");
  StageGuard sg(STG_FORCES);
  if (need_grad) {
    if (E == 0) CUDA_OK(c, cudaMemsetAsync(c->hedge.p, 0, sizeof(float4), st));
    launch_forces(st, n, P<int32_t>(c->arow), P<float4>(c->ar), P<int32_t>(c->arev), P<float4>(c->hedge),
                  P<float>(c->force_s), P<double>(c->vpart), kPartials, P<int>(c->status));
  }
  launch_sum_partials(st, kPartials, 1, P<double>(c->epart), P<double>(c->out_e), 1.0);
  if (need_grad) launch_sum_partials(st, kPartials, 9, P<double>(c->vpart), P<double>(c->out_w), 1.0);
  CUDA_OK(c, cudaGetLastError());
  return CTD_OK;
}

int evaluate(ctd_ctx* c, bool need_grad) {
  if (c->local()) return evaluate_local(c, need_grad);
  cudaStream_t st = c->st;
  const int64_t n = c->n, n1 = n > 0 ? n : 1, e1 = c->n_verlet > 0 ? c->n_verlet : 1;
  const int F = c->desc.F, T = c->desc.T;
  const int nb = model_buffer_count();
  if ((int)c->mbuf.size() < nb) c->mbuf.resize(nb);
  std::vector<float*> ptrs(nb, nullptr);
  for (int b = 0; b < nb; ++b) {
    int64_t per = model_buffer_floats_per_atom(b, c->mw, F, T, c->desc.precision);
    if (per == 0) continue;
    size_t bytes = sizeof(float) * (size_t)per * (size_t)n1;
    ENSURE(c, c->mbuf[b], bytes);
    ptrs[b] = P<float>(c->mbuf[b]);
  }
  ENSURE(c, c->hedge, sizeof(float4) * e1);
  ENSURE(c, c->force_s, sizeof(float) * 3 * n1);
  ENSURE(c, c->eatom, sizeof(float) * n1);
  ENSURE(c, c->epart, sizeof(double) * kPartials);
  ENSURE(c, c->vpart, sizeof(double) * 9 * kPartials);
  ENSURE(c, c->out_e, sizeof(double) * 4);
  ENSURE(c, c->out_w, sizeof(double) * 9);
  if (T == 0) CUDA_OK(c, cudaMemsetAsync(c->hedge.p, 0, sizeof(float4) * e1, st));
  const float* ew = c->use_ew ? P<float>(c->ew) : nullptr;
  // Edge filters stored for the adjoint when asked for and when they fit: within the HBM
  // budget if one is set, and within 80 % of the device's free memory; recomputed otherwise.
  float* wst = nullptr;
  const int64_t wlayer = e1 * 6 * (int64_t)F;
  c->last_stored = false;
  if (model_stores_edges(c->mw, c->desc.precision) && need_grad && T > 0) {
    const size_t want = sizeof(float) * (size_t)wlayer * (size_t)T;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const bool fits_budget = !c->budget || c->held - c->wstore.bytes + want <= c->budget;
    const bool fits_device = want <= c->wstore.bytes || (double)want <= 0.8 * (double)(free_b + c->wstore.bytes);
    if (fits_budget && fits_device) {
      ENSURE(c, c->wstore, want);
      wst = P<float>(c->wstore);
      c->last_stored = true;
    }
  }
  if (c->desc.precision == CTD_PREC_BF16) {
    const int nbb = model_bf16_buffer_count();
    if ((int)c->mbufb.size() < nbb) c->mbufb.resize(nbb);
    std::vector<__nv_bfloat16*> bptrs(nbb, nullptr);
    for (int b = 0; b < nbb; ++b) {
      int64_t per = model_bf16_buffer_elems_per_atom(b, F, T, model_uses_msg_mma(c->mw));
      if (per == 0) continue;
      ENSURE(c, c->mbufb[b], sizeof(__nv_bfloat16) * (size_t)per * (size_t)n1);
      bptrs[b] = P<__nv_bfloat16>(c->mbufb[b]);
    }
    int bad = model_forward_backward_bf16(st, c->mw, n, P<int32_t>(c->z_s), P<int32_t>(c->arow), P<int32_t>(c->acol),
                                          P<float4>(c->ar), P<int32_t>(c->arev), ptrs.data(), bptrs.data(), need_grad,
                                          P<double>(c->epart), kPartials, P<float4>(c->hedge), P<float>(c->force_s),
                                          P<double>(c->vpart), kPartials, P<float>(c->eatom), P<int>(c->status),
                                          wst, wlayer, P<int32_t>(c->aend), ew);
    if (bad) return fail(c, CTD_ERR_INVALID_ARG, "BF16 path: unsupported GEMM shape");
  } else {
    model_forward_backward_fp32(st, c->mw, n, P<int32_t>(c->z_s), P<int32_t>(c->arow), P<int32_t>(c->acol),
                                P<float4>(c->ar), P<int32_t>(c->arev), ptrs.data(), need_grad, P<double>(c->epart),
                                kPartials, P<float4>(c->hedge), P<float>(c->force_s), P<double>(c->vpart),
                                kPartials, P<float>(c->eatom), P<int>(c->status), wst, wlayer, ew);
  }
  StageGuard sg(STG_FORCES);
  launch_sum_partials(st, kPartials, 1, P<double>(c->epart), P<double>(c->out_e), 1.0);
  if (need_grad) launch_sum_partials(st, kPartials, 9, P<double>(c->vpart), P<double>(c->out_w), 1.0);
  CUDA_OK(c, cudaGetLastError());
  return CTD_OK;
}

// positions (device, caller order) are in c->x_user: decide on a rebuild, gather, prune.
int prepare_step(ctd_ctx* c, int64_t n, const double H[9], bool force_rebuild, int32_t* rebuilt, double* maxdisp) {
  bool need = force_rebuild || !c->have_list || n != c->n || memcmp(H, c->H, sizeof(double) * 9) != 0 ||
              c->cutoff < c->desc.rc;
  *rebuilt = 0;
  if (!need) {
    launch_gather_positions(c->st, n, P<int32_t>(c->perm), P<double>(c->x_user), P<double>(c->x_s));
    double md = 0.0;
    int r = prune(c, &md);
    if (r) return r;
    const double eff_skin = c->cutoff + c->skin - c->desc.rc;
    if (md > 0.5 * eff_skin || !std::isfinite(md)) need = true;
    *maxdisp = md;
  }
  if (need) {
    double skin = c->skin_set ? c->skin : 1.0;
    int r = build_from_device_positions(c, n, H, c->desc.rc, skin);
    if (r) return r;
    *rebuilt = 1;
    launch_gather_positions(c->st, n, P<int32_t>(c->perm), P<double>(c->x_user), P<double>(c->x_s));
    double md = 0.0;
    r = prune(c, &md);
    if (r) return r;
    *maxdisp = md;
  }
  return CTD_OK;
}

// Parameters of the strictly local edge model ("CTDLOCAL" blob, matrices [in][out]).
int load_local_params(ctd_ctx* c, const char* b, size_t nbytes) {
  if (memcmp(b, "CTDLOCAL", 8) != 0) return fail(c, CTD_ERR_INVALID_ARG, "bad parameter blob magic");
  int32_t hdr[6];
  memcpy(hdr, b + 8, sizeof(hdr));
  double rc, unused, esc;
  int64_t nval;
  memcpy(&rc, b + 32, 8);
  memcpy(&unused, b + 40, 8);
  memcpy(&esc, b + 48, 8);
  memcpy(&nval, b + 56, 8);
  const int F = hdr[1], K = hdr[2], L = hdr[3], S = hdr[4], C = hdr[5];
  const ctd_model_desc& d = c->desc;
  if (hdr[0] != 1 || F != d.F || K != d.K || L != d.T || S != d.n_species || C != d.channels || rc != d.rc)
    return fail(c, CTD_ERR_INVALID_ARG, "parameter blob header does not match the model description");
  const bool bf16 = d.precision == CTD_PREC_BF16;
  const int C2 = 2 * C, FX = F + C2, Fh = F / 2, KA0 = K + 2 * S, KA = local_ka(K, S, bf16);
  int64_t expect = (int64_t)KA0 * F + F + (int64_t)F * C2 + (int64_t)F * Fh + Fh + Fh + 1;
  for (int l = 1; l <= L; ++l) expect += (int64_t)F * C2 + (int64_t)FX * F + F + (l < L ? 2 * C2 * C : 0);
  if (nval != expect || nbytes < 64 + (size_t)nval * 8)
    return fail(c, CTD_ERR_INVALID_ARG, "parameter blob has the wrong number of values");
  std::vector<double> v((size_t)nval);
  memcpy(v.data(), b + 64, (size_t)nval * 8);
  for (double x : v)
    if (!std::isfinite(x)) return fail(c, CTD_ERR_INVALID_ARG, "non-finite parameter");
  std::vector<float> h;
  auto alloc = [&](size_t cnt) {
    size_t off = (h.size() + 7) / 8 * 8;   // 32-byte aligned arrays (GEMM operands are read as float4)
    h.resize(off + cnt, 0.0f);
    return off;
  };
  const double* p = v.data();
  // a [rows][cols] matrix, stored as is (padded to prow rows) and transposed ([cols][prow])
  auto mat = [&](int rows, int cols, int prow, size_t* t_off) {
    const double* src = p;
    p += (size_t)rows * cols;
    size_t off = alloc((size_t)prow * cols);
    for (int r = 0; r < rows; ++r)
      for (int k = 0; k < cols; ++k) h[off + (size_t)r * cols + k] = (float)src[(size_t)r * cols + k];
    if (t_off) {
      *t_off = alloc((size_t)cols * prow);
      for (int r = 0; r < rows; ++r)
        for (int k = 0; k < cols; ++k) h[*t_off + (size_t)k * prow + r] = (float)src[(size_t)r * cols + k];
    }
    return off;
  };
  auto vec = [&](int cnt) { return mat(1, cnt, 1, nullptr); };
  size_t oA0t, oP0t, oR1t;
  const size_t oA0 = mat(KA0, F, KA, &oA0t), oc0 = vec(F), oP0 = mat(F, C2, F, &oP0t);
  struct LOff { size_t Q, Qt, M, Mt, m, Gs, Gst, Gv, Gvt; } lo[kMaxT] = {};
  for (int l = 1; l <= L; ++l) {
    LOff& o = lo[l - 1];
    o.Q = mat(F, C2, F, &o.Qt);
    o.M = mat(FX, F, FX, &o.Mt);
    o.m = vec(F);
    if (l < L) {
      o.Gs = mat(C2, C, C2, &o.Gst);
      o.Gv = mat(C2, C, C2, &o.Gvt);
    }
  }
  const size_t oR1 = mat(F, Fh, F, &oR1t), od1 = vec(Fh), oR2 = vec(Fh), od2 = vec(1);
  ENSURE(c, c->params, h.size() * sizeof(float));
  CUDA_OK(c, cudaMemcpyAsync(c->params.p, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  const float* base = P<float>(c->params);
  LocalW& w = c->lw;
  w.F = F; w.K = K; w.KA = KA; w.L = L; w.S = S; w.C = C;
  w.rc = (float)rc; w.e_scale = (float)esc;
  w.A0 = base + oA0; w.A0t = base + oA0t; w.c0 = base + oc0; w.P0 = base + oP0; w.P0t = base + oP0t;
  for (int l = 1; l <= L; ++l) {
    const LOff& o = lo[l - 1];
    LocalLayerW& q = w.Lw[l - 1];
    q.Q = base + o.Q; q.Qt = base + o.Qt; q.M = base + o.M; q.Mt = base + o.Mt; q.m = base + o.m;
    q.Gs = l < L ? base + o.Gs : nullptr; q.Gst = l < L ? base + o.Gst : nullptr;
    q.Gv = l < L ? base + o.Gv : nullptr; q.Gvt = l < L ? base + o.Gvt : nullptr;
  }
  w.R1 = base + oR1; w.R1t = base + oR1t; w.d1 = base + od1; w.R2 = base + oR2; w.d2 = base + od2;
  w.bf16 = bf16;
  if (bf16) {
    // BF16 GEMM operands W [N][K]: forward the [out][in] arrays, adjoint the [in][out] ones, each
    // row zero-padded to at least 64 columns
    w.KAb = KA < 64 ? 64 : KA;
    w.Kh = Fh < 64 ? 64 : Fh;
    std::vector<uint16_t> hb;
    auto put = [&](size_t off, int rows, int cols, int kpad) {
      size_t o = (hb.size() + 7) / 8 * 8;   // 16-byte aligned rows
      hb.resize(o + (size_t)rows * kpad, 0);
      for (int r = 0; r < rows; ++r)
        for (int k = 0; k < cols; ++k) hb[o + (size_t)r * kpad + k] = to_bf16_bits(h[off + (size_t)r * cols + k]);
      return o;
    };
    // the transposed arrays are stored [cols][prow]: A0t [F][KA], P0t [2C][F], Qt [2C][F],
    // Mt [F][FX], R1t [F/2][F]; the plain ones [rows][cols]: A0 [KA][F], P0 [F][2C], Q [F][2C],
    // M [FX][F], R1 [F][F/2]
    const size_t bA0t = put(oA0t, F, KA, w.KAb), bP0t = put(oP0t, C2, F, F), bR1t = put(oR1t, Fh, F, F);
    const size_t bA0 = put(oA0, KA, F, F), bP0 = put(oP0, F, C2, 64 > C2 ? 64 : C2), bR1 = put(oR1, F, Fh, w.Kh);
    size_t bQt[kMaxT], bMt[kMaxT], bQ[kMaxT], bM[kMaxT];
    for (int l = 1; l <= L; ++l) {
      const LOff& o = lo[l - 1];
      bQt[l - 1] = put(o.Qt, C2, F, F);
      bMt[l - 1] = put(o.Mt, F, FX, FX);
      bQ[l - 1] = put(o.Q, F, C2, 64 > C2 ? 64 : C2);
      bM[l - 1] = put(o.M, FX, F, F);
    }
    ENSURE(c, c->params_bf, hb.size() * sizeof(uint16_t));
    CUDA_OK(c, cudaMemcpyAsync(c->params_bf.p, hb.data(), hb.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, c->st));
    CUDA_OK(c, cudaStreamSynchronize(c->st));
    const __nv_bfloat16* bb = P<__nv_bfloat16>(c->params_bf);
    w.wb.A0t = bb + bA0t; w.wb.P0t = bb + bP0t; w.wb.R1t = bb + bR1t;
    w.wb.A0 = bb + bA0; w.wb.P0 = bb + bP0; w.wb.R1 = bb + bR1;
    for (int l = 1; l <= L; ++l) {
      w.wb.Qt[l - 1] = bb + bQt[l - 1]; w.wb.Mt[l - 1] = bb + bMt[l - 1];
      w.wb.Q[l - 1] = bb + bQ[l - 1]; w.wb.M[l - 1] = bb + bM[l - 1];
    }
  }
  c->e_scale = esc;
  c->have_params = true;
  return CTD_OK;
}

int load_params_impl(ctd_ctx* c, const void* blob, size_t nbytes) {
  if (!blob || nbytes < 64) return fail(c, CTD_ERR_INVALID_ARG, "parameter blob too short");
  const char* b = static_cast<const char*>(blob);
  if (c->local()) return load_local_params(c, b, nbytes);
  if (memcmp(b, "CTDPAINN", 8) != 0) return fail(c, CTD_ERR_INVALID_ARG, "bad parameter blob magic");
  int32_t hdr[6];
  memcpy(hdr, b + 8, sizeof(hdr));
  double rc, eps, esc;
  int64_t nval;
  memcpy(&rc, b + 32, 8);
  memcpy(&eps, b + 40, 8);
  memcpy(&esc, b + 48, 8);
  memcpy(&nval, b + 56, 8);
  const int F = hdr[1], K = hdr[2], T = hdr[3], S = hdr[4];
  const ctd_model_desc& d = c->desc;
  if (hdr[0] != 1 || F != d.F || K != d.K || T != d.T || S != d.n_species || rc != d.rc)
    return fail(c, CTD_ERR_INVALID_ARG, "parameter blob header does not match the model description");
  int64_t per = (int64_t)F * F + F + 3 * F * F + 3 * F + 3 * F * K + 3 * F + 2 * F * F + 2 * F * F + F +
                3 * F * F + 3 * F;
  int64_t expect = (int64_t)S * F + T * per + (F / 2) * F + F / 2 + F / 2 + 1;
  if (nval != expect || nbytes < 64 + (size_t)nval * 8)
    return fail(c, CTD_ERR_INVALID_ARG, "parameter blob has the wrong number of values");
  std::vector<double> v((size_t)nval);
  memcpy(v.data(), b + 64, (size_t)nval * 8);
  for (double x : v)
    if (!std::isfinite(x)) return fail(c, CTD_ERR_INVALID_ARG, "non-finite parameter");
  const int KP = (K + 3) / 4 * 4;
  // host staging of every FP32 array, 16-byte aligned offsets
  std::vector<float> h;
  auto alloc = [&](size_t cnt) {
    size_t off = (h.size() + 7) / 8 * 8;   // 32 B: the BF16 twin of every array is 16-byte aligned
    h.resize(off + cnt, 0.0f);
    return off;
  };
  const double* p = v.data();
  auto take = [&](size_t cnt) {
    const double* q = p;
    p += cnt;
    return q;
  };
  auto put = [&](const double* src, int rows, int cols, bool transpose) {
    size_t off = alloc((size_t)rows * cols);
    for (int r = 0; r < rows; ++r)
      for (int k = 0; k < cols; ++k) {
        float x = (float)src[(size_t)r * cols + k];
        if (transpose) h[off + (size_t)k * rows + r] = x;
        else h[off + (size_t)r * cols + k] = x;
      }
    return off;
  };
  struct Off {
    size_t W1, W1t, b1, W2, W2t, b2, Wf, Wf64, bf, UV, UVt, A1, A1t, c1, A2, A2t, c2;
  } lo[kMaxT];
  size_t o_emb = put(take((size_t)S * F), S, F, false);
  for (int t = 0; t < T; ++t) {
    const double* W1 = take((size_t)F * F);
    const double* b1 = take(F);
    const double* W2 = take((size_t)3 * F * F);
    const double* b2 = take(3 * F);
    const double* Wf = take((size_t)3 * F * K);
    const double* bf = take(3 * F);
    const double* U = take((size_t)F * F);
    const double* V = take((size_t)F * F);
    const double* A1 = take((size_t)2 * F * F);
    const double* c1 = take(F);
    const double* A2 = take((size_t)3 * F * F);
    const double* c2 = take(3 * F);
    Off& o = lo[t];
    o.W1 = put(W1, F, F, false);
    o.W1t = put(W1, F, F, true);
    o.b1 = put(b1, 1, F, false);
    o.W2 = put(W2, 3 * F, F, false);
    o.W2t = put(W2, 3 * F, F, true);
    o.b2 = put(b2, 1, 3 * F, false);
    o.Wf = alloc((size_t)3 * F * KP);
    for (int r = 0; r < 3 * F; ++r)
      for (int k = 0; k < K; ++k) h[o.Wf + (size_t)r * KP + k] = (float)Wf[(size_t)r * K + k];
    // [3F][64] zero-padded copy whose BF16 twin is the tensor-core filter operand
    o.Wf64 = alloc((size_t)3 * F * 64);
    for (int r = 0; r < 3 * F; ++r)
      for (int k = 0; k < K && k < 64; ++k) h[o.Wf64 + (size_t)r * 64 + k] = (float)Wf[(size_t)r * K + k];
    // the filter bias in column K: kernels that fold it put f_c at basis index K, the others 0
    if (K < 32)
      for (int r = 0; r < 3 * F; ++r) h[o.Wf64 + (size_t)r * 64 + K] = (float)bf[r];
    o.bf = put(bf, 1, 3 * F, false);
    o.UV = alloc((size_t)2 * F * F);
    o.UVt = alloc((size_t)2 * F * F);
    for (int r = 0; r < F; ++r)
      for (int k = 0; k < F; ++k) {
        h[o.UV + (size_t)r * F + k] = (float)U[(size_t)r * F + k];
        h[o.UV + (size_t)(F + r) * F + k] = (float)V[(size_t)r * F + k];
        h[o.UVt + (size_t)k * 2 * F + r] = (float)U[(size_t)r * F + k];
        h[o.UVt + (size_t)k * 2 * F + F + r] = (float)V[(size_t)r * F + k];
      }
    o.A1 = put(A1, F, 2 * F, false);
    o.A1t = put(A1, F, 2 * F, true);
    o.c1 = put(c1, 1, F, false);
    o.A2 = put(A2, 3 * F, F, false);
    o.A2t = put(A2, 3 * F, F, true);
    o.c2 = put(c2, 1, 3 * F, false);
  }
  const double* R1 = take((size_t)(F / 2) * F);
  size_t o_R1 = put(R1, F / 2, F, false), o_R1t = put(R1, F / 2, F, true);
  size_t o_d1 = put(take(F / 2), 1, F / 2, false);
  size_t o_R2 = put(take(F / 2), 1, F / 2, false);
  size_t o_d2 = put(take(1), 1, 1, false);
  ENSURE(c, c->params, h.size() * sizeof(float));
  CUDA_OK(c, cudaMemcpyAsync(c->params.p, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, c->st));
  // BF16 twin: element k of the BF16 buffer is element k of the FP32 buffer, rounded
  std::vector<uint16_t> hb(h.size());
  for (size_t k = 0; k < h.size(); ++k) hb[k] = to_bf16_bits(h[k]);
  ENSURE(c, c->params_bf, hb.size() * sizeof(uint16_t));
  CUDA_OK(c, cudaMemcpyAsync(c->params_bf.p, hb.data(), hb.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  const __nv_bfloat16* bbase = P<__nv_bfloat16>(c->params_bf);
  // FP16 copies of the zero-padded radial filters [3F][64] for the tensor-core adjoint; a filter
  // weight beyond FP16's range keeps that model on the CUDA-core adjoint (FP32 weights)
  std::vector<__half> hh((size_t)T * 3 * F * 64);
  bool f16_ok = true;
  for (int t = 0; t < T; ++t)
    for (size_t k = 0; k < (size_t)3 * F * 64; ++k) {
      const float x = h[lo[t].Wf64 + k];
      if (!(std::fabs(x) <= 65504.0f)) f16_ok = false;
      hh[(size_t)t * 3 * F * 64 + k] = __float2half_rn(x);
    }
  if (T > 0) {
    ENSURE(c, c->params_h, hh.size() * sizeof(__half));
    CUDA_OK(c, cudaMemcpyAsync(c->params_h.p, hh.data(), hh.size() * sizeof(__half), cudaMemcpyHostToDevice, c->st));
    CUDA_OK(c, cudaStreamSynchronize(c->st));
  }
  const float* base = P<float>(c->params);
  ModelW& m = c->mw;
  m.F = F; m.K = K; m.KP = KP; m.T = T; m.S = S;
  m.rc = (float)rc; m.eps = (float)eps; m.e_scale = (float)esc;
  m.emb = base + o_emb;
  for (int t = 0; t < T; ++t) {
    const Off& o = lo[t];
    LayerW& L = m.L[t];
    L.W1 = base + o.W1; L.W1t = base + o.W1t; L.b1 = base + o.b1;
    L.W2 = base + o.W2; L.W2t = base + o.W2t; L.b2 = base + o.b2;
    L.Wf = base + o.Wf; L.bf = base + o.bf;
    L.UV = base + o.UV; L.UVt = base + o.UVt;
    L.A1 = base + o.A1; L.A1t = base + o.A1t; L.c1 = base + o.c1;
    L.A2 = base + o.A2; L.A2t = base + o.A2t; L.c2 = base + o.c2;
    L.W1b = bbase + o.W1; L.W1tb = bbase + o.W1t; L.W2b = bbase + o.W2; L.W2tb = bbase + o.W2t;
    L.UVb = bbase + o.UV; L.UVtb = bbase + o.UVt; L.A1b = bbase + o.A1; L.A1tb = bbase + o.A1t;
    L.A2b = bbase + o.A2; L.A2tb = bbase + o.A2t;
    L.Wfb = bbase + o.Wf64;
    L.Wfh = f16_ok ? P<__half>(c->params_h) + (size_t)t * 3 * F * 64 : nullptr;
  }
  if (!f16_ok) m.tc_adjoint = false;
  m.R1 = base + o_R1; m.R1t = base + o_R1t; m.d1 = base + o_d1; m.R2 = base + o_R2; m.d2 = base + o_d2;
  m.R1b = bbase + o_R1; m.R1tb = bbase + o_R1t;
  c->eps = eps;
  c->e_scale = esc;
  c->have_params = true;
  return CTD_OK;
}

}  // namespace ctd

// ============================================================================== C ABI
extern "C" {

int ctd_create(ctd_ctx** out, const ctd_model_desc* desc, size_t hbm_budget_bytes, void* cuda_stream) {
  if (!out || !desc) return CTD_ERR_INVALID_ARG;
  *out = nullptr;
  const int F = desc->F;
  if (desc->family == CTD_FAMILY_LOCAL) {
    // edge rows of width F, F/2, 2C, K + 2S (rounded up to 4) feed the SIMT GEMM
    const int C = desc->channels;
    if (F < 8 || F > 256 || F % 8 != 0 || C < 4 || C > 64 || C % 4 != 0 || desc->K < 2 || desc->K > kMaxKP ||
        desc->T < 1 || desc->T > kMaxT || desc->n_species < 1 || desc->n_species > 64 || !(desc->rc > 0.0) ||
        (desc->precision != CTD_PREC_FP32 && desc->precision != CTD_PREC_BF16))
      return CTD_ERR_INVALID_ARG;
    // BF16: every tensor-core GEMM width (F, F/2, 2C, F + 2C, the padded two-body input) a
    // multiple of 32
    if (desc->precision == CTD_PREC_BF16 && (!bf16_available() || !(F == 64 || F == 128) || C % 16 != 0))
      return CTD_ERR_INVALID_ARG;
  } else if (desc->family != CTD_FAMILY_PAINN ||
             !(F == 32 || F == 64 || F == 128 || F == 256) || desc->K < 2 || desc->K > kMaxKP || desc->T < 0 ||
             desc->T > kMaxT || desc->n_species < 1 || !(desc->rc > 0.0) ||
             (desc->precision != CTD_PREC_FP32 && desc->precision != CTD_PREC_BF16)) {
    return CTD_ERR_INVALID_ARG;
  }
  if (desc->precision == CTD_PREC_BF16 && (!bf16_available() || !(F == 64 || F == 128)))
    return CTD_ERR_INVALID_ARG;
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
    cudaGetLastError();
    return CTD_ERR_CUDA;
  }
  ctd_ctx* c = new ctd_ctx();
  c->desc = *desc;
  c->budget = hbm_budget_bytes;
  c->mw.tc_adjoint = true;   // BF16 path, F = 128: tensor-core adjoint and message contraction
  c->mw.tc_message = true;
  c->mw.edge_chunk_rows = 32;
  cudaGetDevice(&c->device);
  if (cuda_stream) {
    c->st = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return CTD_ERR_CUDA;
    }
    c->own_stream = true;
  }
  *out = c;
  return CTD_OK;
}

void ctd_destroy(ctd_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  c->prof.collect();
  for (DBuf* b : c->all)
    if (b->p) cudaFree(b->p);
  for (DBuf& b : c->mbuf)
    if (b.p) cudaFree(b.p);
  for (DBuf& b : c->mbufb)
    if (b.p) cudaFree(b.p);
  if (c->own_stream) cudaStreamDestroy(c->st);
  delete c;
}

const char* ctd_last_error(ctd_ctx* c) { return c ? c->err.c_str() : "null context"; }

int ctd_load_params(ctd_ctx* c, const void* blob, size_t nbytes) {
  if (!c) return CTD_ERR_INVALID_ARG;
  Bind bind_(c);
  return load_params_impl(c, blob, nbytes);
}

int ctd_build_neighbors(ctd_ctx* c, int64_t n, const double* positions, const double cell[9], double cutoff,
                        double skin, int32_t flags, int64_t* n_pairs_out) {
  if (!c) return CTD_ERR_INVALID_ARG;
  Bind bind_(c);
  if (n < 0 || (n > 0 && !positions) || !cell) return fail(c, CTD_ERR_INVALID_ARG, "bad positions / cell");
  if (n > (int64_t)INT32_MAX / 4) return fail(c, CTD_ERR_INVALID_ARG, "too many atoms");
  const bool dev = flags & CTD_DEVICE_PTRS;
  ENSURE(c, c->x_user, sizeof(double) * 3 * (n > 0 ? n : 1));
  int r = copy_in(c, c->x_user.p, positions, sizeof(double) * 3 * n, dev);
  if (r) return r;
  r = build_from_device_positions(c, n, cell, cutoff, skin);
  if (r) return r;
  c->skin = skin;
  c->skin_set = true;
  if (n_pairs_out) *n_pairs_out = c->n_verlet;
  return CTD_OK;
}

int ctd_get_pairs(ctd_ctx* c, int32_t* pi, int32_t* pj, int8_t* shift, int64_t cap) {
  if (!c) return CTD_ERR_INVALID_ARG;
  Bind bind_(c);
  if (!c->have_list) return fail(c, CTD_ERR_STATE, "no neighbour list");
  if (cap < c->n_verlet) return fail(c, CTD_ERR_CAPACITY, "output arrays shorter than the pair list");
  if (!pi || !pj || !shift) return fail(c, CTD_ERR_INVALID_ARG, "null output array");
  const int64_t n = c->n, E = c->n_verlet;
  std::vector<int32_t> row(n + 1), col(E), perm(n);
  std::vector<uint32_t> img(E);
  CUDA_OK(c, cudaMemcpyAsync(row.data(), c->vrow.p, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, c->st));
  if (E) {
    CUDA_OK(c, cudaMemcpyAsync(col.data(), c->vcol.p, sizeof(int32_t) * E, cudaMemcpyDeviceToHost, c->st));
    CUDA_OK(c, cudaMemcpyAsync(img.data(), c->vimg.p, sizeof(uint32_t) * E, cudaMemcpyDeviceToHost, c->st));
  }
  if (n) CUDA_OK(c, cudaMemcpyAsync(perm.data(), c->perm.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  struct Rec {
    int32_t i, j;
    int8_t s[3];
  };
  std::vector<Rec> rec((size_t)E);
  for (int64_t k = 0; k < n; ++k)
    for (int32_t e = row[k]; e < row[k + 1]; ++e) {
      Rec& q = rec[(size_t)e];
      q.i = perm[k];
      q.j = perm[col[e]];
      q.s[0] = (int8_t)(img[e] & 0xff);
      q.s[1] = (int8_t)((img[e] >> 8) & 0xff);
      q.s[2] = (int8_t)((img[e] >> 16) & 0xff);
    }
  std::sort(rec.begin(), rec.end(), [](const Rec& a, const Rec& b) {
    if (a.i != b.i) return a.i < b.i;
    if (a.j != b.j) return a.j < b.j;
    for (int k = 0; k < 3; ++k)
      if (a.s[k] != b.s[k]) return a.s[k] < b.s[k];
    return false;
  });
  for (int64_t e = 0; e < E; ++e) {
    pi[e] = rec[(size_t)e].i;
    pj[e] = rec[(size_t)e].j;
    for (int k = 0; k < 3; ++k) shift[3 * e + k] = rec[(size_t)e].s[k];
  }
  return CTD_OK;
}

int ctd_set_option(ctd_ctx* c, int32_t option, int64_t value) {
  if (!c) return CTD_ERR_INVALID_ARG;
  switch (option) {
    case CTD_OPT_EDGE_CHUNK_ROWS:
      if (value < 0 || value > (1 << 30)) return fail(c, CTD_ERR_INVALID_ARG, "CTD_OPT_EDGE_CHUNK_ROWS out of range");
      c->mw.edge_chunk_rows = value;
      return CTD_OK;
    case CTD_OPT_TC_MESSAGE:
      if (value < 0 || value > 1) return fail(c, CTD_ERR_INVALID_ARG, "CTD_OPT_TC_MESSAGE takes 0 or 1");
      c->mw.tc_message = value != 0;
      return CTD_OK;
    case CTD_OPT_EDGE_STORE:
      if (value < 0 || value > 1) return fail(c, CTD_ERR_INVALID_ARG, "CTD_OPT_EDGE_STORE takes 0 or 1");
      c->mw.edge_store = value != 0;
      return CTD_OK;
    case CTD_OPT_TC_ADJOINT:
      if (value < 0 || value > 1) return fail(c, CTD_ERR_INVALID_ARG, "CTD_OPT_TC_ADJOINT takes 0 or 1");
      c->mw.tc_adjoint = value != 0;
      return CTD_OK;
    default:
      return fail(c, CTD_ERR_INVALID_ARG, "unknown option");
  }
}

int ctd_profile_enable(ctd_ctx* c, int32_t enable) {
  if (!c) return CTD_ERR_INVALID_ARG;
  c->prof.collect();
  c->prof.on = enable != 0;
  return CTD_OK;
}

int ctd_profile_read(ctd_ctx* c, double* ms, int64_t* launches, int32_t reset) {
  if (!c) return CTD_ERR_INVALID_ARG;
  c->prof.collect();
  for (int s = 0; s < STG_COUNT; ++s) {
    if (ms) ms[s] = c->prof.ms[s];
    if (launches) launches[s] = c->prof.launches[s];
    if (reset) {
      c->prof.ms[s] = 0.0;
      c->prof.launches[s] = 0;
    }
  }
  return CTD_OK;
}

int ctd_gemm_bf16(ctd_ctx* c, int64_t M, int32_t N, int32_t K, const void* A, int64_t lda, const void* B,
                  float* C, int64_t ldc) {
  if (!c) return CTD_ERR_INVALID_ARG;
  Bind bind_(c);
  if (M < 0 || !gemm_bf16_supported(N, K) || (M > 0 && (!A || !B || !C)) || lda < K || ldc < N || ldc % 4)
    return fail(c, CTD_ERR_INVALID_ARG, "gemm: K must be a multiple of 32 and at least 64, N a multiple of 32 (<= 512)");
  ENSURE(c, c->status, sizeof(int32_t) * 4);
  CUDA_OK(c, cudaMemsetAsync(c->status.p, 0, sizeof(int32_t), c->st));
  int r = gemm_bf16<0>(c->st, M, N, K, static_cast<const __nv_bfloat16*>(A), lda,
                       static_cast<const __nv_bfloat16*>(B), nullptr, nullptr, 0, C, (int)ldc, nullptr, 0,
                       P<int>(c->status));
  if (r) return fail(c, CTD_ERR_INVALID_ARG, "gemm: unsupported shape or alignment");
  CUDA_OK(c, cudaGetLastError());
  int st = 0;
  CUDA_OK(c, cudaMemcpyAsync(&st, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  if (st & ST_TIMEOUT) return fail(c, CTD_ERR_TIMEOUT, "gemm: a bounded device wait gave up");
  return CTD_OK;
}

int ctd_set_energy_out(ctd_ctx* c, double* energies) {
  if (!c) return CTD_ERR_INVALID_ARG;
  c->energy_out_user = energies;
  return CTD_OK;
}

int ctd_compute(ctd_ctx* c, int64_t n, const int32_t* species, const double* positions, const double cell[9],
                int32_t flags, double* energy, double* forces, double* virial, ctd_stats* stats) {
  if (!c) return CTD_ERR_INVALID_ARG;
  Bind bind_(c);
  if (!c->have_params) return fail(c, CTD_ERR_STATE, "parameters not loaded");
  if (n < 0 || (n > 0 && (!positions || !species)) || !cell || !energy)
    return fail(c, CTD_ERR_INVALID_ARG, "bad arguments");
  if (((flags & CTD_NEED_FORCES) && !forces) || ((flags & CTD_NEED_VIRIAL) && !virial))
    return fail(c, CTD_ERR_INVALID_ARG, "forces / virial requested without an output array");
  if (n > (int64_t)INT32_MAX / 4) return fail(c, CTD_ERR_INVALID_ARG, "too many atoms");
  cudaEvent_t ev[3];
  bool timing = stats != nullptr;
  if (timing)
    for (auto& e : ev) cudaEventCreate(&e);
  const bool dev = flags & CTD_DEVICE_PTRS;
  const int64_t n1 = n > 0 ? n : 1;
  ENSURE(c, c->x_user, sizeof(double) * 3 * n1);
  ENSURE(c, c->z_user, sizeof(int32_t) * n1);
  int r = copy_in(c, c->x_user.p, positions, sizeof(double) * 3 * n, dev);
  if (r) return r;
  r = copy_in(c, c->z_user.p, species, sizeof(int32_t) * n, dev);
  if (r) return r;
  if (timing) cudaEventRecord(ev[0], c->st);
  int32_t rebuilt = 0;
  double md = 0.0;
  r = prepare_step(c, n, cell, flags & CTD_REBUILD, &rebuilt, &md);
  if (r) return r;
  launch_gather_i32(c->st, n, P<int32_t>(c->perm), P<int32_t>(c->z_user), P<int32_t>(c->z_s));
  if (timing) cudaEventRecord(ev[1], c->st);
  const bool need_grad = flags & (CTD_NEED_FORCES | CTD_NEED_VIRIAL);
  CUDA_OK(c, cudaMemsetAsync(c->status.p, 0, sizeof(int32_t), c->st));
  r = evaluate(c, need_grad);
  if (r) return r;
  if (timing) cudaEventRecord(ev[2], c->st);
  // outputs
  ENSURE(c, c->out_f, sizeof(double) * 3 * n1);
  ENSURE(c, c->out_eatom, sizeof(double) * n1);
  double* fdst = (flags & CTD_NEED_FORCES) ? (dev ? forces : P<double>(c->out_f)) : nullptr;
  if (fdst) launch_scatter_rows(c->st, n, 3, P<int32_t>(c->perm), P<float>(c->force_s), fdst);
  double* edst = c->energy_out_user ? (dev ? c->energy_out_user : P<double>(c->out_eatom)) : nullptr;
  if (edst) launch_scatter_rows(c->st, n, 1, P<int32_t>(c->perm), P<float>(c->eatom), edst);
  launch_check_finite(c->st, 1, P<double>(c->out_e), P<int>(c->status));
  if (fdst) launch_check_finite(c->st, 3 * n, fdst, P<int>(c->status));
  if (dev) {
    CUDA_OK(c, cudaMemcpyAsync(energy, c->out_e.p, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    if (flags & CTD_NEED_VIRIAL)
      CUDA_OK(c, cudaMemcpyAsync(virial, c->out_w.p, sizeof(double) * 9, cudaMemcpyDeviceToDevice, c->st));
  } else {
    CUDA_OK(c, cudaMemcpyAsync(energy, c->out_e.p, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (flags & CTD_NEED_VIRIAL)
      CUDA_OK(c, cudaMemcpyAsync(virial, c->out_w.p, sizeof(double) * 9, cudaMemcpyDeviceToHost, c->st));
    if (flags & CTD_NEED_FORCES)
      CUDA_OK(c, cudaMemcpyAsync(forces, c->out_f.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->st));
    if (c->energy_out_user)
      CUDA_OK(c, cudaMemcpyAsync(c->energy_out_user, c->out_eatom.p, sizeof(double) * n, cudaMemcpyDeviceToHost,
                                 c->st));
  }
  r = check_status(c);   // synchronises the stream
  if (r) return r;
  if (stats) {
    int32_t act = 0;
    CUDA_OK(c, cudaMemcpy(&act, P<int32_t>(c->arow) + n, sizeof(int32_t), cudaMemcpyDeviceToHost));
    stats->n_atoms = n;
    stats->n_verlet_edges = c->n_verlet;
    stats->n_active_edges = act;
    stats->rebuilt = rebuilt;
    stats->retries = 0;
    stats->max_displacement = md;
    stats->bytes_allocated = (int64_t)c->held;
    stats->bytes_in_use = (int64_t)c->used;
    stats->edges_stored = c->last_stored ? 1 : 0;
    cudaEventElapsedTime(&stats->ms_neighbors, ev[0], ev[1]);
    cudaEventElapsedTime(&stats->ms_model, ev[1], ev[2]);
    for (auto& e : ev) cudaEventDestroy(e);
  }
  return CTD_OK;
}

// ------------------------------------------------------------------------------ NVE
int ctd_md_set_state(ctd_ctx* c, int64_t n, const int32_t* species, const double* masses, const double* positions,
                     const double* velocities, const double cell[9], double skin) {
  if (!c) return CTD_ERR_INVALID_ARG;
  Bind bind_(c);
  if (!c->have_params) return fail(c, CTD_ERR_STATE, "parameters not loaded");
  if (n <= 0 || !species || !masses || !positions || !velocities || !cell || !(skin >= 0.0))
    return fail(c, CTD_ERR_INVALID_ARG, "bad MD state");
  for (int64_t k = 0; k < n; ++k)
    if (!(masses[k] > 0.0)) return fail(c, CTD_ERR_INVALID_ARG, "masses must be positive");
  ENSURE(c, c->x_user, sizeof(double) * 3 * n);
  ENSURE(c, c->z_user, sizeof(int32_t) * n);
  ENSURE(c, c->md_x_user, sizeof(double) * 3 * n);
  ENSURE(c, c->md_v_user, sizeof(double) * 3 * n);
  ENSURE(c, c->md_tmp, sizeof(double) * 3 * n);
  ENSURE(c, c->md_v, sizeof(double) * 3 * n);
  ENSURE(c, c->md_m, sizeof(double) * n);
  int r = copy_in(c, c->x_user.p, positions, sizeof(double) * 3 * n, false);
  if (r) return r;
  r = copy_in(c, c->z_user.p, species, sizeof(int32_t) * n, false);
  if (r) return r;
  r = copy_in(c, c->md_v_user.p, velocities, sizeof(double) * 3 * n, false);
  if (r) return r;
  r = copy_in(c, c->md_tmp.p, masses, sizeof(double) * n, false);
  if (r) return r;
  r = build_from_device_positions(c, n, cell, c->desc.rc, skin);
  if (r) return r;
  c->skin = skin;
  c->skin_set = true;
  launch_gather_positions(c->st, n, P<int32_t>(c->perm), P<double>(c->x_user), P<double>(c->x_s));
  launch_gather_rows_d(c->st, n, 3, P<int32_t>(c->perm), P<double>(c->md_v_user), P<double>(c->md_v));
  launch_gather_rows_d(c->st, n, 1, P<int32_t>(c->perm), P<double>(c->md_tmp), P<double>(c->md_m));
  launch_gather_i32(c->st, n, P<int32_t>(c->perm), P<int32_t>(c->z_user), P<int32_t>(c->z_s));
  CUDA_OK(c, cudaGetLastError());
  c->md_ready = true;
  c->md_forces_valid = false;
  if (c->nhc_state.p) CUDA_OK(c, cudaMemsetAsync(c->nhc_state.p, 0, c->nhc_state.bytes, c->st));   // new trajectory
  return CTD_OK;
}

int ctd_md_set_thermostat(ctd_ctx* c, double temperature, double tau, int32_t chain) {
  if (!c) return CTD_ERR_INVALID_ARG;
  Bind bind_(c);
  if (chain < 0 || chain > 16) return fail(c, CTD_ERR_INVALID_ARG, "chain length must be 0..16");
  if (chain > 0 && !(temperature > 0.0 && std::isfinite(temperature) && tau > 0.0 && std::isfinite(tau)))
    return fail(c, CTD_ERR_INVALID_ARG, "temperature and tau must be positive and finite");
  ENSURE(c, c->nhc_state, sizeof(double) * 40);
  CUDA_OK(c, cudaMemsetAsync(c->nhc_state.p, 0, c->nhc_state.bytes, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  c->nhc_M = chain;
  c->nhc_T = temperature;
  c->nhc_tau = tau;
  return CTD_OK;
}

int ctd_md_set_thermostat_state(ctd_ctx* c, const double* xi, const double* vxi) {
  if (!c) return CTD_ERR_INVALID_ARG;
  Bind bind_(c);
  if (c->nhc_M == 0) return fail(c, CTD_ERR_STATE, "no thermostat set");
  if (!xi || !vxi) return fail(c, CTD_ERR_INVALID_ARG, "xi and vxi are required");
  const int M = c->nhc_M;
  for (int j = 0; j < M; ++j)
    if (!std::isfinite(xi[j]) || !std::isfinite(vxi[j])) return fail(c, CTD_ERR_INVALID_ARG, "non-finite chain state");
  CUDA_OK(c, cudaMemcpyAsync(c->nhc_state.p, xi, sizeof(double) * M, cudaMemcpyHostToDevice, c->st));
  CUDA_OK(c, cudaMemcpyAsync(P<double>(c->nhc_state) + M, vxi, sizeof(double) * M, cudaMemcpyHostToDevice, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  return CTD_OK;
}

int ctd_md_get_thermostat(ctd_ctx* c, double* xi, double* vxi, double* ethermo) {
  if (!c) return CTD_ERR_INVALID_ARG;
  Bind bind_(c);
  if (c->nhc_M == 0) return fail(c, CTD_ERR_STATE, "no thermostat set");
  const int M = c->nhc_M;
  if (xi) CUDA_OK(c, cudaMemcpyAsync(xi, c->nhc_state.p, sizeof(double) * M, cudaMemcpyDeviceToHost, c->st));
  if (vxi)
    CUDA_OK(c, cudaMemcpyAsync(vxi, P<double>(c->nhc_state) + M, sizeof(double) * M, cudaMemcpyDeviceToHost, c->st));
  if (ethermo && c->md_last_steps >= 0)
    CUDA_OK(c, cudaMemcpyAsync(ethermo, c->md_eth.p, sizeof(double) * (c->md_last_steps + 1), cudaMemcpyDeviceToHost,
                               c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  return CTD_OK;
}

namespace {
// Rebuild the list from the resident sorted state (x_s, v, m, z) and re-sort that state.
int md_rebuild(ctd_ctx* c) {
  const int64_t n = c->n;
  cudaStream_t st = c->st;
  int32_t* perm = P<int32_t>(c->perm);
  // back to caller order
  launch_scatter_rows_d(st, n, 3, perm, P<double>(c->x_s), P<double>(c->x_user));
  launch_scatter_rows_d(st, n, 3, perm, P<double>(c->md_v), P<double>(c->md_v_user));
  launch_scatter_rows_d(st, n, 1, perm, P<double>(c->md_m), P<double>(c->md_tmp));
  double H[9];
  memcpy(H, c->H, sizeof(H));
  int r = build_from_device_positions(c, n, H, c->desc.rc, c->skin);
  if (r) return r;
  perm = P<int32_t>(c->perm);
  launch_gather_positions(st, n, perm, P<double>(c->x_user), P<double>(c->x_s));
  launch_gather_rows_d(st, n, 3, perm, P<double>(c->md_v_user), P<double>(c->md_v));
  launch_gather_rows_d(st, n, 1, perm, P<double>(c->md_tmp), P<double>(c->md_m));
  launch_gather_i32(st, n, perm, P<int32_t>(c->z_user), P<int32_t>(c->z_s));
  return CTD_OK;
}

int md_forces(ctd_ctx* c, int32_t* rebuilds) {
  double md = 0.0;
  int r = prune(c, &md);
  if (r) return r;
  if (md > 0.5 * c->skin || !std::isfinite(md)) {
    if (!std::isfinite(md)) return fail(c, CTD_ERR_NONFINITE, "non-finite positions in MD");
    r = md_rebuild(c);
    if (r) return r;
    ++*rebuilds;
    r = prune(c, nullptr);
    if (r) return r;
  }
  return evaluate(c, true);
}
}  // namespace

int ctd_md_run(ctd_ctx* c, int32_t nsteps, double dt, double* epot, double* ekin, int32_t* n_rebuilds) {
  if (!c) return CTD_ERR_INVALID_ARG;
  Bind bind_(c);
  if (!c->md_ready) return fail(c, CTD_ERR_STATE, "no MD state");
  if (nsteps < 0 || !(dt > 0.0)) return fail(c, CTD_ERR_INVALID_ARG, "bad step count or time step");
  const int64_t n = c->n;
  cudaStream_t st = c->st;
  ENSURE(c, c->md_ep, sizeof(double) * ((size_t)nsteps + 1));
  ENSURE(c, c->md_ek, sizeof(double) * ((size_t)nsteps + 1));
  ENSURE(c, c->kpart, sizeof(double) * kPartials);
  int32_t rebuilds = 0;
  int r;
  ENSURE(c, c->status, sizeof(int32_t) * 4);
  CUDA_OK(c, cudaMemsetAsync(c->status.p, 0, sizeof(int32_t), st));
  if (!c->md_forces_valid) {
    r = md_forces(c, &rebuilds);
    if (r) return r;
    c->md_forces_valid = true;
  }
  StageGuard sg(STG_MD);
  // NVT: Nose-Hoover chain half steps around velocity Verlet (Nf = 3n - 3: centre of mass at rest)
  const bool nvt = c->nhc_M > 0;
  NhcParams np{};
  if (nvt) {
    if (n < 2) return fail(c, CTD_ERR_INVALID_ARG, "a thermostat needs at least two atoms");
    np.M = c->nhc_M;
    np.kT = 8.617333262e-5 * c->nhc_T;
    np.Nf = 3.0 * (double)n - 3.0;
    for (int j = 0; j < np.M; ++j) np.Q[j] = (j == 0 ? np.Nf : 1.0) * np.kT * c->nhc_tau * c->nhc_tau;
    ENSURE(c, c->nhc_ke, sizeof(double) * 4);
    ENSURE(c, c->md_eth, sizeof(double) * ((size_t)nsteps + 1));
  }
  double* gscale = nvt ? P<double>(c->nhc_state) + np.M * 2 : nullptr;
  auto record = [&](int step) {
    cudaMemcpyAsync(P<double>(c->md_ep) + step, c->out_e.p, sizeof(double), cudaMemcpyDeviceToDevice, st);
    launch_kinetic(st, n, P<double>(c->md_m), P<double>(c->md_v), P<double>(c->kpart), kPartials);
    launch_sum_partials(st, kPartials, 1, P<double>(c->kpart), P<double>(c->md_ek) + step, 1.0);
    if (nvt) launch_nhc_energy(st, np, P<double>(c->nhc_state), P<double>(c->md_eth) + step);
  };
  record(0);
  for (int32_t s = 0; s < nsteps; ++s) {
    if (nvt) launch_nhc_half(st, np, 0.5 * dt, P<double>(c->md_ek) + s, P<double>(c->nhc_state));
    launch_kick_drift(st, n, dt, P<float>(c->force_s), P<double>(c->md_m), gscale, P<double>(c->x_s),
                      P<double>(c->md_v));
    r = md_forces(c, &rebuilds);
    if (r) return r;
    launch_kick(st, n, dt, P<float>(c->force_s), P<double>(c->md_m), P<double>(c->md_v));
    if (nvt) {
      launch_kinetic(st, n, P<double>(c->md_m), P<double>(c->md_v), P<double>(c->kpart), kPartials);
      launch_sum_partials(st, kPartials, 1, P<double>(c->kpart), P<double>(c->nhc_ke), 1.0);
      launch_nhc_half(st, np, 0.5 * dt, P<double>(c->nhc_ke), P<double>(c->nhc_state));
      launch_scale_v(st, n, gscale, P<double>(c->md_v));
    }
    record(s + 1);
  }
  c->md_last_steps = nvt ? nsteps : -1;
  CUDA_OK(c, cudaGetLastError());
  if (epot) CUDA_OK(c, cudaMemcpyAsync(epot, c->md_ep.p, sizeof(double) * (nsteps + 1), cudaMemcpyDeviceToHost, st));
  if (ekin) CUDA_OK(c, cudaMemcpyAsync(ekin, c->md_ek.p, sizeof(double) * (nsteps + 1), cudaMemcpyDeviceToHost, st));
  r = check_status(c);
  if (r) return r;
  if (n_rebuilds) *n_rebuilds = rebuilds;
  return CTD_OK;
}

int ctd_md_get_state(ctd_ctx* c, double* positions, double* velocities) {
  if (!c) return CTD_ERR_INVALID_ARG;
  Bind bind_(c);
  if (!c->md_ready) return fail(c, CTD_ERR_STATE, "no MD state");
  const int64_t n = c->n;
  int32_t* perm = P<int32_t>(c->perm);
  launch_scatter_rows_d(c->st, n, 3, perm, P<double>(c->x_s), P<double>(c->md_x_user));
  launch_scatter_rows_d(c->st, n, 3, perm, P<double>(c->md_v), P<double>(c->md_v_user));
  if (positions)
    CUDA_OK(c, cudaMemcpyAsync(positions, c->md_x_user.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->st));
  if (velocities)
    CUDA_OK(c, cudaMemcpyAsync(velocities, c->md_v_user.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  return CTD_OK;
}

}  // extern "C"
