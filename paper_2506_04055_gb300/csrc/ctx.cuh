// ctx.cuh -- the engine context behind the C ABI (internal): grow-only device buffers, model
// weights, the neighbour-list and MD state, and the host-side stages shared by the single-system
// calls (api.cu) and the multi-replica serving loop (serve.cu).
#pragma once
#include <string>
#include <vector>

#include "ctd_internal.cuh"
#include "../../include/painn.h"

namespace ctd {
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  size_t need = 0;   // bytes the last request asked for (the rest of `bytes` is growth headroom)
};

constexpr int kPartials = 152 * 4;   // fixed block count of the reductions (deterministic)

bool bf16_available();
uint16_t to_bf16_bits(float f);

}  // namespace ctd

struct ctd_ctx {
  using DBuf = ctd::DBuf;
  using ProfState = ctd::ProfState;
  using ModelW = ctd::ModelW;
  using CellGeom = ctd::CellGeom;
  ctd_model_desc desc{};
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  size_t budget = 0, held = 0, used = 0;   // used: the buffers' last requests
  std::string err;
  // While a served step is being captured into a CUDA graph, a buffer that would have to grow
  // fails instead of reallocating (the capture is then abandoned); alloc_gen counts every
  // (re)allocation and free, so that a graph is replayed only over the buffers it captured.
  bool capturing = false;
  uint64_t alloc_gen = 0;
  std::vector<DBuf*> all;

  // parameters
  bool have_params = false;
  double eps = 1e-8, e_scale = 1.0;
  DBuf params, params_bf, params_h;   // FP32 weights, their BF16 twin, FP16 copies of the filters
  ModelW mw{};
  // strictly local edge model (desc.family == CTD_FAMILY_LOCAL): weights and edge buffers
  ctd::LocalW lw{};
  DBuf lbuf;
  bool local() const { return desc.family == CTD_FAMILY_LOCAL; }

  // neighbour state
  bool have_list = false;
  int64_t n = 0, n_verlet = 0;
  double H[9] = {0};
  double cutoff = 0.0, skin = 1.0;
  bool skin_set = false;
  CellGeom geom{};
  int64_t ncell = 0;
  double last_maxdisp = 0.0;

  DBuf x_user, z_user, xw, wrapm, cellid, cell_count, cell_start, cursor, tmp_idx, perm, inv_perm;
  DBuf xw_s, xref_s, z_s, x_s, count, vrow, vcol, vimg, vbase, vrev, v2a, status, delta, maxd;
  DBuf acount, arow, acol, ar, vidx, arev, aend, hedge, force_s, eatom, epart, vpart, kpart, scan_tmp;
  DBuf out_e, out_f, out_w, out_eatom;
  DBuf wstore;              // per-edge filters [T][E][6F] when edge storage is on
  DBuf ew, near;            // per-atom energy weights and hop flags of a spatial decomposition
  bool use_ew = false, use_near = false;
  bool last_stored = false;  // the last evaluation stored edge filters
  std::vector<DBuf> mbuf, mbufb;
  double* energy_out_user = nullptr;

  ProfState prof;

  // MD state (sorted order)
  bool md_ready = false, md_forces_valid = false;
  DBuf md_v, md_m, md_x_user, md_v_user, md_ep, md_ek, md_tmp;
  // Nose-Hoover chain (chain length 0: NVE)
  int nhc_M = 0;
  double nhc_T = 0.0, nhc_tau = 0.0;
  int32_t md_last_steps = -1;
  DBuf nhc_state, nhc_ke, md_eth;

  ctd_ctx() {
    DBuf* list[] = {&params, &params_bf, &params_h, &x_user, &z_user, &xw, &wrapm, &cellid, &cell_count, &cell_start, &cursor,
                    &tmp_idx, &perm, &inv_perm, &xw_s, &xref_s, &z_s, &x_s, &count, &vrow, &vcol, &vimg,
                    &vbase, &vrev, &v2a, &status, &delta, &maxd, &acount, &arow, &acol, &ar, &vidx, &arev, &aend,
                    &hedge, &force_s, &eatom, &epart, &vpart, &kpart, &scan_tmp, &out_e, &out_f, &out_w,
                    &out_eatom, &wstore, &ew, &near, &md_v, &md_m, &md_x_user, &md_v_user, &md_ep, &md_ek, &md_tmp,
                    &nhc_state, &nhc_ke, &md_eth, &lbuf};
    for (DBuf* b : list) all.push_back(b);
  }
};

namespace ctd {

// Binds the calling thread's launch accounting to a context for the duration of an API call.
struct Bind {
  explicit Bind(ctd_ctx* c) { prof_bind(c ? &c->prof : nullptr); }
  ~Bind() { prof_bind(nullptr); }
};

int fail(ctd_ctx* c, int code, const std::string& msg);
int ensure(ctd_ctx* c, DBuf& b, size_t bytes);
template <class T>
T* P(DBuf& b) {
  return static_cast<T*>(b.p);
}
void inv_transpose(const double H[9], double G[9]);
bool finite_cell(const double H[9]);
int setup_geometry_into(ctd_ctx* c, CellGeom& g, int64_t* ncell, const double H[9], double R);
int check_status(ctd_ctx* c);
int copy_in(ctd_ctx* c, void* dst, const void* src, size_t bytes, bool device);
int prune(ctd_ctx* c, double* maxdisp_out);
int evaluate(ctd_ctx* c, bool need_grad);
size_t model_bytes_per_atom(const ctd_ctx* c);

}  // namespace ctd

#define CUDA_OK(ctx, call)                                                                     \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return ctd::fail(ctx, CTD_ERR_CUDA, std::string(#call " -> ") + cudaGetErrorString(e_)); \
  } while (0)

#define ENSURE(c, b, bytes)                \
  do {                                     \
    int r_ = ctd::ensure((c), (b), (bytes)); \
    if (r_ != CTD_OK) return r_;           \
  } while (0)
