// domain.cu -- spatial domain decomposition with copied atoms, evaluated on one GPU.
//
// arXiv 2506.04055, Results "Distributed potential computation": the system is split into
// non-overlapping domains, each atom is owned by exactly one; every domain also holds copies of
// all atoms (and periodic images) within a communication distance R_comm >= T R of its
// boundary, so that each owned atom's T-hop environment is complete.  The total energy is the
// sum of the owned atoms' U_i over the domains, and the force on an atom is the sum of the
// partial forces on all of its copies (sum-rule equation).  Copies that are more than T hops
// from every owned atom are dropped (the pseudo-message pruning).  "Parallelization cost"
// estimates the extra work of the copies; ctd_domains_info reports the counts it predicts.
//
// GB300 realisation: all domains live on one GPU as one batched system (the same batching as
// the serving loop: atoms concatenated, per-domain neighbour lists concatenated with offsets),
// so every model kernel runs once over all domains.  The two exchanges of a multi-processor
// run become two kernels: before the step, copies take their owners' positions plus their
// image shift; after it, a gather over a per-atom list of copies adds up the partial forces in
// a fixed order (no atomics).  Each domain is an open subsystem in a cell scaled from the
// global one with a margin wider than the neighbour cutoff, so its neighbour search finds no
// periodic image.
//
// Decomposition (on the first call, on CTD_REBUILD, and whenever an atom has moved more than
// half the skin since the last one):
//   k_dom_frac        s = G x, f = s - floor(s) (canonical FP64 order), owner domain of f
//   k_dom_candidates  count / fill every image f + n inside a domain's box widened by the halo
//                     h_a = R_comm |G_a| (R_comm = T rc + skin: valid until the next rebuild)
//   per domain        Verlet list of the candidates in the domain's own cell
//   k_hop_step        hop levels from the owned atoms over the Verlet graph (a superset of
//                     every active graph until the next rebuild, so levels are never larger)
//   compact           keep level <= T; rebuild; near = level <= T - 1 (the per-step prune keeps
//                     an edge only if one of its atoms is near)
//   copies            per global atom, the batch indices of its copies, ascending
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.cuh"

namespace ctd {

constexpr int kDomMaxImg = 8;   // image range per direction searched for copies

struct DomBox {
  double lo[3], hi[3];   // fractional window [q/p - h, (q+1)/p + h) of the global cell
  double origin[3];      // Cartesian origin of the domain's cell
};

struct DomEdges {
  const int32_t* vrow;
  const int32_t* vcol;
  const float4* vbase;
  const int32_t* vrev;
  int64_t atom_off, edge_off;
  int32_t n, nv;
};

static inline unsigned dblk(int64_t w) { return (unsigned)((w + kThreads - 1) / kThreads); }

__device__ __forceinline__ double canon_frac(const CellGeom& g, int a, const double* x) {
  return __dadd_rn(__dadd_rn(__dmul_rn(g.G[3 * a], x[0]), __dmul_rn(g.G[3 * a + 1], x[1])),
                   __dmul_rn(g.G[3 * a + 2], x[2]));
}

// Wrapped fractional coordinates, wrap image and owner domain of every atom.
__global__ void k_dom_frac(int64_t n, const double* __restrict__ x, CellGeom g, int p0, int p1, int p2,
                           double* __restrict__ f, int32_t* __restrict__ wimg, int32_t* __restrict__ owner,
                           int* __restrict__ status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  const int p[3] = {p0, p1, p2};
  int q[3];
  bool ok = true;
  for (int a = 0; a < 3; ++a) {
    const double s = canon_frac(g, a, xi);
    ok = ok && isfinite(s) && fabs(s) < 1e9;
    const double fl = ok ? floor(s) : 0.0;
    const double fa = ok ? __dsub_rn(s, fl) : 0.0;
    f[3 * i + a] = fa;
    wimg[3 * i + a] = (int32_t)fl;
    int qa = (int)floor(fa * (double)p[a]);
    q[a] = qa < 0 ? 0 : (qa >= p[a] ? p[a] - 1 : qa);
  }
  if (!ok) atomicOr(status, (int)ST_NONFINITE);
  owner[i] = (q[0] * p1 + q[1]) * p2 + q[2];
}

// Images n (per direction, -m..m) of atom i that fall inside domain d's widened box.
__device__ __forceinline__ int dom_axis_images(double fa, double lo, double hi, int m, int* out) {
  int c = 0;
  for (int k = -m; k <= m; ++k) {
    const double u = __dadd_rn(fa, (double)k);
    if (u >= lo && u < hi) out[c++] = k;
  }
  return c;
}

// Count (FILL = false) or write (FILL = true) the copies of every atom in every domain.  Grid:
// x over atoms, y over domains.  count / off are [nd][n] (off = exclusive scan of count, nd n + 1
// entries).  A copy records its atom, its Cartesian shift (image of the raw position, minus the
// domain cell's origin) and whether it is the owned copy.
template <bool FILL>
__global__ void k_dom_candidates(int64_t n, const double* __restrict__ f, const int32_t* __restrict__ wimg,
                                 const int32_t* __restrict__ owner, const DomBox* __restrict__ boxes, int m0,
                                 int m1, int m2, CellGeom g, int32_t* __restrict__ count,
                                 const int32_t* __restrict__ off, int32_t* __restrict__ csrc,
                                 double* __restrict__ cshift, uint8_t* __restrict__ cown) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int d = blockIdx.y;
  if (i >= n) return;
  const DomBox B = boxes[d];
  const int mm[3] = {m0, m1, m2};
  int img[3][2 * kDomMaxImg + 1];
  int c[3];
  for (int a = 0; a < 3; ++a) c[a] = dom_axis_images(f[3 * i + a], B.lo[a], B.hi[a], mm[a], img[a]);
  const int64_t slot = (int64_t)d * n + i;
  if (!FILL) {
    count[slot] = c[0] * c[1] * c[2];
    return;
  }
  int64_t pos = off[slot];
  const bool mine = owner[i] == d;
  for (int u = 0; u < c[0]; ++u)
    for (int v = 0; v < c[1]; ++v)
      for (int w = 0; w < c[2]; ++w) {
        const int n0 = img[0][u], n1 = img[1][v], n2 = img[2][w];
        const double s0 = (double)(n0 - wimg[3 * i]), s1 = (double)(n1 - wimg[3 * i + 1]),
                     s2 = (double)(n2 - wimg[3 * i + 2]);
        for (int k = 0; k < 3; ++k)
          cshift[3 * pos + k] = __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(s0, g.H[k]), __dmul_rn(s1, g.H[3 + k])),
                                                    __dmul_rn(s2, g.H[6 + k])),
                                          B.origin[k]);
        csrc[pos] = (int32_t)i;
        cown[pos] = (mine && n0 == 0 && n1 == 0 && n2 == 0) ? 1 : 0;
        ++pos;
      }
}

// out[d] = off[d n] for d = 0..nd (domain boundaries of the scanned [nd][n] counts).
__global__ void k_dom_bounds(int nd, int64_t n, const int32_t* __restrict__ off, int64_t* __restrict__ out) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d <= nd) out[d] = off[(int64_t)d * n];
}

// out[d] = pos[at[d]] for d = 0..nd (domain boundaries after compaction).
__global__ void k_dom_gather_at(int nd, const int64_t* __restrict__ at, const int32_t* __restrict__ pos,
                                int64_t* __restrict__ out) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d <= nd) out[d] = pos[at[d]];
}

// Positions of copies: x[k] = x_glob[src[k]] + shift[k] (FP64).  Used at build and every step.
__global__ void k_dom_positions(int64_t m, const int32_t* __restrict__ src, const double* __restrict__ shift,
                                const double* __restrict__ xg, double* __restrict__ x) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= m) return;
  const int64_t i = src[k];
  for (int c = 0; c < 3; ++c) x[3 * k + c] = __dadd_rn(xg[3 * i + c], shift[3 * k + c]);
}

// Sorted copy metadata of one domain: out[k] = in[perm[k]] for the atom, shift and ownership.
__global__ void k_dom_gather_meta(int64_t n, const int32_t* __restrict__ perm, const int32_t* __restrict__ csrc,
                                  const double* __restrict__ cshift, const uint8_t* __restrict__ cown,
                                  int32_t* __restrict__ bsrc, double* __restrict__ bshift, uint8_t* __restrict__ bown) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t j = perm[k];
  bsrc[k] = csrc[j];
  for (int c = 0; c < 3; ++c) bshift[3 * k + c] = cshift[3 * j + c];
  bown[k] = cown[j];
}

__global__ void k_hop_init(int64_t n, const uint8_t* __restrict__ own, int32_t* __restrict__ lev) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n) lev[k] = own[k] ? 0 : 0x3fffffff;
}

// One warp per atom: an atom not yet reached gets level t if a neighbour has level t - 1.
// Levels set in this launch are t, never t - 1, so the result does not depend on the order.
__global__ void k_hop_step(int64_t n, const int32_t* __restrict__ vrow, const int32_t* __restrict__ vcol, int t,
                           int32_t* __restrict__ lev) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n || lev[i] < t) return;
  bool hit = false;
  for (int e = vrow[i] + lane; e < vrow[i + 1] && !hit; e += 32) hit = lev[vcol[e]] == t - 1;
  if (__any_sync(__activemask(), hit) && lane == 0) lev[i] = t;
}

// keep[perm[k]] = level[k] <= T (back to the candidate order of the domain).
__global__ void k_hop_keep(int64_t n, const int32_t* __restrict__ perm, const int32_t* __restrict__ lev, int T,
                           int32_t* __restrict__ keep) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n) keep[perm[k]] = lev[k] <= T ? 1 : 0;
}

// Compaction of the candidate arrays by the scanned keep flags.
__global__ void k_dom_compact(int64_t m, const int32_t* __restrict__ keep, const int32_t* __restrict__ pos,
                              const int32_t* __restrict__ csrc, const double* __restrict__ cshift,
                              const uint8_t* __restrict__ cown, int32_t* __restrict__ nsrc,
                              double* __restrict__ nshift, uint8_t* __restrict__ nown) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= m || !keep[k]) return;
  const int64_t p = pos[k];
  nsrc[p] = csrc[k];
  for (int c = 0; c < 3; ++c) nshift[3 * p + c] = cshift[3 * k + c];
  nown[p] = cown[k];
}

__global__ void k_dom_weights(int64_t n, const uint8_t* __restrict__ own, const int32_t* __restrict__ lev, int T,
                              float* __restrict__ ew, uint8_t* __restrict__ near) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  ew[k] = own[k] ? 1.0f : 0.0f;
  if (near) near[k] = lev[k] <= T - 1 ? 1 : 0;
}

__global__ void k_dom_concat(const DomEdges* __restrict__ doms, int32_t* __restrict__ vrow, int32_t* __restrict__ vcol,
                             float4* __restrict__ vbase, int32_t* __restrict__ vrev) {
  const DomEdges d = doms[blockIdx.y];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= (int64_t)d.n || k < d.nv;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (k <= d.n) vrow[d.atom_off + k] = (int32_t)(d.edge_off + d.vrow[k]);
    if (k < d.nv) {
      vcol[d.edge_off + k] = (int32_t)(d.atom_off + d.vcol[k]);
      vbase[d.edge_off + k] = d.vbase[k];
      vrev[d.edge_off + k] = (int32_t)(d.edge_off + d.vrev[k]);
    }
  }
}

// Copies of each global atom: counts, then a fill whose order within an atom is made
// ascending in the batch index by a rank sort (an atom has a handful of copies).
__global__ void k_copies_count(int64_t m, const int32_t* __restrict__ bsrc, int32_t* __restrict__ cnt) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < m) atomicAdd(&cnt[bsrc[k]], 1);
}
__global__ void k_copies_place(int64_t m, const int32_t* __restrict__ bsrc, const int32_t* __restrict__ cptr,
                               int32_t* __restrict__ cursor, int32_t* __restrict__ tmp) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= m) return;
  const int i = bsrc[k];
  tmp[cptr[i] + atomicAdd(&cursor[i], 1)] = (int32_t)k;
}
__global__ void k_copies_sort(int64_t n, const int32_t* __restrict__ cptr, const int32_t* __restrict__ tmp,
                              const uint8_t* __restrict__ bown, int32_t* __restrict__ clist,
                              int32_t* __restrict__ owned_copy, int* __restrict__ status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = cptr[i], e = cptr[i + 1];
  int own = -1, nown = 0;
  for (int k = b; k < e; ++k) {
    const int v = tmp[k];
    int rank = 0;
    for (int l = b; l < e; ++l) rank += tmp[l] < v;
    clist[b + rank] = v;
    if (bown[v]) {
      own = v;
      ++nown;
    }
  }
  owned_copy[i] = own;
  if (nown != 1) atomicOr(status, (int)ST_OWNERSHIP);   // every atom is owned exactly once
}

// Reverse exchange: F_i = sum over the copies of atom i of their partial forces (FP64, in the
// ascending batch order of the copies); optional per-atom energies from the owned copy.
__global__ void k_dom_forces(int64_t n, const int32_t* __restrict__ cptr, const int32_t* __restrict__ clist,
                             const float* __restrict__ fb, double* __restrict__ fout,
                             const int32_t* __restrict__ owned_copy, const float* __restrict__ eatom,
                             double* __restrict__ eout) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (fout) {
    double fx = 0.0, fy = 0.0, fz = 0.0;
    for (int k = cptr[i]; k < cptr[i + 1]; ++k) {
      const int64_t c = clist[k];
      fx += (double)fb[3 * c];
      fy += (double)fb[3 * c + 1];
      fz += (double)fb[3 * c + 2];
    }
    fout[3 * i] = fx;
    fout[3 * i + 1] = fy;
    fout[3 * i + 2] = fz;
  }
  if (eout) {
    const int oc = owned_copy[i];
    eout[i] = oc >= 0 ? (double)eatom[oc] : __longlong_as_double(0x7ff8000000000000LL);
  }
}

// Active edge offsets of the domains after a prune: out[d] = arow[atom_off[d]].
__global__ void k_dom_active(int nd, const int64_t* __restrict__ aoff, const int32_t* __restrict__ arow,
                             int64_t* __restrict__ out) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d <= nd) out[d] = arow[aoff[d]];
}

}  // namespace ctd

using namespace ctd;

namespace {

struct Dom {
  int64_t atom_off = 0, n = 0, n_owned = 0, n_candidates = 0, nv = 0, n_active = 0;
  CellGeom geom{};
  int64_t ncell = 0;
  double H[9];
  DBuf vrow, vcol, vbase, vrev;
};

}  // namespace

struct ctd_domains {
  ctd_ctx* c = nullptr;
  int p[3] = {1, 1, 1};
  int nd = 1;
  bool hop_prune = true;
  double skin = 1.0;
  std::string err;
  // global system (caller order)
  bool decomposed = false;
  int64_t N = 0;
  double H[9] = {0};
  DBuf x_glob, z_glob, f_out, e_out, frac, wimg, owner;
  // candidates (domain-major) and their compacted copy
  DBuf ccount, coff, csrc, cshift, cown, keep, kpos, nsrc, nshift, nown, bounds;
  // batch (per batched atom, sorted within each domain)
  DBuf bsrc, bshift, bown, lev, xc;
  // copies of each global atom
  DBuf cptr, clist, ccur, ctmp, owned_copy;
  // per-domain build scratch
  DBuf b_xw, b_wrap, b_cell, b_ccount, b_cstart, b_cursor, b_tmp, b_perm, b_inv, b_xws, b_count, b_img, b_scan;
  DBuf dtable, aoff, aout;
  std::vector<Dom> doms;
  std::vector<DBuf*> bufs() {
    return {&x_glob, &z_glob, &f_out, &e_out, &frac, &wimg, &owner, &ccount, &coff, &csrc, &cshift, &cown,
            &keep, &kpos, &nsrc, &nshift, &nown, &bounds, &bsrc, &bshift, &bown, &lev, &xc, &cptr, &clist,
            &ccur, &ctmp, &owned_copy, &b_xw, &b_wrap, &b_cell, &b_ccount, &b_cstart, &b_cursor, &b_tmp,
            &b_perm, &b_inv, &b_xws, &b_count, &b_img, &b_scan, &dtable, &aoff, &aout};
  }
};

namespace {

int dfail(ctd_domains* D, int code, const std::string& msg) {
  D->err = msg;
  return code;
}

void dfree(ctd_ctx* c, DBuf& b) {
  if (b.p) {
    cudaFree(b.p);
    c->held -= b.bytes;
    c->used -= b.need;
    b.p = nullptr;
    b.bytes = 0;
    b.need = 0;
  }
}

// Verlet list of domain d's atoms: positions of the copies in candidate order at xcand (FP64),
// ownership and sources in candidate order at (csrc, cshift, cown) + atom_off.  Writes the
// batch arrays (sorted positions, sources, shifts, ownership) at the domain's atom offset and
// the domain's own lists (local indices).
int build_domain(ctd_domains* D, Dom& M, const double* xcand, const int32_t* csrc, const double* cshift,
                 const uint8_t* cown) {
  ctd_ctx* c = D->c;
  cudaStream_t st = c->st;
  const int64_t n = M.n, off = M.atom_off, n1 = n > 0 ? n : 1;
  ENSURE(c, D->b_xw, sizeof(double) * 3 * n1);
  ENSURE(c, D->b_wrap, sizeof(int32_t) * 3 * n1);
  ENSURE(c, D->b_cell, sizeof(int32_t) * n1);
  ENSURE(c, D->b_ccount, sizeof(int32_t) * (M.ncell + 1));
  ENSURE(c, D->b_cstart, sizeof(int32_t) * (M.ncell + 1));
  ENSURE(c, D->b_cursor, sizeof(int32_t) * (M.ncell + 1));
  ENSURE(c, D->b_tmp, sizeof(int32_t) * n1);
  ENSURE(c, D->b_perm, sizeof(int32_t) * n1);
  ENSURE(c, D->b_inv, sizeof(int32_t) * n1);
  ENSURE(c, D->b_xws, sizeof(double) * 3 * n1);
  ENSURE(c, D->b_count, sizeof(int32_t) * n1);
  ENSURE(c, D->b_scan, scan_temp_bytes(std::max<int64_t>(n1, M.ncell)) + 64);
  ENSURE(c, M.vrow, sizeof(int32_t) * (n1 + 1));
  CUDA_OK(c, cudaMemsetAsync(D->b_ccount.p, 0, sizeof(int32_t) * M.ncell, st));
  CUDA_OK(c, cudaMemsetAsync(D->b_cursor.p, 0, sizeof(int32_t) * M.ncell, st));
  launch_wrap_bin(st, n, xcand, M.geom, P<double>(D->b_xw), P<int32_t>(D->b_wrap), P<int32_t>(D->b_cell),
                  P<int32_t>(D->b_ccount));
  launch_exclusive_scan(st, M.ncell, P<int32_t>(D->b_ccount), P<int32_t>(D->b_cstart), D->b_scan.p);
  launch_place(st, n, P<int32_t>(D->b_cell), P<int32_t>(D->b_cstart), P<int32_t>(D->b_cursor), P<int32_t>(D->b_tmp));
  launch_sort_cells(st, M.ncell, P<int32_t>(D->b_cstart), P<int32_t>(D->b_tmp), P<int32_t>(D->b_perm));
  // sorted positions: wrapped (pair search) and raw (= reference and current positions)
  launch_gather_sorted(st, n, P<int32_t>(D->b_perm), P<double>(D->b_xw), xcand, nullptr, P<double>(D->b_xws),
                       P<double>(c->xref_s) + 3 * off, nullptr, P<int32_t>(D->b_inv));
  CUDA_OK(c, cudaMemcpyAsync(P<double>(c->x_s) + 3 * off, P<double>(c->xref_s) + 3 * off, sizeof(double) * 3 * n,
                             cudaMemcpyDeviceToDevice, st));
  if (n > 0) {
    LaunchScope ls_(st);
    k_dom_gather_meta<<<dblk(n), kThreads, 0, st>>>(n, P<int32_t>(D->b_perm), csrc + off, cshift + 3 * off,
                                                   cown + off, P<int32_t>(D->bsrc) + off,
                                                   P<double>(D->bshift) + 3 * off, P<uint8_t>(D->bown) + off);
  }
  launch_pair_search(st, false, n, P<double>(D->b_xws), P<int32_t>(D->b_cstart), M.geom, P<int32_t>(D->b_count),
                     nullptr, nullptr, nullptr, nullptr);
  launch_exclusive_scan(st, n, P<int32_t>(D->b_count), P<int32_t>(M.vrow), D->b_scan.p);
  int32_t total = 0;
  CUDA_OK(c, cudaMemcpyAsync(&total, P<int32_t>(M.vrow) + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CUDA_OK(c, cudaStreamSynchronize(st));
  if (total < 0) return fail(c, CTD_ERR_CAPACITY, "domain has more than 2^31 neighbour pairs");
  const int64_t e1 = total > 0 ? total : 1;
  ENSURE(c, M.vcol, sizeof(int32_t) * e1);
  ENSURE(c, M.vbase, sizeof(float4) * e1);
  ENSURE(c, M.vrev, sizeof(int32_t) * e1);
  ENSURE(c, D->b_img, sizeof(uint32_t) * e1);
  launch_pair_search(st, true, n, P<double>(D->b_xws), P<int32_t>(D->b_cstart), M.geom, P<int32_t>(D->b_count),
                     P<int32_t>(M.vrow), P<int32_t>(M.vcol), P<uint32_t>(D->b_img), P<float4>(M.vbase));
  launch_reverse(st, n, P<int32_t>(M.vrow), P<int32_t>(M.vcol), P<uint32_t>(D->b_img), P<int32_t>(M.vrev),
                 P<int>(c->status));
  M.nv = total;
  return CTD_OK;
}

// Hop levels of one domain's atoms (batch arrays at its offset) over its Verlet list.
void hop_levels(ctd_domains* D, Dom& M, int T) {
  cudaStream_t st = D->c->st;
  if (M.n == 0) return;
  int32_t* lev = P<int32_t>(D->lev) + M.atom_off;
  { LaunchScope ls_(st); k_hop_init<<<dblk(M.n), kThreads, 0, st>>>(M.n, P<uint8_t>(D->bown) + M.atom_off, lev); }
  for (int t = 1; t <= T; ++t) {
    LaunchScope ls_(st);
    k_hop_step<<<dblk(M.n * 32), kThreads, 0, st>>>(M.n, P<int32_t>(M.vrow), P<int32_t>(M.vcol), t, lev);
  }
}

// Size the batch arrays for the current candidate set and set each domain's geometry.
int layout_batch(ctd_domains* D, const std::vector<int64_t>& counts) {
  ctd_ctx* c = D->c;
  int64_t off = 0;
  for (int d = 0; d < D->nd; ++d) {
    D->doms[d].atom_off = off;
    D->doms[d].n = counts[d];
    off += counts[d];
  }
  if (off > (int64_t)INT32_MAX / 4) return fail(c, CTD_ERR_CAPACITY, "decomposition has too many atoms and copies");
  const int64_t m1 = off > 0 ? off : 1;
  ENSURE(c, c->x_s, sizeof(double) * 3 * m1);
  ENSURE(c, c->xref_s, sizeof(double) * 3 * m1);
  ENSURE(c, c->z_s, sizeof(int32_t) * m1);
  ENSURE(c, D->bsrc, sizeof(int32_t) * m1);
  ENSURE(c, D->bshift, sizeof(double) * 3 * m1);
  ENSURE(c, D->bown, sizeof(uint8_t) * m1);
  ENSURE(c, D->lev, sizeof(int32_t) * m1);
  ENSURE(c, D->xc, sizeof(double) * 3 * m1);
  c->n = off;
  return CTD_OK;
}

// Hops of the model's receptive field: T layers of message passing reach T cutoffs; the strictly
// local family reaches one, whatever its layer count.
static int receptive_hops(const ctd_ctx* c) { return c->local() ? 1 : c->desc.T; }

// Build every domain on the candidates (src, shift, own) laid out domain-major per layout_batch,
// with hop levels; keep (optional, candidate order) receives level <= T.
int build_all(ctd_domains* D, const int32_t* src, const double* shift, const uint8_t* own, int32_t* keep) {
  ctd_ctx* c = D->c;
  cudaStream_t st = c->st;
  if (c->n > 0) {
    LaunchScope ls_(st);
    k_dom_positions<<<dblk(c->n), kThreads, 0, st>>>(c->n, src, shift, P<double>(D->x_glob), P<double>(D->xc));
  }
  for (Dom& M : D->doms) {
    int r = build_domain(D, M, P<double>(D->xc) + 3 * M.atom_off, src, shift, own);
    if (r) return r;
    hop_levels(D, M, receptive_hops(c));
    if (keep && M.n > 0) {   // the domain's sort permutation is still in b_perm here
      LaunchScope ls_(st);
      k_hop_keep<<<dblk(M.n), kThreads, 0, st>>>(M.n, P<int32_t>(D->b_perm), P<int32_t>(D->lev) + M.atom_off,
                                                 receptive_hops(c), keep + M.atom_off);
    }
  }
  return CTD_OK;
}

// Concatenate the domains' Verlet lists into the batch list (global indices).
int concat_domains(ctd_domains* D) {
  ctd_ctx* c = D->c;
  cudaStream_t st = c->st;
  std::vector<DomEdges> t;
  int64_t E = 0, maxw = 1;
  for (Dom& M : D->doms) {
    DomEdges q;
    q.vrow = P<int32_t>(M.vrow);
    q.vcol = P<int32_t>(M.vcol);
    q.vbase = P<float4>(M.vbase);
    q.vrev = P<int32_t>(M.vrev);
    q.atom_off = M.atom_off;
    q.edge_off = E;
    q.n = (int32_t)M.n;
    q.nv = (int32_t)M.nv;
    t.push_back(q);
    E += M.nv;
    maxw = std::max<int64_t>(maxw, std::max<int64_t>(M.n + 1, M.nv));
  }
  if (E > INT32_MAX) return fail(c, CTD_ERR_CAPACITY, "decomposition has more than 2^31 neighbour pairs");
  const int64_t N1 = c->n > 0 ? c->n : 1, E1 = E > 0 ? E : 1;
  ENSURE(c, c->vrow, sizeof(int32_t) * (N1 + 1));
  ENSURE(c, c->vcol, sizeof(int32_t) * E1);
  ENSURE(c, c->vbase, sizeof(float4) * E1);
  ENSURE(c, c->vrev, sizeof(int32_t) * E1);
  ENSURE(c, c->v2a, sizeof(int32_t) * E1);
  ENSURE(c, c->scan_tmp, scan_temp_bytes(N1) + 64);
  CUDA_OK(c, cudaMemsetAsync(c->vrow.p, 0, sizeof(int32_t), st));
  CUDA_OK(c, cudaMemcpyAsync(D->dtable.p, t.data(), sizeof(DomEdges) * t.size(), cudaMemcpyHostToDevice, st));
  {
    dim3 grid((unsigned)std::min<int64_t>((maxw + kThreads - 1) / kThreads, 4096), (unsigned)t.size());
    LaunchScope ls_(st);
    k_dom_concat<<<grid, kThreads, 0, st>>>(P<DomEdges>(D->dtable), P<int32_t>(c->vrow), P<int32_t>(c->vcol),
                                            P<float4>(c->vbase), P<int32_t>(c->vrev));
  }
  CUDA_OK(c, cudaStreamSynchronize(st));   // the descriptor table is host memory until here
  c->n_verlet = E;
  return CTD_OK;
}

// Per global atom, the batch indices of its copies (ascending) and of its owned copy.
int build_copies(ctd_domains* D) {
  ctd_ctx* c = D->c;
  cudaStream_t st = c->st;
  const int64_t N = D->N, N1 = N > 0 ? N : 1, M = c->n, M1 = M > 0 ? M : 1;
  ENSURE(c, D->ccur, sizeof(int32_t) * N1);
  ENSURE(c, D->cptr, sizeof(int32_t) * (N1 + 1));
  ENSURE(c, D->clist, sizeof(int32_t) * M1);
  ENSURE(c, D->ctmp, sizeof(int32_t) * M1);
  ENSURE(c, D->owned_copy, sizeof(int32_t) * N1);
  ENSURE(c, c->scan_tmp, scan_temp_bytes(N1) + 64);
  CUDA_OK(c, cudaMemsetAsync(D->ccur.p, 0, sizeof(int32_t) * N1, st));
  if (M > 0) {
    LaunchScope ls_(st);
    k_copies_count<<<dblk(M), kThreads, 0, st>>>(M, P<int32_t>(D->bsrc), P<int32_t>(D->ccur));
  }
  launch_exclusive_scan(st, N, P<int32_t>(D->ccur), P<int32_t>(D->cptr), c->scan_tmp.p);
  CUDA_OK(c, cudaMemsetAsync(D->ccur.p, 0, sizeof(int32_t) * N1, st));
  if (M > 0) {
    LaunchScope ls_(st);
    k_copies_place<<<dblk(M), kThreads, 0, st>>>(M, P<int32_t>(D->bsrc), P<int32_t>(D->cptr), P<int32_t>(D->ccur),
                                                P<int32_t>(D->ctmp));
  }
  if (N > 0) {
    LaunchScope ls_(st);
    k_copies_sort<<<dblk(N), kThreads, 0, st>>>(N, P<int32_t>(D->cptr), P<int32_t>(D->ctmp), P<uint8_t>(D->bown),
                                               P<int32_t>(D->clist), P<int32_t>(D->owned_copy), P<int>(c->status));
  }
  return CTD_OK;
}

int decompose(ctd_domains* D) {
  ctd_ctx* c = D->c;
  cudaStream_t st = c->st;
  StageGuard sg(STG_BUILD);
  D->decomposed = false;   // until every buffer below is consistent again
  const int64_t N = D->N, N1 = N > 0 ? N : 1;
  const int nd = D->nd, T = receptive_hops(c);
  const double rcomm = T * c->desc.rc + D->skin;
  const double R = c->desc.rc + D->skin;
  CellGeom g{};
  int64_t nc_unused = 0;
  int r = setup_geometry_into(c, g, &nc_unused, D->H, R);
  if (r) return r;
  double h[3], margin[3];
  int m[3];
  for (int a = 0; a < 3; ++a) {
    const double gn =
        std::sqrt(g.G[3 * a] * g.G[3 * a] + g.G[3 * a + 1] * g.G[3 * a + 1] + g.G[3 * a + 2] * g.G[3 * a + 2]);
    h[a] = rcomm * gn;
    margin[a] = 1.05 * R * gn + 1e-9;
    m[a] = (int)std::ceil(h[a]) + 1;
    if (m[a] > kDomMaxImg)
      return fail(c, CTD_ERR_CELL_TOO_SMALL, "halo spans more than 7 cell widths along a lattice direction");
  }
  std::vector<DomBox> boxes(nd);
  D->doms.resize(nd);
  for (int q0 = 0; q0 < D->p[0]; ++q0)
    for (int q1 = 0; q1 < D->p[1]; ++q1)
      for (int q2 = 0; q2 < D->p[2]; ++q2) {
        const int d = (q0 * D->p[1] + q1) * D->p[2] + q2;
        const int q[3] = {q0, q1, q2};
        DomBox& B = boxes[d];
        double Hd[9], lo_cell[3];
        for (int a = 0; a < 3; ++a) {
          B.lo[a] = (double)q[a] / D->p[a] - h[a];
          B.hi[a] = (double)(q[a] + 1) / D->p[a] + h[a];
          const double alpha = (B.hi[a] - B.lo[a]) + margin[a];
          lo_cell[a] = B.lo[a] - 0.5 * margin[a];
          for (int k = 0; k < 3; ++k) Hd[3 * a + k] = alpha * D->H[3 * a + k];
        }
        for (int k = 0; k < 3; ++k)
          B.origin[k] = (lo_cell[0] * D->H[k] + lo_cell[1] * D->H[3 + k]) + lo_cell[2] * D->H[6 + k];
        Dom& M = D->doms[d];
        memcpy(M.H, Hd, sizeof(Hd));
        r = setup_geometry_into(c, M.geom, &M.ncell, Hd, R);
        if (r) return r;
      }
  // 1. fractional coordinates and owners
  ENSURE(c, D->frac, sizeof(double) * 3 * N1);
  ENSURE(c, D->wimg, sizeof(int32_t) * 3 * N1);
  ENSURE(c, D->owner, sizeof(int32_t) * N1);
  ENSURE(c, c->status, sizeof(int32_t) * 4);
  CUDA_OK(c, cudaMemsetAsync(c->status.p, 0, sizeof(int32_t), st));
  if (N > 0) {
    LaunchScope ls_(st);
    k_dom_frac<<<dblk(N), kThreads, 0, st>>>(N, P<double>(D->x_glob), g, D->p[0], D->p[1], D->p[2],
                                            P<double>(D->frac), P<int32_t>(D->wimg), P<int32_t>(D->owner),
                                            P<int>(c->status));
  }
  r = check_status(c);
  if (r) return r;
  // 2. candidate copies: count, scan, fill (domain-major)
  const int64_t PN = (int64_t)nd * N;
  if (PN >= (int64_t)INT32_MAX) return fail(c, CTD_ERR_CAPACITY, "domains x atoms exceeds 2^31");
  ENSURE(c, D->ccount, sizeof(int32_t) * (PN > 0 ? PN : 1));
  ENSURE(c, D->coff, sizeof(int32_t) * (PN + 1));
  ENSURE(c, D->bounds, sizeof(int64_t) * (nd + 1));
  ENSURE(c, D->dtable, std::max(sizeof(DomBox), sizeof(DomEdges)) * nd);
  ENSURE(c, c->scan_tmp, scan_temp_bytes(std::max<int64_t>(PN, N1)) + 64);
  CUDA_OK(c, cudaMemcpyAsync(D->dtable.p, boxes.data(), sizeof(DomBox) * nd, cudaMemcpyHostToDevice, st));
  const dim3 grid(dblk(N1), (unsigned)nd);
  {
    LaunchScope ls_(st);
    k_dom_candidates<false><<<grid, kThreads, 0, st>>>(N, P<double>(D->frac), P<int32_t>(D->wimg),
                                                      P<int32_t>(D->owner), P<DomBox>(D->dtable), m[0], m[1], m[2],
                                                      g, P<int32_t>(D->ccount), nullptr, nullptr, nullptr, nullptr);
  }
  launch_exclusive_scan(st, PN, P<int32_t>(D->ccount), P<int32_t>(D->coff), c->scan_tmp.p);
  {
    LaunchScope ls_(st);
    k_dom_bounds<<<dblk(nd + 1), kThreads, 0, st>>>(nd, N, P<int32_t>(D->coff), P<int64_t>(D->bounds));
  }
  std::vector<int64_t> bnd(nd + 1);
  CUDA_OK(c, cudaMemcpyAsync(bnd.data(), D->bounds.p, sizeof(int64_t) * (nd + 1), cudaMemcpyDeviceToHost, st));
  CUDA_OK(c, cudaStreamSynchronize(st));   // also: the box table is host memory until here
  if (bnd[nd] < 0) return fail(c, CTD_ERR_CAPACITY, "more than 2^31 copies");
  const int64_t M0 = bnd[nd], M01 = M0 > 0 ? M0 : 1;
  ENSURE(c, D->csrc, sizeof(int32_t) * M01);
  ENSURE(c, D->cshift, sizeof(double) * 3 * M01);
  ENSURE(c, D->cown, sizeof(uint8_t) * M01);
  {
    LaunchScope ls_(st);
    k_dom_candidates<true><<<grid, kThreads, 0, st>>>(N, P<double>(D->frac), P<int32_t>(D->wimg),
                                                     P<int32_t>(D->owner), P<DomBox>(D->dtable), m[0], m[1], m[2],
                                                     g, nullptr, P<int32_t>(D->coff), P<int32_t>(D->csrc),
                                                     P<double>(D->cshift), P<uint8_t>(D->cown));
  }
  std::vector<int64_t> counts(nd);
  for (int d = 0; d < nd; ++d) {
    counts[d] = bnd[d + 1] - bnd[d];
    D->doms[d].n_candidates = counts[d];
  }
  r = layout_batch(D, counts);
  if (r) return r;
  if (D->hop_prune) {
    // 3. hop pruning: keep the copies within T hops of an owned atom and build again
    ENSURE(c, D->keep, sizeof(int32_t) * M01);
    ENSURE(c, D->kpos, sizeof(int32_t) * (M0 + 1));
    ENSURE(c, c->scan_tmp, scan_temp_bytes(M01) + 64);   // M0 can exceed domains x atoms
    r = build_all(D, P<int32_t>(D->csrc), P<double>(D->cshift), P<uint8_t>(D->cown), P<int32_t>(D->keep));
    if (r) return r;
    launch_exclusive_scan(st, M0, P<int32_t>(D->keep), P<int32_t>(D->kpos), c->scan_tmp.p);
    std::vector<int64_t> kb(nd + 1);
    ENSURE(c, D->aout, sizeof(int64_t) * (nd + 1));
    {
      LaunchScope ls_(st);
      k_dom_gather_at<<<dblk(nd + 1), kThreads, 0, st>>>(nd, P<int64_t>(D->bounds), P<int32_t>(D->kpos),
                                                        P<int64_t>(D->aout));
    }
    CUDA_OK(c, cudaMemcpyAsync(kb.data(), D->aout.p, sizeof(int64_t) * (nd + 1), cudaMemcpyDeviceToHost, st));
    CUDA_OK(c, cudaStreamSynchronize(st));
    const int64_t M1 = kb[nd] > 0 ? kb[nd] : 1;
    ENSURE(c, D->nsrc, sizeof(int32_t) * M1);
    ENSURE(c, D->nshift, sizeof(double) * 3 * M1);
    ENSURE(c, D->nown, sizeof(uint8_t) * M1);
    if (M0 > 0) {
      LaunchScope ls_(st);
      k_dom_compact<<<dblk(M0), kThreads, 0, st>>>(M0, P<int32_t>(D->keep), P<int32_t>(D->kpos), P<int32_t>(D->csrc),
                                                   P<double>(D->cshift), P<uint8_t>(D->cown), P<int32_t>(D->nsrc),
                                                   P<double>(D->nshift), P<uint8_t>(D->nown));
    }
    for (int d = 0; d < nd; ++d) counts[d] = kb[d + 1] - kb[d];
    r = layout_batch(D, counts);
    if (r) return r;
    r = build_all(D, P<int32_t>(D->nsrc), P<double>(D->nshift), P<uint8_t>(D->nown), nullptr);
    if (r) return r;
  } else {
    r = build_all(D, P<int32_t>(D->csrc), P<double>(D->cshift), P<uint8_t>(D->cown), nullptr);
    if (r) return r;
  }
  // 4. energy weights, near flags, batch lists, copies of each atom
  const int64_t Mb = c->n, Mb1 = Mb > 0 ? Mb : 1;
  ENSURE(c, c->ew, sizeof(float) * Mb1);
  ENSURE(c, c->near, sizeof(uint8_t) * Mb1);
  if (Mb > 0) {
    LaunchScope ls_(st);
    k_dom_weights<<<dblk(Mb), kThreads, 0, st>>>(Mb, P<uint8_t>(D->bown), P<int32_t>(D->lev), T, P<float>(c->ew),
                                                 D->hop_prune ? P<uint8_t>(c->near) : nullptr);
  }
  c->use_ew = true;
  c->use_near = D->hop_prune;
  r = concat_domains(D);
  if (r) return r;
  r = build_copies(D);
  if (r) return r;
  r = check_status(c);
  if (r) return r;
  for (Dom& M : D->doms) M.n_owned = 0;
  {
    std::vector<int32_t> own(N1);
    CUDA_OK(c, cudaMemcpyAsync(own.data(), D->owner.p, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st));
    CUDA_OK(c, cudaStreamSynchronize(st));
    for (int64_t i = 0; i < N; ++i) ++D->doms[own[i]].n_owned;
  }
  c->have_list = true;
  D->decomposed = true;
  return CTD_OK;
}

}  // namespace

extern "C" {

int ctd_domains_create(ctd_domains** out, const ctd_model_desc* desc, const void* params, size_t nbytes,
                       size_t hbm_budget_bytes, const int32_t grid[3], int32_t hop_prune, double skin,
                       void* cuda_stream) {
  if (!out || !desc || !grid || !(skin >= 0.0) || !std::isfinite(skin)) return CTD_ERR_INVALID_ARG;
  *out = nullptr;
  for (int a = 0; a < 3; ++a)
    if (grid[a] < 1 || grid[a] > 64) return CTD_ERR_INVALID_ARG;
  if ((int64_t)grid[0] * grid[1] * grid[2] > 4096) return CTD_ERR_INVALID_ARG;
  ctd_ctx* c = nullptr;
  int r = ctd_create(&c, desc, hbm_budget_bytes, cuda_stream);
  if (r) return r;
  r = ctd_load_params(c, params, nbytes);
  if (r) {
    ctd_destroy(c);
    return r;
  }
  ctd_domains* D = new ctd_domains();
  D->c = c;
  for (int a = 0; a < 3; ++a) D->p[a] = grid[a];
  D->nd = grid[0] * grid[1] * grid[2];
  D->hop_prune = hop_prune != 0;
  D->skin = skin;
  *out = D;
  return CTD_OK;
}

void ctd_domains_destroy(ctd_domains* D) {
  if (!D) return;
  if (D->c) cudaStreamSynchronize(D->c->st);
  for (Dom& M : D->doms) {
    dfree(D->c, M.vrow);
    dfree(D->c, M.vcol);
    dfree(D->c, M.vbase);
    dfree(D->c, M.vrev);
  }
  for (DBuf* b : D->bufs()) dfree(D->c, *b);
  ctd_destroy(D->c);
  delete D;
}

const char* ctd_domains_last_error(ctd_domains* D) {
  if (!D) return "null decomposition";
  return D->err.empty() ? ctd_last_error(D->c) : D->err.c_str();
}

ctd_ctx* ctd_domains_context(ctd_domains* D) { return D ? D->c : nullptr; }

int ctd_domains_compute(ctd_domains* D, int64_t n, const int32_t* species, const double* positions,
                        const double cell[9], int32_t flags, double* energy, double* forces, double* virial,
                        ctd_stats* stats) {
  if (!D) return CTD_ERR_INVALID_ARG;
  ctd_ctx* c = D->c;
  Bind bind_(c);
  D->err.clear();
  if (n < 0 || (n > 0 && (!positions || !species)) || !cell || !energy)
    return dfail(D, CTD_ERR_INVALID_ARG, "bad arguments");
  if (((flags & CTD_NEED_FORCES) && !forces) || ((flags & CTD_NEED_VIRIAL) && !virial))
    return dfail(D, CTD_ERR_INVALID_ARG, "forces / virial requested without an output array");
  if (!finite_cell(cell)) return dfail(D, CTD_ERR_INVALID_ARG, "cell is singular or not finite");
  if (n > (int64_t)INT32_MAX / 64) return dfail(D, CTD_ERR_INVALID_ARG, "too many atoms");
  cudaStream_t st = c->st;
  const bool dev = flags & CTD_DEVICE_PTRS;
  if (n == 0) {   // nothing to decompose: zero energy and virial
    const double zero[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const cudaMemcpyKind k = dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    CUDA_OK(c, cudaMemcpy(energy, zero, sizeof(double), k));
    if (flags & CTD_NEED_VIRIAL) CUDA_OK(c, cudaMemcpy(virial, zero, sizeof(zero), k));
    if (stats) memset(stats, 0, sizeof(*stats));
    return CTD_OK;
  }
  const int64_t n1 = n;
  cudaEvent_t ev[3];
  const bool timing = stats != nullptr;
  if (timing)
    for (auto& e : ev) cudaEventCreate(&e);
  ENSURE(c, D->x_glob, sizeof(double) * 3 * n1);
  ENSURE(c, D->z_glob, sizeof(int32_t) * n1);
  int r = copy_in(c, D->x_glob.p, positions, sizeof(double) * 3 * n, dev);
  if (r) return r;
  r = copy_in(c, D->z_glob.p, species, sizeof(int32_t) * n, dev);
  if (r) return r;
  if (timing) cudaEventRecord(ev[0], st);
  bool need = (flags & CTD_REBUILD) || !D->decomposed || n != D->N || memcmp(cell, D->H, sizeof(double) * 9) != 0;
  int32_t rebuilt = 0;
  double md = 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    if (need) {
      D->N = n;
      memcpy(D->H, cell, sizeof(double) * 9);
      r = decompose(D);
      if (r) return r;
      rebuilt = 1;
    }
    // forward exchange: every copy takes its atom's position plus its image shift
    if (c->n > 0) {
      StageGuard sg(STG_PRUNE);
      LaunchScope ls_(st);
      k_dom_positions<<<dblk(c->n), kThreads, 0, st>>>(c->n, P<int32_t>(D->bsrc), P<double>(D->bshift),
                                                      P<double>(D->x_glob), P<double>(c->x_s));
    }
    r = prune(c, &md);
    if (r) return r;
    if (need) break;
    if (!(md <= 0.5 * D->skin)) need = true;   // also catches non-finite displacements
    else break;
  }
  launch_gather_i32(st, c->n, P<int32_t>(D->bsrc), P<int32_t>(D->z_glob), P<int32_t>(c->z_s));
  if (timing) cudaEventRecord(ev[1], st);
  const bool need_grad = flags & (CTD_NEED_FORCES | CTD_NEED_VIRIAL);
  CUDA_OK(c, cudaMemsetAsync(c->status.p, 0, sizeof(int32_t), st));
  r = evaluate(c, need_grad);
  if (r) return r;
  // reverse exchange: partial forces of the copies summed onto their atoms
  ENSURE(c, D->f_out, sizeof(double) * 3 * n1);
  ENSURE(c, D->e_out, sizeof(double) * n1);
  double* fdst = (flags & CTD_NEED_FORCES) ? (dev ? forces : P<double>(D->f_out)) : nullptr;
  double* edst = c->energy_out_user ? (dev ? c->energy_out_user : P<double>(D->e_out)) : nullptr;
  if (n > 0 && (fdst || edst)) {
    StageGuard sg(STG_FORCES);
    LaunchScope ls_(st);
    k_dom_forces<<<dblk(n), kThreads, 0, st>>>(n, P<int32_t>(D->cptr), P<int32_t>(D->clist), P<float>(c->force_s),
                                              fdst, P<int32_t>(D->owned_copy), P<float>(c->eatom), edst);
  }
  if (timing) cudaEventRecord(ev[2], st);
  launch_check_finite(st, 1, P<double>(c->out_e), P<int>(c->status));
  if (fdst) launch_check_finite(st, 3 * n, fdst, P<int>(c->status));
  const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CUDA_OK(c, cudaMemcpyAsync(energy, c->out_e.p, sizeof(double), kind, st));
  if (flags & CTD_NEED_VIRIAL) CUDA_OK(c, cudaMemcpyAsync(virial, c->out_w.p, sizeof(double) * 9, kind, st));
  if (!dev && (flags & CTD_NEED_FORCES))
    CUDA_OK(c, cudaMemcpyAsync(forces, D->f_out.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
  if (!dev && c->energy_out_user)
    CUDA_OK(c, cudaMemcpyAsync(c->energy_out_user, D->e_out.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  // active edges per domain
  const int nd = D->nd;
  ENSURE(c, D->aoff, sizeof(int64_t) * (nd + 1));
  ENSURE(c, D->aout, sizeof(int64_t) * (nd + 1));
  std::vector<int64_t> ao(nd + 1), act(nd + 1);
  for (int d = 0; d < nd; ++d) ao[d] = D->doms[d].atom_off;
  ao[nd] = c->n;
  CUDA_OK(c, cudaMemcpyAsync(D->aoff.p, ao.data(), sizeof(int64_t) * (nd + 1), cudaMemcpyHostToDevice, st));
  {
    LaunchScope ls_(st);
    k_dom_active<<<dblk(nd + 1), kThreads, 0, st>>>(nd, P<int64_t>(D->aoff), P<int32_t>(c->arow), P<int64_t>(D->aout));
  }
  CUDA_OK(c, cudaMemcpyAsync(act.data(), D->aout.p, sizeof(int64_t) * (nd + 1), cudaMemcpyDeviceToHost, st));
  r = check_status(c);   // synchronises the stream
  if (r) return r;
  for (int d = 0; d < nd; ++d) D->doms[d].n_active = act[d + 1] - act[d];
  if (stats) {
    stats->n_atoms = c->n;
    stats->n_verlet_edges = c->n_verlet;
    stats->n_active_edges = act[nd];
    stats->rebuilt = rebuilt;
    stats->retries = 0;
    stats->max_displacement = md;
    stats->bytes_allocated = (int64_t)c->held;
    stats->edges_stored = c->last_stored ? 1 : 0;
    cudaEventElapsedTime(&stats->ms_neighbors, ev[0], ev[1]);
    cudaEventElapsedTime(&stats->ms_model, ev[1], ev[2]);
    for (auto& e : ev) cudaEventDestroy(e);
  }
  return CTD_OK;
}

int ctd_domains_info(ctd_domains* D, int32_t domain, ctd_domain_info* info) {
  if (!D || !info) return CTD_ERR_INVALID_ARG;
  if (!D->decomposed) return dfail(D, CTD_ERR_STATE, "no decomposition yet");
  if (domain < 0 || domain >= D->nd) return dfail(D, CTD_ERR_INVALID_ARG, "domain index out of range");
  const Dom& M = D->doms[domain];
  info->n_owned = M.n_owned;
  info->n_copies = M.n - M.n_owned;
  info->n_candidates = M.n_candidates - M.n_owned;
  info->n_verlet_edges = M.nv;
  info->n_active_edges = M.n_active;
  for (int a = 0; a < 3; ++a) info->grid_index[a] = 0;
  int d = domain;
  info->grid_index[2] = d % D->p[2];
  d /= D->p[2];
  info->grid_index[1] = d % D->p[1];
  info->grid_index[0] = d / D->p[1];
  return CTD_OK;
}

}  // extern "C"
