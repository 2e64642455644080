/*
 * oracle.c -- plain, slow FP64 CPU reference for the PaiNN-form energy / force / virial path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or execute this file;
 * it is used by tests/, by __graft_entry__.smoke() and by the benchmark's CPU-baseline leg.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Compile with -ffp-contract=off: the canonical pair test below must round every product and
 * sum separately so that its result is reproducible bit for bit.
 *
 * What it computes (arXiv 2506.04055, Methods "(Semi-)Local Potential Models", Eq. for U;
 * Results "Distributed potential computation", sum-rule Eq. for f_i):
 *   U = sum_i U_i(r_i, A_i) over a periodic neighbour graph with cutoff R (5 A, Sec. "Training
 *   Details"), forces f_i = -dU/dr_i (the sum-rule equation's sign; the Methods line that
 *   writes f_i = dU/dr_i without the minus is read as a typo), virial W = -sum_e r_e (x) dU/dr_e.
 * The message-passing form (Methods "Graph Neural Networks", message and update equations) is
 * instantiated as PaiNN (cited in "Chosen Architectures"); the paper prints no PaiNN equations,
 * so the layer below follows the PaiNN definition with these readings:
 *   rbf_k(d) = exp(-(d-mu_k)^2 / (2 sigma^2)), mu_k = k rc/(K-1), sigma = rc/(K-1)
 *   f_c(d)   = (cos(pi d / rc) + 1) / 2 for d < rc, else 0
 *   message : phi_j = W2 silu(W1 s_j + b1) + b2 = [phi_s | phi_vv | phi_vs]
 *             W_e   = (Wf rbf(d_e) + bf) f_c(d_e)  = [W_s | W_vv | W_vs]
 *             s_i  += sum_e phi_s,j W_s,e
 *             v_i  += sum_e ( v_j phi_vv,j W_vv,e + u_e (x) phi_vs,j W_vs,e ),  u_e = r_e / d_e
 *   update  : Uv = U v, Vv = V v (per spatial component), nV = sqrt(sum_a Vv_a^2 + eps)
 *             a = A2 silu(A1 [s ; nV] + c1) + c2 = [a_vv | a_sv | a_ss]
 *             v += a_vv Uv ;  s += a_ss + a_sv <Uv, Vv>
 *   readout : U_i = e_scale (R2 . silu(R1 s_i + d1) + d2)
 * Edge e = (i <- j, n) has r_e = x_j - x_i + n1 a + n2 b + n3 c (cell rows a, b, c).
 *
 * The backward pass is reverse-mode differentiation of exactly these loops, written by hand.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_MAXT 16

/* ------------------------------------------------------------------------------------------
 * Cell geometry: G = H^{-T} by cofactors (rows of H are the lattice vectors), so that the
 * fractional coordinates of x are s = G x.  The expression order is fixed; see the pair test.
 * ---------------------------------------------------------------------------------------- */
void orc_inv_transpose(const double H[9], double G[9]) {
  double c00 = H[4] * H[8] - H[5] * H[7];
  double c01 = H[5] * H[6] - H[3] * H[8];
  double c02 = H[3] * H[7] - H[4] * H[6];
  double c10 = H[2] * H[7] - H[1] * H[8];
  double c11 = H[0] * H[8] - H[2] * H[6];
  double c12 = H[1] * H[6] - H[0] * H[7];
  double c20 = H[1] * H[5] - H[2] * H[4];
  double c21 = H[2] * H[3] - H[0] * H[5];
  double c22 = H[0] * H[4] - H[1] * H[3];
  double det = (H[0] * c00 + H[1] * c01) + H[2] * c02;
  G[0] = c00 / det; G[1] = c01 / det; G[2] = c02 / det;
  G[3] = c10 / det; G[4] = c11 / det; G[5] = c12 / det;
  G[6] = c20 / det; G[7] = c21 / det; G[8] = c22 / det;
}

/* Perpendicular width of the cell along lattice direction a: 1 / |row a of G|. */
static double perp_width(const double G[9], int a) {
  return 1.0 / sqrt(G[3 * a] * G[3 * a] + G[3 * a + 1] * G[3 * a + 1] + G[3 * a + 2] * G[3 * a + 2]);
}

/* Wrap positions into the cell: s = G x, f = s - floor(s), xw = f1 a + f2 b + f3 c.
 * Also returns the integer lattice translation m = floor(s) removed from each atom. */
void orc_wrap(int64_t n, const double *x, const double H[9], double *xw, int32_t *m) {
  double G[9];
  orc_inv_transpose(H, G);
  for (int64_t i = 0; i < n; ++i) {
    double f[3];
    for (int a = 0; a < 3; ++a) {
      double s = (G[3 * a] * x[3 * i] + G[3 * a + 1] * x[3 * i + 1]) + G[3 * a + 2] * x[3 * i + 2];
      double fl = floor(s);
      f[a] = s - fl;
      if (m) m[3 * i + a] = (int32_t)fl;
    }
    for (int c = 0; c < 3; ++c)
      xw[3 * i + c] = (f[0] * H[c] + f[1] * H[3 + c]) + f[2] * H[6 + c];
  }
}

/* Canonical pair test (the neighbour criterion "closer than a cutoff", Methods Eq. for U and
 * Results "Distributed potential computation"):
 *   d_c = (xw_j,c - xw_i,c) + ((n1 a_c + n2 b_c) + n3 c_c),  d2 = (d_0^2 + d_1^2) + d_2^2,
 *   keep iff d2 < R*R, excluding i == j with n = 0.                                         */
static int pair_keep(const double *xi, const double *xj, const double H[9], int n1, int n2, int n3,
                     double R2) {
  double d2 = 0.0, d[3];
  for (int c = 0; c < 3; ++c) {
    double sh = ((double)n1 * H[c] + (double)n2 * H[3 + c]) + (double)n3 * H[6 + c];
    d[c] = (xj[c] - xi[c]) + sh;
  }
  d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
  return d2 < R2;
}

/* Brute-force O(N^2 * images) search over wrapped positions.  Images n_a in [-m_a, m_a] with
 * m_a = ceil(R / w_a) + 1, which covers every image within R.  Output is ordered by
 * (i, j, n1, n2, n3) by construction.  Returns the number of pairs; writes at most cap. */
int64_t orc_pairs_brute(int64_t n, const double *xw, const double H[9], double R, int32_t *pi,
                        int32_t *pj, int8_t *pn, int64_t cap) {
  double G[9];
  orc_inv_transpose(H, G);
  int m[3];
  for (int a = 0; a < 3; ++a) m[a] = (int)ceil(R / perp_width(G, a)) + 1;
  double R2 = R * R;
  int64_t cnt = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j)
      for (int n1 = -m[0]; n1 <= m[0]; ++n1)
        for (int n2 = -m[1]; n2 <= m[1]; ++n2)
          for (int n3 = -m[2]; n3 <= m[2]; ++n3) {
            if (i == j && n1 == 0 && n2 == 0 && n3 == 0) continue;
            if (!pair_keep(&xw[3 * i], &xw[3 * j], H, n1, n2, n3, R2)) continue;
            if (cnt < cap) {
              pi[cnt] = (int32_t)i; pj[cnt] = (int32_t)j;
              pn[3 * cnt] = (int8_t)n1; pn[3 * cnt + 1] = (int8_t)n2; pn[3 * cnt + 2] = (int8_t)n3;
            }
            ++cnt;
          }
  return cnt;
}

/* Linked-cell search over the same wrapped positions and the same pair test.  The cell is cut
 * into nc_a = max(1, floor(w_a / (R (1+1e-6)))) slabs per lattice direction; an atom is in
 * slab floor(f_a nc_a) (clamped).  Neighbour slabs within +-M_a = ceil(R nc_a (1+1e-6) / w_a)
 * are visited; slab index c + dc maps to slab (c+dc) mod nc_a seen through image
 * floor((c+dc)/nc_a).  Output order is unspecified (callers sort). */
int64_t orc_pairs_cells(int64_t n, const double *xw, const double H[9], double R, int32_t *pi,
                        int32_t *pj, int8_t *pn, int64_t cap) {
  double G[9];
  orc_inv_transpose(H, G);
  int nc[3], M[3];
  for (int a = 0; a < 3; ++a) {
    double w = perp_width(G, a);
    nc[a] = (int)floor(w / (R * (1.0 + 1e-6)));
    if (nc[a] < 1) nc[a] = 1;
    M[a] = (int)ceil(R * nc[a] * (1.0 + 1e-6) / w);
  }
  int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
  int64_t *head = (int64_t *)malloc(sizeof(int64_t) * ncell);
  int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  int32_t *cid = (int32_t *)malloc(sizeof(int32_t) * 3 * (n > 0 ? n : 1));
  if (!head || !next || !cid) { free(head); free(next); free(cid); return ORC_ENOMEM; }
  for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
  for (int64_t i = n - 1; i >= 0; --i) {
    for (int a = 0; a < 3; ++a) {
      double s = (G[3 * a] * xw[3 * i] + G[3 * a + 1] * xw[3 * i + 1]) + G[3 * a + 2] * xw[3 * i + 2];
      int c = (int)floor(s * nc[a]);
      if (c < 0) c = 0;
      if (c >= nc[a]) c = nc[a] - 1;
      cid[3 * i + a] = c;
    }
    int64_t lin = ((int64_t)cid[3 * i] * nc[1] + cid[3 * i + 1]) * nc[2] + cid[3 * i + 2];
    next[i] = head[lin];
    head[lin] = i;
  }
  double R2 = R * R;
  int64_t cnt = 0;
  for (int64_t i = 0; i < n; ++i) {
    for (int d0 = -M[0]; d0 <= M[0]; ++d0)
      for (int d1 = -M[1]; d1 <= M[1]; ++d1)
        for (int d2 = -M[2]; d2 <= M[2]; ++d2) {
          int cc[3] = {cid[3 * i] + d0, cid[3 * i + 1] + d1, cid[3 * i + 2] + d2};
          int img[3], w[3];
          for (int a = 0; a < 3; ++a) {
            /* floor division and non-negative remainder */
            int q = cc[a] >= 0 ? cc[a] / nc[a] : -((-cc[a] + nc[a] - 1) / nc[a]);
            img[a] = q;
            w[a] = cc[a] - q * nc[a];
          }
          int64_t lin = ((int64_t)w[0] * nc[1] + w[1]) * nc[2] + w[2];
          for (int64_t j = head[lin]; j >= 0; j = next[j]) {
            if (i == j && img[0] == 0 && img[1] == 0 && img[2] == 0) continue;
            if (!pair_keep(&xw[3 * i], &xw[3 * j], H, img[0], img[1], img[2], R2)) continue;
            if (cnt < cap) {
              pi[cnt] = (int32_t)i; pj[cnt] = (int32_t)j;
              pn[3 * cnt] = (int8_t)img[0]; pn[3 * cnt + 1] = (int8_t)img[1]; pn[3 * cnt + 2] = (int8_t)img[2];
            }
            ++cnt;
          }
        }
  }
  free(head); free(next); free(cid);
  return cnt;
}

/* ------------------------------------------------------------------------------------------
 * PaiNN-form potential.  Parameter vector layout (float64, matrices row-major [out][in]):
 *   emb[S][F]; per layer t: W1[F][F] b1[F] W2[3F][F] b2[3F] Wf[3F][K] bf[3F] U[F][F] V[F][F]
 *   A1[F][2F] c1[F] A2[3F][F] c2[3F]; then R1[F/2][F] d1[F/2] R2[F/2] d2[1].
 * ---------------------------------------------------------------------------------------- */
typedef struct {
  int32_t F, K, T, S;
  double rc, eps, e_scale;
} orc_model;

typedef struct {
  const double *W1, *b1, *W2, *b2, *Wf, *bf, *U, *V, *A1, *c1, *A2, *c2;
} orc_layer;

typedef struct {
  const double *emb, *R1, *d1, *R2, *d2;
  orc_layer L[ORC_MAXT];
} orc_params;

int64_t orc_param_count(int32_t F, int32_t K, int32_t T, int32_t S) {
  int64_t per = (int64_t)F * F + F + 3 * F * F + 3 * F + 3 * F * K + 3 * F + 2 * F * F +
                2 * F * F + F + 3 * F * F + 3 * F;
  return (int64_t)S * F + T * per + (F / 2) * F + F / 2 + F / 2 + 1;
}

static void bind_params(const orc_model *md, const double *p, orc_params *P) {
  int F = md->F, K = md->K;
  P->emb = p; p += md->S * F;
  for (int t = 0; t < md->T; ++t) {
    orc_layer *L = &P->L[t];
    L->W1 = p; p += F * F;  L->b1 = p; p += F;
    L->W2 = p; p += 3 * F * F; L->b2 = p; p += 3 * F;
    L->Wf = p; p += 3 * F * K; L->bf = p; p += 3 * F;
    L->U = p; p += F * F;   L->V = p; p += F * F;
    L->A1 = p; p += 2 * F * F; L->c1 = p; p += F;
    L->A2 = p; p += 3 * F * F; L->c2 = p; p += 3 * F;
  }
  P->R1 = p; p += (F / 2) * F; P->d1 = p; p += F / 2; P->R2 = p; p += F / 2; P->d2 = p;
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }
static double silu(double x) { return x * sigmoid(x); }
static double dsilu(double x) { double s = sigmoid(x); return s * (1.0 + x * (1.0 - s)); }

/* y[o] = sum_i W[o][i] x[i] (+ b[o]) */
static void matvec(const double *W, const double *b, const double *x, int nout, int nin, double *y) {
  for (int o = 0; o < nout; ++o) {
    double acc = b ? b[o] : 0.0;
    for (int i = 0; i < nin; ++i) acc += W[(int64_t)o * nin + i] * x[i];
    y[o] = acc;
  }
}
/* y[i] += sum_o W[o][i] g[o]   (transpose product, for the backward pass) */
static void matvec_T_add(const double *W, const double *g, int nout, int nin, double *y) {
  for (int o = 0; o < nout; ++o)
    for (int i = 0; i < nin; ++i) y[i] += W[(int64_t)o * nin + i] * g[o];
}

/* Edge geometry and radial filter for one edge: r, d, u, rbf[K], f_c, wt = Wf rbf + bf (3F). */
typedef struct { double r[3], d, u[3], fc, dfc; } edge_geom;

static int edge_geometry(const double *x, const double H[9], int32_t i, int32_t j, const int8_t *n,
                         double rc, edge_geom *g) {
  for (int c = 0; c < 3; ++c)
    g->r[c] = x[3 * j + c] - x[3 * i + c] + (n[0] * H[c] + n[1] * H[3 + c] + n[2] * H[6 + c]);
  g->d = sqrt(g->r[0] * g->r[0] + g->r[1] * g->r[1] + g->r[2] * g->r[2]);
  if (!(g->d < rc)) return 0;                 /* f_c = 0 beyond the cutoff: no contribution */
  for (int c = 0; c < 3; ++c) g->u[c] = g->r[c] / g->d;
  g->fc = 0.5 * (cos(M_PI * g->d / rc) + 1.0);
  g->dfc = -0.5 * (M_PI / rc) * sin(M_PI * g->d / rc);
  return 1;
}

static void radial(const orc_model *md, const orc_layer *L, double d, double fc, double *rb,
                   double *wt, double *W) {
  int K = md->K, F3 = 3 * md->F;
  double sig = md->rc / (K - 1);
  for (int k = 0; k < K; ++k) {
    double mu = k * md->rc / (K - 1);
    rb[k] = exp(-(d - mu) * (d - mu) / (2.0 * sig * sig));
  }
  matvec(L->Wf, L->bf, rb, F3, K, wt);
  for (int c = 0; c < F3; ++c) W[c] = wt[c] * fc;
}

/* Energy, per-atom energies, forces and virial for the pair list (i <- j, n).  The list may
 * contain edges longer than rc (a Verlet list); they contribute nothing.
 * w[n] (may be NULL = all ones): per-atom weights of the energy, E = sum_i w_i U_i, and the
 * forces and virial are those of that weighted sum.  With w = 1 on the atoms a processor owns
 * and 0 on its copied atoms this is one processor's share of the spatial decomposition (Results,
 * "Distributed potential computation": the total energy is the sum of the owned atoms' U_i, the
 * total force on an atom the sum of its copies' partial forces).
 * E: scalar; Ei[n] (unweighted U_i, may be NULL); Fo[n][3] (may be NULL); Wv[9] row-major
 * (may be NULL). */
int orc_painn(const orc_model *md, const double *params, int64_t n, const int32_t *Z,
              const double *x, const double H[9], int64_t ne, const int32_t *pi, const int32_t *pj,
              const int8_t *pn, const double *w, double *E, double *Ei, double *Fo, double *Wv) {
  const int F = md->F, K = md->K, T = md->T, F3 = 3 * F, Fh = F / 2;
  if (T < 0 || T > ORC_MAXT || F < 2 || F > 512 || (F % 2) || K < 2 || K > 256) return ORC_EINVAL;
  orc_params P;
  bind_params(md, params, &P);
  int64_t nF = n * F;
  /* stored activations per layer */
  double *s_in = calloc((size_t)(T + 1) * nF, sizeof(double));      /* s at the start of layer t; s_in[T] = final s */
  double *v_in = calloc((size_t)(T + 1) * 3 * nF, sizeof(double));  /* v at the start of layer t, [n][3][F] */
  double *h1 = calloc((size_t)T * nF, sizeof(double));
  double *phi = calloc((size_t)T * 3 * nF, sizeof(double));
  double *sm = calloc((size_t)T * nF, sizeof(double));
  double *vm = calloc((size_t)T * 3 * nF, sizeof(double));
  double *h2 = calloc((size_t)T * nF, sizeof(double));
  double *h3 = calloc((size_t)n * Fh, sizeof(double));
  double *tmp = calloc((size_t)(8 * F + 2 * K + 8), sizeof(double));
  if (!s_in || !v_in || !h1 || !phi || !sm || !vm || !h2 || !h3 || !tmp) {
    free(s_in); free(v_in); free(h1); free(phi); free(sm); free(vm); free(h2); free(h3); free(tmp);
    return ORC_ENOMEM;
  }
  double *rb = tmp, *wt = rb + K, *W = wt + F3;

  /* embedding: s^0_i = emb[Z_i], v^0 = 0 (Methods "Graph Neural Networks": h^0 = f_h(Z)) */
  for (int64_t i = 0; i < n; ++i)
    for (int f = 0; f < F; ++f) s_in[i * F + f] = P.emb[(int64_t)Z[i] * F + f];

  for (int t = 0; t < T; ++t) {
    const orc_layer *L = &P.L[t];
    double *s = s_in + t * nF, *v = v_in + t * 3 * nF;
    double *H1 = h1 + t * nF, *PH = phi + t * 3 * nF, *SM = sm + t * nF, *VM = vm + t * 3 * nF;
    double *H2 = h2 + t * nF;
    /* message function phi_j on every atom */
    for (int64_t j = 0; j < n; ++j) {
      double a1[1024];
      matvec(L->W1, L->b1, &s[j * F], F, F, &H1[j * F]);
      for (int f = 0; f < F; ++f) a1[f] = silu(H1[j * F + f]);
      matvec(L->W2, L->b2, a1, F3, F, &PH[j * F3]);
    }
    /* residual: s^m = s + sum_e ..., v^m = v + sum_e ... (synchronous: uses v before block) */
    memcpy(SM, s, sizeof(double) * nF);
    memcpy(VM, v, sizeof(double) * 3 * nF);
    for (int64_t e = 0; e < ne; ++e) {
      edge_geom g;
      int32_t i = pi[e], j = pj[e];
      if (!edge_geometry(x, H, i, j, &pn[3 * e], md->rc, &g)) continue;
      radial(md, L, g.d, g.fc, rb, wt, W);
      const double *ph = &PH[(int64_t)j * F3];
      for (int f = 0; f < F; ++f) SM[i * F + f] += ph[f] * W[f];
      for (int a = 0; a < 3; ++a)
        for (int f = 0; f < F; ++f)
          VM[(i * 3 + a) * F + f] += v[(j * 3 + a) * F + f] * ph[F + f] * W[F + f] +
                                     g.u[a] * ph[2 * F + f] * W[2 * F + f];
    }
    /* update function */
    double *sn = s_in + (t + 1) * nF, *vn = v_in + (t + 1) * 3 * nF;
    for (int64_t i = 0; i < n; ++i) {
      double Uv[3][512], Vv[3][512], z[1024], a2[512], av[1536], nV[512];
      for (int a = 0; a < 3; ++a) {
        matvec(L->U, NULL, &VM[(i * 3 + a) * F], F, F, Uv[a]);
        matvec(L->V, NULL, &VM[(i * 3 + a) * F], F, F, Vv[a]);
      }
      for (int f = 0; f < F; ++f) {
        nV[f] = sqrt(Vv[0][f] * Vv[0][f] + Vv[1][f] * Vv[1][f] + Vv[2][f] * Vv[2][f] + md->eps);
        z[f] = SM[i * F + f];
        z[F + f] = nV[f];
      }
      matvec(L->A1, L->c1, z, F, 2 * F, &H2[i * F]);
      for (int f = 0; f < F; ++f) a2[f] = silu(H2[i * F + f]);
      matvec(L->A2, L->c2, a2, F3, F, av);
      for (int f = 0; f < F; ++f) {
        double sp = Uv[0][f] * Vv[0][f] + Uv[1][f] * Vv[1][f] + Uv[2][f] * Vv[2][f];
        sn[i * F + f] = SM[i * F + f] + av[2 * F + f] + av[F + f] * sp;
        for (int a = 0; a < 3; ++a)
          vn[(i * 3 + a) * F + f] = VM[(i * 3 + a) * F + f] + av[f] * Uv[a][f];
      }
    }
  }

  /* readout: U_i = e_scale (R2 . silu(R1 s_i + d1) + d2), U = sum_i w_i U_i */
  double *sT = s_in + (int64_t)T * nF;
  double Etot = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    matvec(P.R1, P.d1, &sT[i * F], Fh, F, &h3[i * Fh]);
    double ei = P.d2[0];
    for (int k = 0; k < Fh; ++k) ei += P.R2[k] * silu(h3[i * Fh + k]);
    ei *= md->e_scale;
    if (Ei) Ei[i] = ei;
    Etot += w ? w[i] * ei : ei;
  }
  *E = Etot;

  if (Fo || Wv) {
    double *gs = calloc((size_t)nF, sizeof(double)), *gv = calloc((size_t)3 * nF, sizeof(double));
    double *gsm = calloc((size_t)nF, sizeof(double)), *gvm = calloc((size_t)3 * nF, sizeof(double));
    double *gph = calloc((size_t)3 * nF, sizeof(double));
    double Wacc[9] = {0};
    if (Fo) memset(Fo, 0, sizeof(double) * 3 * n);
    /* dU/ds^T, seeded with dU/dU_i = w_i */
    for (int64_t i = 0; i < n; ++i) {
      double g3[512];
      const double wi = w ? w[i] : 1.0;
      for (int k = 0; k < Fh; ++k) g3[k] = wi * md->e_scale * P.R2[k] * dsilu(h3[i * Fh + k]);
      matvec_T_add(P.R1, g3, Fh, F, &gs[i * F]);
    }
    for (int t = T - 1; t >= 0; --t) {
      const orc_layer *L = &P.L[t];
      double *s = s_in + t * nF, *v = v_in + t * 3 * nF;
      double *H1 = h1 + t * nF, *PH = phi + t * 3 * nF, *SM = sm + t * nF, *VM = vm + t * 3 * nF;
      double *H2 = h2 + t * nF;
      (void)s;
      /* update backward: (gs, gv) w.r.t. layer output -> (gsm, gvm) w.r.t. s^m, v^m */
      for (int64_t i = 0; i < n; ++i) {
        double Uv[3][512], Vv[3][512], a2[512], av[1536], nV[512];
        double gUv[3][512], gVv[3][512], ga[1536], ga2[512], gz[1024];
        for (int a = 0; a < 3; ++a) {
          matvec(L->U, NULL, &VM[(i * 3 + a) * F], F, F, Uv[a]);
          matvec(L->V, NULL, &VM[(i * 3 + a) * F], F, F, Vv[a]);
        }
        for (int f = 0; f < F; ++f)
          nV[f] = sqrt(Vv[0][f] * Vv[0][f] + Vv[1][f] * Vv[1][f] + Vv[2][f] * Vv[2][f] + md->eps);
        for (int f = 0; f < F; ++f) a2[f] = silu(H2[i * F + f]);
        matvec(L->A2, L->c2, a2, F3, F, av);
        for (int f = 0; f < F; ++f) {
          double gsf = gs[i * F + f];
          double sp = Uv[0][f] * Vv[0][f] + Uv[1][f] * Vv[1][f] + Uv[2][f] * Vv[2][f];
          double gsp = gsf * av[F + f];
          ga[2 * F + f] = gsf;          /* a_ss */
          ga[F + f] = gsf * sp;         /* a_sv */
          double gavv = 0.0;
          for (int a = 0; a < 3; ++a) {
            double gvf = gv[(i * 3 + a) * F + f];
            gavv += gvf * Uv[a][f];
            gUv[a][f] = gvf * av[f] + gsp * Vv[a][f];
            gVv[a][f] = gsp * Uv[a][f];
          }
          ga[f] = gavv;                 /* a_vv */
        }
        for (int k = 0; k < F; ++k) ga2[k] = 0.0;
        matvec_T_add(L->A2, ga, F3, F, ga2);
        for (int k = 0; k < F; ++k) ga2[k] *= dsilu(H2[i * F + k]);
        for (int k = 0; k < 2 * F; ++k) gz[k] = 0.0;
        matvec_T_add(L->A1, ga2, F, 2 * F, gz);
        for (int f = 0; f < F; ++f) {
          gsm[i * F + f] = gs[i * F + f] + gz[f];
          for (int a = 0; a < 3; ++a) gVv[a][f] += gz[F + f] * Vv[a][f] / nV[f];
        }
        for (int a = 0; a < 3; ++a) {
          double *g = &gvm[(i * 3 + a) * F];
          for (int f = 0; f < F; ++f) g[f] = gv[(i * 3 + a) * F + f];
          matvec_T_add(L->U, gUv[a], F, F, g);
          matvec_T_add(L->V, gVv[a], F, F, g);
        }
      }
      /* message backward: residual passes gsm, gvm straight through */
      memcpy(gs, gsm, sizeof(double) * nF);
      memcpy(gv, gvm, sizeof(double) * 3 * nF);
      memset(gph, 0, sizeof(double) * 3 * nF);
      for (int64_t e = 0; e < ne; ++e) {
        edge_geom g;
        int32_t i = pi[e], j = pj[e];
        if (!edge_geometry(x, H, i, j, &pn[3 * e], md->rc, &g)) continue;
        radial(md, L, g.d, g.fc, rb, wt, W);
        const double *ph = &PH[(int64_t)j * F3];
        double *gp = &gph[(int64_t)j * F3];
        double gW[1536], gu[3] = {0, 0, 0};
        for (int f = 0; f < F; ++f) {
          double gsf = gsm[i * F + f];
          gW[f] = gsf * ph[f];
          gp[f] += gsf * W[f];
          double gWvv = 0.0, gWvs = 0.0, gpvv = 0.0, gpvs = 0.0;
          for (int a = 0; a < 3; ++a) {
            double gvf = gvm[(i * 3 + a) * F + f];
            double vj = v[(j * 3 + a) * F + f];
            gWvv += gvf * vj * ph[F + f];
            gpvv += gvf * vj * W[F + f];
            gv[(j * 3 + a) * F + f] += gvf * ph[F + f] * W[F + f];
            gWvs += gvf * g.u[a] * ph[2 * F + f];
            gpvs += gvf * g.u[a] * W[2 * F + f];
            gu[a] += gvf * ph[2 * F + f] * W[2 * F + f];
          }
          gW[F + f] = gWvv;
          gW[2 * F + f] = gWvs;
          gp[F + f] += gpvv;
          gp[2 * F + f] += gpvs;
        }
        /* W = wt * fc, wt = Wf rbf + bf */
        double gfc = 0.0, grb[256];
        for (int k = 0; k < K; ++k) grb[k] = 0.0;
        for (int c = 0; c < F3; ++c) {
          gfc += gW[c] * wt[c];
          double gwt = gW[c] * g.fc;
          for (int k = 0; k < K; ++k) grb[k] += L->Wf[(int64_t)c * K + k] * gwt;
        }
        double sig = md->rc / (K - 1), gd = gfc * g.dfc;
        for (int k = 0; k < K; ++k) {
          double mu = k * md->rc / (K - 1);
          gd += grb[k] * rb[k] * (-(g.d - mu) / (sig * sig));
        }
        /* r -> (d, u):  dU/dr = gd u + (gu - (gu.u) u) / d */
        double gudotu = gu[0] * g.u[0] + gu[1] * g.u[1] + gu[2] * g.u[2];
        double gr[3];
        for (int c = 0; c < 3; ++c) gr[c] = gd * g.u[c] + (gu[c] - gudotu * g.u[c]) / g.d;
        /* r_e = x_j - x_i + shift:  f_i += dU/dr, f_j -= dU/dr;  W -= r (x) dU/dr */
        if (Fo)
          for (int c = 0; c < 3; ++c) { Fo[3 * i + c] += gr[c]; Fo[3 * j + c] -= gr[c]; }
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) Wacc[3 * a + b] -= g.r[a] * gr[b];
      }
      /* phi_j backward: phi = W2 silu(W1 s + b1) + b2 */
      for (int64_t j = 0; j < n; ++j) {
        double ga1[512];
        for (int k = 0; k < F; ++k) ga1[k] = 0.0;
        matvec_T_add(L->W2, &gph[j * F3], F3, F, ga1);
        for (int k = 0; k < F; ++k) ga1[k] *= dsilu(H1[j * F + k]);
        matvec_T_add(L->W1, ga1, F, F, &gs[j * F]);
      }
    }
    if (Wv) memcpy(Wv, Wacc, sizeof(Wacc));
    free(gs); free(gv); free(gsm); free(gvm); free(gph);
  }
  free(s_in); free(v_in); free(h1); free(phi); free(sm); free(vm); free(h2); free(h3); free(tmp);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------
 * NVE velocity Verlet (the MD loop that consumes the forces; Results "Distributed potential
 * computation": forces drive every MD step).  Units: A, fs, amu, eV.  The pair list is
 * rebuilt from scratch every step (no skin) with the linked-cell search above.
 * x, vel: [n][3], updated in place.  epot/ekin: [nsteps+1] energies along the trajectory.
 * ---------------------------------------------------------------------------------------- */
#define ORC_ACC 9.648533212331002e-3   /* (eV / A) / amu in A / fs^2 */

static int forces_at(const orc_model *md, const double *params, int64_t n, const int32_t *Z,
                     const double *x, const double H[9], double *E, double *Fo) {
  double *xw = malloc(sizeof(double) * 3 * n);
  int32_t *m = malloc(sizeof(int32_t) * 3 * n);
  if (!xw || !m) { free(xw); free(m); return ORC_ENOMEM; }
  orc_wrap(n, x, H, xw, m);
  int64_t np = orc_pairs_cells(n, xw, H, md->rc, NULL, NULL, NULL, 0);
  int32_t *pi = malloc(sizeof(int32_t) * (np + 1)), *pj = malloc(sizeof(int32_t) * (np + 1));
  int8_t *pn = malloc(3 * (np + 1));
  if (!pi || !pj || !pn) { free(xw); free(m); free(pi); free(pj); free(pn); return ORC_ENOMEM; }
  orc_pairs_cells(n, xw, H, md->rc, pi, pj, pn, np);
  int rc = orc_painn(md, params, n, Z, xw, H, np, pi, pj, pn, NULL, E, NULL, Fo, NULL);
  free(xw); free(m); free(pi); free(pj); free(pn);
  return rc;
}

int orc_nve(const orc_model *md, const double *params, int64_t n, const int32_t *Z,
            const double *mass, const double H[9], double *x, double *vel, double dt, int32_t nsteps,
            double *epot, double *ekin) {
  double *Fo = malloc(sizeof(double) * 3 * n);
  if (!Fo) return ORC_ENOMEM;
  double E;
  int rc = forces_at(md, params, n, Z, x, H, &E, Fo);
  for (int32_t step = 0; step <= nsteps && rc == ORC_OK; ++step) {
    double ke = 0.0;
    for (int64_t i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c) ke += 0.5 * mass[i] * vel[3 * i + c] * vel[3 * i + c];
    if (epot) epot[step] = E;
    if (ekin) ekin[step] = ke / ORC_ACC;   /* amu A^2/fs^2 -> eV */
    if (step == nsteps) break;
    for (int64_t i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c) {
        vel[3 * i + c] += 0.5 * dt * ORC_ACC * Fo[3 * i + c] / mass[i];
        x[3 * i + c] += dt * vel[3 * i + c];
      }
    rc = forces_at(md, params, n, Z, x, H, &E, Fo);
    for (int64_t i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c) vel[3 * i + c] += 0.5 * dt * ORC_ACC * Fo[3 * i + c] / mass[i];
  }
  free(Fo);
  return rc;
}

/* ------------------------------------------------------------------------------------------
 * NVT with a Nose-Hoover chain thermostat (Methods, "MD simulations": NVT ensemble, Nose-Hoover
 * thermostat with a temperature damping parameter tau).  The paper names neither the chain
 * length nor the integrator; this follows the Martyna-Tuckerman-Klein (1996) equations of a
 * chain of M thermostats,
 *   dv_i/dt   = F_i/m_i - vxi_1 v_i
 *   dvxi_1/dt = (2 K - Nf kT)/Q_1 - vxi_2 vxi_1
 *   dvxi_j/dt = (Q_{j-1} vxi_{j-1}^2 - kT)/Q_j - vxi_{j+1} vxi_j      (vxi_{M+1} = 0)
 *   dxi_j/dt  = vxi_j
 * with Q_1 = Nf kT tau^2, Q_j = kT tau^2, Nf = 3n - 3 (centre of mass at rest), integrated by
 * the symmetric Trotter splitting: a chain half step over dt/2, velocity Verlet, a chain half
 * step.  The chain half step of length h updates vxi_M, then vxi_{M-1} .. vxi_1 (each between two
 * factors exp(-h vxi_{j+1}/4)), scales the velocities by exp(-h vxi_1), advances every xi_j by
 * h vxi_j, and sweeps the chain back up in the mirrored order.  Conserved quantity:
 *   H = K + U + sum_j Q_j vxi_j^2 / 2 + Nf kT xi_1 + kT sum_{j>1} xi_j.
 * ---------------------------------------------------------------------------------------- */
#define ORC_KB 8.617333262e-5   /* eV / K */

static double chain_force(int j, double KE, double Nf, double kT, const double *Q, const double *vxi) {
  if (j == 0) return (2.0 * KE - Nf * kT) / Q[0];
  return (Q[j - 1] * vxi[j - 1] * vxi[j - 1] - kT) / Q[j];
}

/* One chain half step of length h; returns the factor that scales every velocity. */
static double chain_half(int M, double h, double KE, double Nf, double kT, const double *Q, double *xi,
                         double *vxi) {
  vxi[M - 1] += 0.5 * h * chain_force(M - 1, KE, Nf, kT, Q, vxi);
  for (int j = M - 2; j >= 0; --j) {
    double e = exp(-0.25 * h * vxi[j + 1]);
    vxi[j] *= e;
    vxi[j] += 0.5 * h * chain_force(j, KE, Nf, kT, Q, vxi);
    vxi[j] *= e;
  }
  double scale = exp(-h * vxi[0]);
  KE *= scale * scale;
  for (int j = 0; j < M; ++j) xi[j] += h * vxi[j];
  for (int j = 0; j < M - 1; ++j) {
    double e = exp(-0.25 * h * vxi[j + 1]);
    vxi[j] *= e;
    vxi[j] += 0.5 * h * chain_force(j, KE, Nf, kT, Q, vxi);
    vxi[j] *= e;
  }
  vxi[M - 1] += 0.5 * h * chain_force(M - 1, KE, Nf, kT, Q, vxi);
  return scale;
}

static double kinetic(int64_t n, const double *mass, const double *vel) {
  double ke = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < 3; ++c) ke += 0.5 * mass[i] * vel[3 * i + c] * vel[3 * i + c];
  return ke / ORC_ACC;
}

static double chain_energy(int M, double Nf, double kT, const double *Q, const double *xi, const double *vxi) {
  double e = 0.0;
  for (int j = 0; j < M; ++j) e += 0.5 * Q[j] * vxi[j] * vxi[j] + (j == 0 ? Nf * kT : kT) * xi[j];
  return e;
}

/* temperature (K), tau (fs), chain length M (1..16).  xi, vxi: [M] chain state, updated in place
 * (start from zeros for a fresh chain).  epot / ekin / eth: [nsteps+1] (eth = chain energy). */
int orc_nvt(const orc_model *md, const double *params, int64_t n, const int32_t *Z, const double *mass,
            const double H[9], double *x, double *vel, double dt, int32_t nsteps, double temperature,
            double tau, int32_t M, double *xi, double *vxi, double *epot, double *ekin, double *eth) {
  if (M < 1 || M > 16 || n < 2 || !(tau > 0.0) || !(temperature > 0.0)) return ORC_EINVAL;
  const double kT = ORC_KB * temperature, Nf = 3.0 * (double)n - 3.0;
  double Q[16];
  for (int j = 0; j < M; ++j) Q[j] = (j == 0 ? Nf : 1.0) * kT * tau * tau;
  double *Fo = malloc(sizeof(double) * 3 * n);
  if (!Fo) return ORC_ENOMEM;
  double E;
  int rc = forces_at(md, params, n, Z, x, H, &E, Fo);
  for (int32_t step = 0; step <= nsteps && rc == ORC_OK; ++step) {
    if (epot) epot[step] = E;
    if (ekin) ekin[step] = kinetic(n, mass, vel);
    if (eth) eth[step] = chain_energy(M, Nf, kT, Q, xi, vxi);
    if (step == nsteps) break;
    double s = chain_half(M, 0.5 * dt, kinetic(n, mass, vel), Nf, kT, Q, xi, vxi);
    for (int64_t i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c) {
        vel[3 * i + c] = s * vel[3 * i + c] + 0.5 * dt * ORC_ACC * Fo[3 * i + c] / mass[i];
        x[3 * i + c] += dt * vel[3 * i + c];
      }
    rc = forces_at(md, params, n, Z, x, H, &E, Fo);
    for (int64_t i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c) vel[3 * i + c] += 0.5 * dt * ORC_ACC * Fo[3 * i + c] / mass[i];
    s = chain_half(M, 0.5 * dt, kinetic(n, mass, vel), Nf, kT, Q, xi, vxi);
    for (int64_t i = 0; i < 3 * n; ++i) vel[i] *= s;
  }
  free(Fo);
  return rc;
}

