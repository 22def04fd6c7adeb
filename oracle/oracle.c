/*
 * HODLR2D CPU oracle (FP64, single thread).  TEST INFRASTRUCTURE ONLY: only
 * the tests, the smoke check and the benchmark's CPU legs may load it.  It
 * shares no code with the CUDA library.
 *
 * Every routine follows one passage of "HODLR2D: A new class of hierarchical
 * matrices" (arXiv 2204.05536) and favours obviousness over speed:
 *   orc_entry            - kernel entries: Sec. 3, Eq. 1byr, Eq. ker (phi_1, phi_2)
 *   orc_direct_*         - the explicit product K psi of Sec. 5.1
 *   build_tree           - Sec. 4 quadtree, Fig. sdomain01 numbering, Alg. 1
 *   build_lists          - Defs. ec / vc / wc / cc / ic, Eq. ilist
 *   orc_aca              - ACA (Alg. 1, compression step)
 *   orc_matvec           - Alg. 2
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - the square root box is the bounding square of the points (centred on
 *     the bounding box) unless the caller gives one;
 *   - a point maps to box floor((x - x0)/w * 2^l), clamped to [0, 2^l - 1];
 *   - kappa is the smallest depth whose leaves all hold <= N_max points;
 *   - within a box, points are ordered by ascending original index;
 *   - ACA is the partially pivoted variant: first row = the box's first
 *     point, column pivot = argmax |residual row| (first on ties), next row =
 *     argmax |residual column| over unused rows (first on ties), stop when
 *     |u| |v| <= eps |S_k|_F or the rank reaches min(m, n);
 *   - the kernels are radial, so A(Y,X) = A(X,Y)^T: each unordered pair is
 *     compressed once, rows = the box with the smaller Morton key, and the
 *     pair (Y,X) is applied as V U^T;
 *   - Alg. 2 loops i = 1..4^kappa at every level; read as 4^l.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Kernel entries                                                            */
/* ------------------------------------------------------------------------ */

/* phi as a function of the squared distance r2 (r2 > 0 off the diagonal). */
static double phi_r2(const orc_kernel* k, double r2) {
  const double a = k->a;
  double r;
  switch (k->kind) {
    case ORC_IMQ: /* inverse multiquadric */
      return 1.0 / sqrt(r2 + a * a);
    case ORC_MQ: /* multiquadric */
      return sqrt(r2 + a * a);
    case ORC_LOG: /* log |r_i - r_j|, Sec. 3 */
      return 0.5 * log(r2);
    case ORC_INV_R: /* 1 / r_ij, Eq. 1byr */
      return 1.0 / sqrt(r2);
    case ORC_PHI1: /* phi_1, Sec. 5.2 */
      r = sqrt(r2);
      if (r >= a) return log(r) / log(a);
      return (r * log(r) - 1.0) / (a * log(a) - 1.0);
    case ORC_PHI2: /* phi_2, Sec. 5.2 */
      r = sqrt(r2);
      if (r >= a) return a / r;
      return r / a;
  }
  return NAN;
}

/* The diagonal.  diag_mode 1: a constant (beta of Eq. ker, or a panel
 * self-term).  diag_mode 0: phi(0) where it is finite (IMQ 1/a, MQ a,
 * phi_1 -1/(a log a - 1) with r log r -> 0, phi_2 0), and 0 for the singular
 * kernels, as Sec. 3 and Eq. 1byr set it. */
static double diag_entry(const orc_kernel* k) {
  if (k->diag_mode == 1) return k->diag_value;
  switch (k->kind) {
    case ORC_IMQ: return 1.0 / k->a;
    case ORC_MQ: return k->a;
    case ORC_PHI1: return -1.0 / (k->a * log(k->a) - 1.0);
    default: return 0.0;
  }
}

double orc_entry(const orc_kernel* k, const double* pts, int64_t i, int64_t j) {
  if (i == j) return diag_entry(k);
  const double dx = pts[2 * i] - pts[2 * j];
  const double dy = pts[2 * i + 1] - pts[2 * j + 1];
  return phi_r2(k, dx * dx + dy * dy);
}

/* ------------------------------------------------------------------------ */
/* Direct product (Sec. 5.1: b = K psi by explicit matrix-vector product)    */
/* ------------------------------------------------------------------------ */

void orc_direct_rows(int64_t n, const double* pts, const orc_kernel* k,
                     const double* x, int nrhs, int64_t nrows,
                     const int64_t* rows, double* y) {
  for (int c = 0; c < nrhs; ++c) {
    for (int64_t r = 0; r < nrows; ++r) {
      const int64_t i = rows[r];
      double s = 0.0;
      for (int64_t j = 0; j < n; ++j) s += orc_entry(k, pts, i, j) * x[j + n * c];
      y[r + nrows * c] = s;
    }
  }
}

void orc_direct_matvec(int64_t n, const double* pts, const orc_kernel* k,
                       const double* x, double* y, int nrhs) {
  for (int c = 0; c < nrhs; ++c) {
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t j = 0; j < n; ++j) s += orc_entry(k, pts, i, j) * x[j + n * c];
      y[i + n * c] = s;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Box numbering of Fig. sdomain01: children of box b are 4b + c with        */
/* c = 0 bottom-left, 1 bottom-right, 2 top-right, 3 top-left.              */
/* ------------------------------------------------------------------------ */

int64_t orc_paper_index(int l, int32_t ix, int32_t iy) {
  int64_t b = 0;
  for (int s = l - 1; s >= 0; --s) {
    const int bx = (ix >> s) & 1, by = (iy >> s) & 1;
    int c;
    if (!by && !bx) c = 0;      /* bottom-left  */
    else if (!by && bx) c = 1;  /* bottom-right */
    else if (by && bx) c = 2;   /* top-right    */
    else c = 3;                 /* top-left     */
    b = 4 * b + c;
  }
  return b;
}

void orc_paper_coords(int l, int64_t b, int32_t* ix, int32_t* iy) {
  int32_t x = 0, y = 0;
  for (int s = 0; s < l; ++s) {
    const int c = (int)((b >> (2 * s)) & 3);
    const int bx = (c == 1 || c == 2), by = (c == 2 || c == 3);
    x |= bx << s;
    y |= by << s;
  }
  *ix = x;
  *iy = y;
}

/* Morton key (x bits even, y bits odd): fixes which box of a pair is the row
 * side of its single stored factorisation. */
static uint64_t morton(int l, int32_t ix, int32_t iy) {
  uint64_t key = 0;
  for (int s = 0; s < l; ++s) {
    key |= (uint64_t)((ix >> s) & 1) << (2 * s);
    key |= (uint64_t)((iy >> s) & 1) << (2 * s + 1);
  }
  return key;
}

/* ------------------------------------------------------------------------ */
/* The handle                                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
  int level;
  int64_t bx, by; /* paper indices: bx = row box (smaller Morton key) */
  int64_t nx, ny;
  int rank;
  double* U; /* nx x rank, column-major */
  double* V; /* ny x rank, column-major */
} orc_pair;

struct orc_h2d {
  int64_t n;
  double* pts;
  orc_kernel k;
  int kappa;
  double x0, y0, w;
  double eps;
  int64_t** off; /* off[l][b]: start of box b in idx[l]; size 4^l + 1 */
  int64_t** idx; /* idx[l]: point indices grouped by box, ascending inside */
  int64_t** e_off;
  int64_t** e_lst; /* edge sharers (non-empty boxes), Def. ec */
  int64_t** i_off;
  int64_t** i_lst;  /* interaction list, Eq. ilist */
  int64_t** i_pair; /* stored pair serving (b, i_lst entry) */
  int64_t npairs, cap_pairs;
  orc_pair* pairs;
};

static int64_t nboxes(int l) { return (int64_t)1 << (2 * l); }

static int64_t box_count(const orc_h2d* h, int l, int64_t b) {
  return h->off[l][b + 1] - h->off[l][b];
}

/* ------------------------------------------------------------------------ */
/* Tree (Sec. 4, Alg. 1): uniform subdivision of the square B; kappa is the  */
/* smallest depth at which every leaf holds at most N_max points.           */
/* ------------------------------------------------------------------------ */

static int32_t cell_of(double v, double v0, double w, int l) {
  const double m = (double)((int64_t)1 << l);
  const double f = floor((v - v0) / w * m);
  if (f < 0.0) return 0;
  if (f > m - 1.0) return (int32_t)(m - 1.0);
  return (int32_t)f;
}

static int build_tree(orc_h2d* h, int leaf_size, int levels) {
  const int64_t n = h->n;
  const int max_levels = 14;
  int kappa;
  if (levels >= 0) {
    kappa = levels;
  } else {
    int64_t* cnt = NULL;
    for (kappa = 0; kappa <= max_levels; ++kappa) {
      const int64_t nb = nboxes(kappa);
      cnt = (int64_t*)calloc((size_t)nb, sizeof(int64_t));
      if (!cnt) return -2;
      int64_t mx = 0;
      for (int64_t i = 0; i < n; ++i) {
        const int32_t ix = cell_of(h->pts[2 * i], h->x0, h->w, kappa);
        const int32_t iy = cell_of(h->pts[2 * i + 1], h->y0, h->w, kappa);
        const int64_t b = orc_paper_index(kappa, ix, iy);
        if (++cnt[b] > mx) mx = cnt[b];
      }
      free(cnt);
      if (mx <= leaf_size) break;
    }
    if (kappa > max_levels) return -3;
  }
  h->kappa = kappa;
  h->off = (int64_t**)calloc((size_t)kappa + 1, sizeof(int64_t*));
  h->idx = (int64_t**)calloc((size_t)kappa + 1, sizeof(int64_t*));
  if (!h->off || !h->idx) return -2;
  int64_t* box = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  if (!box) return -2;
  for (int l = 0; l <= kappa; ++l) {
    const int64_t nb = nboxes(l);
    h->off[l] = (int64_t*)calloc((size_t)nb + 1, sizeof(int64_t));
    h->idx[l] = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    if (!h->off[l] || !h->idx[l]) { free(box); return -2; }
    for (int64_t i = 0; i < n; ++i) {
      const int32_t ix = cell_of(h->pts[2 * i], h->x0, h->w, l);
      const int32_t iy = cell_of(h->pts[2 * i + 1], h->y0, h->w, l);
      box[i] = orc_paper_index(l, ix, iy);
      h->off[l][box[i] + 1] += 1;
    }
    for (int64_t b = 0; b < nb; ++b) h->off[l][b + 1] += h->off[l][b];
    /* counting sort in ascending point order: each box keeps its points in
     * ascending original index */
    int64_t* fill = (int64_t*)malloc((size_t)nb * sizeof(int64_t));
    if (!fill) { free(box); return -2; }
    memcpy(fill, h->off[l], (size_t)nb * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) h->idx[l][fill[box[i]]++] = i;
    free(fill);
  }
  free(box);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Lists (Defs. ec, vc, wc, cc, ic; Eq. ilist)                               */
/* ------------------------------------------------------------------------ */

enum { REL_SELF = 0, REL_EDGE = 1, REL_VERTEX = 2, REL_FAR = 3 };

/* Relation of two same-level boxes [ax,ax+1]x[ay,ay+1] and [bx,bx+1]x[by,by+1]
 * from their closed intersection: a square (same box), a segment (they share
 * an edge, Def. ec), a point (they share a vertex only, Def. vc) or empty
 * (well separated, Def. wc). */
static int relation(int32_t ax, int32_t ay, int32_t bx, int32_t by) {
  const int32_t lox = ax > bx ? ax : bx, hix = (ax < bx ? ax : bx) + 1;
  const int32_t loy = ay > by ? ay : by, hiy = (ay < by ? ay : by) + 1;
  if (lox > hix || loy > hiy) return REL_FAR;
  const int32_t lenx = hix - lox, leny = hiy - loy;
  if (lenx > 0 && leny > 0) return REL_SELF;
  if (lenx > 0 || leny > 0) return REL_EDGE;
  return REL_VERTEX;
}

static int in_grid(int l, int32_t ix, int32_t iy) {
  const int32_t m = (int32_t)1 << l;
  return ix >= 0 && iy >= 0 && ix < m && iy < m;
}

/* Clan set of box (cx, cy) at level l >= 1 (Def. cc): the siblings of the
 * box and the children of every edge sharer of its parent.  Written as grid
 * coordinates; returns the count. */
static int clan_set(int l, int32_t cx, int32_t cy, int32_t* ox, int32_t* oy) {
  int c = 0;
  const int32_t px = cx >> 1, py = cy >> 1;
  for (int ch = 0; ch < 4; ++ch) { /* siblings */
    const int32_t sx = 2 * px + (ch & 1), sy = 2 * py + (ch >> 1);
    if (sx == cx && sy == cy) continue;
    ox[c] = sx; oy[c] = sy; ++c;
  }
  static const int dxs[4] = {1, -1, 0, 0}, dys[4] = {0, 0, 1, -1};
  for (int e = 0; e < 4; ++e) { /* children of E_parent(C) */
    const int32_t qx = px + dxs[e], qy = py + dys[e];
    if (!in_grid(l - 1, qx, qy)) continue;
    for (int ch = 0; ch < 4; ++ch) {
      ox[c] = 2 * qx + (ch & 1); oy[c] = 2 * qy + (ch >> 1); ++c;
    }
  }
  return c;
}

static int cmp_i64(const void* a, const void* b) {
  const int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

static int build_lists(orc_h2d* h) {
  const int kappa = h->kappa;
  h->e_off = (int64_t**)calloc((size_t)kappa + 1, sizeof(int64_t*));
  h->e_lst = (int64_t**)calloc((size_t)kappa + 1, sizeof(int64_t*));
  h->i_off = (int64_t**)calloc((size_t)kappa + 1, sizeof(int64_t*));
  h->i_lst = (int64_t**)calloc((size_t)kappa + 1, sizeof(int64_t*));
  h->i_pair = (int64_t**)calloc((size_t)kappa + 1, sizeof(int64_t*));
  if (!h->e_off || !h->e_lst || !h->i_off || !h->i_lst || !h->i_pair) return -2;
  for (int l = 0; l <= kappa; ++l) {
    const int64_t nb = nboxes(l);
    h->e_off[l] = (int64_t*)calloc((size_t)nb + 1, sizeof(int64_t));
    h->i_off[l] = (int64_t*)calloc((size_t)nb + 1, sizeof(int64_t));
    /* list storage grows with the non-empty boxes (deep trees are sparse) */
    int64_t cap = 64;
    h->e_lst[l] = (int64_t*)malloc((size_t)cap * 4 * sizeof(int64_t));
    h->i_lst[l] = (int64_t*)malloc((size_t)cap * 15 * sizeof(int64_t));
    if (!h->e_off[l] || !h->i_off[l] || !h->e_lst[l] || !h->i_lst[l]) return -2;
    int64_t ne = 0, ni = 0, nonempty = 0;
    for (int64_t b = 0; b < nb; ++b) {
      h->e_off[l][b] = ne;
      h->i_off[l][b] = ni;
      if (box_count(h, l, b) == 0) continue;
      if (++nonempty > cap) {
        cap *= 2;
        int64_t* ne_ = (int64_t*)realloc(h->e_lst[l], (size_t)cap * 4 * sizeof(int64_t));
        if (ne_) h->e_lst[l] = ne_;
        int64_t* ni_ = (int64_t*)realloc(h->i_lst[l], (size_t)cap * 15 * sizeof(int64_t));
        if (ni_) h->i_lst[l] = ni_;
        if (!ne_ || !ni_) return -2;
      }
      int32_t cx, cy;
      orc_paper_coords(l, b, &cx, &cy);
      /* E_C: same-level boxes sharing an edge with C (at most 4) */
      const int64_t e0 = ne;
      static const int dxs[4] = {1, -1, 0, 0}, dys[4] = {0, 0, 1, -1};
      for (int e = 0; e < 4; ++e) {
        const int32_t qx = cx + dxs[e], qy = cy + dys[e];
        if (!in_grid(l, qx, qy)) continue;
        const int64_t q = orc_paper_index(l, qx, qy);
        if (box_count(h, l, q) == 0) continue;
        if (relation(cx, cy, qx, qy) != REL_EDGE) continue;
        h->e_lst[l][ne++] = q;
      }
      qsort(h->e_lst[l] + e0, (size_t)(ne - e0), sizeof(int64_t), cmp_i64);
      if (l == 0) continue;
      /* I_C = (clan ∩ V_C) ∪ (clan ∩ W_C) */
      int32_t ox[19], oy[19];
      const int nc = clan_set(l, cx, cy, ox, oy);
      const int64_t i0 = ni;
      for (int c = 0; c < nc; ++c) {
        const int rel = relation(cx, cy, ox[c], oy[c]);
        if (rel != REL_VERTEX && rel != REL_FAR) continue;
        const int64_t q = orc_paper_index(l, ox[c], oy[c]);
        if (box_count(h, l, q) == 0) continue;
        h->i_lst[l][ni++] = q;
      }
      qsort(h->i_lst[l] + i0, (size_t)(ni - i0), sizeof(int64_t), cmp_i64);
    }
    h->e_off[l][nb] = ne;
    h->i_off[l][nb] = ni;
    h->i_pair[l] = (int64_t*)malloc((size_t)(ni + 1) * sizeof(int64_t));
    if (!h->i_pair[l]) return -2;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* ACA: partially pivoted adaptive cross approximation of A(I, J).           */
/* Rank-one terms u v^T with u the residual column and v the residual row    */
/* divided by its pivot; |S_k|_F^2 updated from the new term and its inner   */
/* products with the earlier ones.                                          */
/* ------------------------------------------------------------------------ */

int orc_aca(const orc_kernel* k, const double* pts, int64_t m, const int64_t* I,
            int64_t n, const int64_t* J, double eps, double* U, double* V) {
  const int64_t kmax = m < n ? m : n;
  char* used = (char*)calloc((size_t)m, 1);
  double* r = (double*)malloc((size_t)n * sizeof(double));
  if (!used || !r) { free(used); free(r); return -2; }
  int64_t rank = 0, nused = 0, i = 0;
  double S2 = 0.0;
  while (rank < kmax && nused < m) {
    /* residual row i */
    for (int64_t j = 0; j < n; ++j) {
      double s = orc_entry(k, pts, I[i], J[j]);
      for (int64_t q = 0; q < rank; ++q) s -= U[i + m * q] * V[j + n * q];
      r[j] = s;
    }
    used[i] = 1;
    ++nused;
    int64_t jp = 0;
    for (int64_t j = 1; j < n; ++j)
      if (fabs(r[j]) > fabs(r[jp])) jp = j;
    if (r[jp] == 0.0) { /* zero residual row: try the next unused row */
      for (i = 0; i < m && used[i]; ++i) {}
      continue;
    }
    const double piv = r[jp];
    double* v = V + n * rank;
    double* u = U + m * rank;
    for (int64_t j = 0; j < n; ++j) v[j] = r[j] / piv;
    /* residual column jp */
    for (int64_t t = 0; t < m; ++t) {
      double s = orc_entry(k, pts, I[t], J[jp]);
      for (int64_t q = 0; q < rank; ++q) s -= U[t + m * q] * V[jp + n * q];
      u[t] = s;
    }
    double uu = 0.0, vv = 0.0;
    for (int64_t t = 0; t < m; ++t) uu += u[t] * u[t];
    for (int64_t j = 0; j < n; ++j) vv += v[j] * v[j];
    double cross = 0.0;
    for (int64_t q = 0; q < rank; ++q) {
      double du = 0.0, dv = 0.0;
      for (int64_t t = 0; t < m; ++t) du += U[t + m * q] * u[t];
      for (int64_t j = 0; j < n; ++j) dv += V[j + n * q] * v[j];
      cross += du * dv;
    }
    S2 += 2.0 * cross + uu * vv;
    ++rank;
    if (sqrt(uu) * sqrt(vv) <= eps * sqrt(S2 > 0.0 ? S2 : 0.0)) break;
    /* next row: largest |u| among the unused rows, first on ties */
    int64_t best = -1;
    for (int64_t t = 0; t < m; ++t) {
      if (used[t]) continue;
      if (best < 0 || fabs(u[t]) > fabs(u[best])) best = t;
    }
    if (best < 0) break;
    i = best;
  }
  free(used);
  free(r);
  return (int)rank;
}

/* ------------------------------------------------------------------------ */
/* InitializeHODLR2D (Alg. 1)                                                */
/* ------------------------------------------------------------------------ */

static int add_pair(orc_h2d* h, int l, int64_t bx, int64_t by) {
  if (h->npairs == h->cap_pairs) {
    const int64_t nc = h->cap_pairs ? 2 * h->cap_pairs : 64;
    orc_pair* np = (orc_pair*)realloc(h->pairs, (size_t)nc * sizeof(orc_pair));
    if (!np) return -2;
    h->pairs = np;
    h->cap_pairs = nc;
  }
  orc_pair* p = &h->pairs[h->npairs++];
  memset(p, 0, sizeof(*p));
  p->level = l;
  p->bx = bx;
  p->by = by;
  p->nx = box_count(h, l, bx);
  p->ny = box_count(h, l, by);
  return 0;
}

static int compress_pair(orc_h2d* h, orc_pair* p) {
  const int64_t kmax = p->nx < p->ny ? p->nx : p->ny;
  double* U = (double*)malloc((size_t)(p->nx * kmax) * sizeof(double));
  double* V = (double*)malloc((size_t)(p->ny * kmax) * sizeof(double));
  if (!U || !V) { free(U); free(V); return -2; }
  const int64_t* I = h->idx[p->level] + h->off[p->level][p->bx];
  const int64_t* J = h->idx[p->level] + h->off[p->level][p->by];
  const int r = orc_aca(&h->k, h->pts, p->nx, I, p->ny, J, h->eps, U, V);
  if (r < 0) { free(U); free(V); return r; }
  p->rank = r;
  p->U = U;
  p->V = V;
  return 0;
}

int orc_build(int64_t n, const double* pts, const orc_kernel* k, int leaf_size,
              double eps, const double* root, int levels, int compress,
              orc_h2d** out) {
  if (n < 1 || !pts || !k || !out || leaf_size < 1 || !(eps > 0.0)) return -1;
  orc_h2d* h = (orc_h2d*)calloc(1, sizeof(orc_h2d));
  if (!h) return -2;
  h->n = n;
  h->k = *k;
  h->eps = eps;
  h->pts = (double*)malloc((size_t)(2 * n) * sizeof(double));
  if (!h->pts) { orc_free(h); return -2; }
  memcpy(h->pts, pts, (size_t)(2 * n) * sizeof(double));
  if (root) {
    h->x0 = root[0]; h->y0 = root[1]; h->w = root[2];
  } else {
    double xmin = pts[0], xmax = pts[0], ymin = pts[1], ymax = pts[1];
    for (int64_t i = 1; i < n; ++i) {
      xmin = fmin(xmin, pts[2 * i]); xmax = fmax(xmax, pts[2 * i]);
      ymin = fmin(ymin, pts[2 * i + 1]); ymax = fmax(ymax, pts[2 * i + 1]);
    }
    double w = fmax(xmax - xmin, ymax - ymin);
    if (!(w > 0.0)) w = 1.0;
    h->w = w;
    h->x0 = 0.5 * (xmin + xmax) - 0.5 * w;
    h->y0 = 0.5 * (ymin + ymax) - 0.5 * w;
  }
  int rc = build_tree(h, leaf_size, levels);
  if (!rc) rc = build_lists(h);
  /* stored pairs: every unordered interaction-list pair once, rows = the box
   * with the smaller Morton key; levels kappa down to 1 as in Alg. 1 */
  for (int l = h->kappa; !rc && l >= 1; --l) {
    const int64_t nb = nboxes(l);
    for (int64_t b = 0; !rc && b < nb; ++b) {
      int32_t bx, by;
      orc_paper_coords(l, b, &bx, &by);
      for (int64_t t = h->i_off[l][b]; !rc && t < h->i_off[l][b + 1]; ++t) {
        const int64_t q = h->i_lst[l][t];
        int32_t qx, qy;
        orc_paper_coords(l, q, &qx, &qy);
        if (morton(l, bx, by) < morton(l, qx, qy)) rc = add_pair(h, l, b, q);
      }
    }
  }
  /* link every (box, list entry) to the pair that serves it */
  for (int64_t p = 0; !rc && p < h->npairs; ++p) {
    const orc_pair* pp = &h->pairs[p];
    const int l = pp->level;
    for (int side = 0; side < 2; ++side) {
      const int64_t b = side ? pp->by : pp->bx, q = side ? pp->bx : pp->by;
      for (int64_t t = h->i_off[l][b]; t < h->i_off[l][b + 1]; ++t)
        if (h->i_lst[l][t] == q) h->i_pair[l][t] = p;
    }
  }
  if (compress)
    for (int64_t p = 0; !rc && p < h->npairs; ++p) rc = compress_pair(h, &h->pairs[p]);
  if (rc) { orc_free(h); return rc; }
  *out = h;
  return 0;
}

void orc_free(orc_h2d* h) {
  if (!h) return;
  for (int l = 0; l <= h->kappa; ++l) {
    if (h->off) free(h->off[l]);
    if (h->idx) free(h->idx[l]);
    if (h->e_off) free(h->e_off[l]);
    if (h->e_lst) free(h->e_lst[l]);
    if (h->i_off) free(h->i_off[l]);
    if (h->i_lst) free(h->i_lst[l]);
    if (h->i_pair) free(h->i_pair[l]);
  }
  free(h->off); free(h->idx); free(h->e_off); free(h->e_lst);
  free(h->i_off); free(h->i_lst); free(h->i_pair);
  for (int64_t p = 0; p < h->npairs; ++p) { free(h->pairs[p].U); free(h->pairs[p].V); }
  free(h->pairs);
  free(h->pts);
  free(h);
}

/* ------------------------------------------------------------------------ */
/* MatVec (Alg. 2)                                                           */
/* ------------------------------------------------------------------------ */

/* b(X) += K(X,Y) psi(Y), entries evaluated from the points */
static void dense_block(const orc_h2d* h, int l, int64_t bx, int64_t by,
                        const double* x, double* y, int nrhs) {
  const int64_t* X = h->idx[l] + h->off[l][bx];
  const int64_t* Y = h->idx[l] + h->off[l][by];
  const int64_t nx = box_count(h, l, bx), ny = box_count(h, l, by);
  for (int c = 0; c < nrhs; ++c)
    for (int64_t i = 0; i < nx; ++i) {
      double s = 0.0;
      for (int64_t j = 0; j < ny; ++j) s += orc_entry(&h->k, h->pts, X[i], Y[j]) * x[Y[j] + h->n * c];
      y[X[i] + h->n * c] += s;
    }
}

/* b(X) += U (V^T psi(Y)) for the list entry t of box b at level l */
static void lowrank_block(const orc_h2d* h, int l, int64_t b, int64_t t,
                          const double* x, double* y, int nrhs) {
  const orc_pair* p = &h->pairs[h->i_pair[l][t]];
  const int row = (p->bx == b); /* X is the row side of the stored pair */
  const double* L = row ? p->U : p->V; /* applied on X's side */
  const double* R = row ? p->V : p->U; /* projected against psi(Y) */
  const int64_t nX = row ? p->nx : p->ny, nY = row ? p->ny : p->nx;
  const int64_t* X = h->idx[l] + h->off[l][b];
  const int64_t* Y = h->idx[l] + h->off[l][h->i_lst[l][t]];
  double* tmp = (double*)malloc((size_t)(p->rank > 0 ? p->rank : 1) * sizeof(double));
  for (int c = 0; c < nrhs; ++c) {
    for (int q = 0; q < p->rank; ++q) {
      double s = 0.0;
      for (int64_t j = 0; j < nY; ++j) s += R[j + nY * q] * x[Y[j] + h->n * c];
      tmp[q] = s;
    }
    for (int64_t i = 0; i < nX; ++i) {
      double s = 0.0;
      for (int q = 0; q < p->rank; ++q) s += L[i + nX * q] * tmp[q];
      y[X[i] + h->n * c] += s;
    }
  }
  free(tmp);
}

void orc_matvec_far_levels(const orc_h2d* h, const double* x, double* y,
                           int nrhs, int l0, int l1) {
  for (int l = l0; l <= l1 && l <= h->kappa; ++l) {
    if (l < 1) continue;
    for (int64_t b = 0; b < nboxes(l); ++b)
      for (int64_t t = h->i_off[l][b]; t < h->i_off[l][b + 1]; ++t)
        lowrank_block(h, l, b, t, x, y, nrhs);
  }
}

void orc_matvec(const orc_h2d* h, const double* x, double* y, int nrhs) {
  const int kappa = h->kappa;
  memset(y, 0, (size_t)(h->n * nrhs) * sizeof(double));
  /* full-rank products at the leaf level: self and edge sharers */
  for (int64_t b = 0; b < nboxes(kappa); ++b) {
    if (box_count(h, kappa, b) == 0) continue;
    dense_block(h, kappa, b, b, x, y, nrhs);
    for (int64_t t = h->e_off[kappa][b]; t < h->e_off[kappa][b + 1]; ++t)
      dense_block(h, kappa, b, h->e_lst[kappa][t], x, y, nrhs);
  }
  /* low-rank products, levels 1..kappa */
  orc_matvec_far_levels(h, x, y, nrhs, 1, kappa);
}

/* ------------------------------------------------------------------------ */
/* Introspection                                                             */
/* ------------------------------------------------------------------------ */

void orc_info(const orc_h2d* h, int* kappa, double* root3, int64_t* npairs,
              int64_t* nvalues) {
  if (kappa) *kappa = h->kappa;
  if (root3) { root3[0] = h->x0; root3[1] = h->y0; root3[2] = h->w; }
  if (npairs) *npairs = h->npairs;
  if (nvalues) {
    int64_t s = 0;
    for (int64_t p = 0; p < h->npairs; ++p)
      s += (h->pairs[p].nx + h->pairs[p].ny) * h->pairs[p].rank;
    *nvalues = s;
  }
}

void orc_box_counts(const orc_h2d* h, int l, int64_t* counts) {
  for (int64_t b = 0; b < nboxes(l); ++b) counts[b] = box_count(h, l, b);
}

int64_t orc_box_points(const orc_h2d* h, int l, int64_t b, int64_t* out) {
  const int64_t c = box_count(h, l, b);
  if (out) memcpy(out, h->idx[l] + h->off[l][b], (size_t)c * sizeof(int64_t));
  return c;
}

int orc_edge_list(const orc_h2d* h, int l, int64_t b, int64_t* out, int cap) {
  const int64_t s = h->e_off[l][b], e = h->e_off[l][b + 1];
  for (int64_t t = s; t < e && t - s < cap; ++t) out[t - s] = h->e_lst[l][t];
  return (int)(e - s);
}

int orc_interaction_list(const orc_h2d* h, int l, int64_t b, int64_t* out, int cap) {
  if (l == 0) return 0;
  const int64_t s = h->i_off[l][b], e = h->i_off[l][b + 1];
  for (int64_t t = s; t < e && t - s < cap; ++t) out[t - s] = h->i_lst[l][t];
  return (int)(e - s);
}

void orc_level_counts(const orc_h2d* h, int l, int64_t* out4) {
  out4[0] = out4[1] = out4[2] = out4[3] = 0;
  for (int64_t b = 0; b < nboxes(l); ++b) {
    if (box_count(h, l, b) == 0) continue;
    out4[0] += 1;
    out4[1] += h->e_off[l][b + 1] - h->e_off[l][b];
    if (l == 0) continue;
    int32_t cx, cy;
    orc_paper_coords(l, b, &cx, &cy);
    for (int64_t t = h->i_off[l][b]; t < h->i_off[l][b + 1]; ++t) {
      int32_t qx, qy;
      orc_paper_coords(l, h->i_lst[l][t], &qx, &qy);
      out4[relation(cx, cy, qx, qy) == REL_VERTEX ? 2 : 3] += 1;
    }
  }
}

static void mark_block(const orc_h2d* h, int l, int64_t bx, int64_t by, int32_t* mark) {
  const int64_t* X = h->idx[l] + h->off[l][bx];
  const int64_t* Y = h->idx[l] + h->off[l][by];
  for (int64_t i = 0; i < box_count(h, l, bx); ++i)
    for (int64_t j = 0; j < box_count(h, l, by); ++j) mark[X[i] * h->n + Y[j]] += 1;
}

void orc_coverage(const orc_h2d* h, int32_t* mark) {
  const int kappa = h->kappa;
  for (int64_t b = 0; b < nboxes(kappa); ++b) {
    if (box_count(h, kappa, b) == 0) continue;
    mark_block(h, kappa, b, b, mark);
    for (int64_t t = h->e_off[kappa][b]; t < h->e_off[kappa][b + 1]; ++t)
      mark_block(h, kappa, b, h->e_lst[kappa][t], mark);
  }
  for (int l = 1; l <= kappa; ++l)
    for (int64_t b = 0; b < nboxes(l); ++b)
      for (int64_t t = h->i_off[l][b]; t < h->i_off[l][b + 1]; ++t)
        mark_block(h, l, b, h->i_lst[l][t], mark);
}

void orc_pair_info(const orc_h2d* h, int64_t p, int32_t* info6, int64_t* nx,
                   int64_t* ny) {
  const orc_pair* pp = &h->pairs[p];
  int32_t ax, ay, bx, by;
  orc_paper_coords(pp->level, pp->bx, &ax, &ay);
  orc_paper_coords(pp->level, pp->by, &bx, &by);
  info6[0] = pp->level; info6[1] = ax; info6[2] = ay;
  info6[3] = bx; info6[4] = by; info6[5] = pp->rank;
  if (nx) *nx = pp->nx;
  if (ny) *ny = pp->ny;
}

void orc_pair_factors(const orc_h2d* h, int64_t p, double* U, double* V) {
  const orc_pair* pp = &h->pairs[p];
  if (pp->rank == 0) return;
  memcpy(U, pp->U, (size_t)(pp->nx * pp->rank) * sizeof(double));
  memcpy(V, pp->V, (size_t)(pp->ny * pp->rank) * sizeof(double));
}

void orc_export_factors(const orc_h2d* h, int32_t* info, int64_t* offsets, double* values) {
  offsets[0] = 0;
  for (int64_t p = 0; p < h->npairs; ++p) {
    const orc_pair* pp = &h->pairs[p];
    orc_pair_info(h, p, info + 6 * p, NULL, NULL);
    const int64_t nu = pp->nx * pp->rank, nv = pp->ny * pp->rank;
    if (values) orc_pair_factors(h, p, values + offsets[p], values + offsets[p] + nu);
    offsets[p + 1] = offsets[p] + nu + nv;
  }
}
