/*
 * HODLR2D CPU oracle: plain, slow, FP64 reference of the method.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference legs may load this library.  It shares
 * no code, header, table or helper with the CUDA library; the only thing the
 * two sides have in common is the seeded input generator (a separate Python
 * module with none of the method's arithmetic).
 *
 * Paper: "HODLR2D: A new class of hierarchical matrices" (arXiv 2204.05536).
 *   - kernel functions: Sec. 3 (log r, zero diagonal), Eq. 1byr (1/r, zero
 *     diagonal), Eq. ker with phi_1 / phi_2 (RBF system, beta on the diagonal);
 *     inverse multiquadric and multiquadric are the RBFs the workloads name.
 *   - tree: Sec. 4, Fig. sdomain01 (counter-clockwise child numbering),
 *     Alg. 1 (balanced quadtree, every leaf holds at most N_max points).
 *   - lists: Defs. ec, vc, wc, cc, ic and Eq. ilist.
 *   - compression: Alg. 1 (ACA at tolerance eps for every interaction-list pair).
 *   - matvec: Alg. 2.
 */
#ifndef HODLR2D_ORACLE_H
#define HODLR2D_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_IMQ = 0,   /* 1/sqrt(r^2+a^2)                                   */
  ORC_MQ = 1,    /* sqrt(r^2+a^2)                                     */
  ORC_LOG = 2,   /* log r                 (Sec. 3)                    */
  ORC_INV_R = 3, /* 1/r                   (Eq. 1byr)                  */
  ORC_PHI1 = 4,  /* phi_1 of Sec. 5.2                                 */
  ORC_PHI2 = 5   /* phi_2 of Sec. 5.2                                 */
};

typedef struct {
  int kind;
  double a;          /* shape parameter (IMQ, MQ, PHI1, PHI2)              */
  int diag_mode;     /* 0: phi(0) (0 for LOG / INV_R), 1: diag_value     */
  double diag_value; /* e.g. beta = N of Eq. ker                          */
} orc_kernel;

/* Entry A_ij of the dense matrix.  pts is N x 2 row-major. */
double orc_entry(const orc_kernel* k, const double* pts, int64_t i, int64_t j);

/* Direct O(N^2) product y = A x, j summed in ascending order.
 * x, y: n x nrhs column-major.  The reference for Sec. 5.1's error ε_r. */
void orc_direct_matvec(int64_t n, const double* pts, const orc_kernel* k,
                       const double* x, double* y, int nrhs);

/* Same, for a list of rows only: y is nrows x nrhs column-major. */
void orc_direct_rows(int64_t n, const double* pts, const orc_kernel* k,
                     const double* x, int nrhs, int64_t nrows,
                     const int64_t* rows, double* y);

typedef struct orc_h2d orc_h2d;

/* InitializeHODLR2D of Alg. 1.
 *   root:      NULL, or {x0, y0, w}: the square [x0,x0+w] x [y0,y0+w].
 *   levels:    <0 picks kappa by the leaf rule of Alg. 1; >=0 forces kappa.
 *   compress:  0 builds tree and lists only (no ACA).
 * Returns 0, or a negative code (-1 bad argument, -2 out of memory,
 * -3 no kappa <= max_levels satisfies the leaf rule). */
int orc_build(int64_t n, const double* pts, const orc_kernel* k, int leaf_size,
              double eps, const double* root, int levels, int compress,
              orc_h2d** out);
void orc_free(orc_h2d* h);

/* MatVec of Alg. 2: y = K_hat x.  x, y: n x nrhs column-major. */
void orc_matvec(const orc_h2d* h, const double* x, double* y, int nrhs);

/* Same product over the levels [l0, l1] of the far field only (near field
 * excluded); y is accumulated into, not overwritten.  Used to time a bounded
 * sample of the product. */
void orc_matvec_far_levels(const orc_h2d* h, const double* x, double* y,
                           int nrhs, int l0, int l1);

/* ----- introspection for tests ----- */
void orc_info(const orc_h2d* h, int* kappa, double* root3, int64_t* npairs,
              int64_t* nvalues);
/* number of points in every box of level l, indexed by the paper's numbering */
void orc_box_counts(const orc_h2d* h, int l, int64_t* counts);
/* points of box b (paper numbering) at level l, ascending original index */
int64_t orc_box_points(const orc_h2d* h, int l, int64_t b, int64_t* out);
/* paper numbering <-> grid coordinates (Fig. sdomain01) */
int64_t orc_paper_index(int l, int32_t ix, int32_t iy);
void orc_paper_coords(int l, int64_t b, int32_t* ix, int32_t* iy);
/* edge-sharer and interaction lists of box b at level l (paper numbering);
 * returns the list length, writes at most cap entries */
int orc_edge_list(const orc_h2d* h, int l, int64_t b, int64_t* out, int cap);
int orc_interaction_list(const orc_h2d* h, int l, int64_t b, int64_t* out, int cap);
/* ordered-pair counts at level l: [0] self, [1] edge sharers,
 * [2] vertex sharers in I, [3] well separated in I */
void orc_level_counts(const orc_h2d* h, int l, int64_t* out4);
/* mark[i*n + j] += 1 for every matrix entry covered by a dense leaf block or
 * by one interaction-list block; exact once-coverage means all ones */
void orc_coverage(const orc_h2d* h, int32_t* mark);
/* stored pair p: info = {level, ixX, iyX, ixY, iyY, rank}, sizes nX, nY */
void orc_pair_info(const orc_h2d* h, int64_t p, int32_t* info6, int64_t* nx,
                   int64_t* ny);
/* U (nX x k) and V (nY x k), column-major, rows in ascending original index */
void orc_pair_factors(const orc_h2d* h, int64_t p, double* U, double* V);
/* every stored pair in one flat layout: info[6p..6p+5] as orc_pair_info,
 * values[offsets[p] .. offsets[p+1]) = U then V of pair p as orc_pair_factors
 * gives them; offsets has npairs + 1 entries.  values may be NULL (sizes
 * only). */
void orc_export_factors(const orc_h2d* h, int32_t* info, int64_t* offsets, double* values);

/* Stand-alone ACA of A(I,J) (rows I, columns J given as point indices).
 * U: m x kmax, V: n x kmax column-major (caller sized with kmax=min(m,n)).
 * Returns the rank. */
int orc_aca(const orc_kernel* k, const double* pts, int64_t m, const int64_t* I,
            int64_t n, const int64_t* J, double eps, double* U, double* V);

#ifdef __cplusplus
}
#endif
#endif
