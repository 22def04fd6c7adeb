/*
 * hodlr2d.h -- C ABI of the GB300 (sm_103a) HODLR2D library.
 *
 * HODLR2D ("HODLR2D: A new class of hierarchical matrices", arXiv 2204.05536)
 * represents the dense N x N matrix A_ij = phi(|x_i - x_j|) of a 2D point set
 * on a balanced quadtree (Sec. 4):
 *   - at every level l = 1..kappa, the interaction of a box C with each box of
 *     its interaction list I_C (Def. ic, Eq. ilist: clan members that share
 *     only a vertex with C or are well separated from it) is a low-rank block
 *     U V^T obtained by ACA at tolerance eps (Alg. 1);
 *   - at the leaf level the self block and the edge-sharing blocks (Def. ec)
 *     stay dense (Remark in Sec. 4.1); they are evaluated from the kernel when
 *     the product runs, not stored;
 *   - the product b = K psi follows Alg. 2.
 *
 * Conventions (all entry points):
 *   - Return HODLR2D_OK (0) or a negative HODLR2D_ERR_* code; hodlr2d_strerror
 *     names it.  No entry point aborts, traps or prints.
 *   - Pointers marked "host or device" may be either; the library asks the
 *     CUDA runtime which one it was given.  Device pointers must be on the
 *     handle's device.
 *   - Matrices of right-hand sides are n x nrhs, column-major (column c starts
 *     at c * n), in the caller's point order.
 *   - A handle owns all of its device memory.  A handle is not thread-safe;
 *     separate handles may run concurrently on separate streams.
 *   - Work is queued on the handle's stream (hodlr2d_set_stream, default: the
 *     legacy default stream).  Calls that return host-visible results
 *     synchronise that stream before returning.
 */
#ifndef HODLR2D_H
#define HODLR2D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----- error codes ----- */
#define HODLR2D_OK 0
#define HODLR2D_ERR_ARG (-1)     /* invalid argument (null, size, NaN, ...)       */
#define HODLR2D_ERR_OOM (-2)     /* device or host allocation failed             */
#define HODLR2D_ERR_CUDA (-3)    /* a CUDA runtime call failed                   */
#define HODLR2D_ERR_NOCONV (-4)  /* an iteration did not reach its tolerance     */
#define HODLR2D_ERR_TIMEOUT (-5) /* a bounded device-side wait gave up         */
#define HODLR2D_ERR_DEPTH (-6)   /* no depth <= 14 meets the leaf rule           */
#define HODLR2D_ERR_STATE (-7)   /* handle not ready (e.g. no factors yet)       */

/* ----- kernel functions ----- */
typedef enum {
  HODLR2D_IMQ = 0,   /* 1 / sqrt(r^2 + a^2)                                      */
  HODLR2D_MQ = 1,    /* sqrt(r^2 + a^2)                                          */
  HODLR2D_LOG = 2,   /* log r                     (Sec. 3, zero diagonal)        */
  HODLR2D_INV_R = 3, /* 1 / r                     (Eq. 1byr, zero diagonal)      */
  HODLR2D_PHI1 = 4,  /* log r / log a (r >= a), (r log r - 1)/(a log a - 1) else */
  HODLR2D_PHI2 = 5   /* a / r (r >= a), r / a else            (Sec. 5.2, Eq. ker) */
} hodlr2d_kernel_kind;

typedef struct {
  int kind;          /* hodlr2d_kernel_kind                                    */
  double a;          /* shape parameter of IMQ, MQ, PHI1, PHI2                 */
  int diag_mode;     /* 0: A_ii = phi(0) (IMQ 1/a, MQ a, PHI1 -1/(a log a - 1),
                        PHI2 0; LOG and INV_R 0); 1: A_ii = diag_value
                        (beta of Eq. ker, or a panel self-term)                */
  double diag_value;
} hodlr2d_kernel;

/* ----- arithmetic of the product ----- */
typedef enum {
  /* factors stored in IEEE binary64, products and sums in binary64 */
  HODLR2D_MODE_F64 = 0,
  /* factors stored as unevaluated float pairs hi + lo (8 bytes, ~48-bit
     significand), products and sums in float-float arithmetic (Dekker 1971
     products, Knuth two-sum); the near field in the same arithmetic */
  HODLR2D_MODE_DF32 = 1,
  /* factors stored in binary32, binary32 products and sums */
  HODLR2D_MODE_F32 = 2,
  /* factors stored in bfloat16, binary32 products and sums */
  HODLR2D_MODE_BF16 = 3
} hodlr2d_mode;

/* ----- build options ----- */
typedef struct {
  double root[3];  /* {x0, y0, w}: the root box [x0,x0+w] x [y0,y0+w].  w <= 0:
                      the bounding square of the points (centred on their
                      bounding box) -- the default.                            */
  int levels;      /* < 0 (default): kappa = smallest depth whose leaves all
                      hold <= leaf_size points (Alg. 1); >= 0: force kappa.    */
  int compress;    /* 1 (default): run ACA; 0: tree and lists only, factors
                      come from hodlr2d_import_factors.                        */
  int max_rank;    /* ACA rank cap per block (default 256).  A block that hits
                      the cap before eps is counted in stats.unconverged.      */
  int mode;        /* hodlr2d_mode used by hodlr2d_matvec (default F64).      */
  void* rank_model; /* NULL (default), or a hodlr2d_rank_model_t: each ACA runs
                      with the rank cap the model predicts (workspace sized up
                      front); a pair that reaches it without meeting eps is
                      redone with the full cap, so the factors are those of
                      the build without a model.                              */
} hodlr2d_opts;

typedef struct hodlr2d* hodlr2d_t;

/* Fill *opts with the defaults listed above. */
void hodlr2d_default_opts(hodlr2d_opts* opts);

/* InitializeHODLR2D (Alg. 1): quadtree, edge and interaction lists (Defs. ec,
 * ic), ACA of every admissible pair at tolerance eps.
 *   points:    N x 2 row-major {x_i, y_i}, host or device; copied.
 *   n:         N >= 1.
 *   kernel:    entry rule; a > 0 where the kind uses it.
 *   leaf_size: N_max >= 1 of Alg. 1.
 *   eps:       ACA tolerance, 0 < eps < 1.
 *   out:       receives the handle (unchanged on error).
 * The kernels are radial, so A(Y,X) = A(X,Y)^T: each unordered admissible
 * pair is compressed once (rows: the box with the smaller Morton key) and
 * serves both directions.  Errors: ARG, OOM, CUDA, DEPTH. */
int hodlr2d_build(const double* points, int64_t n, hodlr2d_kernel kernel,
                  int leaf_size, double eps, hodlr2d_t* out);

/* As hodlr2d_build with options (opts may be NULL for the defaults). */
int hodlr2d_build_ex(const double* points, int64_t n, hodlr2d_kernel kernel,
                     int leaf_size, double eps, const hodlr2d_opts* opts,
                     hodlr2d_t* out);

/* MatVec (Alg. 2): y = K_hat x in the handle's default mode.
 *   x: n x nrhs column-major, host or device (read only).
 *   y: n x nrhs column-major, host or device (overwritten).
 *   nrhs >= 1.
 * With device x and y the call is asynchronous on the handle's stream; with a
 * host x or y it returns after y is written.  Errors: ARG, STATE, CUDA. */
int hodlr2d_matvec(hodlr2d_t h, const double* x, double* y, int nrhs);

/* As hodlr2d_matvec in an explicit hodlr2d_mode.  Modes other than F64 need a
 * prior hodlr2d_prepare(h, mode) (else HODLR2D_ERR_STATE). */
int hodlr2d_matvec_ex(hodlr2d_t h, const double* x, double* y, int nrhs, int mode);

/* Make the factor copy that a mode reads (allocates device memory once; the
 * F64 factors stay).  Errors: ARG, OOM, CUDA, STATE (no factors, or the F64
 * factors were released and this copy was not made before). */
int hodlr2d_prepare(hodlr2d_t h, int mode);

/* Free the device memory of one mode's factors (hodlr2d_mode), e.g. the
 * F64 factors once the float-float copy exists, which halves the factor
 * memory of a float-float-only handle (15.5 GB at N = 2^20, eps 1e-8).  The
 * mode's products then return HODLR2D_ERR_STATE; a released F64 copy cannot
 * come back (later hodlr2d_prepare of a new mode, hodlr2d_export_factors,
 * hodlr2d_matvec_noalloc and GMRES refinement around F32 / BF16 products,
 * which need the F64 factors, return HODLR2D_ERR_STATE); a released other
 * copy can be prepared again while the F64 factors exist.  Synchronises the
 * handle's stream.  Errors: ARG, STATE (no factors). */
int hodlr2d_release(hodlr2d_t h, int mode);

/* Restarted GMRES for A x = b with the HODLR2D product (Sec. 5.2, 5.3), all
 * in FP64 on the GPU.  b, x: n vectors, host or device; x holds x0 on entry
 * and the solution on return.  Stops at |b - A x| <= tol |b|.
 * hodlr2d_gmres uses restart 50 and maxit = min(10 n, 100000) matvecs. */
int hodlr2d_gmres(hodlr2d_t h, const double* b, double* x, double tol);

/* As hodlr2d_gmres with explicit restart length, matvec cap, and outputs
 * (iters: matvecs used, relres: final |b - A x| / |b|; either may be NULL).
 * inner_mode: the hodlr2d_mode of the products inside each cycle.  F64 and
 * DF32 (binary64-level accuracy) run plain GMRES with that product; F32 and
 * BF16 run iterative refinement: residuals r = b - A x with the F64 product,
 * corrections solved with inner_mode to a relative residual of 1e-5 (F32) or
 * 1e-2 (BF16).  Products of a zero vector are skipped and not counted.  The
 * Krylov workspace ((restart + 6) n doubles) is kept by the handle until
 * hodlr2d_free.  Returns HODLR2D_ERR_NOCONV (with x and the outputs filled)
 * when maxit is reached first. */
int hodlr2d_gmres_ex(hodlr2d_t h, const double* b, double* x, double tol,
                     int restart, int maxit, int inner_mode, int* iters,
                     double* relres);

/* ----- statistics (Sec. 5 notation: kappa, r_m, CR, memory, T_I) ----- */
#define HODLR2D_MAX_LEVELS 15
typedef struct {
  int64_t n;
  int kappa;
  double root[3];
  int64_t npairs;                            /* stored (unordered) pairs      */
  int64_t pairs_per_level[HODLR2D_MAX_LEVELS];
  int64_t values_per_level[HODLR2D_MAX_LEVELS]; /* sum (|X|+|Y|) k           */
  int max_rank_per_level[HODLR2D_MAX_LEVELS];
  int max_rank;                              /* r_m                           */
  int64_t far_values;                        /* stored factor values          */
  int64_t near_entries;                      /* dense leaf entries per product */
  int64_t unconverged;                       /* pairs that hit max_rank       */
  double compression_ratio;                  /* (far_values + near_entries)/N^2 */
  double build_ms[4];                        /* tree, lists, ACA, pack        */
  int64_t bytes_per_matvec[4];               /* algorithmic bytes, per mode   */
  int64_t aca_fallbacks;                     /* pairs redone after a predicted
                                                cap (rank model) was too small */
  int64_t aca_workspace_values;              /* largest ACA workspace batch   */
} hodlr2d_stats;

int hodlr2d_get_stats(hodlr2d_t h, hodlr2d_stats* s);

/* ----- tracing: per-phase device time of the product -----
 * Phases of one product (one kernel, or one per pair size class): 0 gather
 * x, 1 near field, 2 far-field projection (coarse levels), 3 projection
 * sums, 4 far-field expansion (coarse levels), 5 combine and scatter y,
 * 6 single-read far field, one block per pair (mid levels), 7 single-read
 * far field of the finest levels (boxes of at most 64 points: one warp per
 * box in binary64, sub-warp pairs otherwise), 8 as 6 for smaller boxes,
 * 9 unused.  While
 * enabled, each phase is bracketed by CUDA events and the product runs on the
 * handle's stream alone (no side streams), so each time is that of its
 * kernel running by itself.  hodlr2d_profile(h, 1) resets and starts
 * recording, (h, 0) stops.  hodlr2d_get_profile synchronises the stream and
 * returns, per phase, the summed milliseconds, the number of kernel launches,
 * and the summed algorithmic bytes of those launches (arrays of
 * HODLR2D_NPHASE entries; any may be NULL). */
#define HODLR2D_NPHASE 10
int hodlr2d_profile(hodlr2d_t h, int enable);
int hodlr2d_get_profile(hodlr2d_t h, double* ms, int64_t* launches, int64_t* bytes);
/* Per phase, the summed algorithmic floating-point operations of the
 * recorded launches (flops: HODLR2D_NPHASE entries): 4 per stored factor
 * value and right-hand side in the far field (each value takes part in one
 * multiply-add of a projection and one of an expansion), and per near-field
 * entry c_K + 2 per right-hand side, c_K the operations of the kernel's
 * formula with each elementary function (sqrt, log, a division) counted as
 * one: 7 for MQ, INV_R, LOG and PHI2, 8 for IMQ and PHI1. */
int hodlr2d_get_profile_flops(hodlr2d_t h, int64_t* flops);

/* Synchronise the handle's stream and report whether a product kernel gave
 * up a bounded device-side wait since the last check (the tensor-core
 * kernels of the bfloat16 many-RHS product wait on mbarriers for their
 * MMAs): HODLR2D_ERR_TIMEOUT, whose products since the previous check are
 * not to be trusted, or HODLR2D_OK.  Clears the flag.  Errors: ARG, CUDA. */
int hodlr2d_check(hodlr2d_t h);

/* Queue the handle's work on a cudaStream_t (passed as void*). */
int hodlr2d_set_stream(hodlr2d_t h, void* stream);

/* ----- tree introspection (tests, tools) ----- */
/* perm[i] = original index of the point at tree position i (Morton order of
 * the leaves, ascending original index inside a leaf).  perm: n int64, host. */
int hodlr2d_get_perm(hodlr2d_t h, int64_t* perm);
/* Stored pairs: for pair p, info[6p..6p+5] = {level, ixX, iyX, ixY, iyY, rank}
 * with X the row side.  Pass info = NULL to get the count in *npairs. */
int hodlr2d_get_pairs(hodlr2d_t h, int64_t* npairs, int32_t* info);

/* ----- factor exchange (checkpoint / resume, and tests) -----
 * Flat layout shared by import and export: npairs pairs, each
 *   info[6p..6p+5] = {level, ixX, iyX, ixY, iyY, rank},
 *   values[offsets[p] .. offsets[p+1]) = U (|X| x rank) then V (|Y| x rank),
 *   each column-major, rows ordered by ascending original point index.
 * Import requires a handle built with the same points, kernel and tree and
 * exactly its set of stored pairs (any order); all host pointers.
 * Errors: ARG (pair set or sizes differ), OOM, CUDA. */
int hodlr2d_import_factors(hodlr2d_t h, int64_t npairs, const int32_t* info,
                           const int64_t* offsets, const double* values);
/* Export: pass values = NULL to get *npairs and *nvalues only. */
int hodlr2d_export_factors(hodlr2d_t h, int64_t* npairs, int64_t* nvalues,
                           int32_t* info, int64_t* offsets, double* values);

/* ----- learned rank predictor (spec extension; not in the paper) -----
 * An 8 -> H -> H -> 1 ReLU network in binary32 mapping the geometry of an
 * admissible block to log2(rank + 1) of its ACA factorisation.  Features per
 * pair (hodlr2d_pair_features): level/16, (ixY - ixX)/3, (iyY - iyX)/3,
 * log2|X|/16, log2|Y|/16, min(a / box width, 4)/4, -log10(eps)/16, kind/8.
 * Parameters: one flat vector W1 (8 x H row-major), b1, W2 (H x H), b2, w3,
 * b3.  Training (forward, backward, Adam) runs on the GPU; loss is the mean
 * squared error.  feats are n x 8 row-major binary32, targets and predictions
 * n binary32; host or device pointers.  Every reduction runs in a fixed
 * order, so results are reproducible bit for bit. */
typedef struct hodlr2d_rank_model* hodlr2d_rank_model_t;
/* params: NULL (zeros) or the initial flat vector (host or device). */
int hodlr2d_rank_model_create(int hidden, const float* params, hodlr2d_rank_model_t* out);
/* Current parameters (params may be NULL to query the count). */
int hodlr2d_rank_model_params(hodlr2d_rank_model_t m, float* params, int64_t* nparams);
/* Loss and its gradient (host outputs, either may be NULL) on one batch. */
int hodlr2d_rank_model_loss_grad(hodlr2d_rank_model_t m, const float* feats,
                                 const float* targets, int64_t n, float* loss,
                                 float* grad);
/* epochs passes of Adam over the data in the given order, mini-batches of
 * batch rows, learning rate lr; *loss_out (may be NULL) = final loss. */
int hodlr2d_rank_model_train(hodlr2d_rank_model_t m, const float* feats,
                             const float* targets, int64_t n, int batch,
                             int epochs, float lr, float* loss_out);
int hodlr2d_rank_model_predict(hodlr2d_rank_model_t m, const float* feats,
                               int64_t n, float* pred);
void hodlr2d_rank_model_free(hodlr2d_rank_model_t m);
/* Training data from a built handle: per stored pair (in hodlr2d_get_pairs
 * order) its 8 features and log2(rank + 1).  feats / log2rank: host arrays of
 * 8 * npairs / npairs floats, or NULL to query *npairs. */
int hodlr2d_pair_features(hodlr2d_t h, int64_t* npairs, float* feats, float* log2rank);

/* ----- many independent matrices (point sets of uneven size) -----
 * Not in the paper (deployment batching).  Each set's product is the Alg. 2
 * product of its own handle.  Two forms:
 *   HODLR2D_BATCH_GRAPH: the first hodlr2d_batch_matvec (and any call whose
 *     pointers, nrhs or mode differ from the recorded ones) runs the products
 *     once, then records them into a CUDA graph (sets spread over eight
 *     forked streams); later calls replay that graph on the batch's stream.
 *     Every mode.  Bit for bit the handles' own products.
 *   HODLR2D_BATCH_PERSISTENT: one cooperative kernel launch multiplies all
 *     sets (recorded into a graph when the driver allows it), in five phases
 *     separated by grid barriers: gather; pairs, projections and near field;
 *     chunk sums; expansions; combine (see hodlr2d_batch_set_shapes).  Modes
 *     F64 and F32 only (others: ARG).  Within rounding of the handles' own
 *     products (its sums run in another order).  Each barrier wait is
 *     bounded (hodlr2d_batch_set_wait_limit); a block whose wait gives up
 *     records it and the launch ends without writing y:
 *     hodlr2d_batch_check then returns HODLR2D_ERR_TIMEOUT.
 *   HODLR2D_BATCH_AUTO (the default): GRAPH, which measured faster on the
 *     benchmark's 256 sets, until hodlr2d_batch_autotune has timed both
 *     forms on the caller's inputs; then the faster of the two.
 * Either form is set up again when a handle's plans, working memory or
 * factor copies have changed since the recording.  A handle may appear once
 * in a batch (repeats: ARG; its working memory serves one product at a
 * time).  The handles must outlive
 * the batch and must not be used concurrently with it.  x[i], y[i]: device
 * pointers, n_i x nrhs[i] column-major.  Profiling (hodlr2d_profile) must be
 * off on every handle.  Errors: ARG, STATE, CUDA. */
typedef struct hodlr2d_batch* hodlr2d_batch_t;
#define HODLR2D_BATCH_AUTO 0
#define HODLR2D_BATCH_GRAPH 1
#define HODLR2D_BATCH_PERSISTENT 2
int hodlr2d_batch_create(const hodlr2d_t* handles, int count, hodlr2d_batch_t* out);
int hodlr2d_batch_set_stream(hodlr2d_batch_t b, void* stream);
/* form: one of HODLR2D_BATCH_*; ARG otherwise. */
int hodlr2d_batch_set_form(hodlr2d_batch_t b, int form);
/* Polls of a grid-barrier wait of the persistent form before it gives up
 * (default 4194304, each poll followed by a sleep of about 64 ns, so at
 * least a quarter of a second).  0 makes every wait give up at once: a
 * self-test of the timeout path that leaves the context usable. */
int hodlr2d_batch_set_wait_limit(hodlr2d_batch_t b, uint32_t polls);
int hodlr2d_batch_matvec(hodlr2d_batch_t b, const double* const* x, double* const* y,
                         const int* nrhs, int mode);
/* Synchronises the batch's stream; HODLR2D_ERR_TIMEOUT if a persistent
 * product since the previous check gave up a barrier wait (its y is not
 * written), else OK.  Clears the record. */
int hodlr2d_batch_check(hodlr2d_batch_t b);
/* The form the last hodlr2d_batch_matvec ran (HODLR2D_BATCH_GRAPH or
 * HODLR2D_BATCH_PERSISTENT), or -1 before the first. */
int hodlr2d_batch_last_form(hodlr2d_batch_t b);
/* 1 if the persistent form's launch is recorded in a CUDA graph (stream
 * capture of the cooperative launch, replayed with one graph launch), 0 if
 * the driver refused the capture and it is launched directly, -1 before the
 * first persistent product. */
int hodlr2d_batch_persistent_recorded(hodlr2d_batch_t b);
/* Work shapes of the persistent form by box size: the levels whose boxes
 * hold at most pair_rows points (0 <= pair_rows <= 2048; binary64 uses at
 * most 1024) run as pairs, each stored pair read once (t1 = V^T x_Y,
 * t2 = U^T x_X, then U t1 and V t2): pairs of at most warp_rows points
 * (0 <= warp_rows <= 64) one per warp, of at most 128 points four per
 * 256-thread unit, of at most 256 two per unit, larger ones one per unit;
 * coarser levels run in two passes (projections over 512-row chunks, chunk
 * sums, expansions over 256-row chunks).  Defaults 384 and 64.  Takes effect
 * at the next product. */
int hodlr2d_batch_set_shapes(hodlr2d_batch_t b, int pair_rows, int warp_rows);
int hodlr2d_batch_get_shapes(hodlr2d_batch_t b, int* pair_rows, int* warp_rows);
/* Resident 256-thread blocks per SM of the persistent kernel: 2, 3 (the
 * default) or 4, i.e. at most 128, 80 or 64 registers a thread. */
int hodlr2d_batch_set_blocks_per_sm(hodlr2d_batch_t b, int blocks);
/* Phase of the work that depends only on the gathered x (0-3): bit 0 runs
 * the near field beside the expansions (phase 3) instead of beside the
 * projections (phase 1); bit 1 runs the one-warp pairs beside the chunk sums
 * (phase 2).  Default 0. */
int hodlr2d_batch_set_placement(hodlr2d_batch_t b, int place);
/* Autotuner of those settings: times reps persistent products (CUDA events
 * on the batch's stream, after one untimed product) for each candidate
 * pair_rows in {0, 128, 256, 512, 1024, 2048} and warp_rows in {0, 48, 64}
 * (warp_rows <= pair_rows) at the current blocks per SM and placement,
 * then the other blocks-per-SM values at the fastest shapes, then the other
 * placements; keeps the fastest and writes its time per product to *best_ms
 * (may be NULL).  Then times the graph form once (its table row has -1 for
 * the four settings), and HODLR2D_BATCH_AUTO runs the faster form from then
 * on.  Arguments as in
 * hodlr2d_batch_matvec (y is overwritten); modes F64 and F32 only.
 * Synchronises the stream.  Errors: ARG, STATE, CUDA, TIMEOUT. */
int hodlr2d_batch_autotune(hodlr2d_batch_t b, const double* const* x, double* const* y,
                           const int* nrhs, int mode, int reps, double* best_ms);
/* The candidates of the last hodlr2d_batch_autotune with their times per
 * product.  *count: in, the room of the five host arrays; out, the number
 * of candidates timed (arrays may be NULL to query it). */
int hodlr2d_batch_tune_table(hodlr2d_batch_t b, int* count, int* pair_rows, int* warp_rows,
                             int* blocks, int* place, double* ms);
/* Milliseconds of the five phases of the last persistent product (gather;
 * pairs, projections and near field; chunk sums; expansions; combine), read
 * from the device clock at the grid barriers.  ms: host array of 5.
 * Synchronises the stream.  STATE before the first persistent product. */
int hodlr2d_batch_phase_ms(hodlr2d_batch_t b, double* ms);
void hodlr2d_batch_free(hodlr2d_batch_t b);

/* ----- product without any device allocation -----
 * The paper has no counterpart: this is a deployment aid.  hodlr2d_matvec may
 * allocate its working memory on first use (and again when nrhs grows).  Some
 * callers must not allocate device memory while they run -- a serving loop
 * that cannot take the implicit device-wide synchronisation of cudaMalloc /
 * cudaFree, or a host framework that owns the device-memory budget and
 * forbids allocations outside its own pool.  hodlr2d_matvec_noalloc computes
 * the same Alg. 2 product in binary64, within rounding of hodlr2d_matvec's F64
 * mode but not bit for bit: it runs a simpler, slower set of binary64 kernels
 * (near field, per-chunk projections, chunk sums, expansions) whose sums run
 * in another order.  Its working memory is one statically sized device array
 * of HODLR2D_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library
 * holds until the process exits.  It never calls cudaMalloc, cudaFree or any
 * allocating routine.
 *   h:    a handle with factors; its device must be the current device.
 *   x, y: DEVICE pointers only, n x nrhs column-major (host pointers: ARG).
 * The working memory needed is about 8 n nrhs (kappa + 2) bytes plus
 * 8 nrhs (2 x sum of the pair ranks, summed over row chunks) bytes -- for the
 * N = 2^16, leaf 64, eps 1e-8 multiquadric workload about 30 MiB at nrhs = 1.
 * A call that would need more than HODLR2D_NOALLOC_SCRATCH_BYTES returns
 * HODLR2D_ERR_ARG and does nothing.
 * The first call on a device looks up the array's device address (once per
 * device, under a lock); make that first call before any stream capture.
 * The call is asynchronous on the handle's stream.  All calls share the one
 * array: calls whose kernels overlap on the GPU (other streams, handles or
 * threads) race on it and produce wrong results -- serialise them.  Each call
 * writes every scratch word it reads, so leftovers of earlier calls are
 * harmless.  Errors: ARG, STATE, CUDA. */
#define HODLR2D_NOALLOC_SCRATCH_BYTES (32u << 20)
int hodlr2d_matvec_noalloc(hodlr2d_t h, const double* x, double* y, int nrhs);

void hodlr2d_free(hodlr2d_t h);
const char* hodlr2d_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* HODLR2D_H */
