// Internal handle layout shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "arith.cuh"
#include "common.cuh"

namespace h2d {

__host__ __device__ __forceinline__ int64_t ldpad(int64_t r) { return r + (r & 1); }

// One row box of a box-mode level: its row pairs are meta[p0 .. p0 + np).
struct BoxWork {
  int64_t p0;
  int32_t level, np, xs, m;
};

// Everything a product kernel needs about one stored pair, in one record.
struct PairMeta {
  int64_t foff;   // first value of U (V follows at foff + ldpad(m) k)
  int64_t ppx;    // partial-result offset of the X rows (pair mode)
  int64_t ppy;    // partial-result offset of the Y rows
  int32_t k, xs, m, ys, n, pad;
};

// One unit of the expansion pass: rows [r0, r0 + nr) of one box.
struct ExpTask {
  int32_t level;
  int32_t box;
  int32_t r0, nr;
};

// Stored factors of one level: pairs sorted by (row box, column box) in
// Morton order.  Columns are padded to an even length ld(r) = r + (r & 1)
// (pad entries are zero) so that every column starts on a 16-byte boundary:
// pair p's U (|X| x k, column-major, leading dimension ld(|X|)) starts at
// foff[p] and its V (|Y| x k, leading dimension ld(|Y|)) at
// foff[p] + ld(|X|) k.
struct Level {
  int l = 0;
  int64_t npairs = 0;
  int32_t* d_px = nullptr;       // row box (Morton id at level l)
  int32_t* d_py = nullptr;       // column box
  int32_t* d_rank = nullptr;     // k per pair
  int64_t* d_foff = nullptr;     // npairs + 1 value offsets
  int64_t* d_toff = nullptr;     // npairs + 1 offsets into the projection buffer
  double* d_fac = nullptr;       // F64 factor values
  void* d_fac_mode[4] = {nullptr, nullptr, nullptr, nullptr};  // per hodlr2d_mode copy
  int64_t nvalues = 0;   // allocated values, padding included
  int64_t nstored = 0;   // sum (|X| + |Y|) k: the values the method stores
  int max_rank = 0;
  int64_t* d_prow = nullptr;   // 4^l + 1: first stored pair of each row box
  int64_t* d_ppoff = nullptr;  // npairs + 1: partial-result offsets (|Y| per pair)
  PairMeta* d_meta = nullptr;  // npairs: per-pair records for the product
  int64_t npart = 0;
  // per box: entries (pair * 2 + side) of its interaction list, ascending
  // partner; side 0 = the box is the row side (applies U), 1 = column (V)
  int32_t* d_ent_off = nullptr;  // 4^l + 1
  int32_t* d_ent = nullptr;
  int64_t nent = 0;
  int64_t* d_entpp = nullptr;  // per entry: partial offset << 1 | side (pair-planned levels)
  std::vector<int32_t> h_rank;   // host copy of the ranks
  std::vector<int64_t> h_foff;
};

// One unit of the projection pass: rows [r0, r0 + nr) of one factor matrix.
struct ProjTask {
  int32_t level;
  int32_t side;   // 0: V of the pair against x_Y -> t1 ; 1: U against x_X -> t2
  int64_t pair;
  int32_t r0, nr;
  int64_t out;    // offset of its k partial sums (per right-hand side)
  int64_t mat;    // first value of the matrix (U or V) in the level's factors
  int32_t ld;     // its (padded) column length
  int32_t base;   // tree position of its first row
  int32_t k;
  int32_t pad;
};

// Plan and scratch of the second-generation product (product.cu).
// Pair-mode work of one level: (level, pair) of every stored pair of rank > 0,
// sorted into size classes by max(|X|, |Y|) (bounds kPairClassRows), so that
// each class runs with a block shape fitted to its boxes.
constexpr int kPairClasses = 11;
constexpr int kPairClassRows[kPairClasses] = {16,  32,   48,   64,   128, 256,
                                              384, 1280, 2560, 4608, 1 << 30};
struct PairLevel {
  int2* d_work = nullptr;              // all classes, class by class
  int64_t nwork = 0;
  int max_rows = 0;                    // largest box of the level
  int64_t off[kPairClasses + 1] = {};  // class c: work [off[c], off[c + 1])
  int cls_rows[kPairClasses] = {};     // largest box of class c
  std::vector<int2> h_work;            // host copy of the work list
};

struct V2Plan {
  bool ready = false;
  int lfuse = 1;   // first single-read level
  int ldual = 1;   // first two-pass level that also has a pair plan (<= lfuse)
  int l2max = 1;   // two-pass plans exist for levels [1, l2max) (>= lfuse)
  int l2few = 1;   // first level of boxes <= 1024 points (>= lfuse): few-RHS pair levels
  // two-pass task counts of the levels below l (level-ordered list prefixes)
  int64_t pre_proj[HODLR2D_MAX_LEVELS + 1] = {}, pre_exp[HODLR2D_MAX_LEVELS + 1] = {};
  int64_t pre_part[HODLR2D_MAX_LEVELS + 1] = {}, pre_tsum[HODLR2D_MAX_LEVELS + 1] = {};
  ProjTask* d_proj = nullptr;
  ExpTask* d_exp = nullptr;
  int64_t* d_red = nullptr;
  int64_t nproj = 0, nexp = 0, proj_partials = 0, nsides = 0, ntsum = 0;
  // binary64 projection work (task, first column) per column group, and the
  // groups of the tasks below each level
  int2* d_pgrp = nullptr;
  int64_t pre_pgrp[HODLR2D_MAX_LEVELS + 1] = {};
  int32_t* d_wtask = nullptr;  // task of each projection warp
  int64_t* d_sideq = nullptr;  // (pair side, column) of each chunk-sum warp
  int lmode[HODLR2D_MAX_LEVELS] = {};  // per level: base mode (two-pass, pair or box)
  int lpair_small = 1 << 20;           // first pair level of boxes <= 256 points (profiling)
  BoxWork* d_bw = nullptr;     // box-mode work, boxes <= 64 points
  int64_t nbw = 0;
  int nsm = 1;  // streaming multiprocessors of the device
  int2* d_nearw = nullptr;     // near-field work: (leaf, first target), <= 32 targets
  int64_t nnearw = 0;
  int64_t near_entries = 0;    // dense leaf entries of one product
  int* d_status = nullptr;     // set by a product kernel whose bounded wait gave up
  // tensor-core projection groups (tasks sharing a box and row chunk): task
  // order, {first, tasks, rows, level} per group, groups below each level
  int32_t* d_gtask = nullptr;
  int4* d_grp = nullptr;
  int64_t pre_grp[HODLR2D_MAX_LEVELS + 1] = {};
  bool grp_ok = true;  // every task fits one group
  int two_levels = 0;  // the two-pass plan covers levels [1, two_levels)
  bool zero_partials = false;
  int64_t pstride = 1;
  int32_t* d_leaf_of = nullptr;
  int scratch_nrhs = 0;
  void* d_xt = nullptr;
  void* d_yl = nullptr;
  void* d_ppart = nullptr;
  void* d_part = nullptr;
  void* d_t = nullptr;
  void* d_xf = nullptr;  // float-float coordinates (DF32)
  void* d_yf = nullptr;
  KernelFF kff{};
  void* d_x32 = nullptr;  // binary32 coordinates (F32 / BF16 modes)
  void* d_y32 = nullptr;
  KernelF32 kf32{};
  PairLevel plev[HODLR2D_MAX_LEVELS];
  // side streams: near field, and the single-read far-field levels
  cudaStream_t s_near = nullptr, s_far = nullptr;
  cudaEvent_t ev_in = nullptr, ev_near = nullptr, ev_far = nullptr;
};

// A persistent batch product (product.cu): device descriptors of the sets,
// the unit descriptors of the five phases, the pair items, the barrier words.
struct BatchPersist {
  void* d_sets = nullptr;
  int64_t* d_pre = nullptr;   // the six phase offsets into d_tab
  uint64_t* d_tab = nullptr;  // unit descriptors
  void* d_sync = nullptr;
  void* d_work = nullptr;
  int count = 0, mode = -1, grid = 0;
  uint32_t polls = 1u << 22;  // polls of a barrier wait before it gives up
  // shapes by size class: levels whose boxes hold at most pair_rows points
  // run as pairs (one pair per 256-thread unit, or per warp for pairs of at
  // most warp_rows points); coarser levels run in two passes
  int pair_rows = 384, warp_rows = 64;
  int minb = 3;  // resident blocks per SM (2, 3 or 4: 128, 80 or 64 registers a thread)
  int place = 0;  // bit 0: near field beside the expansions; bit 1: warp pairs beside chunk sums
};
int batch_persist_setup(hodlr2d* const* hs, int count, const double* const* x, double* const* y,
                        const int* nrhs, int mode, BatchPersist* bp);
int batch_persist_launch(const BatchPersist& bp, cudaStream_t s);
int batch_persist_status(const BatchPersist& bp, cudaStream_t s);
int batch_persist_phase_ms(const BatchPersist& bp, cudaStream_t s, double* ms);
void batch_persist_free(BatchPersist* bp);

}  // namespace h2d

struct hodlr2d {
  int device = 0;
  cudaStream_t stream = 0;
  int64_t n = 0;
  hodlr2d_kernel kern{};
  h2d::KernelParams kp{};
  int leaf_size = 0;
  double eps = 0;
  hodlr2d_opts opts{};
  int kappa = 0;
  double root[3] = {0, 0, 0};

  // tree (device)
  double* d_x = nullptr;      // coordinates in tree order
  double* d_y = nullptr;
  int64_t* d_perm = nullptr;  // tree position -> original index
  int32_t* d_leaf_off = nullptr;  // 4^kappa + 1 leaf offsets (Morton order)
  std::vector<int32_t> h_leaf_off;

  h2d::Level lev[HODLR2D_MAX_LEVELS];
  h2d::V2Plan v2;
  bool has_factors = false;
  bool prepared[4] = {true, false, false, false};
  bool f64_released = false;  // hodlr2d_release dropped the binary64 factors
  // bumped whenever device buffers a recorded batch product points to may
  // have moved (plans, scratch, factor copies)
  uint64_t gen = 0;

  // matvec plan
  int64_t nproj = 0, nexp = 0;
  h2d::ProjTask* d_proj = nullptr;
  h2d::ExpTask* d_exp = nullptr;
  int64_t proj_partials = 0;   // sum of k over projection tasks
  int64_t t_total = 0;         // sum of 2 k over pairs
  int64_t* d_tred = nullptr;   // per (pair, side): first task and task count
  int64_t nt_sides = 0;

  // matvec scratch, sized for scratch_nrhs right-hand sides
  int scratch_nrhs = 0;
  double* d_xt = nullptr;      // n x nrhs, tree order
  double* d_yl = nullptr;      // (kappa + 1) x n x nrhs, per-level results
  double* d_part = nullptr;    // proj_partials x nrhs
  double* d_t = nullptr;       // t_total x nrhs
  double* d_io = nullptr;      // staging for host x / y (n x nrhs each)
  int io_nrhs = 0;
  double* d_gm = nullptr;      // GMRES workspace (Krylov basis and vectors)
  int64_t gm_values = 0;

  hodlr2d_stats st{};

  // tracing (hodlr2d_profile)
  struct ProfRec {
    int phase;
    cudaEvent_t a, b;
  };
  bool prof_on = false;
  std::vector<ProfRec> prof;
  double prof_ms[HODLR2D_NPHASE] = {};
  int64_t prof_launches[HODLR2D_NPHASE] = {};
  int64_t prof_bytes[HODLR2D_NPHASE] = {};
  int64_t prof_flops[HODLR2D_NPHASE] = {};
};

namespace h2d {
// Brackets the launches of one phase with events while profiling is on.
struct PhaseScope {
  hodlr2d* h;
  int phase;
  int nlaunch;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t st;
  PhaseScope(hodlr2d* h_, int phase_, int nlaunch_, int64_t bytes, cudaStream_t s_)
      : h(h_), phase(phase_), nlaunch(nlaunch_), st(s_) {
    if (!h->prof_on) return;
    h->prof_bytes[phase] += bytes;
    if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
      cudaEventRecord(a, st);
  }
  PhaseScope(hodlr2d* h_, int phase_, int nlaunch_, int64_t bytes)
      : PhaseScope(h_, phase_, nlaunch_, bytes, h_->stream) {}
  // algorithmic floating-point operations of the phase's launches
  void flops(int64_t f) {
    if (h->prof_on) h->prof_flops[phase] += f;
  }
  ~PhaseScope() {
    if (!h->prof_on || !a || !b) return;
    cudaEventRecord(b, st);
    h->prof.push_back({phase, a, b});
    h->prof_launches[phase] += nlaunch;
  }
};
}  // namespace h2d
