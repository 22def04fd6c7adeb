// Many independent HODLR2D matrices (point sets of uneven size) multiplied
// as one unit, in one of two forms: the products of all sets recorded once
// into a CUDA graph (sets spread over kLanes forked streams, each set's own
// near/far streams nested inside) and replayed with one graph launch per
// call; or one persistent cooperative kernel over all sets (product.cu),
// itself recorded into a graph.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace h2d {
bool is_device_ptr(const void* p);
int matvec_mode_device(hodlr2d* h, const double* x, double* y, int nrhs, int mode);
}  // namespace h2d

struct hodlr2d_batch {
  int device = 0;
  std::vector<hodlr2d*> sets;
  cudaStream_t stream = 0;  // the caller's stream
  static constexpr int kLanes = 8;
  cudaStream_t lanes[kLanes] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kLanes] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // what the recorded graph was made for
  std::vector<const double*> gx;
  std::vector<double*> gy;
  std::vector<int> gnrhs;
  int gmode = -1;
  cudaStream_t gstream = 0;
  std::vector<uint64_t> ggen;  // the handles' buffer generations
  // persistent form, what its descriptors were made for, and its launch
  // recorded into a graph (when the driver takes a cooperative launch in a
  // capture; else it is launched directly)
  int form = HODLR2D_BATCH_AUTO;
  int auto_form = HODLR2D_BATCH_GRAPH;  // what AUTO runs (hodlr2d_batch_autotune may change it)
  int last_form = -1;
  bool coop = false;  // the device supports cooperative launches
  h2d::BatchPersist bp;
  std::vector<const double*> px;
  std::vector<double*> py;
  std::vector<int> pnrhs;
  std::vector<uint64_t> pgen;
  cudaGraph_t pgraph = nullptr;
  cudaGraphExec_t pexec = nullptr;
  // the last autotuning: (pair_rows, warp_rows, blocks per SM, ms per
  // product) per candidate
  std::vector<int> tune_pair, tune_warp, tune_minb, tune_place;
  std::vector<double> tune_ms;
};

// True when every handle's buffers are those a recording was made for.
static bool gens_match(const std::vector<hodlr2d*>& sets, const std::vector<uint64_t>& g) {
  if (g.size() != sets.size()) return false;
  for (size_t i = 0; i < sets.size(); ++i)
    if (sets[i]->gen != g[i]) return false;
  return true;
}
static std::vector<uint64_t> gens_of(const std::vector<hodlr2d*>& sets) {
  std::vector<uint64_t> g(sets.size());
  for (size_t i = 0; i < sets.size(); ++i) g[i] = sets[i]->gen;
  return g;
}

using namespace h2d;

static void batch_drop_graph(hodlr2d_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}
static void batch_drop_persistent(hodlr2d_batch* b) {
  if (b->pexec) cudaGraphExecDestroy(b->pexec);
  if (b->pgraph) cudaGraphDestroy(b->pgraph);
  b->pexec = nullptr;
  b->pgraph = nullptr;
  batch_persist_free(&b->bp);
  b->px.clear();
}

extern "C" {

int hodlr2d_batch_create(const hodlr2d_t* handles, int count, hodlr2d_batch_t* out) {
  if (!handles || count < 1 || !out) return HODLR2D_ERR_ARG;
  hodlr2d_batch* b = new (std::nothrow) hodlr2d_batch();
  if (!b) return HODLR2D_ERR_OOM;
  cudaGetDevice(&b->device);
  for (int i = 0; i < count; ++i) {
    if (!handles[i] || !handles[i]->has_factors || handles[i]->device != b->device) {
      delete b;
      return HODLR2D_ERR_ARG;
    }
    b->sets.push_back(handles[i]);
  }
  {  // a handle's working memory serves one product at a time: no repeats
    std::vector<hodlr2d*> sorted(b->sets);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
      delete b;
      return HODLR2D_ERR_ARG;
    }
  }
  int rc = HODLR2D_OK;
  for (int j = 0; j < hodlr2d_batch::kLanes && !rc; ++j) {
    if (cudaStreamCreateWithFlags(&b->lanes[j], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join[j], cudaEventDisableTiming) != cudaSuccess)
      rc = HODLR2D_ERR_CUDA;
  }
  if (!rc && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
    rc = HODLR2D_ERR_CUDA;
  int coop = 0;
  if (!rc && cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device) != cudaSuccess)
    rc = HODLR2D_ERR_CUDA;
  b->coop = coop != 0;
  if (rc) {
    (void)cudaGetLastError();
    hodlr2d_batch_free(b);
    return rc;
  }
  *out = b;
  return HODLR2D_OK;
}

int hodlr2d_batch_set_stream(hodlr2d_batch_t b, void* stream) {
  if (!b) return HODLR2D_ERR_ARG;
  b->stream = (cudaStream_t)stream;
  return HODLR2D_OK;
}

int hodlr2d_batch_set_form(hodlr2d_batch_t b, int form) {
  if (!b || form < HODLR2D_BATCH_AUTO || form > HODLR2D_BATCH_PERSISTENT) return HODLR2D_ERR_ARG;
  b->form = form;
  return HODLR2D_OK;
}

int hodlr2d_batch_set_wait_limit(hodlr2d_batch_t b, uint32_t polls) {
  if (!b) return HODLR2D_ERR_ARG;
  if (b->bp.polls != polls) b->px.clear();  // the recorded launch holds the old limit
  b->bp.polls = polls;
  return HODLR2D_OK;
}

int hodlr2d_batch_last_form(hodlr2d_batch_t b) { return b ? b->last_form : -1; }

int hodlr2d_batch_persistent_recorded(hodlr2d_batch_t b) {
  if (!b) return HODLR2D_ERR_ARG;
  if (!b->bp.d_sets) return -1;
  return b->pexec ? 1 : 0;
}

int hodlr2d_batch_check(hodlr2d_batch_t b) {
  if (!b) return HODLR2D_ERR_ARG;
  H2D_CK(cudaStreamSynchronize(b->stream));
  return batch_persist_status(b->bp, b->stream);
}

int hodlr2d_batch_phase_ms(hodlr2d_batch_t b, double* ms) {
  if (!b || !ms) return HODLR2D_ERR_ARG;
  return batch_persist_phase_ms(b->bp, b->stream, ms);
}

// Records the persistent launch into a graph on a private stream; false (and
// no graph) when the capture or instantiation is refused.
static bool batch_record_persistent(hodlr2d_batch* b) {
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  cudaGraph_t g = nullptr;
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    const int rc = batch_persist_launch(b->bp, cs);
    ok = cudaStreamEndCapture(cs, &g) == cudaSuccess && rc == HODLR2D_OK && g;
  }
  if (ok) ok = cudaGraphInstantiate(&b->pexec, g, 0) == cudaSuccess;
  if (!ok) {
    (void)cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    b->pexec = nullptr;
    g = nullptr;
  }
  b->pgraph = g;
  cudaStreamDestroy(cs);
  return ok;
}

// One persistent product of all sets; descriptors (and the recorded launch)
// are rebuilt when the pointers, nrhs, mode or the handles' buffers change.
static int batch_persistent(hodlr2d_batch* b, const double* const* x, double* const* y,
                            const int* nrhs, int mode) {
  const int count = (int)b->sets.size();
  bool same = b->bp.d_sets && b->bp.mode == mode && !b->px.empty() &&
              gens_match(b->sets, b->pgen);
  for (int i = 0; same && i < count; ++i)
    same = b->px[i] == x[i] && b->py[i] == y[i] && b->pnrhs[i] == nrhs[i];
  if (!same) {
    for (hodlr2d* h : b->sets) H2D_CK(cudaStreamSynchronize(h->stream));
    H2D_CK(cudaStreamSynchronize(b->stream));
    batch_drop_persistent(b);
    H2D_TRY(batch_persist_setup(b->sets.data(), count, x, y, nrhs, mode, &b->bp));
    b->px.assign(x, x + count);
    b->py.assign(y, y + count);
    b->pnrhs.assign(nrhs, nrhs + count);
    b->pgen = gens_of(b->sets);
    batch_record_persistent(b);
  }
  if (b->pexec) {
    H2D_CK(cudaGraphLaunch(b->pexec, b->stream));
    return HODLR2D_OK;
  }
  return batch_persist_launch(b->bp, b->stream);
}

int hodlr2d_batch_set_shapes(hodlr2d_batch_t b, int pair_rows, int warp_rows) {
  if (!b || pair_rows < 0 || warp_rows < 0 || warp_rows > 64 || pair_rows > 2048)
    return HODLR2D_ERR_ARG;
  if (b->bp.pair_rows != pair_rows || b->bp.warp_rows != warp_rows) b->px.clear();
  b->bp.pair_rows = pair_rows;
  b->bp.warp_rows = warp_rows;
  return HODLR2D_OK;
}

int hodlr2d_batch_set_blocks_per_sm(hodlr2d_batch_t b, int blocks) {
  if (!b || blocks < 2 || blocks > 4) return HODLR2D_ERR_ARG;
  if (b->bp.minb != blocks) b->px.clear();
  b->bp.minb = blocks;
  return HODLR2D_OK;
}

int hodlr2d_batch_set_placement(hodlr2d_batch_t b, int place) {
  if (!b || place < 0 || place > 3) return HODLR2D_ERR_ARG;
  if (b->bp.place != place) b->px.clear();
  b->bp.place = place;
  return HODLR2D_OK;
}

int hodlr2d_batch_get_shapes(hodlr2d_batch_t b, int* pair_rows, int* warp_rows) {
  if (!b || !pair_rows || !warp_rows) return HODLR2D_ERR_ARG;
  *pair_rows = b->bp.pair_rows;
  *warp_rows = b->bp.warp_rows;
  return HODLR2D_OK;
}

// Times reps products with the current settings (after one untimed product
// that also sets up); ms per product.
static int batch_time(hodlr2d_batch* b, const double* const* x, double* const* y,
                      const int* nrhs, int mode, int reps, cudaEvent_t e0, cudaEvent_t e1,
                      float* ms) {
  H2D_TRY(hodlr2d_batch_matvec(b, x, y, nrhs, mode));
  H2D_TRY(hodlr2d_batch_check(b));
  H2D_CK(cudaEventRecord(e0, b->stream));
  for (int r = 0; r < reps; ++r) H2D_TRY(hodlr2d_batch_matvec(b, x, y, nrhs, mode));
  H2D_CK(cudaEventRecord(e1, b->stream));
  H2D_TRY(hodlr2d_batch_check(b));
  H2D_CK(cudaEventElapsedTime(ms, e0, e1));
  *ms /= reps;
  b->tune_pair.push_back(b->bp.pair_rows);
  b->tune_warp.push_back(b->bp.warp_rows);
  b->tune_minb.push_back(b->bp.minb);
  b->tune_place.push_back(b->bp.place);
  b->tune_ms.push_back(*ms);
  return HODLR2D_OK;
}

int hodlr2d_batch_autotune(hodlr2d_batch_t b, const double* const* x, double* const* y,
                           const int* nrhs, int mode, int reps, double* best_ms) {
  if (!b || !x || !y || !nrhs || reps < 1) return HODLR2D_ERR_ARG;
  if ((mode != HODLR2D_MODE_F64 && mode != HODLR2D_MODE_F32) || !b->coop) return HODLR2D_ERR_ARG;
  static const int kPair[] = {0, 128, 256, 512, 1024, 2048};
  static const int kWarp[] = {0, 48, 64};
  const int form = b->form;
  b->form = HODLR2D_BATCH_PERSISTENT;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = HODLR2D_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    rc = HODLR2D_ERR_CUDA;
  b->tune_pair.clear();
  b->tune_warp.clear();
  b->tune_minb.clear();
  b->tune_place.clear();
  b->tune_ms.clear();
  float best = -1.f, ms = 0.f;
  int bpr = b->bp.pair_rows, bwr = b->bp.warp_rows, bmb = b->bp.minb, bpl = b->bp.place;
  // shapes at the current occupancy and placement, then the occupancy at the
  // best shapes, then the placement
  for (int pr : kPair)
    for (int wr : kWarp) {
      if (rc || wr > pr) continue;
      rc = hodlr2d_batch_set_shapes(b, pr, wr);
      if (!rc) rc = batch_time(b, x, y, nrhs, mode, reps, e0, e1, &ms);
      if (!rc && (best < 0.f || ms < best)) {
        best = ms;
        bpr = pr;
        bwr = wr;
      }
    }
  if (!rc) rc = hodlr2d_batch_set_shapes(b, bpr, bwr);
  const int mb0 = bmb;
  for (int mb = 2; mb <= 4 && !rc; ++mb) {
    if (mb == mb0) continue;
    rc = hodlr2d_batch_set_blocks_per_sm(b, mb);
    if (!rc) rc = batch_time(b, x, y, nrhs, mode, reps, e0, e1, &ms);
    if (!rc && ms < best) {
      best = ms;
      bmb = mb;
    }
  }
  if (!rc) rc = hodlr2d_batch_set_blocks_per_sm(b, bmb);
  const int pl0 = bpl;
  for (int pl = 0; pl <= 3 && !rc; ++pl) {
    if (pl == pl0) continue;
    rc = hodlr2d_batch_set_placement(b, pl);
    if (!rc) rc = batch_time(b, x, y, nrhs, mode, reps, e0, e1, &ms);
    if (!rc && ms < best) {
      best = ms;
      bpl = pl;
    }
  }
  if (!rc) rc = hodlr2d_batch_set_placement(b, bpl);
  // the graph form on the same inputs decides what AUTO runs
  float gms = 0.f;
  if (!rc) {
    b->form = HODLR2D_BATCH_GRAPH;
    rc = batch_time(b, x, y, nrhs, mode, reps, e0, e1, &gms);
    if (!rc) {
      b->tune_pair.back() = b->tune_warp.back() = b->tune_minb.back() = b->tune_place.back() = -1;
      b->auto_form = gms < best ? HODLR2D_BATCH_GRAPH : HODLR2D_BATCH_PERSISTENT;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  b->form = form;
  if (rc) return rc;
  if (best_ms) *best_ms = best;
  return HODLR2D_OK;
}

int hodlr2d_batch_tune_table(hodlr2d_batch_t b, int* count, int* pair_rows, int* warp_rows,
                             int* blocks, int* place, double* ms) {
  if (!b || !count) return HODLR2D_ERR_ARG;
  const int n = (int)b->tune_ms.size();
  if (pair_rows && warp_rows && blocks && place && ms)
    for (int i = 0; i < std::min(n, *count); ++i) {
      pair_rows[i] = b->tune_pair[i];
      warp_rows[i] = b->tune_warp[i];
      blocks[i] = b->tune_minb[i];
      place[i] = b->tune_place[i];
      ms[i] = b->tune_ms[i];
    }
  *count = n;
  return HODLR2D_OK;
}

int hodlr2d_batch_matvec(hodlr2d_batch_t b, const double* const* x, double* const* y,
                         const int* nrhs, int mode) {
  if (!b || !x || !y || !nrhs || mode < 0 || mode > 3) return HODLR2D_ERR_ARG;
  const int count = (int)b->sets.size();
  for (int i = 0; i < count; ++i) {
    hodlr2d* h = b->sets[i];
    if (!x[i] || !y[i] || nrhs[i] < 1 || !is_device_ptr(x[i]) || !is_device_ptr(y[i]))
      return HODLR2D_ERR_ARG;
    if (!h->prepared[mode]) return HODLR2D_ERR_STATE;
    if (h->prof_on) return HODLR2D_ERR_STATE;  // event timing cannot be recorded
  }
  const bool mode_ok = mode == HODLR2D_MODE_F64 || mode == HODLR2D_MODE_F32;
  if (b->form == HODLR2D_BATCH_PERSISTENT && (!mode_ok || !b->coop)) return HODLR2D_ERR_ARG;
  const bool pers = b->form == HODLR2D_BATCH_PERSISTENT ||
                    (b->form == HODLR2D_BATCH_AUTO && b->auto_form == HODLR2D_BATCH_PERSISTENT &&
                     mode_ok && b->coop);
  if (pers) {
    H2D_TRY(batch_persistent(b, x, y, nrhs, mode));
    b->last_form = HODLR2D_BATCH_PERSISTENT;
    return HODLR2D_OK;
  }
  b->last_form = HODLR2D_BATCH_GRAPH;
  bool same = b->exec && b->gmode == mode && b->gstream == b->stream &&
              gens_match(b->sets, b->ggen);
  for (int i = 0; same && i < count; ++i)
    same = b->gx[i] == x[i] && b->gy[i] == y[i] && b->gnrhs[i] == nrhs[i];
  if (!same) {
    batch_drop_graph(b);
    std::vector<cudaStream_t> saved(count);
    for (int i = 0; i < count; ++i) saved[i] = b->sets[i]->stream;
    struct Restore {  // the handles keep their own streams afterwards
      std::vector<hodlr2d*>& s;
      std::vector<cudaStream_t>& v;
      ~Restore() {
        for (size_t i = 0; i < s.size(); ++i) s[i]->stream = v[i];
      }
    } restore{b->sets, saved};
    // one ordinary pass first: plans and scratch are allocated outside capture
    for (int i = 0; i < count; ++i) {
      hodlr2d* h = b->sets[i];
      h->stream = b->lanes[i % hodlr2d_batch::kLanes];
      H2D_TRY(matvec_mode_device(h, x[i], y[i], nrhs[i], mode));
    }
    for (int j = 0; j < hodlr2d_batch::kLanes; ++j) H2D_CK(cudaStreamSynchronize(b->lanes[j]));
    // record: fork the lanes off the caller's stream, join them back
    cudaStream_t cs = b->stream;
    cudaStream_t cap = nullptr;
    if (!cs) {  // the legacy default stream cannot be captured: use a private one
      H2D_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      cs = cap;
    }
    int rc = HODLR2D_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      rc = HODLR2D_ERR_CUDA;
    if (!rc && cudaEventRecord(b->fork, cs) != cudaSuccess) rc = HODLR2D_ERR_CUDA;
    for (int j = 0; j < hodlr2d_batch::kLanes && !rc; ++j)
      if (cudaStreamWaitEvent(b->lanes[j], b->fork, 0) != cudaSuccess) rc = HODLR2D_ERR_CUDA;
    for (int i = 0; i < count && !rc; ++i)
      rc = matvec_mode_device(b->sets[i], x[i], y[i], nrhs[i], mode);
    for (int j = 0; j < hodlr2d_batch::kLanes && !rc; ++j) {
      if (cudaEventRecord(b->join[j], b->lanes[j]) != cudaSuccess ||
          cudaStreamWaitEvent(cs, b->join[j], 0) != cudaSuccess)
        rc = HODLR2D_ERR_CUDA;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (!rc && e != cudaSuccess) rc = HODLR2D_ERR_CUDA;
    if (!rc && cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) rc = HODLR2D_ERR_CUDA;
    if (rc) {
      (void)cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      if (cap) cudaStreamDestroy(cap);
      b->exec = nullptr;
      return rc;
    }
    b->graph = g;
    b->gx.assign(x, x + count);
    b->gy.assign(y, y + count);
    b->gnrhs.assign(nrhs, nrhs + count);
    b->gmode = mode;
    b->gstream = b->stream;
    b->ggen = gens_of(b->sets);
    if (cap) {  // replay on the legacy stream, then drop the private one
      H2D_CK(cudaStreamSynchronize(cap));
      cudaStreamDestroy(cap);
    }
  }
  H2D_CK(cudaGraphLaunch(b->exec, b->stream));
  return HODLR2D_OK;
}

void hodlr2d_batch_free(hodlr2d_batch_t b) {
  if (!b) return;
  batch_drop_graph(b);
  batch_drop_persistent(b);
  for (int j = 0; j < hodlr2d_batch::kLanes; ++j) {
    if (b->lanes[j]) cudaStreamDestroy(b->lanes[j]);
    if (b->join[j]) cudaEventDestroy(b->join[j]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

}  // extern "C"
