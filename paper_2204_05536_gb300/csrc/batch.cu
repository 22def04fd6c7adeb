// Many independent HODLR2D matrices (point sets of uneven size) multiplied
// as one unit: the products of all sets are recorded once into a CUDA graph
// (sets spread over kLanes forked streams, each set's own near/far streams
// nested inside) and replayed with one graph launch per call.
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
};

using namespace h2d;

static void batch_drop_graph(hodlr2d_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
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
  int rc = HODLR2D_OK;
  for (int j = 0; j < hodlr2d_batch::kLanes && !rc; ++j) {
    if (cudaStreamCreateWithFlags(&b->lanes[j], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join[j], cudaEventDisableTiming) != cudaSuccess)
      rc = HODLR2D_ERR_CUDA;
  }
  if (!rc && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
    rc = HODLR2D_ERR_CUDA;
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
  bool same = b->exec && b->gmode == mode && b->gstream == b->stream;
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
  for (int j = 0; j < hodlr2d_batch::kLanes; ++j) {
    if (b->lanes[j]) cudaStreamDestroy(b->lanes[j]);
    if (b->join[j]) cudaEventDestroy(b->join[j]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

}  // extern "C"
