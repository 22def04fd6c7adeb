// Rank predictor: an 8 -> H -> H -> 1 ReLU network that maps the geometry
// of an admissible block to log2(rank + 1) of its ACA factorisation, trained
// on the GPU by the kernels below (forward, backward, Adam), all binary32.
//
//   h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), y = h2 . w3 + b3,
//   loss = (1/B) sum (y - t)^2.
// Parameters are one flat vector: W1 (8 x H, row-major), b1, W2 (H x H,
// row-major), b2, w3, b3.  Every reduction over the batch is a fixed-order
// block tree, so training is bitwise reproducible.
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"

struct hodlr2d_rank_model {
  int device = 0;
  int H = 64;
  int64_t np = 0;
  float* d_theta = nullptr;
  float* d_grad = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  int64_t step = 0;
  // activations of the largest batch seen
  int64_t cap = 0;
  float *d_x = nullptr, *d_t = nullptr, *d_z1 = nullptr, *d_z2 = nullptr, *d_y = nullptr;
  float *d_dz2 = nullptr, *d_dz1 = nullptr, *d_loss = nullptr;
};

namespace h2d {

bool is_device_ptr(const void* p);
constexpr int kNF = 8;

static int64_t mlp_nparams(int H) { return (int64_t)kNF * H + H + (int64_t)H * H + H + H + 1; }

struct MlpView {
  const float* W1;
  const float* b1;
  const float* W2;
  const float* b2;
  const float* w3;
  const float* b3;
  int H;
};
static MlpView mlp_view(const float* th, int H) {
  MlpView v;
  v.W1 = th;
  v.b1 = v.W1 + kNF * H;
  v.W2 = v.b1 + H;
  v.b2 = v.W2 + (int64_t)H * H;
  v.w3 = v.b2 + H;
  v.b3 = v.w3 + H;
  v.H = H;
  return v;
}

// z1 = x W1 + b1 (one thread per sample and unit)
__global__ void k_mlp_l1(MlpView w, const float* __restrict__ x, int64_t B, float* __restrict__ z1) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= B * w.H) return;
  const int64_t s = g / w.H;
  const int j = (int)(g - s * w.H);
  float a = w.b1[j];
  for (int f = 0; f < kNF; ++f) a = __fmaf_rn(x[s * kNF + f], w.W1[f * w.H + j], a);
  z1[g] = a;
}

// z2 = relu(z1) W2 + b2
__global__ void k_mlp_l2(MlpView w, const float* __restrict__ z1, int64_t B, float* __restrict__ z2) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= B * w.H) return;
  const int64_t s = g / w.H;
  const int j = (int)(g - s * w.H);
  float a = w.b2[j];
  const float* h1 = z1 + s * w.H;
  for (int i = 0; i < w.H; ++i) a = __fmaf_rn(fmaxf(h1[i], 0.f), w.W2[i * w.H + j], a);
  z2[g] = a;
}

// y = relu(z2) . w3 + b3; with targets: dy = 2 (y - t) / B and squared error
__global__ void k_mlp_l3(MlpView w, const float* __restrict__ z2, int64_t B, float* __restrict__ y,
                         const float* __restrict__ t, float* __restrict__ dy,
                         float* __restrict__ sqerr) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= B) return;
  float a = w.b3[0];
  const float* h2 = z2 + s * w.H;
  for (int i = 0; i < w.H; ++i) a = __fmaf_rn(fmaxf(h2[i], 0.f), w.w3[i], a);
  y[s] = a;
  if (t) {
    const float r = a - t[s];
    dy[s] = 2.0f * r / (float)B;
    sqerr[s] = r * r;
  }
}

// dz2[s, j] = dy[s] w3[j] [z2 > 0]
__global__ void k_mlp_bz2(MlpView w, const float* __restrict__ dy, const float* __restrict__ z2,
                          int64_t B, float* __restrict__ dz2) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= B * w.H) return;
  const int64_t s = g / w.H;
  const int j = (int)(g - s * w.H);
  dz2[g] = z2[g] > 0.f ? dy[s] * w.w3[j] : 0.f;
}

// dz1[s, i] = (sum_j dz2[s, j] W2[i, j]) [z1 > 0]
__global__ void k_mlp_bz1(MlpView w, const float* __restrict__ dz2, const float* __restrict__ z1,
                          int64_t B, float* __restrict__ dz1) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= B * w.H) return;
  const int64_t s = g / w.H;
  const int i = (int)(g - s * w.H);
  float a = 0.f;
  const float* d = dz2 + s * w.H;
  for (int j = 0; j < w.H; ++j) a = __fmaf_rn(d[j], w.W2[i * w.H + j], a);
  dz1[g] = z1[g] > 0.f ? a : 0.f;
}

// out[o] = sum_s L(s, o / C) R(s, o % C) in a fixed order: one block per
// output, thread strides over the batch, then a shared-memory tree.
// L(s, i) = Lm[s * ldl + i] (relu'd if lrelu; 1 if Lm is null),
// R(s, j) = Rm[s * ldr + j] (relu'd if rrelu).
constexpr int kRedThreads = 256;
__global__ void __launch_bounds__(kRedThreads)
    k_mlp_outer(const float* __restrict__ Lm, int ldl, int lrelu, const float* __restrict__ Rm,
                int ldr, int rrelu, int C, int64_t B, float* __restrict__ out) {
  __shared__ float red[kRedThreads];
  const int o = blockIdx.x;
  const int i = o / C, j = o - i * C;
  float a = 0.f;
  for (int64_t s = threadIdx.x; s < B; s += kRedThreads) {
    float lv = Lm ? Lm[s * ldl + i] : 1.f;
    if (lrelu) lv = fmaxf(lv, 0.f);
    float rv = Rm[s * ldr + j];
    if (rrelu) rv = fmaxf(rv, 0.f);
    a = __fmaf_rn(lv, rv, a);
  }
  red[threadIdx.x] = a;
  __syncthreads();
  for (int st = kRedThreads / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[o] = red[0];
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float c1,
                       float c2, float eps) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

static int mlp_reserve(hodlr2d_rank_model* M, int64_t B) {
  if (M->cap >= B) return HODLR2D_OK;
  float** bufs[] = {&M->d_x, &M->d_t, &M->d_z1, &M->d_z2, &M->d_y, &M->d_dz2, &M->d_dz1, &M->d_loss};
  for (auto b : bufs) {
    cudaFree(*b);
    *b = nullptr;
  }
  M->cap = 0;
  const int64_t H = M->H;
  H2D_CK(cudaMalloc(&M->d_x, 4 * B * kNF));
  H2D_CK(cudaMalloc(&M->d_t, 4 * B));
  H2D_CK(cudaMalloc(&M->d_z1, 4 * B * H));
  H2D_CK(cudaMalloc(&M->d_z2, 4 * B * H));
  H2D_CK(cudaMalloc(&M->d_y, 4 * B));
  H2D_CK(cudaMalloc(&M->d_dz2, 4 * B * H));
  H2D_CK(cudaMalloc(&M->d_dz1, 4 * B * H));
  H2D_CK(cudaMalloc(&M->d_loss, 4 * (B + 1)));
  M->cap = B;
  return HODLR2D_OK;
}

// forward on the device copy d_x (B samples); with targets also the loss
// gradient into d_grad and the per-sample squared errors into d_loss
static int mlp_forward_backward(hodlr2d_rank_model* M, int64_t B, bool grad, cudaStream_t s) {
  const MlpView w = mlp_view(M->d_theta, M->H);
  const int H = M->H;
  const unsigned gbh = (unsigned)((B * H + 255) / 256), gb = (unsigned)((B + 255) / 256);
  k_mlp_l1<<<gbh, 256, 0, s>>>(w, M->d_x, B, M->d_z1);
  k_mlp_l2<<<gbh, 256, 0, s>>>(w, M->d_z1, B, M->d_z2);
  k_mlp_l3<<<gb, 256, 0, s>>>(w, M->d_z2, B, M->d_y, grad ? M->d_t : nullptr, M->d_dz2 /*dy*/,
                              M->d_loss);
  if (!grad) return cudaGetLastError() == cudaSuccess ? HODLR2D_OK : HODLR2D_ERR_CUDA;
  // dy lives in d_dz2[0 .. B); keep it in d_y's place before dz2 overwrites it
  H2D_CK(cudaMemcpyAsync(M->d_t, M->d_dz2, 4 * B, cudaMemcpyDeviceToDevice, s));
  const float* dy = M->d_t;
  float* g = M->d_grad;
  float* gW1 = g;
  float* gb1 = gW1 + kNF * H;
  float* gW2 = gb1 + H;
  float* gb2 = gW2 + (int64_t)H * H;
  float* gw3 = gb2 + H;
  float* gb3 = gw3 + H;
  // output layer: dw3 = relu(z2)^T dy, db3 = sum dy
  k_mlp_outer<<<H, kRedThreads, 0, s>>>(dy, 1, 0, M->d_z2, H, 1, H, B, gw3);
  k_mlp_outer<<<1, kRedThreads, 0, s>>>(nullptr, 0, 0, dy, 1, 0, 1, B, gb3);
  k_mlp_bz2<<<gbh, 256, 0, s>>>(w, dy, M->d_z2, B, M->d_dz2);
  // hidden layer 2: dW2 = relu(z1)^T dz2, db2 = sum dz2
  k_mlp_outer<<<H * H, kRedThreads, 0, s>>>(M->d_z1, H, 1, M->d_dz2, H, 0, H, B, gW2);
  k_mlp_outer<<<H, kRedThreads, 0, s>>>(nullptr, 0, 0, M->d_dz2, H, 0, H, B, gb2);
  k_mlp_bz1<<<gbh, 256, 0, s>>>(w, M->d_dz2, M->d_z1, B, M->d_dz1);
  // hidden layer 1: dW1 = x^T dz1, db1 = sum dz1
  k_mlp_outer<<<kNF * H, kRedThreads, 0, s>>>(M->d_x, kNF, 0, M->d_dz1, H, 0, H, B, gW1);
  k_mlp_outer<<<H, kRedThreads, 0, s>>>(nullptr, 0, 0, M->d_dz1, H, 0, H, B, gb1);
  H2D_CK(cudaGetLastError());
  return HODLR2D_OK;
}

static int copy_in(float* dst, const float* src, int64_t count, cudaStream_t s) {
  const cudaMemcpyKind kind = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  H2D_CK(cudaMemcpyAsync(dst, src, 4 * count, kind, s));
  return HODLR2D_OK;
}

// log2(rank + 1) predictions for n feature rows (device output)
int mlp_predict_device(hodlr2d_rank_model* M, const float* d_feats, int64_t n, float* d_out,
                       cudaStream_t s) {
  const int64_t chunk = 1 << 16;
  for (int64_t o = 0; o < n; o += chunk) {
    const int64_t b = std::min(chunk, n - o);
    H2D_TRY(mlp_reserve(M, b));
    H2D_CK(cudaMemcpyAsync(M->d_x, d_feats + o * kNF, 4 * b * kNF, cudaMemcpyDeviceToDevice, s));
    H2D_TRY(mlp_forward_backward(M, b, false, s));
    H2D_CK(cudaMemcpyAsync(d_out + o, M->d_y, 4 * b, cudaMemcpyDeviceToDevice, s));
  }
  return HODLR2D_OK;
}

}  // namespace h2d

using namespace h2d;

extern "C" {

int hodlr2d_rank_model_create(int hidden, const float* params, hodlr2d_rank_model_t* out) {
  if (!out || hidden < 1 || hidden > 1024) return HODLR2D_ERR_ARG;
  hodlr2d_rank_model* M = new (std::nothrow) hodlr2d_rank_model();
  if (!M) return HODLR2D_ERR_OOM;
  cudaGetDevice(&M->device);
  M->H = hidden;
  M->np = mlp_nparams(hidden);
  if (cudaMalloc(&M->d_theta, 4 * M->np) != cudaSuccess ||
      cudaMalloc(&M->d_grad, 4 * M->np) != cudaSuccess ||
      cudaMalloc(&M->d_m, 4 * M->np) != cudaSuccess ||
      cudaMalloc(&M->d_v, 4 * M->np) != cudaSuccess) {
    (void)cudaGetLastError();
    hodlr2d_rank_model_free(M);
    return HODLR2D_ERR_OOM;
  }
  cudaMemset(M->d_m, 0, 4 * M->np);
  cudaMemset(M->d_v, 0, 4 * M->np);
  cudaMemset(M->d_grad, 0, 4 * M->np);
  int rc = params ? copy_in(M->d_theta, params, M->np, 0)
                  : (cudaMemset(M->d_theta, 0, 4 * M->np) == cudaSuccess ? HODLR2D_OK
                                                                         : HODLR2D_ERR_CUDA);
  if (rc == HODLR2D_OK && cudaDeviceSynchronize() != cudaSuccess) rc = HODLR2D_ERR_CUDA;
  if (rc) {
    hodlr2d_rank_model_free(M);
    return rc;
  }
  *out = M;
  return HODLR2D_OK;
}

int hodlr2d_rank_model_params(hodlr2d_rank_model_t M, float* params, int64_t* nparams) {
  if (!M || !nparams) return HODLR2D_ERR_ARG;
  *nparams = M->np;
  if (!params) return HODLR2D_OK;
  H2D_CK(cudaMemcpy(params, M->d_theta, 4 * M->np, cudaMemcpyDeviceToHost));
  return HODLR2D_OK;
}

int hodlr2d_rank_model_loss_grad(hodlr2d_rank_model_t M, const float* feats, const float* targets,
                                 int64_t n, float* loss, float* grad) {
  if (!M || !feats || !targets || n < 1) return HODLR2D_ERR_ARG;
  H2D_TRY(mlp_reserve(M, n));
  H2D_TRY(copy_in(M->d_x, feats, n * kNF, 0));
  H2D_TRY(copy_in(M->d_t, targets, n, 0));
  H2D_TRY(mlp_forward_backward(M, n, true, 0));
  if (loss) {  // fixed-order sum of the squared errors, divided by n
    float* d_sum = M->d_loss + n;
    k_mlp_outer<<<1, kRedThreads>>>(nullptr, 0, 0, M->d_loss, 1, 0, 1, n, d_sum);
    float sum = 0.f;
    H2D_CK(cudaMemcpy(&sum, d_sum, 4, cudaMemcpyDeviceToHost));
    *loss = sum / (float)n;
  }
  if (grad) H2D_CK(cudaMemcpy(grad, M->d_grad, 4 * M->np, cudaMemcpyDeviceToHost));
  H2D_CK(cudaDeviceSynchronize());
  return HODLR2D_OK;
}

int hodlr2d_rank_model_train(hodlr2d_rank_model_t M, const float* feats, const float* targets,
                             int64_t n, int batch, int epochs, float lr, float* loss_out) {
  if (!M || !feats || !targets || n < 1 || batch < 1 || epochs < 0 || !(lr > 0.f))
    return HODLR2D_ERR_ARG;
  // whole data set on the device once
  float *d_f = nullptr, *d_tg = nullptr;
  H2D_CK(cudaMalloc(&d_f, 4 * n * kNF));
  H2D_CK(cudaMalloc(&d_tg, 4 * n));
  int rc = copy_in(d_f, feats, n * kNF, 0);
  if (!rc) rc = copy_in(d_tg, targets, n, 0);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int e = 0; e < epochs && !rc; ++e) {
    for (int64_t o = 0; o < n && !rc; o += batch) {
      const int64_t b = std::min<int64_t>(batch, n - o);
      rc = mlp_reserve(M, b);
      if (rc) break;
      cudaMemcpyAsync(M->d_x, d_f + o * kNF, 4 * b * kNF, cudaMemcpyDeviceToDevice, 0);
      cudaMemcpyAsync(M->d_t, d_tg + o, 4 * b, cudaMemcpyDeviceToDevice, 0);
      rc = mlp_forward_backward(M, b, true, 0);
      if (rc) break;
      M->step += 1;
      const float c1 = 1.f - powf(b1, (float)M->step), c2 = 1.f - powf(b2, (float)M->step);
      k_adam<<<(unsigned)((M->np + 255) / 256), 256>>>(M->d_theta, M->d_grad, M->d_m, M->d_v, M->np,
                                                       lr, b1, b2, c1, c2, eps);
      if (cudaGetLastError() != cudaSuccess) rc = HODLR2D_ERR_CUDA;
    }
  }
  cudaFree(d_f);
  cudaFree(d_tg);
  if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = HODLR2D_ERR_CUDA;
  if (!rc && loss_out) rc = hodlr2d_rank_model_loss_grad(M, feats, targets, n, loss_out, nullptr);
  return rc;
}

int hodlr2d_rank_model_predict(hodlr2d_rank_model_t M, const float* feats, int64_t n, float* pred) {
  if (!M || !feats || !pred || n < 1) return HODLR2D_ERR_ARG;
  float *d_f = nullptr, *d_p = nullptr;
  H2D_CK(cudaMalloc(&d_f, 4 * n * kNF));
  H2D_CK(cudaMalloc(&d_p, 4 * n));
  int rc = copy_in(d_f, feats, n * kNF, 0);
  if (!rc) rc = mlp_predict_device(M, d_f, n, d_p, 0);
  if (!rc) {
    const cudaMemcpyKind kind = is_device_ptr(pred) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (cudaMemcpy(pred, d_p, 4 * n, kind) != cudaSuccess) rc = HODLR2D_ERR_CUDA;
  }
  cudaFree(d_f);
  cudaFree(d_p);
  return rc;
}

void hodlr2d_rank_model_free(hodlr2d_rank_model_t M) {
  if (!M) return;
  cudaFree(M->d_theta);
  cudaFree(M->d_grad);
  cudaFree(M->d_m);
  cudaFree(M->d_v);
  float* bufs[] = {M->d_x, M->d_t, M->d_z1, M->d_z2, M->d_y, M->d_dz2, M->d_dz1, M->d_loss};
  for (auto b : bufs) cudaFree(b);
  delete M;
}

}  // extern "C"
