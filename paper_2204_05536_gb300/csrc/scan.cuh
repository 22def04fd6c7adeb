// Exclusive prefix sums for the build: a block-local scan of 2048 items per
// 256-thread block, a recursive scan of the block totals, and a fix-up pass.
// Deterministic (integer adds only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace h2d {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__global__ void k_scan_tile(const T* __restrict__ in, T* __restrict__ out,
                            T* __restrict__ tile_sum, int64_t n) {
  __shared__ T warp_tot[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t g = base + i;
    const T x = g < n ? in[g] : T(0);
    v[i] = run;
    run += x;
  }
  // inclusive scan of per-thread totals across the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T w = lane < kScanThreads / 32 ? warp_tot[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = w;
  }
  __syncthreads();
  const T excl = incl - run + (warp > 0 ? warp_tot[warp - 1] : T(0));
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t g = base + i;
    if (g < n) out[g] = v[i] + excl;
  }
  if (threadIdx.x == kScanThreads - 1) tile_sum[blockIdx.x] = excl + run;
}

template <typename T>
__global__ void k_scan_add(T* __restrict__ out, const T* __restrict__ tile_off, int64_t n) {
  const int64_t g = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  const T add = tile_off[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t x = g + (int64_t)i * kScanThreads;
    if (x < n) out[x] += add;
  }
}

// out[i] = in[0] + ... + in[i-1] for i < n, and out[n] = total (out has n + 1
// slots).  in and out may alias.  Build-time helper: allocates its temporaries.
template <typename T>
int scan_exclusive(const T* d_in, T* d_out, int64_t n, cudaStream_t s) {
  if (n <= 0) {
    H2D_CK(cudaMemsetAsync(d_out, 0, sizeof(T), s));
    return HODLR2D_OK;
  }
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  T* d_tile = nullptr;
  H2D_CK(cudaMalloc(&d_tile, sizeof(T) * (tiles + 1)));
  k_scan_tile<T><<<(unsigned)tiles, kScanThreads, 0, s>>>(d_in, d_out, d_tile, n);
  int rc = cudaGetLastError() == cudaSuccess ? HODLR2D_OK : HODLR2D_ERR_CUDA;
  if (tiles > 1) {
    // scan the tile totals (d_tile[tiles] receives the grand total), then
    // add each tile's offset to its items
    if (rc == HODLR2D_OK) rc = scan_exclusive<T>(d_tile, d_tile, tiles, s);
    if (rc == HODLR2D_OK) {
      k_scan_add<T><<<(unsigned)tiles, kScanThreads, 0, s>>>(d_out, d_tile, n);
      if (cudaGetLastError() != cudaSuccess) rc = HODLR2D_ERR_CUDA;
    }
  }
  // a single tile's total is d_tile[0]; otherwise the scan left it in d_tile[tiles]
  const T* total = d_tile + (tiles > 1 ? tiles : 0);
  if (rc == HODLR2D_OK &&
      cudaMemcpyAsync(d_out + n, total, sizeof(T), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    rc = HODLR2D_ERR_CUDA;
  cudaStreamSynchronize(s);
  cudaFree(d_tile);
  return rc;
}

}  // namespace h2d
