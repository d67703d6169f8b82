// Automated equilibration detection ("Equilibration and production"): for each of S series and each
// candidate start t0 = c * stride, the statistical inefficiency g of the tail a[t0:],
//   g = 1 + 2 sum_{t >= 1} (1 - t/N) C(t),  C(t) = sum_i (a_i - mu)(a_{i+t} - mu) / ((N - t) var),
// summed until C(t) first drops to <= 0 (N = T - t0, mu and var of the tail); then per series the
// t0 that maximises N_eff = N / g (Chodera 2016).
//
// One warp per (series, candidate).  The tail is centred in FP64 (mean, variance) and staged in
// shared memory as FP32; the lag products accumulate per lane in FP32 (at most N/32 terms) and
// across the warp in FP64, so that a long positive autocorrelation (a drifting series) costs FP32
// work, not FP64 work, on this part.
#include "internal.cuh"

namespace algdock {
namespace {

constexpr unsigned kFullMask = 0xffffffffu;

__device__ inline double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
  return v;
}

__global__ void __launch_bounds__(32) tail_inefficiency_kernel(int64_t T, int64_t S, const double* __restrict__ a,
                                                                int64_t stride, int n_cand, double* g_out) {
  extern __shared__ float v[];
  const int lane = threadIdx.x;
  const int cand = blockIdx.x;
  const int64_t s = blockIdx.y;
  const int64_t t0 = (int64_t)cand * stride;
  const int64_t N = T - t0;
  double g = 1.0;
  if (N >= 2) {
    double sum = 0.0;
    for (int64_t i = lane; i < N; i += 32) sum += a[(t0 + i) * S + s];
    const double mu = warp_sum_d(sum) / (double)N;
    double var = 0.0;
    for (int64_t i = lane; i < N; i += 32) {
      const double d = a[(t0 + i) * S + s] - mu;
      var += d * d;
      v[i] = (float)d;
    }
    var = warp_sum_d(var) / (double)N;
    __syncwarp();
    if (var > 0.0) {
      for (int64_t t = 1; t < N; ++t) {
        float cl = 0.f;
        for (int64_t i = lane; i + t < N; i += 32) cl = fmaf(v[i], v[i + t], cl);
        const double c = warp_sum_d((double)cl) / ((double)(N - t) * var);
        if (c <= 0.0) break;  // the same value on every lane
        g += 2.0 * c * (1.0 - (double)t / (double)N);
      }
      if (g < 1.0) g = 1.0;
    }
  }
  if (lane == 0) g_out[s * n_cand + cand] = g;
}

// Per series: the candidate with the largest N_eff (the earliest on ties).
__global__ void best_start_kernel(int64_t T, int64_t S, int64_t stride, int n_cand, const double* __restrict__ g,
                                  int64_t* t0_best, double* neff_best) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  double best = -1.0;
  int64_t bt = 0;
  for (int c = 0; c < n_cand; ++c) {
    const int64_t t0 = (int64_t)c * stride;
    const double ne = (double)(T - t0) / g[s * n_cand + c];
    if (ne > best) {
      best = ne;
      bt = t0;
    }
  }
  if (t0_best) t0_best[s] = bt;
  if (neff_best) neff_best[s] = best;
}

}  // namespace

size_t equilibration_smem(int64_t T) { return (size_t)T * sizeof(float); }

cudaError_t launch_equilibration(cudaStream_t st, int64_t T, int64_t S, const double* a, int64_t stride, int n_cand,
                                 double* g, int64_t* t0_best, double* neff_best) {
  const size_t smem = equilibration_smem(T);
  cudaError_t e = cudaFuncSetAttribute(tail_inefficiency_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  tail_inefficiency_kernel<<<dim3((unsigned)n_cand, (unsigned)S), 32, smem, st>>>(T, S, a, stride, n_cand, g);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  best_start_kernel<<<(unsigned)((S + 127) / 128), 128, 0, st>>>(T, S, stride, n_cand, g, t0_best, neff_best);
  return cudaGetLastError();
}

}  // namespace algdock
