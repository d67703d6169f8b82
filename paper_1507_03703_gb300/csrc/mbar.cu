// MBAR (Shirts & Chodera 2008; "Estimation") by self-consistent iteration in log-sum-exp form.
//
// One iteration is four kernels on the stream:
//   1. log_denominators: for every sample n, log D_n = ln sum_k N_k exp(f_k - u_kn)   (one thread per n)
//   2. state_partials:   for every state i and a chunk of samples, the (max, sum) pair of
//                        exp(-u_in - log D_n)                                       (block per (chunk, i))
//   3. merge_chunks:     f_i <- -ln sum_n ..., the chunks' pairs of each state merged (one warp per state)
//   4. finalize:         gauge f_0 = 0, convergence flag                             (one block)
// Every kernel returns at once when the device flag says the iteration has converged, so the host
// can enqueue iterations in batches and poll the flag between batches.
#include <math.h>

#include <mutex>
#include <string>

#include "internal.cuh"

namespace algdock {
namespace {

constexpr int kPartialThreads = 256;
// Samples per state_partials block: the largest power of two in [8192, 32768] that still gives a
// full wave of blocks (K x chunks >= 152 SMs x 8 resident blocks), so that large solves spread
// each block's merge over more loads and small ones keep every SM busy.
inline int64_t mbar_chunk(int K, int64_t N) {
  int64_t c = 32768;
  while (c > 8192 && (int64_t)K * ((N + c - 1) / c) < 152 * 8) c >>= 1;
  return c;
}

struct MbarState {
  int converged;
  int iters;
  int _pad[2];
};

// Online log-sum-exp accumulator: value = m + log(s).
struct Lse {
  double m, s;
};
__device__ inline void lse_add(Lse& a, double x, int mode) {
  if (x == -INFINITY) return;
  if (x <= a.m) {
    a.s += mode ? (double)__expf((float)(x - a.m)) : exp(x - a.m);
  } else {
    a.s = a.s * (mode ? (double)__expf((float)(a.m - x)) : exp(a.m - x)) + 1.0;
    a.m = x;
  }
}
__device__ inline Lse lse_merge(Lse a, Lse b) {
  if (b.m == -INFINITY) return a;
  if (a.m == -INFINITY) return b;
  if (a.m >= b.m) return Lse{a.m, a.s + b.s * exp(b.m - a.m)};
  return Lse{b.m, b.s + a.s * exp(a.m - b.m)};
}

__global__ void log_denominators(int K, int64_t N, const double* __restrict__ u, const double* __restrict__ logNk,
                                 const double* __restrict__ f, double* logD, const MbarState* st, int mode) {
  if (st->converged) return;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  Lse a{-INFINITY, 0.0};
  // eight independent loads in flight, then the updates in the same order as one at a time
  constexpr int kAhead = 8;
  const double* col = u + n;
  int k = 0;
  for (; k + kAhead <= K; k += kAhead) {
    double v[kAhead];
#pragma unroll
    for (int j = 0; j < kAhead; ++j) v[j] = __ldg(col + (int64_t)(k + j) * N);
#pragma unroll
    for (int j = 0; j < kAhead; ++j) lse_add(a, logNk[k + j] + f[k + j] - v[j], mode);
  }
  for (; k < K; ++k) lse_add(a, logNk[k] + f[k] - __ldg(col + (int64_t)k * N), mode);
  logD[n] = a.m + log(a.s);
}

__global__ void __launch_bounds__(kPartialThreads) state_partials(int64_t N, int64_t chunk_len,
                                                                  const double* __restrict__ u,
                                                                  const double* __restrict__ logD, double2* part,
                                                                  int n_chunks, const MbarState* st, int mode) {
  if (st->converged) return;
  const int i = blockIdx.y, chunk = blockIdx.x;
  const int64_t begin = (int64_t)chunk * chunk_len;
  const int64_t end = min(N, begin + chunk_len);
  Lse a{-INFINITY, 0.0};
  const double* ui = u + (int64_t)i * N;
  constexpr int kAhead = 8;
  const int64_t stride = blockDim.x;
  int64_t n = begin + threadIdx.x;
  for (; n + (kAhead - 1) * stride < end; n += kAhead * stride) {
    double v[kAhead], d[kAhead];
#pragma unroll
    for (int j = 0; j < kAhead; ++j) {
      v[j] = __ldg(ui + n + j * stride);
      d[j] = __ldg(logD + n + j * stride);
    }
#pragma unroll
    for (int j = 0; j < kAhead; ++j) lse_add(a, -v[j] - d[j], mode);
  }
  for (; n < end; n += stride) lse_add(a, -ui[n] - logD[n], mode);
  __shared__ double sm[kPartialThreads], ss[kPartialThreads];
  sm[threadIdx.x] = a.m;
  ss[threadIdx.x] = a.s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      const Lse r = lse_merge(Lse{sm[threadIdx.x], ss[threadIdx.x]}, Lse{sm[threadIdx.x + w], ss[threadIdx.x + w]});
      sm[threadIdx.x] = r.m;
      ss[threadIdx.x] = r.s;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)i * n_chunks + chunk] = make_double2(sm[0], ss[0]);
}

// The gauge f_0 = 0 and the convergence test on f^new (formed by merge_chunks).
__global__ void finalize(int K, double* f, double* fnew, MbarState* st, double tol, int max_iter) {
  if (st->converged) return;
  __shared__ double s_delta[256];
  __syncthreads();
  const double f0 = fnew[0];
  double dmax = 0.0;
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    const double v = fnew[i] - f0;
    const double d = fabs(v - f[i]);
    dmax = (d > dmax || isnan(d)) ? d : dmax;
  }
  s_delta[threadIdx.x] = dmax;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      const double o = s_delta[threadIdx.x + w];
      if (o > s_delta[threadIdx.x] || isnan(o)) s_delta[threadIdx.x] = o;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < K; i += blockDim.x) f[i] = fnew[i] - f0;
  __syncthreads();
  if (threadIdx.x == 0) {
    st->iters += 1;
    if (s_delta[0] < tol) st->converged = 1;
    else if (st->iters >= max_iter) st->converged = 2;  // stop: not converged
  }
}

// ---------------------------------------------------------------- precision mode 2: FP32
// Every sample's column of u_kn is shifted once by its minimum s_n (in FP64) and stored as FP32,
// w_kn = u_kn - s_n.  The shift cancels exactly: log D_n and the state sums change by -s_n and +s_n
// in turn.  The iterations then run in FP32 (arguments, exponentials, Kahan-compensated sums),
// with FP64 only where the per-thread partial sums meet.  That halves the bytes read per
// iteration and removes FP64 work from the inner loops.
__global__ void shift_columns(int K, int64_t N, const double* __restrict__ u, float* w) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double m = INFINITY;
  for (int k = 0; k < K; ++k) m = fmin(m, u[(int64_t)k * N + n]);
  if (!isfinite(m)) m = 0.0;
  for (int k = 0; k < K; ++k) w[(int64_t)k * N + n] = (float)(u[(int64_t)k * N + n] - m);
}

// Online log-sum-exp in FP32, value m + log(s - c) with the Kahan compensation c.
struct LseF {
  float m, s, c;
};
__device__ inline void lsef_add(LseF& a, float x) {
  if (x == -INFINITY) return;
  if (x <= a.m) {
    const float y = __expf(x - a.m) - a.c;
    const float t = a.s + y;
    a.c = (t - a.s) - y;
    a.s = t;
  } else {
    const float r = a.m == -INFINITY ? 0.f : __expf(a.m - x);
    a.s = a.s * r + 1.f;
    a.c *= r;
    a.m = x;
  }
}

// One (max, sum) pair from every thread's (m, s): the exact maximum M (a float), then
// sum_t s_t exp(m_t - M) with the factor in FP32 (about 1e-7 relative, independent between
// threads) and the sum in FP64, over the warp by shuffles and over the warps in shared memory.
// The result is valid in thread 0; every thread of the block must call it.
__device__ inline Lse block_merge_f32(float m, double s) {
  __shared__ float s_m[kPartialThreads / 32];
  __shared__ double s_s[kPartialThreads / 32];
  const unsigned full = 0xffffffffu;
  float wm = m;
  for (int o = 16; o > 0; o >>= 1) wm = fmaxf(wm, __shfl_xor_sync(full, wm, o));
  double t = (m == -INFINITY) ? 0.0 : s * (double)expf(m - wm);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(full, t, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_m[warp] = wm;
    s_s[warp] = t;
  }
  __syncthreads();
  Lse r{-INFINITY, 0.0};
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    const float pm = lane < nw ? s_m[lane] : -INFINITY;
    const double ps = lane < nw ? s_s[lane] : 0.0;
    float bm = pm;
    for (int o = 16; o > 0; o >>= 1) bm = fmaxf(bm, __shfl_xor_sync(full, bm, o));
    double u = (pm == -INFINITY) ? 0.0 : ps * (double)expf(pm - bm);
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(full, u, o);
    r = Lse{bm == -INFINITY ? -INFINITY : (double)bm, u};
  }
  return r;
}

__global__ void log_denominators_f32(int K, int64_t N, const float* __restrict__ w, const double* __restrict__ logNk,
                                     const double* __restrict__ f, float* logD, const MbarState* st) {
  if (st->converged) return;
  extern __shared__ float g_k[];
  for (int k = threadIdx.x; k < K; k += blockDim.x) g_k[k] = (float)(logNk[k] + f[k]);
  __syncthreads();
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  LseF a{-INFINITY, 0.f, 0.f};
  // eight independent loads in flight before the dependent log-sum-exp updates (each thread walks
  // its column; a warp's loads of one state are one coalesced row segment)
  constexpr int kAhead = 8;
  const float* col = w + n;
  int k = 0;
  for (; k + kAhead <= K; k += kAhead) {
    float v[kAhead];
#pragma unroll
    for (int j = 0; j < kAhead; ++j) v[j] = __ldg(col + (int64_t)(k + j) * N);
#pragma unroll
    for (int j = 0; j < kAhead; ++j) lsef_add(a, g_k[k + j] - v[j]);
  }
  for (; k < K; ++k) lsef_add(a, g_k[k] - __ldg(col + (int64_t)k * N));
  logD[n] = a.m + logf(a.s - a.c);
}

__global__ void __launch_bounds__(kPartialThreads) state_partials_f32(int64_t N, int64_t chunk_len,
                                                                      const float* __restrict__ w,
                                                                      const float* __restrict__ logD, double2* part,
                                                                      int n_chunks, const MbarState* st) {
  if (st->converged) return;
  const int i = blockIdx.y, chunk = blockIdx.x;
  const int64_t begin = (int64_t)chunk * chunk_len;
  const int64_t end = min(N, begin + chunk_len);
  LseF a{-INFINITY, 0.f, 0.f};
  const float* wi = w + (int64_t)i * N;
  // eight independent pairs of loads in flight per thread, then the dependent updates
  constexpr int kAhead = 8;
  const int64_t stride = blockDim.x;
  int64_t n = begin + threadIdx.x;
  for (; n + (kAhead - 1) * stride < end; n += kAhead * stride) {
    float v[kAhead], d[kAhead];
#pragma unroll
    for (int j = 0; j < kAhead; ++j) {
      v[j] = __ldg(wi + n + j * stride);
      d[j] = __ldg(logD + n + j * stride);
    }
#pragma unroll
    for (int j = 0; j < kAhead; ++j) lsef_add(a, -v[j] - d[j]);
  }
  for (; n < end; n += stride) lsef_add(a, -wi[n] - logD[n]);
  // block merge without FP64 exponentials (slow on this GPU): the exact maximum of the partials'
  // maxima, each partial rescaled by an FP32 exp of its (non-positive) offset, the rescaled sums
  // added in FP64; first within each warp, then over the warps
  const Lse r = block_merge_f32(a.m, (double)a.s - (double)a.c);
  if (threadIdx.x == 0) part[(int64_t)i * n_chunks + chunk] = make_double2(r.m, r.s);
}

// Each state's chunk pairs merged by one warp into f_i^new = -(M + ln S): lanes take every 32nd
// chunk, then a butterfly over the lanes.  F32 (precision mode 2, whose maxima are floats): the
// exact maximum, FP32 rescale factors and an FP64 sum.  Otherwise FP64 log-sum-exp merges (the
// merge is symmetric in its operands, so every lane ends with the same bits).  finalize then
// applies the gauge and the convergence test.
template <bool F32>
__global__ void merge_chunks(int K, int n_chunks, const double2* __restrict__ part, double* fnew,
                             const MbarState* st) {
  if (st->converged) return;
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= K) return;
  const unsigned full = 0xffffffffu;
  const double2* pi = part + (int64_t)i * n_chunks;
  if (F32) {
    float M = -INFINITY;
    for (int c = lane; c < n_chunks; c += 32) M = fmaxf(M, (float)pi[c].x);
    for (int o = 16; o > 0; o >>= 1) M = fmaxf(M, __shfl_xor_sync(full, M, o));
    double S = 0.0;
    if (M != -INFINITY)
      for (int c = lane; c < n_chunks; c += 32)
        if (pi[c].x != -INFINITY) S += pi[c].y * (double)expf((float)pi[c].x - M);
    for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(full, S, o);
    if (lane == 0) fnew[i] = M == -INFINITY ? INFINITY : -((double)M + log(S));
  } else {
    Lse a{-INFINITY, 0.0};
    for (int c = lane; c < n_chunks; c += 32) a = lse_merge(a, Lse{pi[c].x, pi[c].y});
    for (int o = 16; o > 0; o >>= 1) {
      const Lse b{__shfl_xor_sync(full, a.m, o), __shfl_xor_sync(full, a.s, o)};
      a = lse_merge(a, b);
    }
    if (lane == 0) fnew[i] = -(a.m + log(a.s));
  }
}

// Each state's chunk pairs merged into one (max, sum) pair (FP64 log-sum-exp merges, one warp per
// state), for MBAR sharded over samples: the pairs of all processes are merged on the host.
__global__ void merge_chunk_pairs(int K, int n_chunks, const double2* __restrict__ part, double2* out) {
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= K) return;
  const unsigned full = 0xffffffffu;
  const double2* pi = part + (int64_t)i * n_chunks;
  Lse a{-INFINITY, 0.0};
  for (int c = lane; c < n_chunks; c += 32) a = lse_merge(a, Lse{pi[c].x, pi[c].y});
  for (int o = 16; o > 0; o >>= 1) {
    const Lse b{__shfl_xor_sync(full, a.m, o), __shfl_xor_sync(full, a.s, o)};
    a = lse_merge(a, b);
  }
  if (lane == 0) out[i] = make_double2(a.m, a.s);
}

__global__ void init_state(int K, const int64_t* Nk, double* logNk, double* f, MbarState* st) {
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    logNk[k] = Nk[k] > 0 ? log((double)Nk[k]) : -INFINITY;
    f[k] = 0.0;
  }
  if (threadIdx.x == 0) {
    st->converged = 0;
    st->iters = 0;
  }
}

}  // namespace

// Scratch layout (bytes): MbarState | logNk[K] | f[K] | fnew[K] | Nk[K] (int64) | part[K][n_chunks] | logD[N]
// (double; float in mode 2), then in mode 2 the shifted FP32 copy w[K][N] (256-byte aligned).
size_t mbar_scratch_bytes(int K, int64_t N) {
  const int64_t chunk_len = mbar_chunk(K, N);
  const int64_t n_chunks = (N + chunk_len - 1) / chunk_len;
  return 64 + 4 * (size_t)K * 8 + (size_t)K * n_chunks * 16 + (size_t)N * 8 + 256;
}
size_t mbar_scratch_bytes_mode(int K, int64_t N, int mode) {
  return mbar_scratch_bytes(K, N) + (mode == 2 ? (size_t)K * N * sizeof(float) + 256 : 0);
}

// One iteration's (max, sum) pair per state over these N samples, given the global N_k and the
// current f (host arrays): sum_n exp(-u_in - log D_n) = sum * exp(max), with log D_n over all K
// states as in the full solve.  Scratch: mbar_pairs_scratch_bytes(K, N).  pairs_host [K][2].
size_t mbar_pairs_scratch_bytes(int K, int64_t N) { return mbar_scratch_bytes(K, N) + 16 * (size_t)K + 256; }

cudaError_t mbar_local_pairs(cudaStream_t s, void* scratch, int K, int64_t N, const double* u_kn,
                             const int64_t* Nk_host, const double* f_host, int mode, double* pairs_host) {
  const int64_t chunk_len = mbar_chunk(K, N);
  const int64_t n_chunks = (N + chunk_len - 1) / chunk_len;
  char* p = (char*)scratch;
  MbarState* st = (MbarState*)p;
  double* logNk = (double*)(p + 64);
  double* f = logNk + K;
  double* fnew = f + K;
  int64_t* Nk = (int64_t*)(fnew + K);
  double2* part = (double2*)(Nk + K);
  double* logD = (double*)(part + (size_t)K * n_chunks);
  const size_t off = ((size_t)((char*)(logD + N) - p) + 255) & ~(size_t)255;
  double2* pairs = (double2*)(p + off);
  cudaError_t e = cudaMemcpyAsync(Nk, Nk_host, sizeof(int64_t) * K, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  init_state<<<1, 256, 0, s>>>(K, Nk, logNk, f, st);
  e = cudaMemcpyAsync(f, f_host, sizeof(double) * K, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const int threads = 256;
  log_denominators<<<(unsigned)((N + threads - 1) / threads), threads, 0, s>>>(K, N, u_kn, logNk, f, logD, st, mode);
  state_partials<<<dim3((unsigned)n_chunks, (unsigned)K), kPartialThreads, 0, s>>>(N, chunk_len, u_kn, logD, part,
                                                                                    (int)n_chunks, st, mode);
  merge_chunk_pairs<<<(unsigned)((K * 32 + 255) / 256), 256, 0, s>>>(K, (int)n_chunks, part, pairs);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(pairs_host, pairs, sizeof(double2) * K, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

// Runs the solver on caller-provided scratch (mbar_scratch_bytes(K, N) bytes, 256-byte aligned).
// h_flag: pinned host int used to poll the device flag.  Returns 0 converged, 1 not converged,
// -1 on a CUDA error (then *err is set).
int mbar_run(cudaStream_t s, void* scratch, int K, int64_t N, const double* u_kn, const int64_t* Nk_host,
             double tol, int max_iter, int mode, double* f_host, int* iters, int* h_flag, cudaError_t* err) {
  const int64_t chunk_len = mbar_chunk(K, N);
  const int64_t n_chunks = (N + chunk_len - 1) / chunk_len;
  char* p = (char*)scratch;
  MbarState* st = (MbarState*)p;
  double* logNk = (double*)(p + 64);
  double* f = logNk + K;
  double* fnew = f + K;
  int64_t* Nk = (int64_t*)(fnew + K);
  double2* part = (double2*)(Nk + K);
  double* logD = (double*)(part + (size_t)K * n_chunks);
  cudaError_t e = cudaMemcpyAsync(Nk, Nk_host, sizeof(int64_t) * K, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) { *err = e; return -1; }
  init_state<<<1, 256, 0, s>>>(K, Nk, logNk, f, st);
  const int threads = 256;
  const unsigned blocks_n = (unsigned)((N + threads - 1) / threads);
  const dim3 grid_p((unsigned)n_chunks, (unsigned)K);
  float* w32 = nullptr;
  if (mode == 2) {
    const size_t off = ((size_t)((char*)(logD + N) - (char*)scratch) + 255) & ~(size_t)255;
    w32 = (float*)((char*)scratch + off);
    shift_columns<<<blocks_n, threads, 0, s>>>(K, N, u_kn, w32);
    e = cudaFuncSetAttribute(log_denominators_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(K * sizeof(float)));
    if (e != cudaSuccess) { *err = e; return -1; }
  }
  int done = 0;
  int issued = 0;
  int batch = 4;
  while (!done) {
    for (int b = 0; b < batch && issued < max_iter; ++b, ++issued) {
      if (mode == 2) {
        log_denominators_f32<<<blocks_n, threads, K * sizeof(float), s>>>(K, N, w32, logNk, f, (float*)logD, st);
        state_partials_f32<<<grid_p, kPartialThreads, 0, s>>>(N, chunk_len, w32, (const float*)logD, part,
                                                              (int)n_chunks, st);
      } else {
        log_denominators<<<blocks_n, threads, 0, s>>>(K, N, u_kn, logNk, f, logD, st, mode);
        state_partials<<<grid_p, kPartialThreads, 0, s>>>(N, chunk_len, u_kn, logD, part, (int)n_chunks, st, mode);
      }
      const unsigned merge_blocks = (unsigned)((K * 32 + 255) / 256);
      if (mode == 2)
        merge_chunks<true><<<merge_blocks, 256, 0, s>>>(K, (int)n_chunks, part, fnew, st);
      else
        merge_chunks<false><<<merge_blocks, 256, 0, s>>>(K, (int)n_chunks, part, fnew, st);
      finalize<<<1, 256, 0, s>>>(K, f, fnew, st, tol, max_iter);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_flag, &st->converged, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { *err = e; return -1; }
    done = (*h_flag != 0) || issued >= max_iter;
    if (batch < 64) batch *= 2;
  }
  MbarState hs;
  e = cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f_host, f, sizeof(double) * K, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { *err = e; return -1; }
  *iters = hs.iters;
  return hs.converged == 1 ? 0 : 1;
}

}  // namespace algdock

// ------------------------------------------------------------------ allocation-free MBAR
// Callers that must not allocate device memory - a host framework whose caching allocator owns
// all device memory and forbids direct cudaMalloc, or a service that reserves its whole memory
// budget at start-up - use algdock_mbar_noalloc.  Its scratch is this fixed array in the
// library's own device memory, present on every GPU that loads the library until the process
// exits.
namespace {

constexpr size_t kNoallocScratchBytes = (size_t)8 << 20;  // 8 MiB
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_mbar_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the array's name is
// only a host-side stand-in, so the address is looked up once per device (with that device
// current) and cached.
cudaError_t noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_mbar_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" algdock_status algdock_mbar_noalloc(algdock_ctx* c, int32_t K, int64_t N, const double* u_kn,
                                               const int64_t* N_k, double tol, int32_t max_iter,
                                               int32_t precision_mode, double* f_k, int32_t* iters) {
  if (!c) return ALGDOCK_E_INVALID;
  try {
    if (K < 1 || N < 1 || !u_kn || !N_k || !f_k || !iters || max_iter < 1 || !(tol > 0)) {
      c->err = "mbar_noalloc: bad arguments";
      return ALGDOCK_E_INVALID;
    }
    if (precision_mode != 0 && precision_mode != 1) {
      c->err = "mbar_noalloc: precision_mode must be 0 or 1 (mode 2 keeps an FP32 copy of u_kn, K*N*4 bytes, "
               "which the fixed scratch array does not hold; use algdock_mbar for mode 2)";
      return ALGDOCK_E_INVALID;
    }
    if (K > algdock::kMbarMaxStates) {
      c->err = "mbar_noalloc: K = " + std::to_string(K) + " exceeds the " + std::to_string(algdock::kMbarMaxStates) +
               " states one launch grid dimension can hold";
      return ALGDOCK_E_INVALID;
    }
    int64_t total = 0;
    for (int k = 0; k < K; ++k) {
      if (N_k[k] < 0) {
        c->err = "mbar_noalloc: negative N_k";
        return ALGDOCK_E_INVALID;
      }
      total += N_k[k];
    }
    if (total != N) {
      c->err = "mbar_noalloc: sum of N_k must equal N";
      return ALGDOCK_E_INVALID;
    }
    const size_t need = algdock::mbar_scratch_bytes(K, N);
    if (need > kNoallocScratchBytes) {
      c->err = "mbar_noalloc: K = " + std::to_string(K) + ", N = " + std::to_string(N) + " needs " +
               std::to_string(need) + " bytes of scratch, more than the fixed " +
               std::to_string(kNoallocScratchBytes) + "-byte buffer; use algdock_mbar";
      return ALGDOCK_E_INVALID;
    }
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, u_kn) != cudaSuccess ||
        (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      c->err = "mbar_noalloc: u_kn must be a device pointer";
      return ALGDOCK_E_INVALID;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    void* scratch = nullptr;
    cudaError_t e = noalloc_scratch(c->device, &scratch);
    cudaError_t err = cudaSuccess;
    int it = 0;
    int r = -1;
    if (e == cudaSuccess) r = algdock::mbar_run(c->stream, scratch, K, N, u_kn, N_k, tol, max_iter, precision_mode,
                                                f_k, &it, c->h_flag, &err);
    else err = e;
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    *iters = it;
    if (r < 0) {
      c->err = std::string("mbar_noalloc: ") + cudaGetErrorString(err);
      return err == cudaErrorMemoryAllocation ? ALGDOCK_E_OOM : ALGDOCK_E_CUDA;
    }
    if (r == 1) {
      c->err = "mbar_noalloc: max_iter reached";
      return ALGDOCK_E_NOT_CONVERGED;
    }
    return ALGDOCK_OK;
  } catch (...) {
    try {
      c->err = "mbar_noalloc: host exception";
    } catch (...) {
    }
    return ALGDOCK_E_INVALID;
  }
}
