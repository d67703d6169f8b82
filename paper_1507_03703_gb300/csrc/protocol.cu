// Protocol initialization ("Initialization"): the per-state reductions of building a protocol
// state by state.
//   state_stats_kernel   sigma[U_L + U_I], sigma[Psi_sg], sigma[Psi_g], sigma[u_k] over a state's
//                        samples (population standard deviations, FP64, two passes)
//   resample_kernel      seeds for the next state by sampling importance resampling: weights
//                        exp(u_from - u_to) of every sample, cumulated in index order, draws from
//                        Philox counter {j, 0, ctr, 6}; the chosen configurations are gathered
//   pacc_kernel          the mean exchange probability of Eq. (repXacc) over pairs of samples
// Each is one block: a state has a few thousand samples.
#include <math.h>

#include "internal.cuh"

namespace algdock {
namespace {

constexpr int kProtoThreads = 256;
constexpr uint32_t kPurposeResample = 6;

__device__ inline double reduced_u(const StateDev& s, const double* c) {
  double e = __dadd_rn(c[0], c[1]);
  if (s.w_sg != 0.0) e = __dadd_rn(e, __dmul_rn(s.w_sg, c[2]));
  if (s.w_g != 0.0) e = __dadd_rn(e, __dmul_rn(s.w_g, c[3]));
  return __dmul_rn(s.beta, e);
}

__device__ inline double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kProtoThreads) state_stats_kernel(int64_t n, const double* __restrict__ comps,
                                                                     const StateDev* __restrict__ states, int k,
                                                                     double* out) {
  __shared__ double sh[kProtoThreads];
  const StateDev st = states[k];
  double m[4] = {0, 0, 0, 0};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double* c = comps + 4 * i;
    m[0] += c[0] + c[1];
    m[1] += c[2];
    m[2] += c[3];
    m[3] += reduced_u(st, c);
  }
  for (int q = 0; q < 4; ++q) m[q] = block_sum(m[q], sh) / (double)n;
  double v[4] = {0, 0, 0, 0};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double* c = comps + 4 * i;
    const double d[4] = {c[0] + c[1] - m[0], c[2] - m[1], c[3] - m[2], reduced_u(st, c) - m[3]};
    for (int q = 0; q < 4; ++q) v[q] += d[q] * d[q];
  }
  for (int q = 0; q < 4; ++q) {
    const double t = block_sum(v[q], sh);
    if (threadIdx.x == 0) out[q] = sqrt(t / (double)n);
  }
}

// work: n doubles (the weights, then their running sums)
__global__ void __launch_bounds__(kProtoThreads) resample_kernel(int64_t n, const double* __restrict__ comps,
                                                                  const StateDev* __restrict__ states, int k_from,
                                                                  int k_to, int n_out, uint64_t seed, uint32_t ctr,
                                                                  double* work, int64_t* idx, int na,
                                                                  const float* __restrict__ x_in, float* x_out) {
  __shared__ double sh[kProtoThreads];
  __shared__ int64_t s_pick[1024];
  const StateDev a = states[k_from], b = states[k_to];
  double mx = -INFINITY;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double lw = reduced_u(a, comps + 4 * i) - reduced_u(b, comps + 4 * i);
    work[i] = lw;
    mx = fmax(mx, lw);
  }
  sh[threadIdx.x] = mx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  mx = sh[0];
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) work[i] = exp(work[i] - mx);
  __syncthreads();
  if (threadIdx.x == 0) {  // running sums in index order
    double tot = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      tot += work[i];
      work[i] = tot;
    }
  }
  __syncthreads();
  const double tot = work[n - 1];
  for (int j = threadIdx.x; j < n_out; j += blockDim.x) {
    const U4 r = philox(seed, (uint32_t)j, 0u, ctr, kPurposeResample);
    const double u = uniform53(r.x, r.y) * tot;
    int64_t lo = 0, hi = n - 1;  // first index with running sum > u
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (u < work[mid]) hi = mid;
      else lo = mid + 1;
    }
    s_pick[j] = lo;
    if (idx) idx[j] = lo;
  }
  __syncthreads();
  if (x_in && x_out)
    for (int64_t e = threadIdx.x; e < (int64_t)n_out * na * 3; e += blockDim.x) {
      const int64_t j = e / (na * 3), r = e % (na * 3);
      x_out[j * na * 3 + r] = x_in[s_pick[j] * na * 3 + r];
    }
}

__global__ void __launch_bounds__(kProtoThreads) pacc_kernel(int64_t n, const double* __restrict__ ca,
                                                              const double* __restrict__ cb,
                                                              const StateDev* __restrict__ states, int ka, int kb,
                                                              double* out) {
  __shared__ double sh[kProtoThreads];
  const StateDev a = states[ka], b = states[kb];
  double t = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double* xa = ca + 4 * i;
    const double* xb = cb + 4 * i;
    const double d = reduced_u(a, xa) + reduced_u(b, xb) - reduced_u(a, xb) - reduced_u(b, xa);
    t += d >= 0.0 ? 1.0 : exp(d);
  }
  t = block_sum(t, sh);
  if (threadIdx.x == 0) *out = t / (double)n;
}

}  // namespace

cudaError_t launch_state_stats(cudaStream_t s, const algdock_ctx& c, int64_t n, const double* comps, int k,
                               double* out) {
  state_stats_kernel<<<1, kProtoThreads, 0, s>>>(n, comps, c.d_states, k, out);
  return cudaGetLastError();
}

cudaError_t launch_resample(cudaStream_t s, const algdock_ctx& c, int64_t n, const double* comps, int k_from,
                            int k_to, int n_out, uint64_t seed, uint32_t ctr, double* work, int64_t* idx,
                            const float* x_in, float* x_out) {
  resample_kernel<<<1, kProtoThreads, 0, s>>>(n, comps, c.d_states, k_from, k_to, n_out, seed, ctr, work, idx,
                                              c.lig.na, x_in, x_out);
  return cudaGetLastError();
}

cudaError_t launch_pacc(cudaStream_t s, const algdock_ctx& c, int64_t n, const double* ca, const double* cb, int ka,
                        int kb, double* out) {
  pacc_kernel<<<1, kProtoThreads, 0, s>>>(n, ca, cb, c.d_states, ka, kb, out);
  return cudaGetLastError();
}

}  // namespace algdock

// ------------------------------------------------------------------ the scalar steps (host)
// Protocol initialization places the states of a leg one thermodynamic-length step apart and
// adapts each state's time step; between cycles it inserts states where neighbours stopped
// exchanging ("Initialization"; "Equilibration and production").  These steps are a few scalar
// operations per state, so they run on the host, in the library, beside the device reductions
// above that supply their inputs.
namespace {

constexpr double kBoltzmannKcal = 0.0019872043;  // kcal/(mol K)

double logistic(double z) { return z >= 0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z)); }

// d alpha_sg / d alpha and d alpha_g / d alpha for alpha_sg = 1 - (2 alpha - 1)^2 and
// alpha_g = (2 alpha - 1)^2 logistic(1000 (alpha - 1/2)), Eq. (protocol).
double d_alpha_sg(double a) { return -4.0 * (2.0 * a - 1.0); }
double d_alpha_g(double a) {
  const double s = 2.0 * a - 1.0;
  const double L = logistic(1000.0 * (a - 0.5));
  return 4.0 * s * L + s * s * 1000.0 * L * (1.0 - L);
}

}  // namespace

extern "C" {

algdock_status algdock_next_temperature(double T, double sigma_U, double speed, double T_end, double* T_next) {
  if (!T_next || !(T > 0) || !isfinite(T) || !(sigma_U >= 0) || !isfinite(sigma_U) || !(speed > 0) ||
      !isfinite(T_end))
    return ALGDOCK_E_INVALID;
  // the thermodynamic length along T changes at sigma[U_S] / (k_B T^2)
  *T_next = sigma_U <= 0.0 ? T_end : fmin(T_end, T + speed * kBoltzmannKcal * T * T / sigma_U);
  return ALGDOCK_OK;
}

algdock_status algdock_next_alpha(double alpha, double sigma_sg, double sigma_g, double sigma_u, double speed,
                                  double T_T, double T_H, double* alpha_next) {
  if (!alpha_next || !(alpha >= 0) || !(alpha <= 1) || !(sigma_sg >= 0) || !(sigma_g >= 0) || !(sigma_u >= 0) ||
      !isfinite(sigma_sg) || !isfinite(sigma_g) || !isfinite(sigma_u) || !(speed > 0) || !(T_T > 0) || !(T_H > 0))
    return ALGDOCK_E_INVALID;
  const double T = (T_T - T_H) * alpha + T_H;
  const double rate = fabs(d_alpha_sg(alpha)) * sigma_sg / (kBoltzmannKcal * T) +
                      fabs(d_alpha_g(alpha)) * sigma_g / (kBoltzmannKcal * T) + fabs(T_T - T_H) * sigma_u / T;
  *alpha_next = rate <= 0.0 ? 1.0 : fmin(1.0, alpha + speed / rate);
  return ALGDOCK_OK;
}

algdock_status algdock_adapt_dt(double dt, double acceptance, double* dt_next) {
  if (!dt_next || !isfinite(dt) || !(acceptance >= 0) || !(acceptance <= 1)) return ALGDOCK_E_INVALID;
  if (acceptance > 0.8) dt += 0.125;
  else if (acceptance < 0.1) dt -= 0.5;
  else if (acceptance < 0.4) dt -= 0.25;
  *dt_next = fmin(5.0, fmax(0.1, dt));
  return ALGDOCK_OK;
}

algdock_status algdock_insert_states(int32_t K, const double* T, const double* alpha, const double* dt,
                                     const int64_t* attempts, const int64_t* accepts, double threshold, double T_T,
                                     double T_H, int32_t capacity, int32_t* K_out, double* T_out, double* alpha_out,
                                     double* dt_out, int32_t* lower) {
  if (K < 1 || !T || !alpha || !dt || (K > 1 && (!attempts || !accepts)) || !K_out || !T_out || !alpha_out ||
      !dt_out || !lower || capacity < 2 * K - 1 || !(threshold >= 0) || !(T_T > 0) || !(T_H > 0))
    return ALGDOCK_E_INVALID;
  int n = 0;
  for (int k = 0; k < K; ++k) {
    T_out[n] = T[k];
    alpha_out[n] = alpha[k];
    dt_out[n] = dt[k];
    lower[n] = -1;
    ++n;
    if (k + 1 < K && attempts[k] > 0 && (double)accepts[k] / (double)attempts[k] < threshold) {
      double t, a;
      if (isnan(alpha[k])) {  // warming leg: the geometric mean keeps the ladder geometric
        t = sqrt(T[k] * T[k + 1]);
        a = alpha[k];
      } else {  // coupling leg: the mean alpha, with its temperature T(alpha)
        a = 0.5 * (alpha[k] + alpha[k + 1]);
        t = T_H + (T_T - T_H) * a;
      }
      T_out[n] = t;
      alpha_out[n] = a;
      dt_out[n] = fmin(dt[k], dt[k + 1]);
      lower[n] = n - 1;
      ++n;
    }
  }
  *K_out = n;
  return ALGDOCK_OK;
}

}  // extern "C"
