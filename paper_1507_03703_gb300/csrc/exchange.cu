// Hamiltonian replica exchange ("Sampling", Eq. (repXacc)): sweeps of swap attempts between
// states 1..min(max_sep, K-1) apart, with the FP64 acceptance test.
//
// Within one (separation, colour) phase the pairs (a, a+s) with floor(a/s) % 2 == colour are
// disjoint, so a warp's lanes attempt them concurrently; phases follow one another in a fixed
// order, which makes the result a deterministic function of the components and the Philox
// counters.  The slot components do not change during the sweeps, so for K <= 160 the reduced
// energies u_k(x_i) of every state and slot are computed once per ladder into shared memory
// (by all four warps of the ladder's block) before one warp runs the sweeps; larger ladders
// evaluate them per attempt.  Both give bit-identical decisions: the same FP64 expression.
#include <math.h>

#include "internal.cuh"

namespace algdock {
namespace {

constexpr int kExMaxWarps = 4;
constexpr int kMatrixMaxK = 160;  // K^2 doubles of shared memory

struct SlotE {
  double e, psg, pg;  // U_L + U_I, Psi_sg, Psi_g of one slot
};

// ((e + w_sg psg) + w_g pg) * beta, in that order and without contraction, a zero weight dropping
// its term: the same rounding as any other correct FP64 evaluation of that expression.
__device__ inline double reduced(double beta, double w_sg, double w_g, const SlotE& c) {
  double e = c.e;
  if (w_sg != 0.0) e = __dadd_rn(e, __dmul_rn(w_sg, c.psg));
  if (w_g != 0.0) e = __dadd_rn(e, __dmul_rn(w_g, c.pg));
  return __dmul_rn(beta, e);
}

// The test u < exp(-d) in FP64.  exp(-d) >= 1 > u whenever d <= 0.  Otherwise an FP32 estimate of
// ln u (error < 1e-5 absolute) decides every case more than 1e-3 away from the boundary ln u = -d;
// the rest (and u = 0) takes the FP64 exponential.  The decision is the FP64 one either way.
__device__ inline bool accept_swap(double d, double u) {
  if (d <= 0.0) return true;
  if (u == 0.0) return 0.0 < exp(-d);
  const float lu = __logf((float)u);
  const float md = (float)(-d);
  if (lu < md - 1e-3f) return true;
  if (lu > md + 1e-3f) return false;
  return u < exp(-d);
}

struct ExArgs {
  const StateDev* states;
  int n_ladders, K, state_offset;
  const double* comps;
  int32_t* config_of;
  int32_t* state_of;
  int n_sweeps, max_sep;
  uint64_t seed;
  uint32_t cycle;
  int64_t ladder_offset;
  int64_t* attempts;
  int64_t* accepts;
};

__device__ inline SlotE load_slot(const double* c) { return SlotE{__dadd_rn(c[0], c[1]), c[2], c[3]}; }

// The sweeps of one ladder by one warp.  U(a, i) returns u_a(x_i).
template <typename UFn>
__device__ inline void sweeps(const ExArgs& A, int64_t l, int* s_cfg, unsigned* s_cnt, UFn U) {
  const int K = A.K, lane = threadIdx.x & 31;
  const int smax = min(A.max_sep, K - 1);
  const uint32_t lid = (uint32_t)(A.ladder_offset + l);
  for (int sw = 0; sw < A.n_sweeps; ++sw) {
    for (int s = 1; s <= smax; ++s) {
      for (int colour = 0; colour < 2; ++colour) {
        for (int a = lane; a + s < K; a += 32) {
          if ((a / s) % 2 != colour) continue;
          const int b = a + s;
          const int xi = s_cfg[a], yi = s_cfg[b];
          const U4 o = philox(A.seed, (uint32_t)((sw * A.max_sep + s - 1) * 65536 + a), lid, A.cycle,
                              kPurposeExchange);
          double d = __dadd_rn(U(a, yi), U(b, xi));
          d = __dsub_rn(d, U(a, xi));
          d = __dsub_rn(d, U(b, yi));
          const bool acc = accept_swap(d, uniform53(o.x, o.y));
          s_cnt[(s - 1) * K + a] += 1u;
          if (acc) {
            s_cfg[a] = yi;
            s_cfg[b] = xi;
            s_cnt[(A.max_sep + s - 1) * K + a] += 1u;
          }
        }
        __syncwarp();
      }
    }
  }
}

__device__ inline void write_back(const ExArgs& A, int64_t l, const int* s_cfg, const unsigned* s_cnt) {
  const int K = A.K, lane = threadIdx.x & 31;
  for (int k = lane; k < K; k += 32) {
    A.config_of[l * K + k] = s_cfg[k];
    if (A.state_of) A.state_of[l * K + s_cfg[k]] = A.state_offset + k;
  }
  for (int i = lane; i < A.max_sep * K; i += 32) {
    if (A.attempts && s_cnt[i]) atomicAdd((unsigned long long*)&A.attempts[i], (unsigned long long)s_cnt[i]);
    const unsigned ac = s_cnt[A.max_sep * K + i];
    if (A.accepts && ac) atomicAdd((unsigned long long*)&A.accepts[i], (unsigned long long)ac);
  }
}

// Loads the ladder's configuration and clears its counters; false if config_of is not a list of
// slots 0..K-1 (then the ladder is left untouched).
__device__ inline bool load_ladder(const ExArgs& A, int64_t l, int* s_cfg, unsigned* s_cnt) {
  const int K = A.K, lane = threadIdx.x & 31;
  bool bad = false;
  for (int i = lane; i < K; i += 32) {
    s_cfg[i] = A.config_of[l * K + i];
    bad |= (unsigned)s_cfg[i] >= (unsigned)K;
  }
  for (int i = lane; i < 2 * A.max_sep * K; i += 32) s_cnt[i] = 0u;
  __syncwarp();
  return !__any_sync(0xffffffffu, bad);
}

// Shared-memory bytes of the fast kernel for a ladder of K states.
__host__ __device__ inline size_t fast_smem_bytes(int K, int n_sweeps, int max_sep) {
  const int smax = max_sep < K - 1 ? max_sep : K - 1;
  return (size_t)K * K * (sizeof(double) + sizeof(float)) +  // u in FP64 and FP32
         (size_t)n_sweeps * (smax > 0 ? smax : 1) * K * sizeof(float) +  // log-uniforms
         (size_t)2 * (smax > 0 ? smax : 1) * K * sizeof(int) +           // pair lists
         (size_t)K * (3 * sizeof(double) + sizeof(SlotE) + sizeof(int)) +   // states, slots, config
         (size_t)max_sep * K * sizeof(unsigned) + 64;                    // accept counters
}

// One ladder per block.  All warps fill u_k(x_i) (FP64, and its FP32 rounding), the pair list of
// every (separation, colour) phase and the FP32 log-uniform of every attempt; warp 0 then sweeps,
// deciding each attempt from the FP32 values when the margin to the boundary exceeds a bound on
// their rounding error, and otherwise exactly as the FP64 test.
__global__ void __launch_bounds__(kExMaxWarps * 32) exchange_fast_kernel(const ExArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = A.K;
  const int smax = min(A.max_sep, K - 1);
  const int sm1 = smax > 0 ? smax : 1;
  double* s_u = (double*)smem_raw;                       // [K][K]
  double* s_st = s_u + (size_t)K * K;                     // [K][3]
  SlotE* s_slot = (SlotE*)(s_st + 3 * K);                 // [K]
  float* s_uf = (float*)(s_slot + K);                     // [K][K]
  float* s_lu = s_uf + (size_t)K * K;                     // [n_sweeps][smax][K]
  int* s_pairs = (int*)(s_lu + (size_t)A.n_sweeps * sm1 * K);  // [smax][2][K/2+1]... stored [smax][2][K]
  int* s_cfg = s_pairs + 2 * sm1 * K;
  unsigned* s_acc = (unsigned*)(s_cfg + K);               // [max_sep][K]
  __shared__ int s_npairs[2 * 8];
  const int64_t l = blockIdx.x;
  const uint32_t lid = (uint32_t)(A.ladder_offset + l);
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const StateDev st = A.states[A.state_offset + k];
    s_st[3 * k] = st.beta;
    s_st[3 * k + 1] = st.w_sg;
    s_st[3 * k + 2] = st.w_g;
    s_slot[k] = load_slot(A.comps + (l * K + k) * 4);
  }
  if (threadIdx.x < 2 * smax) {  // pair list of phase (s, colour), ascending a
    const int s = threadIdx.x / 2 + 1, colour = threadIdx.x % 2;
    int n = 0;
    for (int a = 0; a + s < K; ++a)
      if ((a / s) % 2 == colour) s_pairs[(2 * (s - 1) + colour) * K + n++] = a;
    s_npairs[threadIdx.x] = n;
  }
  const int n_att = A.n_sweeps * smax * K;
  for (int idx = threadIdx.x; idx < n_att; idx += blockDim.x) {
    const int a = idx % K, ss = idx / K;
    const int s = ss % smax + 1, sw = ss / smax;
    float lu = 0.f;
    if (a + s < K) {
      const U4 o = philox(A.seed, (uint32_t)((sw * A.max_sep + s - 1) * 65536 + a), lid, A.cycle, kPurposeExchange);
      // the 53-bit uniform (o.x >> 5) 2^-27 + (o.y >> 6) 2^-53 in FP32: two roundings, 1.2e-7
      // relative, as good as rounding the FP64 value; zero exactly when the uniform is zero
      const float uf = __fmaf_rn((float)(o.x >> 5), 7.450580596923828125e-9f, (float)(o.y >> 6) * 1.1102230246251565e-16f);
      lu = uf == 0.f ? -INFINITY : __logf(uf);
    }
    s_lu[idx] = lu;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int k = e / K, i = e - k * K;
    const double v = reduced(s_st[3 * k], s_st[3 * k + 1], s_st[3 * k + 2], s_slot[i]);
    s_u[e] = v;
    s_uf[e] = (float)v;
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  bool bad = false;
  for (int i = lane; i < K; i += 32) {
    s_cfg[i] = A.config_of[l * K + i];
    bad |= (unsigned)s_cfg[i] >= (unsigned)K;
  }
  for (int i = lane; i < A.max_sep * K; i += 32) s_acc[i] = 0u;
  __syncwarp();
  if (__any_sync(0xffffffffu, bad)) return;  // not a list of slots 0..K-1: leave the ladder untouched
  for (int sw = 0; sw < A.n_sweeps; ++sw) {
    for (int s = 1; s <= smax; ++s) {
      // floor(p / s) = (p * inv_s) >> 16 exactly for p < 1024 and s <= 8
      const int inv_s = (65536 + s - 1) / s;
      for (int colour = 0; colour < 2; ++colour) {
        const int ph = 2 * (s - 1) + colour;
        const int np = s_npairs[ph];
        for (int p = lane; p < np; p += 32) {
          // the p-th pair of the phase, in the order of the list: blocks of s consecutive a whose
          // block index has the colour's parity
          const int t = (p * inv_s) >> 16;
          const int a = s * (colour + 2 * t) + (p - t * s), b = a + s;
          const int xi = s_cfg[a], yi = s_cfg[b];
          const float f1 = s_uf[a * K + yi], f2 = s_uf[b * K + xi], f3 = s_uf[a * K + xi], f4 = s_uf[b * K + yi];
          const float df = ((f1 + f2) - f3) - f4;
          // |df - d| <= 2^-22 (|f1| + |f2| + |f3| + |f4|) from the roundings; ln-uniform error < 2e-5
          const float band = 1e-3f + 1e-6f * (fabsf(f1) + fabsf(f2) + fabsf(f3) + fabsf(f4));
          const float lu = s_lu[((sw * smax) + (s - 1)) * K + a];
          bool acc;
          if (lu != -INFINITY && lu < -df - band) {
            acc = true;
          } else if (lu != -INFINITY && lu > -df + band) {
            acc = false;
          } else {  // close to the boundary, or not finite: the FP64 test itself
            double d = __dadd_rn(s_u[a * K + yi], s_u[b * K + xi]);
            d = __dsub_rn(d, s_u[a * K + xi]);
            d = __dsub_rn(d, s_u[b * K + yi]);
            const U4 o = philox(A.seed, (uint32_t)((sw * A.max_sep + s - 1) * 65536 + a), lid, A.cycle,
                                kPurposeExchange);
            acc = (d <= 0.0) || (uniform53(o.x, o.y) < exp(-d));
          }
          if (acc) {
            s_cfg[a] = yi;
            s_cfg[b] = xi;
            s_acc[(s - 1) * K + a] += 1u;
          }
        }
        __syncwarp();
      }
    }
  }
  for (int k = lane; k < K; k += 32) {
    A.config_of[l * K + k] = s_cfg[k];
    if (A.state_of) A.state_of[l * K + s_cfg[k]] = A.state_offset + k;
  }
  for (int i = lane; i < A.max_sep * K; i += 32) {
    const int s = i / K + 1, a = i % K;
    if (A.attempts && s <= smax && a + s < K) atomicAdd((unsigned long long*)&A.attempts[i], (unsigned long long)A.n_sweeps);
    if (A.accepts && s_acc[i]) atomicAdd((unsigned long long*)&A.accepts[i], (unsigned long long)s_acc[i]);
  }
}

// One ladder per block: all warps fill u[k][i], warp 0 sweeps.
__global__ void __launch_bounds__(kExMaxWarps * 32) exchange_matrix_kernel(const ExArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = A.K;
  double* s_u = (double*)smem_raw;  // [K][K]
  double* s_st = s_u + (size_t)K * K;  // [K][3]: beta, w_sg, w_g
  SlotE* s_slot = (SlotE*)(s_st + 3 * K);
  int* s_cfg = (int*)(s_slot + K);
  unsigned* s_cnt = (unsigned*)(s_cfg + K);
  const int64_t l = blockIdx.x;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const StateDev st = A.states[A.state_offset + k];
    s_st[3 * k] = st.beta;
    s_st[3 * k + 1] = st.w_sg;
    s_st[3 * k + 2] = st.w_g;
    s_slot[k] = load_slot(A.comps + (l * K + k) * 4);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int k = e / K, i = e - k * K;
    s_u[e] = reduced(s_st[3 * k], s_st[3 * k + 1], s_st[3 * k + 2], s_slot[i]);
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  if (!load_ladder(A, l, s_cfg, s_cnt)) return;
  sweeps(A, l, s_cfg, s_cnt, [&](int k, int i) { return s_u[k * K + i]; });
  write_back(A, l, s_cfg, s_cnt);
}

// Several ladders per block, one warp each, reduced energies per attempt (any K up to 1024).
__global__ void __launch_bounds__(kExMaxWarps * 32) exchange_direct_kernel(const ExArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = A.K;
  double* s_beta = (double*)smem_raw;
  double* s_wsg = s_beta + K;
  double* s_wg = s_wsg + K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_warps = blockDim.x >> 5;
  SlotE* s_slot = (SlotE*)(s_wg + K) + (size_t)warp * K;
  int* s_cfg = (int*)((SlotE*)(s_wg + K) + (size_t)n_warps * K) + (size_t)warp * K;
  unsigned* s_cnt = (unsigned*)((int*)((SlotE*)(s_wg + K) + (size_t)n_warps * K) + (size_t)n_warps * K) +
                    (size_t)warp * 2 * A.max_sep * K;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const StateDev st = A.states[A.state_offset + k];
    s_beta[k] = st.beta;
    s_wsg[k] = st.w_sg;
    s_wg[k] = st.w_g;
  }
  __syncthreads();
  const int64_t l = (int64_t)blockIdx.x * n_warps + warp;
  if (l >= A.n_ladders) return;
  for (int i = lane; i < K; i += 32) s_slot[i] = load_slot(A.comps + (l * K + i) * 4);
  if (!load_ladder(A, l, s_cfg, s_cnt)) return;
  sweeps(A, l, s_cfg, s_cnt,
         [&](int k, int i) { return reduced(s_beta[k], s_wsg[k], s_wg[k], s_slot[i]); });
  write_back(A, l, s_cfg, s_cnt);
}

}  // namespace

cudaError_t launch_exchange(cudaStream_t s, const algdock_ctx& c, int n_ladders, int K, int state_offset,
                            const double* comps, int32_t* config_of, int32_t* state_of, int n_sweeps, int max_sep,
                            uint64_t seed, uint64_t cycle, int64_t ladder_offset, int64_t* attempts,
                            int64_t* accepts) {
  if (n_ladders == 0) return cudaSuccess;
  ExArgs A{c.d_states, n_ladders, K, state_offset, comps, config_of, state_of, n_sweeps, max_sep, seed,
           (uint32_t)cycle, ladder_offset, attempts, accepts};
  const size_t counters = (size_t)2 * max_sep * K * sizeof(unsigned);
  const size_t fast = fast_smem_bytes(K, n_sweeps, max_sep);
  if (max_sep <= 8 && fast <= 200 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(exchange_fast_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fast);
    if (e != cudaSuccess) return e;
    exchange_fast_kernel<<<n_ladders, kExMaxWarps * 32, fast, s>>>(A);
    return cudaGetLastError();
  }
  if (K <= kMatrixMaxK) {
    const size_t smem = (size_t)K * K * sizeof(double) + (size_t)K * (3 * sizeof(double) + sizeof(SlotE) + sizeof(int)) +
                        counters;
    cudaError_t e = cudaFuncSetAttribute(exchange_matrix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    exchange_matrix_kernel<<<n_ladders, kExMaxWarps * 32, smem, s>>>(A);
    return cudaGetLastError();
  }
  const size_t fixed = (size_t)3 * K * sizeof(double);
  const size_t per_warp = (size_t)K * (sizeof(SlotE) + sizeof(int)) + counters;
  const size_t budget = 200 * 1024;
  // each ladder is a chain of dependent phases: spread the ladders over all SMs first
  int warps = n_ladders / (2 * 152);
  warps = warps < 1 ? 1 : (warps > kExMaxWarps ? kExMaxWarps : warps);
  while (warps > 1 && fixed + warps * per_warp > budget) --warps;
  if (fixed + warps * per_warp > budget) return cudaErrorInvalidValue;
  const size_t smem = fixed + warps * per_warp;
  cudaError_t e = cudaFuncSetAttribute(exchange_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int blocks = (n_ladders + warps - 1) / warps;
  exchange_direct_kernel<<<blocks, warps * 32, smem, s>>>(A);
  return cudaGetLastError();
}

}  // namespace algdock
