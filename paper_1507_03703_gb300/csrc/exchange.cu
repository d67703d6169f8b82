// Hamiltonian replica exchange ("Sampling", Eq. (repXacc)): sweeps of swap attempts between
// states 1..min(max_sep, K-1) apart, with the FP64 acceptance test.
//
// One warp per ladder.  Within one (separation, colour) phase the pairs (a, a+s) with
// floor(a/s) % 2 == colour are disjoint, so the lanes attempt them concurrently; phases follow
// one another in a fixed order, which is what makes the result a deterministic function of the
// components and the Philox counters.
#include <math.h>

#include "internal.cuh"

namespace algdock {
namespace {

constexpr int kExMaxWarps = 4;

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

__global__ void __launch_bounds__(kExMaxWarps * 32) exchange_kernel(const ExArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = A.K;
  // per block: state table (beta, w_sg, w_g) then per warp: slots, config, counters
  double* s_beta = (double*)smem_raw;
  double* s_wsg = s_beta + K;
  double* s_wg = s_wsg + K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_warps = blockDim.x >> 5;
  const int smax = min(A.max_sep, K - 1);
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
  for (int i = lane; i < K; i += 32) {
    const double* c = A.comps + (l * K + i) * 4;
    s_slot[i] = SlotE{__dadd_rn(c[0], c[1]), c[2], c[3]};
    s_cfg[i] = A.config_of[l * K + i];
  }
  for (int i = lane; i < 2 * A.max_sep * K; i += 32) s_cnt[i] = 0u;
  bool bad = false;
  for (int i = lane; i < K; i += 32) bad |= (unsigned)s_cfg[i] >= (unsigned)K;
  if (__any_sync(0xffffffffu, bad)) return;  // not a permutation of 0..K-1: leave the ladder untouched
  __syncwarp();
  const uint32_t lid = (uint32_t)(A.ladder_offset + l);
  for (int sw = 0; sw < A.n_sweeps; ++sw) {
    for (int s = 1; s <= smax; ++s) {
      for (int colour = 0; colour < 2; ++colour) {
        for (int a = lane; a + s < K; a += 32) {
          if ((a / s) % 2 != colour) continue;
          const int b = a + s;
          const int xi = s_cfg[a], yi = s_cfg[b];
          const SlotE X = s_slot[xi], Y = s_slot[yi];
          double d = __dadd_rn(reduced(s_beta[a], s_wsg[a], s_wg[a], Y), reduced(s_beta[b], s_wsg[b], s_wg[b], X));
          d = __dsub_rn(d, reduced(s_beta[a], s_wsg[a], s_wg[a], X));
          d = __dsub_rn(d, reduced(s_beta[b], s_wsg[b], s_wg[b], Y));
          const U4 o = philox(A.seed, (uint32_t)((sw * A.max_sep + s - 1) * 65536 + a), lid, A.cycle,
                              kPurposeExchange);
          const double u = uniform53(o.x, o.y);
          // The test u < exp(-d) in FP64.  exp(-d) >= 1 > u whenever d <= 0.  Otherwise an FP32
          // estimate of ln u (error < 1e-5 absolute) decides every case more than 1e-3 away from
          // the boundary ln u = -d; the rest takes the FP64 exponential.  The decision is the FP64
          // one either way.
          bool acc;
          if (d <= 0.0) {
            acc = true;
          } else if (u == 0.0) {
            acc = 0.0 < exp(-d);
          } else {
            const float lu = __logf((float)u);
            const float md = (float)(-d);
            if (lu < md - 1e-3f) acc = true;
            else if (lu > md + 1e-3f) acc = false;
            else acc = u < exp(-d);
          }
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

}  // namespace

cudaError_t launch_exchange(cudaStream_t s, const algdock_ctx& c, int n_ladders, int K, int state_offset,
                            const double* comps, int32_t* config_of, int32_t* state_of, int n_sweeps, int max_sep,
                            uint64_t seed, uint64_t cycle, int64_t ladder_offset, int64_t* attempts,
                            int64_t* accepts) {
  if (n_ladders == 0) return cudaSuccess;
  ExArgs A{c.d_states, n_ladders, K, state_offset, comps, config_of, state_of, n_sweeps, max_sep, seed,
           (uint32_t)cycle, ladder_offset, attempts, accepts};
  const size_t fixed = (size_t)3 * K * sizeof(double);
  const size_t per_warp = (size_t)K * (sizeof(SlotE) + sizeof(int)) + (size_t)2 * max_sep * K * sizeof(unsigned);
  const size_t budget = 200 * 1024;
  // Each ladder is a chain of dependent phases, so the launch is latency-bound: spread the
  // ladders over all SMs first (one warp per block until there are two blocks per SM).
  int warps = n_ladders / (2 * 152);
  warps = warps < 1 ? 1 : (warps > kExMaxWarps ? kExMaxWarps : warps);
  while (warps > 1 && fixed + warps * per_warp > budget) --warps;
  if (fixed + warps * per_warp > budget) return cudaErrorInvalidValue;
  const size_t smem = fixed + warps * per_warp;
  cudaError_t e = cudaFuncSetAttribute(exchange_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int blocks = (n_ladders + warps - 1) / warps;
  exchange_kernel<<<blocks, warps * 32, smem, s>>>(A);
  return cudaGetLastError();
}

}  // namespace algdock
