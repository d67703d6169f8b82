// Hamiltonian replica exchange ("Sampling", Eq. (repXacc)): sweeps of swap attempts between
// states 1..min(max_sep, K-1) apart, with the FP64 acceptance test.
//
// Within one (separation, colour) phase the pairs (a, a+s) with floor(a/s) % 2 == colour are
// disjoint, so a warp's lanes attempt them concurrently; phases follow one another in a fixed
// order, which makes the result a deterministic function of the components and the Philox
// counters.  The slot components do not change during the sweeps, so the energies a sweep reads
// are tabulated once per ladder before one warp runs the sweeps:
//  - ladders of up to 128 states (exchange_fast_kernel): FP32 energies shifted per slot, with a
//    bound on their rounding error, and the FP32 log-uniform of every attempt; the sweeping warp
//    keeps the ladder's configuration in registers and decides from the FP32 values wherever the
//    bound allows, otherwise by the FP64 test;
//  - up to 160 states (exchange_matrix_kernel): the FP64 u_k(x_i) of every state and slot;
//  - larger ladders (exchange_direct_kernel): FP64 energies per attempt.
// All three give the decisions of the same FP64 expression, bit for bit.
#include <math.h>

#include "internal.cuh"

namespace algdock {
namespace {

constexpr int kExMaxWarps = 4;
constexpr unsigned kFull = 0xffffffffu;
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

// The fast kernel: one block per ladder of at most kFastMaxK states.
constexpr int kFastMaxK = 128;     // four slots per lane of the sweeping warp
constexpr int kFastThreads = 640;  // twenty warps fill the tables, warp 0 sweeps
constexpr size_t kFastSmemMax = 220 * 1024;

// Shared-memory bytes of the fast kernel for a ladder of K states.
__host__ __device__ inline size_t fast_smem_bytes(int K, int n_sweeps, int max_sep) {
  const int smax = max_sep < K - 1 ? max_sep : K - 1;
  return (size_t)K * (3 * sizeof(double) + sizeof(SlotE)) +          // states and slots in FP64
         (size_t)K * 2 * sizeof(float4) +                             // FP32 state factors, centred slots
         (size_t)K * K * sizeof(float2) +                             // shifted u and its magnitude bound
         (size_t)n_sweeps * (smax > 0 ? smax : 1) * K * sizeof(float) +  // log-uniforms
         (size_t)max_sep * K * sizeof(unsigned) +                     // accept counters
         (size_t)2 * kFastMaxK * sizeof(int) +                        // the team sweep's slot buffers
         (size_t)n_sweeps * sizeof(int);                              // sweeps' log-uniforms ready
}

// The fast kernels' shared memory.
struct FastTables {
  double* st;     // [K][3]: beta, w_sg, w_g
  SlotE* slot;    // [K]
  float4* w;      // [K]: beta, beta w_sg, beta w_g
  float4* d;      // [K]: centred slot components
  float2* fm;     // [K][K]: v_k(x_i), m_k(x_i)
  float* lu;      // [n_sweeps][smax][K]
  unsigned* acc;  // [max_sep][K]
  int* cbuf;      // [2][kFastMaxK]: configurations published by the team sweep, by phase parity
  int* ready;     // [n_sweeps]: drawing warps done with each sweep's log-uniforms
};
__device__ inline FastTables fast_carve(unsigned char* smem, int K, int n_sweeps, int sm1, int max_sep) {
  FastTables T;
  T.st = (double*)smem;
  T.slot = (SlotE*)(T.st + 3 * K);
  T.w = (float4*)(T.slot + K);
  T.d = T.w + K;
  T.fm = (float2*)(T.d + K);
  T.lu = (float*)(T.fm + (size_t)K * K);
  T.acc = (unsigned*)(T.lu + (size_t)n_sweeps * sm1 * K);
  T.cbuf = (int*)(T.acc + (size_t)max_sep * K);
  T.ready = T.cbuf + 2 * kFastMaxK;
  return T;
}

// The FP64 test of one attempt (pair a, a + s of sweep sw; configurations x at a and y at a + s),
// for the decisions the FP32 estimate leaves open.  Out of line: it is rare, and one copy serves
// every unrolled phase of the sweep loop.
__device__ __noinline__ bool exact_swap(const ExArgs& A, const double* s_st, const SlotE* s_slot, uint32_t lid, int sw,
                                        int s, int a, int x, int y) {
  auto U = [&](int k, int i) { return reduced(s_st[3 * k], s_st[3 * k + 1], s_st[3 * k + 2], s_slot[i]); };
  const int b = a + s;
  double d = __dadd_rn(U(a, y), U(b, x));
  d = __dsub_rn(d, U(a, x));
  d = __dsub_rn(d, U(b, y));
  const U4 o = philox(A.seed, (uint32_t)((sw * A.max_sep + s - 1) * 65536 + a), lid, A.cycle, kPurposeExchange);
  return (d <= 0.0) || (uniform53(o.x, o.y) < exp(-d));
}

// One ladder per block.  The energy difference of a swap,
//   d = u_a(y) + u_b(x) - u_a(x) - u_b(y),
// is unchanged when a constant per state or per slot is subtracted from every u_k(x_i).  The
// block therefore tabulates, in FP32, v_k(x_i) = beta_k (e_i + w_sg,k psg_i + w_g,k pg_i) with each
// slot component taken relative to its minimum over the ladder (e = U_L + U_I), together with
// m_k(x_i) = |beta_k e_i| + |beta_k w_sg,k psg_i| + |beta_k w_g,k pg_i| in the same shifted
// variables.  Each entry is within 5 2^-24 m of the exact shifted value (one rounding of each
// centred component and each factor, three products, two sums), and the estimate of d from four
// entries within 7 2^-24 of the sum of their m.  With the FP32 log-uniform (error below 2e-5) a
// decision is taken from the estimate when its margin to the boundary ln u = -d exceeds
// 1e-4 + 1e-6 sum(m); otherwise from the FP64 test itself, so every decision is the FP64 one.
// The tables of one ladder are built by all threads of the block (ends with a block barrier).
// Attempt idx's FP32 log-uniform (idx = (sweep smax + s - 1) K + a: pair a, a + s of the sweep).
__device__ inline float log_uniform(const ExArgs& A, int idx, int K, int smax, uint32_t lid) {
  const int a = idx % K, ss = idx / K;
  const int s = ss % smax + 1, sw = ss / smax;
  if (a + s >= K) return 0.f;
  const U4 o = philox(A.seed, (uint32_t)((sw * A.max_sep + s - 1) * 65536 + a), lid, A.cycle, kPurposeExchange);
  // the 53-bit uniform (o.x >> 5) 2^-27 + (o.y >> 6) 2^-53 in FP32: two roundings, 1.2e-7
  // relative, as good as rounding the FP64 value; zero exactly when the uniform is zero
  const float uf = __fmaf_rn((float)(o.x >> 5), 7.450580596923828125e-9f, (float)(o.y >> 6) * 1.1102230246251565e-16f);
  return uf == 0.f ? -INFINITY : __logf(uf);
}

// The warps that do not sweep draw the log-uniforms of sweeps 1.. while the sweep runs, sweep by
// sweep; each publishes its share of a sweep by one shared-memory counter (after a block fence).
__device__ inline void draw_sweeps(const ExArgs& A, const FastTables& T, int K, int smax, uint32_t lid, int first_warp) {
  const int lane = threadIdx.x & 31, w = (threadIdx.x >> 5) - first_warp;
  const int n_w = (int)(blockDim.x >> 5) - first_warp;
  const int per = smax * K;
  for (int sw = 1; sw < A.n_sweeps; ++sw) {
    for (int idx = sw * per + 32 * w + lane; idx < (sw + 1) * per; idx += 32 * n_w)
      T.lu[idx] = log_uniform(A, idx, K, smax, lid);
    __syncwarp();
    __threadfence_block();
    if (lane == 0) atomicAdd(&T.ready[sw], 1);
  }
}

// Before sweep sw (>= 1): waits, bounded, until all n_w drawing warps have published its
// log-uniforms; if the wait runs out, the sweeping warp draws them itself (the same values).
__device__ inline void await_sweep(const ExArgs& A, const FastTables& T, int K, int smax, uint32_t lid, int sw,
                                   int n_w) {
  const volatile int* r = T.ready + sw;
  int spins = 0;
  while (*r < n_w && spins < (1 << 20)) {
    __nanosleep(64);
    ++spins;
  }
  __threadfence_block();
  if (*r < n_w) {
    const int per = smax * K;
    for (int idx = sw * per + (threadIdx.x & 31); idx < (sw + 1) * per; idx += 32)
      T.lu[idx] = log_uniform(A, idx, K, smax, lid);
    __syncwarp();
  }
}

__device__ inline void fast_tables(const ExArgs& A, const FastTables& T, int K, int smax, uint32_t lid,
                                   int n_drawn) {
  const int64_t l = blockIdx.x;
  const int lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const StateDev st = A.states[A.state_offset + k];
    T.st[3 * k] = st.beta;
    T.st[3 * k + 1] = st.w_sg;
    T.st[3 * k + 2] = st.w_g;
    T.w[k] = make_float4((float)st.beta, (float)(st.beta * st.w_sg), (float)(st.beta * st.w_g), 0.f);
    T.slot[k] = load_slot(A.comps + (l * K + k) * 4);
  }
  for (int i = threadIdx.x; i < A.max_sep * K; i += blockDim.x) T.acc[i] = 0u;
  for (int i = threadIdx.x; i < A.n_sweeps; i += blockDim.x) T.ready[i] = 0;
  // the log-uniforms of the first n_drawn sweeps; the team kernels draw the later sweeps' beside
  // the sweeps (draw_sweeps)
  const int n_first = min(n_drawn, A.n_sweeps) * smax * K;
  for (int idx = threadIdx.x; idx < n_first; idx += blockDim.x) T.lu[idx] = log_uniform(A, idx, K, smax, lid);
  __syncthreads();
  {  // every warp forms the minima (fmin skips NaN; a non-finite slot only sends its pairs to FP64)
    double me = INFINITY, msg = INFINITY, mg = INFINITY;
    for (int i = lane; i < K; i += 32) {
      me = fmin(me, T.slot[i].e);
      msg = fmin(msg, T.slot[i].psg);
      mg = fmin(mg, T.slot[i].pg);
    }
    for (int o = 16; o > 0; o >>= 1) {
      me = fmin(me, __shfl_xor_sync(kFull, me, o));
      msg = fmin(msg, __shfl_xor_sync(kFull, msg, o));
      mg = fmin(mg, __shfl_xor_sync(kFull, mg, o));
    }
    for (int i = threadIdx.x; i < K; i += blockDim.x)
      T.d[i] = make_float4((float)(T.slot[i].e - me), (float)(T.slot[i].psg - msg), (float)(T.slot[i].pg - mg), 0.f);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int k = e / K, i = e - k * K;
    const float4 w = T.w[k], d = T.d[i];
    const float t0 = w.x * d.x, t1 = w.y * d.y, t2 = w.z * d.z;
    T.fm[e] = make_float2((t0 + t1) + t2, (fabsf(t0) + fabsf(t1)) + fabsf(t2));
  }
  __syncthreads();
}

// Ladders of up to 32 states: warp 0 sweeps with the ladder's configuration in registers, slot
// k = 32 g + lane in register g.  In the phase (s, colour) a slot k is the lower member a of a
// pair when floor(k/s) has the colour's parity and k + s < K, the upper member b when it has the
// other parity and k >= s.  Each member reads its partner's configuration by a shuffle, then its
// own row's entry at that configuration and the partner's row at both configurations, so both
// members form d from the same four entries (FP32 addition commutes), take the same decision and
// update their own register.
template <int KG>
__global__ void __launch_bounds__(kFastThreads) exchange_fast_kernel(const ExArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = A.K;
  const int smax = min(A.max_sep, K - 1);
  const int sm1 = smax > 0 ? smax : 1;
  const FastTables T = fast_carve(smem_raw, K, A.n_sweeps, sm1, A.max_sep);
  const double* s_st = T.st;
  const SlotE* s_slot = T.slot;
  const float2* s_fm = T.fm;
  const float* s_lu = T.lu;
  unsigned* s_acc = T.acc;
  const int64_t l = blockIdx.x;
  const uint32_t lid = (uint32_t)(A.ladder_offset + l);
  const int lane = threadIdx.x & 31;
  // every sweep's log-uniforms first: beside a one-warp sweep the drawing warps gained nothing
  fast_tables(A, T, K, smax, lid, A.n_sweeps);
  if (threadIdx.x >= 32) return;
  int cfg[KG];
  float uo[KG], mo[KG];  // the entry of the slot's own state at its own configuration
  bool bad = false;
#pragma unroll
  for (int g = 0; g < KG; ++g) {
    const int k = 32 * g + lane;
    cfg[g] = k < K ? A.config_of[l * K + k] : 0;
    bad |= (unsigned)cfg[g] >= (unsigned)K;
  }
  if (__any_sync(kFull, bad)) return;  // not a list of slots 0..K-1: leave the ladder untouched
#pragma unroll
  for (int g = 0; g < KG; ++g) {
    const int k = 32 * g + lane;
    const float2 v = s_fm[(k < K ? k : 0) * K + cfg[g]];
    uo[g] = v.x;
    mo[g] = v.y;
  }
  // the lane's role in every phase: bit (2 (s - 1) + colour) KG + g of `lower` when its slot of
  // group g is the lower member of a pair, of `active` when it is either member
  uint64_t lower_bits = 0, active_bits = 0;
  for (int s = 1; s <= smax; ++s)
    for (int colour = 0; colour < 2; ++colour)
#pragma unroll
      for (int g = 0; g < KG; ++g) {
        const int k = 32 * g + lane;
        const bool own = (k / s) % 2 == colour;
        const bool lo = own && k + s < K, hi = !own && k >= s && k < K;
        const int bit = (2 * (s - 1) + colour) * KG + g;
        lower_bits |= (uint64_t)lo << bit;
        active_bits |= (uint64_t)(lo || hi) << bit;
      }
  for (int sw = 0; sw < A.n_sweeps; ++sw) {
    const float* lu_sw = s_lu + (size_t)sw * smax * K;
    uint32_t acc_bits = 0;  // bit (s - 1) KG + g: the pair whose lower member is this slot was accepted
    for (int s = 1; s <= smax; ++s) {
      const bool wrap_up = lane + s >= 32, wrap_dn = lane < s;
      const float* lu_s = lu_sw + (s - 1) * K;
#pragma unroll
      for (int colour = 0; colour < 2; ++colour) {
        const int ph = 2 * (s - 1) + colour;
        int cu[KG], cd[KG];
#pragma unroll
        for (int g = 0; g < KG; ++g) {
          cu[g] = __shfl_sync(kFull, cfg[g], (lane + s) & 31);
          cd[g] = __shfl_sync(kFull, cfg[g], (lane - s) & 31);
        }
        // every group's partner, table entries and log-uniform first, then the decisions: the loads
        // of all groups are in flight together
        bool act[KG], lo[KG];
        int pc[KG], own[KG], a[KG];
        float2 f_kp[KG], f_po[KG], f_pp[KG];
        float lu[KG];
#pragma unroll
        for (int g = 0; g < KG; ++g) {
          act[g] = (active_bits >> (ph * KG + g)) & 1u;
          lo[g] = (lower_bits >> (ph * KG + g)) & 1u;
          // the partner: state k + s (lower member) or k - s (upper member), holding configuration
          // pc; the other group's register where the partner's lane wraps (never for an active
          // slot at the first or last group)
          const int k = 32 * g + lane;
          const int vu = wrap_up ? cu[g + 1 < KG ? g + 1 : g] : cu[g];
          const int vd = wrap_dn ? cd[g > 0 ? g - 1 : 0] : cd[g];
          pc[g] = act[g] ? (lo[g] ? vu : vd) : 0;
          own[g] = act[g] ? cfg[g] : 0;
          const int ks = act[g] ? k : 0, ps = act[g] ? (lo[g] ? k + s : k - s) : 0;
          f_kp[g] = s_fm[ks * K + pc[g]];      // own state at the partner's configuration
          f_po[g] = s_fm[ps * K + own[g]];     // partner's state at this configuration
          f_pp[g] = s_fm[ps * K + pc[g]];      // partner's state at its own configuration
          a[g] = lo[g] ? k : k - s;
          lu[g] = lu_s[act[g] ? a[g] : 0];
        }
        bool acc[KG];
        unsigned open = 0u;  // groups whose decision needs the FP64 test
#pragma unroll
        for (int g = 0; g < KG; ++g) {
          // this member's half of d and the partner's, each formed from the same two entries on
          // both lanes (uo is the stored entry at the own configuration), added in either order
          const float df = (f_kp[g].x - uo[g]) + (f_po[g].x - f_pp[g].x);
          const float band = 1e-4f + 1e-6f * ((f_kp[g].y + mo[g]) + (f_po[g].y + f_pp[g].y));
          const bool sure_acc = lu[g] != -INFINITY && lu[g] < -df - band;
          const bool sure_rej = lu[g] != -INFINITY && lu[g] > -df + band;
          acc[g] = sure_acc;
          open |= (unsigned)(act[g] && !sure_acc && !sure_rej) << g;
        }
        if (__any_sync(kFull, open != 0u)) {  // close to the boundary, or not finite: the FP64 test itself
#pragma unroll
          for (int g = 0; g < KG; ++g)
            if ((open >> g) & 1u)
              acc[g] = exact_swap(A, s_st, s_slot, lid, sw, s, a[g], lo[g] ? own[g] : pc[g], lo[g] ? pc[g] : own[g]);
        }
#pragma unroll
        for (int g = 0; g < KG; ++g) {
          const bool take = acc[g] && act[g];
          cfg[g] = take ? pc[g] : cfg[g];
          uo[g] = take ? f_kp[g].x : uo[g];
          mo[g] = take ? f_kp[g].y : mo[g];
          acc_bits |= (uint32_t)(take && lo[g]) << ((s - 1) * KG + g);
        }
      }
    }
    while (acc_bits) {  // this sweep's accepts into the counters (one lane per lower member)
      const int bit = __ffs(acc_bits) - 1;
      acc_bits &= acc_bits - 1;
      s_acc[(bit / KG) * K + 32 * (bit % KG) + lane] += 1u;
    }
  }
  __syncwarp();
#pragma unroll
  for (int g = 0; g < KG; ++g) {
    const int k = 32 * g + lane;
    if (k >= K) continue;
    A.config_of[l * K + k] = cfg[g];
    if (A.state_of) A.state_of[l * K + cfg[g]] = A.state_offset + k;
  }
  for (int i = lane; i < A.max_sep * K; i += 32) {
    const int s = i / K + 1, a = i % K;
    if (A.attempts && s <= smax && a + s < K) atomicAdd((unsigned long long*)&A.attempts[i], (unsigned long long)A.n_sweeps);
    if (A.accepts && s_acc[i]) atomicAdd((unsigned long long*)&A.accepts[i], (unsigned long long)s_acc[i]);
  }
}

// The sweeps of a ladder of more than 32 states by a team of KG warps, warp w holding slot
// k = 32 w + lane in one register.  The roles, table entries and decisions are those of the
// single-warp sweep; what differs is how a member learns its partner's configuration: at every
// phase each warp publishes its slots' configurations to one of two shared-memory buffers
// (alternating by phase parity), the team meets at a named barrier, and each member reads its
// partner's entry.  A warp can reach the next phase's write only after every warp has passed the
// barrier of the current one, so the buffer it writes is no longer read.  Every team warp runs the
// same block-uniform loops with one barrier per phase, and none leaves before the end.
constexpr int kTeamBarrier = 1;
template <int KG>
__global__ void __launch_bounds__(kFastThreads) exchange_team_kernel(const ExArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = A.K;
  const int smax = min(A.max_sep, K - 1);
  const int sm1 = smax > 0 ? smax : 1;
  const FastTables T = fast_carve(smem_raw, K, A.n_sweeps, sm1, A.max_sep);
  const int64_t l = blockIdx.x;
  const uint32_t lid = (uint32_t)(A.ladder_offset + l);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  fast_tables(A, T, K, smax, lid, 1);
  const int k = 32 * warp + lane;
  int cfg = warp < KG && k < K ? A.config_of[l * K + k] : 0;
  const bool bad = warp < KG && k < K && (unsigned)cfg >= (unsigned)K;
  // not a list of slots 0..K-1: every thread leaves, the ladder untouched
  if (__syncthreads_or(bad)) return;
  if (warp >= KG) {
    if (smax > 0) draw_sweeps(A, T, K, smax, lid, KG);
    return;
  }
  const float2 own0 = T.fm[(k < K ? k : 0) * K + cfg];
  float uo = own0.x, mo = own0.y;
  // the slot's role in every phase: bit 2 (s - 1) + colour of `lower` / `active`
  uint32_t lower_bits = 0, active_bits = 0;
  for (int s = 1; s <= smax; ++s)
    for (int colour = 0; colour < 2; ++colour) {
      const bool own = (k / s) % 2 == colour;
      const bool lo = own && k + s < K, hi = !own && k >= s && k < K;
      lower_bits |= (uint32_t)lo << (2 * (s - 1) + colour);
      active_bits |= (uint32_t)(lo || hi) << (2 * (s - 1) + colour);
    }
  int phase = 0;
  for (int sw = 0; sw < A.n_sweeps; ++sw) {
    if (sw > 0 && smax > 0) await_sweep(A, T, K, smax, lid, sw, (int)(blockDim.x >> 5) - KG);
    const float* lu_sw = T.lu + (size_t)sw * smax * K;
    uint32_t acc_bits = 0;  // bit s - 1: the pair whose lower member is this slot was accepted
    for (int s = 1; s <= smax; ++s) {
      const float* lu_s = lu_sw + (s - 1) * K;
#pragma unroll
      for (int colour = 0; colour < 2; ++colour, ++phase) {
        int* buf = T.cbuf + (phase & 1) * kFastMaxK;
        buf[k] = cfg;
        asm volatile("bar.sync %0, %1;" ::"r"(kTeamBarrier), "r"(32 * KG) : "memory");
        const int ph = 2 * (s - 1) + colour;
        const bool act = (active_bits >> ph) & 1u;
        const bool lo = (lower_bits >> ph) & 1u;
        const int pslot = lo ? k + s : k - s;
        const int pc = act ? buf[pslot] : 0;
        const int ks = act ? k : 0, ps = act ? pslot : 0, own = act ? cfg : 0;
        const float2 f_kp = T.fm[ks * K + pc];   // own state at the partner's configuration
        const float2 f_po = T.fm[ps * K + own];  // partner's state at this configuration
        const float2 f_pp = T.fm[ps * K + pc];   // partner's state at its own configuration
        const int a = lo ? k : k - s;
        const float lu = lu_s[act ? a : 0];
        const float df = (f_kp.x - uo) + (f_po.x - f_pp.x);
        const float band = 1e-4f + 1e-6f * ((f_kp.y + mo) + (f_po.y + f_pp.y));
        const bool sure_acc = lu != -INFINITY && lu < -df - band;
        const bool sure_rej = lu != -INFINITY && lu > -df + band;
        bool acc = sure_acc;
        if (act && !sure_acc && !sure_rej)  // close to the boundary, or not finite: the FP64 test itself
          acc = exact_swap(A, T.st, T.slot, lid, sw, s, a, lo ? own : pc, lo ? pc : own);
        const bool take = acc && act;
        cfg = take ? pc : cfg;
        uo = take ? f_kp.x : uo;
        mo = take ? f_kp.y : mo;
        acc_bits |= (uint32_t)(take && lo) << (s - 1);
      }
    }
    while (acc_bits) {  // this sweep's accepts of the pairs this slot leads
      const int bit = __ffs(acc_bits) - 1;
      acc_bits &= acc_bits - 1;
      T.acc[bit * K + k] += 1u;
    }
  }
  if (k < K) {
    A.config_of[l * K + k] = cfg;
    if (A.state_of) A.state_of[l * K + cfg] = A.state_offset + k;
    for (int s = 1; s <= A.max_sep; ++s) {
      const int i = (s - 1) * K + k;
      if (A.attempts && s <= smax && k + s < K)
        atomicAdd((unsigned long long*)&A.attempts[i], (unsigned long long)A.n_sweeps);
      if (A.accepts && T.acc[i]) atomicAdd((unsigned long long*)&A.accepts[i], (unsigned long long)T.acc[i]);
    }
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
  if (K <= kFastMaxK && max_sep <= 8 && fast <= kFastSmemMax) {
    const int kg = (K + 31) / 32;
    void (*fn)(ExArgs) = kg == 1   ? exchange_fast_kernel<1>
                         : kg == 2 ? exchange_team_kernel<2>
                         : kg == 3 ? exchange_team_kernel<3>
                                   : exchange_team_kernel<4>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fast);
    if (e != cudaSuccess) return e;
    fn<<<n_ladders, kFastThreads, fast, s>>>(A);
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
