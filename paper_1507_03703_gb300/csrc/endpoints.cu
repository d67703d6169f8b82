// End-point corrections of the thermodynamic cycle: the receptor-ligand interaction of the target
// force field, computed directly ("Thermodynamic Cycle": the target force field evaluates
// receptor-ligand interactions directly, the sampling force field by grid interpolation), and the
// Zwanzig free energy perturbation that carries milestone samples into the target force field
// ("Estimation": f_AB and f_DE by free energy perturbation).
#include <math.h>

#include "internal.cuh"

namespace algdock {
namespace {

constexpr int kTIThreads = 128;                     // threads of a target-interaction block
constexpr int kTIPer = 4;                           // (configuration, atom) points per thread
constexpr int kTIPoints = kTIPer * kTIThreads;      // points per block
constexpr int kRecPairTile = 128;                   // receptor atom pairs staged per shared-memory tile
constexpr int kFepThreads = 256;
constexpr int kFepMaxBlocks = 2 * 152;

__device__ __forceinline__ float rcp_approx(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

// Each thread evaluates kTIPer (configuration, atom) points against every receptor atom, two
// receptor atoms per paired instruction.  A block holds whole configurations (spb of them,
// spb * na <= 512 points), so the per-configuration sums stay inside the block and are taken in a
// fixed order.  Receptor atoms j, j' = 2k, 2k + 1 (see ReceptorPair): x = x_hi + x_lo is the FP64
// coordinate, so that the difference (x_L - x_hi) - x_lo carries the rounding of the difference
// rather than of the coordinate.  Each term is FP32 (one approximate reciprocal; the floors of the
// attractive and electrostatic sums at 2 A are minima of the reciprocal powers, which equal the
// powers of max(r, 2)); a tile's terms are summed in FP32 and tiles in FP64.
__global__ void __launch_bounds__(kTIThreads) target_interaction_kernel(
    int64_t N, int na, int spb, const float* __restrict__ x, const TargetFactors* __restrict__ lig_fac,
    const ReceptorPair* __restrict__ rec, const float2* __restrict__ rec_q, int n_pairs, double* __restrict__ psi) {
  __shared__ ReceptorPair s_p[kRecPairTile];
  __shared__ float2 s_q[kRecPairTile];
  __shared__ double s_e[kTIPoints];
  const int tid = threadIdx.x;
  const int64_t s0 = (int64_t)blockIdx.x * spb;
  const int nsamp = (int)min((int64_t)spb, N - s0);
  const int npts = nsamp * na;
  const float* xb = x + 3 * (s0 * na);
  const float rmin2 = (float)(kRepulsiveMinDist * kRepulsiveMinDist);
  const float amin2_inv = (float)(1.0 / (kAttractiveMinDist * kAttractiveMinDist));
  const float amin6_inv = amin2_inv * amin2_inv * amin2_inv;
  f32x2 X[kTIPer], Y[kTIPer], Z[kTIPer];
  double dr[kTIPer], da[kTIPer], de[kTIPer];
#pragma unroll
  for (int k = 0; k < kTIPer; ++k) {
    const int p = tid + k * kTIThreads;
    const bool v = p < npts;
    const float a = v ? xb[3 * p] : 0.f, b = v ? xb[3 * p + 1] : 0.f, c = v ? xb[3 * p + 2] : 0.f;
    X[k] = pack2(a, a);
    Y[k] = pack2(b, b);
    Z[k] = pack2(c, c);
    dr[k] = da[k] = de[k] = 0.0;
  }
  for (int base = 0; base < n_pairs; base += kRecPairTile) {
    const int m = min(kRecPairTile, n_pairs - base);
    __syncthreads();
    for (int t = tid; t < m; t += kTIThreads) {
      s_p[t] = rec[base + t];
      s_q[t] = rec_q[base + t];
    }
    __syncthreads();
    f32x2 fr[kTIPer], fa[kTIPer], fe[kTIPer];
#pragma unroll
    for (int k = 0; k < kTIPer; ++k) fr[k] = fa[k] = fe[k] = 0ull;
#pragma unroll 2
    for (int t = 0; t < m; ++t) {
      const ReceptorPair R = s_p[t];
      const float2 q = s_q[t];
      const f32x2 hx = pack2(R.c0.x, R.c0.y), hy = pack2(R.c0.z, R.c0.w), hz = pack2(R.c1.x, R.c1.y);
      const f32x2 lx = pack2(R.c1.z, R.c1.w), ly = pack2(R.c2.x, R.c2.y), lz = pack2(R.c2.z, R.c2.w);
      const f32x2 A = pack2(R.c3.x, R.c3.y), B = pack2(R.c3.z, R.c3.w), Q = pack2(q.x, q.y);
#pragma unroll
      for (int k = 0; k < kTIPer; ++k) {
        const f32x2 dx = sub2(sub2(X[k], hx), lx), dy = sub2(sub2(Y[k], hy), ly), dz = sub2(sub2(Z[k], hz), lz);
        const f32x2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        float ra, rb;
        unpack2(r2, ra, rb);
        const float ia = rcp_approx(fmaxf(ra, rmin2)), ib = rcp_approx(fmaxf(rb, rmin2));
        const f32x2 i2 = pack2(ia, ib);
        const f32x2 i6 = mul2(mul2(i2, i2), i2);
        fr[k] = fma2(A, mul2(i6, i6), fr[k]);
        float sa, sb;
        unpack2(i6, sa, sb);
        fa[k] = fma2(B, pack2(fminf(sa, amin6_inv), fminf(sb, amin6_inv)), fa[k]);
        fe[k] = fma2(Q, pack2(fminf(ia, amin2_inv), fminf(ib, amin2_inv)), fe[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < kTIPer; ++k) {
      float a, b;
      unpack2(fr[k], a, b);
      dr[k] += (double)a + (double)b;
      unpack2(fa[k], a, b);
      da[k] += (double)a + (double)b;
      unpack2(fe[k], a, b);
      de[k] += (double)a + (double)b;
    }
  }
  // atom energy sqrt(A_i) LJr - sqrt(B_i) |LJa| + 332.0637 q_i elec
#pragma unroll
  for (int k = 0; k < kTIPer; ++k) {
    const int p = tid + k * kTIThreads;
    if (p < npts) {
      const TargetFactors f = lig_fac[p % na];
      s_e[p] = f.sA * dr[k] - f.sB * da[k] + f.qC * de[k];
    }
  }
  __syncthreads();
  for (int k = tid; k < nsamp; k += kTIThreads) {  // up to 512 configurations (one-atom ligands)
    double s = 0.0;
    for (int i = 0; i < na; ++i) s += s_e[k * na + i];
    psi[s0 + k] = s;
  }
}

// ------------------------------------------------------------------ FEP reduction
// Running log-sum-exp state of weights w = exp(-du): m = smallest du so far, s1 = sum exp(m - du),
// s2 = sum exp(2 (m - du)); m = +inf with s1 = s2 = 0 is the empty state.  du = +inf has weight 0;
// NaN and -inf are counted as invalid.
struct Lse {
  double m, s1, s2;
  int bad;
};

__device__ __forceinline__ void lse_add(Lse& a, double du) {
  if (isnan(du) || du == -INFINITY) {
    ++a.bad;
    return;
  }
  if (du == INFINITY) return;
  if (du < a.m) {
    const double r = a.s1 > 0.0 ? exp(du - a.m) : 0.0;
    a.s1 = a.s1 * r + 1.0;
    a.s2 = a.s2 * (r * r) + 1.0;
    a.m = du;
  } else {
    const double w = exp(a.m - du);
    a.s1 += w;
    a.s2 += w * w;
  }
}

__device__ __forceinline__ void lse_merge(Lse& a, const Lse& b) {
  a.bad += b.bad;
  if (!(b.s1 > 0.0)) return;
  if (!(a.s1 > 0.0)) {
    a.m = b.m;
    a.s1 = b.s1;
    a.s2 = b.s2;
    return;
  }
  const double m = fmin(a.m, b.m);
  const double ra = exp(m - a.m), rb = exp(m - b.m);
  a.s1 = a.s1 * ra + b.s1 * rb;
  a.s2 = a.s2 * (ra * ra) + b.s2 * (rb * rb);
  a.m = m;
}

__device__ __forceinline__ Lse lse_shfl_down(const Lse& a, int o) {
  Lse b;
  b.m = __shfl_down_sync(0xffffffffu, a.m, o);
  b.s1 = __shfl_down_sync(0xffffffffu, a.s1, o);
  b.s2 = __shfl_down_sync(0xffffffffu, a.s2, o);
  b.bad = __shfl_down_sync(0xffffffffu, a.bad, o);
  return b;
}

// Block-wide merge in a fixed tree; the result is valid in thread 0.
__device__ Lse lse_block(Lse a) {
  __shared__ Lse s_w[kFepThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    const Lse b = lse_shfl_down(a, o);
    lse_merge(a, b);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_w[warp] = a;
  __syncthreads();
  if (warp == 0) {
    a = lane < kFepThreads / 32 ? s_w[lane] : Lse{INFINITY, 0.0, 0.0, 0};
    for (int o = 16; o > 0; o >>= 1) {
      const Lse b = lse_shfl_down(a, o);
      lse_merge(a, b);
    }
  }
  return a;
}

// du_n = beta (u_t[n st] - u_s[n ss]) (u_s may be null: 0); each block merges a strided share.
__global__ void __launch_bounds__(kFepThreads) fep_partial_kernel(int64_t N, const double* __restrict__ ut, int64_t st,
                                                                  const double* __restrict__ us, int64_t ss,
                                                                  double beta, Lse* partial) {
  Lse a{INFINITY, 0.0, 0.0, 0};
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const double d = ut[n * st] - (us ? us[n * ss] : 0.0);
    lse_add(a, beta * d);
  }
  a = lse_block(a);
  if (threadIdx.x == 0) partial[blockIdx.x] = a;
}

// out: f, sigma, n_eff, du_min, invalid count (as a double).
__global__ void __launch_bounds__(kFepThreads) fep_final_kernel(int64_t N, int n_part, const Lse* __restrict__ partial,
                                                                double* out) {
  Lse a{INFINITY, 0.0, 0.0, 0};
  for (int b = threadIdx.x; b < n_part; b += blockDim.x) lse_merge(a, partial[b]);
  a = lse_block(a);
  if (threadIdx.x == 0) {
    const double n = (double)N;
    if (a.s1 > 0.0) {
      const double n_eff = a.s1 * a.s1 / a.s2;
      out[0] = a.m - log(a.s1 / n);
      out[1] = N > 1 ? sqrt(fmax(n / n_eff - 1.0, 0.0) / (n - 1.0)) : NAN;
      out[2] = n_eff;
    } else {
      out[0] = INFINITY;
      out[1] = NAN;
      out[2] = 0.0;
    }
    out[3] = a.m;
    out[4] = (double)a.bad;
  }
}

}  // namespace

int target_samples_per_block(int na) { return na > 0 ? kTIPoints / na : 0; }

cudaError_t launch_target_interaction(cudaStream_t s, int64_t N, int na, const float* x, const TargetFactors* lig_fac,
                                      const ReceptorPair* rec, const float2* rec_q, int n_pairs, double* psi) {
  if (N <= 0) return cudaSuccess;
  const int spb = target_samples_per_block(na);
  const int64_t blocks = (N + spb - 1) / spb;
  target_interaction_kernel<<<(unsigned)blocks, kTIThreads, 0, s>>>(N, na, spb, x, lig_fac, rec, rec_q, n_pairs,
                                                                   psi);
  return cudaGetLastError();
}

size_t fep_scratch_bytes() { return sizeof(Lse) * kFepMaxBlocks + 8 * sizeof(double); }

cudaError_t launch_fep(cudaStream_t s, int64_t N, const double* ut, int64_t st, const double* us, int64_t ss,
                       double beta, void* scratch, double* out_dev) {
  Lse* part = (Lse*)scratch;
  const int64_t want = (N + kFepThreads - 1) / kFepThreads;  // one sample per thread up to 304 blocks
  const int blocks = (int)max((int64_t)1, min(want, (int64_t)kFepMaxBlocks));
  fep_partial_kernel<<<blocks, kFepThreads, 0, s>>>(N, ut, st, us, ss, beta, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  fep_final_kernel<<<1, kFepThreads, 0, s>>>(N, blocks, part, out_dev);
  return cudaGetLastError();
}

}  // namespace algdock
