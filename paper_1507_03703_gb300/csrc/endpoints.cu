// End-point corrections of the thermodynamic cycle: the receptor-ligand interaction of the target
// force field, computed directly ("Thermodynamic Cycle": the target force field evaluates
// receptor-ligand interactions directly, the sampling force field by grid interpolation), and the
// Zwanzig free energy perturbation that carries milestone samples into the target force field
// ("Estimation": f_AB and f_DE by free energy perturbation).
#include <math.h>

#include "internal.cuh"

namespace algdock {
namespace {

constexpr int kTIThreads = 256;                     // threads of a target-interaction block
constexpr int kTIPoints = 2 * kTIThreads;           // (sample, atom) points per block, two per thread
constexpr int kRecTile = 256;                       // receptor atoms staged per shared-memory tile
constexpr int kFepThreads = 256;
constexpr int kFepMaxBlocks = 2 * 152;

__device__ __forceinline__ float rcp_approx(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

// One thread evaluates two (sample, atom) points against every receptor atom.  A block holds whole
// samples (spb of them, spb * na <= 512 points), so the per-sample sums stay inside the block and
// are taken in a fixed order.  Receptor atom j: a[j] = (x_hi, y_hi, z_hi, sqrt(A_j)), b[j] = (x_lo,
// y_lo, z_lo, sqrt(B_j)), q[j] = q_j / 4, with x = x_hi + x_lo the FP64 coordinate, so that the
// difference (x_L - x_hi) - x_lo carries the rounding of the difference rather than of the
// coordinate.  Each term is FP32 (one approximate reciprocal; the attractive and electrostatic
// floors at 2 A reuse it); a tile's terms are summed in FP32 and tiles in FP64.
__global__ void __launch_bounds__(kTIThreads) target_interaction_kernel(
    int64_t N, int na, int spb, const float* __restrict__ x, const TargetFactors* __restrict__ lig_fac,
    const float4* __restrict__ rec_a, const float4* __restrict__ rec_b, const float* __restrict__ rec_q, int n_rec,
    double* __restrict__ psi) {
  __shared__ float4 s_a[kRecTile];
  __shared__ float4 s_b[kRecTile];
  __shared__ float s_q[kRecTile];
  __shared__ double s_e[kTIPoints];
  const int tid = threadIdx.x;
  const int64_t s0 = (int64_t)blockIdx.x * spb;
  const int nsamp = (int)min((int64_t)spb, N - s0);
  const int npts = nsamp * na;
  const int p0 = tid, p1 = tid + kTIThreads;
  const bool v0 = p0 < npts, v1 = p1 < npts;
  const float* xb = x + 3 * (s0 * na);
  const float x0 = v0 ? xb[3 * p0] : 0.f, y0 = v0 ? xb[3 * p0 + 1] : 0.f, z0 = v0 ? xb[3 * p0 + 2] : 0.f;
  const float x1 = v1 ? xb[3 * p1] : 0.f, y1 = v1 ? xb[3 * p1 + 1] : 0.f, z1 = v1 ? xb[3 * p1 + 2] : 0.f;
  const float rmin2 = (float)(kRepulsiveMinDist * kRepulsiveMinDist);
  const float amin2 = (float)(kAttractiveMinDist * kAttractiveMinDist);
  const float amin2_inv = 1.0f / amin2;
  const float amin6_inv = amin2_inv * amin2_inv * amin2_inv;
  double r0 = 0.0, a0 = 0.0, e0 = 0.0, r1 = 0.0, a1 = 0.0, e1 = 0.0;
  for (int base = 0; base < n_rec; base += kRecTile) {
    const int m = min(kRecTile, n_rec - base);
    __syncthreads();
    for (int t = tid; t < m; t += kTIThreads) {
      s_a[t] = rec_a[base + t];
      s_b[t] = rec_b[base + t];
      s_q[t] = rec_q[base + t];
    }
    __syncthreads();
    float fr0 = 0.f, fa0 = 0.f, fe0 = 0.f, fr1 = 0.f, fa1 = 0.f, fe1 = 0.f;
#pragma unroll 4
    for (int t = 0; t < m; ++t) {
      const float4 A = s_a[t];
      const float4 B = s_b[t];
      const float Q = s_q[t];
      {
        const float dx = (x0 - A.x) - B.x, dy = (y0 - A.y) - B.y, dz = (z0 - A.z) - B.z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float i2 = rcp_approx(fmaxf(r2, rmin2));
        const float i6 = i2 * i2 * i2;
        const bool far = r2 >= amin2;
        fr0 = fmaf(A.w, i6 * i6, fr0);
        fa0 = fmaf(B.w, far ? i6 : amin6_inv, fa0);
        fe0 = fmaf(Q, far ? i2 : amin2_inv, fe0);
      }
      {
        const float dx = (x1 - A.x) - B.x, dy = (y1 - A.y) - B.y, dz = (z1 - A.z) - B.z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float i2 = rcp_approx(fmaxf(r2, rmin2));
        const float i6 = i2 * i2 * i2;
        const bool far = r2 >= amin2;
        fr1 = fmaf(A.w, i6 * i6, fr1);
        fa1 = fmaf(B.w, far ? i6 : amin6_inv, fa1);
        fe1 = fmaf(Q, far ? i2 : amin2_inv, fe1);
      }
    }
    r0 += (double)fr0;
    a0 += (double)fa0;
    e0 += (double)fe0;
    r1 += (double)fr1;
    a1 += (double)fa1;
    e1 += (double)fe1;
  }
  // atom energy sqrt(A_i) LJr - sqrt(B_i) |LJa| + 332.0637 q_i elec
  if (v0) {
    const TargetFactors f = lig_fac[p0 % na];
    s_e[p0] = f.sA * r0 - f.sB * a0 + f.qC * e0;
  }
  if (v1) {
    const TargetFactors f = lig_fac[p1 % na];
    s_e[p1] = f.sA * r1 - f.sB * a1 + f.qC * e1;
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
                                      const float4* rec_a, const float4* rec_b, const float* rec_q, int n_rec,
                                      double* psi) {
  if (N <= 0) return cudaSuccess;
  const int spb = target_samples_per_block(na);
  const int64_t blocks = (N + spb - 1) / spb;
  target_interaction_kernel<<<(unsigned)blocks, kTIThreads, 0, s>>>(N, na, spb, x, lig_fac, rec_a, rec_b, rec_q,
                                                                   n_rec, psi);
  return cudaGetLastError();
}

size_t fep_scratch_bytes() { return sizeof(Lse) * kFepMaxBlocks + 8 * sizeof(double); }

cudaError_t launch_fep(cudaStream_t s, int64_t N, const double* ut, int64_t st, const double* us, int64_t ss,
                       double beta, void* scratch, double* out_dev) {
  Lse* part = (Lse*)scratch;
  const int64_t want = (N + 4 * kFepThreads - 1) / (4 * kFepThreads);
  const int blocks = (int)max((int64_t)1, min(want, (int64_t)kFepMaxBlocks));
  fep_partial_kernel<<<blocks, kFepThreads, 0, s>>>(N, ut, st, us, ss, beta, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  fep_final_kernel<<<1, kFepThreads, 0, s>>>(N, blocks, part, out_dev);
  return cudaGetLastError();
}

}  // namespace algdock
