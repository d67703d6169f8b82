// Learned pose proposal: an extension of the paper's external-coordinate Monte Carlo moves
// ("Sampling": random rotation about the centre of mass plus Gaussian translation, Metropolis
// test).  A network proposes rigid-body and torsion increments; the involutive move
// Apply(x, d) = Rigid(d_r/2) . Tor(d_tau) . Rigid(d_r/2) (Apply(Apply(x, d), -d) = x, unit
// Jacobian) is accepted with min(1, exp(-(u(x') - u(x))) q(-d|x') / q(d|x)).
//
// The network (64 -> 256 -> 256 -> 256 -> 360, ReLU) runs on the tensor cores: a BF16 mma.sync
// GEMM with FP32 accumulation and fused epilogues (bias + ReLU to BF16, bias to FP32, ReLU mask of
// the backward pass).  Training uses the same GEMM for the weight and input gradients.
#include <cuda_bf16.h>
#include <math.h>

#include <vector>

#include "internal.cuh"

namespace algdock {
namespace {

using bf16 = __nv_bfloat16;

constexpr int NFEAT = 64, NHID = 256, NOUT = 360, DMAX = 22, NCOMP = 8;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NHID * NFEAT, OFF_W2 = OFF_B1 + NHID, OFF_B2 = OFF_W2 + NHID * NHID,
              OFF_W3 = OFF_B2 + NHID, OFF_B3 = OFF_W3 + NHID * NHID, OFF_W4 = OFF_B3 + NHID,
              OFF_B4 = OFF_W4 + NOUT * NHID, NPARAMS = OFF_B4 + NOUT;
constexpr int WOFF_1 = 0, WOFF_2 = WOFF_1 + NHID * NFEAT, WOFF_3 = WOFF_2 + NHID * NHID, WOFF_4 = WOFF_3 + NHID * NHID,
              NWEIGHTS = WOFF_4 + NOUT * NHID;
constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kPurposeLearned = 4;
static_assert(NPARAMS == ALGDOCK_MLP_NPARAMS && NWEIGHTS == ALGDOCK_MLP_NWEIGHTS, "parameter layout");

// ------------------------------------------------------------------ BF16 tensor-core GEMM
// C[m][n] = epi(sum_k A(m, k) B(n, k)), A(m, k) = A_T ? A[k * lda + m] : A[m * lda + k], likewise B.
enum Epi { EPI_F32 = 0, EPI_F32_BIAS = 1, EPI_RELU_BF16 = 2, EPI_MASK_BF16 = 3 };

__device__ inline float ld_f(const float* p) { return *p; }
__device__ inline float ld_f(const bf16* p) { return __bfloat162float(*p); }

__device__ inline void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int GT = 64;   // block tile in M and N
constexpr int GK = 32;   // K step
constexpr int GP = 40;   // padded row length of the shared tiles (bf16 elements)

// Eight consecutive elements (from a 16-byte aligned address) as BF16 pairs.
__device__ inline uint4 load8(const bf16* p) { return *(const uint4*)p; }
__device__ inline uint4 load8(const float* p) {
  const float4 a = *(const float4*)p, b = *(const float4*)(p + 4);
  __nv_bfloat162 h0 = __floats2bfloat162_rn(a.x, a.y), h1 = __floats2bfloat162_rn(a.z, a.w);
  __nv_bfloat162 h2 = __floats2bfloat162_rn(b.x, b.y), h3 = __floats2bfloat162_rn(b.z, b.w);
  return make_uint4(*(uint32_t*)&h0, *(uint32_t*)&h1, *(uint32_t*)&h2, *(uint32_t*)&h3);
}

// Rows r0 .. r0+63, columns k0 .. k0+31 of a row-major matrix into a shared tile, 8 elements per
// 16-byte load where the row stride allows it, element by element at the edges.
template <typename T>
__device__ inline void load_rows(bf16 (&S)[GT][GP], const T* __restrict__ X, int ld, int r0, int R, int k0, int K,
                                 int tid) {
  const bool vec = (ld % 8) == 0 && (((uintptr_t)X) & 15) == 0;
  for (int e = tid; e < GT * (GK / 8); e += 128) {
    const int rr = e / (GK / 8), kk = (e % (GK / 8)) * 8;
    const int gr = r0 + rr, gk = k0 + kk;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gr < R) {
      if (vec && gk + 8 <= K) {
        v = load8(X + (size_t)gr * ld + gk);
      } else {
        __nv_bfloat16 h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) h[j] = __float2bfloat16(gk + j < K ? ld_f(X + (size_t)gr * ld + gk + j) : 0.f);
        v = *(uint4*)h;
      }
    }
    *(uint4*)&S[rr][kk] = v;
  }
}

template <typename TA, bool A_T, typename TB, bool B_T, int EPI>
__global__ void __launch_bounds__(128) gemm_kernel(int M, int N, int K, const TA* __restrict__ A, int lda,
                                                   const TB* __restrict__ B, int ldb, void* C, int ldc,
                                                   const float* __restrict__ bias, const bf16* __restrict__ mask,
                                                   int ldm) {
  __shared__ __align__(16) bf16 As[GT][GP];
  __shared__ __align__(16) bf16 Bs[GT][GP];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, t = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
  for (int k0 = 0; k0 < K; k0 += GK) {
    if (A_T) {
      for (int e = tid; e < GT * GK; e += 128) {
        const int kk = e / GT, mm = e % GT;
        const int gm = m0 + mm, gk = k0 + kk;
        const float v = (gm < M && gk < K) ? ld_f(A + (size_t)gk * lda + gm) : 0.f;
        As[mm][kk] = __float2bfloat16(v);
      }
    } else {
      load_rows(As, A, lda, m0, M, k0, K, tid);
    }
    if (B_T) {
      for (int e = tid; e < GT * GK; e += 128) {
        const int kk = e / GT, nn = e % GT;
        const int gn = n0 + nn, gk = k0 + kk;
        const float w = (gn < N && gk < K) ? ld_f(B + (size_t)gk * ldb + gn) : 0.f;
        Bs[nn][kk] = __float2bfloat16(w);
      }
    } else {
      load_rows(Bs, B, ldb, n0, N, k0, K, tid);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; kk += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r = wm + 16 * mi + g;
        a[mi][0] = *(const uint32_t*)&As[r][kk + 2 * t];
        a[mi][1] = *(const uint32_t*)&As[r + 8][kk + 2 * t];
        a[mi][2] = *(const uint32_t*)&As[r][kk + 2 * t + 8];
        a[mi][3] = *(const uint32_t*)&As[r + 8][kk + 2 * t + 8];
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int cidx = wn + 8 * ni + g;
        b[ni][0] = *(const uint32_t*)&Bs[cidx][kk + 2 * t];
        b[ni][1] = *(const uint32_t*)&Bs[cidx][kk + 2 * t + 8];
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], a[mi], b[ni]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int row = m0 + wm + 16 * mi + g + (e >= 2 ? 8 : 0);
        const int col = n0 + wn + 8 * ni + 2 * t + (e & 1);
        if (row >= M || col >= N) continue;
        float v = acc[mi][ni][e];
        if (EPI == EPI_F32_BIAS || EPI == EPI_RELU_BF16) v += bias[col];
        if (EPI == EPI_F32 || EPI == EPI_F32_BIAS) {
          ((float*)C)[(size_t)row * ldc + col] = v;
        } else if (EPI == EPI_RELU_BF16) {
          ((bf16*)C)[(size_t)row * ldc + col] = __float2bfloat16(v > 0.f ? v : 0.f);
        } else {
          const float h = __bfloat162float(mask[(size_t)row * ldm + col]);
          ((bf16*)C)[(size_t)row * ldc + col] = __float2bfloat16(h > 0.f ? v : 0.f);
        }
      }
}

template <typename TA, bool A_T, typename TB, bool B_T, int EPI>
cudaError_t gemm(cudaStream_t s, int M, int N, int K, const TA* A, int lda, const TB* B, int ldb, void* C, int ldc,
                 const float* bias = nullptr, const bf16* mask = nullptr, int ldm = 0) {
  if (M == 0 || N == 0) return cudaSuccess;
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
  gemm_kernel<TA, A_T, TB, B_T, EPI><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, mask, ldm);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ small kernels
// Column sums of G [M][N] into out[n] (bias gradients), scaled.
template <typename T>
__global__ void colsum_kernel(int M, int N, const T* __restrict__ G, float scale, float* out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += ld_f(G + (size_t)m * N + n);
  out[n] = scale * s;
}

__global__ void to_bf16_kernel(int64_t n, const float* __restrict__ in, bf16* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __float2bfloat16(in[i]);
}

// Weight entries (not biases) of the parameter vector, in the order of the BF16 copy.
__device__ inline int weight_index(int p) {
  if (p < OFF_B1) return WOFF_1 + p;
  if (p >= OFF_W2 && p < OFF_B2) return WOFF_2 + (p - OFF_W2);
  if (p >= OFF_W3 && p < OFF_B3) return WOFF_3 + (p - OFF_W3);
  if (p >= OFF_W4 && p < OFF_B4) return WOFF_4 + (p - OFF_W4);
  return -1;
}

__global__ void adam_kernel(float* params, bf16* wbf16, const float* __restrict__ grad, float* m, float* v, float lr,
                            float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAMS) return;
  const float gr = grad[p];
  const float mm = 0.9f * m[p] + 0.1f * gr;
  const float vv = 0.999f * v[p] + 0.001f * gr * gr;
  m[p] = mm;
  v[p] = vv;
  const float w = params[p] - lr * (mm * c1) / (sqrtf(vv * c2) + 1e-8f);
  params[p] = w;
  const int wi = weight_index(p);
  if (wi >= 0) wbf16[wi] = __float2bfloat16(w);
}

// log sigma of a mixture output
__device__ inline double log_sigma(float raw) { return -2.0 + 4.0 * tanh((double)raw / 4.0); }

// Per component c: log w_c + sum_d log N(delta_d; mu, sigma) over D dims (FP64).
__device__ inline double component_logp(const float* o, int D, const float* dl, int c, double logz) {
  double s = (double)o[c] - logz;
  for (int d = 0; d < D; ++d) {
    const double mu = o[NCOMP + c * DMAX + d];
    const double ls = log_sigma(o[NCOMP + NCOMP * DMAX + c * DMAX + d]);
    const double z = ((double)dl[d] - mu) * exp(-ls);
    s += -0.5 * z * z - ls - 0.9189385332046728;  // 0.5 ln(2 pi)
  }
  return s;
}

__device__ inline double logits_lse(const float* o) {
  double m = -INFINITY;
  for (int c = 0; c < NCOMP; ++c) m = fmax(m, (double)o[c]);
  double z = 0.0;
  for (int c = 0; c < NCOMP; ++c) z += exp((double)o[c] - m);
  return m + log(z);
}

// Mean negative log-density of the targets: per row, the gradient -(1/N) dlogq/do (FP32) and
// the row's -log q.
__global__ void nll_kernel(int64_t N, int D, const float* __restrict__ out, const float* __restrict__ delta,
                           float* dout, float* loss_rows) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const float* o = out + n * NOUT;
  const float* dl = delta + n * DMAX;
  float* g = dout + n * NOUT;
  const double logz = logits_lse(o);
  double lp[NCOMP];
  double m = -INFINITY;
  for (int c = 0; c < NCOMP; ++c) {
    lp[c] = component_logp(o, D, dl, c, logz);
    m = fmax(m, lp[c]);
  }
  double ss = 0.0;
  for (int c = 0; c < NCOMP; ++c) ss += exp(lp[c] - m);
  const double lq = m + log(ss);
  const double scale = -1.0 / (double)N;
  for (int i = 0; i < NOUT; ++i) g[i] = 0.f;
  for (int c = 0; c < NCOMP; ++c) {
    const double r = exp(lp[c] - lq);
    // d logq / d logit_c' = r_c' - softmax_c' (summed over c below)
    g[c] += (float)(scale * (r - exp((double)o[c] - logz)));
    for (int d = 0; d < D; ++d) {
      const double mu = o[NCOMP + c * DMAX + d];
      const float raw = o[NCOMP + NCOMP * DMAX + c * DMAX + d];
      const double th = tanh((double)raw / 4.0);
      const double sg = exp(-2.0 + 4.0 * th);
      const double z = ((double)dl[d] - mu) / sg;
      g[NCOMP + c * DMAX + d] = (float)(scale * r * z / sg);
      g[NCOMP + NCOMP * DMAX + c * DMAX + d] = (float)(scale * r * (z * z - 1.0) * (1.0 - th * th));
    }
  }
  loss_rows[n] = (float)(-lq);
}

__global__ void sum_kernel(int64_t N, const float* __restrict__ x, float scale, float* out) {
  __shared__ float sh[256];
  float s = 0.f;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += x[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = scale * sh[0];
}

// ------------------------------------------------------------------ features, targets
struct PoseArgs {
  LigandLayout LL;
  const uint32_t* blob;
  LearnedTopo topo;
};

__device__ inline float atom_mass(const PoseArgs& P, int i) { return ((const float4*)(P.blob + P.LL.off_atom_b))[i].z; }

__global__ void features_kernel(int64_t N, const PoseArgs P, const StateDev* __restrict__ states, int n_states,
                                const int32_t* __restrict__ state_of, const float* __restrict__ x,
                                const double* __restrict__ comps, float* feat) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int na = P.LL.na;
  const float* xn = x + n * na * 3;
  float* f = feat + n * NFEAT;
  for (int i = 0; i < NFEAT; ++i) f[i] = 0.f;
  float cx = 0.f, cy = 0.f, cz = 0.f;
  for (int i = 0; i < na; ++i) {
    const float m = atom_mass(P, i);
    cx += m * xn[3 * i];
    cy += m * xn[3 * i + 1];
    cz += m * xn[3 * i + 2];
  }
  const float invM = 1.f / P.LL.total_mass;
  cx *= invM;
  cy *= invM;
  cz *= invM;
  f[0] = (cx - P.LL.site[0]) / P.LL.d0;
  f[1] = (cy - P.LL.site[1]) / P.LL.d0;
  f[2] = (cz - P.LL.site[2]) / P.LL.d0;
  const int ref[2] = {0, na - 1};
  for (int r = 0; r < 2; ++r) {
    const float vx = xn[3 * ref[r]] - cx, vy = xn[3 * ref[r] + 1] - cy, vz = xn[3 * ref[r] + 2] - cz;
    const float nn = fmaxf(sqrtf(vx * vx + vy * vy + vz * vz), 1e-6f);
    f[3 + 3 * r] = vx / nn;
    f[4 + 3 * r] = vy / nn;
    f[5 + 3 * r] = vz / nn;
  }
  for (int q = 0; q < P.topo.T; ++q) {
    const int* a = P.topo.dih[q];
    float b1[3], b2[3], b3[3];
    for (int d = 0; d < 3; ++d) {
      b1[d] = xn[3 * a[1] + d] - xn[3 * a[0] + d];
      b2[d] = xn[3 * a[2] + d] - xn[3 * a[1] + d];
      b3[d] = xn[3 * a[3] + d] - xn[3 * a[2] + d];
    }
    const float n1[3] = {b1[1] * b2[2] - b1[2] * b2[1], b1[2] * b2[0] - b1[0] * b2[2], b1[0] * b2[1] - b1[1] * b2[0]};
    const float n2[3] = {b2[1] * b3[2] - b2[2] * b3[1], b2[2] * b3[0] - b2[0] * b3[2], b2[0] * b3[1] - b2[1] * b3[0]};
    const float yy = sqrtf(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]) * (b1[0] * n2[0] + b1[1] * n2[1] + b1[2] * n2[2]);
    const float xx = n1[0] * n2[0] + n1[1] * n2[1] + n1[2] * n2[2];
    const float rr = sqrtf(xx * xx + yy * yy);
    f[9 + 2 * q] = rr > 0.f ? xx / rr : 1.f;
    f[10 + 2 * q] = rr > 0.f ? yy / rr : 0.f;
  }
  const int k = state_of ? state_of[n] : 0;
  if ((unsigned)k < (unsigned)n_states) {
    const StateDev st = states[k];
    f[41] = st.w_sg_f;
    f[42] = st.w_g_f;
    f[43] = (float)(300.0 * kBoltzmann / st.kT);
  }
  for (int i = 0; i < 4; ++i) f[44 + i] = asinhf((float)(comps[n * 4 + i] / 10.0));
}

// The move from pose x to pose y, in FP64.
__global__ void pose_delta_kernel(int64_t N, const PoseArgs P, const float* __restrict__ x,
                                  const float* __restrict__ y, float* delta) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int na = P.LL.na;
  const float* X[2] = {x + n * na * 3, y + n * na * 3};
  double C[2][3], F[2][3][3];
  for (int p = 0; p < 2; ++p) {
    double M = 0.0, c[3] = {0, 0, 0};
    for (int i = 0; i < na; ++i) {
      const double m = atom_mass(P, i);
      M += m;
      for (int d = 0; d < 3; ++d) c[d] += m * X[p][3 * i + d];
    }
    for (int d = 0; d < 3; ++d) C[p][d] = c[d] / M;
    double e1[3], e2[3], e3[3];
    for (int d = 0; d < 3; ++d) e1[d] = X[p][d] - C[p][d];
    double nn = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    if (nn < 1e-9) { e1[0] = 1; e1[1] = 0; e1[2] = 0; nn = 1; }
    for (int d = 0; d < 3; ++d) e1[d] /= nn;
    for (int d = 0; d < 3; ++d) e2[d] = X[p][3 * (na - 1) + d] - C[p][d];
    const double pr = e2[0] * e1[0] + e2[1] * e1[1] + e2[2] * e1[2];
    for (int d = 0; d < 3; ++d) e2[d] -= pr * e1[d];
    nn = sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
    if (nn < 1e-9) {
      double a[3] = {0, 0, 1};
      if (fabs(e1[2]) > 0.9) { a[1] = 1; a[2] = 0; }
      e2[0] = e1[1] * a[2] - e1[2] * a[1];
      e2[1] = e1[2] * a[0] - e1[0] * a[2];
      e2[2] = e1[0] * a[1] - e1[1] * a[0];
      nn = sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
    }
    for (int d = 0; d < 3; ++d) e2[d] /= nn;
    e3[0] = e1[1] * e2[2] - e1[2] * e2[1];
    e3[1] = e1[2] * e2[0] - e1[0] * e2[2];
    e3[2] = e1[0] * e2[1] - e1[1] * e2[0];
    for (int d = 0; d < 3; ++d) { F[p][d][0] = e1[d]; F[p][d][1] = e2[d]; F[p][d][2] = e3[d]; }
  }
  float* out = delta + n * DMAX;
  for (int d = 0; d < DMAX; ++d) out[d] = 0.f;
  for (int d = 0; d < 3; ++d) out[d] = (float)(C[1][d] - C[0][d]);
  double R[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) R[a][b] = F[1][a][0] * F[0][b][0] + F[1][a][1] * F[0][b][1] + F[1][a][2] * F[0][b][2];
  const double v[3] = {R[2][1] - R[1][2], R[0][2] - R[2][0], R[1][0] - R[0][1]};
  const double sv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);  // 2 sin(theta)
  const double th = atan2(0.5 * sv, 0.5 * (R[0][0] + R[1][1] + R[2][2] - 1.0));
  if (th > 1e-8 && sv < 1e-8) {  // rotation by pi: axis from the symmetric part
    double ax[3] = {sqrt(fmax(0.0, 0.5 * (R[0][0] + 1))), sqrt(fmax(0.0, 0.5 * (R[1][1] + 1))),
                    sqrt(fmax(0.0, 0.5 * (R[2][2] + 1)))};
    if (R[0][1] < 0) ax[1] = -ax[1];
    if (R[0][2] < 0) ax[2] = -ax[2];
    for (int d = 0; d < 3; ++d) out[3 + d] = (float)(th * ax[d]);
  } else {
    const double f = th < 1e-8 ? 0.5 : th / sv;
    for (int d = 0; d < 3; ++d) out[3 + d] = (float)(f * v[d]);
  }
  for (int q = 0; q < P.topo.T; ++q) {
    double tau[2];
    for (int p = 0; p < 2; ++p) {
      const int* a = P.topo.dih[q];
      double b1[3], b2[3], b3[3];
      for (int d = 0; d < 3; ++d) {
        b1[d] = (double)X[p][3 * a[1] + d] - X[p][3 * a[0] + d];
        b2[d] = (double)X[p][3 * a[2] + d] - X[p][3 * a[1] + d];
        b3[d] = (double)X[p][3 * a[3] + d] - X[p][3 * a[2] + d];
      }
      const double n1[3] = {b1[1] * b2[2] - b1[2] * b2[1], b1[2] * b2[0] - b1[0] * b2[2], b1[0] * b2[1] - b1[1] * b2[0]};
      const double n2[3] = {b2[1] * b3[2] - b2[2] * b3[1], b2[2] * b3[0] - b2[0] * b3[2], b2[0] * b3[1] - b2[1] * b3[0]};
      tau[p] = atan2(sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]) * (b1[0] * n2[0] + b1[1] * n2[1] + b1[2] * n2[2]),
                     n1[0] * n2[0] + n1[1] * n2[1] + n1[2] * n2[2]);
    }
    double d = tau[1] - tau[0];
    while (d > M_PI) d -= 2.0 * M_PI;
    while (d <= -M_PI) d += 2.0 * M_PI;
    out[6 + q] = (float)d;
  }
}

// ------------------------------------------------------------------ the learned MH move
// Rotation of v by the axis-angle vector w (Rodrigues), FP32.
__device__ inline void rotate(float& vx, float& vy, float& vz, float wx, float wy, float wz) {
  const float th2 = wx * wx + wy * wy + wz * wz;
  float a, b;
  if (th2 < 1e-12f) {
    a = 1.f - th2 / 6.f;
    b = 0.5f - th2 / 24.f;
  } else {
    const float th = sqrtf(th2);
    float s, c;
    sincosf(th, &s, &c);
    a = s / th;
    b = (1.f - c) / th2;
  }
  const float cx = wy * vz - wz * vy, cy = wz * vx - wx * vz, cz = wx * vy - wy * vx;
  const float ccx = wy * cz - wz * cy, ccy = wz * cx - wx * cz, ccz = wx * cy - wy * cx;
  vx += a * cx + b * ccx;
  vy += a * cy + b * ccy;
  vz += a * cz + b * ccz;
}

template <int APL>
__device__ inline void rigid(float (&xs)[APL][3], int na, const float* mass, float invM, float tx, float ty, float tz,
                             float wx, float wy, float wz) {
  const int lane = threadIdx.x & 31;
  float cx = 0.f, cy = 0.f, cz = 0.f;
#pragma unroll
  for (int a = 0; a < APL; ++a) {
    const int i = lane + 32 * a;
    if (i < na) {
      cx += mass[a] * xs[a][0];
      cy += mass[a] * xs[a][1];
      cz += mass[a] * xs[a][2];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cx += __shfl_xor_sync(kFull, cx, o);
    cy += __shfl_xor_sync(kFull, cy, o);
    cz += __shfl_xor_sync(kFull, cz, o);
  }
  cx *= invM;
  cy *= invM;
  cz *= invM;
#pragma unroll
  for (int a = 0; a < APL; ++a) {
    float vx = xs[a][0] - cx, vy = xs[a][1] - cy, vz = xs[a][2] - cz;
    rotate(vx, vy, vz, wx, wy, wz);
    xs[a][0] = cx + vx + tx;
    xs[a][1] = cy + vy + ty;
    xs[a][2] = cz + vz + tz;
  }
}

struct MoveArgs {
  PoseArgs P;
  const StateDev* states;
  int n_states;
  int64_t n_rep;
  const int32_t* state_of;
  const float* out;  // network outputs [R][360]
  uint64_t seed;
  uint32_t ctr;
  int64_t rep_offset;
  int t_eff;         // moved torsions (<= topo.T); the mixture uses 6 + t_eff dimensions
};

// Draw d ~ q(. | x), y = Apply(x, d), log q(d | x).  One warp per replica.
template <int APL>
__global__ void sample_apply_kernel(const MoveArgs A, const float* __restrict__ x, float* y, float* delta,
                                    double* logq) {
  __shared__ float s_pos[4][96 * 3];
  __shared__ float s_dl[4][DMAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * 4 + warp;
  if (r >= A.n_rep) return;
  const int na = A.P.LL.na, T = A.t_eff, D = 6 + T;
  const float* o = A.out + r * NOUT;
  const uint32_t rid = (uint32_t)(A.rep_offset + r);
  // component: cumulative softmax in FP64 against a 53-bit uniform
  int comp = NCOMP - 1;
  if (lane == 0) {
    double m = -INFINITY;
    for (int c = 0; c < NCOMP; ++c) m = fmax(m, (double)o[c]);
    double w[NCOMP], z = 0.0;
    for (int c = 0; c < NCOMP; ++c) {
      w[c] = exp((double)o[c] - m);
      z += w[c];
    }
    const U4 rr = philox(A.seed, 100u, rid, A.ctr, kPurposeLearned);
    const double u = uniform53(rr.x, rr.y) * z;
    double cum = 0.0;
    for (int c = 0; c < NCOMP; ++c) {
      cum += w[c];
      if (u < cum) {
        comp = c;
        break;
      }
    }
  }
  comp = __shfl_sync(kFull, comp, 0);
  if (lane < D) {
    const U4 rr = philox(A.seed, (uint32_t)lane, rid, A.ctr, kPurposeLearned);
    const float u1 = ((float)(rr.x >> 9) + 0.5f) * (1.0f / 8388608.0f);
    const float u2 = (float)(rr.y >> 9) * (1.0f / 8388608.0f);
    float sn, cs;
    sincospif(2.f * u2, &sn, &cs);
    const float z0 = sqrtf(-2.f * logf(u1)) * cs;
    const float mu = o[NCOMP + comp * DMAX + lane];
    const float sg = (float)exp(log_sigma(o[NCOMP + NCOMP * DMAX + comp * DMAX + lane]));
    s_dl[warp][lane] = mu + sg * z0;
  } else if (lane < DMAX) {
    s_dl[warp][lane] = 0.f;
  }
  __syncwarp();
  // log q(d | x): component log-probabilities on lanes 0..7, log-sum-exp over the warp (FP64)
  const double logz = logits_lse(o);
  double lp = lane < NCOMP ? component_logp(o, D, s_dl[warp], lane, logz) : -INFINITY;
  double mx = lp;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(kFull, mx, off));
  double e = lane < NCOMP ? exp(lp - mx) : 0.0;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(kFull, e, off);
  if (lane == 0) logq[r] = mx + log(e);
  if (lane < DMAX) delta[r * DMAX + lane] = s_dl[warp][lane];
  // Apply
  float xs[APL][3], mass[APL];
  const float* xr = x + r * na * 3;
#pragma unroll
  for (int a = 0; a < APL; ++a) {
    const int i = lane + 32 * a;
    mass[a] = i < na ? atom_mass(A.P, i) : 0.f;
    for (int d = 0; d < 3; ++d) xs[a][d] = i < na ? xr[3 * i + d] : 0.f;
  }
  const float* dl = s_dl[warp];
  const float invM = 1.f / A.P.LL.total_mass;
  rigid<APL>(xs, na, mass, invM, 0.5f * dl[0], 0.5f * dl[1], 0.5f * dl[2], 0.5f * dl[3], 0.5f * dl[4], 0.5f * dl[5]);
  float* sp = s_pos[warp];
  for (int q = 0; q < T; ++q) {
#pragma unroll
    for (int a = 0; a < APL; ++a) {
      const int i = lane + 32 * a;
      if (i < na)
        for (int d = 0; d < 3; ++d) sp[3 * i + d] = xs[a][d];
    }
    __syncwarp();
    const int pi = A.P.topo.prox[q], di = A.P.topo.dist[q];
    const float px = sp[3 * pi], py = sp[3 * pi + 1], pz = sp[3 * pi + 2];
    float ax = sp[3 * di] - px, ay = sp[3 * di + 1] - py, az = sp[3 * di + 2] - pz;
    const float inv = rsqrtf(ax * ax + ay * ay + az * az) * dl[6 + q];
    ax *= inv;
    ay *= inv;
    az *= inv;
    __syncwarp();
#pragma unroll
    for (int a = 0; a < APL; ++a) {
      const int i = lane + 32 * a;
      if (i < na && ((A.P.topo.moved[q][i >> 5] >> (i & 31)) & 1u)) {
        float vx = xs[a][0] - px, vy = xs[a][1] - py, vz = xs[a][2] - pz;
        rotate(vx, vy, vz, ax, ay, az);
        xs[a][0] = px + vx;
        xs[a][1] = py + vy;
        xs[a][2] = pz + vz;
      }
    }
  }
  rigid<APL>(xs, na, mass, invM, 0.5f * dl[0], 0.5f * dl[1], 0.5f * dl[2], 0.5f * dl[3], 0.5f * dl[4], 0.5f * dl[5]);
  float* yr = y + r * na * 3;
#pragma unroll
  for (int a = 0; a < APL; ++a) {
    const int i = lane + 32 * a;
    if (i < na)
      for (int d = 0; d < 3; ++d) yr[3 * i + d] = xs[a][d];
  }
}

__device__ inline double weighted_u(const double* c, double w_sg, double w_g) {
  double e = __dadd_rn(c[0], c[1]);
  if (w_sg != 0.0) e = __dadd_rn(e, __dmul_rn(w_sg, c[2]));
  if (w_g != 0.0) e = __dadd_rn(e, __dmul_rn(w_g, c[3]));
  return e;
}

// log q(-d | x'), the acceptance test, and the copy of accepted moves.  One warp per replica.
template <int APL>
__global__ void accept_kernel(const MoveArgs A, const float* __restrict__ y, const double* __restrict__ comps_y,
                              const float* __restrict__ delta, const double* __restrict__ logq_f, float* x,
                              double* comps, int32_t* accepted, int64_t* counters) {
  __shared__ float s_dl[4][DMAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * 4 + warp;
  if (r >= A.n_rep) return;
  const int na = A.P.LL.na, D = 6 + A.t_eff;
  const int k = A.state_of[r];
  if ((unsigned)k >= (unsigned)A.n_states) return;
  if (lane < DMAX) s_dl[warp][lane] = -delta[r * DMAX + lane];
  __syncwarp();
  const float* o = A.out + r * NOUT;
  const double logz = logits_lse(o);
  const double lp = lane < NCOMP ? component_logp(o, D, s_dl[warp], lane, logz) : -INFINITY;
  double mx = lp;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(kFull, mx, off));
  double e = lane < NCOMP ? exp(lp - mx) : 0.0;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(kFull, e, off);
  const double lqr = mx + log(e);
  const StateDev st = A.states[k];
  const double du = st.beta * (weighted_u(comps_y + r * 4, st.w_sg, st.w_g) - weighted_u(comps + r * 4, st.w_sg, st.w_g));
  const double lr = (lqr - logq_f[r]) - du;
  const U4 rr = philox(A.seed, 101u, (uint32_t)(A.rep_offset + r), A.ctr, kPurposeLearned);
  const bool acc = uniform53(rr.x, rr.y) < exp(lr);
  if (acc) {
#pragma unroll
    for (int a = 0; a < APL; ++a) {
      const int i = lane + 32 * a;
      if (i < na)
        for (int d = 0; d < 3; ++d) x[(r * na + i) * 3 + d] = y[(r * na + i) * 3 + d];
    }
    if (lane < 4) comps[r * 4 + lane] = comps_y[r * 4 + lane];
  }
  if (lane == 0) {
    if (acc && accepted) accepted[r] += 1;
    if (counters) {
      if (acc) atomicAdd((unsigned long long*)&counters[ALGDOCK_CNT_ACCEPTED], 1ull);
      if (!isfinite(lr)) atomicAdd((unsigned long long*)&counters[ALGDOCK_CNT_NONFINITE], 1ull);
    }
  }
}

PoseArgs pose_args(const algdock_ctx& c) { return PoseArgs{c.lig, c.d_blob, c.ltopo}; }

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

// ------------------------------------------------------------------ host side
void build_learned_topo(int na, int nb, const int32_t* bonds, LearnedTopo* t) {
  std::vector<int> deg(na, 0);
  std::vector<std::vector<int>> nbr(na);
  for (int b = 0; b < nb; ++b) {
    deg[bonds[2 * b]]++;
    deg[bonds[2 * b + 1]]++;
  }
  *t = LearnedTopo{};
  std::vector<int> seen(na), queue(na);
  for (int b = 0; b < nb && t->T < kLearnTmax; ++b) {
    const int j = bonds[2 * b], k = bonds[2 * b + 1];
    if (deg[j] < 2 || deg[k] < 2) continue;
    std::fill(seen.begin(), seen.end(), 0);
    int h = 0, tl = 0;
    seen[0] = 1;
    queue[tl++] = 0;
    while (h < tl) {  // atoms reachable from the root without crossing bond b
      const int u = queue[h++];
      for (int c = 0; c < nb; ++c) {
        if (c == b) continue;
        int v = -1;
        if (bonds[2 * c] == u) v = bonds[2 * c + 1];
        else if (bonds[2 * c + 1] == u) v = bonds[2 * c];
        if (v >= 0 && !seen[v]) {
          seen[v] = 1;
          queue[tl++] = v;
        }
      }
    }
    const int prox = seen[j] ? j : k, dist = seen[j] ? k : j;
    const int T = t->T;
    t->prox[T] = prox;
    t->dist[T] = dist;
    for (int i = 0; i < na; ++i)
      if (!seen[i] && i != dist) t->moved[T][i >> 5] |= 1u << (i & 31);
    int ii = -1, ll = -1;
    for (int c = 0; c < nb; ++c) {
      const int a0 = bonds[2 * c], a1 = bonds[2 * c + 1];
      if (a0 == prox || a1 == prox) {
        const int v = a0 == prox ? a1 : a0;
        if (v != dist && (ii < 0 || v < ii)) ii = v;
      }
      if (a0 == dist || a1 == dist) {
        const int v = a0 == dist ? a1 : a0;
        if (v != prox && (ll < 0 || v < ll)) ll = v;
      }
    }
    t->dih[T][0] = ii;
    t->dih[T][1] = prox;
    t->dih[T][2] = dist;
    t->dih[T][3] = ll;
    t->T++;
  }
}

cudaError_t learned_features(cudaStream_t s, const algdock_ctx& c, int64_t N, const int32_t* state_of,
                             const float* x, const double* comps, float* feat) {
  if (N == 0) return cudaSuccess;
  features_kernel<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(N, pose_args(c), c.d_states, c.K, state_of, x, comps,
                                                              feat);
  return cudaGetLastError();
}

cudaError_t learned_pose_delta(cudaStream_t s, const algdock_ctx& c, int64_t N, const float* x, const float* y,
                               float* delta) {
  if (N == 0) return cudaSuccess;
  pose_delta_kernel<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(N, pose_args(c), x, y, delta);
  return cudaGetLastError();
}

// Scratch of the forward pass: h1, h2, h3 (BF16 [N][256]).
size_t learned_forward_scratch(int64_t N) { return 3 * align256((size_t)N * NHID * sizeof(bf16)); }

static cudaError_t forward_keep(cudaStream_t s, const float* params, const bf16* W, int64_t N, const float* feat,
                                float* out, bf16* h1, bf16* h2, bf16* h3) {
  const int n = (int)N;
  cudaError_t e = gemm<float, false, bf16, false, EPI_RELU_BF16>(s, n, NHID, NFEAT, feat, NFEAT, W + WOFF_1, NFEAT, h1,
                                                                  NHID, params + OFF_B1);
  if (e == cudaSuccess)
    e = gemm<bf16, false, bf16, false, EPI_RELU_BF16>(s, n, NHID, NHID, h1, NHID, W + WOFF_2, NHID, h2, NHID,
                                                       params + OFF_B2);
  if (e == cudaSuccess)
    e = gemm<bf16, false, bf16, false, EPI_RELU_BF16>(s, n, NHID, NHID, h2, NHID, W + WOFF_3, NHID, h3, NHID,
                                                       params + OFF_B3);
  if (e == cudaSuccess)
    e = gemm<bf16, false, bf16, false, EPI_F32_BIAS>(s, n, NOUT, NHID, h3, NHID, W + WOFF_4, NHID, out, NOUT,
                                                      params + OFF_B4);
  return e;
}

cudaError_t learned_forward(cudaStream_t s, const float* params, const uint16_t* wbf16, int64_t N, const float* feat,
                            float* out, void* scratch) {
  if (N == 0) return cudaSuccess;
  char* p = (char*)scratch;
  const size_t hb = align256((size_t)N * NHID * sizeof(bf16));
  return forward_keep(s, params, (const bf16*)wbf16, N, feat, out, (bf16*)p, (bf16*)(p + hb), (bf16*)(p + 2 * hb));
}

// Scratch of the gradient: h1..h3, out (FP32), dout (FP32 and BF16), dh (two BF16 buffers), loss rows.
size_t learned_grad_scratch(int64_t N) {
  return 5 * align256((size_t)N * NHID * sizeof(bf16)) + 2 * align256((size_t)N * NOUT * sizeof(float)) +
         align256((size_t)N * NOUT * sizeof(bf16)) + align256((size_t)N * sizeof(float));
}

cudaError_t learned_grad(cudaStream_t s, const float* params, const uint16_t* wbf16, int64_t N, const float* feat,
                         const float* delta, int D, float* grad, float* loss, void* scratch) {
  if (N == 0) return cudaSuccess;
  const bf16* W = (const bf16*)wbf16;
  char* p = (char*)scratch;
  const size_t hb = align256((size_t)N * NHID * sizeof(bf16));
  const size_t ob = align256((size_t)N * NOUT * sizeof(float));
  bf16* h1 = (bf16*)p;
  bf16* h2 = (bf16*)(p + hb);
  bf16* h3 = (bf16*)(p + 2 * hb);
  bf16* dA = (bf16*)(p + 3 * hb);
  bf16* dB = (bf16*)(p + 4 * hb);
  float* out = (float*)(p + 5 * hb);
  float* dout = (float*)(p + 5 * hb + ob);
  bf16* dout16 = (bf16*)(p + 5 * hb + 2 * ob);
  float* lrow = (float*)(p + 5 * hb + 2 * ob + align256((size_t)N * NOUT * sizeof(bf16)));
  const int n = (int)N;
  cudaError_t e = forward_keep(s, params, W, N, feat, out, h1, h2, h3);
  if (e != cudaSuccess) return e;
  nll_kernel<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(N, D, out, delta, dout, lrow);
  to_bf16_kernel<<<(unsigned)((N * NOUT + 255) / 256), 256, 0, s>>>(N * NOUT, dout, dout16);
  if (loss) sum_kernel<<<1, 256, 0, s>>>(N, lrow, 1.f / (float)N, loss);
  // layer 4: dW4 = dout^T h3, db4 = colsum(dout), dh3 = (dout W4) * [h3 > 0]
  e = gemm<bf16, true, bf16, true, EPI_F32>(s, NOUT, NHID, n, dout16, NOUT, h3, NHID, grad + OFF_W4, NHID);
  colsum_kernel<float><<<(NOUT + 127) / 128, 128, 0, s>>>(n, NOUT, dout, 1.f, grad + OFF_B4);
  if (e == cudaSuccess)
    e = gemm<bf16, false, bf16, true, EPI_MASK_BF16>(s, n, NHID, NOUT, dout16, NOUT, W + WOFF_4, NHID, dA, NHID,
                                                      nullptr, h3, NHID);
  // layer 3
  if (e == cudaSuccess) e = gemm<bf16, true, bf16, true, EPI_F32>(s, NHID, NHID, n, dA, NHID, h2, NHID, grad + OFF_W3, NHID);
  colsum_kernel<bf16><<<(NHID + 127) / 128, 128, 0, s>>>(n, NHID, dA, 1.f, grad + OFF_B3);
  if (e == cudaSuccess)
    e = gemm<bf16, false, bf16, true, EPI_MASK_BF16>(s, n, NHID, NHID, dA, NHID, W + WOFF_3, NHID, dB, NHID, nullptr,
                                                      h2, NHID);
  // layer 2
  if (e == cudaSuccess) e = gemm<bf16, true, bf16, true, EPI_F32>(s, NHID, NHID, n, dB, NHID, h1, NHID, grad + OFF_W2, NHID);
  colsum_kernel<bf16><<<(NHID + 127) / 128, 128, 0, s>>>(n, NHID, dB, 1.f, grad + OFF_B2);
  if (e == cudaSuccess)
    e = gemm<bf16, false, bf16, true, EPI_MASK_BF16>(s, n, NHID, NHID, dB, NHID, W + WOFF_2, NHID, dA, NHID, nullptr,
                                                      h1, NHID);
  // layer 1
  if (e == cudaSuccess)
    e = gemm<bf16, true, float, true, EPI_F32>(s, NHID, NFEAT, n, dA, NHID, feat, NFEAT, grad + OFF_W1, NFEAT);
  colsum_kernel<bf16><<<(NHID + 127) / 128, 128, 0, s>>>(n, NHID, dA, 1.f, grad + OFF_B1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t learned_adam(cudaStream_t s, float* params, uint16_t* wbf16, const float* grad, float* m, float* v, int step,
                         float lr) {
  const float c1 = (float)(1.0 / (1.0 - pow(0.9, step)));
  const float c2 = (float)(1.0 / (1.0 - pow(0.999, step)));
  adam_kernel<<<(NPARAMS + 255) / 256, 256, 0, s>>>(params, (bf16*)wbf16, grad, m, v, lr, c1, c2);
  return cudaGetLastError();
}

// Scratch of one learned move: features, h1..h3, outputs, y, delta, log q, components of y.
size_t learned_propose_scratch(int64_t R, int na) {
  return align256((size_t)R * NFEAT * sizeof(float)) + learned_forward_scratch(R) +
         align256((size_t)R * NOUT * sizeof(float)) + align256((size_t)R * na * 3 * sizeof(float)) +
         align256((size_t)R * DMAX * sizeof(float)) + align256((size_t)R * sizeof(double)) +
         align256((size_t)R * 4 * sizeof(double));
}

cudaError_t learned_propose(cudaStream_t s, const algdock_ctx& c, const float* params, const uint16_t* wbf16,
                            int64_t R, const int32_t* state_of, float* x, double* comps, int n_moves, int t_eff,
                            uint64_t seed, uint64_t cycle, int64_t rep_offset, int32_t* accepted, int64_t* counters,
                            void* scratch) {
  if (R == 0 || n_moves == 0) return cudaSuccess;
  const int na = c.lig.na;
  char* p = (char*)scratch;
  float* feat = (float*)p;
  p += align256((size_t)R * NFEAT * sizeof(float));
  void* fwd = p;
  p += learned_forward_scratch(R);
  float* out = (float*)p;
  p += align256((size_t)R * NOUT * sizeof(float));
  float* y = (float*)p;
  p += align256((size_t)R * na * 3 * sizeof(float));
  float* delta = (float*)p;
  p += align256((size_t)R * DMAX * sizeof(float));
  double* logq = (double*)p;
  p += align256((size_t)R * sizeof(double));
  double* comps_y = (double*)p;
  const int apl = na <= 32 ? 1 : (na <= 64 ? 2 : 3);
  const unsigned blocks = (unsigned)((R + 3) / 4);
  cudaError_t e = cudaSuccess;
  for (int mv = 0; mv < n_moves && e == cudaSuccess; ++mv) {
    MoveArgs A{pose_args(c), c.d_states, c.K, R, state_of, out, seed, (uint32_t)(cycle * (uint64_t)n_moves + mv),
               rep_offset, t_eff};
    e = learned_features(s, c, R, state_of, x, comps, feat);
    if (e == cudaSuccess) e = learned_forward(s, params, wbf16, R, feat, out, fwd);
    if (e != cudaSuccess) break;
    if (apl == 1) sample_apply_kernel<1><<<blocks, 128, 0, s>>>(A, x, y, delta, logq);
    else if (apl == 2) sample_apply_kernel<2><<<blocks, 128, 0, s>>>(A, x, y, delta, logq);
    else sample_apply_kernel<3><<<blocks, 128, 0, s>>>(A, x, y, delta, logq);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_evaluate(s, c, R, y, comps_y);
    if (e == cudaSuccess) e = learned_features(s, c, R, state_of, y, comps_y, feat);
    if (e == cudaSuccess) e = learned_forward(s, params, wbf16, R, feat, out, fwd);
    if (e != cudaSuccess) break;
    if (apl == 1) accept_kernel<1><<<blocks, 128, 0, s>>>(A, y, comps_y, delta, logq, x, comps, accepted, counters);
    else if (apl == 2) accept_kernel<2><<<blocks, 128, 0, s>>>(A, y, comps_y, delta, logq, x, comps, accepted, counters);
    else accept_kernel<3><<<blocks, 128, 0, s>>>(A, y, comps_y, delta, logq, x, comps, accepted, counters);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace algdock
