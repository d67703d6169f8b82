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

#include <atomic>
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

// Columns k0 .. k0+31 of a matrix stored transposed (X[k * ld + r]), rows r0 .. r0+63, into a
// shared tile: 8 consecutive r per 16-byte load where the stride allows it, scattered into the
// tile's rows.
template <typename T>
__device__ inline void load_cols(bf16 (&S)[GT][GP], const T* __restrict__ X, int ld, int r0, int R, int k0, int K,
                                 int tid) {
  const bool vec = (ld % 8) == 0 && (((uintptr_t)X) & 15) == 0;
  for (int e = tid; e < GK * (GT / 8); e += 128) {
    const int kk = e / (GT / 8), rr = (e % (GT / 8)) * 8;
    const int gk = k0 + kk, gr = r0 + rr;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gk < K) {
      if (vec && gr + 8 <= R) {
        v = load8(X + (size_t)gk * ld + gr);
      } else {
        __nv_bfloat16 h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) h[j] = __float2bfloat16(gr + j < R ? ld_f(X + (size_t)gk * ld + gr + j) : 0.f);
        v = *(uint4*)h;
      }
    }
    const bf16* h = (const bf16*)&v;
#pragma unroll
    for (int j = 0; j < 8; ++j) S[rr + j][kk] = h[j];
  }
}

// Block (blockIdx.z) of a split reduction dimension: k in [z * k_len, min(K, (z + 1) * k_len)),
// its result at C + z * c_zstride (FP32 epilogue only).
template <typename TA, bool A_T, typename TB, bool B_T, int EPI>
__global__ void __launch_bounds__(128) gemm_kernel(int M, int N, int K, const TA* __restrict__ A, int lda,
                                                   const TB* __restrict__ B, int ldb, void* C, int ldc,
                                                   const float* __restrict__ bias, const bf16* __restrict__ mask,
                                                   int ldm, int k_len, size_t c_zstride) {
  __shared__ __align__(16) bf16 As[GT][GP];
  __shared__ __align__(16) bf16 Bs[GT][GP];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, t = lane & 3;
  const int kb = blockIdx.z * k_len, ke = min(K, kb + k_len);
  if (EPI == EPI_F32) C = (float*)C + blockIdx.z * c_zstride;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += GK) {
    if (A_T) load_cols(As, A, lda, m0, M, k0, ke, tid);
    else load_rows(As, A, lda, m0, M, k0, ke, tid);
    if (B_T) load_cols(Bs, B, ldb, n0, N, k0, ke, tid);
    else load_rows(Bs, B, ldb, n0, N, k0, ke, tid);
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
  gemm_kernel<TA, A_T, TB, B_T, EPI><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, mask, ldm, K, 0);
  return cudaGetLastError();
}

// Sum of the split partial products part[z][M*N], z in fixed order, into C.
__global__ void splitk_reduce_kernel(int MN, int nz, const float* __restrict__ part, float* C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= MN) return;
  float s = 0.f;
  for (int z = 0; z < nz; ++z) s += part[(size_t)z * MN + i];
  C[i] = s;
}

constexpr int kWgradSplit = 16;  // batch slices of a weight-gradient product

// Weight gradient C[M][N] = sum_k A[k][M] B[k][N] over a long batch dimension K: the batch is
// split into up to kWgradSplit slices (one CTA column each, so the 16-24 output tiles fill the
// GPU), the partial products land in part and are summed in slice order.
template <typename TA, typename TB>
cudaError_t gemm_wgrad(cudaStream_t s, int M, int N, int K, const TA* A, int lda, const TB* B, int ldb, float* C,
                       float* part) {
  if (M == 0 || N == 0) return cudaSuccess;
  const int k_len = ((K + kWgradSplit - 1) / kWgradSplit + GK - 1) / GK * GK;
  const int nz = k_len > 0 ? (K + k_len - 1) / k_len : 0;
  if (nz == 0) {
    cudaError_t e = cudaMemsetAsync(C, 0, sizeof(float) * (size_t)M * N, s);
    return e;
  }
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, nz);
  gemm_kernel<TA, true, TB, true, EPI_F32><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, part, N, nullptr, nullptr, 0,
                                                                k_len, (size_t)M * N);
  splitk_reduce_kernel<<<(M * N + 255) / 256, 256, 0, s>>>(M * N, nz, part, C);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ fused forward pass
// One CTA takes 16 rows through all four layers.  The activations stay in shared memory as BF16.
// The weights are first packed (once per call) into 13 chunks of 64 input columns, each a
// contiguous [rows][72] BF16 block whose rows carry the 8-element padding that keeps ldmatrix free
// of bank conflicts; one cp.async.bulk per chunk (the TMA engine, completion counted on an
// mbarrier) streams them from L2 through a three-stage ring, so a CTA has up to ~100 KB of weights
// in flight from two instructions instead of thousands of 16-byte requests.  The fragments reach
// mma.sync m16n8k16 through ldmatrix.  Eight warps split the output columns: 32 each in the hidden
// layers, 48 in the output layer.  Rounding is that of the layer-by-layer GEMMs: BF16 inputs and
// hidden activations, FP32 accumulation.
constexpr int FM = 16;               // rows per CTA
constexpr int F_MT = FM / 16;        // m16 row tiles per warp
constexpr int FKC = 64;              // input columns per weight chunk
constexpr int FWS = FKC + 8;         // padded row of a weight chunk (bf16): conflict-free ldmatrix
constexpr int FHS = NHID + 8;        // padded row of a hidden activation tile
constexpr int FXS = NFEAT + 8;       // padded row of the input tile
constexpr int F_WARPS = 8;
constexpr int F_STAGES = 3;
constexpr int F_NOUT_ROWS = 368;     // output-layer rows rounded up to the 16-row ldmatrix pair
constexpr int F_CH0 = NFEAT / FKC;   // chunks of the input layer
constexpr int F_CHH = NHID / FKC;    // chunks of each later layer
constexpr int F_NCHUNK = F_CH0 + 3 * F_CHH;
constexpr int F_STAGE_ELEMS = F_NOUT_ROWS * FWS;
constexpr size_t F_SMEM = (size_t)(F_STAGES * F_STAGE_ELEMS + 2 * FM * FHS + FM * FXS) * sizeof(bf16);
// packed weights: chunks of the three 256-row layers, then the four chunks of the 360-row layer
constexpr int F_CHUNK_H = NHID * FWS;                // elements of a 256-row chunk
constexpr int F_CHUNK_O = NOUT * FWS;                // elements of a 360-row chunk
constexpr int F_NCHUNK_H = F_CH0 + 2 * F_CHH;        // chunks of 256 rows
constexpr int F_PACKED = F_NCHUNK_H * F_CHUNK_H + F_CHH * F_CHUNK_O;
static_assert(NFEAT % FKC == 0 && NHID % FKC == 0, "whole chunks");
static_assert(F_SMEM <= 227 * 1024, "shared memory of one CTA");
static_assert((F_CHUNK_H * 2) % 16 == 0 && (F_CHUNK_O * 2) % 16 == 0 && (F_STAGE_ELEMS * 2) % 16 == 0,
              "bulk copies move multiples of 16 bytes between 16-byte aligned addresses");
constexpr long long kMbarSpinLimit = 1ll << 22;      // bounded waits (well over a second in all)

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void ldsm_x4(uint32_t (&r)[4], const bf16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ inline void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false if the limit ran out.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < kMbarSpinLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// One bulk copy global -> this CTA's shared memory, its bytes counted on bar.
__device__ inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

struct FusedArgs {
  const float* params;
  const bf16* Wp;      // packed weights (F_PACKED elements, 16-byte aligned)
  int N;
  const float* feat;
  float* out;
  bf16 *h1, *h2, *h3;  // optional copies of the hidden activations [N][256] (for the backward pass)
};

__device__ inline void f_layer_dims(int layer, int& n_out, int& k_in, int& woff, int& boff) {
  if (layer == 0) { n_out = NHID; k_in = NFEAT; woff = WOFF_1; boff = OFF_B1; }
  else if (layer == 1) { n_out = NHID; k_in = NHID; woff = WOFF_2; boff = OFF_B2; }
  else if (layer == 2) { n_out = NHID; k_in = NHID; woff = WOFF_3; boff = OFF_B3; }
  else { n_out = NOUT; k_in = NHID; woff = WOFF_4; boff = OFF_B4; }
}

__host__ __device__ inline void f_chunk(int c, int& layer, int& kc) {
  layer = c < F_CH0 ? 0 : 1 + (c - F_CH0) / F_CHH;
  kc = c < F_CH0 ? c : (c - F_CH0) % F_CHH;
}

// First element and element count of packed chunk c.
__host__ __device__ inline int f_chunk_off(int c) {
  return c < F_NCHUNK_H ? c * F_CHUNK_H : F_NCHUNK_H * F_CHUNK_H + (c - F_NCHUNK_H) * F_CHUNK_O;
}
__host__ __device__ inline int f_chunk_len(int c) { return c < F_NCHUNK_H ? F_CHUNK_H : F_CHUNK_O; }

// Packed weights from the row-major BF16 copy: chunk c, row n, column k < 64 is W_layer[n][64 kc + k];
// columns 64..71 are zero.
__global__ void pack_weights_kernel(const bf16* __restrict__ W, bf16* Wp) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= F_PACKED) return;
  const int c = e < F_NCHUNK_H * F_CHUNK_H ? e / F_CHUNK_H : F_NCHUNK_H + (e - F_NCHUNK_H * F_CHUNK_H) / F_CHUNK_O;
  const int i = e - f_chunk_off(c), row = i / FWS, col = i % FWS;
  int layer, kc, n_out, k_in, woff, boff;
  f_chunk(c, layer, kc);
  f_layer_dims(layer, n_out, k_in, woff, boff);
  Wp[e] = col < FKC ? W[woff + row * k_in + kc * FKC + col] : __float2bfloat16(0.f);
}

__global__ void __launch_bounds__(F_WARPS * 32) mlp_fused_kernel(const FusedArgs P) {
  extern __shared__ __align__(16) unsigned char f_smem[];
  __shared__ __align__(8) uint64_t full[F_STAGES];
  bf16* const Wst = (bf16*)f_smem;
  bf16* const H0 = Wst + F_STAGES * F_STAGE_ELEMS;
  bf16* const H1 = H0 + FM * FHS;
  bf16* const Xs = H1 + FM * FHS;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int r0 = blockIdx.x * FM;
  if (tid == 0) {
    for (int st = 0; st < F_STAGES; ++st) mbar_init(&full[st], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int c) {  // thread 0: chunk c into its stage
    // the stage's earlier reads (generic proxy, ordered before this thread by the barrier) come
    // before the bulk copy's writes (async proxy)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    uint64_t* bar = &full[c % F_STAGES];
    const uint32_t bytes = (uint32_t)(f_chunk_len(c) * sizeof(bf16));
    mbar_expect_tx(bar, bytes);
    bulk_g2s(Wst + (c % F_STAGES) * F_STAGE_ELEMS, P.Wp + f_chunk_off(c), bytes, bar);
  };
  if (tid == 0)
    for (int c = 0; c < F_STAGES - 1 && c < F_NCHUNK; ++c) issue(c);
  int issued = min(F_STAGES - 1, F_NCHUNK);
  // rows of every stage past the 360 output-layer weight rows: zero (their columns are dropped)
  for (int e = tid; e < F_STAGES * (F_NOUT_ROWS - NOUT) * FWS; e += F_WARPS * 32) {
    const int st = e / ((F_NOUT_ROWS - NOUT) * FWS), i = e % ((F_NOUT_ROWS - NOUT) * FWS);
    Wst[st * F_STAGE_ELEMS + NOUT * FWS + i] = __float2bfloat16(0.f);
  }
  for (int e = tid; e < FM * NFEAT / 4; e += F_WARPS * 32) {
    const int row = e / (NFEAT / 4), col = (e % (NFEAT / 4)) * 4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r0 + row < P.N) v = *(const float4*)(P.feat + (size_t)(r0 + row) * NFEAT + col);
    __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
    *(__nv_bfloat162*)(Xs + row * FXS + col) = lo;
    *(__nv_bfloat162*)(Xs + row * FXS + col + 2) = hi;
  }
  float acc[F_MT][6][4];
#pragma unroll
  for (int mi = 0; mi < F_MT; ++mi)
#pragma unroll
    for (int j = 0; j < 6; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[mi][j][e] = 0.f;
  for (int c = 0; c < F_NCHUNK; ++c) {
    // chunk c has landed; after the barrier every warp is done with chunk c - 1, whose stage takes
    // chunk c + F_STAGES - 1
    const bool ok = mbar_wait(&full[c % F_STAGES], (uint32_t)((c / F_STAGES) & 1));
    if (__syncthreads_or(!ok)) {
      // a copy did not arrive in time: wait (bounded) for the copies still in flight, then mark
      // this CTA's rows as failed (NaN outputs) and leave
      if (tid == 0)
        for (int cc = c; cc < issued; ++cc) mbar_wait(&full[cc % F_STAGES], (uint32_t)((cc / F_STAGES) & 1));
      __syncthreads();
      for (int e = tid; e < FM * NOUT; e += F_WARPS * 32)
        if (r0 + e / NOUT < P.N) P.out[(size_t)r0 * NOUT + e] = __int_as_float(0x7fc00000);
      return;
    }
    if (c + F_STAGES - 1 < F_NCHUNK) {
      if (tid == 0) issue(c + F_STAGES - 1);
      issued = c + F_STAGES;
    }
    int layer, kc, n_out, k_in, woff, boff;
    f_chunk(c, layer, kc);
    f_layer_dims(layer, n_out, k_in, woff, boff);
    const bf16* Ain = layer == 0 ? Xs : (((layer - 1) & 1) ? H1 : H0);
    const int as = layer == 0 ? FXS : FHS;
    const bf16* Wc = Wst + (c % F_STAGES) * F_STAGE_ELEMS;
    const int ntile = layer == 3 ? 6 : 4;            // n8 tiles per warp
    const int nbase = warp * ntile * 8;
    // pairs of n8 tiles this warp multiplies (warp-uniform): 2 in the hidden layers, up to 3 in
    // the output layer (the last warp's third pair would start past the 360 outputs)
    const int npair = min(ntile / 2, (n_out - nbase + 15) / 16);
#pragma unroll
    for (int kk = 0; kk < FKC; kk += 16) {
      uint32_t a[F_MT][4];
#pragma unroll
      for (int mi = 0; mi < F_MT; ++mi) ldsm_x4(a[mi], Ain + (16 * mi + (lane & 15)) * as + kc * FKC + kk + (lane >> 4) * 8);
#pragma unroll
      for (int jp = 0; jp < 3; ++jp) {
        if (jp < npair) {
          uint32_t b[4];
          ldsm_x4(b, Wc + (nbase + 16 * jp + (lane & 7) + ((lane >> 4) << 3)) * FWS + kk + ((lane >> 3) & 1) * 8);
          const uint32_t b0[2] = {b[0], b[1]}, b1[2] = {b[2], b[3]};
#pragma unroll
          for (int mi = 0; mi < F_MT; ++mi) {
            mma_bf16(acc[mi][2 * jp], a[mi], b0);
            mma_bf16(acc[mi][2 * jp + 1], a[mi], b1);
          }
        }
      }
    }
    const bool last = kc == (layer == 0 ? F_CH0 : F_CHH) - 1;
    if (last) {
#pragma unroll
      for (int mi = 0; mi < F_MT; ++mi)
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (j < ntile) {
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int row = 16 * mi + g + 8 * hh, col = nbase + 8 * j + 2 * t;
            float v0 = acc[mi][j][2 * hh], v1 = acc[mi][j][2 * hh + 1];
            acc[mi][j][2 * hh] = acc[mi][j][2 * hh + 1] = 0.f;
            if (col >= n_out) continue;
            v0 += P.params[boff + col];
            v1 += P.params[boff + col + 1];
            if (layer < 3) {
              const __nv_bfloat162 hv = __floats2bfloat162_rn(fmaxf(v0, 0.f), fmaxf(v1, 0.f));
              *(__nv_bfloat162*)(((layer & 1) ? H1 : H0) + row * FHS + col) = hv;
              bf16* hk = layer == 0 ? P.h1 : (layer == 1 ? P.h2 : P.h3);
              if (hk && r0 + row < P.N) *(__nv_bfloat162*)(hk + (size_t)(r0 + row) * NHID + col) = hv;
            } else if (r0 + row < P.N) {
              *(float2*)(P.out + (size_t)(r0 + row) * NOUT + col) = make_float2(v0, v1);
            }
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------------ small kernels
// Column sums of G [M][N] (bias gradients) in two passes: block (x, y) sums 32 columns over the
// y-th of kColsumSlices row slices (8 warps, then the warps' sums in fixed order) into
// part[y][n]; the split reduction then adds the slices in order.
constexpr int kColsumSlices = 16;

template <typename T>
__global__ void colsum_kernel(int M, int N, const T* __restrict__ G, float* part) {
  __shared__ float ws[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = blockIdx.x * 32 + lane;
  const int len = (M + kColsumSlices - 1) / kColsumSlices;
  const int mb = blockIdx.y * len, me = min(M, mb + len);
  float s = 0.f;
  if (n < N)
    for (int m = mb + warp; m < me; m += 8) s += ld_f(G + (size_t)m * N + n);
  ws[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && n < N) {
    float t = 0.f;
    for (int w = 0; w < 8; ++w) t += ws[w][lane];
    part[(size_t)blockIdx.y * N + n] = t;
  }
}

template <typename T>
cudaError_t colsum(cudaStream_t s, int M, int N, const T* G, float* out, float* part) {
  colsum_kernel<T><<<dim3((N + 31) / 32, kColsumSlices), 256, 0, s>>>(M, N, G, part);
  splitk_reduce_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, kColsumSlices, part, out);
  return cudaGetLastError();
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

// ------------------------------------------------------------------ the mixture density, one warp per row
// The mixture is evaluated in FP32 across the warp: lane = c + 8 j takes component c = lane & 7 and
// the dimensions j, j + 4, j + 8, ...; the four lanes of a component add their partial sums and a
// log-sum-exp over the eight components follows.  (FP64 transcendentals run at a small fraction of
// the FP32 rate on this part; the Metropolis decision itself stays FP64.)
__device__ inline float log_sigma_f(float raw) { return -2.f + 4.f * tanhf(0.25f * raw); }

struct MixtureTerms {
  float lq;   // log q(dl | o)
  float lp;   // log w_c + log N(dl; mu_c, sigma_c) of this lane's component
  float lw;   // log w_c (log-softmax of the logits)
};

__device__ inline float warp8_max(float v) {
  v = fmaxf(v, __shfl_xor_sync(kFull, v, 1));
  v = fmaxf(v, __shfl_xor_sync(kFull, v, 2));
  return fmaxf(v, __shfl_xor_sync(kFull, v, 4));
}

__device__ inline float warp8_sum(float v) {
  v += __shfl_xor_sync(kFull, v, 1);
  v += __shfl_xor_sync(kFull, v, 2);
  return v + __shfl_xor_sync(kFull, v, 4);
}

__device__ inline MixtureTerms mixture_terms(const float* o, int D, const float* dl, int lane) {
  const int c = lane & 7;
  const float lg = o[c];
  const float m = warp8_max(lg);
  const float lz = m + logf(warp8_sum(expf(lg - m)));
  float s = 0.f;
  for (int d = lane >> 3; d < D; d += 4) {
    const float mu = o[NCOMP + c * DMAX + d];
    const float ls = log_sigma_f(o[NCOMP + NCOMP * DMAX + c * DMAX + d]);
    const float z = (dl[d] - mu) * expf(-ls);
    s += -0.5f * z * z - ls;
  }
  s += __shfl_xor_sync(kFull, s, 8);
  s += __shfl_xor_sync(kFull, s, 16);
  MixtureTerms t;
  t.lw = lg - lz;
  t.lp = s + t.lw - 0.9189385332f * (float)D;  // 0.5 ln(2 pi) per dimension
  const float mx = warp8_max(t.lp);
  t.lq = mx + logf(warp8_sum(expf(t.lp - mx)));
  return t;
}

// Mean negative log-density of the targets, one warp per row: the gradient -(1/N) dlogq/do (FP32
// and its BF16 copy for the backward GEMMs) and the row's -log q.
__global__ void nll_kernel(int64_t N, int D, const float* __restrict__ out, const float* __restrict__ delta,
                           float* dout, bf16* dout16, float* loss_rows) {
  __shared__ float s_dl[4][DMAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n = (int64_t)blockIdx.x * 4 + warp;
  if (n >= N) return;
  const float* o = out + n * NOUT;
  if (lane < DMAX) s_dl[warp][lane] = delta[n * DMAX + lane];
  __syncwarp();
  const float* dl = s_dl[warp];
  const MixtureTerms t = mixture_terms(o, D, dl, lane);
  const float scale = -1.f / (float)N;
  const int c = lane & 7;
  const float r = expf(t.lp - t.lq);  // responsibility of component c
  float* g = dout + n * NOUT;
  bf16* g16 = dout16 + n * NOUT;
  if (lane < NCOMP) {
    // d logq / d logit_c = r_c - softmax_c
    const float v = scale * (r - expf(t.lw));
    g[c] = v;
    g16[c] = __float2bfloat16(v);
  }
  for (int d = lane >> 3; d < DMAX; d += 4) {
    float gm = 0.f, gs = 0.f;
    if (d < D) {
      const float mu = o[NCOMP + c * DMAX + d];
      const float th = tanhf(0.25f * o[NCOMP + NCOMP * DMAX + c * DMAX + d]);
      const float inv_sg = expf(2.f - 4.f * th);
      const float z = (dl[d] - mu) * inv_sg;
      gm = scale * r * z * inv_sg;
      gs = scale * r * (z * z - 1.f) * (1.f - th * th);
    }
    g[NCOMP + c * DMAX + d] = gm;
    g[NCOMP + NCOMP * DMAX + c * DMAX + d] = gs;
    g16[NCOMP + c * DMAX + d] = __float2bfloat16(gm);
    g16[NCOMP + NCOMP * DMAX + c * DMAX + d] = __float2bfloat16(gs);
  }
  if (lane == 0) loss_rows[n] = -t.lq;
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

// Pose features, one warp per replica: lanes share the centre-of-mass sums, lanes 3-4 take the two
// reference directions, lanes 8.. one torsion each, and the row leaves through shared memory in two
// coalesced stores.
__global__ void features_kernel(int64_t N, const PoseArgs P, const StateDev* __restrict__ states, int n_states,
                                const int32_t* __restrict__ state_of, const float* __restrict__ x,
                                const double* __restrict__ comps, float* feat) {
  __shared__ float s_f[4][NFEAT];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n = (int64_t)blockIdx.x * 4 + warp;
  if (n >= N) return;
  const int na = P.LL.na;
  const float* xn = x + n * na * 3;
  float* f = s_f[warp];
  f[lane] = 0.f;
  f[lane + 32] = 0.f;
  float cx = 0.f, cy = 0.f, cz = 0.f;
  for (int i = lane; i < na; i += 32) {
    const float m = atom_mass(P, i);
    cx += m * xn[3 * i];
    cy += m * xn[3 * i + 1];
    cz += m * xn[3 * i + 2];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cx += __shfl_xor_sync(kFull, cx, o);
    cy += __shfl_xor_sync(kFull, cy, o);
    cz += __shfl_xor_sync(kFull, cz, o);
  }
  const float invM = 1.f / P.LL.total_mass;
  cx *= invM;
  cy *= invM;
  cz *= invM;
  __syncwarp();
  if (lane < 3) f[lane] = ((lane == 0 ? cx : (lane == 1 ? cy : cz)) - P.LL.site[lane]) / P.LL.d0;
  if (lane == 3 || lane == 4) {
    const int r = lane - 3, a = r ? na - 1 : 0;
    const float vx = xn[3 * a] - cx, vy = xn[3 * a + 1] - cy, vz = xn[3 * a + 2] - cz;
    const float nn = fmaxf(sqrtf(vx * vx + vy * vy + vz * vz), 1e-6f);
    f[3 + 3 * r] = vx / nn;
    f[4 + 3 * r] = vy / nn;
    f[5 + 3 * r] = vz / nn;
  }
  if (lane == 5) {
    const int k = state_of ? state_of[n] : 0;
    if ((unsigned)k < (unsigned)n_states) {
      const StateDev st = states[k];
      f[41] = st.w_sg_f;
      f[42] = st.w_g_f;
      f[43] = (float)(300.0 * kBoltzmann / st.kT);
    }
  }
  if (lane >= 24 && lane < 28) f[44 + lane - 24] = asinhf(0.1f * (float)comps[n * 4 + lane - 24]);
  const int q = lane - 8;
  if (q >= 0 && q < P.topo.T) {
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
  __syncwarp();
  feat[n * NFEAT + lane] = f[lane];
  feat[n * NFEAT + lane + 32] = f[lane + 32];
}

// The move from pose x to pose y: the rigid-body part in FP64, the torsion increments in FP32.
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
  // torsion increments in FP32 (FP64 transcendentals are slow on this part; the angles carry
  // FP32-level error either way, the poses being FP32)
  for (int q = 0; q < P.topo.T; ++q) {
    float tau[2];
    for (int p = 0; p < 2; ++p) {
      const int* a = P.topo.dih[q];
      float b1[3], b2[3], b3[3];
      for (int d = 0; d < 3; ++d) {
        b1[d] = X[p][3 * a[1] + d] - X[p][3 * a[0] + d];
        b2[d] = X[p][3 * a[2] + d] - X[p][3 * a[1] + d];
        b3[d] = X[p][3 * a[3] + d] - X[p][3 * a[2] + d];
      }
      const float n1[3] = {b1[1] * b2[2] - b1[2] * b2[1], b1[2] * b2[0] - b1[0] * b2[2], b1[0] * b2[1] - b1[1] * b2[0]};
      const float n2[3] = {b2[1] * b3[2] - b2[2] * b3[1], b2[2] * b3[0] - b2[0] * b3[2], b2[0] * b3[1] - b2[1] * b3[0]};
      tau[p] = atan2f(sqrtf(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]) * (b1[0] * n2[0] + b1[1] * n2[1] + b1[2] * n2[2]),
                      n1[0] * n2[0] + n1[1] * n2[1] + n1[2] * n2[2]);
    }
    float d = tau[1] - tau[0];
    const float pi = 3.14159265358979f;
    if (d > pi) d -= 2.f * pi;
    if (d <= -pi) d += 2.f * pi;
    out[6 + q] = d;
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
  // component: cumulative softmax in FP64 against a 53-bit uniform, the weights computed one per
  // lane and summed in component order (every lane walks the same sum)
  const float m8 = warp8_max(o[lane & 7]);
  const double w = lane < NCOMP ? exp((double)o[lane] - (double)m8) : 0.0;
  double z = 0.0;
#pragma unroll
  for (int c = 0; c < NCOMP; ++c) z += __shfl_sync(kFull, w, c);
  const U4 ru = philox(A.seed, 100u, rid, A.ctr, kPurposeLearned);
  const double u = uniform53(ru.x, ru.y) * z;
  int comp = NCOMP - 1;
  bool found = false;
  double cum = 0.0;
#pragma unroll
  for (int c = 0; c < NCOMP; ++c) {
    cum += __shfl_sync(kFull, w, c);
    if (!found && u < cum) {
      comp = c;
      found = true;
    }
  }
  if (lane < D) {
    const U4 rr = philox(A.seed, (uint32_t)lane, rid, A.ctr, kPurposeLearned);
    const float u1 = ((float)(rr.x >> 9) + 0.5f) * (1.0f / 8388608.0f);
    const float u2 = (float)(rr.y >> 9) * (1.0f / 8388608.0f);
    float sn, cs;
    sincospif(2.f * u2, &sn, &cs);
    const float z0 = sqrtf(-2.f * logf(u1)) * cs;
    const float mu = o[NCOMP + comp * DMAX + lane];
    const float sg = expf(log_sigma_f(o[NCOMP + NCOMP * DMAX + comp * DMAX + lane]));
    s_dl[warp][lane] = mu + sg * z0;
  } else if (lane < DMAX) {
    s_dl[warp][lane] = 0.f;
  }
  __syncwarp();
  // log q(d | x)
  const MixtureTerms mt = mixture_terms(o, D, s_dl[warp], lane);
  if (lane == 0) logq[r] = (double)mt.lq;
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
  const double lqr = (double)mixture_terms(A.out + r * NOUT, D, s_dl[warp], lane).lq;
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
  features_kernel<<<(unsigned)((N + 3) / 4), 128, 0, s>>>(N, pose_args(c), c.d_states, c.K, state_of, x, comps,
                                                              feat);
  return cudaGetLastError();
}

cudaError_t learned_pose_delta(cudaStream_t s, const algdock_ctx& c, int64_t N, const float* x, const float* y,
                               float* delta) {
  if (N == 0) return cudaSuccess;
  pose_delta_kernel<<<(unsigned)((N + 31) / 32), 32, 0, s>>>(N, pose_args(c), x, y, delta);
  return cudaGetLastError();
}

// Scratch of the forward pass: the packed weights, then h1, h2, h3 (BF16 [N][256]) for the
// layer-by-layer path.
static size_t packed_bytes() { return align256((size_t)F_PACKED * sizeof(bf16)); }
size_t learned_forward_scratch(int64_t N) {
  return packed_bytes() + 3 * align256((size_t)N * NHID * sizeof(bf16)) + align256((size_t)N * NFEAT * sizeof(bf16));
}

// The tensor-core (tcgen05) path: from min_rows rows, on an sm_100-class device, with an error word.
static bool use_tc(int64_t N, const int* err, int64_t min_rows) {
  if (!err || N < min_rows || N > (int64_t)1 << 30) return false;
  static std::atomic<int> ok[64];  // 0 unknown, 1 yes, 2 no
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  int v = ok[dev].load(std::memory_order_acquire);
  if (v == 0) {
    v = umma_supported(dev) ? 1 : 2;
    ok[dev].store(v, std::memory_order_release);
  }
  return v == 1;
}

__global__ void to_bf16_kernel(int64_t n, const float* __restrict__ in, bf16* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __float2bfloat16(in[i]);
}

// The four layers as tcgen05 GEMMs with fused epilogues (BF16 hidden activations, FP32 outputs).
static cudaError_t forward_tc(cudaStream_t s, const float* params, const bf16* W, int64_t N, const float* feat,
                              float* out, bf16* f16, bf16* h1, bf16* h2, bf16* h3, int* err) {
  const int n = (int)N;
  to_bf16_kernel<<<(unsigned)((N * NFEAT + 255) / 256), 256, 0, s>>>(N * NFEAT, feat, f16);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = umma_gemm(s, n, NHID, NFEAT, f16, NFEAT, W + WOFF_1, NFEAT, h1, NHID, EPI_RELU_BF16, params + OFF_B1, nullptr,
                  0, 1, err);
  if (e == cudaSuccess)
    e = umma_gemm(s, n, NHID, NHID, h1, NHID, W + WOFF_2, NHID, h2, NHID, EPI_RELU_BF16, params + OFF_B2, nullptr, 0, 1,
                  err);
  if (e == cudaSuccess)
    e = umma_gemm(s, n, NHID, NHID, h2, NHID, W + WOFF_3, NHID, h3, NHID, EPI_RELU_BF16, params + OFF_B3, nullptr, 0, 1,
                  err);
  if (e == cudaSuccess)
    e = umma_gemm(s, n, NOUT, NHID, h3, NHID, W + WOFF_4, NHID, out, NOUT, EPI_F32_BIAS, params + OFF_B4, nullptr, 0, 1,
                  err);
  return e;
}

static cudaError_t pack_weights(cudaStream_t s, const bf16* W, bf16* Wp) {
  pack_weights_kernel<<<(F_PACKED + 255) / 256, 256, 0, s>>>(W, Wp);
  return cudaGetLastError();
}

// The fused kernel needs 16-byte aligned features (float4 loads) and the opt-in shared-memory
// size, set once per device.
static bool fused_ready(const float* feat) {
  if ((((uintptr_t)feat) & 15) != 0) return false;
  static std::atomic<int> done[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  if (done[dev].load(std::memory_order_acquire) == 1) return true;
  if (cudaFuncSetAttribute(mlp_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F_SMEM) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  done[dev].store(1, std::memory_order_release);
  return true;
}

// Forward pass: the fused kernel on the packed weights Wp, or (misaligned features) the four
// layer GEMMs on the row-major copy W.  keep: also store h1..h3.
static cudaError_t forward_run(cudaStream_t s, const float* params, const bf16* W, const bf16* Wp, int64_t N,
                               const float* feat, float* out, bf16* h1, bf16* h2, bf16* h3, bool keep) {
  const int n = (int)N;
  if (fused_ready(feat)) {
    FusedArgs P{params, Wp, n, feat, out, keep ? h1 : nullptr, keep ? h2 : nullptr, keep ? h3 : nullptr};
    mlp_fused_kernel<<<(unsigned)((N + FM - 1) / FM), F_WARPS * 32, F_SMEM, s>>>(P);
    return cudaGetLastError();
  }
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

// Forward pass with its scratch laid out as learned_forward_scratch; pack: (re)pack the weights
// first (false when an earlier call on the same scratch and weights already did).
static cudaError_t forward_scratch(cudaStream_t s, const float* params, const uint16_t* wbf16, int64_t N,
                                   const float* feat, float* out, void* scratch, bool pack, int* tc_err = nullptr) {
  if (N == 0) return cudaSuccess;
  char* p = (char*)scratch;
  bf16* Wp = (bf16*)p;
  p += packed_bytes();
  const size_t hb = align256((size_t)N * NHID * sizeof(bf16));
  if (use_tc(N, tc_err, kTcMinRowsForward))
    return forward_tc(s, params, (const bf16*)wbf16, N, feat, out, (bf16*)(p + 3 * hb), (bf16*)p, (bf16*)(p + hb),
                      (bf16*)(p + 2 * hb), tc_err);
  if (pack) {
    const cudaError_t e = pack_weights(s, (const bf16*)wbf16, Wp);
    if (e != cudaSuccess) return e;
  }
  return forward_run(s, params, (const bf16*)wbf16, Wp, N, feat, out, (bf16*)p, (bf16*)(p + hb), (bf16*)(p + 2 * hb),
                     false);
}

cudaError_t learned_forward(cudaStream_t s, const float* params, const uint16_t* wbf16, int64_t N, const float* feat,
                            float* out, void* scratch, int* tc_err) {
  return forward_scratch(s, params, wbf16, N, feat, out, scratch, true, tc_err);
}

// Scratch of the gradient: h1..h3, dh (two BF16 buffers), out and dout (FP32), dout (BF16), loss
// rows, and the split partial products of the weight gradients.
static int64_t pad8(int64_t n) { return (n + 7) / 8 * 8; }

size_t learned_grad_scratch(int64_t N) {
  return 5 * align256((size_t)N * NHID * sizeof(bf16)) + 2 * align256((size_t)N * NOUT * sizeof(float)) +
         align256((size_t)N * NOUT * sizeof(bf16)) + align256((size_t)N * sizeof(float)) +
         align256((size_t)kWgradSplit * NOUT * NHID * sizeof(float)) + packed_bytes() +
         // the tensor-core path: operands transposed for the weight gradients, a transposed weight
         // matrix and the BF16 features
         align256((size_t)NOUT * pad8(N) * sizeof(bf16)) + align256((size_t)NHID * pad8(N) * sizeof(bf16)) +
         align256((size_t)NHID * NOUT * sizeof(bf16)) + align256((size_t)N * NFEAT * sizeof(bf16));
}

// Weight gradient C[M][N] = sum_n A[n][M] B[n][N] on tcgen05: both factors transposed to K-major
// ([M][n] and [N][n]), the batch split into FP32 partial products summed in slice order.
static cudaError_t wgrad_tc(cudaStream_t s, int M, int N, int n, const void* A, int lda, bool a_f32, const void* B,
                            int ldb, bool b_f32, float* C, float* part, bf16* TA, bf16* TB, int* err) {
  const int np = (int)pad8(n);
  cudaError_t e = transpose_to_bf16(s, n, M, A, lda, a_f32, TA, np);
  if (e == cudaSuccess) e = transpose_to_bf16(s, n, N, B, ldb, b_f32, TB, np);
  if (e == cudaSuccess) e = umma_gemm(s, M, N, n, TA, np, TB, np, part, N, EPI_F32, nullptr, nullptr, 0, kWgradSplit, err);
  if (e != cudaSuccess) return e;
  const int nz = umma_split_count(n, kWgradSplit);
  splitk_reduce_kernel<<<(M * N + 255) / 256, 256, 0, s>>>(M * N, nz, part, C);
  return cudaGetLastError();
}

// Input gradient dX[n][N] = (dY[n][K] . W[K][N]) masked by H > 0, on tcgen05 with W transposed.
static cudaError_t dgrad_tc(cudaStream_t s, int n, int N, int K, const bf16* dY, const bf16* W, const bf16* H, bf16* dX,
                            bf16* WT, int* err) {
  cudaError_t e = transpose_to_bf16(s, K, N, W, N, false, WT, K);
  if (e == cudaSuccess) e = umma_gemm(s, n, N, K, dY, K, WT, K, dX, N, EPI_MASK_BF16, nullptr, H, N, 1, err);
  return e;
}

cudaError_t learned_grad(cudaStream_t s, const float* params, const uint16_t* wbf16, int64_t N, const float* feat,
                         const float* delta, int D, float* grad, float* loss, void* scratch, int* tc_err) {
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
  float* part = (float*)((char*)lrow + align256((size_t)N * sizeof(float)));
  bf16* Wp = (bf16*)((char*)part + align256((size_t)kWgradSplit * NOUT * NHID * sizeof(float)));
  const int n = (int)N;
  if (use_tc(N, tc_err, kTcMinRowsGrad)) {
    char* q = (char*)Wp + packed_bytes();
    bf16* TA = (bf16*)q;
    q += align256((size_t)NOUT * pad8(N) * sizeof(bf16));
    bf16* TB = (bf16*)q;
    q += align256((size_t)NHID * pad8(N) * sizeof(bf16));
    bf16* WT = (bf16*)q;
    q += align256((size_t)NHID * NOUT * sizeof(bf16));
    bf16* f16 = (bf16*)q;
    cudaError_t e = forward_tc(s, params, W, N, feat, out, f16, h1, h2, h3, tc_err);
    if (e != cudaSuccess) return e;
    nll_kernel<<<(unsigned)((N + 3) / 4), 128, 0, s>>>(N, D, out, delta, dout, dout16, lrow);
    if (loss) sum_kernel<<<1, 256, 0, s>>>(N, lrow, 1.f / (float)N, loss);
    e = wgrad_tc(s, NOUT, NHID, n, dout16, NOUT, false, h3, NHID, false, grad + OFF_W4, part, TA, TB, tc_err);
    if (e == cudaSuccess) e = colsum<float>(s, n, NOUT, dout, grad + OFF_B4, part);
    if (e == cudaSuccess) e = dgrad_tc(s, n, NHID, NOUT, dout16, W + WOFF_4, h3, dA, WT, tc_err);
    if (e == cudaSuccess) e = wgrad_tc(s, NHID, NHID, n, dA, NHID, false, h2, NHID, false, grad + OFF_W3, part, TA, TB,
                                       tc_err);
    if (e == cudaSuccess) e = colsum<bf16>(s, n, NHID, dA, grad + OFF_B3, part);
    if (e == cudaSuccess) e = dgrad_tc(s, n, NHID, NHID, dA, W + WOFF_3, h2, dB, WT, tc_err);
    if (e == cudaSuccess) e = wgrad_tc(s, NHID, NHID, n, dB, NHID, false, h1, NHID, false, grad + OFF_W2, part, TA, TB,
                                       tc_err);
    if (e == cudaSuccess) e = colsum<bf16>(s, n, NHID, dB, grad + OFF_B2, part);
    if (e == cudaSuccess) e = dgrad_tc(s, n, NHID, NHID, dB, W + WOFF_2, h1, dA, WT, tc_err);
    if (e == cudaSuccess) e = wgrad_tc(s, NHID, NFEAT, n, dA, NHID, false, feat, NFEAT, true, grad + OFF_W1, part, TA,
                                       TB, tc_err);
    if (e == cudaSuccess) e = colsum<bf16>(s, n, NHID, dA, grad + OFF_B1, part);
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  cudaError_t e = pack_weights(s, W, Wp);
  if (e == cudaSuccess) e = forward_run(s, params, W, Wp, N, feat, out, h1, h2, h3, true);
  if (e != cudaSuccess) return e;
  nll_kernel<<<(unsigned)((N + 3) / 4), 128, 0, s>>>(N, D, out, delta, dout, dout16, lrow);
  if (loss) sum_kernel<<<1, 256, 0, s>>>(N, lrow, 1.f / (float)N, loss);
  // layer 4: dW4 = dout^T h3, db4 = colsum(dout), dh3 = (dout W4) * [h3 > 0]
  e = gemm_wgrad<bf16, bf16>(s, NOUT, NHID, n, dout16, NOUT, h3, NHID, grad + OFF_W4, part);
  if (e == cudaSuccess) e = colsum<float>(s, n, NOUT, dout, grad + OFF_B4, part);
  if (e == cudaSuccess)
    e = gemm<bf16, false, bf16, true, EPI_MASK_BF16>(s, n, NHID, NOUT, dout16, NOUT, W + WOFF_4, NHID, dA, NHID,
                                                      nullptr, h3, NHID);
  // layer 3
  if (e == cudaSuccess) e = gemm_wgrad<bf16, bf16>(s, NHID, NHID, n, dA, NHID, h2, NHID, grad + OFF_W3, part);
  if (e == cudaSuccess) e = colsum<bf16>(s, n, NHID, dA, grad + OFF_B3, part);
  if (e == cudaSuccess)
    e = gemm<bf16, false, bf16, true, EPI_MASK_BF16>(s, n, NHID, NHID, dA, NHID, W + WOFF_3, NHID, dB, NHID, nullptr,
                                                      h2, NHID);
  // layer 2
  if (e == cudaSuccess) e = gemm_wgrad<bf16, bf16>(s, NHID, NHID, n, dB, NHID, h1, NHID, grad + OFF_W2, part);
  if (e == cudaSuccess) e = colsum<bf16>(s, n, NHID, dB, grad + OFF_B2, part);
  if (e == cudaSuccess)
    e = gemm<bf16, false, bf16, true, EPI_MASK_BF16>(s, n, NHID, NHID, dB, NHID, W + WOFF_2, NHID, dA, NHID, nullptr,
                                                      h1, NHID);
  // layer 1
  if (e == cudaSuccess) e = gemm_wgrad<bf16, float>(s, NHID, NFEAT, n, dA, NHID, feat, NFEAT, grad + OFF_W1, part);
  if (e == cudaSuccess) e = colsum<bf16>(s, n, NHID, dA, grad + OFF_B1, part);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t learned_adam(cudaStream_t s, float* params, uint16_t* wbf16, const float* grad, float* m, float* v, int step,
                         float lr) {
  const float c1 = (float)(1.0 / (1.0 - pow(0.9, step)));
  const float c2 = (float)(1.0 / (1.0 - pow(0.999, step)));
  adam_kernel<<<(NPARAMS + 255) / 256, 256, 0, s>>>(params, (bf16*)wbf16, grad, m, v, lr, c1, c2);
  return cudaGetLastError();
}

// Scratch of one learned move: features, packed weights and h1..h3, outputs, y, delta, log q,
// components of y.
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
    if (e == cudaSuccess) e = forward_scratch(s, params, wbf16, R, feat, out, fwd, mv == 0);
    if (e != cudaSuccess) break;
    if (apl == 1) sample_apply_kernel<1><<<blocks, 128, 0, s>>>(A, x, y, delta, logq);
    else if (apl == 2) sample_apply_kernel<2><<<blocks, 128, 0, s>>>(A, x, y, delta, logq);
    else sample_apply_kernel<3><<<blocks, 128, 0, s>>>(A, x, y, delta, logq);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_evaluate(s, c, R, y, comps_y);
    if (e == cudaSuccess) e = learned_features(s, c, R, state_of, y, comps_y, feat);
    if (e == cudaSuccess) e = forward_scratch(s, params, wbf16, R, feat, out, fwd, false);
    if (e != cudaSuccess) break;
    if (apl == 1) accept_kernel<1><<<blocks, 128, 0, s>>>(A, y, comps_y, delta, logq, x, comps, accepted, counters);
    else if (apl == 2) accept_kernel<2><<<blocks, 128, 0, s>>>(A, y, comps_y, delta, logq, x, comps, accepted, counters);
    else accept_kernel<3><<<blocks, 128, 0, s>>>(A, y, comps_y, delta, logq, x, comps, accepted, counters);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace algdock
