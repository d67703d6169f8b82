// BF16 GEMM on the fifth-generation tensor cores (tcgen05) with tensor-memory accumulators, for
// the learned proposal's network at large row counts (training batches and the proposals of many
// replicas).  The network itself is an extension of the paper's external-coordinate moves
// ("Sampling"); see learned.cu.
//
// D[m][n] = epi(sum_k A[m][k] B[n][k]): A [M][K] and B [N][K] row-major BF16 (both K-major), FP32
// accumulation.  One CTA of four warps computes a 128 x BN tile of D:
//   - one lane of warp 0 loads the operand tiles (128 x 64 and BN x 64 BF16, 128-byte swizzle) by
//     TMA (cp.async.bulk.tensor) into a ring of kStages shared-memory stages, each stage's bytes
//     counted on its "full" barrier;
//   - one lane of warp 1 issues tcgen05.mma (M = 128, N = BN, K = 16, four per stage) into a BN-column
//     tensor-memory accumulator, and commits each stage's MMAs to the stage's "empty" barrier (the
//     stage may then be refilled) and the last ones to the "done" barrier;
//   - all four warps then read the accumulator with tcgen05.ld (warp w holds rows 32w .. 32w + 31)
//     and apply the epilogue: bias, ReLU, the ReLU mask of the backward pass, FP32 or BF16 store.
// A split reduction over K (blockIdx.z) writes partial tiles that the caller sums in fixed order.
// Every wait is bounded: a wait that runs out sets *err and the CTA carries on to its end, where the
// tensor memory is released, so a failure returns an error instead of hanging the GPU.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <mutex>

#include "internal.cuh"

namespace algdock {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kUM = 128;     // tile rows (the MMA's M)
constexpr int kUBK = 64;     // K per stage: one 128-byte swizzle row of BF16
constexpr int kStages = 4;
constexpr long long kSpinLimit = 1ll << 24;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// 2-D tile load (x = the contiguous K coordinate, y = row), completion counted on bar.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
      ::"r"(su32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte swizzle layout: rows
// of 128 bytes, 8-row groups of 1024 bytes (the stride byte offset), tile base 1024-byte aligned;
// descriptor version 1, layout code 2 (128-byte swizzle).  A K = 16 slice starts 32 bytes further.
__device__ __forceinline__ uint64_t sdesc(const void* p) {
  uint64_t d = (uint64_t)((su32(p) >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;              // leading byte offset (16 B; unused by swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // version
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d), "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Sixteen consecutive FP32 columns of this thread's accumulator row.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

struct UmmaArgs {
  int M, N, K;
  void* C;
  int ldc;
  const float* bias;
  const bf16* mask;
  int ldm;
  int k_len;         // K per blockIdx.z slice (a multiple of kUBK)
  size_t c_zstride;  // FP32 partial tiles: element offset between slices
  int* err;
};

template <int BN>
constexpr size_t umma_smem() {
  return 1024 + (size_t)kStages * (kUM + BN) * kUBK * 2 + 256;
}

template <int BN, int EPI>
__global__ void __launch_bounds__(128, 1)
    umma_gemm_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, const UmmaArgs P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + (size_t)kStages * kUM * kUBK * 2;
  uint64_t* full = (uint64_t*)(sB + (size_t)kStages * BN * kUBK * 2);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kUM, n0 = blockIdx.x * BN;
  const int kb = blockIdx.z * P.k_len;
  const int ke = min(P.K, kb + P.k_len);
  const int nk = ke > kb ? (ke - kb + kUBK - 1) / kUBK : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      bar_init(&full[s], 1);
      bar_init(&empty[s], 1);
    }
    bar_init(done, 1);
    tmem_slot[1] = 0;  // stages the MMA issuer consumed
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tmem_slot)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  int issued = 0;  // stages loaded (producer) or consumed (MMA issuer)
  if (warp == 0 && lane == 0) {  // TMA producer
    for (int i = 0; i < nk && ok; ++i) {
      const int s = i % kStages;
      if (i >= kStages) ok = bar_wait(&empty[s], ((i / kStages) & 1) ^ 1);
      if (!ok) break;
      bar_expect_tx(&full[s], (uint32_t)((kUM + BN) * kUBK * 2));
      tma_load_2d(sA + (size_t)s * kUM * kUBK * 2, &tA, kb + i * kUBK, m0, &full[s]);
      tma_load_2d(sB + (size_t)s * BN * kUBK * 2, &tB, kb + i * kUBK, n0, &full[s]);
      issued = i + 1;
    }
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    constexpr uint32_t id = idesc(kUM, BN);
    for (int i = 0; i < nk && ok; ++i) {
      const int s = i % kStages;
      ok = bar_wait(&full[s], (i / kStages) & 1);
      if (!ok) break;
      fence_after();
#pragma unroll
      for (int k = 0; k < kUBK / 16; ++k) {
        const uint64_t a = sdesc(sA + (size_t)s * kUM * kUBK * 2 + 32 * k);
        const uint64_t b = sdesc(sB + (size_t)s * BN * kUBK * 2 + 32 * k);
        mma(tmem, a, b, id, (i > 0 || k > 0) ? 1u : 0u);
      }
      mma_commit(&empty[s]);
      issued = i + 1;
    }
    *(volatile int*)(tmem_slot + 1) = issued;
    if (nk > 0) mma_commit(done);  // arrives once every MMA above has completed
  }
  if (!ok) atomicExch(P.err, 1);
  __syncwarp();
  // epilogue: row m0 + 32 warp + lane; nk == 0 (an empty slice) gives zeros
  bool have = nk > 0;
  if (have && !bar_wait(done, 0)) {
    atomicExch(P.err, 2);
    have = false;
  }
  fence_after();
  const int row = m0 + 32 * warp + lane;
  float* Cf = (float*)P.C + (size_t)blockIdx.z * P.c_zstride;
  bf16* Cb = (bf16*)P.C;
  // vector epilogue: 16-byte aligned rows of C (and of the mask and the bias where they are read)
  const int esz = (EPI == 0 || EPI == 1) ? 4 : 2;
  const bool vec_ok = ((uintptr_t)P.C % 16 == 0) && ((size_t)P.ldc * esz) % 16 == 0 && (n0 * esz) % 16 == 0 &&
                      (EPI != 3 || ((uintptr_t)P.mask % 16 == 0 && ((size_t)P.ldm * 2) % 16 == 0)) &&
                      (!(EPI == 1 || EPI == 2) || (uintptr_t)P.bias % 16 == 0) &&
                      (EPI != 0 || (P.c_zstride * 4) % 16 == 0);
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 16) {
    float v[16];
    if (have) {
      tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = 0.f;
    }
    if (row >= P.M) continue;
    const int col0 = n0 + c0;
    if (col0 + 16 <= P.N && vec_ok) {  // 16-byte loads and stores of the thread's 16 columns
      if (EPI == 1 || EPI == 2) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 b = __ldg((const float4*)(P.bias + col0) + q);
          v[4 * q] += b.x;
          v[4 * q + 1] += b.y;
          v[4 * q + 2] += b.z;
          v[4 * q + 3] += b.w;
        }
      }
      if (EPI == 0 || EPI == 1) {
        float4* dst = (float4*)(Cf + (size_t)row * P.ldc + col0);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      } else {
        if (EPI == 3) {
          const uint4* mk = (const uint4*)(P.mask + (size_t)row * P.ldm + col0);
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const uint4 m = __ldg(mk + q);
            const bf16* mh = (const bf16*)&m;
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (!(__bfloat162float(mh[j]) > 0.f)) v[8 * q + j] = 0.f;
          }
        }
        uint4 out[2];
        bf16* oh = (bf16*)out;
#pragma unroll
        for (int j = 0; j < 16; ++j) oh[j] = __float2bfloat16(EPI == 2 ? (v[j] > 0.f ? v[j] : 0.f) : v[j]);
        uint4* dst = (uint4*)(Cb + (size_t)row * P.ldc + col0);
        dst[0] = out[0];
        dst[1] = out[1];
      }
      continue;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int col = col0 + j;
      if (col >= P.N) break;
      float x = v[j];
      if (EPI == 1 || EPI == 2) x += P.bias[col];
      if (EPI == 0 || EPI == 1) {
        Cf[(size_t)row * P.ldc + col] = x;
      } else if (EPI == 2) {
        Cb[(size_t)row * P.ldc + col] = __float2bfloat16(x > 0.f ? x : 0.f);
      } else {
        const float h = __bfloat162float(P.mask[(size_t)row * P.ldm + col]);
        Cb[(size_t)row * P.ldc + col] = __float2bfloat16(h > 0.f ? x : 0.f);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0 && lane == 0) {
    // after a timeout: wait (bounded) for the copies the MMA issuer never consumed
    for (int i = *(volatile int*)(tmem_slot + 1); i < issued; ++i)
      if (!bar_wait(&full[i % kStages], (i / kStages) & 1)) atomicExch(P.err, 3);
  }
  __syncwarp();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
}

// Out[c][r] = In[r][c] for BF16 (or FP32 converted to BF16) matrices, through a 32 x 33 shared tile.
template <typename T>
__global__ void transpose_kernel(int rows, int cols, const T* __restrict__ in, int ld_in, bf16* out, int ld_out) {
  __shared__ float t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    float v = 0.f;
    if (r < rows && c < cols) {
      if constexpr (sizeof(T) == 4) v = (float)in[(size_t)r * ld_in + c];
      else v = __bfloat162float(in[(size_t)r * ld_in + c]);
    }
    t[i][threadIdx.x] = v;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < ld_out) out[(size_t)c * ld_out + r] = __float2bfloat16(r < rows ? t[threadIdx.x][i] : 0.f);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  });
  return fn;
}

// Tensor map of a row-major BF16 matrix [rows][cols] (row stride ld elements), boxes of box_rows x 64
// with the 128-byte swizzle; out-of-range elements read as zero.
bool make_map(CUtensorMap* m, const void* base, int rows, int cols, int ld, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t stride[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kUBK, (cuuint32_t)box_rows};
  const cuuint32_t estride[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dim, stride, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int EPI>
cudaError_t launch_bn(cudaStream_t s, const CUtensorMap& a, const CUtensorMap& b, const UmmaArgs& P, int nz) {
  static std::atomic<int> ready[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (ready[dev].load(std::memory_order_acquire) == 0) {
    e = cudaFuncSetAttribute(umma_gemm_kernel<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)umma_smem<BN>());
    if (e != cudaSuccess) return e;
    ready[dev].store(1, std::memory_order_release);
  }
  const dim3 grid((unsigned)((P.N + BN - 1) / BN), (unsigned)((P.M + kUM - 1) / kUM), (unsigned)nz);
  umma_gemm_kernel<BN, EPI><<<grid, 128, umma_smem<BN>(), s>>>(a, b, P);
  return cudaGetLastError();
}

template <int EPI>
cudaError_t launch_epi(cudaStream_t s, int bn, const CUtensorMap& a, const CUtensorMap& b, const UmmaArgs& P, int nz) {
  if (bn == 64) return launch_bn<64, EPI>(s, a, b, P, nz);
  if (bn == 128) return launch_bn<128, EPI>(s, a, b, P, nz);
  return launch_bn<256, EPI>(s, a, b, P, nz);
}

}  // namespace

int umma_split_count(int K, int n_split);

bool umma_supported(int device) {
  int major = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return major == 10 && encode_fn() != nullptr;
}

cudaError_t umma_gemm(cudaStream_t s, int M, int N, int K, const void* A, int lda, const void* B, int ldb, void* C,
                      int ldc, int epi, const float* bias, const void* mask, int ldm, int n_split, int* err) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  // the operands' TMA rules: 16-byte aligned bases and row strides
  if (K <= 0 || lda % 8 || ldb % 8 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15) || !err) return cudaErrorInvalidValue;
  // tile width: wider tiles read A fewer times, narrower ones give more CTAs; the widest that still
  // gives about two waves of the 152 SMs, down to 64
  const int mt = (M + kUM - 1) / kUM, zs = n_split < 1 ? 1 : umma_split_count(K, n_split);
  int bn = 64;
  for (int c : {256, 128})
    if (N >= c && (int64_t)mt * ((N + c - 1) / c) * zs >= 2 * 152) {
      bn = c;
      break;
    }
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, M, K, lda, kUM) || !make_map(&mb, B, N, K, ldb, bn)) return cudaErrorInvalidValue;
  n_split = n_split < 1 ? 1 : n_split;
  int k_len = ((K + n_split - 1) / n_split + kUBK - 1) / kUBK * kUBK;
  const int nz = (K + k_len - 1) / k_len;
  UmmaArgs P{M, N, K, C, ldc, bias, (const bf16*)mask, ldm, k_len, (size_t)M * ldc, err};
  switch (epi) {
    case 0: return launch_epi<0>(s, bn, ma, mb, P, nz);
    case 1: return launch_epi<1>(s, bn, ma, mb, P, nz);
    case 2: return launch_epi<2>(s, bn, ma, mb, P, nz);
    default: return launch_epi<3>(s, bn, ma, mb, P, nz);
  }
}

int umma_split_count(int K, int n_split) {
  n_split = n_split < 1 ? 1 : n_split;
  const int k_len = ((K + n_split - 1) / n_split + kUBK - 1) / kUBK * kUBK;
  return (K + k_len - 1) / k_len;
}

cudaError_t transpose_to_bf16(cudaStream_t s, int rows, int cols, const void* in, int ld_in, bool in_f32, void* out,
                              int ld_out) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((ld_out + 31) / 32)), block(32, 8);
  if (in_f32)
    transpose_kernel<float><<<grid, block, 0, s>>>(rows, cols, (const float*)in, ld_in, (bf16*)out, ld_out);
  else
    transpose_kernel<bf16><<<grid, block, 0, s>>>(rows, cols, (const bf16*)in, ld_in, (bf16*)out, ld_out);
  return cudaGetLastError();
}

}  // namespace algdock
