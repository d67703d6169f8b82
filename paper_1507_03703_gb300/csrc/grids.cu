// Receptor grids: direct-sum construction and derivation of the interpolated lattices
// ("Thermodynamic Cycle": electrostatic and van der Waals grids, power-4 transform of the
// repulsive grid, soft tanh-capped grids).
#include <math.h>

#include "internal.cuh"

namespace algdock {
namespace {

constexpr int kBuildThreads = 256;
constexpr int kTile = 256;

struct __align__(16) Pos4 {
  double x, y, z, w;
};

// One thread per node; receptor atoms staged through shared memory in tiles.  The node-atom
// difference is formed in FP64 (an FP32 difference of coordinates ~20 A apart would carry ~1e-6 A
// of rounding, which r^-12 amplifies to ~1e-5 relative); each term is then evaluated in FP32
// (relative error ~1e-6) and summed in FP64, so that sums of thousands of terms of mixed sign
// (the electrostatic grid) keep their precision.
__global__ void __launch_bounds__(kBuildThreads) grid_build_kernel(int nx, int ny, int nz, double h, int n_rec,
                                                                   const Pos4* __restrict__ rec_pos,
                                                                   const float4* __restrict__ rec_abq, float* ljr,
                                                                   float* lja, float* elec) {
  __shared__ Pos4 s_pos[kTile];
  __shared__ float4 s_abq[kTile];
  const int64_t n_nodes = (int64_t)nx * ny * nz;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = p < n_nodes;
  double px = 0.0, py = 0.0, pz = 0.0;
  if (active) {
    const int i = (int)(p % nx);
    const int j = (int)((p / nx) % ny);
    const int k = (int)(p / ((int64_t)nx * ny));
    // node coordinates relative to the lattice origin; receptor atoms are shifted the same way
    px = h * i;
    py = h * j;
    pz = h * k;
  }
  double sr = 0.0, sa = 0.0, se = 0.0;
  const float rmin2 = (float)(kRepulsiveMinDist * kRepulsiveMinDist);
  const float amin2 = (float)(kAttractiveMinDist * kAttractiveMinDist);
  for (int base = 0; base < n_rec; base += kTile) {
    const int m = min(kTile, n_rec - base);
    __syncthreads();
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
      s_pos[t] = rec_pos[base + t];
      s_abq[t] = rec_abq[base + t];
    }
    __syncthreads();
    if (active) {
      for (int t = 0; t < m; ++t) {
        const Pos4 a = s_pos[t];
        const float dx = (float)(px - a.x), dy = (float)(py - a.y), dz = (float)(pz - a.z);
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float rr2 = fmaxf(r2, rmin2);
        const float ra2 = fmaxf(r2, amin2);
        const float inv_r2 = 1.0f / rr2;
        const float inv_r6 = inv_r2 * inv_r2 * inv_r2;
        const float inv_a2 = 1.0f / ra2;
        const float inv_a6 = inv_a2 * inv_a2 * inv_a2;
        const float4 ab = s_abq[t];
        sr += (double)(ab.x * (inv_r6 * inv_r6));
        sa -= (double)(ab.y * inv_a6);
        se += (double)(ab.z * inv_a2);  // q / (eps(r) r) with eps(r) = 4r; the 1/4 is in ab.z
      }
    }
  }
  if (active) {
    ljr[p] = (float)sr;
    lja[p] = (float)sa;
    elec[p] = (float)(kCoulomb * se);
  }
}

// Derived lattices, computed in FP64 and rounded once to FP32.
// Node p's hard values go into its own x-pair record (first half) and into the record of its x - 1
// neighbour in the same row (second half); its soft values go into the (x, y) quad records of
// itself and of its x - 1, y - 1 and (x - 1, y - 1) neighbours in the same plane.  Halves that
// would hold a node past the last one of a row or column are zero (no cell starts there).
__global__ void grid_prepare_kernel(int64_t n, int nx, int ny, const float* __restrict__ ljr,
                                    const float* __restrict__ lja, const float* __restrict__ elec, double vmax_r,
                                    double vmax_e, float4* hard, float4* soft) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double v = (double)ljr[p];
  if (!(v <= kRepulsiveNodeCap)) v = v > 0.0 ? kRepulsiveNodeCap : v;  // caps +inf as well
  if (!(v >= 0.0)) v = 0.0;
  const double e = (double)elec[p];
  const double root = pow(v, 0.25);
  const double soft_r = isinf(vmax_r) ? root : pow(vmax_r * tanh(v / vmax_r), 0.25);
  const double soft_e = isinf(vmax_e) ? e : vmax_e * tanh(e / vmax_e);
  const float4 h = make_float4((float)root, lja[p], elec[p], 0.f);
  const float2 sf = make_float2((float)soft_r, (float)soft_e);
  const int x = (int)(p % nx), y = (int)((p / nx) % ny);
  hard[2 * p] = h;
  if (x > 0) hard[2 * (p - 1) + 1] = h;
  if (x == nx - 1) hard[2 * p + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
  float2* q = (float2*)soft;  // 4 float2 per record: nodes (x, y), (x + 1, y), (x, y + 1), (x + 1, y + 1)
  const float2 zero = make_float2(0.f, 0.f);
  q[4 * p] = sf;
  if (x > 0) q[4 * (p - 1) + 1] = sf;
  if (y > 0) q[4 * (p - nx) + 2] = sf;
  if (x > 0 && y > 0) q[4 * (p - nx - 1) + 3] = sf;
  if (x == nx - 1) q[4 * p + 1] = q[4 * p + 3] = zero;
  if (y == ny - 1) q[4 * p + 2] = q[4 * p + 3] = zero;
}

// Peak rate of the interpolation's gathers, for the gather roofline (not a step of the method):
// each thread reads the 8 corners of cells drawn uniformly over the lattice (hard float4 corners,
// and with soft the float2 corners too, as one atom's interpolation does) and folds them into a
// sum that is stored only if it takes an impossible value, so that no load is dead.  Cells come
// from a per-thread xorshift stream mapped to [0, n - 1) by a multiply-shift (no division).
__device__ __forceinline__ uint32_t xorshift32(uint32_t& s) {
  s ^= s << 13;
  s ^= s >> 17;
  s ^= s << 5;
  return s;
}
__device__ __forceinline__ int below(uint32_t r, int n) { return (int)(((uint64_t)r * (uint32_t)n) >> 32); }

template <bool SOFT>
__global__ void __launch_bounds__(256) gather_probe_kernel(const float4* __restrict__ hard,
                                                           const float4* __restrict__ soft, int nx, int ny, int nz,
                                                           int64_t n_cells, uint32_t seed, float* sink) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t st = (uint32_t)(tid * 2654435761u) ^ seed;
  st = st ? st : 0x9E3779B9u;
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  float acc = 0.f;
  for (int64_t c = tid; c < n_cells; c += stride) {
    const int cx = below(xorshift32(st), nx - 1), cy = below(xorshift32(st), ny - 1),
              cz = below(xorshift32(st), nz - 1);
    const int64_t b = cz * sz + cy * sy + cx;
    // the cell's records, as the interpolation reads them: four 32-byte hard x-pair records and
    // (with SOFT) two 32-byte soft quad records
    float4 h0, h1, h2, h3, h4, h5, h6, h7;
    ldg_pair(hard + 2 * b, h0, h1);
    ldg_pair(hard + 2 * (b + sy), h2, h3);
    ldg_pair(hard + 2 * (b + sz), h4, h5);
    ldg_pair(hard + 2 * (b + sz + sy), h6, h7);
    acc += ((h0.x + h1.y) + (h2.z + h3.x)) + ((h4.y + h5.z) + (h6.x + h7.y));
    if (SOFT) {
      float4 s0, s1, s2, s3;
      ldg_pair(soft + 2 * b, s0, s1);
      ldg_pair(soft + 2 * (b + sz), s2, s3);
      acc += ((s0.x + s1.w) + (s2.x + s3.w)) + ((s0.z + s1.y) + (s2.z + s3.y));
    }
  }
  if (acc == -1.2345e-31f) sink[0] = acc;
}

}  // namespace

cudaError_t launch_grid_build(cudaStream_t s, const algdock_grid_desc& d, int n_rec, const double* xyz,
                              const double* rstar, const double* eps, const double* q, float* ljr, float* lja,
                              float* elec) {
  // Per-atom factors on the host (FP64), positions relative to the origin, then one upload.
  Pos4* d_pos = nullptr;
  float4* d_abq = nullptr;
  const int nr = n_rec > 0 ? n_rec : 1;
  Pos4* h_pos = new Pos4[nr];
  float4* h_abq = new float4[nr];
  for (int j = 0; j < n_rec; ++j) {
    const double two_r = 2.0 * rstar[j];
    const double r6 = two_r * two_r * two_r * two_r * two_r * two_r;
    h_pos[j] = Pos4{xyz[3 * j] - d.origin[0], xyz[3 * j + 1] - d.origin[1], xyz[3 * j + 2] - d.origin[2], 0.0};
    h_abq[j] = make_float4((float)(sqrt(eps[j]) * r6), (float)(sqrt(2.0 * eps[j]) * two_r * two_r * two_r),
                           (float)(q[j] / 4.0), 0.f);
  }
  cudaError_t e = cudaMallocAsync(&d_pos, sizeof(Pos4) * nr, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_abq, sizeof(float4) * nr, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_pos, h_pos, sizeof(Pos4) * nr, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_abq, h_abq, sizeof(float4) * nr, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host staging buffers are freed below
  delete[] h_pos;
  delete[] h_abq;
  if (e == cudaSuccess) {
    const int64_t n = (int64_t)d.n[0] * d.n[1] * d.n[2];
    const int64_t blocks = (n + kBuildThreads - 1) / kBuildThreads;
    grid_build_kernel<<<(unsigned)blocks, kBuildThreads, 0, s>>>(d.n[0], d.n[1], d.n[2], d.spacing, n_rec, d_pos,
                                                                 d_abq, ljr, lja, elec);
    e = cudaGetLastError();
  }
  if (d_pos) cudaFreeAsync(d_pos, s);
  if (d_abq) cudaFreeAsync(d_abq, s);
  return e;
}

cudaError_t launch_grid_prepare(cudaStream_t s, size_t n_nodes, int nx, int ny, const float* ljr, const float* lja,
                                const float* elec, double vmax_r, double vmax_e, float4* hard, float4* soft) {
  const int threads = 256;
  const size_t blocks = (n_nodes + threads - 1) / threads;
  grid_prepare_kernel<<<(unsigned)blocks, threads, 0, s>>>((int64_t)n_nodes, nx, ny, ljr, lja, elec, vmax_r,
                                                            vmax_e, hard, soft);
  return cudaGetLastError();
}

}  // namespace algdock

namespace algdock {
cudaError_t launch_gather_probe(cudaStream_t s, const algdock_ctx& c, int64_t n_cells, bool soft, uint32_t seed,
                                float* sink) {
  const int threads = 256;
  const int blocks = 152 * 8;
  if (soft)
    gather_probe_kernel<true><<<blocks, threads, 0, s>>>(c.d_hard, c.d_soft, c.grid.nx, c.grid.ny, c.grid.nz, n_cells,
                                                          seed, sink);
  else
    gather_probe_kernel<false><<<blocks, threads, 0, s>>>(c.d_hard, c.d_soft, c.grid.nx, c.grid.ny, c.grid.nz,
                                                           n_cells, seed, sink);
  return cudaGetLastError();
}
}  // namespace algdock
