// Internal declarations shared by the CUDA sources of libalgdock (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "algdock.h"

namespace algdock {

// A named NVTX range over one scope (a call or one stage of it): profilers that record NVTX show
// the host-side span in which the stage's work is enqueued.  Without a profiler attached the push
// and pop return at once.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Unit conventions: A, kcal/mol, amu, fs.
constexpr double kBoltzmann = 0.0019872043;        // kcal / (mol K)
constexpr double kCoulomb = 332.0637;              // kcal A / (mol e^2)
constexpr double kForceToAccel = 4.184e-4;         // (kcal/mol/A) / amu -> A / fs^2
constexpr double kKineticToKcal = 1.0 / 4.184e-4;  // amu A^2 / fs^2 -> kcal/mol
constexpr double kRepulsiveNodeCap = 1.0e10;
constexpr double kRepulsiveMinDist = 0.01;         // A
constexpr double kAttractiveMinDist = 2.0;         // A
constexpr int kMaxAtoms = 96;                      // 3 atoms per lane of one warp
constexpr int kMaxLadder = 1024;
constexpr int kMbarMaxStates = 65535;             // MBAR's state_partials grid has one y-index per state

// Two FP32 values in one 64-bit register pair, for the paired FP32 instructions of sm_100-class
// GPUs (add/sub/mul/fma .f32x2, round to nearest): one instruction serves two independent terms.
typedef uint64_t f32x2;
__device__ __forceinline__ f32x2 pack2(float a, float b) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(f32x2 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

enum : uint32_t { kPurposeMomentum = 1, kPurposeAccept = 2, kPurposeExchange = 3, kPurposeExternal = 5 };

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: ten rounds of two 32x32->64 multiplies with a Weyl key
// schedule.  Written from the published definition.
struct U4 {
  uint32_t x, y, z, w;
};

__host__ __device__ inline U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__host__ __device__ inline U4 philox(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) {
  return philox4x32_10(U4{c0, c1, c2, c3}, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Uniform double in [0, 1) from 27 + 26 random bits (exact integer arithmetic).
__host__ __device__ inline double uniform53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

// ------------------------------------------------------------------ device-side tables
// Interpolation lattices, stored as records of neighbouring nodes so that a cell's corners come in
// few loads.  Record b = (z ny + y) nx + x:
//   hard: an x-pair, 2 float4 (32 bytes): (LJr^(1/4), LJa, elec, 0) of nodes x and x + 1 of row (y, z);
//   soft: an (x, y) quad, 2 float4 (32 bytes): (sLJr^(1/4), selec) of nodes (x, y), (x + 1, y),
//         (x, y + 1), (x + 1, y + 1) of plane z.
// Parts that would hold a node past the last one of a row or column are zero (no cell starts there).
struct GridDev {
  const float4* hard;  // [n_nodes][2]
  const float4* soft;  // [n_nodes][2]
  int nx, ny, nz;
  float ox, oy, oz;  // origin, exactly the FP32 value used by the split subtraction
  float inv_h;
};

// One 32-byte lattice record in a single 256-bit load (read-only path; the record is 32-byte
// aligned: each lattice is a cudaMalloc allocation of whole records).
__device__ __forceinline__ void ldg_pair(const float4* p, float4& a, float4& b) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}

// One thermodynamic state as the kernels read it.
struct StateDev {
  double kT;       // k_B T
  double beta;     // 1 / (k_B T)
  double w_sg;     // alpha_sg
  double w_g;      // alpha_g
  double alpha;    // the protocol's alpha (NaN on the warming leg)
  float w_sg_f, w_g_f;
  float dt, sqrt_kT;
};

// Ligand blob header: word offsets (4-byte words, each section 16-byte aligned) into one
// contiguous buffer that a CTA copies into shared memory.
struct LigandLayout {
  int na, nb, nang, ntor;
  int gs_iters;    // iterations (of four entries each) of the bonded-force gather schedule per lane
  int n_slots;     // bonded force slots: 2 nb + 3 nang + 4 ntor (float4 each), then one zero slot
  int off_atom_a;  // float4[na]: (accel factor 4.184e-4/m, q, sqrt(A), sqrt(B))
  int off_atom_b;  // float4[na]: (R*, sqrt(eps), m, sqrt(4.184e-4/m))
  int off_ptype;   // uint8[na][na], [j][i]: 0 nonbonded pair, 1 1-4 pair, 2 excluded (incl. i == j)
  int off_bond;    // float4[nb]: (i, j as int bits, k, r0)
  int off_ang;     // int4[nang] (i, j, k, 0) then float4[nang] (k, theta0, 0, 0)
  int off_tor;     // int4[ntor] (i, j, k, l), float4 (V1/2, V2/2, V3/2, 0), float4 cos(gamma), float4 sin(gamma)
  int off_gs;         // uint16[gs_iters][32][4]: lane l's run of the atom-sorted slot list, 4 per
                      // iteration; bit 15 marks the last entry of an atom within the run (the
                      // run's partial sum is stored in that slot); padding entries name the zero slot
  int off_gp;         // uint16[na][4]: the slots holding atom i's partial sums (padded with the zero slot)
  int words;          // total of the sections above (multiple of 4)
  int off_pair;       // float4[(na + 1) / 2][na], [p][i]: for the partner pair j = 2p, 2p + 1,
                      // (e_ij, e_ij', c_ij, c_ij') with e = 12 eps_ij s_lj and c = 332 q_i q_j s_el,
                      // zero if excluded, i == j or j = na (odd na); after the sections above
  int words_pair;     // total including the pair table
  float total_mass;
  float site[3];
  float k_rest, d0;
};

// Target-force-field factors of one ligand atom (FP64): sqrt(A_i), sqrt(B_i), 332.0637 q_i.
struct __align__(32) TargetFactors {
  double sA, sB, qC, pad;
};

// Two receptor atoms j, j' of the target interaction, laid out for paired FP32 instructions:
// c0 = (x_hi, x_hi', y_hi, y_hi'), c1 = (z_hi, z_hi', x_lo, x_lo'), c2 = (y_lo, y_lo', z_lo, z_lo'),
// c3 = (sqrt(A), sqrt(A'), sqrt(B), sqrt(B')), with x = x_hi + x_lo the FP64 coordinate.  The
// charges q/4 of the pair sit in a float2 array beside.  An odd count ends with a zero atom.
struct __align__(16) ReceptorPair {
  float4 c0, c1, c2, c3;
};

// The all-FP64 evaluation path (the precision study's FP64 arm): the ligand's parameters in FP64,
// as offsets (in doubles) into one device buffer, and FP64 lattices.
struct Lig64 {
  int na, nb, nang, ntor;
  int off_atom;   // [na][6]: mass, q, sqrt(A), sqrt(B), R*, sqrt(eps)
  int off_bond;   // [nb][4]: i, j (as doubles), k, r0
  int off_ang;    // [nang][5]: i, j, k, k_theta, theta0
  int off_tor;    // [ntor][10]: i, j, k, l, V1/2, V2/2, V3/2, gamma1, gamma2, gamma3
  int off_ptype;  // [na][na] pair types as doubles: 0 nonbonded, 1 1-4, 2 excluded
  int n_doubles;
  double total_mass, site[3], k_rest, d0;
};
struct __align__(32) Hard64 {
  double r, a, e, pad;  // LJr^(1/4), LJa, elec
};
struct __align__(16) Soft64 {
  double r, e;  // sLJr^(1/4), selec
};
struct GridDev64 {
  const Hard64* hard;
  const Soft64* soft;
  int nx, ny, nz;
  double ox, oy, oz, h;
};

// Multi-ligand batches: one record per ligand (its layout and where its blob starts in the batch
// blob), and one work item per block (a run of up to WPB consecutive replicas of one ligand).
struct BatchLigand {
  LigandLayout LL;
  int64_t blob_off;  // in 4-byte words, a multiple of 4
  int apl;           // atoms per lane: 1 (<= 32 atoms), 2 (<= 64), 3 (<= 96)
  int cls;           // launch class: 0 (1 atom per lane), 1 (2, pair table fits 16-replica blocks),
                     // 2 (2, it does not), 3 (3)
};
struct BatchItem {
  int32_t lig, r0, count, pad;
};
// Launch shape of one class: replicas (warps) per block and whether the per-pair table is staged
// with the blob.
struct BatchClass {
  int wpb = 0;
  bool table = false;
  BatchItem* d_items = nullptr;
  int n_items = 0;
  size_t smem = 0;
};
constexpr int kBatchClasses = 4;
constexpr int kClassApl[kBatchClasses] = {1, 2, 2, 3};

// Torsion tree of the learned proposal: root atom 0, the first 16 rotatable bonds in bond order.
constexpr int kLearnTmax = 16;
struct LearnedTopo {
  int T;
  int prox[kLearnTmax], dist[kLearnTmax];  // bond atoms on the root side / away from the root
  int dih[kLearnTmax][4];                  // dihedral atoms (features)
  uint32_t moved[kLearnTmax][3];           // bit i: atom i turns with torsion k
};

}  // namespace algdock

// The context (opaque to callers).
struct algdock_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  // grids
  bool has_grid = false;
  algdock::GridDev grid{};
  float4* d_hard = nullptr;  // x-pair records, 2 float4 per node
  float4* d_soft = nullptr;  // (x, y) quad records, 2 float4 per node
  size_t grid_nodes = 0;
  // ligand
  bool has_ligand = false;
  algdock::LigandLayout lig{};
  uint32_t* d_blob = nullptr;
  // states (with the host copy of the table they were set from, for checkpoints)
  int K = 0;
  algdock::StateDev* d_states = nullptr;
  std::vector<double> h_T, h_alpha, h_dt;
  // CRC-32 of the loaded ligand blob and of the lattice descriptor (0: none loaded), for checkpoints
  uint32_t fp_ligand = 0, fp_grid = 0;
  // scratch owned by the MBAR solver, grown on demand
  void* d_mbar = nullptr;
  size_t mbar_bytes = 0;
  // pinned host word for convergence polling
  int* h_flag = nullptr;
  // work counter of the single-ligand HMC launch (replicas handed out to warps; zeroed per launch)
  unsigned long long* d_work = nullptr;
  // device staging of algdock_cycle's host arrays (grown on demand), and the side stream on which
  // its snapshot runs beside the exchange sweeps
  void* d_stage = nullptr;
  size_t stage_bytes = 0;
  // the device reaches host memory over a coherent link (NVLink-C2C on Grace: host-native atomics),
  // so algdock_cycle's kernels read and write pinned host arrays in place instead of staging them
  // (all but the counters, which take atomics)
  bool host_coherent = false;
  cudaStream_t cycle_side = nullptr;
  cudaEvent_t cycle_fork = nullptr, cycle_join = nullptr;
  // the context's seed and the method's adjustable arguments (algdock_create, algdock_set_params)
  uint64_t seed = 0;
  algdock_params params{};
  // replicas owned by the context (algdock_replicas_init), in algdock_cycle's layout: one buffer
  // [x | comps | state_of | config_of | counters]
  bool has_replicas = false;
  algdock_run_desc run{};
  int64_t n_replicas = 0;
  void* d_rbuf = nullptr;
  float* d_rx = nullptr;
  double* d_rcomps = nullptr;
  int32_t* d_rstate = nullptr;
  int32_t* d_rcfg = nullptr;
  int64_t* d_rcnt = nullptr;
  // learned proposal: torsion tree and scratch grown on demand
  algdock::LearnedTopo ltopo{};
  void* d_learn = nullptr;
  size_t learn_bytes = 0;
  // protocol initialization: device results (4 doubles) and resampling weights, grown on demand
  void* d_proto = nullptr;
  size_t proto_bytes = 0;
  // end points: receptor atoms of the target force field (ReceptorPair[n_pairs], float2 q[n_pairs]),
  // the ligand's FP64 target factors (sqrt(A_i), sqrt(B_i), 332.0637 q_i, 0), FEP scratch
  void* d_rec = nullptr;
  int n_rec = -1;  // -1: no receptor loaded
  algdock::TargetFactors* d_lig_fac = nullptr;
  void* d_fep = nullptr;
  // all-FP64 evaluation path: FP64 ligand tables (built with the ligand) and FP64 lattices
  algdock::Lig64 lig64{};
  double* d_lig64 = nullptr;
  bool has_grid64 = false;
  algdock::GridDev64 grid64{};
  void* d_grid64 = nullptr;
  size_t grid64_nodes = 0;
  // multi-ligand batch: ligands, their blobs, the replica layout and one launch shape per class
  int n_batch = 0;
  int batch_max_na = 0;
  std::vector<algdock::BatchLigand> h_batch;
  algdock::BatchLigand* d_batch = nullptr;
  uint32_t* d_batch_blob = nullptr;
  int64_t batch_n_rep = 0;
  int batch_x_stride = 0;
  std::vector<int32_t> batch_lig_of;
  bool batch_uniform = false;
  algdock::BatchClass batch_cls[algdock::kBatchClasses];
  cudaStream_t batch_side[algdock::kBatchClasses] = {};
  cudaEvent_t batch_fork = nullptr;
  cudaEvent_t batch_join[algdock::kBatchClasses] = {};
};

namespace algdock {
// Device-side checks of a cycle's results (params.checks): the flag word in the context's work
// buffer, the check kernel over a run's arrays, and the status a set flag turns into.
int* check_word(algdock_ctx* c);
cudaError_t launch_run_check(cudaStream_t s, const algdock_ctx& c, const algdock_run_desc& d, const float* x,
                             const double* comps, const int32_t* state_of, const int32_t* config_of, int* flag);
algdock_status check_status(algdock_ctx* c, int bits, const char* where);
algdock_status params_check(algdock_ctx* c, const algdock_params& p);

// CRC-32 (the IEEE 802.3 polynomial, reflected, as in zip and PNG) of n bytes, continuing from crc
// (0 to start).
uint32_t crc32_update(uint32_t crc, const void* data, size_t n);
// launchers implemented in the .cu files
cudaError_t launch_grid_build(cudaStream_t s, const algdock_grid_desc& d, int n_rec, const double* xyz,
                              const double* rstar, const double* eps, const double* q, float* ljr, float* lja,
                              float* elec);
cudaError_t launch_grid_prepare(cudaStream_t s, size_t n_nodes, int nx, int ny, const float* ljr, const float* lja,
                                const float* elec, double vmax_r, double vmax_e, float4* hard, float4* soft);
cudaError_t launch_gather_probe(cudaStream_t s, const algdock_ctx& c, int64_t n_cells, bool soft, uint32_t seed,
                                float* sink);
cudaError_t launch_hmc(cudaStream_t s, const algdock_ctx& c, int64_t n_rep, const int32_t* state_of, float* x,
                       double* comps, double* dH, uint8_t* acc, int n_steps, uint64_t seed, uint64_t cycle,
                       int64_t rep_offset, int64_t* counters);
cudaError_t launch_evaluate(cudaStream_t s, const algdock_ctx& c, int64_t N, const float* x, double* comps);
// the one-ligand HMC launch shape: 16-replica blocks with the pair table staged, else 4 without
bool hmc_uses_table(const LigandLayout& L);
// batches: the block shared memory of a class shape, the candidate shapes of a class, and the
// HMC trial of every replica of the batch (classes on forked streams, joined on s)
size_t batch_block_smem(const LigandLayout& L, int apl, int wpb, bool table);
// Dynamic shared memory a batch kernel of this shape may request on the current device: the
// per-block opt-in limit less the kernel's static shared memory (0 if the query fails).
size_t batch_smem_limit(int apl, int wpb, bool table);
// Whether a ligand's pair-table batch kernel fits 16-replica blocks (batch class 1 rather than 2
// for 33-64 atoms).
bool batch_uses_table16(const LigandLayout& L);
int batch_candidates(int cls, int* wpb, bool* table);
// all-FP64 path: lattice derivation and the evaluation of N configurations (one thread each)
cudaError_t launch_grid_prepare64(cudaStream_t s, size_t n_nodes, const double* ljr, const double* lja,
                                  const double* elec, double vmax_r, double vmax_e, Hard64* hard, Soft64* soft);
cudaError_t launch_eval64(cudaStream_t s, const algdock_ctx& c, int64_t N, const int32_t* state_of, const float* x,
                          double* force, double* comps);
cudaError_t batch_set_attributes(const algdock_ctx& c);
cudaError_t launch_hmc_batch(cudaStream_t s, const algdock_ctx& c, const int32_t* state_of, float* x, double* comps,
                             double* dH, uint8_t* acc, int n_steps, uint64_t seed, uint64_t cycle, int64_t rep_offset,
                             int64_t* counters, int only_class);
cudaError_t launch_external(cudaStream_t s, const algdock_ctx& c, int64_t n_rep, const int32_t* state_of, float* x,
                            double* comps, int n_moves, double alpha_max, float sigma, uint64_t seed, uint64_t cycle,
                            int64_t rep_offset, int32_t* accepted, int64_t* counters);
size_t equilibration_smem(int64_t T);
cudaError_t launch_equilibration(cudaStream_t st, int64_t T, int64_t S, const double* a, int64_t stride, int n_cand,
                                 double* g, int64_t* t0_best, double* neff_best);
cudaError_t launch_state_stats(cudaStream_t s, const algdock_ctx& c, int64_t n, const double* comps, int k,
                               double* out);
cudaError_t launch_resample(cudaStream_t s, const algdock_ctx& c, int64_t n, const double* comps, int k_from,
                            int k_to, int n_out, uint64_t seed, uint32_t ctr, double* work, int64_t* idx,
                            const float* x_in, float* x_out);
cudaError_t launch_pacc(cudaStream_t s, const algdock_ctx& c, int64_t n, const double* ca, const double* cb, int ka,
                        int kb, double* out);
cudaError_t launch_energy_force(cudaStream_t s, const algdock_ctx& c, int64_t N, const int32_t* state_of,
                                const float* x, float* force, double* comps);
cudaError_t launch_ukn(cudaStream_t s, const algdock_ctx& c, int64_t N, const double* comps, int k_begin,
                       int k_count, double* u_kn);
void build_learned_topo(int na, int nb, const int32_t* bonds, LearnedTopo* t);
cudaError_t learned_features(cudaStream_t s, const algdock_ctx& c, int64_t N, const int32_t* state_of,
                             const float* x, const double* comps, float* feat);
cudaError_t learned_pose_delta(cudaStream_t s, const algdock_ctx& c, int64_t N, const float* x, const float* y,
                               float* delta);
// tcgen05 BF16 GEMM (umma.cu): C = epi(A . B^T), A [M][K], B [N][K] row-major BF16; epi 0: FP32,
// 1: FP32 + bias, 2: BF16 ReLU(+ bias), 3: BF16 masked by mask > 0; n_split > 1 splits K into FP32
// partial tiles C + z M ldc.  *err (device int) is set if a bounded wait runs out.
bool umma_supported(int device);
cudaError_t umma_gemm(cudaStream_t s, int M, int N, int K, const void* A, int lda, const void* B, int ldb, void* C,
                      int ldc, int epi, const float* bias, const void* mask, int ldm, int n_split, int* err);
int umma_split_count(int K, int n_split);
cudaError_t transpose_to_bf16(cudaStream_t s, int rows, int cols, const void* in, int ld_in, bool in_f32, void* out,
                              int ld_out);
// Rows from which the learned network's gradient and forward pass run on tcgen05 (with tc_err set):
// measured against the mma.sync kernels on one GB300, the gradient ties at 4096 rows and wins from
// 8192 (2.2x at 65536); the forward ties at 8192 and wins from 16384 (1.6x at 65536).
constexpr int64_t kTcMinRowsGrad = 4096;
constexpr int64_t kTcMinRowsForward = 8192;
size_t learned_forward_scratch(int64_t N);
cudaError_t learned_forward(cudaStream_t s, const float* params, const uint16_t* wbf16, int64_t N, const float* feat,
                            float* out, void* scratch, int* tc_err = nullptr);
size_t learned_grad_scratch(int64_t N);
cudaError_t learned_grad(cudaStream_t s, const float* params, const uint16_t* wbf16, int64_t N, const float* feat,
                         const float* delta, int D, float* grad, float* loss, void* scratch, int* tc_err = nullptr);
cudaError_t learned_adam(cudaStream_t s, float* params, uint16_t* wbf16, const float* grad, float* m, float* v, int step,
                         float lr);
size_t learned_propose_scratch(int64_t n_rep, int na);
cudaError_t learned_propose(cudaStream_t s, const algdock_ctx& c, const float* params, const uint16_t* wbf16,
                            int64_t n_rep, const int32_t* state_of, float* x, double* comps, int n_moves,
                            int n_torsions, uint64_t seed, uint64_t cycle, int64_t rep_offset, int32_t* accepted,
                            int64_t* counters, void* scratch);
int target_samples_per_block(int na);
cudaError_t launch_target_interaction(cudaStream_t s, int64_t N, int na, const float* x, const TargetFactors* lig_fac,
                                      const ReceptorPair* rec, const float2* rec_q, int n_pairs, double* psi);
size_t fep_scratch_bytes();
cudaError_t launch_fep(cudaStream_t s, int64_t N, const double* ut, int64_t st, const double* us, int64_t ss,
                       double beta, void* scratch, double* out_dev);
cudaError_t launch_exchange(cudaStream_t s, const algdock_ctx& c, int n_ladders, int K, int state_offset,
                            const double* comps, int32_t* config_of, int32_t* state_of, int n_sweeps, int max_sep,
                            uint64_t seed, uint64_t cycle, int64_t ladder_offset, int64_t* attempts,
                            int64_t* accepts);
}  // namespace algdock
