// The context's own run.  The paper's protocol is a loop of cycles over every replica of every
// thermodynamic state ("Equilibration and production"): an HMC move, external-coordinate moves at
// the weakly coupled states ("Sampling"), replica-exchange sweeps, and the snapshot whose reduced
// energies feed MBAR ("Estimation").  algdock_cycle runs one such cycle over arrays the caller
// owns; this file keeps the same arrays inside the context (algdock_replicas_init), runs any
// number of cycles over them with the context's seed and adjustable arguments (algdock_params),
// copies them out, and saves or restores them through the checkpoint format.  It also holds the
// device-side checks of a cycle's results that the params' `checks` setting turns on.
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "internal.cuh"

namespace algdock {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct CheckLegs {
  int n_legs;
  int K[ALGDOCK_MAX_LEGS];
  int off[ALGDOCK_MAX_LEGS];
  int64_t base[ALGDOCK_MAX_LEGS + 1];  // first replica of each leg; base[n_legs] = R
  int n_chains;
  int K_table;
};

// One thread per replica slot r.  Bits of *flag:
//   1  a non-finite position;   2  a non-finite energy component;
//   4  a state index outside the state table;
//   8  a ladder whose config_of is not a permutation of its slots, or whose state_of disagrees.
// config_of[base + c K + i] = v must lie in [0, K) and state_of[base + c K + v] must be the ladder's
// state i; together over i this also makes config_of injective, hence a permutation.
__global__ void run_check_kernel(CheckLegs L, int na, const float* __restrict__ x, const double* __restrict__ comps,
                                 const int32_t* __restrict__ state_of, const int32_t* __restrict__ config_of,
                                 int* flag) {
  const int64_t R = L.base[L.n_legs];
  int bits = 0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
    for (int j = 0; j < 3 * na; ++j)
      if (!isfinite(x[r * 3 * na + j])) bits |= 1;
    for (int j = 0; j < 4; ++j)
      if (!isfinite(comps[4 * r + j])) bits |= 2;
    const int st = state_of[r];
    if (st < 0 || st >= L.K_table) bits |= 4;
    int l = 0;
    while (l + 1 < L.n_legs && r >= L.base[l + 1]) ++l;
    const int K = L.K[l];
    const int64_t rel = r - L.base[l];
    const int64_t ladder = L.base[l] + (rel / K) * K;
    const int i = (int)(rel % K);
    const int v = config_of[r];
    if (v < 0 || v >= K || state_of[ladder + v] != L.off[l] + i) bits |= 8;
  }
  for (int o = 16; o > 0; o >>= 1) bits |= __shfl_xor_sync(kFull, bits, o);
  if ((threadIdx.x & 31) == 0 && bits) atomicOr(flag, bits);
}

struct Device {
  int prev = -1;
  explicit Device(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~Device() {
    int cur;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

algdock_status run_fail(algdock_ctx* c, algdock_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}
algdock_status run_cuda_fail(algdock_ctx* c, cudaError_t e, const char* where) {
  cudaGetLastError();
  return run_fail(c, ALGDOCK_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Replica buffers: [x | comps | state_of | config_of | counters], 256-byte aligned pieces.
size_t piece(size_t bytes) { return (bytes + 255) & ~(size_t)255; }

void replicas_free(algdock_ctx* c) {
  cudaFree(c->d_rbuf);
  c->d_rbuf = nullptr;
  c->has_replicas = false;
  c->n_replicas = 0;
}

// Validates a layout against the context and allocates the buffers for it.
algdock_status replicas_alloc(algdock_ctx* c, const algdock_run_desc& d, const char* where) {
  if (d.n_legs < 1 || d.n_legs > ALGDOCK_MAX_LEGS || d.n_chains < 1 || d.rep_offset < 0 || d.ladder_offset < 0)
    return run_fail(c, ALGDOCK_E_INVALID, std::string(where) + ": bad layout");
  int64_t R = 0;
  for (int l = 0; l < d.n_legs; ++l) {
    if (d.K[l] < 1 || d.K[l] > kMaxLadder || d.state_offset[l] < 0 || d.state_offset[l] + d.K[l] > c->K)
      return run_fail(c, ALGDOCK_E_INVALID, std::string(where) + ": leg outside the state table");
    R += (int64_t)d.n_chains * d.K[l];
  }
  const size_t na = (size_t)c->lig.na;
  const size_t bytes =
      piece(R * na * 12) + piece(R * 32) + piece(R * 4) + piece(R * 4) + piece(ALGDOCK_N_COUNTERS * 8);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return run_cuda_fail(c, e, where);
  replicas_free(c);
  e = cudaMalloc(&c->d_rbuf, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->d_rbuf = nullptr;
    return run_fail(c, ALGDOCK_E_OOM, std::string(where) + ": " + std::to_string(bytes) + " bytes");
  }
  char* p = (char*)c->d_rbuf;
  c->d_rx = (float*)p;
  p += piece(R * na * 12);
  c->d_rcomps = (double*)p;
  p += piece(R * 32);
  c->d_rstate = (int32_t*)p;
  p += piece(R * 4);
  c->d_rcfg = (int32_t*)p;
  p += piece(R * 4);
  c->d_rcnt = (int64_t*)p;
  c->run = d;
  c->n_replicas = R;
  c->has_replicas = true;
  return ALGDOCK_OK;
}

// The run descriptor of the context's replicas with the current params and seed.
algdock_run_desc run_desc_now(const algdock_ctx* c) {
  algdock_run_desc d = c->run;
  d.n_steps = c->params.n_steps;
  d.n_sweeps = c->params.n_sweeps;
  d.max_sep = c->params.max_sep;
  d.n_external = c->params.n_external;
  d.alpha_max = c->params.alpha_max;
  d.sigma_ext = c->params.sigma_ext;
  d.seed = c->seed;
  return d;
}

// The layout as stored in a checkpoint: n_legs, n_chains, rep_offset, ladder_offset, K[n_legs],
// state_offset[n_legs].
std::vector<int64_t> layout_words(const algdock_run_desc& d) {
  std::vector<int64_t> w = {d.n_legs, d.n_chains, d.rep_offset, d.ladder_offset};
  for (int l = 0; l < d.n_legs; ++l) w.push_back(d.K[l]);
  for (int l = 0; l < d.n_legs; ++l) w.push_back(d.state_offset[l]);
  return w;
}

void fill_arrays(algdock_ctx* c, algdock_array* A, int64_t* layout, int64_t n_layout) {
  const int64_t R = c->n_replicas, na = c->lig.na;
  const char* names[6] = {"replicas.layout", "replicas.x", "replicas.comps", "replicas.state_of",
                          "replicas.config_of", "replicas.counters"};
  const int32_t types[6] = {ALGDOCK_I64, ALGDOCK_F32, ALGDOCK_F64, ALGDOCK_I32, ALGDOCK_I32, ALGDOCK_I64};
  const int64_t counts[6] = {n_layout, R * na * 3, R * 4, R, R, ALGDOCK_N_COUNTERS};
  void* data[6] = {layout, c->d_rx, c->d_rcomps, c->d_rstate, c->d_rcfg, c->d_rcnt};
  for (int i = 0; i < 6; ++i) {
    memset(A[i].name, 0, sizeof(A[i].name));
    strncpy(A[i].name, names[i], sizeof(A[i].name) - 1);
    A[i].dtype = types[i];
    A[i].count = counts[i];
    A[i].data = data[i];
  }
}

}  // namespace

int* check_word(algdock_ctx* c) { return (int*)((char*)c->d_work + 128); }

cudaError_t launch_run_check(cudaStream_t s, const algdock_ctx& c, const algdock_run_desc& d, const float* x,
                             const double* comps, const int32_t* state_of, const int32_t* config_of, int* flag) {
  CheckLegs L{};
  L.n_legs = d.n_legs;
  L.n_chains = d.n_chains;
  L.K_table = c.K;
  int64_t base = 0;
  for (int l = 0; l < d.n_legs; ++l) {
    L.K[l] = d.K[l];
    L.off[l] = d.state_offset[l];
    L.base[l] = base;
    base += (int64_t)d.n_chains * d.K[l];
  }
  L.base[d.n_legs] = base;
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (e != cudaSuccess || base == 0) return e;
  const int threads = 256;
  const int64_t want = (base + threads - 1) / threads;
  const int blocks = (int)(want < 4096 ? want : 4096);
  run_check_kernel<<<blocks, threads, 0, s>>>(L, c.lig.na, x, comps, state_of, config_of, flag);
  return cudaGetLastError();
}

algdock_status check_status(algdock_ctx* c, int bits, const char* where) {
  if (bits == 0) return ALGDOCK_OK;
  std::string m = std::string(where) + ": device checks failed:";
  if (bits & 1) m += " non-finite positions;";
  if (bits & 2) m += " non-finite energy components;";
  if (bits & 4) m += " a state index outside the state table;";
  if (bits & 8) m += " a ladder's config_of is not a permutation matching state_of;";
  c->err = m;
  return (bits & 3) ? ALGDOCK_E_NUMERIC : ALGDOCK_E_STATE;
}

algdock_status params_check(algdock_ctx* c, const algdock_params& p) {
  if (p.n_steps < 0 || p.n_sweeps < 0 || p.max_sep < 1 || (int64_t)p.n_sweeps * p.max_sep >= 65536 ||
      p.n_external < 0 || isnan(p.alpha_max) || !(p.sigma_ext >= 0.0) || !isfinite(p.sigma_ext) ||
      !(p.mbar_tol > 0.0) || p.mbar_max_iter < 1 || p.mbar_precision < 0 || p.mbar_precision > 2)
    return run_fail(c, ALGDOCK_E_INVALID,
                    "params: need n_steps >= 0, n_sweeps >= 0, max_sep >= 1, n_sweeps * max_sep < 65536, "
                    "n_external >= 0, alpha_max not NaN, finite sigma_ext >= 0, mbar_tol > 0, "
                    "mbar_max_iter >= 1, mbar_precision 0..2");
  return ALGDOCK_OK;
}

}  // namespace algdock

using namespace algdock;

extern "C" {

algdock_status algdock_params_default(algdock_params* p) {
  if (!p) return ALGDOCK_E_INVALID;
  memset(p, 0, sizeof(*p));
  p->n_steps = 50;
  p->n_sweeps = 25;
  p->max_sep = 5;
  p->n_external = 0;
  p->alpha_max = 0.01;
  p->sigma_ext = 0.6;
  p->mbar_tol = 1e-10;
  p->mbar_max_iter = 10000;
  p->mbar_precision = 0;
  p->checks = 0;
  return ALGDOCK_OK;
}

algdock_status algdock_set_params(algdock_ctx* c, const algdock_params* p) {
  if (!c || !p) return ALGDOCK_E_INVALID;
  const algdock_status st = params_check(c, *p);
  if (st != ALGDOCK_OK) return st;
  c->params = *p;
  return ALGDOCK_OK;
}

algdock_status algdock_get_params(algdock_ctx* c, algdock_params* p, uint64_t* seed) {
  if (!c) return ALGDOCK_E_INVALID;
  if (p) *p = c->params;
  if (seed) *seed = c->seed;
  return ALGDOCK_OK;
}

algdock_status algdock_replicas_init(algdock_ctx* c, int32_t n_legs, const int32_t* K, const int32_t* state_offset,
                                     int32_t n_chains, int64_t rep_offset, int64_t ladder_offset, const float* x0) {
  if (!c) return ALGDOCK_E_INVALID;
  try {
    if (!c->has_grid || !c->has_ligand || c->K == 0)
      return run_fail(c, ALGDOCK_E_STATE, "replicas_init: load grids, ligand and states first");
    if (!K || !state_offset || !x0 || n_legs < 1 || n_legs > ALGDOCK_MAX_LEGS)
      return run_fail(c, ALGDOCK_E_INVALID, "replicas_init: bad arguments");
    algdock_run_desc d{};
    d.n_legs = n_legs;
    for (int l = 0; l < n_legs; ++l) {
      d.K[l] = K[l];
      d.state_offset[l] = state_offset[l];
    }
    d.n_chains = n_chains;
    d.rep_offset = rep_offset;
    d.ladder_offset = ladder_offset;
    Device g(c->device);
    algdock_status st = replicas_alloc(c, d, "replicas_init");
    if (st != ALGDOCK_OK) return st;
    const int64_t R = c->n_replicas;
    std::vector<int32_t> h_state(R), h_cfg(R);
    int64_t base = 0;
    for (int l = 0; l < n_legs; ++l)
      for (int ch = 0; ch < n_chains; ++ch)
        for (int i = 0; i < K[l]; ++i, ++base) {
          h_state[base] = state_offset[l] + i;
          h_cfg[base] = i;
        }
    cudaError_t e = cudaMemcpyAsync(c->d_rx, x0, (size_t)R * c->lig.na * 12, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->d_rstate, h_state.data(), (size_t)R * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_rcfg, h_cfg.data(), (size_t)R * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_rcnt, 0, ALGDOCK_N_COUNTERS * 8, c->stream);
    if (e == cudaSuccess) e = launch_evaluate(c->stream, *c, R, c->d_rx, c->d_rcomps);
    if (e == cudaSuccess && c->params.checks)
      e = launch_run_check(c->stream, *c, c->run, c->d_rx, c->d_rcomps, c->d_rstate, c->d_rcfg, check_word(c));
    if (e == cudaSuccess && c->params.checks)
      e = cudaMemcpyAsync(c->h_flag, check_word(c), sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // the host vectors leave scope
    if (e != cudaSuccess) {
      replicas_free(c);
      return run_cuda_fail(c, e, "replicas_init");
    }
    if (c->params.checks) return check_status(c, *c->h_flag, "replicas_init");
    return ALGDOCK_OK;
  } catch (...) {
    return run_fail(c, ALGDOCK_E_OOM, "replicas_init: host allocation failed");
  }
}

algdock_status algdock_run(algdock_ctx* c, int32_t n_cycles, uint64_t first_cycle, double* u_kn) {
  if (!c) return ALGDOCK_E_INVALID;
  if (!c->has_replicas) return run_fail(c, ALGDOCK_E_STATE, "run: call algdock_replicas_init first");
  if (n_cycles < 0) return run_fail(c, ALGDOCK_E_INVALID, "run: n_cycles < 0");
  const algdock_run_desc d = run_desc_now(c);
  int64_t words = 0;
  for (int l = 0; l < d.n_legs; ++l) words += (int64_t)d.K[l] * d.n_chains * d.K[l];
  NvtxRange range("algdock_run");
  for (int i = 0; i < n_cycles; ++i) {
    const algdock_status st = algdock_cycle(c, &d, first_cycle + (uint64_t)i, c->d_rx, c->d_rcomps, c->d_rstate,
                                            c->d_rcfg, c->d_rcnt, u_kn ? u_kn + (size_t)i * words : nullptr);
    if (st != ALGDOCK_OK) return st;
  }
  return ALGDOCK_OK;
}

algdock_status algdock_replicas_get(algdock_ctx* c, float* x, double* comps, int32_t* state_of, int32_t* config_of,
                                    int64_t* counters) {
  if (!c) return ALGDOCK_E_INVALID;
  if (!c->has_replicas) return run_fail(c, ALGDOCK_E_STATE, "replicas_get: call algdock_replicas_init first");
  Device g(c->device);
  const int64_t R = c->n_replicas;
  struct {
    void* dst;
    const void* src;
    size_t bytes;
  } P[5] = {{x, c->d_rx, (size_t)R * c->lig.na * 12},
            {comps, c->d_rcomps, (size_t)R * 32},
            {state_of, c->d_rstate, (size_t)R * 4},
            {config_of, c->d_rcfg, (size_t)R * 4},
            {counters, c->d_rcnt, (size_t)ALGDOCK_N_COUNTERS * 8}};
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 5 && e == cudaSuccess; ++i)
    if (P[i].dst) e = cudaMemcpyAsync(P[i].dst, P[i].src, P[i].bytes, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return run_cuda_fail(c, e, "replicas_get");
  return ALGDOCK_OK;
}

algdock_status algdock_replicas_save(algdock_ctx* c, const char* path, uint64_t next_cycle) {
  if (!c || !path) return run_fail(c, ALGDOCK_E_INVALID, "replicas_save: bad arguments");
  if (!c->has_replicas) return run_fail(c, ALGDOCK_E_STATE, "replicas_save: call algdock_replicas_init first");
  std::vector<int64_t> layout = layout_words(c->run);
  algdock_array A[6];
  fill_arrays(c, A, layout.data(), (int64_t)layout.size());
  return algdock_checkpoint_save(c, path, c->seed, next_cycle, 6, A);
}

algdock_status algdock_replicas_load(algdock_ctx* c, const char* path, uint64_t* next_cycle) {
  if (!c || !path) return run_fail(c, ALGDOCK_E_INVALID, "replicas_load: bad arguments");
  if (!c->has_grid || !c->has_ligand)
    return run_fail(c, ALGDOCK_E_STATE, "replicas_load: load grids and ligand first");
  algdock_array q{};
  strncpy(q.name, "replicas.layout", sizeof(q.name) - 1);
  q.dtype = ALGDOCK_I64;
  algdock_status st = algdock_checkpoint_load(c, path, nullptr, nullptr, 1, &q);  // sizes only
  if (st != ALGDOCK_OK) return st;
  if (q.dtype != ALGDOCK_I64 || q.count < 6 || q.count > 4 + 2 * ALGDOCK_MAX_LEGS)
    return run_fail(c, ALGDOCK_E_INVALID, "replicas_load: no replica layout in the checkpoint");
  std::vector<int64_t> w((size_t)q.count);
  q.data = w.data();
  st = algdock_checkpoint_load(c, path, nullptr, nullptr, 1, &q);
  if (st != ALGDOCK_OK) return st;
  algdock_run_desc d{};
  d.n_legs = (int)w[0];
  if (d.n_legs < 1 || d.n_legs > ALGDOCK_MAX_LEGS || q.count != 4 + 2 * d.n_legs || w[1] < 1 || w[1] > INT32_MAX)
    return run_fail(c, ALGDOCK_E_INVALID, "replicas_load: bad replica layout");
  d.n_chains = (int)w[1];
  d.rep_offset = w[2];
  d.ladder_offset = w[3];
  for (int l = 0; l < d.n_legs; ++l) {
    if (w[4 + l] < 1 || w[4 + l] > INT32_MAX || w[4 + d.n_legs + l] < 0 || w[4 + d.n_legs + l] > INT32_MAX)
      return run_fail(c, ALGDOCK_E_INVALID, "replicas_load: bad replica layout");
    d.K[l] = (int)w[4 + l];
    d.state_offset[l] = (int)w[4 + d.n_legs + l];
  }
  Device g(c->device);
  st = replicas_alloc(c, d, "replicas_load");
  if (st != ALGDOCK_OK) return st;
  algdock_array A[6];
  fill_arrays(c, A, w.data(), (int64_t)w.size());
  uint64_t seed = 0;
  st = algdock_checkpoint_load(c, path, &seed, next_cycle, 6, A);
  if (st != ALGDOCK_OK) {
    replicas_free(c);
    return st;
  }
  c->seed = seed;
  return ALGDOCK_OK;
}

}  // extern "C"
