// C ABI of libalgdock: argument checking, device-memory ownership, host-side preparation of the
// ligand tables and state weights, and dispatch to the kernels.  See include/algdock.h.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <initializer_list>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace algdock {
size_t mbar_scratch_bytes(int K, int64_t N);
size_t mbar_scratch_bytes_mode(int K, int64_t N, int mode);
size_t mbar_pairs_scratch_bytes(int K, int64_t N);
cudaError_t mbar_local_pairs(cudaStream_t s, void* scratch, int K, int64_t N, const double* u_kn,
                             const int64_t* Nk_host, const double* f_host, int mode, double* pairs_host);
int mbar_run(cudaStream_t s, void* scratch, int K, int64_t N, const double* u_kn, const int64_t* Nk_host,
             double tol, int max_iter, int mode, double* f_host, int* iters, int* h_flag, cudaError_t* err);
}  // namespace algdock

using namespace algdock;

namespace {

algdock_status fail(algdock_ctx* c, algdock_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

algdock_status cuda_fail(algdock_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation) return fail(c, ALGDOCK_E_OOM, std::string(where) + ": out of device memory");
  return fail(c, ALGDOCK_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define ALGDOCK_TRY(c) \
  if (!(c)) return ALGDOCK_E_INVALID; \
  try {
#define ALGDOCK_CATCH(c)                                                   \
  }                                                                        \
  catch (const std::bad_alloc&) {                                          \
    return fail(c, ALGDOCK_E_OOM, "host allocation failed");               \
  }                                                                        \
  catch (...) {                                                            \
    return fail(c, ALGDOCK_E_INVALID, "unexpected exception");             \
  }

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
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

// A device copy of `bytes` from p (host or device); returns the device pointer to use and fills
// `owned` if a temporary was allocated (freed by the caller after the stream is synchronised).
cudaError_t device_view(cudaStream_t s, const void* p, size_t bytes, const void** out, void** owned) {
  *owned = nullptr;
  if (is_device_ptr(p)) {
    *out = p;
    return cudaSuccess;
  }
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, bytes ? bytes : 1);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    cudaFree(d);
    return e;
  }
  *owned = d;
  *out = d;
  return cudaSuccess;
}

// The device word where the tensor-core (tcgen05) GEMMs report a bounded wait that ran out, and its
// check: synchronises the context's stream and turns a set word into ALGDOCK_E_CUDA.
int* tc_err_word(algdock_ctx* c) { return (int*)((char*)c->d_work + 64); }
algdock_status tc_check(algdock_ctx* c, const char* where) {
  cudaError_t e = cudaMemcpyAsync(c->h_flag, tc_err_word(c), sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  if (*c->h_flag != 0)
    return fail(c, ALGDOCK_E_CUDA, std::string(where) + ": a tensor-core GEMM wait timed out (code " +
                                       std::to_string(*c->h_flag) + ")");
  return ALGDOCK_OK;
}

// Host copy of a (host or device) double array.
cudaError_t host_view(cudaStream_t s, const double* p, size_t n, std::vector<double>& out) {
  out.resize(n);
  if (n == 0) return cudaSuccess;
  if (is_device_ptr(p)) {
    cudaError_t e = cudaMemcpyAsync(out.data(), p, n * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
  }
  memcpy(out.data(), p, n * sizeof(double));
  return cudaSuccess;
}

double alpha_sg_of(double a) {
  if (isnan(a)) return 0.0;
  const double s = 2.0 * a - 1.0;
  return 1.0 - s * s;
}
double alpha_g_of(double a) {
  if (isnan(a)) return 0.0;
  const double s = 2.0 * a - 1.0;
  const double z = 1000.0 * (a - 0.5);
  // logistic 1/(1 + e^{-z}) in the form that cannot overflow
  const double logistic = z >= 0.0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z));
  return s * s * logistic;
}

double sqrtA(double rstar, double eps) {
  const double t = 2.0 * rstar;
  return sqrt(eps) * (t * t * t * t * t * t);
}

// SplitMix64 (Steele, Lea and Flood, 2014): the deterministic stream of the gather-layout search.
uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
int below(uint64_t& s, int n) { return (int)(((splitmix64(s) >> 32) * (uint64_t)n) >> 32); }

// Wavefronts of one quarter-warp's 16-byte shared-memory load of bonded slots: 16-byte slots fall
// into 8 bank groups (slot mod 8), the lanes that read one slot share a wavefront, and distinct
// slots of one group take one wavefront each.
int wavefronts(const uint32_t* id, int n) {
  int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0}, worst = 0;
  for (int a = 0; a < n; ++a) {
    bool seen = false;
    for (int b = 0; b < a; ++b) seen = seen || id[b] == id[a];
    if (!seen) worst = std::max(worst, ++cnt[id[a] & 7]);
  }
  return worst;
}

// Layout of the bonded terms and their force gather, chosen against shared-memory bank conflicts.  In
// each round of the bonded terms a quarter-warp loads the positions of its 8 terms' atoms, role by
// role (16 bytes per atom); the kernel's lane l then adds the entries of run lane_run[l] of the
// atom-sorted slot list, so at run position j the four quarter-warps each load 8 slots; the owner
// lanes then load the atoms' partial sums.  Three choices keep every force term (only the order of
// the FP32 additions moves) and move the loads among the 8 bank groups: the order of the terms
// of each kind (a term's slots are base + role n + position), the order of the entries within an
// atom's block, and which lane adds which run.  A simulated annealing over swaps of each kind, with
// integer acceptance (a worsening by d wavefronts is taken with probability 2^-(d b), b rising from 1
// to 32, then greedy) and a fixed seed, minimises the total wavefronts; the result depends on the
// topology only.
struct GatherPlan {
  bool ok = true;
  int na = 0, Lr = 0, n_slots = 0, ng = 0;
  int base[3] = {0, 0, 0}, n[3] = {0, 0, 0}, roles[3] = {2, 3, 4};
  std::vector<int> term_at[3];  // per kind: the input term at each position
  std::vector<uint32_t> ent;    // slot of each entry of the atom-sorted list
  std::vector<int> pos_of;      // entry holding each slot
  std::vector<int> blk0, blk1;  // each atom's block of entries
  std::vector<int> atom_of;     // atom of each entry
  std::vector<int> lane_run, run_lane;
  std::vector<int> part_pos;    // [na][4]: entry whose slot receives the atom's k-th partial sum, or -1
  std::vector<int> part_grp;    // per entry: the partial-sum load group that reads it, or -1
  std::vector<int> tatom[3];    // per kind: the atoms of each input term, roles[kind] per term
  int toff[3] = {0, 0, 0};      // first position-load group of each kind
  std::vector<int> cost;        // wavefronts per load group
  int wf_before = 0, wf_after = 0;  // total wavefronts of the input order and of the layout

  int gather_group(int e) const { return (e % Lr) * 4 + run_lane[e / Lr] / 8; }
  // the load group of the role-r positions read by the quarter-warp holding term position p
  int term_group(int kind, int p, int r) const { return toff[kind] + ((p / 32) * roles[kind] + r) * 4 + (p % 32) / 8; }
  int group_cost(int g) const {
    uint32_t id[8];
    int m = 0;
    if (g >= toff[0]) {  // a bonded-term round's load of one role's atom positions (16 bytes per atom)
      const int kind = g >= toff[2] ? 2 : (g >= toff[1] ? 1 : 0);
      const int h = g - toff[kind], q = h % 4, r = (h / 4) % roles[kind], round = h / (4 * roles[kind]);
      for (int p = 32 * round + 8 * q; p < 32 * round + 8 * q + 8 && p < n[kind]; ++p)
        id[m++] = (uint32_t)tatom[kind][(size_t)term_at[kind][p] * roles[kind] + r];
    } else if (g < 4 * Lr) {
      const int j = g / 4, q = g % 4;
      for (int l = 8 * q; l < 8 * q + 8; ++l) {
        const int e = lane_run[l] * Lr + j;
        id[m++] = e < n_slots ? ent[e] : (uint32_t)n_slots;
      }
    } else {
      const int h = g - 4 * Lr, k = (h / 4) % 4;
      for (int i = 32 * (h / 16) + 8 * (h % 4), i1 = i + 8; i < i1 && i < na; ++i) {
        const int e = part_pos[4 * i + k];
        id[m++] = e >= 0 ? ent[e] : (uint32_t)n_slots;
      }
    }
    return m ? wavefronts(id, m) : 0;
  }

  void swap_entries(int e1, int e2) {
    std::swap(ent[e1], ent[e2]);
    pos_of[ent[e1]] = e1;
    pos_of[ent[e2]] = e2;
  }
  void swap_terms(int kind, int p1, int p2) {
    for (int r = 0; r < roles[kind]; ++r)
      swap_entries(pos_of[base[kind] + r * n[kind] + p1], pos_of[base[kind] + r * n[kind] + p2]);
    std::swap(term_at[kind][p1], term_at[kind][p2]);
  }
  void swap_lanes(int l1, int l2) {
    std::swap(lane_run[l1], lane_run[l2]);
    run_lane[lane_run[l1]] = l1;
    run_lane[lane_run[l2]] = l2;
  }

  // Releases what only the search uses; the build reads term_at, ent, lane_run, part_pos, part_grp.
  void compact() {
    for (auto* v : {&pos_of, &blk0, &blk1, &atom_of, &run_lane, &cost, &tatom[0], &tatom[1], &tatom[2]})
      std::vector<int>().swap(*v);
  }

  void optimise() {
    cost.resize(ng);
    int cur = 0, lower = 0;  // lower: one wavefront per load that reads anything
    for (int g = 0; g < ng; ++g) {
      cost[g] = group_cost(g);
      cur += cost[g];
      lower += cost[g] > 0 ? 1 : 0;
    }
    wf_before = cur;
    int best = cur;
    GatherPlan keep = *this;
    const int terms = n[0] + n[1] + n[2];
    const long iters = std::min<long>(200000, 300L * n_slots);
    uint64_t rs = 0x5deece66dull ^ (uint64_t)n_slots;
    std::vector<int> aff, fresh;
    auto add = [&](int g) {
      if (std::find(aff.begin(), aff.end(), g) == aff.end()) aff.push_back(g);
    };
    auto touch = [&](int e) {
      add(gather_group(e));
      if (part_grp[e] >= 0) add(part_grp[e]);
    };
    for (long it = 0; it < iters && best > lower; ++it) {
      aff.clear();
      // half of the entry and term swaps start from a conflicted load: an entry of a gather load,
      // or a term of a position load
      int tgt = -1, tkind = -1, tpos = -1;
      if (splitmix64(rs) & 1)
        for (int k = 0; k < 8 && tgt < 0 && tkind < 0; ++k) {
          const int g = below(rs, ng);
          if (cost[g] <= 1) continue;
          if (g < 4 * Lr) {
            const int e = lane_run[8 * (g % 4) + below(rs, 8)] * Lr + g / 4;
            if (e < n_slots) tgt = e;
          } else if (g >= toff[0]) {
            const int kd = g >= toff[2] ? 2 : (g >= toff[1] ? 1 : 0);
            const int h = g - toff[kd];
            const int p = 32 * (h / (4 * roles[kd])) + 8 * (h % 4) + below(rs, 8);
            if (p < n[kd]) {
              tkind = kd;
              tpos = p;
            }
          }
        }
      int m = below(rs, 20);
      if (tkind >= 0) m = 8;
      int kind = -1, a1 = 0, a2 = 0;
      if (m < 8) {  // two entries of one atom's block
        const int i = tgt >= 0 ? atom_of[tgt] : below(rs, na);
        const int len = blk1[i] - blk0[i];
        if (len < 2) continue;
        a1 = tgt >= 0 ? tgt : blk0[i] + below(rs, len);
        a2 = blk0[i] + below(rs, len - 1);
        if (a2 >= a1) ++a2;
        touch(a1);
        touch(a2);
        swap_entries(a1, a2);
      } else if (m < 17) {  // two terms of one kind
        if (tkind >= 0) {
          kind = tkind;
        } else if (tgt >= 0) {
          const int id = (int)ent[tgt];
          kind = id < base[1] ? 0 : (id < base[2] ? 1 : 2);
        } else {
          const int u = below(rs, terms);
          kind = u < n[0] ? 0 : (u < n[0] + n[1] ? 1 : 2);
        }
        if (n[kind] < 2) continue;
        a1 = tkind >= 0 ? tpos : (tgt >= 0 ? ((int)ent[tgt] - base[kind]) % n[kind] : below(rs, n[kind]));
        a2 = below(rs, n[kind] - 1);
        if (a2 >= a1) ++a2;
        for (int r = 0; r < roles[kind]; ++r) {
          touch(pos_of[base[kind] + r * n[kind] + a1]);
          touch(pos_of[base[kind] + r * n[kind] + a2]);
          add(term_group(kind, a1, r));
          add(term_group(kind, a2, r));
        }
        swap_terms(kind, a1, a2);
      } else {  // the runs of two lanes in different quarter-warps
        kind = 3;
        a1 = below(rs, 32);
        a2 = 8 * ((a1 / 8 + 1 + below(rs, 3)) % 4) + below(rs, 8);
        for (int j = 0; j < Lr; ++j) {
          add(j * 4 + a1 / 8);
          add(j * 4 + a2 / 8);
        }
        swap_lanes(a1, a2);
      }
      int d = 0;
      fresh.resize(aff.size());
      for (size_t k = 0; k < aff.size(); ++k) {
        fresh[k] = group_cost(aff[k]);
        d += fresh[k] - cost[aff[k]];
      }
      const int b = it < iters * 9 / 10 ? 1 + (int)(32 * it / iters) : 64;
      const bool take = d <= 0 || (d * b < 64 && (splitmix64(rs) >> (64 - d * b)) == 0);
      if (take) {
        for (size_t k = 0; k < aff.size(); ++k) cost[aff[k]] = fresh[k];
        cur += d;
        if (cur < best) {
          best = cur;
          keep = *this;
        }
      } else if (kind < 0) {
        swap_entries(a1, a2);
      } else if (kind < 3) {
        swap_terms(kind, a1, a2);
      } else {
        swap_lanes(a1, a2);
      }
    }
    if (best < cur) *this = keep;
    wf_after = best;
  }
};

// The gather plan of a ligand whose atom indices are in range.  ok is false if an atom's entries
// would meet more than 4 runs.
GatherPlan make_plan(const algdock_ligand* L) {
  const int na = L->n_atoms, nb = L->n_bonds, nang = L->n_angles, ntor = L->n_torsions;
  // per-atom lists of the bonded force slots that act on it (role-major slot numbering by term
  // position: bond role r -> r nb + p; angle -> 2 nb + r nang + p; torsion -> 2 nb + 3 nang + r ntor + p)
  std::vector<std::vector<uint32_t>> inc(na);
  for (int t = 0; t < nb; ++t)
    for (int r = 0; r < 2; ++r) inc[L->bonds[2 * t + r]].push_back((uint32_t)(r * nb + t));
  for (int t = 0; t < nang; ++t)
    for (int r = 0; r < 3; ++r) inc[L->angles[3 * t + r]].push_back((uint32_t)(2 * nb + r * nang + t));
  for (int t = 0; t < ntor; ++t)
    for (int r = 0; r < 4; ++r)
      inc[L->torsions[4 * t + r]].push_back((uint32_t)(2 * nb + 3 * nang + r * ntor + t));
  // Gather schedule of the bonded forces: every slot belongs to exactly one atom, so the slots
  // sorted by atom form one list of n_slots entries.  It is cut into runs of Lr entries, one run
  // per lane, which balances the per-lane work however the slots are spread over atoms.  A lane
  // adds its entries in order and, at the last entry of each atom within its run, stores the
  // partial sum in that entry's slot (which no other lane reads).  Lr is at least a third of the
  // largest atom's count, so that an atom's entries meet at most 4 runs: its owner then adds at
  // most 4 partial sums, in run order.  The term order, the entry order within each atom and the
  // lane of each run are then chosen against shared-memory bank conflicts (GatherPlan).
  const int n_slots = 2 * nb + 3 * nang + 4 * ntor;
  GatherPlan P;
  P.na = na;
  P.n_slots = n_slots;
  P.base[1] = 2 * nb;
  P.base[2] = 2 * nb + 3 * nang;
  P.n[0] = nb;
  P.n[1] = nang;
  P.n[2] = ntor;
  for (int k = 0; k < 3; ++k)
    for (int t = 0; t < P.n[k]; ++t) P.term_at[k].push_back(t);
  P.tatom[0].assign(L->bonds, L->bonds + 2 * nb);
  P.tatom[1].assign(L->angles, L->angles + 3 * nang);
  P.tatom[2].assign(L->torsions, L->torsions + 4 * ntor);
  std::vector<int>& ent_atom = P.atom_of;
  int max_inc = 0;
  for (int i = 0; i < na; ++i) {
    max_inc = std::max(max_inc, (int)inc[i].size());
    P.blk0.push_back((int)P.ent.size());
    for (uint32_t code : inc[i]) {
      P.ent.push_back(code);
      ent_atom.push_back(i);
    }
    P.blk1.push_back((int)P.ent.size());
  }
  const int Lr = n_slots == 0 ? 0 : std::max((n_slots + 31) / 32, (max_inc + 2) / 3);
  P.Lr = Lr;
  if (n_slots > 0) {
    P.pos_of.assign(n_slots + 1, -1);
    for (int e = 0; e < n_slots; ++e) P.pos_of[P.ent[e]] = e;
    P.part_pos.assign((size_t)na * 4, -1);
    P.part_grp.assign(n_slots, -1);
    std::vector<int> n_part(na, 0);
    for (int e = 0; e < n_slots; ++e)
      if (e % Lr == Lr - 1 || e + 1 == n_slots || ent_atom[e + 1] != ent_atom[e]) {
        const int a = ent_atom[e];
        if (n_part[a] >= 4) {
          P.ok = false;
          return P;
        }
        P.part_pos[4 * a + n_part[a]] = e;
        P.part_grp[e] = 4 * Lr + ((a / 32) * 4 + n_part[a]) * 4 + (a % 32) / 8;
        ++n_part[a];
      }
    P.ng = 4 * Lr + 16 * ((na + 31) / 32);
    for (int k = 0; k < 3; ++k) {
      P.toff[k] = P.ng;
      P.ng += ((P.n[k] + 31) / 32) * P.roles[k] * 4;
    }
    for (int l = 0; l < 32; ++l) {
      P.lane_run.push_back(l);
      P.run_lane.push_back(l);
    }
    P.optimise();
  }
  return P;
}

// Plans by topology: the layout depends on the terms' atom indices only, so the contexts of one
// process and the ligands of a batch that share a topology share one search.  At most 1024
// topologies are kept, each with only what the ligand build reads.
std::mutex& plan_mutex() {
  static std::mutex m;
  return m;
}
std::map<std::vector<int32_t>, GatherPlan>& plan_cache() {
  static auto* m = new std::map<std::vector<int32_t>, GatherPlan>();
  return *m;
}
std::vector<int32_t> plan_key(const algdock_ligand* L) {
  std::vector<int32_t> k = {L->n_atoms, L->n_bonds, L->n_angles, L->n_torsions};
  if (L->n_bonds > 0) k.insert(k.end(), L->bonds, L->bonds + 2 * L->n_bonds);
  if (L->n_angles > 0) k.insert(k.end(), L->angles, L->angles + 3 * L->n_angles);
  if (L->n_torsions > 0) k.insert(k.end(), L->torsions, L->torsions + 4 * L->n_torsions);
  return k;
}
GatherPlan cached_plan(const algdock_ligand* L) {
  const std::vector<int32_t> key = plan_key(L);
  {
    std::lock_guard<std::mutex> g(plan_mutex());
    const auto it = plan_cache().find(key);
    if (it != plan_cache().end()) return it->second;
  }
  GatherPlan P = make_plan(L);
  P.compact();
  std::lock_guard<std::mutex> g(plan_mutex());
  if (plan_cache().size() >= 1024) plan_cache().clear();
  plan_cache().emplace(key, P);
  return P;
}

// Whether make_plan can run on L: non-null index arrays, counts in range, indices within the atoms.
bool plannable(const algdock_ligand* L) {
  const int na = L->n_atoms;
  if (na < 1 || na > kMaxAtoms || L->n_bonds < 0 || L->n_angles < 0 || L->n_torsions < 0) return false;
  if ((L->n_bonds && !L->bonds) || (L->n_angles && !L->angles) || (L->n_torsions && !L->torsions)) return false;
  if (2 * L->n_bonds + 3 * L->n_angles + 4 * L->n_torsions >= 0x7fff) return false;
  auto in_range = [&](const int32_t* idx, int n) {
    for (int t = 0; t < n; ++t)
      if (idx[t] < 0 || idx[t] >= na) return false;
    return true;
  };
  return in_range(L->bonds, 2 * L->n_bonds) && in_range(L->angles, 3 * L->n_angles) &&
         in_range(L->torsions, 4 * L->n_torsions);
}

// Searches the plans of a batch's distinct uncached topologies on the host's cores.  A ligand that
// cannot be planned is left to build_ligand, which reports it.
void plan_all(const algdock_ligand* ligs, int n) {
  std::vector<int> todo;
  {
    std::set<std::vector<int32_t>> seen;
    std::lock_guard<std::mutex> g(plan_mutex());
    for (int l = 0; l < n; ++l) {
      if (!plannable(&ligs[l])) continue;
      std::vector<int32_t> key = plan_key(&ligs[l]);
      if (plan_cache().count(key) || seen.count(key)) continue;
      seen.insert(std::move(key));
      todo.push_back(l);
    }
  }
  const int nt = std::min<int>((int)todo.size(), std::max(1u, std::thread::hardware_concurrency()));
  if (nt <= 1) return;
  std::atomic<int> next(0);
  auto work = [&]() {
    try {
      for (int k = next++; k < (int)todo.size(); k = next++) cached_plan(&ligs[todo[k]]);
    } catch (...) {  // a plan that failed to allocate is searched again by build_ligand
    }
  };
  std::vector<std::thread> pool;
  try {
    for (int t = 0; t < nt; ++t) pool.emplace_back(work);
  } catch (...) {  // fewer threads than asked: those started take the whole list
  }
  for (auto& th : pool) th.join();
}

// Validates one ligand and its restraint and builds its device tables: the layout, the blob (atom
// records, pair types, bonded terms, the bonded-force gather schedule, then the per-pair table) and the FP64
// target-force-field factors of each atom.
algdock_status build_ligand(algdock_ctx* c, const algdock_ligand* L, const algdock_restraint* R, const std::string& who,
                            LigandLayout& Y, std::vector<uint32_t>& blob, std::vector<TargetFactors>& fac,
                            Lig64* Y64 = nullptr, std::vector<double>* blob64 = nullptr) {
  if (!L || !R) return fail(c, ALGDOCK_E_INVALID, who + ": null argument");
  const int na = L->n_atoms, nb = L->n_bonds, nang = L->n_angles, ntor = L->n_torsions;
  if (na < 1 || na > kMaxAtoms) return fail(c, ALGDOCK_E_INVALID, who + ": need 1 <= n_atoms <= 96");
  if (nb < 0 || nang < 0 || ntor < 0) return fail(c, ALGDOCK_E_INVALID, who + ": negative term count");
  if (!L->mass || !L->charge || !L->rstar || !L->eps || (nb && (!L->bonds || !L->bond_k || !L->bond_r0)) ||
      (nang && (!L->angles || !L->angle_k || !L->angle_theta0)) ||
      (ntor && (!L->torsions || !L->torsion_V || !L->torsion_gamma)))
    return fail(c, ALGDOCK_E_INVALID, who + ": null array");
  auto bad_idx = [&](const int32_t* idx, int n, int w) {
    for (int t = 0; t < n * w; ++t)
      if (idx[t] < 0 || idx[t] >= na) return true;
    return false;
  };
  if (bad_idx(L->bonds, nb, 2) || bad_idx(L->angles, nang, 3) || bad_idx(L->torsions, ntor, 4))
    return fail(c, ALGDOCK_E_INVALID, who + ": atom index out of range");
  double M = 0.0;
  for (int i = 0; i < na; ++i) {
    if (!(L->mass[i] > 0) || !isfinite(L->mass[i]) || !isfinite(L->charge[i]) || !isfinite(L->rstar[i]) ||
        !(L->eps[i] >= 0) || !isfinite(L->eps[i]))
      return fail(c, ALGDOCK_E_NUMERIC, who + ": non-finite or invalid atom parameter");
    M += L->mass[i];
  }
  for (int t = 0; t < nb; ++t)
    if (!isfinite(L->bond_k[t]) || !isfinite(L->bond_r0[t])) return fail(c, ALGDOCK_E_NUMERIC, who + ": bond");
  for (int t = 0; t < nang; ++t)
    if (!isfinite(L->angle_k[t]) || !isfinite(L->angle_theta0[t]))
      return fail(c, ALGDOCK_E_NUMERIC, who + ": angle");
  for (int t = 0; t < 3 * ntor; ++t)
    if (!isfinite(L->torsion_V[t]) || !isfinite(L->torsion_gamma[t]))
      return fail(c, ALGDOCK_E_NUMERIC, who + ": torsion");
  if (!isfinite(R->k) || !isfinite(R->d0) || !isfinite(R->site[0]) || !isfinite(R->site[1]) || !isfinite(R->site[2]))
    return fail(c, ALGDOCK_E_NUMERIC, who + ": restraint");

  // graph distances (breadth-first over the bonds): exclusions within two bonds, 1-4 at three
  std::vector<std::vector<int>> nbr(na);
  for (int t = 0; t < nb; ++t) {
    nbr[L->bonds[2 * t]].push_back(L->bonds[2 * t + 1]);
    nbr[L->bonds[2 * t + 1]].push_back(L->bonds[2 * t]);
  }
  // pair type [j][i]: 0 nonbonded, 1 1-4 (three bonds apart), 2 excluded (within two bonds, or i == j)
  std::vector<uint8_t> ptype((size_t)na * na, 0);
  std::vector<int> dist(na), queue(na);
  for (int i = 0; i < na; ++i) {
    std::fill(dist.begin(), dist.end(), -1);
    dist[i] = 0;
    int h = 0, t = 0;
    queue[t++] = i;
    while (h < t) {
      const int u = queue[h++];
      if (dist[u] >= 3) continue;
      for (int v : nbr[u])
        if (dist[v] < 0) {
          dist[v] = dist[u] + 1;
          queue[t++] = v;
        }
    }
    for (int j = 0; j < na; ++j) {
      if (dist[j] >= 0 && dist[j] <= 2) ptype[(size_t)j * na + i] = 2;
      else if (dist[j] == 3) ptype[(size_t)j * na + i] = 1;
    }
  }
  // the bonded-force gather schedule of this topology (make_plan)
  const int n_slots = 2 * nb + 3 * nang + 4 * ntor;
  if (n_slots >= 0x7fff) return fail(c, ALGDOCK_E_INVALID, who + ": too many bonded terms");
  const GatherPlan P = cached_plan(L);
  if (!P.ok) return fail(c, ALGDOCK_E_INVALID, who + ": gather schedule overflow");
  const int Lr = P.Lr;
  const int gs_iters = (Lr + 3) / 4;
  std::vector<uint16_t> gs((size_t)gs_iters * 32 * 4, (uint16_t)n_slots);
  std::vector<uint16_t> gp((size_t)na * 4, (uint16_t)n_slots);
  for (int l = 0; l < 32 && Lr > 0; ++l)
    for (int j = 0; j < Lr; ++j) {
      const int e = P.lane_run[l] * Lr + j;
      if (e >= n_slots) break;
      const bool last = P.part_grp[e] >= 0;
      gs[((size_t)(j / 4) * 32 + l) * 4 + (j % 4)] = (uint16_t)(P.ent[e] | (last ? 0x8000u : 0u));
    }
  for (int i = 0; i < 4 * na && Lr > 0; ++i)
    if (P.part_pos[i] >= 0) gp[i] = (uint16_t)P.ent[P.part_pos[i]];

  memset(&Y, 0, sizeof(Y));
  Y.na = na;
  Y.nb = nb;
  Y.nang = nang;
  Y.ntor = ntor;
  Y.gs_iters = gs_iters;
  Y.n_slots = n_slots;
  int w = 0;
  auto take = [&](int words) {
    const int o = w;
    w += (words + 3) & ~3;
    return o;
  };
  Y.off_atom_a = take(4 * na);
  Y.off_atom_b = take(4 * na);
  Y.off_ptype = take((na * na + 3) / 4);
  Y.off_bond = take(4 * nb);
  Y.off_ang = take(8 * nang);
  Y.off_tor = take(16 * ntor);
  Y.off_gs = take(gs_iters * 64);
  Y.off_gp = take(2 * na);
  Y.words = w;
  if ((size_t)w * 4 > 120 * 1024) return fail(c, ALGDOCK_E_INVALID, who + ": topology too large");
  Y.off_pair = take(4 * ((na + 1) / 2) * na);
  Y.words_pair = w;
  blob.assign(w, 0u);
  float* bf = (float*)blob.data();
  int32_t* bi = (int32_t*)blob.data();
  for (int i = 0; i < na; ++i) {
    const double m = L->mass[i];
    const double two_r = 2.0 * L->rstar[i];
    bf[Y.off_atom_a + 4 * i + 0] = (float)(kForceToAccel / m);
    bf[Y.off_atom_a + 4 * i + 1] = (float)L->charge[i];
    bf[Y.off_atom_a + 4 * i + 2] = (float)sqrtA(L->rstar[i], L->eps[i]);
    bf[Y.off_atom_a + 4 * i + 3] = (float)(sqrt(2.0 * L->eps[i]) * two_r * two_r * two_r);
    bf[Y.off_atom_b + 4 * i + 0] = (float)L->rstar[i];
    bf[Y.off_atom_b + 4 * i + 1] = (float)sqrt(L->eps[i]);
    bf[Y.off_atom_b + 4 * i + 2] = (float)m;
    bf[Y.off_atom_b + 4 * i + 3] = (float)sqrt(kForceToAccel / m);
  }
  memcpy((uint8_t*)(blob.data() + Y.off_ptype), ptype.data(), ptype.size());
  // bonded terms at their gather-plan positions (position p holds input term P.term_at[kind][p])
  for (int p = 0; p < nb; ++p) {
    const int t = P.term_at[0][p];
    bi[Y.off_bond + 4 * p + 0] = L->bonds[2 * t];
    bi[Y.off_bond + 4 * p + 1] = L->bonds[2 * t + 1];
    bf[Y.off_bond + 4 * p + 2] = (float)L->bond_k[t];
    bf[Y.off_bond + 4 * p + 3] = (float)L->bond_r0[t];
  }
  for (int p = 0; p < nang; ++p) {
    const int t = P.term_at[1][p];
    for (int k = 0; k < 3; ++k) bi[Y.off_ang + 4 * p + k] = L->angles[3 * t + k];
    bf[Y.off_ang + 4 * nang + 4 * p + 0] = (float)L->angle_k[t];
    bf[Y.off_ang + 4 * nang + 4 * p + 1] = (float)L->angle_theta0[t];
  }
  for (int p = 0; p < ntor; ++p) {
    const int t = P.term_at[2][p];
    for (int k = 0; k < 4; ++k) bi[Y.off_tor + 4 * p + k] = L->torsions[4 * t + k];
    for (int n = 0; n < 3; ++n) {
      const double g = L->torsion_gamma[3 * t + n];
      bf[Y.off_tor + 4 * ntor + 4 * p + n] = (float)(0.5 * L->torsion_V[3 * t + n]);
      bf[Y.off_tor + 8 * ntor + 4 * p + n] = (float)cos(g);
      bf[Y.off_tor + 12 * ntor + 4 * p + n] = (float)sin(g);
    }
  }
  // pair table: the 1-4 scales and the exclusions folded into 8 bytes per ordered pair,
  // (12 eps_ij s_lj, 332 q_i q_j s_el) from FP64, rounded once; excluded pairs (and i == j) hold
  // zeros.  R_ij = R*_i + R*_j is formed in the kernel from the per-atom radii.  Partners are
  // taken two at a time (j = 2p, 2p + 1; an odd na ends with a zero partner j = na), and the two
  // records of atom i share one 16-byte entry (e_ij, e_ij', c_ij, c_ij'), so that one load feeds
  // paired FP32 instructions.
  for (int j = 0; j < 2 * ((na + 1) / 2); ++j)
    for (int i = 0; i < na; ++i) {
      const int ty = j < na ? ptype[(size_t)j * na + i] : 2;
      const double s_lj = ty == 0 ? 1.0 : (ty == 1 ? 0.5 : 0.0);
      const double s_el = ty == 0 ? 1.0 : (ty == 1 ? 1.0 / 1.2 : 0.0);
      float* rec = bf + Y.off_pair + 4 * ((size_t)(j >> 1) * na + i) + (j & 1);
      rec[0] = ty == 2 ? 0.f : (float)(12.0 * s_lj * sqrt(L->eps[i]) * sqrt(L->eps[j]));
      rec[2] = ty == 2 ? 0.f : (float)(kCoulomb * L->charge[i] * L->charge[j] * s_el);
    }
  if (!gs.empty()) memcpy((uint8_t*)(blob.data() + Y.off_gs), gs.data(), gs.size() * sizeof(uint16_t));
  memcpy((uint8_t*)(blob.data() + Y.off_gp), gp.data(), gp.size() * sizeof(uint16_t));
  Y.total_mass = (float)M;
  for (int k = 0; k < 3; ++k) Y.site[k] = (float)R->site[k];
  Y.k_rest = (float)R->k;
  Y.d0 = (float)R->d0;
  fac.resize(na);
  for (int i = 0; i < na; ++i) {
    const double two_r = 2.0 * L->rstar[i];
    fac[i] = TargetFactors{sqrtA(L->rstar[i], L->eps[i]), sqrt(2.0 * L->eps[i]) * two_r * two_r * two_r,
                           kCoulomb * L->charge[i], 0.0};
  }
  if (Y64 && blob64) {  // the all-FP64 path's copy of the parameters, unrounded
    Lig64& G = *Y64;
    std::vector<double>& d = *blob64;
    G.na = na;
    G.nb = nb;
    G.nang = nang;
    G.ntor = ntor;
    G.off_atom = 0;
    G.off_bond = 6 * na;
    G.off_ang = G.off_bond + 4 * nb;
    G.off_tor = G.off_ang + 5 * nang;
    G.off_ptype = G.off_tor + 10 * ntor;
    G.n_doubles = G.off_ptype + na * na;
    d.assign(G.n_doubles > 0 ? G.n_doubles : 1, 0.0);
    for (int i = 0; i < na; ++i) {
      const double two_r = 2.0 * L->rstar[i];
      double* a = &d[G.off_atom + 6 * i];
      a[0] = L->mass[i];
      a[1] = L->charge[i];
      a[2] = sqrtA(L->rstar[i], L->eps[i]);
      a[3] = sqrt(2.0 * L->eps[i]) * two_r * two_r * two_r;
      a[4] = L->rstar[i];
      a[5] = sqrt(L->eps[i]);
    }
    for (int t = 0; t < nb; ++t) {
      double* b = &d[G.off_bond + 4 * t];
      b[0] = L->bonds[2 * t];
      b[1] = L->bonds[2 * t + 1];
      b[2] = L->bond_k[t];
      b[3] = L->bond_r0[t];
    }
    for (int t = 0; t < nang; ++t) {
      double* a = &d[G.off_ang + 5 * t];
      for (int k = 0; k < 3; ++k) a[k] = L->angles[3 * t + k];
      a[3] = L->angle_k[t];
      a[4] = L->angle_theta0[t];
    }
    for (int t = 0; t < ntor; ++t) {
      double* q = &d[G.off_tor + 10 * t];
      for (int k = 0; k < 4; ++k) q[k] = L->torsions[4 * t + k];
      for (int m = 0; m < 3; ++m) {
        q[4 + m] = 0.5 * L->torsion_V[3 * t + m];
        q[7 + m] = L->torsion_gamma[3 * t + m];
      }
    }
    for (int j = 0; j < na; ++j)
      for (int i = 0; i < na; ++i) d[G.off_ptype + (size_t)j * na + i] = ptype[(size_t)j * na + i];
    double M = 0.0;
    for (int i = 0; i < na; ++i) M += L->mass[i];
    G.total_mass = M;
    for (int k = 0; k < 3; ++k) G.site[k] = R->site[k];
    G.k_rest = R->k;
    G.d0 = R->d0;
  }
  return ALGDOCK_OK;
}

// Work items of one batch class: runs of consecutive replicas of one ligand, at most wpb long,
// ordered by decreasing cost (pair work ~ n_atoms^2 plus per-atom work), so that the block scheduler
// starts the longest blocks first.
void batch_items(const algdock_ctx* c, int cls, int wpb, std::vector<BatchItem>& out) {
  out.clear();
  const int64_t n = c->batch_n_rep;
  for (int64_t r = 0; r < n;) {
    const int lig = c->batch_lig_of[r];
    const int k = c->batch_uniform ? kBatchClasses - 1 : c->h_batch[lig].cls;
    int64_t e = r + 1;
    while (e < n && c->batch_lig_of[e] == lig && e - r < wpb) ++e;
    if (k == cls) out.push_back(BatchItem{lig, (int32_t)r, (int32_t)(e - r), 0});
    r = e;
  }
  auto cost = [&](const BatchItem& it) {
    const double na = c->h_batch[it.lig].LL.na;
    return it.count * (na * na + 30.0 * na);
  };
  std::stable_sort(out.begin(), out.end(), [&](const BatchItem& a, const BatchItem& b) { return cost(a) > cost(b); });
}

// The largest block shared memory of a class shape over the ligands it runs (0 if none).
size_t batch_class_smem(const algdock_ctx* c, int cls, int wpb, bool table) {
  size_t m = 0;
  std::vector<char> used(c->n_batch, 0);
  for (int64_t r = 0; r < c->batch_n_rep; ++r) used[c->batch_lig_of[r]] = 1;
  for (int l = 0; l < c->n_batch; ++l) {
    if (!used[l]) continue;
    const int k = c->batch_uniform ? kBatchClasses - 1 : c->h_batch[l].cls;
    if (k != cls) continue;
    m = std::max(m, batch_block_smem(c->h_batch[l].LL, kClassApl[cls], wpb, table));
  }
  return m;
}

// Sets a class's shape and uploads its items.
cudaError_t batch_set_class(algdock_ctx* c, int cls, int wpb, bool table) {
  BatchClass& B = c->batch_cls[cls];
  std::vector<BatchItem> items;
  batch_items(c, cls, wpb, items);
  cudaFree(B.d_items);
  B.d_items = nullptr;
  B.n_items = (int)items.size();
  B.wpb = wpb;
  B.table = table;
  B.smem = batch_class_smem(c, cls, wpb, table);
  if (items.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(&B.d_items, sizeof(BatchItem) * items.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(B.d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice);
  return e;
}

void batch_free(algdock_ctx* c) {
  cudaFree(c->d_batch);
  cudaFree(c->d_batch_blob);
  c->d_batch = nullptr;
  c->d_batch_blob = nullptr;
  for (int k = 0; k < kBatchClasses; ++k) {
    cudaFree(c->batch_cls[k].d_items);
    c->batch_cls[k] = BatchClass{};
  }
  c->n_batch = 0;
  c->batch_n_rep = 0;
  c->h_batch.clear();
  c->batch_lig_of.clear();
}

}  // namespace

extern "C" {

algdock_status algdock_create(int device, uint64_t seed, const algdock_params* params, algdock_ctx** out) {
  if (!out) return ALGDOCK_E_INVALID;
  *out = nullptr;
  algdock_params p;
  algdock_params_default(&p);
  if (params) {
    if (params_check(nullptr, *params) != ALGDOCK_OK) return ALGDOCK_E_INVALID;
    p = *params;
  }
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return ALGDOCK_E_CUDA;
  }
  algdock_ctx* c = new (std::nothrow) algdock_ctx();
  if (!c) return ALGDOCK_E_OOM;
  c->device = device;
  c->seed = seed;
  c->params = p;
  Device g(device);
  int coherent = 0, mappable = 0;
  if (cudaDeviceGetAttribute(&coherent, cudaDevAttrHostNativeAtomicSupported, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&mappable, cudaDevAttrCanMapHostMemory, device) != cudaSuccess) {
    cudaGetLastError();
    coherent = mappable = 0;
  }
  c->host_coherent = coherent && mappable;
  if (cudaMallocHost(&c->h_flag, sizeof(int)) != cudaSuccess) {
    delete c;
    return ALGDOCK_E_CUDA;
  }
  if (cudaMalloc(&c->d_work, 256) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(c->h_flag);
    delete c;
    return ALGDOCK_E_OOM;
  }
  *out = c;
  return ALGDOCK_OK;
}

void algdock_destroy(algdock_ctx* c) {
  if (!c) return;
  Device g(c->device);
  cudaStreamSynchronize(c->stream);
  cudaFree(c->d_hard);
  cudaFree(c->d_soft);
  cudaFree(c->d_blob);
  cudaFree(c->d_states);
  cudaFree(c->d_mbar);
  cudaFree(c->d_learn);
  cudaFree(c->d_proto);
  cudaFree(c->d_rec);
  cudaFree(c->d_lig_fac);
  cudaFree(c->d_fep);
  cudaFree(c->d_lig64);
  cudaFree(c->d_grid64);
  batch_free(c);
  for (int k = 0; k < kBatchClasses; ++k) {
    if (c->batch_side[k]) cudaStreamDestroy(c->batch_side[k]);
    if (c->batch_join[k]) cudaEventDestroy(c->batch_join[k]);
  }
  if (c->batch_fork) cudaEventDestroy(c->batch_fork);
  cudaFreeHost(c->h_flag);
  cudaFree(c->d_work);
  cudaFree(c->d_stage);
  cudaFree(c->d_rbuf);
  if (c->cycle_side) cudaStreamDestroy(c->cycle_side);
  if (c->cycle_fork) cudaEventDestroy(c->cycle_fork);
  if (c->cycle_join) cudaEventDestroy(c->cycle_join);
  delete c;
}

algdock_status algdock_set_stream(algdock_ctx* c, void* stream) {
  if (!c) return ALGDOCK_E_INVALID;
  c->stream = (cudaStream_t)stream;
  return ALGDOCK_OK;
}

const char* algdock_last_error(const algdock_ctx* c) { return c ? c->err.c_str() : "null context"; }

algdock_status algdock_soft_elec_cap(const algdock_ligand* lig, double vmax_r, double* vmax_e) {
  if (!lig || !vmax_e || lig->n_atoms < 1 || !lig->rstar || !lig->eps || !lig->charge) return ALGDOCK_E_INVALID;
  double best = INFINITY;
  for (int i = 0; i < lig->n_atoms; ++i) {
    if (lig->charge[i] == 0.0) continue;
    const double r = sqrtA(lig->rstar[i], lig->eps[i]) / fabs(lig->charge[i]);
    if (r < best) best = r;
  }
  *vmax_e = vmax_r * best;
  return ALGDOCK_OK;
}

algdock_status algdock_gather_layout(const algdock_ligand* lig, int32_t* term_order, uint16_t* slots,
                                     int32_t* lane_run, int32_t* wavefronts) {
  try {
    if (!lig || !plannable(lig)) return ALGDOCK_E_INVALID;
    const GatherPlan P = cached_plan(lig);
    if (!P.ok) return ALGDOCK_E_INVALID;
    if (term_order) {
      int o = 0;
      for (int k = 0; k < 3; ++k)
        for (int t : P.term_at[k]) term_order[o++] = t;
    }
    if (slots)
      for (size_t e = 0; e < P.ent.size(); ++e) slots[e] = (uint16_t)P.ent[e];
    if (lane_run)
      for (int l = 0; l < 32; ++l) lane_run[l] = P.lane_run.empty() ? l : P.lane_run[l];
    if (wavefronts) {
      wavefronts[0] = P.wf_before;
      wavefronts[1] = P.wf_after;
    }
    return ALGDOCK_OK;
  } catch (...) {
    return ALGDOCK_E_OOM;
  }
}

algdock_status algdock_grids_build(algdock_ctx* c, const algdock_grid_desc* d, int32_t n_rec, const double* xyz,
                                   const double* rstar, const double* eps, const double* q, float* ljr, float* lja,
                                   float* elec) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_grids_build");
  if (!d || n_rec < 0 || (n_rec > 0 && (!xyz || !rstar || !eps || !q)) || !ljr || !lja || !elec)
    return fail(c, ALGDOCK_E_INVALID, "grids_build: null argument");
  if (d->n[0] < 2 || d->n[1] < 2 || d->n[2] < 2 || !(d->spacing > 0))
    return fail(c, ALGDOCK_E_INVALID, "grids_build: lattice needs n >= 2 and spacing > 0");
  if (!is_device_ptr(ljr) || !is_device_ptr(lja) || !is_device_ptr(elec))
    return fail(c, ALGDOCK_E_INVALID, "grids_build: outputs must be device pointers");
  Device g(c->device);
  std::vector<double> hx, hr, he, hq;
  cudaError_t e = host_view(c->stream, xyz, 3 * (size_t)n_rec, hx);
  if (e == cudaSuccess) e = host_view(c->stream, rstar, n_rec, hr);
  if (e == cudaSuccess) e = host_view(c->stream, eps, n_rec, he);
  if (e == cudaSuccess) e = host_view(c->stream, q, n_rec, hq);
  if (e != cudaSuccess) return cuda_fail(c, e, "grids_build");
  for (int j = 0; j < n_rec; ++j)
    if (!isfinite(hx[3 * j]) || !isfinite(hx[3 * j + 1]) || !isfinite(hx[3 * j + 2]) || !isfinite(hr[j]) ||
        !isfinite(he[j]) || !isfinite(hq[j]) || he[j] < 0)
      return fail(c, ALGDOCK_E_NUMERIC, "grids_build: non-finite or negative receptor parameter");
  e = launch_grid_build(c->stream, *d, n_rec, hx.data(), hr.data(), he.data(), hq.data(), ljr, lja, elec);
  if (e != cudaSuccess) return cuda_fail(c, e, "grids_build");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_grids_load(algdock_ctx* c, const algdock_grid_desc* d, const float* ljr, const float* lja,
                                  const float* elec, double vmax_r, double vmax_e) {
  ALGDOCK_TRY(c)
  if (!d || !ljr || !lja || !elec) return fail(c, ALGDOCK_E_INVALID, "grids_load: null argument");
  if (d->n[0] < 2 || d->n[1] < 2 || d->n[2] < 2 || !(d->spacing > 0))
    return fail(c, ALGDOCK_E_INVALID, "grids_load: lattice needs n >= 2 and spacing > 0");
  if (!(vmax_r > 0) || !(vmax_e > 0)) return fail(c, ALGDOCK_E_INVALID, "grids_load: caps must be > 0");
  for (int k = 0; k < 3; ++k)
    if ((float)d->origin[k] != d->origin[k])
      return fail(c, ALGDOCK_E_INVALID, "grids_load: origin must be exactly representable in FP32");
  const size_t n = (size_t)d->n[0] * d->n[1] * d->n[2];
  if (n > ((size_t)1 << 31)) return fail(c, ALGDOCK_E_INVALID, "grids_load: lattice too large");
  Device g(c->device);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "grids_load");
  if (n != c->grid_nodes) {
    cudaFree(c->d_hard);
    cudaFree(c->d_soft);
    c->d_hard = nullptr;
    c->d_soft = nullptr;
    c->has_grid = false;
    e = cudaMalloc(&c->d_hard, 2 * n * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_soft, 2 * n * sizeof(float4));
    if (e != cudaSuccess) return cuda_fail(c, e, "grids_load");
    c->grid_nodes = n;
  }
  const void *pr, *pa, *pe;
  void *or_ = nullptr, *oa = nullptr, *oe = nullptr;
  e = device_view(c->stream, ljr, n * 4, &pr, &or_);
  if (e == cudaSuccess) e = device_view(c->stream, lja, n * 4, &pa, &oa);
  if (e == cudaSuccess) e = device_view(c->stream, elec, n * 4, &pe, &oe);
  if (e == cudaSuccess)
    e = launch_grid_prepare(c->stream, n, d->n[0], d->n[1], (const float*)pr, (const float*)pa, (const float*)pe,
                            vmax_r, vmax_e, c->d_hard, c->d_soft);
  if (or_ || oa || oe) {
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = e2;
    cudaFree(or_);
    cudaFree(oa);
    cudaFree(oe);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "grids_load");
  GridDev G;
  G.hard = c->d_hard;
  G.soft = c->d_soft;
  G.nx = d->n[0];
  G.ny = d->n[1];
  G.nz = d->n[2];
  G.ox = (float)d->origin[0];
  G.oy = (float)d->origin[1];
  G.oz = (float)d->origin[2];
  G.inv_h = (float)(1.0 / d->spacing);
  c->grid = G;
  c->has_grid = true;
  const double fpd[6] = {d->origin[0], d->origin[1], d->origin[2], d->spacing, vmax_r, vmax_e};
  const int32_t fpn[3] = {d->n[0], d->n[1], d->n[2]};
  c->fp_grid = crc32_update(crc32_update(0, fpd, sizeof(fpd)), fpn, sizeof(fpn));
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_grids_load_f64(algdock_ctx* c, const algdock_grid_desc* d, const double* ljr, const double* lja,
                                      const double* elec, double vmax_r, double vmax_e) {
  ALGDOCK_TRY(c)
  if (!d || !ljr || !lja || !elec) return fail(c, ALGDOCK_E_INVALID, "grids_load_f64: null argument");
  if (d->n[0] < 2 || d->n[1] < 2 || d->n[2] < 2 || !(d->spacing > 0))
    return fail(c, ALGDOCK_E_INVALID, "grids_load_f64: lattice needs n >= 2 and spacing > 0");
  if (!(vmax_r > 0) || !(vmax_e > 0)) return fail(c, ALGDOCK_E_INVALID, "grids_load_f64: caps must be > 0");
  const size_t n = (size_t)d->n[0] * d->n[1] * d->n[2];
  if (n > ((size_t)1 << 31)) return fail(c, ALGDOCK_E_INVALID, "grids_load_f64: lattice too large");
  Device g(c->device);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "grids_load_f64");
  if (n != c->grid64_nodes) {
    cudaFree(c->d_grid64);
    c->d_grid64 = nullptr;
    c->has_grid64 = false;
    e = cudaMalloc(&c->d_grid64, n * (sizeof(Hard64) + sizeof(Soft64)));
    if (e != cudaSuccess) return cuda_fail(c, e, "grids_load_f64");
    c->grid64_nodes = n;
  }
  Hard64* hard = (Hard64*)c->d_grid64;
  Soft64* soft = (Soft64*)((uint8_t*)c->d_grid64 + n * sizeof(Hard64));
  const void *pr, *pa, *pe;
  void *or_ = nullptr, *oa = nullptr, *oe = nullptr;
  e = device_view(c->stream, ljr, n * 8, &pr, &or_);
  if (e == cudaSuccess) e = device_view(c->stream, lja, n * 8, &pa, &oa);
  if (e == cudaSuccess) e = device_view(c->stream, elec, n * 8, &pe, &oe);
  if (e == cudaSuccess)
    e = launch_grid_prepare64(c->stream, n, (const double*)pr, (const double*)pa, (const double*)pe, vmax_r, vmax_e,
                              hard, soft);
  if (or_ || oa || oe) {
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = e2;
    cudaFree(or_);
    cudaFree(oa);
    cudaFree(oe);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "grids_load_f64");
  GridDev64 G;
  G.hard = hard;
  G.soft = soft;
  G.nx = d->n[0];
  G.ny = d->n[1];
  G.nz = d->n[2];
  G.ox = d->origin[0];
  G.oy = d->origin[1];
  G.oz = d->origin[2];
  G.h = d->spacing;
  c->grid64 = G;
  c->has_grid64 = true;
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_energy_force_f64(algdock_ctx* c, int64_t N, const int32_t* state_of, const float* x,
                                        double* force, double* comps) {
  ALGDOCK_TRY(c)
  if (!c->has_grid64 || !c->has_ligand || (state_of && c->K == 0))
    return fail(c, ALGDOCK_E_STATE, "energy_force_f64: load FP64 grids, the ligand (and states) first");
  if (N < 0 || !comps) return fail(c, ALGDOCK_E_INVALID, "energy_force_f64: need N >= 0 and comps");
  if (N == 0) return ALGDOCK_OK;
  if (!is_device_ptr(x) || !is_device_ptr(comps) || (state_of && !is_device_ptr(state_of)) ||
      (force && !is_device_ptr(force)))
    return fail(c, ALGDOCK_E_INVALID, "energy_force_f64: arrays must be device pointers");
  Device g(c->device);
  cudaError_t e = launch_eval64(c->stream, *c, N, state_of, x, force, comps);
  if (e != cudaSuccess) return cuda_fail(c, e, "energy_force_f64");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_gather_probe(algdock_ctx* c, int64_t n_cells, int32_t soft, uint64_t seed, float* sink) {
  ALGDOCK_TRY(c)
  if (!c->has_grid) return fail(c, ALGDOCK_E_STATE, "gather_probe: load grids first");
  if (n_cells < 0 || !sink || !is_device_ptr(sink))
    return fail(c, ALGDOCK_E_INVALID, "gather_probe: need n_cells >= 0 and a device sink");
  Device g(c->device);
  cudaError_t e = launch_gather_probe(c->stream, *c, n_cells, soft != 0, (uint32_t)seed, sink);
  if (e != cudaSuccess) return cuda_fail(c, e, "gather_probe");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_ligand_load(algdock_ctx* c, const algdock_ligand* L, const algdock_restraint* R) {
  ALGDOCK_TRY(c)
  LigandLayout Y;
  std::vector<uint32_t> blob;
  std::vector<TargetFactors> fac;
  Lig64 Y64{};
  std::vector<double> blob64;
  algdock_status st = build_ligand(c, L, R, "ligand_load", Y, blob, fac, &Y64, &blob64);
  if (st != ALGDOCK_OK) return st;
  const int na = Y.na, nb = Y.nb, w = Y.words_pair;

  Device g(c->device);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "ligand_load");
  cudaFree(c->d_blob);
  cudaFree(c->d_lig_fac);
  c->d_blob = nullptr;
  c->d_lig_fac = nullptr;
  c->has_ligand = false;
  e = cudaMalloc(&c->d_blob, (size_t)w * 4);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_blob, blob.data(), (size_t)w * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_lig_fac, sizeof(TargetFactors) * na);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_lig_fac, fac.data(), sizeof(TargetFactors) * na, cudaMemcpyHostToDevice);
  cudaFree(c->d_lig64);
  c->d_lig64 = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&c->d_lig64, sizeof(double) * blob64.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(c->d_lig64, blob64.data(), sizeof(double) * blob64.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(c, e, "ligand_load");
  c->lig = Y;
  c->lig64 = Y64;
  build_learned_topo(na, nb, L->bonds, &c->ltopo);
  c->has_ligand = true;
  c->fp_ligand = crc32_update(crc32_update(0, blob.data(), blob.size() * 4), &Y, sizeof(Y));
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_states_set(algdock_ctx* c, int32_t K, const double* T, const double* alpha,
                                  const double* dt_fs) {
  ALGDOCK_TRY(c)
  if (K < 1 || !T || !alpha || !dt_fs) return fail(c, ALGDOCK_E_INVALID, "states_set: bad arguments");
  std::vector<StateDev> h(K);
  for (int k = 0; k < K; ++k) {
    if (!(T[k] > 0) || !isfinite(T[k]) || !(dt_fs[k] >= 0) || !isfinite(dt_fs[k]) ||
        (!isnan(alpha[k]) && !isfinite(alpha[k])))
      return fail(c, ALGDOCK_E_INVALID, "states_set: need T > 0, dt >= 0, finite alpha or NaN");
    StateDev s;
    s.kT = kBoltzmann * T[k];
    s.beta = 1.0 / (kBoltzmann * T[k]);
    s.w_sg = alpha_sg_of(alpha[k]);
    s.w_g = alpha_g_of(alpha[k]);
    s.alpha = alpha[k];
    s.w_sg_f = (float)s.w_sg;
    s.w_g_f = (float)s.w_g;
    s.dt = (float)dt_fs[k];
    s.sqrt_kT = (float)sqrt(s.kT);
    h[k] = s;
  }
  Device g(c->device);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "states_set");
  cudaFree(c->d_states);
  c->d_states = nullptr;
  c->K = 0;
  e = cudaMalloc(&c->d_states, sizeof(StateDev) * K);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_states, h.data(), sizeof(StateDev) * K, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(c, e, "states_set");
  c->K = K;
  c->h_T.assign(T, T + K);
  c->h_alpha.assign(alpha, alpha + K);
  c->h_dt.assign(dt_fs, dt_fs + K);
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_hmc_cycle(algdock_ctx* c, int64_t n_rep, const int32_t* state_of, float* x, double* comps,
                                 double* dH, uint8_t* accepted, int32_t n_steps, uint64_t seed, uint64_t cycle,
                                 int64_t rep_offset, int64_t* counters) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_hmc_cycle");
  if (!c->has_grid || !c->has_ligand || c->K == 0)
    return fail(c, ALGDOCK_E_STATE, "hmc_cycle: load grids, ligand and states first");
  if (n_rep < 0 || n_steps < 0 || rep_offset < 0) return fail(c, ALGDOCK_E_INVALID, "hmc_cycle: negative size");
  if (n_rep == 0) return ALGDOCK_OK;
  if (!is_device_ptr(state_of) || !is_device_ptr(x) || !is_device_ptr(comps) || (dH && !is_device_ptr(dH)) ||
      (accepted && !is_device_ptr(accepted)) || (counters && !is_device_ptr(counters)))
    return fail(c, ALGDOCK_E_INVALID, "hmc_cycle: arrays must be device pointers");
  Device g(c->device);
  cudaError_t e = launch_hmc(c->stream, *c, n_rep, state_of, x, comps, dH, accepted, n_steps, seed, cycle,
                             rep_offset, counters);
  if (e != cudaSuccess) return cuda_fail(c, e, "hmc_cycle");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_external_moves(algdock_ctx* c, int64_t n_rep, const int32_t* state_of, float* x,
                                      double* comps, int32_t n_moves, double alpha_max, double sigma, uint64_t seed,
                                      uint64_t cycle, int64_t rep_offset, int32_t* accepted, int64_t* counters) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_external_moves");
  if (!c->has_grid || !c->has_ligand || c->K == 0)
    return fail(c, ALGDOCK_E_STATE, "external_moves: load grids, ligand and states first");
  if (n_rep < 0 || n_moves < 0 || rep_offset < 0) return fail(c, ALGDOCK_E_INVALID, "external_moves: negative size");
  if (!(sigma >= 0.0) || !isfinite(sigma) || isnan(alpha_max))
    return fail(c, ALGDOCK_E_INVALID, "external_moves: need finite sigma >= 0 and alpha_max not NaN");
  if (n_rep == 0 || n_moves == 0) return ALGDOCK_OK;
  if (!is_device_ptr(state_of) || !is_device_ptr(x) || !is_device_ptr(comps) ||
      (accepted && !is_device_ptr(accepted)) || (counters && !is_device_ptr(counters)))
    return fail(c, ALGDOCK_E_INVALID, "external_moves: arrays must be device pointers");
  Device g(c->device);
  cudaError_t e = launch_external(c->stream, *c, n_rep, state_of, x, comps, n_moves, alpha_max, (float)sigma, seed,
                                  cycle, rep_offset, accepted, counters);
  if (e != cudaSuccess) return cuda_fail(c, e, "external_moves");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_detect_equilibration(algdock_ctx* c, int64_t T, int64_t S, const double* series,
                                            int64_t stride, int32_t n_cand, double* g, int64_t* t0_best,
                                            double* neff_best) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_detect_equilibration");
  if (T < 2 || T > 50000 || S < 1 || S > 65535 || stride < 1 || n_cand < 1 || (int64_t)(n_cand - 1) * stride > T - 2)
    return fail(c, ALGDOCK_E_INVALID, "detect_equilibration: need 2 <= T <= 50000, 1 <= S <= 65535, stride >= 1, "
                                      "n_cand >= 1, (n_cand - 1) * stride <= T - 2");
  if (!is_device_ptr(series) || !is_device_ptr(g) || (t0_best && !is_device_ptr(t0_best)) ||
      (neff_best && !is_device_ptr(neff_best)))
    return fail(c, ALGDOCK_E_INVALID, "detect_equilibration: arrays must be device pointers");
  Device dg(c->device);
  cudaError_t e = launch_equilibration(c->stream, T, S, series, stride, n_cand, g, t0_best, neff_best);
  if (e != cudaSuccess) return cuda_fail(c, e, "detect_equilibration");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

// Protocol scratch: 4 result doubles, then n weights.
static algdock_status proto_scratch(algdock_ctx* c, int64_t n, const char* where) {
  const size_t need = 256 + (size_t)n * sizeof(double);
  if (need <= c->proto_bytes) return ALGDOCK_OK;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  cudaFree(c->d_proto);
  c->d_proto = nullptr;
  c->proto_bytes = 0;
  e = cudaMalloc(&c->d_proto, need);
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  c->proto_bytes = need;
  return ALGDOCK_OK;
}

static algdock_status proto_check(algdock_ctx* c, int64_t N, std::initializer_list<int> ks, const char* where) {
  if (c->K == 0) return fail(c, ALGDOCK_E_STATE, std::string(where) + ": set the states first");
  if (N < 1) return fail(c, ALGDOCK_E_INVALID, std::string(where) + ": N < 1");
  for (int k : ks)
    if (k < 0 || k >= c->K) return fail(c, ALGDOCK_E_INVALID, std::string(where) + ": state index out of range");
  return ALGDOCK_OK;
}

algdock_status algdock_state_statistics(algdock_ctx* c, int64_t N, const double* comps, int32_t k, double* sigma) {
  ALGDOCK_TRY(c)
  algdock_status st = proto_check(c, N, {k}, "state_statistics");
  if (st != ALGDOCK_OK) return st;
  if (!sigma || !is_device_ptr(comps)) return fail(c, ALGDOCK_E_INVALID, "state_statistics: bad pointers");
  Device g(c->device);
  if ((st = proto_scratch(c, 1, "state_statistics")) != ALGDOCK_OK) return st;
  double* out = (double*)c->d_proto;
  cudaError_t e = launch_state_stats(c->stream, *c, N, comps, k, out);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sigma, out, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "state_statistics");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_resample(algdock_ctx* c, int64_t N, const double* comps, int32_t k_from, int32_t k_to,
                                int32_t n_out, uint64_t seed, uint32_t counter, const float* x_in, float* x_out,
                                int64_t* idx) {
  ALGDOCK_TRY(c)
  algdock_status st = proto_check(c, N, {k_from, k_to}, "resample");
  if (st != ALGDOCK_OK) return st;
  if (n_out < 1 || n_out > 1024) return fail(c, ALGDOCK_E_INVALID, "resample: need 1 <= n_out <= 1024");
  if ((x_in || x_out) && !c->has_ligand) return fail(c, ALGDOCK_E_STATE, "resample: load the ligand first");
  if (!is_device_ptr(comps) || (idx && !is_device_ptr(idx)) || (x_in && !is_device_ptr(x_in)) ||
      (x_out && !is_device_ptr(x_out)) || (!x_in != !x_out))
    return fail(c, ALGDOCK_E_INVALID, "resample: arrays must be device pointers (x_in and x_out together)");
  Device g(c->device);
  if ((st = proto_scratch(c, N, "resample")) != ALGDOCK_OK) return st;
  double* work = (double*)((char*)c->d_proto + 256);
  cudaError_t e = launch_resample(c->stream, *c, N, comps, k_from, k_to, n_out, seed, counter, work, idx, x_in, x_out);
  if (e != cudaSuccess) return cuda_fail(c, e, "resample");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_mean_pacc(algdock_ctx* c, int64_t N, const double* comps_a, const double* comps_b, int32_t ka,
                                 int32_t kb, double* p) {
  ALGDOCK_TRY(c)
  algdock_status st = proto_check(c, N, {ka, kb}, "mean_pacc");
  if (st != ALGDOCK_OK) return st;
  if (!p || !is_device_ptr(comps_a) || !is_device_ptr(comps_b)) return fail(c, ALGDOCK_E_INVALID, "mean_pacc: bad pointers");
  Device g(c->device);
  if ((st = proto_scratch(c, 1, "mean_pacc")) != ALGDOCK_OK) return st;
  double* out = (double*)c->d_proto;
  cudaError_t e = launch_pacc(c->stream, *c, N, comps_a, comps_b, ka, kb, out);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p, out, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "mean_pacc");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_receptor_load(algdock_ctx* c, int32_t n_rec, const double* xyz, const double* rstar,
                                    const double* eps, const double* q) {
  ALGDOCK_TRY(c)
  if (n_rec < 0 || (n_rec > 0 && (!xyz || !rstar || !eps || !q)))
    return fail(c, ALGDOCK_E_INVALID, "receptor_load: null argument");
  Device g(c->device);
  std::vector<double> hx, hr, he, hq;
  cudaError_t e = host_view(c->stream, xyz, 3 * (size_t)n_rec, hx);
  if (e == cudaSuccess) e = host_view(c->stream, rstar, n_rec, hr);
  if (e == cudaSuccess) e = host_view(c->stream, eps, n_rec, he);
  if (e == cudaSuccess) e = host_view(c->stream, q, n_rec, hq);
  if (e != cudaSuccess) return cuda_fail(c, e, "receptor_load");
  for (int j = 0; j < n_rec; ++j)
    if (!isfinite(hx[3 * j]) || !isfinite(hx[3 * j + 1]) || !isfinite(hx[3 * j + 2]) || !isfinite(hr[j]) ||
        !isfinite(he[j]) || !isfinite(hq[j]) || he[j] < 0)
      return fail(c, ALGDOCK_E_NUMERIC, "receptor_load: non-finite or negative receptor parameter");
  // pairs of atoms (2k, 2k + 1) for the paired FP32 instructions; an odd count ends with a zero
  // atom (no coefficients), whose terms vanish
  const size_t n_pairs = n_rec > 0 ? ((size_t)n_rec + 1) / 2 : 1;
  std::vector<ReceptorPair> hp(n_pairs);
  std::vector<float2> hq2(n_pairs, make_float2(0.f, 0.f));
  float hi[2][3], lo[2][3], sa[2], sb[2], qq[2];
  for (size_t k = 0; k < n_pairs; ++k) {
    for (int u = 0; u < 2; ++u) {
      const size_t j = 2 * k + u;
      const bool real = j < (size_t)n_rec;
      for (int d = 0; d < 3; ++d) {
        hi[u][d] = real ? (float)hx[3 * j + d] : 0.f;
        lo[u][d] = real ? (float)(hx[3 * j + d] - (double)hi[u][d]) : 0.f;
      }
      const double two_r = real ? 2.0 * hr[j] : 0.0;
      sa[u] = real ? (float)sqrtA(hr[j], he[j]) : 0.f;
      sb[u] = real ? (float)(sqrt(2.0 * he[j]) * two_r * two_r * two_r) : 0.f;
      qq[u] = real ? (float)(hq[j] / 4.0) : 0.f;
    }
    hp[k].c0 = make_float4(hi[0][0], hi[1][0], hi[0][1], hi[1][1]);
    hp[k].c1 = make_float4(hi[0][2], hi[1][2], lo[0][0], lo[1][0]);
    hp[k].c2 = make_float4(lo[0][1], lo[1][1], lo[0][2], lo[1][2]);
    hp[k].c3 = make_float4(sa[0], sa[1], sb[0], sb[1]);
    hq2[k] = make_float2(qq[0], qq[1]);
  }
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "receptor_load");
  cudaFree(c->d_rec);
  c->d_rec = nullptr;
  c->n_rec = -1;
  const size_t bytes = sizeof(ReceptorPair) * n_pairs + sizeof(float2) * n_pairs;
  e = cudaMalloc(&c->d_rec, bytes);
  uint8_t* base = (uint8_t*)c->d_rec;
  if (e == cudaSuccess) e = cudaMemcpy(base, hp.data(), sizeof(ReceptorPair) * n_pairs, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(base + sizeof(ReceptorPair) * n_pairs, hq2.data(), sizeof(float2) * n_pairs, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(c, e, "receptor_load");
  c->n_rec = n_rec;
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_target_interaction(algdock_ctx* c, int64_t N, const float* x, double* psi) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_target_interaction");
  if (!c->has_ligand || c->n_rec < 0)
    return fail(c, ALGDOCK_E_STATE, "target_interaction: load the ligand and the receptor first");
  if (N < 0) return fail(c, ALGDOCK_E_INVALID, "target_interaction: N < 0");
  if (N == 0) return ALGDOCK_OK;
  if (!is_device_ptr(x) || !is_device_ptr(psi))
    return fail(c, ALGDOCK_E_INVALID, "target_interaction: x and psi must be device pointers");
  Device g(c->device);
  const size_t n_pairs = c->n_rec > 0 ? ((size_t)c->n_rec + 1) / 2 : 1;
  const uint8_t* base = (const uint8_t*)c->d_rec;
  cudaError_t e = launch_target_interaction(c->stream, N, c->lig.na, x, c->d_lig_fac, (const ReceptorPair*)base,
                                            (const float2*)(base + sizeof(ReceptorPair) * n_pairs),
                                            c->n_rec > 0 ? (int)n_pairs : 0, psi);
  if (e != cudaSuccess) return cuda_fail(c, e, "target_interaction");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_fep(algdock_ctx* c, int64_t N, const double* u_target, int64_t stride_target,
                           const double* u_sampling, int64_t stride_sampling, double beta, double* result) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_fep");
  if (N < 1 || !u_target || !result || stride_target < 0 || stride_sampling < 0 || !isfinite(beta))
    return fail(c, ALGDOCK_E_INVALID, "fep: need N >= 1, strides >= 0, finite beta and non-null arrays");
  if (!is_device_ptr(u_target) || (u_sampling && !is_device_ptr(u_sampling)))
    return fail(c, ALGDOCK_E_INVALID, "fep: energies must be device pointers");
  Device g(c->device);
  cudaError_t e = cudaSuccess;
  if (!c->d_fep) e = cudaMalloc(&c->d_fep, fep_scratch_bytes());
  if (e != cudaSuccess) return cuda_fail(c, e, "fep");
  double* out = (double*)((uint8_t*)c->d_fep + fep_scratch_bytes() - 8 * sizeof(double));
  double h[5];
  e = launch_fep(c->stream, N, u_target, stride_target, u_sampling, stride_sampling, beta, c->d_fep, out);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "fep");
  for (int k = 0; k < 4; ++k) result[k] = h[k];
  if (h[4] > 0) return fail(c, ALGDOCK_E_NUMERIC, "fep: NaN or -inf energy difference");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_batch_load(algdock_ctx* c, int32_t n_ligands, const algdock_ligand* ligands,
                                  const algdock_restraint* rest) {
  ALGDOCK_TRY(c)
  if (n_ligands < 1 || !ligands || !rest) return fail(c, ALGDOCK_E_INVALID, "batch_load: need n_ligands >= 1");
  std::vector<BatchLigand> recs(n_ligands);
  std::vector<uint32_t> all;
  int max_na = 0;
  Device g(c->device);  // the class test queries the batch kernels' limits on this device
  plan_all(ligands, n_ligands);
  for (int l = 0; l < n_ligands; ++l) {
    LigandLayout Y;
    std::vector<uint32_t> blob;
    std::vector<TargetFactors> fac;
    algdock_status st = build_ligand(c, &ligands[l], rest, "batch_load: ligand " + std::to_string(l), Y, blob, fac);
    if (st != ALGDOCK_OK) return st;
    recs[l].LL = Y;
    recs[l].blob_off = (int64_t)all.size();  // blob sizes are multiples of 4 words: 16-byte aligned
    recs[l].apl = Y.na <= 32 ? 1 : (Y.na <= 64 ? 2 : 3);
    recs[l].cls = recs[l].apl == 1 ? 0 : (recs[l].apl == 3 ? 3 : (batch_uses_table16(Y) ? 1 : 2));
    all.insert(all.end(), blob.begin(), blob.end());
    max_na = std::max(max_na, Y.na);
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "batch_load");
  batch_free(c);
  for (int k = 0; k < kBatchClasses && e == cudaSuccess; ++k) {
    if (!c->batch_side[k]) e = cudaStreamCreateWithFlags(&c->batch_side[k], cudaStreamNonBlocking);
    if (e == cudaSuccess && !c->batch_join[k]) e = cudaEventCreateWithFlags(&c->batch_join[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess && !c->batch_fork) e = cudaEventCreateWithFlags(&c->batch_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_batch, sizeof(BatchLigand) * n_ligands);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_batch_blob, all.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_batch, recs.data(), sizeof(BatchLigand) * n_ligands, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_batch_blob, all.data(), all.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    batch_free(c);
    return cuda_fail(c, e, "batch_load");
  }
  c->h_batch = recs;
  c->n_batch = n_ligands;
  c->batch_max_na = max_na;
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_batch_layout(algdock_ctx* c, int64_t n_rep, const int32_t* lig_of, int32_t x_stride,
                                    int32_t uniform) {
  ALGDOCK_TRY(c)
  if (c->n_batch == 0) return fail(c, ALGDOCK_E_STATE, "batch_layout: load a batch first");
  if (n_rep < 1 || n_rep > INT32_MAX || !lig_of || x_stride < 1 || x_stride > kMaxAtoms)
    return fail(c, ALGDOCK_E_INVALID, "batch_layout: need n_rep >= 1, lig_of and 1 <= x_stride <= 96");
  if (is_device_ptr(lig_of)) return fail(c, ALGDOCK_E_INVALID, "batch_layout: lig_of must be a host array");
  for (int64_t r = 0; r < n_rep; ++r) {
    if (lig_of[r] < 0 || lig_of[r] >= c->n_batch)
      return fail(c, ALGDOCK_E_INVALID, "batch_layout: ligand index out of range");
    if (c->h_batch[lig_of[r]].LL.na > x_stride)
      return fail(c, ALGDOCK_E_INVALID, "batch_layout: x_stride is smaller than a ligand's atom count");
  }
  Device g(c->device);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "batch_layout");
  c->batch_lig_of.assign(lig_of, lig_of + n_rep);
  c->batch_n_rep = n_rep;
  c->batch_x_stride = x_stride;
  c->batch_uniform = uniform != 0;
  // default shape per class: the first candidate whose shared memory fits every ligand it runs
  for (int k = 0; k < kBatchClasses && e == cudaSuccess; ++k) {
    int wpb[4];
    bool table[4];
    const int nc = c->batch_uniform && k < kBatchClasses - 1 ? 0 : batch_candidates(k, wpb, table);
    int pick = -1;
    for (int t = 0; t < nc && pick < 0; ++t)
      if (batch_class_smem(c, k, wpb[t], table[t]) <= batch_smem_limit(kClassApl[k], wpb[t], table[t])) pick = t;
    if (pick < 0) {
      e = batch_set_class(c, k, 4, false);
      if (e == cudaSuccess && c->batch_cls[k].n_items > 0 &&
          c->batch_cls[k].smem > batch_smem_limit(kClassApl[k], 4, false)) {
        batch_free(c);
        return fail(c, ALGDOCK_E_INVALID, "batch_layout: a ligand's tables exceed shared memory");
      }
    } else {
      e = batch_set_class(c, k, wpb[pick], table[pick]);
    }
  }
  if (e == cudaSuccess) e = batch_set_attributes(*c);
  if (e != cudaSuccess) return cuda_fail(c, e, "batch_layout");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_batch_hmc_cycle(algdock_ctx* c, const int32_t* state_of, float* x, double* comps, double* dH,
                                       uint8_t* acc, int32_t n_steps, uint64_t seed, uint64_t cycle,
                                       int64_t rep_offset, int64_t* counters) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_batch_hmc_cycle");
  if (!c->has_grid || c->K == 0 || c->batch_n_rep == 0)
    return fail(c, ALGDOCK_E_STATE, "batch_hmc_cycle: load grids, states, a batch and its layout first");
  if (n_steps < 0 || rep_offset < 0) return fail(c, ALGDOCK_E_INVALID, "batch_hmc_cycle: negative argument");
  if (!is_device_ptr(state_of) || !is_device_ptr(x) || !is_device_ptr(comps) || (dH && !is_device_ptr(dH)) ||
      (acc && !is_device_ptr(acc)) || (counters && !is_device_ptr(counters)))
    return fail(c, ALGDOCK_E_INVALID, "batch_hmc_cycle: arrays must be device pointers");
  Device g(c->device);
  cudaError_t e = launch_hmc_batch(c->stream, *c, state_of, x, comps, dH, acc, n_steps, seed, cycle, rep_offset,
                                   counters, -1);
  if (e != cudaSuccess) return cuda_fail(c, e, "batch_hmc_cycle");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_hmc_shape(algdock_ctx* c, int32_t* shape) {
  ALGDOCK_TRY(c)
  if (!shape) return fail(c, ALGDOCK_E_INVALID, "hmc_shape: null argument");
  if (!c->has_ligand) return fail(c, ALGDOCK_E_STATE, "hmc_shape: load a ligand first");
  const bool table = hmc_uses_table(c->lig);
  shape[0] = table ? 16 : 4;
  shape[1] = table ? 1 : 0;
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_batch_shapes(algdock_ctx* c, int32_t* shapes) {
  ALGDOCK_TRY(c)
  if (!shapes) return fail(c, ALGDOCK_E_INVALID, "batch_shapes: null argument");
  if (c->batch_n_rep == 0) return fail(c, ALGDOCK_E_STATE, "batch_shapes: set a batch layout first");
  for (int k = 0; k < kBatchClasses; ++k) {
    const BatchClass& B = c->batch_cls[k];
    shapes[2 * k] = B.n_items ? B.wpb : 0;
    shapes[2 * k + 1] = B.n_items && B.table ? 1 : 0;
  }
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_batch_tune(algdock_ctx* c, const int32_t* state_of, const float* x, int32_t n_steps,
                                  int32_t n_timed, int32_t* chosen, float* ms) {
  ALGDOCK_TRY(c)
  if (!c->has_grid || c->K == 0 || c->batch_n_rep == 0)
    return fail(c, ALGDOCK_E_STATE, "batch_tune: load grids, states, a batch and its layout first");
  if (n_steps < 0 || n_timed < 1 || !is_device_ptr(state_of) || !is_device_ptr(x))
    return fail(c, ALGDOCK_E_INVALID, "batch_tune: bad arguments");
  Device g(c->device);
  const int64_t R = c->batch_n_rep;
  const size_t xbytes = (size_t)R * c->batch_x_stride * 3 * sizeof(float);
  float* xs = nullptr;
  double* cs = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaMalloc(&xs, xbytes);
  if (e == cudaSuccess) e = cudaMalloc(&cs, (size_t)R * 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  // time of the whole batch launch (every class, overlapped as in production) with the current
  // shapes: the median of n_timed launches after one warm-up, each from the same copy of x
  auto whole = [&](float* out) {
    std::vector<float> t;
    for (int rep = 0; rep <= n_timed && e == cudaSuccess; ++rep) {
      e = cudaMemcpyAsync(xs, x, xbytes, cudaMemcpyDeviceToDevice, c->stream);
      if (e == cudaSuccess) e = cudaEventRecord(t0, c->stream);
      if (e == cudaSuccess)
        e = launch_hmc_batch(c->stream, *c, state_of, xs, cs, nullptr, nullptr, n_steps, 0x7E57u, rep, 0, nullptr, -1);
      if (e == cudaSuccess) e = cudaEventRecord(t1, c->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      float el = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&el, t0, t1);
      if (rep > 0) t.push_back(el);
    }
    std::sort(t.begin(), t.end());
    *out = t.empty() ? 0.f : t[t.size() / 2];
  };
  // coordinate descent: each class in turn takes the candidate that minimises the whole launch,
  // the others held at their current shapes; a candidate must beat the incumbent by 2 % (launch
  // times of equal shapes scatter by about that much)
  float best_ms = 0.f;
  whole(&best_ms);
  for (int k = 0; k < kBatchClasses && e == cudaSuccess; ++k) {
    BatchClass& B = c->batch_cls[k];
    if (B.n_items == 0) continue;
    int wpb[4];
    bool table[4];
    const int nc = batch_candidates(k, wpb, table);
    int best_w = B.wpb;
    bool best_t = B.table;
    for (int t = 0; t < nc && e == cudaSuccess; ++t) {
      if (wpb[t] == best_w && table[t] == best_t) continue;
      if (batch_class_smem(c, k, wpb[t], table[t]) > batch_smem_limit(kClassApl[k], wpb[t], table[t])) continue;
      e = batch_set_class(c, k, wpb[t], table[t]);
      if (e == cudaSuccess) e = batch_set_attributes(*c);
      float m = 0.f;
      if (e == cudaSuccess) whole(&m);
      if (e == cudaSuccess && m < 0.98f * best_ms) {
        best_ms = m;
        best_w = wpb[t];
        best_t = table[t];
      }
    }
    if (e == cudaSuccess) e = batch_set_class(c, k, best_w, best_t);
    if (e == cudaSuccess) e = batch_set_attributes(*c);
  }
  for (int k = 0; k < kBatchClasses && chosen; ++k) {
    const BatchClass& B = c->batch_cls[k];
    chosen[2 * k] = B.n_items ? B.wpb : 0;
    chosen[2 * k + 1] = B.n_items && B.table ? 1 : 0;
  }
  if (ms) *ms = best_ms;
  cudaFree(xs);
  cudaFree(cs);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (e != cudaSuccess) return cuda_fail(c, e, "batch_tune");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_energy_force(algdock_ctx* c, int64_t N, const int32_t* state_of, const float* x, float* force,
                                    double* comps) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_energy_force");
  if (!c->has_grid || !c->has_ligand || c->K == 0)
    return fail(c, ALGDOCK_E_STATE, "energy_force: load grids, ligand and states first");
  if (N < 0) return fail(c, ALGDOCK_E_INVALID, "energy_force: N < 0");
  if (N == 0) return ALGDOCK_OK;
  if (!is_device_ptr(state_of) || !is_device_ptr(x) || !is_device_ptr(force) || (comps && !is_device_ptr(comps)))
    return fail(c, ALGDOCK_E_INVALID, "energy_force: arrays must be device pointers");
  Device g(c->device);
  cudaError_t e = launch_energy_force(c->stream, *c, N, state_of, x, force, comps);
  if (e != cudaSuccess) return cuda_fail(c, e, "energy_force");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_exchange(algdock_ctx* c, int32_t n_ladders, int32_t K, int32_t state_offset,
                                const double* comps, int32_t* config_of, int32_t* state_of, int32_t n_sweeps,
                                int32_t max_sep, uint64_t seed, uint64_t cycle, int64_t ladder_offset,
                                int64_t* attempts, int64_t* accepts) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_exchange");
  if (c->K == 0) return fail(c, ALGDOCK_E_STATE, "exchange: set states first");
  if (n_ladders < 0 || K < 1 || K > kMaxLadder || state_offset < 0 || state_offset + K > c->K || n_sweeps < 0 ||
      max_sep < 1 || (int64_t)n_sweeps * max_sep >= 65536 || ladder_offset < 0)
    return fail(c, ALGDOCK_E_INVALID, "exchange: bad sizes");
  if (n_ladders == 0) return ALGDOCK_OK;
  if (!is_device_ptr(comps) || !is_device_ptr(config_of) || (state_of && !is_device_ptr(state_of)) ||
      (attempts && !is_device_ptr(attempts)) ||
      (accepts && !is_device_ptr(accepts)))
    return fail(c, ALGDOCK_E_INVALID, "exchange: arrays must be device pointers");
  Device g(c->device);
  cudaError_t e = launch_exchange(c->stream, *c, n_ladders, K, state_offset, comps, config_of, state_of, n_sweeps,
                                  max_sep, seed, cycle, ladder_offset, attempts, accepts);
  if (e != cudaSuccess) return cuda_fail(c, e, "exchange");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_reduced_energies(algdock_ctx* c, int64_t N, const float* x, double* comps, int32_t k_begin,
                                        int32_t k_count, double* u_kn) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_reduced_energies");
  if (N < 0) return fail(c, ALGDOCK_E_INVALID, "reduced_energies: N < 0");
  if (N == 0) return ALGDOCK_OK;
  if (!x && !comps) return fail(c, ALGDOCK_E_INVALID, "reduced_energies: need x or comps");
  if (u_kn && (k_begin < 0 || k_count < 0 || k_begin + k_count > c->K))
    return fail(c, ALGDOCK_E_INVALID, "reduced_energies: state range outside the state table");
  if (x && (!c->has_grid || !c->has_ligand)) return fail(c, ALGDOCK_E_STATE, "reduced_energies: load grids and ligand");
  if ((x && !is_device_ptr(x)) || (comps && !is_device_ptr(comps)) || (u_kn && !is_device_ptr(u_kn)))
    return fail(c, ALGDOCK_E_INVALID, "reduced_energies: arrays must be device pointers");
  Device g(c->device);
  cudaError_t e = cudaSuccess;
  double* tmp = nullptr;
  double* cp = comps;
  if (x) {
    if (!cp) {
      e = cudaMallocAsync(&tmp, (size_t)N * 4 * sizeof(double), c->stream);
      cp = tmp;
    }
    if (e == cudaSuccess) e = launch_evaluate(c->stream, *c, N, x, cp);
  }
  if (e == cudaSuccess && u_kn) e = launch_ukn(c->stream, *c, N, cp, k_begin, k_count, u_kn);
  if (tmp) cudaFreeAsync(tmp, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "reduced_energies");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

// ------------------------------------------------------------------ learned proposal
static algdock_status learn_scratch(algdock_ctx* c, size_t need, const char* where) {
  if (need <= c->learn_bytes) return ALGDOCK_OK;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  cudaFree(c->d_learn);
  c->d_learn = nullptr;
  c->learn_bytes = 0;
  e = cudaMalloc(&c->d_learn, need);
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  c->learn_bytes = need;
  return ALGDOCK_OK;
}

algdock_status algdock_learned_ntorsions(algdock_ctx* c, int32_t* T) {
  ALGDOCK_TRY(c)
  if (!T) return fail(c, ALGDOCK_E_INVALID, "learned_ntorsions: null argument");
  if (!c->has_ligand) return fail(c, ALGDOCK_E_STATE, "learned_ntorsions: load the ligand first");
  *T = c->ltopo.T;
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_learned_features(algdock_ctx* c, int64_t N, const int32_t* state_of, const float* x,
                                        const double* comps, float* feat) {
  ALGDOCK_TRY(c)
  if (!c->has_ligand || c->K == 0) return fail(c, ALGDOCK_E_STATE, "learned_features: load ligand and states first");
  if (N < 0) return fail(c, ALGDOCK_E_INVALID, "learned_features: N < 0");
  if (N == 0) return ALGDOCK_OK;
  if (!is_device_ptr(state_of) || !is_device_ptr(x) || !is_device_ptr(comps) || !is_device_ptr(feat))
    return fail(c, ALGDOCK_E_INVALID, "learned_features: arrays must be device pointers");
  Device g(c->device);
  cudaError_t e = learned_features(c->stream, *c, N, state_of, x, comps, feat);
  if (e != cudaSuccess) return cuda_fail(c, e, "learned_features");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_pose_delta(algdock_ctx* c, int64_t N, const float* x, const float* y, float* delta) {
  ALGDOCK_TRY(c)
  if (!c->has_ligand) return fail(c, ALGDOCK_E_STATE, "pose_delta: load the ligand first");
  if (N < 0) return fail(c, ALGDOCK_E_INVALID, "pose_delta: N < 0");
  if (N == 0) return ALGDOCK_OK;
  if (!is_device_ptr(x) || !is_device_ptr(y) || !is_device_ptr(delta))
    return fail(c, ALGDOCK_E_INVALID, "pose_delta: arrays must be device pointers");
  Device g(c->device);
  cudaError_t e = learned_pose_delta(c->stream, *c, N, x, y, delta);
  if (e != cudaSuccess) return cuda_fail(c, e, "pose_delta");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_mlp_forward(algdock_ctx* c, const float* params, const uint16_t* wbf16, int64_t N,
                                   const float* feat, float* out) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_mlp_forward");
  if (N < 0 || N > (int64_t)1 << 30) return fail(c, ALGDOCK_E_INVALID, "mlp_forward: bad N");
  if (N == 0) return ALGDOCK_OK;
  if (!is_device_ptr(params) || !is_device_ptr(wbf16) || !is_device_ptr(feat) || !is_device_ptr(out))
    return fail(c, ALGDOCK_E_INVALID, "mlp_forward: arrays must be device pointers");
  Device g(c->device);
  algdock_status st = learn_scratch(c, learned_forward_scratch(N), "mlp_forward");
  if (st != ALGDOCK_OK) return st;
  const bool tc = N >= kTcMinRowsForward;
  cudaError_t e = tc ? cudaMemsetAsync(tc_err_word(c), 0, sizeof(int), c->stream) : cudaSuccess;
  if (e == cudaSuccess) e = learned_forward(c->stream, params, wbf16, N, feat, out, c->d_learn, tc_err_word(c));
  if (e != cudaSuccess) return cuda_fail(c, e, "mlp_forward");
  return tc ? tc_check(c, "mlp_forward") : ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_mlp_grad(algdock_ctx* c, const float* params, const uint16_t* wbf16, int64_t N, const float* feat,
                                const float* delta, int32_t D, float* grad, float* loss) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_mlp_grad");
  if (N < 1 || N > (int64_t)1 << 30 || D < 1 || D > ALGDOCK_MLP_DMAX)
    return fail(c, ALGDOCK_E_INVALID, "mlp_grad: bad N or D");
  if (!is_device_ptr(params) || !is_device_ptr(wbf16) || !is_device_ptr(feat) || !is_device_ptr(delta) ||
      !is_device_ptr(grad) || (loss && !is_device_ptr(loss)))
    return fail(c, ALGDOCK_E_INVALID, "mlp_grad: arrays must be device pointers");
  Device g(c->device);
  algdock_status st = learn_scratch(c, learned_grad_scratch(N), "mlp_grad");
  if (st != ALGDOCK_OK) return st;
  const bool tc = N >= kTcMinRowsGrad;
  cudaError_t e = tc ? cudaMemsetAsync(tc_err_word(c), 0, sizeof(int), c->stream) : cudaSuccess;
  if (e == cudaSuccess)
    e = learned_grad(c->stream, params, wbf16, N, feat, delta, D, grad, loss, c->d_learn, tc_err_word(c));
  if (e != cudaSuccess) return cuda_fail(c, e, "mlp_grad");
  return tc ? tc_check(c, "mlp_grad") : ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_mlp_adam(algdock_ctx* c, float* params, uint16_t* wbf16, const float* grad, float* m, float* v,
                                int32_t step, float lr) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_mlp_adam");
  if (step < 1 || !(lr >= 0.f)) return fail(c, ALGDOCK_E_INVALID, "mlp_adam: step >= 1 and lr >= 0");
  if (!is_device_ptr(params) || !is_device_ptr(wbf16) || !is_device_ptr(grad) || !is_device_ptr(m) ||
      !is_device_ptr(v))
    return fail(c, ALGDOCK_E_INVALID, "mlp_adam: arrays must be device pointers");
  Device g(c->device);
  cudaError_t e = learned_adam(c->stream, params, wbf16, grad, m, v, step, lr);
  if (e != cudaSuccess) return cuda_fail(c, e, "mlp_adam");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_propose_learned(algdock_ctx* c, const float* params, const uint16_t* wbf16, int64_t n_rep,
                                       const int32_t* state_of, float* x, double* comps, int32_t n_moves,
                                       int32_t n_torsions, uint64_t seed, uint64_t cycle, int64_t rep_offset,
                                       int32_t* accepted, int64_t* counters) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_propose_learned");
  if (!c->has_grid || !c->has_ligand || c->K == 0)
    return fail(c, ALGDOCK_E_STATE, "propose_learned: load grids, ligand and states first");
  if (n_rep < 0 || n_rep > (int64_t)1 << 30 || n_moves < 0 || rep_offset < 0)
    return fail(c, ALGDOCK_E_INVALID, "propose_learned: bad sizes");
  if (n_rep == 0 || n_moves == 0) return ALGDOCK_OK;
  if (!is_device_ptr(params) || !is_device_ptr(wbf16) || !is_device_ptr(state_of) || !is_device_ptr(x) ||
      !is_device_ptr(comps) || (accepted && !is_device_ptr(accepted)) || (counters && !is_device_ptr(counters)))
    return fail(c, ALGDOCK_E_INVALID, "propose_learned: arrays must be device pointers");
  Device g(c->device);
  algdock_status st = learn_scratch(c, learned_propose_scratch(n_rep, c->lig.na), "propose_learned");
  if (st != ALGDOCK_OK) return st;
  const int t_eff = (n_torsions < 0 || n_torsions > c->ltopo.T) ? c->ltopo.T : n_torsions;
  cudaError_t e = learned_propose(c->stream, *c, params, wbf16, n_rep, state_of, x, comps, n_moves, t_eff, seed,
                                  cycle, rep_offset, accepted, counters, c->d_learn);
  if (e != cudaSuccess) return cuda_fail(c, e, "propose_learned");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_mbar(algdock_ctx* c, int32_t K, int64_t N, const double* u_kn, const int64_t* N_k, double tol,
                            int32_t max_iter, int32_t precision_mode, double* f_k, int32_t* iters) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_mbar");
  if (tol == 0.0) tol = c->params.mbar_tol;
  if (max_iter == 0) max_iter = c->params.mbar_max_iter;
  if (precision_mode == -1) precision_mode = c->params.mbar_precision;
  if (K < 1 || N < 1 || !u_kn || !N_k || !f_k || !iters || max_iter < 1 || !(tol > 0) ||
      precision_mode < 0 || precision_mode > 2)
    return fail(c, ALGDOCK_E_INVALID, "mbar: bad arguments");
  if (precision_mode == 2 && K > 16384) return fail(c, ALGDOCK_E_INVALID, "mbar: precision mode 2 takes K <= 16384");
  if (K > kMbarMaxStates)
    return fail(c, ALGDOCK_E_INVALID, "mbar: K = " + std::to_string(K) + " exceeds the " +
                                          std::to_string(kMbarMaxStates) + " states one launch grid dimension can hold");
  if (!is_device_ptr(u_kn)) return fail(c, ALGDOCK_E_INVALID, "mbar: u_kn must be a device pointer");
  int64_t total = 0;
  for (int k = 0; k < K; ++k) {
    if (N_k[k] < 0) return fail(c, ALGDOCK_E_INVALID, "mbar: negative N_k");
    total += N_k[k];
  }
  if (total != N) return fail(c, ALGDOCK_E_INVALID, "mbar: sum of N_k must equal N");
  Device g(c->device);
  const size_t need = mbar_scratch_bytes_mode(K, N, precision_mode);
  if (need > c->mbar_bytes) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "mbar");
    cudaFree(c->d_mbar);
    c->d_mbar = nullptr;
    c->mbar_bytes = 0;
    e = cudaMalloc(&c->d_mbar, need);
    if (e != cudaSuccess) return cuda_fail(c, e, "mbar");
    c->mbar_bytes = need;
  }
  cudaError_t err = cudaSuccess;
  int it = 0;
  const int r = mbar_run(c->stream, c->d_mbar, K, N, u_kn, N_k, tol, max_iter, precision_mode, f_k, &it, c->h_flag,
                         &err);
  *iters = it;
  if (r < 0) return cuda_fail(c, err, "mbar");
  if (r == 1) return fail(c, ALGDOCK_E_NOT_CONVERGED, "mbar: max_iter reached");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_cycle(algdock_ctx* c, const algdock_run_desc* d, uint64_t cycle, float* x, double* comps,
                             int32_t* state_of, int32_t* config_of, int64_t* counters, double* u_kn) {
  ALGDOCK_TRY(c)
  if (!c->has_grid || !c->has_ligand || c->K == 0)
    return fail(c, ALGDOCK_E_STATE, "cycle: load grids, ligand and states first");
  if (!d || !x || !comps || !state_of || !config_of || d->n_legs < 1 || d->n_legs > ALGDOCK_MAX_LEGS ||
      d->n_chains < 1 || d->n_steps < 0 || d->n_sweeps < 0 || d->max_sep < 1 ||
      (int64_t)d->n_sweeps * d->max_sep >= 65536 || d->rep_offset < 0 || d->ladder_offset < 0 ||
      d->n_external < 0 || (d->n_external > 0 && (isnan(d->alpha_max) || !(d->sigma_ext >= 0.0) ||
                                                    !isfinite(d->sigma_ext))))
    return fail(c, ALGDOCK_E_INVALID, "cycle: bad arguments");
  NvtxRange range("algdock_cycle");
  int64_t R = 0, ukn_words = 0;
  for (int l = 0; l < d->n_legs; ++l) {
    if (d->K[l] < 1 || d->K[l] > kMaxLadder || d->state_offset[l] < 0 || d->state_offset[l] + d->K[l] > c->K)
      return fail(c, ALGDOCK_E_INVALID, "cycle: leg outside the state table");
    R += (int64_t)d->n_chains * d->K[l];
    ukn_words += (int64_t)d->K[l] * d->n_chains * d->K[l];
  }
  const int na = c->lig.na;
  // each array device-resident as given; or, for the positions, components, permutations and u_kn
  // in pinned host memory on a device with a coherent host link, read and written in place by the
  // kernels (plain loads and stores only; the counters take atomics); or else staged: [x | comps |
  // state_of | config_of | counters | u_kn], 256-byte aligned pieces
  struct Piece {
    void* user;
    size_t bytes;
    bool host;
    size_t off;
    void* mapped;
  };
  constexpr int kPieces = 6;
  Piece P[kPieces] = {{x, (size_t)R * na * 3 * 4, false, 0, nullptr},
                      {comps, (size_t)R * 32, false, 0, nullptr},
                      {state_of, (size_t)R * 4, false, 0, nullptr},
                      {config_of, (size_t)R * 4, false, 0, nullptr},
                      {counters, counters ? (size_t)ALGDOCK_N_COUNTERS * 8 : 0, false, 0, nullptr},
                      {u_kn, u_kn ? (size_t)ukn_words * 8 : 0, false, 0, nullptr}};
  size_t need = 0;
  bool any_mapped = false;
  for (int i = 0; i < kPieces; ++i) {
    if (!P[i].user) continue;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, P[i].user) != cudaSuccess) {
      cudaGetLastError();
      a.type = cudaMemoryTypeUnregistered;
      a.devicePointer = nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) continue;
    if (i != 4 && c->host_coherent && a.type == cudaMemoryTypeHost && a.devicePointer) {
      P[i].mapped = a.devicePointer;
      any_mapped = true;
      continue;
    }
    P[i].host = true;
    P[i].off = need;
    need += (P[i].bytes + 255) & ~(size_t)255;
  }
  Device g(c->device);
  cudaError_t e = cudaSuccess;
  if (need > c->stage_bytes) {
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cycle");
    cudaFree(c->d_stage);
    c->d_stage = nullptr;
    c->stage_bytes = 0;
    e = cudaMalloc(&c->d_stage, need);
    if (e != cudaSuccess) return cuda_fail(c, e, "cycle");
    c->stage_bytes = need;
  }
  auto dev_of = [&](int i) {
    return P[i].mapped ? P[i].mapped : (P[i].host ? (void*)((char*)c->d_stage + P[i].off) : P[i].user);
  };
  bool any_host = false;
  for (int i = 0; i < kPieces && e == cudaSuccess; ++i)
    if (P[i].host && P[i].user) {  // inputs in (u_kn is output only; its host copy goes out below)
      any_host = true;
      if (i != 5) e = cudaMemcpyAsync(dev_of(i), P[i].user, P[i].bytes, cudaMemcpyHostToDevice, c->stream);
    }
  float* dx = (float*)dev_of(0);
  double* dc = (double*)dev_of(1);
  int32_t* ds = (int32_t*)dev_of(2);
  int32_t* dcfg = (int32_t*)dev_of(3);
  int64_t* dcnt = (int64_t*)dev_of(4);
  if (e == cudaSuccess) {
    NvtxRange r("algdock_cycle: HMC trial");
    e = launch_hmc(c->stream, *c, R, ds, dx, dc, nullptr, nullptr, d->n_steps, d->seed, cycle, d->rep_offset, dcnt);
  }
  if (e == cudaSuccess && d->n_external > 0) {
    NvtxRange r("algdock_cycle: external moves");
    e = launch_external(c->stream, *c, R, ds, dx, dc, d->n_external, d->alpha_max, (float)d->sigma_ext, d->seed,
                        cycle, d->rep_offset, nullptr, dcnt);
  }
  // the snapshot reads only the components of the configurations, which the exchange does not
  // move, so it runs on a side stream beside the exchange sweeps
  // the positions and components are final once the trial and the moves are done (the exchange
  // permutes states, not configurations): host copies of them go back on the side stream too,
  // beside the sweeps
  const bool early_out = P[0].host || P[1].host;
  const bool side = u_kn || early_out;
  cudaStream_t snap_s = c->stream;
  if (e == cudaSuccess && side) {
    if (!c->cycle_side) e = cudaStreamCreateWithFlags(&c->cycle_side, cudaStreamNonBlocking);
    if (e == cudaSuccess && !c->cycle_fork) e = cudaEventCreateWithFlags(&c->cycle_fork, cudaEventDisableTiming);
    if (e == cudaSuccess && !c->cycle_join) e = cudaEventCreateWithFlags(&c->cycle_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(c->cycle_fork, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->cycle_side, c->cycle_fork, 0);
    if (e == cudaSuccess) snap_s = c->cycle_side;
  }
  int64_t base = 0, cbase = 0, ubase = 0;
  if (e == cudaSuccess && u_kn) {
    // the snapshot: u_kn per leg from the components of every configuration, which the trial's
    // final energy evaluation (and the external moves) left in comps; U_k is linear in them, so
    // no configuration is evaluated a second time
    NvtxRange r("algdock_cycle: snapshot");
    for (int l = 0; l < d->n_legs && e == cudaSuccess; ++l) {
      const int64_t n = (int64_t)d->n_chains * d->K[l];
      e = launch_ukn(snap_s, *c, n, dc + 4 * base, d->state_offset[l], d->K[l], (double*)dev_of(5) + ubase);
      base += n;
      ubase += (int64_t)d->K[l] * n;
    }
  }
  for (int i = 0; i < 2 && e == cudaSuccess && side; ++i)
    if (P[i].host && P[i].user) e = cudaMemcpyAsync(P[i].user, dev_of(i), P[i].bytes, cudaMemcpyDeviceToHost, snap_s);
  if (e == cudaSuccess && side) e = cudaEventRecord(c->cycle_join, snap_s);
  base = 0;
  NvtxRange rx("algdock_cycle: exchange");
  for (int l = 0; l < d->n_legs && e == cudaSuccess; ++l) {
    e = launch_exchange(c->stream, *c, d->n_chains, d->K[l], d->state_offset[l], dc + 4 * base, dcfg + cbase,
                        ds + base, d->n_sweeps, d->max_sep, d->seed, cycle, d->ladder_offset + (int64_t)l * d->n_chains,
                        nullptr, nullptr);
    base += (int64_t)d->n_chains * d->K[l];
    cbase += (int64_t)d->n_chains * d->K[l];
  }
  if (e == cudaSuccess && side) e = cudaStreamWaitEvent(c->stream, c->cycle_join, 0);
  const bool checks = c->params.checks != 0;
  if (e == cudaSuccess && checks) {
    e = launch_run_check(c->stream, *c, *d, dx, dc, ds, dcfg, check_word(c));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->h_flag, check_word(c), sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  }
  for (int i = side ? 2 : 0; i < kPieces && e == cudaSuccess; ++i)
    if (P[i].host && P[i].user) e = cudaMemcpyAsync(P[i].user, dev_of(i), P[i].bytes, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && (any_host || any_mapped || checks)) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cycle");
  if (checks) return check_status(c, *c->h_flag, "cycle");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_gemm_bf16(algdock_ctx* c, int32_t M, int32_t N, int32_t K, const uint16_t* A, int32_t lda,
                                 const uint16_t* B, int32_t ldb, void* C, int32_t ldc, int32_t epilogue,
                                 const float* bias, const uint16_t* mask, int32_t ldm, int32_t n_split) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_gemm_bf16");
  if (M < 0 || N < 0 || K < 1 || lda < K || ldb < K || lda % 8 || ldb % 8 || epilogue < 0 || epilogue > 3 ||
      ldc < N || n_split < 1 || ((epilogue == 1 || epilogue == 2) && !bias) || (epilogue == 3 && (!mask || ldm < N)) ||
      (n_split > 1 && epilogue != 0))
    return fail(c, ALGDOCK_E_INVALID, "gemm_bf16: bad arguments");
  if (M == 0 || N == 0) return ALGDOCK_OK;
  if (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(C) || (bias && !is_device_ptr(bias)) ||
      (mask && !is_device_ptr(mask)))
    return fail(c, ALGDOCK_E_INVALID, "gemm_bf16: arrays must be device pointers");
  if ((((uintptr_t)A) | ((uintptr_t)B)) & 15) return fail(c, ALGDOCK_E_INVALID, "gemm_bf16: A and B 16-byte aligned");
  Device g(c->device);
  if (!umma_supported(c->device)) return fail(c, ALGDOCK_E_INVALID, "gemm_bf16: needs an sm_100-class device");
  cudaError_t e = cudaMemsetAsync(tc_err_word(c), 0, sizeof(int), c->stream);
  if (e == cudaSuccess)
    e = umma_gemm(c->stream, M, N, K, A, lda, B, ldb, C, ldc, epilogue, bias, mask, ldm, n_split, tc_err_word(c));
  if (e != cudaSuccess) return cuda_fail(c, e, "gemm_bf16");
  return tc_check(c, "gemm_bf16");
  ALGDOCK_CATCH(c)
}

algdock_status algdock_mbar_partials(algdock_ctx* c, int32_t K, int64_t N, const double* u_kn, const int64_t* N_k,
                                     const double* f, int32_t precision_mode, double* pairs) {
  ALGDOCK_TRY(c)
  NvtxRange range("algdock_mbar_partials");
  if (K < 1 || N < 0 || !N_k || !f || !pairs || (N > 0 && !u_kn) || (precision_mode != 0 && precision_mode != 1))
    return fail(c, ALGDOCK_E_INVALID, "mbar_partials: bad arguments (precision_mode 0 or 1)");
  if (K > kMbarMaxStates)
    return fail(c, ALGDOCK_E_INVALID, "mbar_partials: K = " + std::to_string(K) + " exceeds " +
                                          std::to_string(kMbarMaxStates));
  for (int k = 0; k < K; ++k) {
    if (N_k[k] < 0) return fail(c, ALGDOCK_E_INVALID, "mbar_partials: negative N_k");
    if (!isfinite(f[k])) return fail(c, ALGDOCK_E_NUMERIC, "mbar_partials: non-finite f");
  }
  if (N == 0) {  // no samples here: the empty pair of every state
    for (int k = 0; k < K; ++k) {
      pairs[2 * k] = -INFINITY;
      pairs[2 * k + 1] = 0.0;
    }
    return ALGDOCK_OK;
  }
  if (!is_device_ptr(u_kn)) return fail(c, ALGDOCK_E_INVALID, "mbar_partials: u_kn must be a device pointer");
  Device g(c->device);
  const size_t need = mbar_pairs_scratch_bytes(K, N);
  if (need > c->mbar_bytes) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "mbar_partials");
    cudaFree(c->d_mbar);
    c->d_mbar = nullptr;
    c->mbar_bytes = 0;
    e = cudaMalloc(&c->d_mbar, need);
    if (e != cudaSuccess) return cuda_fail(c, e, "mbar_partials");
    c->mbar_bytes = need;
  }
  const cudaError_t e = mbar_local_pairs(c->stream, c->d_mbar, K, N, u_kn, N_k, f, precision_mode, pairs);
  if (e != cudaSuccess) return cuda_fail(c, e, "mbar_partials");
  return ALGDOCK_OK;
  ALGDOCK_CATCH(c)
}

algdock_status algdock_mbar_update(int32_t K, int32_t n_parts, const double* pairs, const double* f_old,
                                   double* f_new, double* delta) {
  if (K < 1 || n_parts < 1 || !pairs || !f_old || !f_new || !delta) return ALGDOCK_E_INVALID;
  std::vector<double> fn(K);
  for (int i = 0; i < K; ++i) {
    double M = -INFINITY;
    for (int p = 0; p < n_parts; ++p) M = std::max(M, pairs[((size_t)p * K + i) * 2]);
    double S = 0.0;
    if (M != -INFINITY)
      for (int p = 0; p < n_parts; ++p) {
        const double m = pairs[((size_t)p * K + i) * 2], sp = pairs[((size_t)p * K + i) * 2 + 1];
        if (m != -INFINITY) S += sp * exp(m - M);
      }
    fn[i] = M == -INFINITY ? INFINITY : -(M + log(S));
  }
  double d = 0.0;
  const double f0 = fn[0];
  for (int i = 0; i < K; ++i) {
    const double v = fn[i] - f0;
    const double di = fabs(v - f_old[i]);
    d = (di > d || isnan(di)) ? di : d;
    f_new[i] = v;
  }
  *delta = d;
  return ALGDOCK_OK;
}

}  // extern "C"
