// Checkpoint and resume of a sampling run.  The paper's protocol stores each stage's data between
// cycles so that a calculation interrupted on a shared or opportunistic machine restarts where it
// stopped ("Stages"; "Equilibration and production").  A checkpoint here holds what a run needs
// to continue bit for bit: the context's state table (T, alpha and each state's time step), the
// run's seed and next cycle, a fingerprint of the loaded ligand and lattice, and any number of
// named arrays of the caller (positions, components, permutations, counters, stored components).
//
// File layout, little-endian throughout (both supported hosts, x86-64 and AArch64, are):
//   "ALGDCKPT" | u32 version (1) | u32 K | u64 seed | u64 cycle | u32 ligand CRC | u32 lattice CRC |
//   u32 n_arrays | f64 T[K] | f64 alpha[K] | f64 dt[K] |
//   n_arrays x { char name[32] | u32 dtype | u32 element bytes | u64 count | data } |
//   u32 CRC-32 of every preceding byte.
#include <stdio.h>
#include <string.h>
#include <unistd.h>

#include <array>
#include <string>
#include <vector>

#include "internal.cuh"

namespace algdock {

// CRC-32, reflected polynomial 0xEDB88320 (bit-reversed 0x04C11DB7), initial value and final XOR
// 0xFFFFFFFF: the checksum of zip, gzip and PNG.  Table-driven, one byte at a time.
uint32_t crc32_update(uint32_t crc, const void* data, size_t n) {
  static const std::array<uint32_t, 256> table = [] {
    std::array<uint32_t, 256> t{};
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t r = i;
      for (int k = 0; k < 8; ++k) r = (r & 1u) ? (r >> 1) ^ 0xEDB88320u : r >> 1;
      t[i] = r;
    }
    return t;
  }();
  const uint8_t* p = (const uint8_t*)data;
  uint32_t c = ~crc;
  for (size_t i = 0; i < n; ++i) c = table[(c ^ p[i]) & 0xffu] ^ (c >> 8);
  return ~c;
}

}  // namespace algdock

using namespace algdock;

namespace {

constexpr char kMagic[8] = {'A', 'L', 'G', 'D', 'C', 'K', 'P', 'T'};
constexpr uint32_t kVersion = 1;
constexpr size_t kNameBytes = 32;

algdock_status ck_fail(algdock_ctx* c, algdock_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

size_t dtype_bytes(int32_t t) {
  switch (t) {
    case ALGDOCK_F32:
    case ALGDOCK_I32:
      return 4;
    case ALGDOCK_F64:
    case ALGDOCK_I64:
      return 8;
    case ALGDOCK_U8:
      return 1;
    default:
      return 0;
  }
}

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void put(std::vector<uint8_t>& b, const void* p, size_t n) {
  const uint8_t* q = (const uint8_t*)p;
  b.insert(b.end(), q, q + n);
}
template <typename T>
void put_v(std::vector<uint8_t>& b, T v) {
  put(b, &v, sizeof(T));
}

// A checkpoint read into memory and checked: magic, version, sizes and the CRC trailer.
struct Parsed {
  uint32_t K = 0, fp_ligand = 0, fp_grid = 0;
  uint64_t seed = 0, cycle = 0;
  std::vector<double> T, alpha, dt;
  struct Arr {
    std::string name;
    uint32_t dtype = 0, esize = 0;
    uint64_t count = 0;
    size_t offset = 0;  // of the data within the file image
  };
  std::vector<Arr> arrays;
  std::vector<uint8_t> image;
};

algdock_status parse(algdock_ctx* c, const char* path, Parsed& P) {
  FILE* f = fopen(path, "rb");
  if (!f) return ck_fail(c, ALGDOCK_E_INVALID, std::string("checkpoint: cannot open ") + path);
  std::vector<uint8_t>& b = P.image;
  uint8_t buf[1 << 16];
  size_t got;
  while ((got = fread(buf, 1, sizeof(buf), f)) > 0) b.insert(b.end(), buf, buf + got);
  const bool read_err = ferror(f) != 0;
  fclose(f);
  if (read_err) return ck_fail(c, ALGDOCK_E_INVALID, "checkpoint: read error");
  const size_t head = 8 + 4 + 4 + 8 + 8 + 4 + 4 + 4;
  if (b.size() < head + 4) return ck_fail(c, ALGDOCK_E_INVALID, "checkpoint: truncated (shorter than its header)");
  uint32_t stored;
  memcpy(&stored, b.data() + b.size() - 4, 4);
  if (crc32_update(0, b.data(), b.size() - 4) != stored)
    return ck_fail(c, ALGDOCK_E_INVALID, "checkpoint: CRC mismatch (corrupt or truncated file)");
  if (memcmp(b.data(), kMagic, 8) != 0) return ck_fail(c, ALGDOCK_E_INVALID, "checkpoint: not a checkpoint file");
  size_t o = 8;
  auto get = [&](void* dst, size_t n) {
    if (o + n > b.size() - 4) return false;
    memcpy(dst, b.data() + o, n);
    o += n;
    return true;
  };
  uint32_t version = 0, n_arr = 0;
  get(&version, 4);
  if (version != kVersion) return ck_fail(c, ALGDOCK_E_INVALID, "checkpoint: unsupported version");
  get(&P.K, 4);
  get(&P.seed, 8);
  get(&P.cycle, 8);
  get(&P.fp_ligand, 4);
  get(&P.fp_grid, 4);
  get(&n_arr, 4);
  if ((uint64_t)P.K * 24 > b.size()) return ck_fail(c, ALGDOCK_E_INVALID, "checkpoint: bad state count");
  P.T.resize(P.K);
  P.alpha.resize(P.K);
  P.dt.resize(P.K);
  if (!get(P.T.data(), 8 * (size_t)P.K) || !get(P.alpha.data(), 8 * (size_t)P.K) ||
      !get(P.dt.data(), 8 * (size_t)P.K))
    return ck_fail(c, ALGDOCK_E_INVALID, "checkpoint: truncated state table");
  for (uint32_t a = 0; a < n_arr; ++a) {
    Parsed::Arr A;
    char name[kNameBytes];
    if (!get(name, kNameBytes) || !get(&A.dtype, 4) || !get(&A.esize, 4) || !get(&A.count, 8))
      return ck_fail(c, ALGDOCK_E_INVALID, "checkpoint: truncated array header");
    if (name[kNameBytes - 1] != 0 || dtype_bytes((int32_t)A.dtype) != A.esize || A.esize == 0)
      return ck_fail(c, ALGDOCK_E_INVALID, "checkpoint: bad array header");
    A.name = name;
    if (A.count > (b.size() - 4 - o) / A.esize) return ck_fail(c, ALGDOCK_E_INVALID, "checkpoint: truncated array");
    A.offset = o;
    o += (size_t)A.count * A.esize;
    P.arrays.push_back(A);
  }
  if (o != b.size() - 4) return ck_fail(c, ALGDOCK_E_INVALID, "checkpoint: trailing bytes");
  return ALGDOCK_OK;
}

}  // namespace

extern "C" {

algdock_status algdock_checkpoint_save(algdock_ctx* c, const char* path, uint64_t seed, uint64_t cycle,
                                       int32_t n_arrays, const algdock_array* arrays) {
  try {
    if (!path || n_arrays < 0 || (n_arrays > 0 && !arrays))
      return ck_fail(c, ALGDOCK_E_INVALID, "checkpoint_save: bad arguments");
    std::vector<uint8_t> b;
    put(b, kMagic, 8);
    put_v<uint32_t>(b, kVersion);
    const uint32_t K = c ? (uint32_t)c->K : 0u;
    put_v<uint32_t>(b, K);
    put_v<uint64_t>(b, seed);
    put_v<uint64_t>(b, cycle);
    put_v<uint32_t>(b, c && c->has_ligand ? c->fp_ligand : 0u);
    put_v<uint32_t>(b, c && c->has_grid ? c->fp_grid : 0u);
    put_v<uint32_t>(b, (uint32_t)n_arrays);
    if (K) {
      put(b, c->h_T.data(), 8 * (size_t)K);
      put(b, c->h_alpha.data(), 8 * (size_t)K);
      put(b, c->h_dt.data(), 8 * (size_t)K);
    }
    if (c) {
      cudaError_t e = cudaStreamSynchronize(c->stream);  // the arrays' producers have finished
      if (e != cudaSuccess) return ck_fail(c, ALGDOCK_E_CUDA, std::string("checkpoint_save: ") + cudaGetErrorString(e));
    }
    for (int32_t a = 0; a < n_arrays; ++a) {
      const algdock_array& A = arrays[a];
      const size_t es = dtype_bytes(A.dtype);
      const size_t nl = strnlen(A.name, kNameBytes);
      if (es == 0 || A.count < 0 || nl == 0 || nl >= kNameBytes || (A.count > 0 && !A.data))
        return ck_fail(c, ALGDOCK_E_INVALID, "checkpoint_save: bad array " + std::to_string(a));
      for (int32_t q = 0; q < a; ++q)
        if (strncmp(arrays[q].name, A.name, kNameBytes) == 0)
          return ck_fail(c, ALGDOCK_E_INVALID, std::string("checkpoint_save: duplicate array name ") + A.name);
      char name[kNameBytes] = {0};
      memcpy(name, A.name, nl);
      put(b, name, kNameBytes);
      put_v<uint32_t>(b, (uint32_t)A.dtype);
      put_v<uint32_t>(b, (uint32_t)es);
      put_v<uint64_t>(b, (uint64_t)A.count);
      const size_t bytes = es * (size_t)A.count;
      const size_t at = b.size();
      b.resize(at + bytes);
      if (bytes == 0) continue;
      if (on_device(A.data)) {
        cudaError_t e = cudaMemcpy(b.data() + at, A.data, bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
          return ck_fail(c, ALGDOCK_E_CUDA, std::string("checkpoint_save: ") + cudaGetErrorString(e));
      } else {
        memcpy(b.data() + at, A.data, bytes);
      }
    }
    put_v<uint32_t>(b, crc32_update(0, b.data(), b.size()));
    // write a temporary file beside the target, then rename it over the target
    const std::string tmp = std::string(path) + ".tmp" + std::to_string((long)getpid());
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return ck_fail(c, ALGDOCK_E_INVALID, std::string("checkpoint_save: cannot write ") + tmp);
    const bool ok = fwrite(b.data(), 1, b.size(), f) == b.size();
    const bool closed = fclose(f) == 0;
    if (!ok || !closed || rename(tmp.c_str(), path) != 0) {
      remove(tmp.c_str());
      return ck_fail(c, ALGDOCK_E_INVALID, std::string("checkpoint_save: cannot write ") + path);
    }
    return ALGDOCK_OK;
  } catch (...) {
    return ck_fail(c, ALGDOCK_E_OOM, "checkpoint_save: host allocation failed");
  }
}

algdock_status algdock_checkpoint_load(algdock_ctx* c, const char* path, uint64_t* seed, uint64_t* cycle,
                                       int32_t n_arrays, algdock_array* arrays) {
  try {
    if (!path || n_arrays < 0 || (n_arrays > 0 && !arrays))
      return ck_fail(c, ALGDOCK_E_INVALID, "checkpoint_load: bad arguments");
    Parsed P;
    algdock_status st = parse(c, path, P);
    if (st != ALGDOCK_OK) return st;
    if (c) {
      if (P.fp_ligand && c->has_ligand && P.fp_ligand != c->fp_ligand)
        return ck_fail(c, ALGDOCK_E_STATE, "checkpoint_load: the context's ligand differs from the checkpoint's");
      if (P.fp_grid && c->has_grid && P.fp_grid != c->fp_grid)
        return ck_fail(c, ALGDOCK_E_STATE, "checkpoint_load: the context's lattice differs from the checkpoint's");
    }
    // every requested array must be present with its dtype and count (data == NULL: query)
    std::vector<const Parsed::Arr*> src(n_arrays, nullptr);
    for (int32_t a = 0; a < n_arrays; ++a) {
      algdock_array& A = arrays[a];
      const std::string name(A.name, strnlen(A.name, kNameBytes));
      for (const auto& B : P.arrays)
        if (B.name == name) src[a] = &B;
      if (!A.data) {
        A.dtype = src[a] ? (int32_t)src[a]->dtype : 0;
        A.count = src[a] ? (int64_t)src[a]->count : -1;
        continue;
      }
      if (!src[a]) return ck_fail(c, ALGDOCK_E_INVALID, "checkpoint_load: no array named " + name);
      if ((uint32_t)A.dtype != src[a]->dtype || A.count < 0 || (uint64_t)A.count != src[a]->count)
        return ck_fail(c, ALGDOCK_E_INVALID, "checkpoint_load: array " + name + " has another dtype or count");
    }
    if (c && P.K > 0) {  // the state table first: a failure leaves the caller's arrays untouched
      st = algdock_states_set(c, (int32_t)P.K, P.T.data(), P.alpha.data(), P.dt.data());
      if (st != ALGDOCK_OK) return st;
    }
    for (int32_t a = 0; a < n_arrays; ++a) {
      algdock_array& A = arrays[a];
      if (!A.data) continue;
      const size_t bytes = (size_t)src[a]->count * src[a]->esize;
      if (bytes == 0) continue;
      const uint8_t* from = P.image.data() + src[a]->offset;
      if (on_device(A.data)) {
        cudaError_t e = c ? cudaMemcpyAsync(A.data, from, bytes, cudaMemcpyHostToDevice, c->stream)
                          : cudaMemcpy(A.data, from, bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && c) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess)
          return ck_fail(c, ALGDOCK_E_CUDA, std::string("checkpoint_load: ") + cudaGetErrorString(e));
      } else {
        memcpy(A.data, from, bytes);
      }
    }
    if (seed) *seed = P.seed;
    if (cycle) *cycle = P.cycle;
    return ALGDOCK_OK;
  } catch (...) {
    return ck_fail(c, ALGDOCK_E_OOM, "checkpoint_load: host allocation failed");
  }
}

}  // extern "C"
