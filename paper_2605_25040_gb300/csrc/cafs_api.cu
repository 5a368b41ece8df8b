// Host runtime and C ABI (include/cafs.h): argument checks, per-(device,
// stream) workspaces, launch of the pipeline kernels, report read-back.

#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "cafs.h"
#include "cafs_argsort.h"
#include "cafs_internal.h"
#include "cafs_transform.h"

namespace cafs {
namespace {

std::atomic<uint64_t> g_launches{0};
uint64_t g_hash_seed = 0;        // 0: the golden-ratio multipliers
uint64_t g_hash_calls = 0;

// SplitMix64 (Steele, Lea, Flood 2014) finaliser: draws the multipliers.
uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// g_mu held.
void next_hash_multipliers_locked(unsigned long long* hash_mult, unsigned* local_mult) {
  if (g_hash_seed == 0) {
    *hash_mult = 0;
    *local_mult = 0;
    return;
  }
  const uint64_t a = mix64(g_hash_seed ^ mix64(++g_hash_calls));
  *hash_mult = a | 1ull;
  *local_mult = (unsigned)(mix64(a) >> 32) | 1u;
}
std::mutex g_mu;
unsigned g_test_flags = 0;
unsigned long long g_timeout_ns = 1000000000ull;  // bounded device waits: 1 s

struct DeviceInfo {
  bool ready = false;
  int sms = 0;
  int max_grid[2] = {0, 0};
  int max_grid_arg[2] = {0, 0};   // argsort kernels
};
std::map<int, DeviceInfo> g_dev;

struct Workspace {
  int device = -1;
  unsigned gen = 0;
  // capacities
  unsigned long long n_cap = 0;        // keys the radix temp holds (per dtype bytes)
  size_t tmp_bytes = 0;
  unsigned long long table_cap = 0;
  unsigned long long pair_cap = 0;
  unsigned long long lookback_cap = 0;
  size_t io_bytes = 0;
  // device buffers
  Ctrl* ctrl = nullptr;        // two blocks: launch i uses ctrl[cur] and zeroes the other
  int cur = 0;
  Ctrl* last = nullptr;        // the block of the last launch (its record is the report)
  unsigned long long* tkeys = nullptr;
  unsigned* tcounts = nullptr;
  unsigned* claimed = nullptr;
  void* pkeys_a = nullptr; unsigned* pvals_a = nullptr;
  void* pkeys_b = nullptr; unsigned* pvals_b = nullptr;
  void* skeys = nullptr; unsigned* svals = nullptr;
  unsigned* offsets = nullptr;
  void* tmp = nullptr;
  unsigned long long* lookback = nullptr;
  long long* sample_keys = nullptr;
  void* io = nullptr;
  unsigned* arg = nullptr;     // argsort scratch: 4 arrays of arg_n words
  unsigned long long arg_n = 0;
  Record* host_rec = nullptr;  // pinned
};
std::map<std::pair<int, uintptr_t>, Workspace*> g_ws;

template <typename T>
void free_dev(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

void release_buffers(Workspace* w) {
  free_dev(w->ctrl); free_dev(w->tkeys); free_dev(w->tcounts); free_dev(w->claimed);
  free_dev(w->pkeys_a); free_dev(w->pvals_a); free_dev(w->pkeys_b); free_dev(w->pvals_b);
  free_dev(w->skeys); free_dev(w->svals); free_dev(w->offsets); free_dev(w->tmp);
  free_dev(w->lookback); free_dev(w->sample_keys); free_dev(w->arg);
  w->arg_n = 0;
  w->n_cap = 0; w->tmp_bytes = 0; w->table_cap = 0; w->pair_cap = 0; w->lookback_cap = 0;
}

cafs_status ensure_device(int dev, DeviceInfo** out) {
  DeviceInfo& d = g_dev[dev];
  if (!d.ready) {
    if (prepare_kernels() != cudaSuccess || prepare_argsort_kernels() != cudaSuccess) return CAFS_ERR_CUDA;
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CAFS_ERR_CUDA;
    for (int t = 0; t < 2; ++t) {
      int bps = 0;
      if (pipeline_occupancy(t, &bps) != cudaSuccess || bps < 1) return CAFS_ERR_CUDA;
      long long g = (long long)bps * d.sms;
      if (g > 1024) g = 1024;  // Ctrl::chunk_sums holds one partial sum per CTA
      d.max_grid[t] = (int)g;
      if (argsort_occupancy(t, &bps) != cudaSuccess || bps < 1) return CAFS_ERR_CUDA;
      g = (long long)bps * d.sms;
      d.max_grid_arg[t] = (int)(g > 1024 ? 1024 : g);
    }
    d.ready = true;
  }
  *out = &d;
  return CAFS_OK;
}

template <typename T>
cudaError_t alloc(T** p, size_t bytes) {
  return cudaMalloc((void**)p, bytes < 16 ? 16 : bytes);
}

// Makes the workspace big enough for n keys of dtype; call with g_mu held.
cafs_status ensure_workspace(Workspace* w, unsigned long long n, int dtype, cudaStream_t s,
                             bool need_io) {
  const size_t kb = dtype == CAFS_INT64 ? 8 : 4;
  const unsigned long long tcap = table_capacity(n, dtype);
  const unsigned long long pcap = pair_capacity(tcap);
  const unsigned long long lcap = lookback_words(n > pcap ? n : pcap);
  const size_t tmp_bytes = (size_t)n * kb;
  const bool grow = !w->ctrl || tcap > w->table_cap || pcap > w->pair_cap ||
                    lcap > w->lookback_cap || tmp_bytes > w->tmp_bytes;
  if (grow) {
    if (w->ctrl && cudaStreamSynchronize(s) != cudaSuccess) return CAFS_ERR_CUDA;
    const unsigned long long ntc = tcap > w->table_cap ? tcap : w->table_cap;
    const unsigned long long npc = pcap > w->pair_cap ? pcap : w->pair_cap;
    const unsigned long long nlc = lcap > w->lookback_cap ? lcap : w->lookback_cap;
    const size_t ntb = tmp_bytes > w->tmp_bytes ? tmp_bytes : w->tmp_bytes;
    release_buffers(w);
    bool ok = alloc(&w->ctrl, 2 * sizeof(Ctrl)) == cudaSuccess &&
              alloc(&w->tkeys, ntc * 8) == cudaSuccess &&
              alloc(&w->tcounts, ntc * 4) == cudaSuccess &&
              alloc(&w->claimed, ntc * 4) == cudaSuccess &&
              alloc(&w->pkeys_a, npc * 8) == cudaSuccess &&
              alloc(&w->pvals_a, npc * 4) == cudaSuccess &&
              alloc(&w->pkeys_b, npc * 8) == cudaSuccess &&
              alloc(&w->pvals_b, npc * 4) == cudaSuccess &&
              alloc(&w->skeys, npc * 8) == cudaSuccess &&
              alloc(&w->svals, npc * 4) == cudaSuccess &&
              alloc(&w->offsets, (npc + 2) * 4) == cudaSuccess &&
              alloc(&w->tmp, ntb) == cudaSuccess &&
              alloc(&w->lookback, nlc * 8) == cudaSuccess &&
              alloc(&w->sample_keys, kSamples * 8) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      release_buffers(w);
      return CAFS_ERR_OUT_OF_MEMORY;
    }
    // Empty table: every key slot holds the empty marker, every count 0.
    if (launch_fill_u64(w->tkeys, ntc, 0x8000000000000000ull, s) != cudaSuccess) return CAFS_ERR_CUDA;
    g_launches++;
    if (cudaMemsetAsync(w->tcounts, 0, ntc * 4, s) != cudaSuccess) return CAFS_ERR_CUDA;
    if (cudaMemsetAsync(w->lookback, 0, nlc * 8, s) != cudaSuccess) return CAFS_ERR_CUDA;
    if (cudaMemsetAsync(w->ctrl, 0, 2 * sizeof(Ctrl), s) != cudaSuccess) return CAFS_ERR_CUDA;
    w->cur = 0;
    w->last = w->ctrl;
    w->table_cap = ntc; w->pair_cap = npc; w->lookback_cap = nlc; w->tmp_bytes = ntb;
    w->n_cap = n;
  }
  if (!w->host_rec) {
    if (cudaMallocHost((void**)&w->host_rec, sizeof(Record)) != cudaSuccess) return CAFS_ERR_OUT_OF_MEMORY;
  }
  if (need_io && (size_t)n * kb > w->io_bytes) {
    if (w->io) {
      if (cudaStreamSynchronize(s) != cudaSuccess) return CAFS_ERR_CUDA;
      cudaFree(w->io);
      w->io = nullptr;
    }
    if (alloc(&w->io, (size_t)n * kb) != cudaSuccess) {
      cudaGetLastError();
      w->io_bytes = 0;
      return CAFS_ERR_OUT_OF_MEMORY;
    }
    w->io_bytes = (size_t)n * kb;
  }
  return CAFS_OK;
}

Workspace* workspace_for(int dev, cudaStream_t s) {
  auto key = std::make_pair(dev, reinterpret_cast<uintptr_t>(s));
  auto it = g_ws.find(key);
  if (it != g_ws.end()) return it->second;
  Workspace* w = new Workspace();
  w->device = dev;
  g_ws[key] = w;
  return w;
}

// Key types: element width, the signed type the pipeline sorts (0: int32,
// 1: int64) and the order map onto it (0: none, 1: unsigned, 2: IEEE float).
bool known_type(cafs_dtype t) { return key_type_known(t); }
size_t type_width(cafs_dtype t) { return key_type_width(t); }
int base_type(cafs_dtype t) { return key_type_base(t); }
int order_kind(cafs_dtype t) { return key_type_kind(t); }

// `any_type`: the entry point takes every key type (else int32/int64 only).
cafs_status check_args_impl(const void* keys, size_t n, cafs_dtype dtype, const void* out, bool need_out,
                            bool any_type = false) {
  if (any_type ? !known_type(dtype) : (dtype != CAFS_INT32 && dtype != CAFS_INT64))
    return CAFS_ERR_UNSUPPORTED_DTYPE;
  if (n == 0) return CAFS_OK;
  if ((unsigned long long)n > 0xFFFFFFFFull) return CAFS_ERR_TOO_LARGE;
  const size_t kb = type_width(dtype);
  if (!keys || (need_out && !out)) return CAFS_ERR_INVALID_ARGUMENT;
  if (reinterpret_cast<uintptr_t>(keys) % kb) return CAFS_ERR_INVALID_ARGUMENT;
  if (need_out) {
    if (reinterpret_cast<uintptr_t>(out) % kb) return CAFS_ERR_INVALID_ARGUMENT;
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(keys), b0 = reinterpret_cast<uintptr_t>(out);
    const uintptr_t bytes = (uintptr_t)n * kb;
    if (a0 != b0 && a0 < b0 + bytes && b0 < a0 + bytes) return CAFS_ERR_ALIAS;
  }
  return CAFS_OK;
}

void fill_estimate(const Record& r, cafs_estimate* e) {
  e->n = r.n;
  e->stride = r.stride;
  e->n_samples = r.n_samples;
  e->u = r.u;
  e->f1 = r.f1;
  e->f2 = r.f2;
  e->k_hat = r.k_hat;
  e->saturated = r.saturated;
  e->sample_nondecreasing = r.sample_nondecreasing;
  e->M = r.M;
  e->C = r.C;
  e->L = r.L;
  e->dispatch = (cafs_path)r.dispatch;
}

// Kernel parameters of one column over workspace w (g_mu held).
Params pipeline_params(Workspace* w, const void* keys, void* out, unsigned long long n, int mode) {
  Params p;
  std::memset(&p, 0, sizeof(p));
  p.keys = keys;
  p.out = out;
  p.n = n;
  p.ctrl = w->ctrl + w->cur;
  p.ctrl_next = w->ctrl + (w->cur ^ 1);
  p.tkeys = w->tkeys;
  p.tcounts = w->tcounts;
  p.claimed = w->claimed;
  p.table_cap = w->table_cap;
  p.pkeys_a = w->pkeys_a; p.pvals_a = w->pvals_a;
  p.pkeys_b = w->pkeys_b; p.pvals_b = w->pvals_b;
  p.skeys = w->skeys; p.svals = w->svals;
  p.offsets = w->offsets;
  p.pair_cap = w->pair_cap;
  p.tmp = w->tmp;
  p.lookback = w->lookback;
  p.lookback_cap = w->lookback_cap;
  p.sample_keys = w->sample_keys;
  p.gen = ++w->gen;
  p.mode = mode;
  p.test_flags = g_test_flags;
  p.local_slots_max = kLocalSlotsMax;
  p.replicas_max = kDefaultReplicasMax;
  p.emit_tile_vec = kEmitTileVecDefault;
  p.timeout_ns = g_timeout_ns;
  next_hash_multipliers_locked(&p.hash_mult, &p.local_mult);
  return p;
}

// CTAs of a cooperative launch over n keys: one per 16384 keys, at most
// one per SM (the persistent kernels' occupancy).
int launch_grid(unsigned long long n, int max_grid) {
  long long grid = (long long)((n + 16383) / 16384);
  if (grid > max_grid) grid = max_grid;
  return grid < 1 ? 1 : (int)grid;
}

// The launch just enqueued used ctrl[cur] and zeroes the other block: the
// next launch takes that one (g_mu held).
void advance_ctrl(Workspace* w) {
  w->last = w->ctrl + w->cur;
  w->cur ^= 1;
}

// Enqueues one pipeline run on stream s (g_mu held).  The control block it
// uses was zeroed by the previous launch on this workspace (or at
// allocation).
cafs_status enqueue(Workspace* w, const DeviceInfo* d, const void* keys, void* out,
                    unsigned long long n, int dtype, int mode, cudaStream_t s) {
  const Params p = pipeline_params(w, keys, out, n, mode);
  cudaError_t e;
  if (n < kSmallN) {
    e = launch_small(p, dtype, s);
  } else {
    e = launch_pipeline(p, dtype, launch_grid(n, d->max_grid[dtype]), s);
  }
  if (e != cudaSuccess) return CAFS_ERR_CUDA;
  advance_ctrl(w);
  g_launches++;
  return CAFS_OK;
}

cafs_status read_record(Workspace* w, cudaStream_t s, Record* r) {
  if (cudaMemcpyAsync(w->host_rec, &w->last->rec, sizeof(Record), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CAFS_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CAFS_ERR_CUDA;
  *r = *w->host_rec;
  return CAFS_OK;
}

void fill_report_impl(const Record& r, cafs_report* rep) {
  std::memset(rep, 0, sizeof(*rep));
  fill_estimate(r, &rep->est);
  rep->path = (cafs_path)r.path;
  rep->k_distinct = r.k_distinct;
  rep->device_status = (cafs_status)r.status;
  for (int i = 0; i < 6; ++i) rep->timeline_ns[i] = r.timeline[i];
}

// The order map of key type t applied to n keys src -> dst (counted launch).
cafs_status map_keys(const void* src, void* dst, unsigned long long n, cafs_dtype t, cudaStream_t s) {
  if (launch_order_map(src, dst, n, (int)type_width(t), order_kind(t), s) != cudaSuccess) return CAFS_ERR_CUDA;
  g_launches++;
  return CAFS_OK;
}

cafs_status sort_impl(const void* keys, size_t n, cafs_dtype dtype, void* out, cafs_report* report,
                      void* stream) {
  cafs_status st = check_args_impl(keys, n, dtype, out, true, true);
  if (st != CAFS_OK) return st;
  if (n == 0) {
    if (report) {
      std::memset(report, 0, sizeof(*report));
      report->path = CAFS_PATH_EMPTY;
      report->est.dispatch = CAFS_PATH_EMPTY;
    }
    return CAFS_OK;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CAFS_ERR_CUDA;
  DeviceInfo* d = nullptr;
  if ((st = ensure_device(dev, &d)) != CAFS_OK) return st;
  Workspace* w = workspace_for(dev, s);
  const int bt = base_type(dtype);
  if ((st = ensure_workspace(w, n, bt, s, false)) != CAFS_OK) return st;
  if (order_kind(dtype)) {
    // keys -> out in the signed order, sorted in place, mapped back
    if ((st = map_keys(keys, out, n, dtype, s)) != CAFS_OK) return st;
    if ((st = enqueue(w, d, out, out, n, bt, kModeSort, s)) != CAFS_OK) return st;
    if ((st = map_keys(out, out, n, dtype, s)) != CAFS_OK) return st;
  } else if ((st = enqueue(w, d, keys, out, n, bt, kModeSort, s)) != CAFS_OK) {
    return st;
  }
  if (report) {
    Record r;
    if ((st = read_record(w, s, &r)) != CAFS_OK) return st;
    fill_report_impl(r, report);
  }
  return CAFS_OK;
}

// Stable argsort of one column (keys, out and perm pairwise disjoint).
cafs_status argsort_impl(const void* keys, size_t n, cafs_dtype dtype, void* out, uint32_t* perm,
                         cafs_report* report, void* stream) {
  cafs_status st = check_args_impl(keys, n, dtype, out, true, true);
  if (st != CAFS_OK) return st;
  if (n == 0) {
    if (report) {
      std::memset(report, 0, sizeof(*report));
      report->path = CAFS_PATH_EMPTY;
      report->est.dispatch = CAFS_PATH_EMPTY;
    }
    return CAFS_OK;
  }
  if (!perm || reinterpret_cast<uintptr_t>(perm) % 4) return CAFS_ERR_INVALID_ARGUMENT;
  const uintptr_t kb = type_width(dtype);
  const uintptr_t k0 = reinterpret_cast<uintptr_t>(keys), o0 = reinterpret_cast<uintptr_t>(out);
  const uintptr_t p0 = reinterpret_cast<uintptr_t>(perm);
  const uintptr_t kbytes = (uintptr_t)n * kb, pbytes = (uintptr_t)n * 4;
  auto overlap = [](uintptr_t a, uintptr_t an, uintptr_t b, uintptr_t bn) { return a < b + bn && b < a + an; };
  if (overlap(k0, kbytes, o0, kbytes) || overlap(p0, pbytes, k0, kbytes) || overlap(p0, pbytes, o0, kbytes))
    return CAFS_ERR_ALIAS;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CAFS_ERR_CUDA;
  DeviceInfo* d = nullptr;
  if ((st = ensure_device(dev, &d)) != CAFS_OK) return st;
  Workspace* w = workspace_for(dev, s);
  const int bt = base_type(dtype);
  const bool mapped = order_kind(dtype) != 0;
  if ((st = ensure_workspace(w, n, bt, s, mapped)) != CAFS_OK) return st;
  if ((unsigned long long)n > w->arg_n) {
    if (w->arg) {
      if (cudaStreamSynchronize(s) != cudaSuccess) return CAFS_ERR_CUDA;
      free_dev(w->arg);
      w->arg_n = 0;
    }
    if (alloc(&w->arg, (size_t)n * 16) != cudaSuccess) {
      cudaGetLastError();
      return CAFS_ERR_OUT_OF_MEMORY;
    }
    w->arg_n = n;
  }
  // other key types: their signed images in the io buffer (the kernel reads
  // the keys again after the sorted keys are written)
  const void* src = keys;
  if (mapped) {
    if ((st = map_keys(keys, w->io, n, dtype, s)) != CAFS_OK) return st;
    src = w->io;
  }
  ArgsortParams ap;
  ap.p = pipeline_params(w, src, out, n, kModeSort);
  ap.perm = perm;
  ap.rk = w->arg;
  ap.iv = w->arg + n;
  ap.tv = w->arg + 2 * (size_t)n;
  ap.rk2 = w->arg + 3 * (size_t)n;
  cudaError_t e;
  if (n < kSmallN) e = launch_small_argsort(ap, bt, s);
  else e = launch_argsort(ap, bt, launch_grid(n, d->max_grid_arg[bt]), s);
  if (e != cudaSuccess) return CAFS_ERR_CUDA;
  advance_ctrl(w);
  g_launches++;
  if (mapped && (st = map_keys(out, out, n, dtype, s)) != CAFS_OK) return st;
  if (report) {
    Record r;
    if ((st = read_record(w, s, &r)) != CAFS_OK) return st;
    fill_report_impl(r, report);
  }
  return CAFS_OK;
}

}  // namespace

void count_launches(unsigned k) { g_launches += k; }
void next_hash_multipliers(unsigned long long* hash_mult, unsigned* local_mult) {
  std::lock_guard<std::mutex> lock(g_mu);
  next_hash_multipliers_locked(hash_mult, local_mult);
}
unsigned long long wait_timeout_ns() {
  std::lock_guard<std::mutex> lock(g_mu);
  return g_timeout_ns;
}
cafs_status check_args(const void* keys, size_t n, cafs_dtype dtype, const void* out, bool need_out) {
  return check_args_impl(keys, n, dtype, out, need_out);
}
cafs_status check_args_typed(const void* keys, size_t n, cafs_dtype dtype, const void* out, bool need_out) {
  return check_args_impl(keys, n, dtype, out, need_out, true);
}
void fill_report(const Record& r, cafs_report* rep) { fill_report_impl(r, rep); }

}  // namespace cafs

using namespace cafs;

extern "C" {

cafs_status cafs_sort(const void* keys, size_t n, cafs_dtype dtype, void* out, void* stream) {
  return sort_impl(keys, n, dtype, out, nullptr, stream);
}

cafs_status cafs_sort_ex(const void* keys, size_t n, cafs_dtype dtype, void* out,
                         cafs_report* report, void* stream) {
  return sort_impl(keys, n, dtype, out, report, stream);
}

cafs_status cafs_argsort(const void* keys, size_t n, cafs_dtype dtype, void* out, uint32_t* perm,
                         cafs_report* report, void* stream) {
  return argsort_impl(keys, n, dtype, out, perm, report, stream);
}

cafs_status cafs_estimate_k(const void* keys, size_t n, cafs_dtype dtype, cafs_estimate* est,
                            void* stream) {
  if (!est) return CAFS_ERR_INVALID_ARGUMENT;
  cafs_status st = check_args_impl(keys, n, dtype, nullptr, false, true);
  if (st != CAFS_OK) return st;
  std::memset(est, 0, sizeof(*est));
  if (n == 0) {
    est->dispatch = CAFS_PATH_EMPTY;
    return CAFS_OK;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CAFS_ERR_CUDA;
  DeviceInfo* d = nullptr;
  if ((st = ensure_device(dev, &d)) != CAFS_OK) return st;
  Workspace* w = workspace_for(dev, s);
  const int bt = base_type(dtype);
  const bool mapped = order_kind(dtype) != 0;
  if ((st = ensure_workspace(w, n, bt, s, mapped)) != CAFS_OK) return st;
  const void* src = keys;
  if (mapped) {
    if ((st = map_keys(keys, w->io, n, dtype, s)) != CAFS_OK) return st;
    src = w->io;
  }
  if ((st = enqueue(w, d, src, nullptr, n, bt, kModeEstimate, s)) != CAFS_OK) return st;
  Record r;
  if ((st = read_record(w, s, &r)) != CAFS_OK) return st;
  if (r.status != kDevOk) return (cafs_status)r.status;
  fill_estimate(r, est);
  return CAFS_OK;
}

cafs_status cafs_sort_host(const void* host_keys, size_t n, cafs_dtype dtype, void* host_out,
                           cafs_report* report, void* stream) {
  cafs_status st = check_args_impl(host_keys, n, dtype, host_out, false, true);
  if (st != CAFS_OK) return st;
  if (n && !host_out) return CAFS_ERR_INVALID_ARGUMENT;
  if (n == 0) {
    if (report) {
      std::memset(report, 0, sizeof(*report));
      report->path = CAFS_PATH_EMPTY;
    }
    return CAFS_OK;
  }
  const size_t bytes = n * type_width(dtype);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CAFS_ERR_CUDA;
  DeviceInfo* d = nullptr;
  if ((st = ensure_device(dev, &d)) != CAFS_OK) return st;
  Workspace* w = workspace_for(dev, s);
  const int bt = base_type(dtype);
  if ((st = ensure_workspace(w, n, bt, s, true)) != CAFS_OK) return st;
  if (cudaMemcpyAsync(w->io, host_keys, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return CAFS_ERR_CUDA;
  if (order_kind(dtype) && (st = map_keys(w->io, w->io, n, dtype, s)) != CAFS_OK) return st;
  if ((st = enqueue(w, d, w->io, w->io, n, bt, kModeSort, s)) != CAFS_OK) return st;
  if (order_kind(dtype) && (st = map_keys(w->io, w->io, n, dtype, s)) != CAFS_OK) return st;
  if (cudaMemcpyAsync(host_out, w->io, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CAFS_ERR_CUDA;
  Record r;
  if ((st = read_record(w, s, &r)) != CAFS_OK) return st;
  if (report) fill_report_impl(r, report);
  return CAFS_OK;
}

void cafs_set_hash_seed(uint64_t seed) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_hash_seed = seed;
  g_hash_calls = 0;
}

void cafs_set_test_hooks(uint32_t flags, uint64_t wait_timeout_ns) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_test_flags = flags;
  g_timeout_ns = wait_timeout_ns ? wait_timeout_ns : 1000000000ull;
}

uint64_t cafs_kernel_launch_count(void) { return g_launches.load(); }

const char* cafs_status_string(cafs_status s) {
  switch (s) {
    case CAFS_OK: return "ok";
    case CAFS_ERR_INVALID_ARGUMENT: return "invalid argument";
    case CAFS_ERR_UNSUPPORTED_DTYPE: return "unsupported dtype";
    case CAFS_ERR_TOO_LARGE: return "n exceeds 2^32-1";
    case CAFS_ERR_ALIAS: return "keys and out overlap partially";
    case CAFS_ERR_OUT_OF_MEMORY: return "out of device memory";
    case CAFS_ERR_CUDA: return "CUDA runtime error";
    case CAFS_ERR_TIMEOUT: return "bounded device wait timed out";
    case CAFS_ERR_INTERNAL: return "internal error";
    case CAFS_ERR_BUSY: return "busy";
  }
  return "unknown status";
}

const char* cafs_path_string(cafs_path p) {
  switch (p) {
    case CAFS_PATH_EMPTY: return "empty";
    case CAFS_PATH_BYPASS_SORTED: return "bypass_sorted";
    case CAFS_PATH_SMALL_N: return "small_n";
    case CAFS_PATH_TINY: return "tiny";
    case CAFS_PATH_MAIN: return "main";
    case CAFS_PATH_HIGH_ENTROPY_RADIX: return "high_entropy_radix";
    case CAFS_PATH_MAIN_OVERFLOW_RADIX: return "main_overflow_radix";
    case CAFS_PATH_TINY_MISS_MAIN: return "tiny_miss_main";
    case CAFS_PATH_TINY_MISS_MAIN_OVERFLOW_RADIX: return "tiny_miss_main_overflow_radix";
  }
  return "unknown path";
}

}  // extern "C"
