// cafs_sort_noalloc: the same sort for callers that must not allocate device
// memory, with every byte of scratch in one file-scope device array.
//
// Some callers cannot call cudaMalloc at all: engines that hand out only
// pre-reserved pools and forbid any other allocation, processes held to a
// fixed device-memory budget, and latency-critical loops that cannot afford
// the implicit device synchronisation of cudaMalloc/cudaFree.  For them this
// entry point takes its scratch (control block, hash table, pair arrays,
// radix buffers) from `g_noalloc_scratch`, a static __device__ array that
// every GPU loading the library holds until the process exits.  Columns are
// limited to kNoAllocMaxKeys keys.  Calls share the array, so calls whose
// work overlaps on the GPU (different streams, different host threads) race
// with each other and must be serialised by the caller.

#include <cstdint>
#include <cstring>
#include <mutex>

#include "cafs.h"
#include "cafs_internal.h"

namespace cafs {
namespace {

// Largest column this entry point accepts.
constexpr unsigned long long kNoAllocMaxKeys = 1ull << 19;

constexpr unsigned long long align256(unsigned long long x) { return (x + 255) & ~255ull; }

// Scratch layout for the largest column (int64 needs the most bytes).
constexpr unsigned long long kTab = table_capacity(kNoAllocMaxKeys, 1) > table_capacity(kNoAllocMaxKeys, 0)
                                        ? table_capacity(kNoAllocMaxKeys, 1)
                                        : table_capacity(kNoAllocMaxKeys, 0);
constexpr unsigned long long kPairs = pair_capacity(kTab);
constexpr unsigned long long kLook = lookback_words(kNoAllocMaxKeys > kPairs ? kNoAllocMaxKeys : kPairs);
constexpr unsigned long long kOffCtrl = 0;
constexpr unsigned long long kOffTKeys = align256(kOffCtrl + sizeof(Ctrl));
constexpr unsigned long long kOffTCounts = align256(kOffTKeys + kTab * 8);
constexpr unsigned long long kOffClaimed = align256(kOffTCounts + kTab * 4);
constexpr unsigned long long kOffPKA = align256(kOffClaimed + kTab * 4);
constexpr unsigned long long kOffPVA = align256(kOffPKA + kPairs * 8);
constexpr unsigned long long kOffPKB = align256(kOffPVA + kPairs * 4);
constexpr unsigned long long kOffPVB = align256(kOffPKB + kPairs * 8);
constexpr unsigned long long kOffSK = align256(kOffPVB + kPairs * 4);
constexpr unsigned long long kOffSV = align256(kOffSK + kPairs * 8);
constexpr unsigned long long kOffOff = align256(kOffSV + kPairs * 4);
constexpr unsigned long long kOffTmp = align256(kOffOff + (kPairs + 2) * 4);
constexpr unsigned long long kOffLook = align256(kOffTmp + kNoAllocMaxKeys * 8);
constexpr unsigned long long kOffSample = align256(kOffLook + kLook * 8);
constexpr unsigned long long kScratchBytes = align256(kOffSample + kSamples * 8);
static_assert(kScratchBytes <= (32ull << 20), "no-alloc scratch stays modest (<= 32 MiB)");

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct NoAllocDevice {
  bool ready = false;
  unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
  int max_grid[2] = {0, 0};
  unsigned gen = 0;
};
constexpr int kMaxDevices = 64;
NoAllocDevice g_noalloc[kMaxDevices];
std::mutex g_noalloc_mu;

// Once per device, with that device current: resolve the array's device
// address (host code must never use the symbol itself as a pointer) and the
// launch limits.
cafs_status noalloc_setup(int dev, NoAllocDevice** out) {
  if (dev < 0 || dev >= kMaxDevices) return CAFS_ERR_INVALID_ARGUMENT;
  NoAllocDevice& d = g_noalloc[dev];
  if (!d.ready) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return CAFS_ERR_CUDA;
    if (prepare_kernels() != cudaSuccess) return CAFS_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CAFS_ERR_CUDA;
    for (int t = 0; t < 2; ++t) {
      int bps = 0;
      if (pipeline_occupancy(t, &bps) != cudaSuccess || bps < 1) return CAFS_ERR_CUDA;
      long long g = (long long)bps * sms;
      if (g > 1024) g = 1024;
      d.max_grid[t] = (int)g;
    }
    d.scratch = static_cast<unsigned char*>(ptr);
    d.ready = true;
  }
  *out = &d;
  return CAFS_OK;
}

}  // namespace
}  // namespace cafs

using namespace cafs;

extern "C" cafs_status cafs_sort_noalloc(const void* keys, size_t n, cafs_dtype dtype, void* out,
                                         void* stream) {
  if (dtype != CAFS_INT32 && dtype != CAFS_INT64) return CAFS_ERR_UNSUPPORTED_DTYPE;
  if (n == 0) return CAFS_OK;
  if ((unsigned long long)n > kNoAllocMaxKeys) return CAFS_ERR_TOO_LARGE;
  const size_t kb = dtype == CAFS_INT64 ? 8 : 4;
  if (!keys || !out) return CAFS_ERR_INVALID_ARGUMENT;
  if (reinterpret_cast<uintptr_t>(keys) % kb || reinterpret_cast<uintptr_t>(out) % kb)
    return CAFS_ERR_INVALID_ARGUMENT;
  {
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(keys), b0 = reinterpret_cast<uintptr_t>(out);
    const uintptr_t bytes = (uintptr_t)n * kb;
    if (a0 != b0 && a0 < b0 + bytes && b0 < a0 + bytes) return CAFS_ERR_ALIAS;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CAFS_ERR_CUDA;
  NoAllocDevice* d = nullptr;
  cafs_status st = noalloc_setup(dev, &d);
  if (st != CAFS_OK) return st;

  unsigned char* base = d->scratch;
  Params p;
  std::memset(&p, 0, sizeof(p));
  p.keys = keys;
  p.out = out;
  p.n = n;
  p.ctrl = reinterpret_cast<Ctrl*>(base + kOffCtrl);
  p.tkeys = reinterpret_cast<unsigned long long*>(base + kOffTKeys);
  p.tcounts = reinterpret_cast<unsigned*>(base + kOffTCounts);
  p.claimed = reinterpret_cast<unsigned*>(base + kOffClaimed);
  p.table_cap = kTab;
  p.pkeys_a = base + kOffPKA;
  p.pvals_a = reinterpret_cast<unsigned*>(base + kOffPVA);
  p.pkeys_b = base + kOffPKB;
  p.pvals_b = reinterpret_cast<unsigned*>(base + kOffPVB);
  p.skeys = base + kOffSK;
  p.svals = reinterpret_cast<unsigned*>(base + kOffSV);
  p.offsets = reinterpret_cast<unsigned*>(base + kOffOff);
  p.pair_cap = kPairs;
  p.tmp = base + kOffTmp;
  p.lookback = reinterpret_cast<unsigned long long*>(base + kOffLook);
  p.lookback_cap = kLook;
  p.sample_keys = reinterpret_cast<long long*>(base + kOffSample);
  p.gen = ++d->gen;
  p.mode = kModeSort;
  p.test_flags = 0;
  p.local_slots_max = kLocalSlotsMax;
  p.replicas_max = kDefaultReplicasMax;
  p.emit_tile_vec = kEmitTileVecDefault;
  p.timeout_ns = wait_timeout_ns();
  next_hash_multipliers(&p.hash_mult, &p.local_mult);

  // The array keeps the previous call's contents: the control block must
  // start at zero and the hash table empty (every key slot the empty marker,
  // every count zero).  The rest of the scratch needs no clearing: every
  // radix pass writes each CTA's digit counts and bases (and the pair bucket
  // sort its per-CTA counts) before any CTA reads them, with a grid barrier
  // in between, and the pair and temp arrays are written before they are
  // read within a call.
  if (cudaMemsetAsync(p.ctrl, 0, sizeof(Ctrl), s) != cudaSuccess) return CAFS_ERR_CUDA;
  if (n >= kSmallN) {
    const unsigned long long tcap = table_capacity(n, dtype);
    if (launch_fill_u64(p.tkeys, tcap, 0x8000000000000000ull, s) != cudaSuccess) return CAFS_ERR_CUDA;
    count_launches(1);
    if (cudaMemsetAsync(p.tcounts, 0, tcap * 4, s) != cudaSuccess) return CAFS_ERR_CUDA;
  }
  cudaError_t e;
  if (n < kSmallN) {
    e = launch_small(p, dtype, s);
  } else {
    long long grid = (long long)((n + 16383) / 16384);
    if (grid > d->max_grid[dtype]) grid = d->max_grid[dtype];
    if (grid < 1) grid = 1;
    e = launch_pipeline(p, dtype, (int)grid, s);
  }
  if (e != cudaSuccess) return CAFS_ERR_CUDA;
  count_launches(1);
  return CAFS_OK;
}
