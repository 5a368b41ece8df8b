// Internal definitions shared by the kernels (cafs_pipeline.cu) and the host
// runtime (cafs_api.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "cafs.h"

namespace cafs {

// Algorithm 2: number of strided samples s.
constexpr int kSamples = 1024;
// Table 2 / Algorithm 3: below this length the sampler is skipped.
constexpr uint64_t kSmallN = 2048;
// Table 2: tiny-count branch limit on K_hat and u.
constexpr int kTinyMax = 8;
// Tiny path: the sampled keys are hashed collision-free into this many
// buckets (log2: kTinyBucketBits) by a multiplier found during sampling.
constexpr int kTinyBucketBits = 4;
constexpr int kTinyBuckets = 1 << kTinyBucketBits;

// Threads per CTA of every kernel in the library (one CTA per SM).
constexpr int kThreads = 1024;
// Largest grid of the persistent pipeline (per-CTA arrays are sized by it).
constexpr int kMaxGrid = 1024;
constexpr int kWarps = kThreads / 32;

// Dynamic shared memory of the persistent pipeline kernel (bytes): during
// the count phase it holds the bulk-copy ring and the per-CTA hash table.
constexpr int kPipelineSmem = 226 * 1024;
// Count phase: one producer warp streams the CTA's share of the column
// through a ring of chunks with cp.async.bulk; the other warps
// consume.  A chunk is kVecsPerThread 16-byte vectors per consumer thread.
constexpr int kConsumerWarps = kWarps - 1;
constexpr int kVecsPerThread = 2;
constexpr int kChunkVecs = kConsumerWarps * 32 * kVecsPerThread;
constexpr int kChunkBytes = kChunkVecs * 16;
// The ring sits at the top of shared memory (about 128 KB must be in flight
// per SM to reach full read bandwidth); it is filled from the start of the
// launch, while CTA 0 samples, and never overlaps the sampler's or the count
// phase's tables below it.
constexpr int kRingStages = 4;
constexpr int kRingBytes = kRingStages * kChunkBytes;
// Just below the ring: its mbarriers (full and empty per stage) and the
// shared copy of the skip flag.
constexpr int kRingReserve = 256;
static_assert(2 * kRingStages * 8 + 4 <= kRingReserve, "ring barriers below the ring");
// Shared-memory budget of the per-CTA hash table (keys + counters), of the
// small bookkeeping area before it, and of the tiny path's table (the tiny
// path's per-thread bucket counters follow it inside the table budget).
constexpr int kLocalTableBytes = 96 * 1024;
constexpr int kSmallTableBytes = 48 * 1024;   // R is trimmed to this for S <= 2048
constexpr int kMiscBytes = 512;
constexpr int kTinyTableBytes = 36 * 1024;
// Largest per-CTA shared hash table (slots).
constexpr int kLocalSlotsMax = 8192;
// Pair counts up to this size are ordered by an all-CTA rank computation;
// larger counts go through the LSD radix sort.
constexpr int kRankPairs = 4096;
// Columns shorter than this are sorted by one CTA in shared memory.
constexpr int kSmallCap = 2048;
// Pair arrays hold at least this many entries.
constexpr int kSmallPairs = 8192;
// Radix sort: 8-bit digits; items per thread per tile.
constexpr int kRadixBits = 8;
constexpr int kRadixDigits = 1 << kRadixBits;
constexpr int kRadixItems = 8;
constexpr int kRadixTile = kThreads * kRadixItems;
// Emit: elements per output tile and pairs staged per tile in shared memory.
constexpr int kEmitStagePairs = 4096;

// Device status codes (match cafs_status values).
constexpr unsigned kDevOk = 0;
constexpr unsigned kDevTimeout = 7;
constexpr unsigned kDevInternal = 8;

// Pipeline modes.
constexpr int kModeSort = 0;
constexpr int kModeEstimate = 1;

// Test hooks (bit flags in Params::test_flags).
constexpr unsigned kTestSkipBarrier = 1u;   // CTA 0 never arrives: the others time out

// Result of the sampler / dispatcher, written by the device.
struct Record {
  unsigned long long n, stride, k_hat, M, C, L;
  unsigned n_samples, u, f1, f2;
  int saturated, sample_nondecreasing;
  int dispatch;   // Algorithm 3 decision
  int path;       // final branch
  int n_tiny;
  int pad0;
  long long tiny_keys[kTinyMax];  // the u <= 8 distinct sample values (first-sample order)
  unsigned long long tiny_mult;   // odd multiplier hashing the tiny keys to distinct
  int tiny_hash_ok;               //   buckets of kTinyBuckets (0: none found)
  int pad_t;
  unsigned long long k_distinct;  // distinct keys counted (K')
  unsigned long long n_pairs;     // entries in the sorted pair arrays (padded)
  unsigned status;                // kDevOk / kDevTimeout / ...
  unsigned pad1;
  unsigned long long timeline[8]; // globaltimer ns at phase boundaries
};

// Control block: zeroed by the host before every pipeline launch.
struct Ctrl {
  Record rec;
  unsigned bar_count;
  unsigned bar_epoch;
  unsigned occupancy;           // global-table slots claimed
  unsigned overflow;            // guard fired (distinct keys > L or table full)
  unsigned inversion;           // IsMonotone found a descent
  unsigned pad2;
  unsigned long long special;   // keys equal to the type minimum (the empty marker)
  unsigned long long key_or;     // radix (all CTAs): OR of the order-mapped keys
  unsigned long long key_nor;    //   and OR of their complements (bits that vary)
  unsigned unused_tickets[14];
  unsigned hist[8][kRadixDigits];  // radix: global digit counts per pass
  unsigned long long chunk_sums[1024];  // scan: per-CTA partial sums
};

struct Params {
  const void* keys;
  void* out;
  unsigned long long n;
  Ctrl* ctrl;
  // A second control block that CTA 0 zeroes at the start of the launch, for
  // the launch after this one (nullptr: none; the host zeroes ctrl instead).
  Ctrl* ctrl_next;
  // global hash table (C slots used, capacity table_cap)
  unsigned long long* tkeys;
  unsigned* tcounts;
  unsigned* claimed;
  unsigned long long table_cap;
  // pair arrays: A (gathered), B (radix temp), S (sorted) + offsets
  void* pkeys_a; unsigned* pvals_a;
  void* pkeys_b; unsigned* pvals_b;
  void* skeys;   unsigned* svals;
  unsigned* offsets;
  unsigned long long pair_cap;
  // radix fallback temp buffer (n keys) and look-back status words
  void* tmp;
  unsigned long long* lookback;       // radix scratch: per-CTA digit counts and bases
  unsigned long long lookback_cap;   // words
  long long* sample_keys;            // kSamples: distinct sampled keys (FreqSet slot order)
  unsigned gen;          // call counter (diagnostic)
  int mode;
  unsigned test_flags;
  // Scheduling knobs (never change a result): cap on the per-CTA shared
  // hash table (slots, power of two in [256, kLocalSlotsMax]), cap on its
  // counter replicas per slot (power of two in [1, 32]) and the emit tile
  // (16-byte vectors, multiple of kThreads, <= kEmitTileVecMax).
  unsigned local_slots_max;
  unsigned replicas_max;
  unsigned emit_tile_vec;
  // Odd multipliers of the per-CTA shared table's bucket hash and of the
  // global table's Eq. 4 hash (0: the golden-ratio constants).  A per-call
  // seed draws them; no count, result or path depends on them.
  unsigned local_mult;
  unsigned long long timeout_ns;
  unsigned long long hash_mult;
};

// Default scheduling knobs.
constexpr unsigned kDefaultReplicasMax = 32;
constexpr unsigned kEmitTileVecDefault = 4096;
constexpr unsigned kEmitTileVecMax = 8192;

// ---------------------------------------------------------------------------
// Workspace sizing shared by the host entry points.
// ---------------------------------------------------------------------------
constexpr unsigned long long bit_ceil_host(unsigned long long x) {
  unsigned long long r = 1;
  while (r < x) r <<= 1;
  return r;
}

// Largest Chao1 estimate short of saturation: u = 1022 distinct samples, 1021
// of them seen once and one seen three times (Eq. 5 maximised over the sample
// spectra with u < 1024).  Any main-path table is sized from K_hat <= this.
constexpr unsigned long long kMaxUnsaturatedKhat = 522242ull;

// Slots of the largest global table a column of n keys can need (Eq. 6 with
// K_hat <= kMaxUnsaturatedKhat and the clamps).  dtype 1 = int64, 0 = int32.
constexpr unsigned long long table_capacity(unsigned long long n, int dtype) {
  const unsigned long long cap = dtype == 1 ? 4 : 8;
  unsigned long long m = bit_ceil_host((8ull * kMaxUnsaturatedKhat) / cap);
  const unsigned long long upper = bit_ceil_host((n + cap - 1) / cap);
  if (m > upper) m = upper;
  if (m < 8) m = 8;
  return m * cap;
}

// Entries of the pair arrays for a table of tcap slots (L + the type minimum).
constexpr unsigned long long pair_capacity(unsigned long long tcap) {
  return tcap / 2 + 2 > (unsigned long long)kSmallPairs ? tcap / 2 + 2 : (unsigned long long)kSmallPairs;
}

// The pair bucket sort (K' > kRankPairs) runs on grids of up to this many
// CTAs; its scratch holds, per producer CTA and bucket, a pair count, a key
// count sum and a base (three G x G arrays of 32-bit words), then the bucket
// totals and their key-count sums (64-bit words).
constexpr unsigned kBucketMaxGrid = 256;
__host__ __device__ constexpr unsigned long long bucket_scratch_words(unsigned long long G) {
  return (3ull * G * G + 2ull * G + 1ull) / 2ull + 1ull;
}

// 64-bit words of the radix scratch of a scope of `parts` CTAs: per-CTA
// digit counts and bases, two [parts][kRadixDigits] arrays of 32-bit words,
// then the pair bucket sort's scratch (grids up to kBucketMaxGrid CTAs),
// then the grid-wide sampler's kSamples gathered keys in the last kSamples
// words (apart, because a CTA may start counting digits while another still
// reads the samples).
constexpr unsigned long long radix_scratch_words(unsigned long long parts) {
  return parts * kRadixDigits + bucket_scratch_words(parts < kBucketMaxGrid ? parts : kBucketMaxGrid) +
         (unsigned long long)kSamples;
}

// The same for any grid up to kMaxGrid (independent of n).
constexpr unsigned long long lookback_words(unsigned long long /*items*/) {
  return radix_scratch_words(kMaxGrid);
}

// ---------------------------------------------------------------------------
// Batched form: many columns in one persistent cooperative launch.  Columns
// with n >= grid_min_n are sorted one after another by all CTAs together;
// the others form a work queue (longest first) from which every CTA takes
// whole columns and sorts each alone; radix-fallback columns of that queue
// with n >= defer_min_n are put aside and radix-sorted by all CTAs at the
// end.
// ---------------------------------------------------------------------------
struct BatchColumn {
  const void* keys;
  void* out;
  unsigned long long n;
  int dtype;   // 0 int32, 1 int64
  int pad;
};

// Byte offsets of one column workspace ("slot") and its capacities.  The
// radix temp buffer shares its bytes with the pair arrays: a column uses
// one or the other, never both.  A per-CTA slot may hold a smaller table
// than its longest column could need (Eq. 6); such a column is set aside
// after sampling and sorted by all CTAs.
struct SlotLayout {
  unsigned long long ctrl, tkeys, tcounts, claimed;
  unsigned long long pka, pva, pkb, pvb, sk, sv, off, tmp, look, sample;
  unsigned long long table_cap, pair_cap, lookback_cap, n_cap, bytes;
};

struct BatchState {     // zeroed before every batched launch
  unsigned next;        // work-queue cursor
  unsigned ndeferred;   // columns deferred to the all-CTA radix phase
  unsigned status;      // first device failure (kDevOk when none)
  unsigned pad;
};

struct BatchParams {
  const BatchColumn* cols;
  const unsigned* grid_items;   // columns sorted by all CTAs, in order
  const unsigned* cta_items;    // work queue, longest column first
  unsigned* deferred;           // >= n_cta entries
  Record* records;              // one per column
  BatchState* state;
  unsigned char* grid_slot;
  unsigned char* cta_slots;     // slot b at cta_slots + b * cta_layout.bytes
  SlotLayout grid_layout;
  SlotLayout cta_layout;
  unsigned n_grid, n_cta;
  unsigned long long defer_min_n;
  unsigned local_slots_max, replicas_max, emit_tile_vec, local_mult;
  unsigned long long timeout_ns;
  unsigned long long hash_mult;
};

// Slot layout: a hash table of table_cap slots (with pair arrays for its
// L + 1 pairs), a radix temp buffer of tmp_keys keys (either dtype), radix
// scratch for up to `parts` CTAs.
SlotLayout slot_layout(unsigned long long table_cap, unsigned long long tmp_keys, unsigned parts);
// Largest table any column of up to n keys can need (either dtype).
constexpr unsigned long long table_capacity_any(unsigned long long n) {
  return table_capacity(n, 0) > table_capacity(n, 1) ? table_capacity(n, 0) : table_capacity(n, 1);
}

// Host-side launchers (defined in cafs_pipeline.cu and cafs_batch.cu).
cudaError_t launch_pipeline(const Params& p, int dtype, int grid, cudaStream_t s);
cudaError_t launch_small(const Params& p, int dtype, cudaStream_t s);
cudaError_t pipeline_occupancy(int dtype, int* blocks_per_sm);
cudaError_t prepare_kernels();
cudaError_t launch_fill_u64(unsigned long long* ptr, unsigned long long n, unsigned long long v,
                            cudaStream_t s);
cudaError_t prepare_batch_kernel();
cudaError_t batch_occupancy(int* blocks_per_sm);
cudaError_t launch_batch(const BatchParams& bp, int dtype, int grid, cudaStream_t s);

// Shared by the host entry points (defined in cafs_api.cu).
void count_launches(unsigned k);
// The hash multipliers of the next call: both 0 (the golden-ratio constants)
// unless a seed was set (cafs_set_hash_seed), then odd values drawn from the
// seed and a per-process call counter.
void next_hash_multipliers(unsigned long long* hash_mult, unsigned* local_mult);
unsigned long long wait_timeout_ns();
cafs_status check_args(const void* keys, size_t n, cafs_dtype dtype, const void* out, bool need_out);
void fill_report(const Record& r, cafs_report* rep);

}  // namespace cafs
