// The phases of the CAFS count-and-emit frequency sort on one GB300 (sm_103a),
// shared by the single-column kernels and the batched kernel.
//
// For one column of N >= 2048 keys the CTAs of a scope (the whole cooperative
// grid, or one CTA) run the pipeline of Sec. 4.1; phases are separated by a
// bounded grid barrier:
//
//   0  sampler + Chao1 + dispatcher record (Alg. 2, Eq. 5, Eq. 6, Alg. 3):
//      the CTAs gather the 1024 strided samples together, then every CTA
//      computes the same estimate and dispatch decision itself
//   1  IsMonotone full scan, only when the 1024 samples ascend (Alg. 3);
//      a sorted column is copied through (bypass)
//   2  count: every CTA streams its share of the column through a shared
//      memory ring filled by bulk copies (cp.async.bulk + mbarrier) and counts
//      it against the <= 8 sampled keys (tiny path, Sec. 4.4) or in a per-CTA
//      table (main path, Sec. 4.2: a direct table of the sampled keys, linear
//      probing over 16-byte buckets, or two-choice buckets) that is merged
//      into a global table hashed with Eq. 4; above what a CTA's table holds,
//      every key goes to the global table, runs of equal keys folded first
//      (Sec. 4.4).  The global table counts distinct keys; the branch is the
//      overflow branch when they exceed L = C/2 (Eq. 6, Alg. 4)
//   3  the K' (key, count) pairs are put in key order and their counts
//      exclusive-scanned (Alg. 4): for K' <= 4096 every CTA computes, for its
//      share of the pairs, the rank and the run offset directly (number of
//      smaller keys and the sum of their counts); larger K' go through a
//      splitter bucket sort (one key range per CTA, sorted in shared memory)
//   4  emit: every output tile looks up its runs and writes them with 16-byte
//      streaming stores (the paper's fill_n per pair)
//   R  radix fallback (the paper's pdqsort: 2*K_hat > N, or the guard fired):
//      LSD radix sort, 8-bit digits; per pass a reduce-then-scan over per-CTA
//      digit counts (pass 0's count read also finds the key bits that vary,
//      so passes whose digit is constant are skipped) and an in-order stable
//      scatter.
//
// Columns with N < 2048 are sorted by a single CTA in shared memory
// (Table 2: "sampling does not amortize").
//
// All device waits (grid barrier, mbarriers) are bounded by a
// timeout; a wait that runs out records kDevTimeout and the launch ends early
// after draining its own bulk copies.

#pragma once

#include <type_traits>

#include "cafs_device.cuh"
#include "cafs_internal.h"

namespace cafs {

// ---------------------------------------------------------------------------
// Phase 0: sampler, spectrum, Chao1, Eq. 6, provisional dispatch (one CTA).
// ---------------------------------------------------------------------------
// The strided samples of Alg. 2 that fall in part `part` of `nparts`: part b
// loads samples [1024 b / nparts, 1024 (b + 1) / nparts), which lie in its own
// share of the column, into `buf` (global).
template <typename K>
__device__ __forceinline__ void gather_samples(const Params& p, const K* keys, long long* buf,
                                               unsigned part, unsigned nparts) {
  const unsigned long long n = p.n;
  const unsigned long long stride = n / kSamples > 0 ? n / kSamples : 1ull;
  const int ns = n < (unsigned long long)kSamples ? (int)n : kSamples;
  const int i0 = (int)((unsigned long long)ns * part / nparts);
  const int i1 = (int)((unsigned long long)ns * (part + 1) / nparts);
  for (int i = i0 + (int)threadIdx.x; i < i1; i += kThreads)
    buf[i] = (long long)keys[(unsigned long long)i * stride];
}

// Every CTA that calls this computes the same record, sample-key list and
// tiny-path multiplier from the same samples, so the grid needs no barrier
// after it: the spectrum does not depend on where the parallel inserts put
// the keys, and the distinct keys are listed in the order of their first
// sample position (the FreqSet's slot order would depend on which of two
// colliding keys was inserted first).  `gathered` (global, may be null)
// holds the samples already; otherwise they are read from the column.
constexpr int kFreqSlots = 4096;
// FreqSet keys, counts and first positions, the samples, each sample's slot,
// the scratch words.
constexpr int kSampleSmem = kFreqSlots * (8 + 4 + 4) + kSamples * (8 + 4) + 256;
static_assert(kSamples == kThreads, "one sample position per thread in the listing scan");
static_assert(kSampleSmem + kRingReserve <= kPipelineSmem - kRingBytes, "sampler below the ring");

template <typename K>
__device__ void phase_sample(const Params& p, const K* keys, unsigned char* smem,
                             const long long* gathered = nullptr) {
  using T = KeyTraits<K>;
  // Algorithm 2's FreqSet: a 4096-slot open-addressing table in shared
  // memory, filled with the 1024 strided samples in parallel.  The empty
  // marker is the type minimum; samples equal to it are counted on the side.
  long long* fkey = reinterpret_cast<long long*>(smem);                 // kFreqSlots
  unsigned* fcnt = reinterpret_cast<unsigned*>(fkey + kFreqSlots);      // kFreqSlots
  int* ffirst = reinterpret_cast<int*>(fcnt + kFreqSlots);              // kFreqSlots: first position
  long long* s = reinterpret_cast<long long*>(ffirst + kFreqSlots);     // kSamples, position order
  int* sslot = reinterpret_cast<int*>(s + kSamples);                    // kSamples: slot of each sample
  int* scratch = sslot + kSamples;                                      // kWarps + 2
  const int t = threadIdx.x;
  const unsigned long long n = p.n;
  const unsigned long long stride = n / kSamples > 0 ? n / kSamples : 1ull;
  const int ns = n < (unsigned long long)kSamples ? (int)n : kSamples;
  const long long kmin = (long long)T::min_key();

  for (int i = t; i < kFreqSlots; i += kThreads) {
    fkey[i] = kmin;
    fcnt[i] = 0u;
    ffirst[i] = INT_MAX;
  }
  if (t == 0) {
    scratch[kWarps] = 0;              // samples equal to the type minimum
    scratch[kWarps + 1] = INT_MAX;    // first position of such a sample
  }
  for (int i = t; i < kSamples; i += kThreads)
    s[i] = i < ns ? (gathered ? __ldcg(gathered + i) : (long long)keys[(unsigned long long)i * stride])
                  : LLONG_MAX;
  __syncthreads();
  int asc = 1;
  for (int i = t; i + 1 < ns; i += kThreads) asc &= (s[i] <= s[i + 1]);
  const int hint = __syncthreads_and(asc);

  // Linear-probe insert (Alg. 2), load <= 1/4.
  for (int i = t; i < ns; i += kThreads) {
    const long long x = s[i];
    if (x == kmin) {
      atomicAdd(scratch + kWarps, 1);
      atomicMin(scratch + kWarps + 1, i);
      sslot[i] = -1;
      continue;
    }
    unsigned slot = (unsigned)hash_slot((unsigned long long)x, 12);
    for (int probe = 0; probe < kFreqSlots; ++probe, slot = (slot + 1) & (kFreqSlots - 1)) {
      const long long k = *reinterpret_cast<volatile long long*>(fkey + slot);
      if (k == x) break;
      if (k == kmin) {
        const long long old = (long long)atomicCAS(reinterpret_cast<unsigned long long*>(fkey + slot),
                                                   (unsigned long long)kmin, (unsigned long long)x);
        if (old == kmin || old == x) break;
      }
    }
    atomicAdd(fcnt + slot, 1u);
    atomicMin(ffirst + slot, i);
    sslot[i] = (int)slot;
  }
  __syncthreads();
  // Spectrum: occupied slots (u), slots seen once (f1) and twice (f2).
  int cu = 0, c1 = 0, c2 = 0;
  for (int i = t; i < kFreqSlots; i += kThreads) {
    const unsigned c = fcnt[i];
    cu += c > 0u;
    c1 += c == 1u;
    c2 += c == 2u;
  }
  const int nmin = scratch[kWarps];
  int u = block_sum(cu, scratch) + (nmin > 0);
  const int f1 = block_sum(c1, scratch) + (nmin == 1);
  const int f2 = block_sum(c2, scratch) + (nmin == 2);

  // The distinct sample values in the order of their first sample position
  // (a block scan over the positions, one per thread): all of them go to
  // the workspace (they seed the count tables), and when u <= 8 also to the
  // record (tiny path).
  Record& r = p.ctrl->rec;
  long long* tiny_list = reinterpret_cast<long long*>(fkey);   // reuses the FreqSet keys
  {
    const int i = t;   // kSamples == kThreads
    bool first = false;
    if (i < ns) first = sslot[i] < 0 ? scratch[kWarps + 1] == i : ffirst[sslot[i]] == i;
    int tot_unused;
    const int idx = block_exclusive_scan(first ? 1 : 0, scratch, &tot_unused);   // barrier first
    if (first) {
      const long long v = s[i];
      if (p.sample_keys) p.sample_keys[idx] = v;
      if (u <= kTinyMax) {
        r.tiny_keys[idx] = v;
        tiny_list[idx] = v;
      }
    }
  }
  // Tiny path: find an odd multiplier that sends the u <= 8 sampled keys to
  // distinct buckets (Eq. 4's multiplicative hash with other multipliers).
  __syncthreads();
  if (u <= kTinyMax && t < 32) {
    unsigned long long tkv[kTinyMax];
    #pragma unroll
    for (int j = 0; j < kTinyMax; ++j)
      tkv[j] = j < u ? (unsigned long long)(typename T::U)(K)tiny_list[j] : 0ull;
    bool found = false;
    for (int round = 0; round < 16 && !found; ++round) {
      const unsigned long long m = (kPhi * (2ull * (unsigned long long)(round * 32 + t) + 1ull)) | 1ull;
      unsigned mask = 0;
      bool ok = true;
      #pragma unroll
      for (int j = 0; j < kTinyMax; ++j) {
        if (j < u) {
          const unsigned b = (unsigned)((tkv[j] * m) >> (64 - kTinyBucketBits));
          ok = ok && !((mask >> b) & 1u);
          mask |= 1u << b;
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, ok);
      if (bal) {
        if (t == __ffs(bal) - 1) {
          r.tiny_mult = m;
          r.tiny_hash_ok = 1;
        }
        found = true;
      }
    }
  }
  if (t == 0) {
    const bool saturated = (u == kSamples);
    const unsigned long long k_hat =
        saturated ? n : (unsigned long long)u + ((unsigned long long)f1 * f1) / (2ull * (f2 + 1));
    const unsigned long long cap = T::kCap;
    unsigned long long m = bit_ceil_u64((8ull * k_hat) / cap);
    if (m < 8) m = 8;
    const unsigned long long upper = bit_ceil_u64((n + cap - 1) / cap);
    if (m > upper) m = upper;
    r.n = n;
    r.stride = stride;
    r.n_samples = ns;
    r.u = u;
    r.f1 = f1;
    r.f2 = f2;
    r.k_hat = k_hat;
    r.saturated = saturated;
    r.M = m;
    r.C = m * cap;
    r.L = (m * cap) / 2;
    r.sample_nondecreasing = hint;
    r.n_tiny = u <= kTinyMax ? u : 0;
    int d;
    if (k_hat <= (unsigned long long)kTinyMax && u <= kTinyMax) d = 3;   // TINY
    else if (2ull * k_hat > n) d = 5;                                   // HIGH_ENTROPY
    else d = 4;                                                         // MAIN
    r.dispatch = d;
    r.path = d;
  }
  __syncthreads();
}

// Which CTAs work on the current column (a compile-time policy of every
// phase): GridScope = all CTAs of the cooperative launch, phases separated
// by the bounded grid barrier; CtaScope = this CTA alone (the batched form's
// per-column work items), phases separated by __syncthreads.
struct GridScope {
  __device__ __forceinline__ unsigned part() const { return blockIdx.x; }
  __device__ __forceinline__ unsigned nparts() const { return gridDim.x; }
  __device__ __forceinline__ unsigned long long gthread() const {
    return (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  }
  __device__ __forceinline__ unsigned long long gthreads() const {
    return (unsigned long long)gridDim.x * blockDim.x;
  }
  __device__ __forceinline__ bool lead() const { return blockIdx.x == 0 && threadIdx.x == 0; }
  __device__ __forceinline__ bool sync(Ctrl* c, unsigned& epoch, unsigned long long timeout_ns) const {
    return grid_sync(c, epoch, timeout_ns);
  }
};

struct CtaScope {
  __device__ __forceinline__ unsigned part() const { return 0u; }
  __device__ __forceinline__ unsigned nparts() const { return 1u; }
  __device__ __forceinline__ unsigned long long gthread() const { return threadIdx.x; }
  __device__ __forceinline__ unsigned long long gthreads() const { return blockDim.x; }
  __device__ __forceinline__ bool lead() const { return threadIdx.x == 0; }
  __device__ __forceinline__ bool sync(Ctrl* c, unsigned&, unsigned long long) const {
    __syncthreads();
    const bool ok = !device_failed(c);
    __syncthreads();
    return ok;
  }
};

// Geometry of one CTA's share of a column: `head` scalar elements before the
// first 16-byte boundary, then whole 16-byte vectors [v0, v1) of this CTA,
// then the ragged tail [tail0, n) handled by the last CTA.
template <typename K>
struct Share {
  unsigned long long head, nvec, tail0, v0, v1;
  template <class S>
  __device__ Share(const K* keys, unsigned long long n, const S& sc) {
    constexpr int VPE = KeyTraits<K>::kVec;
    const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
    head = ((16u - (addr & 15u)) & 15u) / sizeof(K);
    if (head > n) head = n;
    nvec = (n - head) / VPE;
    tail0 = head + nvec * VPE;
    const unsigned nb = sc.nparts(), b = sc.part();
    v0 = nvec * b / nb;
    v1 = nvec * (b + 1) / nb;
  }
};

// ---------------------------------------------------------------------------
// The bulk-copy ring: this CTA's vectors of the column stream through
// kRingStages chunks of shared memory.  Warp kConsumerWarps (the last) issues
// cp.async.bulk copies, warps 0..kConsumerWarps-1 consume.  start() issues the
// first kRingStages chunks (at launch, before the sampler's grid barrier);
// run() streams the whole share through a counting functor; drain() waits for
// copies that will not be consumed.  Every wait is bounded.
// ---------------------------------------------------------------------------
template <typename K>
struct Ring {
  unsigned char* buf;           // kRingBytes
  unsigned long long* full;     // kRingStages
  unsigned long long* empty;    // kRingStages
  unsigned* skip_flag;          // shared copy of the caller's skip flag
  const unsigned char* src;     // first byte of this CTA's vector range
  unsigned long long total;     // bytes of this CTA's vector range
  unsigned long long nchunks;
  unsigned long long issued;    // producer lane only
  bool live;

  __device__ __forceinline__ bool producer() const {
    return threadIdx.x == kConsumerWarps * 32;
  }

  template <class S>
  __device__ void start(const Params& p, const K* keys, unsigned char* smem, const S& sc) {
    const Share<K> sh(keys, p.n, sc);
    buf = smem + (kPipelineSmem - kRingBytes);
    full = reinterpret_cast<unsigned long long*>(buf - kRingReserve);
    empty = full + kRingStages;
    skip_flag = reinterpret_cast<unsigned*>(empty + kRingStages);
    src = reinterpret_cast<const unsigned char*>(keys + sh.head) + sh.v0 * 16ull;
    total = (sh.v1 - sh.v0) * 16ull;
    nchunks = (total + kChunkBytes - 1) / kChunkBytes;
    issued = 0;
    live = true;
    if (threadIdx.x == 0) {
      for (int s = 0; s < kRingStages; ++s) {
        mbar_init(full + s, 1);
        mbar_init(empty + s, kConsumerWarps);
      }
      fence_mbar_init();
      *skip_flag = 0u;
    }
    // The ring's bytes may hold an earlier phase's (or column's) generic
    // stores: every thread fences them against the coming bulk copies.
    fence_proxy_async_smem();
    __syncthreads();
    if (producer())
      while (issued < nchunks && issued < (unsigned long long)kRingStages) issue(issued++);
  }

  __device__ __forceinline__ unsigned bytes_of(unsigned long long ch) const {
    const unsigned long long off = ch * (unsigned long long)kChunkBytes;
    return (unsigned)((total - off) < (unsigned long long)kChunkBytes ? (total - off) : kChunkBytes);
  }

  __device__ __forceinline__ void issue(unsigned long long ch) {
    const int s = (int)(ch % kRingStages);
    const unsigned bytes = bytes_of(ch);
    mbar_arrive_expect_tx(full + s, bytes);
    bulk_g2s(buf + (size_t)s * kChunkBytes, src + ch * (unsigned long long)kChunkBytes, bytes, full + s);
  }

  // Waits for the copies that may still be in flight (the last kRingStages
  // issued chunks; every earlier chunk was consumed before its stage was
  // reused), then retires the barriers.
  __device__ void drain(const Params& p) {
    if (!live) return;
    if (producer()) {
      const unsigned long long first = issued > (unsigned long long)kRingStages ? issued - kRingStages : 0ull;
      for (unsigned long long ch = first; ch < issued; ++ch)
        mbar_wait(full + (ch % kRingStages), (unsigned)(ch / kRingStages) & 1u, p.timeout_ns, p.ctrl);
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int s = 0; s < kRingStages; ++s) {
        mbar_inval(full + s);
        mbar_inval(empty + s);
      }
    __syncthreads();
    live = false;
  }

  // Streams the whole share; consumers call f.chunk() on each chunk and
  // f.single() on the scalar head/tail elements.  When `*skip` becomes
  // non-zero the consumers stop counting (the stream still runs to its end).
  template <typename F, class S>
  __device__ bool run(const Params& p, const K* keys, const unsigned* skip, F& f, const S& sc) {
    using T = KeyTraits<K>;
    constexpr int kConsumers = kConsumerWarps * 32;
    Ctrl* c = p.ctrl;
    const unsigned long long n = p.n;
    const Share<K> sh(keys, n, sc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool consumer = warp < kConsumerWarps;
    const int ctid = threadIdx.x;
    if (consumer) {
      if (sc.part() == 0)
        for (unsigned long long i = ctid; i < sh.head; i += kConsumers) f.single(keys[i]);
      if (sc.part() == sc.nparts() - 1)
        for (unsigned long long i = sh.tail0 + ctid; i < n; i += kConsumers) f.single(keys[i]);
    }
    bool ok = true;
    if (!consumer) {
      if (producer()) {
        // The producer mirrors the (global) skip flag into shared memory,
        // one chunk late: its L2 read overlaps the wait for a free stage,
        // and the consumers only read shared memory (a global read per
        // chunk and warp cost 13 us of a 70 us count phase).
        unsigned fl = skip ? ld_relaxed_u32(skip) : 0u;
        for (; issued < nchunks; ++issued) {
          const int s = (int)(issued % kRingStages);
          const unsigned k = (unsigned)(issued / kRingStages);
          if (!mbar_wait(empty + s, (k - 1) & 1u, p.timeout_ns, c)) { ok = false; break; }
          if (skip) {
            // set only: a consumer may have raised it already
            if (fl) *reinterpret_cast<volatile unsigned*>(skip_flag) = 1u;
            fl = ld_relaxed_u32(skip);
          }
          issue(issued);
        }
      }
    } else {
      for (unsigned long long ch = 0; ch < nchunks; ++ch) {
        const int s = (int)(ch % kRingStages);
        const unsigned k = (unsigned)(ch / kRingStages);
        if (!mbar_wait(full + s, k & 1u, p.timeout_ns, c)) { ok = false; break; }
        const unsigned sk = __shfl_sync(0xffffffffu, *reinterpret_cast<volatile unsigned*>(skip_flag), 0);
        if (!sk) {
          const unsigned nv = bytes_of(ch) / 16u;
          const typename T::Vec* cv = reinterpret_cast<const typename T::Vec*>(buf + (size_t)s * kChunkBytes);
          f.template chunk<kVecsPerThread, kConsumers>(
              cv + ctid, nv > (unsigned)ctid ? (nv - ctid + kConsumers - 1) / kConsumers : 0u);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + s);
      }
    }
    drain(p);
    return ok && !device_failed(c);
  }
};

// ---------------------------------------------------------------------------
// Phase 1: IsMonotone (Alg. 3) over the whole column; early exit on the
// first descent found by any thread.
// ---------------------------------------------------------------------------
template <typename K, class S>
__device__ void phase_monotone(const Params& p, const K* keys, const S& sc) {
  Ctrl* c = p.ctrl;
  const unsigned long long n = p.n;
  const unsigned long long G = sc.gthreads();
  const unsigned long long gt = sc.gthread();
  unsigned iter = 0;
  for (unsigned long long i = gt; i + 1 < n; i += G) {
    if (((++iter) & 15u) == 0 && ld_relaxed_u32(&c->inversion)) break;
    if (keys[i] > keys[i + 1]) {
      atomicExch(&c->inversion, 1u);
      break;
    }
  }
}

// Grid-stride copy src -> dst (both n elements of K).
template <typename K, class S>
__device__ void grid_copy(const K* src, K* dst, unsigned long long n, const S& sc) {
  using T = KeyTraits<K>;
  using V = typename T::Vec;
  const unsigned long long G = sc.gthreads();
  const unsigned long long gt = sc.gthread();
  const uintptr_t as = reinterpret_cast<uintptr_t>(src), ad = reinterpret_cast<uintptr_t>(dst);
  if (((as ^ ad) & 15u) == 0) {
    unsigned long long head = ((16u - (ad & 15u)) & 15u) / sizeof(K);
    if (head > n) head = n;
    const unsigned long long nvec = (n - head) / T::kVec;
    const V* vs = reinterpret_cast<const V*>(src + head);
    V* vd = reinterpret_cast<V*>(dst + head);
    for (unsigned long long i = gt; i < nvec; i += G) __stcs(vd + i, __ldcg(vs + i));
    for (unsigned long long i = gt; i < head; i += G) dst[i] = src[i];
    for (unsigned long long i = head + nvec * T::kVec + gt; i < n; i += G) dst[i] = src[i];
  } else {
    for (unsigned long long i = gt; i < n; i += G) dst[i] = __ldcg(src + i);
  }
}

// ---------------------------------------------------------------------------
// Global table insert (Eq. 4 hash, linear probing).  Every successful claim
// of an empty slot increments the occupancy counter and records the slot; the
// guard fires once more than L slots are claimed or the table is full.
// ---------------------------------------------------------------------------
struct GlobalTable {
  unsigned long long* keys;
  unsigned* counts;
  unsigned* claimed;
  Ctrl* ctrl;
  unsigned long long C;     // Eq. 6's slots
  unsigned long long cap;   // slots the workspace's table holds (>= C)
  int logC;
  unsigned long long mult;   // Eq. 4 multiplier (odd)
  // The CTA's shared copy of the guard (null: none).  Once the guard has
  // fired the inserts stop at a shared-memory read: every thread of every
  // CTA probing a small, full table in L2 (the overflow case) queues on the
  // same few lines, hundreds of microseconds for one column.
  unsigned* stop;
};

__device__ __forceinline__ GlobalTable global_table(const Params& p) {
  GlobalTable g;
  g.keys = p.tkeys;
  g.counts = p.tcounts;
  g.claimed = p.claimed;
  g.ctrl = p.ctrl;
  g.C = p.ctrl->rec.C;
  g.cap = p.table_cap;
  g.logC = log2_pow2(g.C);
  g.mult = p.hash_mult ? (p.hash_mult | 1ull) : kPhi;
  g.stop = nullptr;
  return g;
}

// Slots of the global table in use.  Tables of Eq. 6 up to kSlackMaxC slots
// belong to columns counted in shared tables (K_hat within one CTA's table,
// whose C is at most 65536 slots for either key width); they use up to
// kGuardSlack times C slots, within the workspace's table, and the count goes
// on until half of those are claimed.  Alg. 4's guard (distinct keys >
// L = C/2) still decides the branch, but when the count completes below the
// larger limit its counts are emitted instead of running the radix fallback
// on the whole column (Chao1 underestimates K on skewed data by a few times:
// the Zipf(1.1) columns of K = 1e4 .. 1.3e5 at N = 3e7 hold 1.2 to 7.9 times
// L distinct keys).  Such a global table only holds the keys the shared
// tables flush or spill, so its size does not slow the count.  Larger Eq. 6
// tables belong to columns counted in the global table alone, where the
// table is the hot structure and keeps its Eq. 6 size.  Every insert of a
// call computes the same size from the same (C, cap).
constexpr unsigned long long kGuardSlack = 8;
constexpr unsigned long long kSlackMaxC = 65536;

__device__ __forceinline__ int table_log2(unsigned long long C, unsigned long long cap, int logC) {
  if (C > kSlackMaxC) return logC;
  const unsigned long long big = C * kGuardSlack;
  return log2_pow2(big < cap ? big : (cap > C ? cap : C));
}

// Counter increment without a returned value: a reduction that L2 applies
// on its own, no response back to the SM.
__device__ __forceinline__ void red_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

static __device__ __noinline__ void global_insert(GlobalTable g, unsigned long long key64, unsigned inc) {
  Ctrl* c = g.ctrl;
  const int lg = table_log2(g.C, g.cap, g.logC);
  const unsigned long long size = 1ull << lg;
  const unsigned long long limit = size / 2;
  const unsigned long long mask = size - 1;
  const unsigned long long h = hash_slot_m(key64, g.mult, lg);
  for (unsigned long long probe = 0; probe < size; ++probe) {
    // Once the guard has fired the counts are discarded: stop probing.
    if (g.stop && *reinterpret_cast<volatile unsigned*>(g.stop)) return;
    if ((probe & 3ull) == 3ull && ld_relaxed_u32(&c->overflow)) {
      if (g.stop) *reinterpret_cast<volatile unsigned*>(g.stop) = 1u;
      return;
    }
    const unsigned long long slot = (h + probe) & mask;
    const unsigned long long k = ld_relaxed_u64(g.keys + slot);
    if (k == key64) {
      red_add_u32(g.counts + slot, inc);
      return;
    }
    if (k == kEmpty64) {
      const unsigned long long old = atomicCAS(g.keys + slot, kEmpty64, key64);
      if (old == kEmpty64) {
        // The lanes of the warp that claim a slot together take their
        // occupancy indices with one atomic: every claim of every CTA goes
        // to this one counter, whose atomics the L2 serialises.
        const unsigned grp = __activemask();
        const int lead = __ffs(grp) - 1;
        unsigned first = 0;
        if ((int)(threadIdx.x & 31u) == lead) first = atomicAdd(&c->occupancy, (unsigned)__popc(grp));
        const unsigned idx = __shfl_sync(grp, first, lead) + (unsigned)__popc(grp & lanemask_lt());
        if (idx < size) g.claimed[idx] = (unsigned)slot;
        red_add_u32(g.counts + slot, inc);
        if (idx >= limit) {
          if (!ld_relaxed_u32(&c->overflow)) atomicExch(&c->overflow, 1u);
          if (g.stop) *reinterpret_cast<volatile unsigned*>(g.stop) = 1u;
        }
        return;
      }
      if (old == key64) {
        red_add_u32(g.counts + slot, inc);
        return;
      }
    }
  }
  atomicExch(&c->overflow, 1u);
  if (g.stop) *reinterpret_cast<volatile unsigned*>(g.stop) = 1u;
}

// ---------------------------------------------------------------------------
// Phase 2: count (tiny or main).
// ---------------------------------------------------------------------------

// The CTA's shared counting table: NB buckets of kBucketSlots keys (one
// 16-byte shared-memory load reads a bucket: 4 int32 or 2 int64 keys, the
// GPU form of Sec. 4.2's one-line bucket), each slot with R counter replicas
// (lane % R) so that lanes of a warp hitting the same key do not serialise.
// A key lives in one of two buckets, chosen by two multiplicative hashes of
// its 32-bit fold: the lookup reads both with two independent loads, so that
// every key costs the same (a probe sequence of data-dependent length makes
// the whole warp wait for its longest one; measured 50 us for a column of
// 3e7 keys in a table with every key in its first slot, 73-120 us with
// linear probing).  Passed by value to the non-inlined slow path so that the
// hot loop stays small.
template <typename K>
constexpr int bucket_slots() { return 16 / (int)sizeof(K); }

template <typename K>
struct LocalTable {
  static constexpr int kBucketSlots = bucket_slots<K>();
  K* keys;          // NB * kBucketSlots, bucket-major; nullptr: no shared table
  unsigned* cnt;    // NB * kBucketSlots * R
  unsigned* occ;    // distinct keys held
  unsigned limit;   // at most this many distinct keys (half the slots)
  int logNB, NB, R, lane_rep;
  unsigned mult;    // first bucket hash multiplier (odd); the second is derived
  int two;          // 1: two-choice buckets; 0: linear probing over buckets
  GlobalTable gt;

  __device__ __forceinline__ unsigned first(unsigned x32) const {
    return local_bucket_m(x32, mult, logNB);
  }
  __device__ __forceinline__ unsigned second(unsigned x32) const {
    return local_bucket_m(x32, (mult * 0xA3B195A5u) | 1u, logNB);
  }
  __device__ __forceinline__ void add(unsigned slot) const {
    atomicAdd(cnt + slot * R + lane_rep, 1u);
  }
};

// Reads the keys of one bucket with a single 16-byte load.
__device__ __forceinline__ void load_bucket(const long long* kb, long long* k) {
  const longlong2 a = *reinterpret_cast<const longlong2*>(kb);
  k[0] = a.x; k[1] = a.y;
}
__device__ __forceinline__ void load_bucket(const int* kb, int* k) {
  const int4 a = *reinterpret_cast<const int4*>(kb);
  k[0] = a.x; k[1] = a.y; k[2] = a.z; k[3] = a.w;
}

// Slow path of one key (not the type minimum) that was not found by the
// fast lookup: scan its buckets in a fixed order (two-choice: its first
// bucket, then its second; otherwise linear probing over buckets from the
// first) and claim the first empty slot while the table holds fewer than
// `limit` distinct keys; otherwise (or when its buckets are full) count it in
// the global table.  Slots are never emptied and always tried in the same
// order, so a key occupies at most one slot: a later scan of it passes the
// same occupied slots and meets it before any empty one.  `inc` is 0 when
// the table is being seeded with the sampled keys.
template <typename K>
__device__ __forceinline__ void slow_insert(K x, const LocalTable<K>& t, unsigned inc) {
  using T = KeyTraits<K>;
  constexpr int kBucketSlots = LocalTable<K>::kBucketSlots;
  const K kmin = T::min_key();
  if (t.keys) {
    const unsigned x32 = fold32((typename T::U)x);
    const unsigned b1 = t.first(x32), b2 = t.second(x32);
    const int nprobe = t.two ? 2 : t.NB;
    for (int c = 0; c < nprobe; ++c) {
      const unsigned b = t.two ? (c ? b2 : b1) : ((b1 + (unsigned)c) & (unsigned)(t.NB - 1));
      for (int j = 0; j < kBucketSlots; ++j) {
        K* slotp = t.keys + b * kBucketSlots + j;
        const K k = *reinterpret_cast<volatile K*>(slotp);
        if (k == x) {
          if (inc) t.add(b * kBucketSlots + j);
          return;
        }
        if (k == kmin) {
          if (*reinterpret_cast<volatile unsigned*>(t.occ) >= t.limit) {
            if (inc) global_insert(t.gt, (unsigned long long)(long long)x, inc);
            return;
          }
          K old;
          if constexpr (sizeof(K) == 8) {
            old = (K)atomicCAS(reinterpret_cast<unsigned long long*>(slotp),
                               (unsigned long long)kmin, (unsigned long long)x);
          } else {
            old = (K)atomicCAS(reinterpret_cast<unsigned*>(slotp), (unsigned)kmin, (unsigned)x);
          }
          if (old == kmin) atomicAdd(t.occ, 1u);
          if (old == kmin || old == x) {
            if (inc) t.add(b * kBucketSlots + j);
            return;
          }
          // another key took the slot: carry on with the next one
        }
      }
    }
  }
  if (inc) global_insert(t.gt, (unsigned long long)(long long)x, inc);
}

// Per-key counting of one thread.  TINY: the <= 8 sampled keys are looked
// up through a collision-free multiplicative hash into kTinyBuckets buckets
// and counted in this thread's own shared-memory counters (Sec. 4.4, the
// paper's eight branchless counters).  Main path (and tiny misses): read the
// key's home bucket and add to the matching slot's counter (Sec. 4.2's bucket
// update).  Keys that miss are handled afterwards in one loop per chunk, so
// that a warp's misses at different positions share one pass of the slow
// path.  Keys equal to the type minimum (the tables' empty marker) are only
// counted.
// Direct table of the main path when the sample holds few distinct keys
// (u <= kDirectMaxKeys): a multiplier that sends every sampled key to its
// own slot of kDirectSlots is searched for, and a slot holds the key's index
// in a dense list (kDirectMaxKeys means none; that entry holds the type
// minimum, which no looked-up key equals).  A lookup is one byte load, one
// key compare and one counter atomic on a lane-private replica (the bank is
// the lane); keys outside the sample fall through to the bucket table.
constexpr int kDirectSlotBits = 14;
constexpr int kDirectSlots = 1 << kDirectSlotBits;
constexpr int kDirectMaxKeys = 255;
constexpr int kDirectBytes = kDirectSlots + 256 * 8 + 256 * 32 * 4;   // index, keys, counters

template <typename K, bool TINY>
struct KeyCounter {
  using T = KeyTraits<K>;
  LocalTable<K> lt;
  // direct table (main path; dslot == nullptr: none)
  const unsigned char* dslot;
  const K* dkey;
  unsigned* dcnt;
  unsigned dmult;
  int lane;
  // tiny path
  unsigned long long tmult;
  unsigned tvalid;
  const K* tkey;        // kTinyBuckets keys by bucket
  unsigned* tcnt;       // this thread's counters, stride kConsumerWarps*32
  unsigned long long special;

  // Fast path; returns false when the key must take the slow path.
  __device__ __forceinline__ bool fast(K x) {
    if constexpr (TINY) {
      const unsigned long long ux = (unsigned long long)(typename T::U)x;
      const unsigned b = (unsigned)((ux * tmult) >> (64 - kTinyBucketBits));
      if (((tvalid >> b) & 1u) && tkey[b] == x) {
        tcnt[b * (kConsumerWarps * 32)] += 1u;
        return true;
      }
    }
    if (x == T::min_key()) {
      ++special;
      return true;
    }
    if (!TINY && dslot) {
      const unsigned i = dslot[local_bucket_m(fold32((typename T::U)x), dmult, kDirectSlotBits)];
      if (dkey[i] == x) {
        atomicAdd(dcnt + i * 32u + (unsigned)lane, 1u);
        return true;
      }
    }
    if (!TINY && !lt.two) {
      // Linear probing over buckets (load <= 1/4): a key sits in the first
      // bucket from its home on that had a free slot when it came, so a
      // bucket whose last slot is free ends the search; up to kFastBuckets
      // buckets here, the rest in the slow path.
      constexpr int kBucketSlots = LocalTable<K>::kBucketSlots;
      constexpr int kFastBuckets = 3;
      unsigned b = lt.first(fold32((typename T::U)x));
      #pragma unroll
      for (int probe = 0; probe < kFastBuckets; ++probe) {
        K k[kBucketSlots];
        load_bucket(lt.keys + b * kBucketSlots, k);
        int hit = -1;
        #pragma unroll
        for (int j = kBucketSlots - 1; j >= 0; --j)
          if (k[j] == x) hit = j;
        if (hit >= 0) {
          lt.add(b * kBucketSlots + hit);
          return true;
        }
        if (k[kBucketSlots - 1] == T::min_key()) break;
        b = (b + 1) & (unsigned)(lt.NB - 1);
      }
      return false;
    }
    if (!TINY) {
      // Two-choice buckets (load up to 1/2): both candidate buckets with two
      // independent 16-byte loads; a key found in either is counted.
      constexpr int kBucketSlots = LocalTable<K>::kBucketSlots;
      const unsigned x32 = fold32((typename T::U)x);
      const unsigned b1 = lt.first(x32), b2 = lt.second(x32);
      K k1[kBucketSlots], k2[kBucketSlots];
      load_bucket(lt.keys + b1 * kBucketSlots, k1);
      load_bucket(lt.keys + b2 * kBucketSlots, k2);
      int hit = -1;
      #pragma unroll
      for (int j = kBucketSlots - 1; j >= 0; --j) {
        if (k2[j] == x) hit = (int)(b2 * kBucketSlots) + j;
      }
      #pragma unroll
      for (int j = kBucketSlots - 1; j >= 0; --j) {
        if (k1[j] == x) hit = (int)(b1 * kBucketSlots) + j;
      }
      if (hit >= 0) {
        lt.add((unsigned)hit);
        return true;
      }
    }
    return false;
  }

  __device__ __forceinline__ void single(K x) {
    if (!fast(x)) slow_insert<K>(x, lt, 1u);
  }

  // The 16-byte vectors src[0], src[STRIDE], ..., src[(cnt-1)*STRIDE]
  // (cnt <= NV) of a chunk in shared memory, one vector load each.
  template <int NV, int STRIDE>
  __device__ __forceinline__ void chunk(const typename T::Vec* src, unsigned cnt) {
    constexpr int VPE = T::kVec;
    static_assert(NV * VPE <= 32, "miss mask");
    unsigned miss = 0;
    #pragma unroll
    for (int i = 0; i < NV; ++i) {
      if ((unsigned)i < cnt) {
        K e[VPE];
        unpack(src[i * STRIDE], e);
        #pragma unroll
        for (int q = 0; q < VPE; ++q)
          if (!fast(e[q])) miss |= 1u << (i * VPE + q);
      }
    }
    while (miss) {
      const int i = __ffs(miss) - 1;
      miss &= miss - 1;
      slow_insert<K>(reinterpret_cast<const K*>(src + (i / VPE) * STRIDE)[i % VPE], lt, 1u);
    }
  }
};

// Count phase without a shared table (K_hat above what one CTA's table
// holds; Sec. 4.5's L2-level table): every key is inserted into the global
// Eq. 4 table.  A functor of its own, so that the shared-table counter's
// loop never has to allow for a missing table (measured: 8-12 us less per
// 3e7-key count for K <= 1000).  Streaming the share with plain loads and
// several probes in flight per thread measured slower than this (about 1 ms
// against 0.62-0.71 ms for K = 1e4..1.3e5).
//
// Runs of equal keys (Sec. 4.4's run-length case: grouped input, the output
// of a group-by) are folded before the insert: the lanes of a warp hold
// 32 * VPE consecutive keys, and when any key in that window equals the one
// before it, each run in the window is inserted once with its length, so the
// inserts fall from one per key towards one per run.  A window without such
// a pair (the usual case off grouped input) costs one shuffle and one vote.
// The shared-table counter has no such step: every form of it measured
// slowed its loop by 10-20 % through register pressure.
template <typename K>
struct GlobalCounter {
  using T = KeyTraits<K>;
  GlobalTable g;
  unsigned long long special;

  __device__ __forceinline__ void insert(K x, unsigned inc) {
    if (x == T::min_key()) special += inc;
    else global_insert(g, (unsigned long long)(long long)x, inc);
  }
  __device__ __forceinline__ void single(K x) { insert(x, 1u); }

  // The vectors src[0], src[STRIDE], ... (cnt <= NV of them, fewer only in
  // the higher lanes at the end of a chunk); lane l's vector i follows lane
  // l - 1's in the column.
  template <int NV, int STRIDE>
  __device__ __forceinline__ void chunk(const typename T::Vec* src, unsigned cnt) {
    constexpr int VPE = T::kVec;
    constexpr unsigned kAll = (1u << VPE) - 1u;
    const unsigned lane = threadIdx.x & 31u;
    #pragma unroll
    for (int i = 0; i < NV; ++i) {
      const bool have = (unsigned)i < cnt;
      K e[VPE];
      if (have) {
        unpack(src[i * STRIDE], e);
      } else {
        #pragma unroll
        for (int q = 0; q < VPE; ++q) e[q] = (K)0;
      }
      // hm bit q: the key at position q of this lane starts a run (a lane
      // without a vector counts as a run start: it ends the window).
      const K prev = __shfl_up_sync(0xffffffffu, e[VPE - 1], 1);
      unsigned hm = (lane == 0u || prev != e[0]) ? 1u : 0u;
      #pragma unroll
      for (int q = 1; q < VPE; ++q) hm |= (e[q] != e[q - 1]) ? (1u << q) : 0u;
      if (!have) hm = 1u;
      if (__all_sync(0xffffffffu, hm == kAll || !have)) {
        if (have) {
          #pragma unroll
          for (int q = 0; q < VPE; ++q) insert(e[q], 1u);
        }
        continue;
      }
      // Window position of the first run start after this lane's keys.
      const unsigned starts = __ballot_sync(0xffffffffu, hm != 0u);
      const unsigned later = starts & ~((2u << lane) - 1u);
      const int nl = later ? __ffs(later) - 1 : 32;
      const int nfirst = __shfl_sync(0xffffffffu, __ffs(hm) - 1, nl & 31);
      const unsigned after = nl < 32 ? (unsigned)(nl * VPE + nfirst) : 32u * VPE;
      if (have) {
        #pragma unroll
        for (int q = 0; q < VPE; ++q) {
          if ((hm >> q) & 1u) {
            const unsigned rest = hm >> (q + 1);   // run starts after q in this lane
            const unsigned end = rest ? lane * VPE + q + 1u + (unsigned)(__ffs(rest) - 1) : after;
            insert(e[q], end - (lane * VPE + q));
          }
        }
      }
    }
  }
};

// Adds this CTA's count of type-minimum keys to the control block.
__device__ __forceinline__ void special_out(Ctrl* c, unsigned long long special, unsigned long long* red) {
  const unsigned long long bs = block_sum(special, red);
  if (threadIdx.x == 0 && bs) atomicAdd(&c->special, bs);
}

template <typename K, bool TINY, class SC>
__device__ bool phase_count(const Params& p, const K* keys, unsigned char* smem, Ring<K>& ring,
                            const SC& sc) {
  using T = KeyTraits<K>;
  Ctrl* c = p.ctrl;
  const Record& r = c->rec;
  const unsigned long long k_hat = r.k_hat;
  const K kmin = T::min_key();
  constexpr int kConsumers = kConsumerWarps * 32;

  // Per-CTA shared table: S slots (power of two, load <= 1/4 when K_hat is
  // right) with R privatised counter replicas per slot (lane % R) so that hot
  // keys do not serialise a warp's atomics.
  constexpr int kKeyBytes = sizeof(K);
  int S = 256;   // slots = buckets * slots per bucket; load <= 1/4 when K_hat is right
  const int smax = (int)p.local_slots_max;
  while (S < smax && (unsigned long long)S < 4ull * k_hat) S <<= 1;
  const int budget = S <= 2048 ? kSmallTableBytes : kLocalTableBytes;
  int R = (int)p.replicas_max;
  while (R > 1 && S * (kKeyBytes + 4 * R) > budget) R >>= 1;
  const bool use_local = TINY || (k_hat <= (unsigned long long)smax);

  // Direct table: few sampled keys, all of them in slots of their own.
  // Its multiplier is searched for first (32 warps, one candidate each per
  // round, a 16384-bit occupancy bitmap per warp in the table's bytes).
  const int u_all = (int)r.u;
  unsigned char* dbase = smem;
  unsigned* dflag = reinterpret_cast<unsigned*>(smem + kLocalTableBytes);   // [0] multiplier, [1] kmin position
  int nd = 0;
  unsigned dmult = 0;
  if (!TINY && use_local && u_all <= kDirectMaxKeys && k_hat <= (unsigned long long)kDirectMaxKeys) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    unsigned* bm = reinterpret_cast<unsigned*>(smem) + w * (kDirectSlots / 32);
    static_assert(kWarps * (kDirectSlots / 8) <= kLocalTableBytes, "search bitmaps in the table's bytes");
    if (threadIdx.x == 0) {
      dflag[0] = 0u;
      dflag[1] = 0xFFFFFFFFu;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < u_all; j += blockDim.x)
      if ((K)__ldcg(p.sample_keys + j) == kmin) dflag[1] = (unsigned)j;
    const unsigned base = p.local_mult ? (p.local_mult | 1u) : 0x9E3779B1u;
    for (int round = 0; round < 4; ++round) {
      const unsigned m = (base * (2u * (unsigned)(round * kWarps + w) + 1u)) | 1u;
      for (int i = l; i < kDirectSlots / 32; i += 32) bm[i] = 0u;
      __syncwarp();
      bool coll = false;
      for (int j = l; j < u_all; j += 32) {
        const K kj = (K)__ldcg(p.sample_keys + j);
        if (kj == kmin) continue;
        const unsigned sl = local_bucket_m(fold32((typename T::U)kj), m, kDirectSlotBits);
        const unsigned bit = 1u << (sl & 31u);
        coll |= (atomicOr(bm + (sl >> 5), bit) & bit) != 0u;
      }
      coll = __any_sync(0xffffffffu, coll);
      __syncthreads();
      if (!coll && l == 0) atomicCAS(dflag, 0u, m);   // any collision-free candidate
      __syncthreads();
      if (dflag[0] != 0u) break;
    }
    dmult = dflag[0];
    nd = dmult ? u_all - (dflag[1] != 0xFFFFFFFFu ? 1 : 0) : 0;
    __syncthreads();
  }
  const bool dmode = nd > 0;
  // Two-choice buckets once the table may pass a quarter full.
  const int two_choice = (!TINY && 4ull * k_hat > (unsigned long long)smax) ? 1 : 0;
  unsigned char* dslot = dbase;
  K* dkey = reinterpret_cast<K*>(dbase + kDirectSlots);
  unsigned* dcnt = reinterpret_cast<unsigned*>(dbase + kDirectSlots + 256 * 8);
  if (dmode) {
    // the bucket table behind it: what is left of the budget, for keys
    // outside the sample
    S = 256;
    while (S < 2048 && (unsigned long long)S < 4ull * k_hat) S <<= 1;
    R = (int)p.replicas_max;
    while (R > 1 && S * (kKeyBytes + 4 * R) > kLocalTableBytes - kDirectBytes) R >>= 1;
  }
  static_assert(kDirectBytes + 2048 * (8 + 4) <= kLocalTableBytes, "direct table and bucket table");

  // Shared memory: [direct table] table (| tiny counters) | misc ... barriers | ring (top).
  unsigned char* tbase = smem + (dmode ? kDirectBytes : 0);
  const int table_bytes = (dmode ? kDirectBytes : 0) +
                          (TINY ? kTinyTableBytes + kTinyBuckets * kConsumers * 4
                                : (use_local ? S * (kKeyBytes + 4 * R) : 0));
  K* lkeys = reinterpret_cast<K*>(tbase);
  unsigned* lcnt = reinterpret_cast<unsigned*>(tbase + (size_t)S * kKeyBytes);
  unsigned* tcnt = reinterpret_cast<unsigned*>(tbase + kTinyTableBytes);           // kTinyBuckets x kConsumers
  unsigned char* mbase = smem + table_bytes;
  unsigned* local_occ = reinterpret_cast<unsigned*>(mbase);                       // 1
  unsigned long long* red = reinterpret_cast<unsigned long long*>(mbase + 8);     // kWarps
  K* tkey = reinterpret_cast<K*>(mbase + 8 + 8 * kWarps);                          // kTinyBuckets
  static_assert(kLocalTableBytes + kMiscBytes + kRingReserve <= kPipelineSmem - kRingBytes, "table under ring");
  static_assert(kTinyTableBytes + kTinyBuckets * kConsumerWarps * 32 * 4 + kMiscBytes + kRingReserve <=
                    kPipelineSmem - kRingBytes, "tiny table under ring");

  const int nt = r.n_tiny;
  const bool tiny_hash = TINY && r.tiny_hash_ok;
  const unsigned long long tmult = r.tiny_mult;
  unsigned tvalid = 0;
  if (tiny_hash) {
    for (int j = 0; j < nt; ++j) {
      const K kj = (K)r.tiny_keys[j];
      tvalid |= 1u << (unsigned)(((unsigned long long)(typename T::U)kj * tmult) >> (64 - kTinyBucketBits));
    }
  }
  if (use_local) {
    for (int i = threadIdx.x; i < S; i += blockDim.x) lkeys[i] = kmin;
    for (int i = threadIdx.x; i < S * R; i += blockDim.x) lcnt[i] = 0u;
  }
  if (tiny_hash) {
    for (int i = threadIdx.x; i < kTinyBuckets * kConsumers; i += blockDim.x) tcnt[i] = 0u;
    if (threadIdx.x < nt) {
      const K kj = (K)r.tiny_keys[threadIdx.x];
      tkey[((unsigned long long)(typename T::U)kj * tmult) >> (64 - kTinyBucketBits)] = kj;
    }
  }
  if (threadIdx.x == 0) *local_occ = 0u;
  if (dmode) {
    for (int i = threadIdx.x; i < kDirectSlots; i += blockDim.x) dslot[i] = (unsigned char)kDirectMaxKeys;
    for (int i = threadIdx.x; i < 256 * 32; i += blockDim.x) dcnt[i] = 0u;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) dkey[i] = kmin;
  }
  __syncthreads();
  if (dmode) {
    const unsigned kpos = dflag[1];
    for (int j = threadIdx.x; j < u_all; j += blockDim.x) {
      if ((unsigned)j == kpos) continue;
      const K kj = (K)__ldcg(p.sample_keys + j);
      const int i = j - ((unsigned)j > kpos && kpos != 0xFFFFFFFFu ? 1 : 0);
      dkey[i] = kj;
      dslot[local_bucket_m(fold32((typename T::U)kj), dmult, kDirectSlotBits)] = (unsigned char)i;
    }
  }
  __syncthreads();
  if (!TINY && use_local && !dmode) {
    // Seed with the distinct sampled keys (counts 0), so that the frequent
    // keys are found in their buckets from the first chunk on.
    LocalTable<K> seed;
    seed.keys = lkeys;
    seed.cnt = lcnt;
    seed.occ = local_occ;
    seed.limit = S / 2;
    seed.NB = S / LocalTable<K>::kBucketSlots;
    seed.logNB = log2_pow2(S / LocalTable<K>::kBucketSlots);
    seed.R = R;
    seed.lane_rep = 0;
    seed.mult = p.local_mult ? (p.local_mult | 1u) : 0x9E3779B1u;
    seed.two = two_choice;
    seed.gt = global_table(p);
    const int u = (int)r.u;
    for (int j = threadIdx.x; j < u; j += blockDim.x) {
      const K kj = (K)__ldcg(p.sample_keys + j);
      if (kj != kmin) slow_insert<K>(kj, seed, 0u);
    }
    __syncthreads();
  }

  const bool ok = [&]() {
    LocalTable<K> lt;
    lt.keys = use_local ? lkeys : nullptr;
    lt.cnt = lcnt;
    lt.occ = local_occ;
    lt.limit = S / 2;
    lt.NB = S / LocalTable<K>::kBucketSlots;
    lt.logNB = log2_pow2(S / LocalTable<K>::kBucketSlots);
    lt.R = R;
    lt.lane_rep = (threadIdx.x & 31) & (R - 1);
    lt.mult = p.local_mult ? (p.local_mult | 1u) : 0x9E3779B1u;
    lt.two = two_choice;
    lt.gt = global_table(p);
    lt.gt.stop = ring.skip_flag;
    if (tiny_hash) {
      KeyCounter<K, true> kc;
      kc.lt = lt;
      kc.tmult = tmult;
      kc.tvalid = tvalid;
      kc.tkey = tkey;
      kc.tcnt = tcnt + (threadIdx.x < kConsumers ? threadIdx.x : 0);
      kc.special = 0;
      kc.dslot = nullptr;
      const bool res = ring.run(p, keys, &c->overflow, kc, sc);
      // Tiny buckets: add up the per-thread counters, insert each sampled key.
      for (int j = 0; j < nt; ++j) {
        const K kj = (K)r.tiny_keys[j];
        const unsigned b = (unsigned)(((unsigned long long)(typename T::U)kj * tmult) >> (64 - kTinyBucketBits));
        const unsigned long long v = threadIdx.x < kConsumers ? tcnt[b * kConsumers + threadIdx.x] : 0u;
        const unsigned long long tot = block_sum(v, red);
        if (threadIdx.x == 0 && tot) {
          if (kj == kmin) kc.special += tot;
          else global_insert(lt.gt, (unsigned long long)(long long)kj, (unsigned)tot);
        }
      }
      special_out(c, kc.special, red);
      return res;
    }
    if (!use_local) {
      GlobalCounter<K> gc;
      gc.g = lt.gt;
      gc.special = 0;
      const bool res = ring.run(p, keys, &c->overflow, gc, sc);
      special_out(c, gc.special, red);
      return res;
    }
    KeyCounter<K, false> kc;
    kc.lt = lt;
    kc.special = 0;
    kc.dslot = dmode ? dslot : nullptr;
    kc.dkey = dkey;
    kc.dcnt = dcnt;
    kc.dmult = dmult;
    kc.lane = threadIdx.x & 31;
    const bool res = ring.run(p, keys, &c->overflow, kc, sc);
    special_out(c, kc.special, red);
    return res;
  }();

  if (dmode) {
    GlobalTable g = global_table(p);
    g.stop = ring.skip_flag;
    const int rot = (int)((sc.part() * 37u) % (unsigned)nd);
    for (int i0 = threadIdx.x; i0 < nd; i0 += blockDim.x) {
      const int i = (i0 + rot) % nd;
      unsigned tot = 0;
      #pragma unroll 8
      for (int q = 0; q < 32; ++q) tot += dcnt[i * 32 + ((q + i) & 31)];
      if (tot) global_insert(g, (unsigned long long)(long long)dkey[i], tot);
    }
  }

  // Flush the shared table into the global table.  CTAs hold mostly the
  // same keys in the same local slots; each starts at its own offset so
  // that they do not all add to the same global slot at the same time.
  if (use_local) {
    GlobalTable g = global_table(p);
    g.stop = ring.skip_flag;
    const int rot = (int)((sc.part() * 977u) & (unsigned)(S - 1));
    for (int i0 = threadIdx.x; i0 < S; i0 += blockDim.x) {
      const int i = (i0 + rot) & (S - 1);
      const K k = lkeys[i];
      if (k != kmin) {
        unsigned tot = 0;
        for (int q = 0; q < R; ++q) tot += lcnt[i * R + q];
        if (tot) global_insert(g, (unsigned long long)(long long)k, tot);
      }
    }
  }
  return ok;
}

// Reset the global-table slots claimed in this call: this CTA's share.
template <class S>
__device__ void reset_claimed(const Params& p, unsigned occ, const S& sc) {
  const unsigned b = sc.part(), nb = sc.nparts();
  const unsigned i0 = (unsigned)((unsigned long long)occ * b / nb);
  const unsigned i1 = (unsigned)((unsigned long long)occ * (b + 1) / nb);
  for (unsigned i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const unsigned slot = __ldcg(p.claimed + i);
    p.tkeys[slot] = kEmpty64;
    p.tcounts[slot] = 0u;
  }
}

// ---------------------------------------------------------------------------
// Phase 3a (K' <= kRankPairs): rank and run offset of every pair, all CTAs.
// Keys in the table are distinct, so pair i goes to position
//   rank_i = #{j : key_j < key_i}   (+1 when the type minimum occurs)
// and its run starts at
//   off_i = sum of count_j over key_j < key_i   (+ count of the minimum).
// This is the sorted order and the exclusive scan of Alg. 4 in one pass.
// CTA b takes pairs [b*K'/G, (b+1)*K'/G); a warp per pair, lanes over j.
// ---------------------------------------------------------------------------
template <typename K, class S>
__device__ void phase_rank_pairs(const Params& p, unsigned occ, unsigned long long special,
                                 unsigned char* smem, const S& sc) {
  using T = KeyTraits<K>;
  const unsigned b = sc.part(), nb = sc.nparts();
  const unsigned i0 = (unsigned)((unsigned long long)occ * b / nb);
  const unsigned i1 = (unsigned)((unsigned long long)occ * (b + 1) / nb);
  K* skeys = reinterpret_cast<K*>(p.skeys);
  const unsigned long long add = special ? 1ull : 0ull;
  if (b == 0 && threadIdx.x == 0) {
    if (special) {
      skeys[0] = T::min_key();
      p.offsets[0] = 0u;
    }
    p.offsets[occ + add] = (unsigned)p.n;
  }
  if (i1 <= i0) return;
  long long* jk = reinterpret_cast<long long*>(smem);
  unsigned* jc = reinterpret_cast<unsigned*>(jk + kRankPairs);
  for (unsigned j = threadIdx.x; j < occ; j += blockDim.x) {
    const unsigned slot = __ldcg(p.claimed + j);
    jk[j] = (long long)__ldcg(p.tkeys + slot);
    jc[j] = __ldcg(p.tcounts + slot);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (unsigned i = i0 + warp; i < i1; i += kWarps) {
    const long long ki = jk[i];
    unsigned rk = 0;
    unsigned long long off = 0;
    #pragma unroll 4
    for (unsigned j = lane; j < occ; j += 32) {
      const bool lt = jk[j] < ki;
      rk += lt ? 1u : 0u;
      off += lt ? jc[j] : 0u;
    }
    rk = __reduce_add_sync(0xffffffffu, rk);
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
    if (lane == 0) {
      skeys[rk + add] = (K)ki;
      p.offsets[rk + add] = (unsigned)(off + special);
    }
  }
}

// ---------------------------------------------------------------------------
// LSD radix sort, 8-bit digits, stable reduce-then-scan passes over tiles
// of kRadixTile items (all CTAs of the scope).
// ---------------------------------------------------------------------------
template <typename K>
__device__ __forceinline__ unsigned radix_digit(K k, int shift) {
  using T = KeyTraits<K>;
  const typename T::U u = (typename T::U)k ^ T::kSign;
  return (unsigned)(u >> shift) & (kRadixDigits - 1);
}

// One stable counting pass on digit `pass` (8 bits at 8*pass), all CTAs.
// CTA b owns the contiguous tiles [b*T/G, (b+1)*T/G) and scatters them in
// order, so each digit's output position is
//   dstart[d] + (keys with digit d in CTAs before b) + (earlier tiles of b)
//   + (rank within the tile).
// (a) every CTA counts digit d over its range; (b) the CTAs scan those
// counts (CTA b takes digits d = b, b + G, ...), with a grid barrier after
// each step; (c) every CTA ranks each tile in shared memory (stable: each
// warp ranks its items by digit, item-major then lane, and the warps' digit
// counts are scanned in warp order) and writes it out.  Per half-tile the
// half meets at four barriers: after the warps' ranking, after the digit
// scan (a thread pair per digit, the digit totals scanned within each warp),
// after taking the digit bases, and after staging the keys in digit order.
// Half-CTA pipelines of a radix pass: the CTA's range is cut into half-tiles
// of kHalfTile keys, taken alternately by the two halves of the CTA (512
// threads each, own shared memory, own named barrier).  A half-tile gets its
// digit bases from the CTA's running cursor, which the halves hand to each
// other in half-tile order through a turn counter, so every digit keeps the
// input order (the pass is stable) while one half waits at its barriers and
// the other ranks or writes.
constexpr int kHalfThreads = kThreads / 2;
constexpr int kHalfWarps = kHalfThreads / 32;
constexpr int kHalfTile = kHalfThreads * kRadixItems;

__device__ __forceinline__ void half_sync(int h) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + h), "r"(kHalfThreads) : "memory");
}

// Lanes of the warp whose digit equals this lane's (digits < 2^9: the
// radix digit, or 256 for no item).  The top digit bits go to one match
// instruction and each low bit to a ballot: ballots and the bit tests around
// them are ALU work, whose pipe a pass of ballots alone keeps busy, while
// the match runs in another unit and costs more the more distinct values the
// warp holds (at most 8 here: 256 >> 5 = 8 tells missing items apart).  On
// 3e7 distinct int64 keys the whole sort took 2.32 ms with eight ballots,
// 2.10 ms with a match of 3 bits and 5 ballots, 2.13 ms with 4 + 4, 2.40 ms
// with 5 + 3, 2.89 ms with a match of each nibble and about 3 ms with one
// match of the whole digit.
__device__ __forceinline__ unsigned digit_peers_ballot(unsigned d) {
  constexpr int kLowBits = 5;
  unsigned peers = __match_any_sync(0xffffffffu, d >> kLowBits);
  #pragma unroll
  for (int bit = 0; bit < kLowBits; ++bit) {
    const unsigned on = (d >> bit) & 1u;
    const unsigned b = __ballot_sync(0xffffffffu, on);
    peers &= on ? b : ~b;
  }
  return peers;
}

// Stable rank of a warp's items within the warp (item-major, then lane):
// rd[j] holds the digit on entry and gets (rank << 16) | digit.  `row` is
// the warp's digit-counter row (zero on entry, the warp's digit counts on
// exit).
template <bool kMatch>
__device__ __forceinline__ void rank_warp_items(unsigned (&rd)[kRadixItems], unsigned short* row, int lane) {
  #pragma unroll
  for (int j = 0; j < kRadixItems; ++j) {
    const unsigned d = rd[j];
    const unsigned peers = kMatch ? __match_any_sync(0xffffffffu, d) : digit_peers_ballot(d);
    const int leader = __ffs(peers) - 1;
    unsigned old = 0;
    if (lane == leader && d < (unsigned)kRadixDigits) {
      old = row[d];
      row[d] = (unsigned short)(old + __popc(peers));
    }
    old = __shfl_sync(0xffffffffu, old, leader);
    __syncwarp();
    rd[j] = d | ((old + __popc(peers & lanemask_lt())) << 16);
  }
}

template <typename K, bool PAY>
struct HalfSmem {
  K stage_k[kHalfTile];
  unsigned stage_v[PAY ? kHalfTile : 1];
  unsigned short wcnt[kHalfWarps * kRadixDigits];
  unsigned tile_start[kRadixDigits];
  unsigned base[kRadixDigits];      // digit destination minus its first stage slot
  unsigned scratch[kHalfWarps];     // per warp: half-tile keys of its 16 digits
  unsigned stop;                    // the half leaves the pass (written before a barrier, read after it)
};

struct PassSmem {
  unsigned running[kRadixDigits];   // the CTA's digit cursor
  unsigned hist[kRadixDigits];
  unsigned scratch[kWarps];
  unsigned turn;                    // next half-tile allowed to take bases
  unsigned failed;
};

// Step (a) of a pass over all CTAs: digit `pass` counted over this CTA's
// range of tiles, stored as the CTA's part counts in the radix scratch and
// added to the pass's global totals (Ctrl::hist).  With kBits, also the OR of
// the order-mapped keys and of their complements (the key bits that vary),
// so that one read of the keys serves pass 0's counts and the choice of
// passes.  The caller's grid barrier publishes all of it.
template <typename K, bool kBits>
__device__ void radix_count(const Params& p, const K* in_k, unsigned long long n, int pass,
                            unsigned char* smem, const GridScope& sc) {
  using T = KeyTraits<K>;
  Ctrl* c = p.ctrl;
  const int shift = pass * kRadixBits;
  const unsigned long long ntiles = (n + kRadixTile - 1) / kRadixTile;
  const unsigned b = sc.part(), nb = sc.nparts();
  const unsigned long long i0 = (ntiles * b / nb) * kRadixTile;
  const unsigned long long i1e = (ntiles * (b + 1) / nb) * kRadixTile;
  const unsigned long long i1 = i1e < n ? i1e : n;
  unsigned* hist = reinterpret_cast<PassSmem*>(smem)->hist;
  if (threadIdx.x < kRadixDigits) hist[threadIdx.x] = 0u;
  __syncthreads();
  unsigned long long o1 = 0ull, o0 = 0ull;
  constexpr int U = 4;
  for (unsigned long long base = i0 + threadIdx.x; base < i1; base += (unsigned long long)U * kThreads) {
    K kk[U];
    #pragma unroll
    for (int j = 0; j < U; ++j) {
      const unsigned long long i = base + (unsigned long long)j * kThreads;
      kk[j] = i < i1 ? __ldcg(in_k + i) : (K)0;
    }
    #pragma unroll
    for (int j = 0; j < U; ++j) {
      if (base + (unsigned long long)j * kThreads < i1) {
        atomicAdd(hist + radix_digit(kk[j], shift), 1u);
        if constexpr (kBits) {
          const typename T::U u = (typename T::U)kk[j] ^ T::kSign;
          o1 |= (unsigned long long)u;
          o0 |= (unsigned long long)(typename T::U)~u;
        }
      }
    }
  }
  if constexpr (kBits) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      o1 |= __shfl_xor_sync(0xffffffffu, o1, o);
      o0 |= __shfl_xor_sync(0xffffffffu, o0, o);
    }
    if ((threadIdx.x & 31) == 0) {
      if (o1) atomicOr(&c->key_or, o1);
      if (o0) atomicOr(&c->key_nor, o0);
    }
  }
  unsigned* cta_cnt = reinterpret_cast<unsigned*>(p.lookback);   // [nb][256]
  __syncthreads();
  if (threadIdx.x < kRadixDigits) {
    const unsigned v = hist[threadIdx.x];
    cta_cnt[b * kRadixDigits + threadIdx.x] = v;
    if (v) atomicAdd(&c->hist[pass][threadIdx.x], v);
  }
}

// `counted`: step (a) of this pass was already done (radix_count).
template <typename K, bool PAY, class S>
__device__ bool radix_pass(const Params& p, const K* in_k, const unsigned* in_v, K* out_k,
                           unsigned* out_v, unsigned long long n, int pass, unsigned char* smem,
                           unsigned& epoch, const S& sc, bool counted) {
  Ctrl* c = p.ctrl;
  const int shift = pass * kRadixBits;
  const unsigned long long ntiles = (n + kRadixTile - 1) / kRadixTile;
  const unsigned b = sc.part(), nb = sc.nparts();
  const unsigned long long tile0 = ntiles * b / nb, tile1 = ntiles * (b + 1) / nb;
  const unsigned long long i0 = tile0 * kRadixTile;
  const unsigned long long i1 = tile1 * kRadixTile < n ? tile1 * kRadixTile : n;
  unsigned* cta_cnt = reinterpret_cast<unsigned*>(p.lookback);       // [nb][256]
  unsigned* cta_base = cta_cnt + nb * kRadixDigits;                   // [nb][256]

  PassSmem* ps = reinterpret_cast<PassSmem*>(smem);
  constexpr size_t kPassBytes = (sizeof(PassSmem) + 127) & ~size_t(127);
  constexpr size_t kHalfBytes = (sizeof(HalfSmem<K, PAY>) + 127) & ~size_t(127);
  static_assert(kPassBytes + 2 * kHalfBytes <= (size_t)kPipelineSmem, "radix pass shared memory");
  unsigned* running = ps->running;
  unsigned* hist = ps->hist;
  unsigned* scratch = ps->scratch;

  if (threadIdx.x == 0) {
    ps->turn = 0u;
    ps->failed = 0u;
  }
  if constexpr (std::is_same<S, CtaScope>::value) {
    // One CTA owns the whole range: the digit starts are the exclusive scan
    // of the pass histogram (counted for all passes up front), so the
    // per-pass count read and the cross-CTA scan are not needed.
    const unsigned v = threadIdx.x < kRadixDigits ? c->hist[pass][threadIdx.x] : 0u;
    unsigned tot;
    const unsigned ex = block_exclusive_scan(v, scratch, &tot);
    if (threadIdx.x < kRadixDigits) running[threadIdx.x] = ex;
  } else {
    // (a) digit counts of this CTA's range (and the pass totals)
    if (!counted) {
      radix_count<K, false>(p, in_k, n, pass, smem, sc);
      if (!sc.sync(c, epoch, p.timeout_ns)) return false;
    }

    // (b) exclusive scan over CTAs of each digit (this CTA's digits), offset
    // by the digit's global start (exclusive scan of the pass histogram)
    {
      const unsigned v = threadIdx.x < kRadixDigits ? ld_relaxed_u32(&c->hist[pass][threadIdx.x]) : 0u;
      unsigned tot;
      const unsigned ex = block_exclusive_scan(v, scratch, &tot);
      if (threadIdx.x < kRadixDigits) hist[threadIdx.x] = ex;   // digit starts
    }
    __syncthreads();
    for (int d = (int)b; d < kRadixDigits; d += (int)nb) {
      const unsigned dstart = hist[d];
      const unsigned v = threadIdx.x < nb ? __ldcg(cta_cnt + threadIdx.x * kRadixDigits + d) : 0u;
      unsigned tot;
      const unsigned ex = block_exclusive_scan(v, scratch, &tot);
      if (threadIdx.x < nb) cta_base[threadIdx.x * kRadixDigits + d] = dstart + ex;
    }
    if (!sc.sync(c, epoch, p.timeout_ns)) return false;
    if (threadIdx.x < kRadixDigits) running[threadIdx.x] = __ldcg(cta_base + b * kRadixDigits + threadIdx.x);
  }
  __syncthreads();

  // (c) rank and scatter the CTA's range in half-tiles
  const int h = threadIdx.x / kHalfThreads;
  const int t = threadIdx.x - h * kHalfThreads;
  const int w = t >> 5, lane = t & 31;
  HalfSmem<K, PAY>* hs = reinterpret_cast<HalfSmem<K, PAY>*>(smem + kPassBytes + (size_t)h * kHalfBytes);
  const unsigned long long nhalf = (i1 - i0 + kHalfTile - 1) / kHalfTile;
  for (unsigned long long q = (unsigned long long)h; q < nhalf; q += 2) {
    const unsigned long long base = i0 + q * kHalfTile;
    const unsigned cnt = (unsigned)((i1 - base) < (unsigned long long)kHalfTile ? (i1 - base) : kHalfTile);
    // No barrier here: another warp's accesses of the previous half-tile's
    // shared arrays all come before it reaches this half-tile's first
    // barrier, and until then this warp writes only its own counter row.
    for (int d = lane; d < kRadixDigits; d += 32) hs->wcnt[w * kRadixDigits + d] = 0;
    __syncwarp();
    K key[kRadixItems];
    unsigned rd[kRadixItems];   // rank within the warp << 16 | digit (256 = no item)
    const unsigned long long wbase = base + (unsigned long long)w * (32 * kRadixItems) + lane;
    #pragma unroll
    for (int j = 0; j < kRadixItems; ++j) {
      const unsigned long long idx = wbase + j * 32;
      const bool valid = idx < i1;
      key[j] = valid ? __ldcg(in_k + idx) : (K)0;
      rd[j] = valid ? radix_digit(key[j], shift) : (unsigned)kRadixDigits;
    }
    // Runs of equal keys (a later pass over repeated keys) leave few
    // distinct digits per warp, where the match instruction is cheaper than
    // the ballots: the warp picks one by how many lanes share the digit of
    // the next lane (item 0).
    const unsigned next_d = __shfl_down_sync(0xffffffffu, rd[0], 1);
    const bool runs = __popc(__ballot_sync(0xffffffffu, lane == 31 || next_d == rd[0])) >= 16;
    if (runs) rank_warp_items<true>(rd, hs->wcnt + w * kRadixDigits, lane);
    else rank_warp_items<false>(rd, hs->wcnt + w * kRadixDigits, lane);
    half_sync(h);
    // Digit d = t / 2: the thread pair (g = t & 1, adjacent lanes) turns the
    // counts of warps 8g .. 8g + 7 into exclusive prefixes over the half's
    // warps, and each warp scans the half-tile totals of its 16 digits, so
    // that one barrier later every thread has its digit's start.
    constexpr int kPairWarps = kHalfWarps / 2;
    static_assert(kHalfThreads == 2 * kRadixDigits && kHalfWarps * 16 == kRadixDigits, "digit pairs");
    const int dg = t >> 1, g = t & 1;
    unsigned run = 0;
    #pragma unroll
    for (int qq = g * kPairWarps; qq < (g + 1) * kPairWarps; ++qq) {
      const unsigned x = hs->wcnt[qq * kRadixDigits + dg];
      hs->wcnt[qq * kRadixDigits + dg] = (unsigned short)run;
      run += x;
    }
    const unsigned other = __shfl_xor_sync(0xffffffffu, run, 1);
    const unsigned tot = run + other;   // the digit's keys in the half-tile
    if (g) {
      #pragma unroll
      for (int qq = kPairWarps; qq < kHalfWarps; ++qq)
        hs->wcnt[qq * kRadixDigits + dg] = (unsigned short)(hs->wcnt[qq * kRadixDigits + dg] + other);
    }
    unsigned incl = g ? 0u : tot;        // inclusive scan over this warp's digits
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) hs->scratch[w] = incl;
    // Take this half-tile's digit bases from the cursor, in half-tile order.
    if (t == 0) {
      const unsigned long long t0 = global_timer_ns();
      unsigned it = 0;
      while (*reinterpret_cast<volatile unsigned*>(&ps->turn) != (unsigned)q) {
        if (*reinterpret_cast<volatile unsigned*>(&ps->failed)) break;
        if ((++it & 255u) == 0 && global_timer_ns() - t0 > p.timeout_ns) {
          atomicExch(&c->rec.status, kDevTimeout);
          *reinterpret_cast<volatile unsigned*>(&ps->failed) = 1u;
          break;
        }
      }
      __threadfence_block();
      // One read of the shared failure flag for the whole half: the other
      // half may raise it while this half's threads read it.
      hs->stop = *reinterpret_cast<volatile unsigned*>(&ps->failed);
    }
    half_sync(h);
    if (hs->stop) break;
    {
      unsigned wt = 0;   // half-tile keys of the digits of warps before this one
      if (lane < w) wt = hs->scratch[lane];
      const unsigned before = __reduce_add_sync(0xffffffffu, wt);
      if (!g) {
        const unsigned start = before + incl - tot;
        hs->tile_start[dg] = start;
        hs->base[dg] = running[dg] - start;   // destination of stage slot i = base[d] + i
        running[dg] += tot;
      }
    }
    half_sync(h);
    if (t == 0) {
      __threadfence_block();
      *reinterpret_cast<volatile unsigned*>(&ps->turn) = (unsigned)q + 1u;
    }
    // Scatter into shared memory in half-tile-sorted order.
    #pragma unroll
    for (int j = 0; j < kRadixItems; ++j) {
      const unsigned d = rd[j] & 0xFFFFu;
      if (d < (unsigned)kRadixDigits) {
        const unsigned pos = hs->tile_start[d] + hs->wcnt[w * kRadixDigits + d] + (rd[j] >> 16);
        hs->stage_k[pos] = key[j];
        if constexpr (PAY) hs->stage_v[pos] = __ldcg(in_v + wbase + j * 32);
      }
    }
    half_sync(h);
    for (unsigned i = t; i < cnt; i += kHalfThreads) {
      const K k = hs->stage_k[i];
      const unsigned d = radix_digit(k, shift);
      const unsigned long long dst = (unsigned long long)(unsigned)(hs->base[d] + i);
      __stcg(out_k + dst, k);
      if constexpr (PAY) __stcg(out_v + dst, hs->stage_v[i]);
    }
  }
  __syncthreads();
  return !ps->failed && !device_failed(c);
}

// Full LSD radix sort src -> dst (tmp as ping-pong), all CTAs.  Returns false
// if a barrier failed (the caller must return).
template <typename K, bool PAY, class S>
__device__ bool radix_sort(const Params& p, const K* src_k, const unsigned* src_v,
                           unsigned long long n, K* dst_k, unsigned* dst_v, K* tmp_k,
                           unsigned* tmp_v, unsigned char* smem, unsigned& epoch,
                           const S& sc) {
  using T = KeyTraits<K>;
  constexpr int NP = T::kPasses;
  constexpr bool kGrid = std::is_same<S, GridScope>::value;
  Ctrl* c = p.ctrl;
  // Plan: a pass whose digit is the same for every key changes nothing.
  unsigned active_bits = 0;  // pass indices, 4 bits each
  int na = 0;
  if constexpr (kGrid) {
    // Pass 0's counts and the key bits that vary, from one read of the keys;
    // every later pass counts its own digit (step (a)).
    radix_count<K, true>(p, src_k, n, 0, smem, sc);
    if (!sc.sync(c, epoch, p.timeout_ns)) return false;
    const unsigned long long vary = ld_relaxed_u64(&c->key_or) & ld_relaxed_u64(&c->key_nor);
    for (int q = 0; q < NP; ++q)
      if ((vary >> (q * kRadixBits)) & (kRadixDigits - 1)) active_bits |= (unsigned)q << (4 * na++);
  } else {
    // One CTA: the histogram of every digit of every pass (one read of the
    // keys) gives each pass its digit starts directly.
    unsigned* sh = reinterpret_cast<unsigned*>(smem);
    for (int i = threadIdx.x; i < NP * kRadixDigits; i += blockDim.x) sh[i] = 0u;
    __syncthreads();
    {
      constexpr int U = 4;
      for (unsigned long long base = threadIdx.x; base < n; base += (unsigned long long)kThreads * U) {
        K kk[U];
        #pragma unroll
        for (int j = 0; j < U; ++j) {
          const unsigned long long i = base + (unsigned long long)j * kThreads;
          kk[j] = i < n ? __ldcg(src_k + i) : (K)0;
        }
        #pragma unroll
        for (int j = 0; j < U; ++j) {
          if (base + (unsigned long long)j * kThreads < n) {
            const typename T::U u = (typename T::U)kk[j] ^ T::kSign;
            #pragma unroll
            for (int q = 0; q < NP; ++q) atomicAdd(sh + q * kRadixDigits + ((u >> (q * kRadixBits)) & 0xFF), 1u);
          }
        }
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NP * kRadixDigits; i += blockDim.x) c->hist[i / kRadixDigits][i % kRadixDigits] = sh[i];
    __syncthreads();
    int* triv = reinterpret_cast<int*>(smem);  // NP flags
    if (threadIdx.x < NP) triv[threadIdx.x] = 0;
    __syncthreads();
    if (threadIdx.x < kRadixDigits)
      for (int q = 0; q < NP; ++q)
        if ((unsigned long long)c->hist[q][threadIdx.x] == n) triv[q] = 1;
    __syncthreads();
    for (int q = 0; q < NP; ++q)
      if (!triv[q]) active_bits |= (unsigned)q << (4 * na++);
    __syncthreads();
  }
  // The last active pass writes dst; earlier ones alternate with tmp.  If the
  // first pass would write over its own input (in-place), every target flips
  // and a final copy tmp -> dst follows.
  bool flip = false;
  if (na > 0) {
    const bool first_to_dst = ((na - 1) % 2) == 0;
    if (first_to_dst && (const void*)src_k == (const void*)dst_k) flip = true;
  }
  const K* cur_k = src_k;
  const unsigned* cur_v = src_v;
  for (int a = 0; a < na; ++a) {
    bool to_dst = ((na - 1 - a) % 2) == 0;
    if (flip) to_dst = !to_dst;
    K* ok_ = to_dst ? dst_k : tmp_k;
    unsigned* ov = to_dst ? dst_v : tmp_v;
    const int pass = (int)((active_bits >> (4 * a)) & 15u);
    if (!radix_pass<K, PAY>(p, cur_k, cur_v, ok_, ov, n, pass, smem, epoch, sc, kGrid && pass == 0))
      return false;
    if (!sc.sync(c, epoch, p.timeout_ns)) return false;
    cur_k = ok_;
    cur_v = ov;
  }
  if ((const void*)cur_k != (const void*)dst_k) {
    grid_copy<K>(cur_k, dst_k, n, sc);
    if constexpr (PAY) {
      const unsigned long long G = sc.gthreads();
      const unsigned long long gt = sc.gthread();
      for (unsigned long long i = gt; i < n; i += G) dst_v[i] = __ldcg(cur_v + i);
    }
    if (!sc.sync(c, epoch, p.timeout_ns)) return false;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Scan of the sorted counts (large pair path): offsets[i] = sum of counts
// before i; offsets[kp] = n.  Two levels with one grid barrier.
// ---------------------------------------------------------------------------
template <class S>
__device__ bool grid_scan_counts(const Params& p, const unsigned* vals, unsigned long long kp,
                                 unsigned char* smem, unsigned& epoch, const S& sc) {
  Ctrl* c = p.ctrl;
  unsigned long long* scratch = reinterpret_cast<unsigned long long*>(smem);
  const unsigned b = sc.part(), nb = sc.nparts();
  const unsigned long long i0 = kp * b / nb, i1 = kp * (b + 1) / nb;
  unsigned long long s = 0;
  for (unsigned long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) s += __ldcg(vals + i);
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) c->chunk_sums[b] = s;
  if (!sc.sync(c, epoch, p.timeout_ns)) return false;
  unsigned long long base = 0;
  for (unsigned q = threadIdx.x; q < b; q += blockDim.x) base += ld_relaxed_u64(&c->chunk_sums[q]);
  base = block_sum(base, scratch + kWarps);
  unsigned long long carry = base;
  for (unsigned long long off = i0; off < i1; off += blockDim.x) {
    const unsigned long long i = off + threadIdx.x;
    const unsigned long long v = i < i1 ? (unsigned long long)__ldcg(vals + i) : 0ull;
    unsigned long long tot;
    const unsigned long long ex = block_exclusive_scan(v, scratch + 2 * kWarps, &tot);
    if (i < i1) p.offsets[i] = (unsigned)(carry + ex);
    carry += tot;
  }
  if (b == 0 && threadIdx.x == 0) p.offsets[kp] = (unsigned)p.n;
  return sc.sync(c, epoch, p.timeout_ns);
}

// How a column's pass through column_body() ended.
enum ColumnEnd : int {
  kColumnDone = 0,     // output written
  kColumnRadix = 1,    // the path ends in the LSD radix fallback, not yet run
  kColumnFailed = 2,   // a bounded wait gave up; the status is in the record
  kColumnTooBig = 3,   // the Eq. 6 table exceeds this workspace's table; nothing
                       // was counted (only the sampler's record was written)
};

// ---------------------------------------------------------------------------
// Phase 3b (K' > kRankPairs, all CTAs of a grid): splitter bucket sort of the
// pairs, the sort and exclusive scan of Alg. 4 without a radix pass.
//   1. the claimed slots are gathered into the pair arrays A (the table is
//      reset on the way);
//   2. every CTA sorts the same evenly spaced sample of A's keys in shared
//      memory and takes G - 1 splitters from it, so bucket g (owned by CTA g)
//      holds a contiguous key range; every CTA counts its share of the pairs
//      per bucket (and the key counts they carry);
//   3. CTA g scans bucket g's counts over the producing CTAs;
//   4. every CTA scatters its share into the buckets (array B);
//   5. CTA g sorts bucket g in shared memory and writes its keys and run
//      offsets (bucket starts and count starts are exclusive scans of the
//      bucket totals, which every CTA computes).
// Keys are distinct, so the order inside a bucket before step 5 does not
// matter.  Five grid barriers in all.  Returns kColumnFailed on a failed
// barrier, kColumnRadix when a bucket is too large for one CTA (the caller
// then sorts A with the radix sort), kColumnDone otherwise.
// ---------------------------------------------------------------------------
constexpr int kBucketSortCap = 16384;   // pairs one CTA sorts in shared memory
constexpr int kPairSamplesPerCta = 16;
constexpr int kPairSamplesMax = 4096;
static_assert(kBucketSortCap * 12 <= kPipelineSmem, "bucket in shared memory");

// Number of splitters <= x among spl[0, P - 1) (P a power of two, entries
// past the G - 1 splitters hold LLONG_MAX), clamped to the last bucket.
__device__ __forceinline__ unsigned bucket_of(const long long* spl, int P, long long x, unsigned G) {
  int pos = 0;
  for (int step = P >> 1; step >= 1; step >>= 1)
    if (spl[pos + step - 1] <= x) pos += step;
  return (unsigned)pos < G ? (unsigned)pos : G - 1u;
}

// In-place ascending bitonic sort of n (a power of two) pairs by key, by all
// threads; entries with value 0 (padding) sort after real entries (values
// >= 1) of an equal key.
__device__ __forceinline__ void bitonic_sort_counted(long long* k, unsigned* v, int n) {
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const long long a = k[i], b = k[j];
          const unsigned va = v[i], vb = v[j];
          const bool a_gt = a > b || (a == b && va == 0u && vb != 0u);
          if (a_gt == up) {
            k[i] = b; k[j] = a;
            v[i] = vb; v[j] = va;
          }
        }
      }
      __syncthreads();
    }
  }
}

// The bucket sort's scratch in p.lookback starts after the radix sort's
// per-CTA digit counts and bases (G x 256 64-bit words), which the radix
// fallback of the pairs writes while other CTAs may still read it.
__device__ __forceinline__ bool bucket_sort_fits(const Params& p, unsigned G) {
  return G <= (unsigned)kBucketMaxGrid &&
         (unsigned long long)G * kRadixDigits + bucket_scratch_words(G) + kSamples <= p.lookback_cap;
}

template <typename K>
__device__ int phase_bucket_pairs(const Params& p, unsigned occ, unsigned long long special,
                                  unsigned long long kp, unsigned char* smem, unsigned& epoch,
                                  const GridScope& sc) {
  using T = KeyTraits<K>;
  Ctrl* c = p.ctrl;
  const unsigned G = sc.nparts(), b = sc.part();
  K* ak = reinterpret_cast<K*>(p.pkeys_a);
  unsigned* av = p.pvals_a;
  K* bk = reinterpret_cast<K*>(p.pkeys_b);
  unsigned* bv = p.pvals_b;

  // 1. gather + reset
  {
    const unsigned long long Gt = sc.gthreads(), gt = sc.gthread();
    for (unsigned long long i = gt; i < occ; i += Gt) {
      const unsigned slot = __ldcg(p.claimed + i);
      ak[i] = (K)(long long)__ldcg(p.tkeys + slot);
      av[i] = __ldcg(p.tcounts + slot);
      p.tkeys[slot] = kEmpty64;
      p.tcounts[slot] = 0u;
    }
    if (special && gt == 0) {
      ak[occ] = T::min_key();
      av[occ] = (unsigned)special;
    }
  }
  if (!sc.sync(c, epoch, p.timeout_ns)) return kColumnFailed;

  unsigned* cnt = reinterpret_cast<unsigned*>(p.lookback + (size_t)G * kRadixDigits);   // [G][G] pairs of b' in g
  unsigned* csm = cnt + (size_t)G * G;                        // [G][G] their key counts
  unsigned* base = csm + (size_t)G * G;                       // [G][G] first position of b' in g
  unsigned* tot = base + (size_t)G * G;                       // [G]
  unsigned* tsum = tot + G;                                   // [G]

  // 2. splitters and per-bucket counts of this CTA's share
  const int P = (int)bit_ceil_u64(G);
  long long* spl = reinterpret_cast<long long*>(smem);                          // P
  unsigned* hcnt = reinterpret_cast<unsigned*>(spl + P);                        // P
  unsigned* hsum = hcnt + P;                                                    // P
  unsigned* aux = hsum + P;                                                     // kWarps + 8
  long long* samp = reinterpret_cast<long long*>(smem + 32 * 1024);             // kPairSamplesMax
  {
    unsigned long long nsamp = (unsigned long long)kPairSamplesPerCta * G;
    if (nsamp > (unsigned long long)kPairSamplesMax) nsamp = kPairSamplesMax;
    if (nsamp > kp) nsamp = kp;
    const int ps = (int)bit_ceil_u64(nsamp);
    for (int j = threadIdx.x; j < ps; j += blockDim.x)
      samp[j] = (unsigned long long)j < nsamp ? (long long)__ldcg(ak + (kp * (unsigned long long)j) / nsamp)
                                              : LLONG_MAX;
    for (int g = threadIdx.x; g < P; g += blockDim.x) {
      hcnt[g] = 0u;
      hsum[g] = 0u;
    }
    __syncthreads();
    bitonic_sort_pairs(samp, nullptr, ps);
    for (int g = threadIdx.x; g < P; g += blockDim.x)
      spl[g] = (unsigned)g + 1u < G ? samp[((unsigned long long)(g + 1) * nsamp) / G] : LLONG_MAX;
    __syncthreads();
  }
  const unsigned long long i0 = kp * b / G, i1 = kp * (b + 1) / G;
  for (unsigned long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const unsigned g = bucket_of(spl, P, (long long)__ldcg(ak + i), G);
    atomicAdd(hcnt + g, 1u);
    atomicAdd(hsum + g, __ldcg(av + i));
  }
  __syncthreads();
  for (unsigned g = threadIdx.x; g < G; g += blockDim.x) {
    cnt[(size_t)b * G + g] = hcnt[g];
    csm[(size_t)b * G + g] = hsum[g];
  }
  if (!sc.sync(c, epoch, p.timeout_ns)) return kColumnFailed;

  // 3. bucket b: exclusive scan of its counts over the producers
  {
    unsigned t = 0;
    const unsigned v = threadIdx.x < G ? __ldcg(cnt + (size_t)threadIdx.x * G + b) : 0u;
    const unsigned s = threadIdx.x < G ? __ldcg(csm + (size_t)threadIdx.x * G + b) : 0u;
    const unsigned ex = block_exclusive_scan(v, aux, &t);
    if (threadIdx.x < G) base[(size_t)threadIdx.x * G + b] = ex;
    const unsigned ss = block_sum(s, aux);
    if (threadIdx.x == 0) {
      tot[b] = t;
      tsum[b] = ss;
    }
  }
  if (!sc.sync(c, epoch, p.timeout_ns)) return kColumnFailed;

  // bucket starts and count starts (every CTA); too large a bucket: radix
  unsigned* bstart = hcnt;   // reuses the histogram arrays
  unsigned* cstart = hsum;
  unsigned* cur = aux + kWarps + 8;   // P cursors
  {
    unsigned t = 0;
    const unsigned v = threadIdx.x < G ? __ldcg(tot + threadIdx.x) : 0u;
    const unsigned s = threadIdx.x < G ? __ldcg(tsum + threadIdx.x) : 0u;
    const int big = __syncthreads_or(v > (unsigned)kBucketSortCap);
    const unsigned ex = block_exclusive_scan(v, aux, &t);
    if (threadIdx.x < G) bstart[threadIdx.x] = ex;
    const unsigned exs = block_exclusive_scan(s, aux, &t);
    if (threadIdx.x < G) {
      cstart[threadIdx.x] = exs;
      cur[threadIdx.x] = ex + __ldcg(base + (size_t)b * G + threadIdx.x);
    }
    __syncthreads();
    if (big) return kColumnRadix;
  }

  // 4. scatter this CTA's share into the buckets
  for (unsigned long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const K x = __ldcg(ak + i);
    const unsigned g = bucket_of(spl, P, (long long)x, G);
    const unsigned pos = atomicAdd(cur + g, 1u);
    bk[pos] = x;
    bv[pos] = __ldcg(av + i);
  }
  const unsigned my_start = bstart[b], my_cstart = cstart[b];
  __syncthreads();
  if (!sc.sync(c, epoch, p.timeout_ns)) return kColumnFailed;

  // 5. sort bucket b in shared memory, write keys and run offsets
  const unsigned m = __ldcg(tot + b);
  if (m > 0) {
    long long* sk = reinterpret_cast<long long*>(smem);
    unsigned* sv = reinterpret_cast<unsigned*>(sk + kBucketSortCap);
    const int pm = (int)bit_ceil_u64(m);
    for (int j = threadIdx.x; j < pm; j += blockDim.x) {
      const bool real = (unsigned)j < m;
      sk[j] = real ? (long long)__ldcg(bk + my_start + j) : LLONG_MAX;
      sv[j] = real ? __ldcg(bv + my_start + j) : 0u;
    }
    __syncthreads();
    bitonic_sort_counted(sk, sv, pm);
    K* skeys = reinterpret_cast<K*>(p.skeys);
    unsigned long long carry = my_cstart;
    unsigned long long* scan_scratch = reinterpret_cast<unsigned long long*>(sv + kBucketSortCap);
    for (unsigned j0 = 0; j0 < m; j0 += blockDim.x) {
      const unsigned j = j0 + threadIdx.x;
      const unsigned long long v = j < m ? (unsigned long long)sv[j] : 0ull;
      unsigned long long t;
      const unsigned long long ex = block_exclusive_scan(v, scan_scratch, &t);
      if (j < m) {
        skeys[my_start + j] = (K)sk[j];
        p.offsets[my_start + j] = (unsigned)(carry + ex);
      }
      carry += t;
    }
  }
  if (b == 0 && threadIdx.x == 0) p.offsets[kp] = (unsigned)p.n;
  if (!sc.sync(c, epoch, p.timeout_ns)) return kColumnFailed;
  return kColumnDone;
}

// ---------------------------------------------------------------------------
// Phase 4: emit.  Output tiles of p.emit_tile_vec 16-byte vectors; each CTA
// looks up the first and last run of each of its tiles (binary search on the
// run offsets), stages the tile's runs in shared memory and writes the
// vectors with streaming stores.
// ---------------------------------------------------------------------------
constexpr int kEmitMaxTilesPerCta = 512;
// Threads that write a tile covered by a single run.
constexpr int kEmitBroadcastThreads = 256;
static_assert(kEmitBroadcastThreads <= kThreads, "broadcast writers");

// Largest j in [lo, hi] with off[j] <= x (off non-decreasing, off[lo] <= x).
__device__ __forceinline__ unsigned long long run_of(const unsigned* off, unsigned long long lo,
                                                     unsigned long long hi, unsigned long long x) {
  while (lo < hi) {
    const unsigned long long mid = (lo + hi + 1) >> 1;
    if ((unsigned long long)__ldcg(off + mid) <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename K, class S>
__device__ void phase_emit(const Params& p, unsigned long long npairs, unsigned char* smem,
                           const S& sc) {
  using T = KeyTraits<K>;
  using V = typename T::Vec;
  constexpr int VPE = T::kVec;
  const K* sk = reinterpret_cast<const K*>(p.skeys);
  const unsigned* off = p.offsets;
  K* out = reinterpret_cast<K*>(p.out);
  const unsigned long long n = p.n;
  const unsigned long long last = npairs - 1;
  const uintptr_t addr = reinterpret_cast<uintptr_t>(out);
  unsigned long long head = ((16u - (addr & 15u)) & 15u) / sizeof(K);
  if (head > n) head = n;
  const unsigned long long nvec = (n - head) / VPE;
  const unsigned long long tail0 = head + nvec * VPE;
  const unsigned nb = sc.nparts(), b = sc.part();
  const unsigned long long tv = p.emit_tile_vec;

  if (b == 0)
    for (unsigned long long i = threadIdx.x; i < head; i += blockDim.x) out[i] = __ldcg(sk + run_of(off, 0, last, i));
  if (b == nb - 1)
    for (unsigned long long i = tail0 + threadIdx.x; i < n; i += blockDim.x) out[i] = __ldcg(sk + run_of(off, 0, last, i));

  const unsigned long long ntile = (nvec + tv - 1) / tv;
  unsigned* tj = reinterpret_cast<unsigned*>(smem);                     // 2 per local tile
  unsigned* soff = tj + 2 * kEmitMaxTilesPerCta;                        // kEmitStagePairs + 1
  K* skey = reinterpret_cast<K*>(soff + kEmitStagePairs + 2);           // kEmitStagePairs
  V* vout = reinterpret_cast<V*>(out + head);

  for (unsigned long long round = 0;; ++round) {
    const unsigned long long first_tile = (unsigned long long)b + round * kEmitMaxTilesPerCta * nb;
    if (first_tile >= ntile) break;
    // Look up the first and last run of up to kEmitMaxTilesPerCta tiles at once.
    for (int q = threadIdx.x; q < 2 * kEmitMaxTilesPerCta; q += blockDim.x) {
      const unsigned long long tile = first_tile + (unsigned long long)(q >> 1) * nb;
      if (tile < ntile) {
        const unsigned long long vb = tile * tv;
        const unsigned long long ve = (vb + tv < nvec) ? vb + tv : nvec;
        const unsigned long long e = (q & 1) ? head + ve * VPE - 1 : head + vb * VPE;
        tj[q] = (unsigned)run_of(off, 0, last, e);
      }
    }
    __syncthreads();
    for (int lt = 0; lt < kEmitMaxTilesPerCta; ++lt) {
      const unsigned long long tile = first_tile + (unsigned long long)lt * nb;
      if (tile >= ntile) break;
      const unsigned long long vb = tile * tv;
      const unsigned long long ve = (vb + tv < nvec) ? vb + tv : nvec;
      const unsigned j0 = tj[2 * lt], j1 = tj[2 * lt + 1];
      const unsigned m = j1 - j0 + 1;
      if (m == 1) {
        const V kv = splat(__ldcg(sk + j0));
        // One run fills the tile: a broadcast store stream.  A quarter of
        // the CTA's threads writes it faster than all of them (measured on
        // GB300: 37 us instead of 52 us per 240 MB column).
        if (threadIdx.x < kEmitBroadcastThreads)
          for (unsigned long long v = vb + threadIdx.x; v < ve; v += kEmitBroadcastThreads) __stcs(vout + v, kv);
      } else if (m <= (unsigned)kEmitStagePairs) {
        for (unsigned i = threadIdx.x; i <= m; i += blockDim.x) {
          soff[i] = (i < m) ? __ldcg(off + j0 + i) : __ldcg(off + j0 + m);
          if (i < m) skey[i] = __ldcg(sk + j0 + i);
        }
        __syncthreads();
        for (unsigned long long v = vb + threadIdx.x; v < ve; v += blockDim.x) {
          const unsigned long long e = head + v * VPE;
          unsigned lo = 0, hi = m - 1;
          while (lo < hi) {
            const unsigned mid = (lo + hi + 1) >> 1;
            if ((unsigned long long)soff[mid] <= e) lo = mid; else hi = mid - 1;
          }
          K vals[VPE];
          #pragma unroll
          for (int q = 0; q < VPE; ++q) {
            while (lo + 1 < m && (unsigned long long)soff[lo + 1] <= e + q) ++lo;
            vals[q] = skey[lo];
          }
          __stcs(vout + v, pack(vals));
        }
        __syncthreads();
      } else {
        for (unsigned long long v = vb + threadIdx.x; v < ve; v += blockDim.x) {
          const unsigned long long e = head + v * VPE;
          unsigned long long j = run_of(off, j0, j1, e);
          K vals[VPE];
          #pragma unroll
          for (int q = 0; q < VPE; ++q) {
            while (j < j1 && (unsigned long long)__ldcg(off + j + 1) <= e + q) ++j;
            vals[q] = __ldcg(sk + j);
          }
          __stcs(vout + v, pack(vals));
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// The persistent pipeline kernel (N >= 2048).
// ---------------------------------------------------------------------------
// CTA 0 zeroes the control block of the next launch on this workspace (two
// blocks alternate, so no separate zeroing step runs between launches).
__device__ __forceinline__ void zero_next_ctrl(const Params& p) {
  if (blockIdx.x != 0 || !p.ctrl_next) return;
  static_assert(sizeof(Ctrl) % 8 == 0, "control block in 8-byte words");
  unsigned long long* w = reinterpret_cast<unsigned long long*>(p.ctrl_next);
  for (int i = threadIdx.x; i < (int)(sizeof(Ctrl) / 8); i += blockDim.x) w[i] = 0ull;
}

template <class S>
__device__ __forceinline__ void mark(Ctrl* c, int i, const S& sc) {
  if (sc.lead()) c->rec.timeline[i] = global_timer_ns();
}

// Algorithm 3 for one column of n >= 2048 keys, run by the CTAs of `sc`:
// sample and estimate, the sortedness bypass, then the tiny or main count,
// the pair sort and scan, and the emit.  A path that ends in the radix
// fallback (2 K_hat > N, or the overflow guard) returns kColumnRadix with
// the table already clean, so that the caller can run the radix sort in
// whatever scope it chooses.  The control block must start zeroed apart
// from the grid-barrier words.
template <typename K, class S>
__device__ int column_body(const Params& p, unsigned char* smem, const S& sc, unsigned& epoch) {
  Ctrl* c = p.ctrl;
  const K* keys = reinterpret_cast<const K*>(p.keys);
  K* out = reinterpret_cast<K*>(p.out);

  // The count phase's first chunks are on their way while the samples are
  // taken.  With the whole grid on one column, every CTA fetches the samples
  // that lie in its own share (one CTA reading all 1024 strided positions,
  // spread over the whole column, spent about 8 us in address-translation
  // misses), then every CTA computes the estimate itself: one barrier, and
  // counting starts right after it.
  constexpr bool kGrid = std::is_same<S, GridScope>::value;
  Ring<K> ring;
  ring.live = false;
  if (p.mode == kModeSort) ring.start(p, keys, smem, sc);
  if constexpr (kGrid) {
    long long* gathered = reinterpret_cast<long long*>(p.lookback + (p.lookback_cap - kSamples));
    gather_samples<K>(p, keys, gathered, sc.part(), sc.nparts());
    if (!sc.sync(c, epoch, p.timeout_ns)) { ring.drain(p); return kColumnFailed; }
    phase_sample<K>(p, keys, smem, gathered);
  } else {
    phase_sample<K>(p, keys, smem);
  }
  mark(c, 1, sc);

  Record& r = c->rec;
  const int hint = r.sample_nondecreasing;
  if (hint) {
    phase_monotone<K>(p, keys, sc);
    if (!sc.sync(c, epoch, p.timeout_ns)) { ring.drain(p); return kColumnFailed; }
    mark(c, 2, sc);
    if (ld_relaxed_u32(&c->inversion) == 0u) {
      if (sc.lead()) {
        r.dispatch = 1;   // BYPASS_SORTED
        r.path = 1;
      }
      ring.drain(p);
      if (p.mode == kModeSort && (const void*)keys != (const void*)out) grid_copy<K>(keys, out, p.n, sc);
      return kColumnDone;
    }
  }
  if (p.mode == kModeEstimate) {
    ring.drain(p);
    return kColumnDone;
  }

  const int d = r.dispatch;
  if (d != 3 && d != 4) {
    ring.drain(p);
    if (sc.lead()) r.path = 5;  // HIGH_ENTROPY_RADIX
    return kColumnRadix;
  }
  if (r.C > p.table_cap) {   // only a capped batch workspace can be too small
    ring.drain(p);
    return kColumnTooBig;
  }
  if (d == 3) phase_count<K, true>(p, keys, smem, ring, sc);
  else phase_count<K, false>(p, keys, smem, ring, sc);
  if (!sc.sync(c, epoch, p.timeout_ns)) return kColumnFailed;
  mark(c, 3, sc);
  // One thread per CTA reads the counters every CTA hammered with atomics;
  // the others take them from shared memory (1024 reads of one hot L2 line
  // per CTA cost several microseconds).
  unsigned long long* cnt_smem = reinterpret_cast<unsigned long long*>(smem + kPipelineSmem - 64);
  if (threadIdx.x == 0) {
    cnt_smem[0] = ld_relaxed_u32(&c->occupancy);
    cnt_smem[1] = ld_relaxed_u64(&c->special);
    cnt_smem[2] = ld_relaxed_u32(&c->overflow);
  }
  __syncthreads();
  const unsigned occ = (unsigned)cnt_smem[0];
  const unsigned long long special = cnt_smem[1];
  const unsigned long long kp = (unsigned long long)occ + (special ? 1ull : 0ull);
  // Alg. 4's guard (distinct keys > L) decides the branch; the count itself
  // stops only past the global table's own limit (see table_log2), and only
  // then is the column left to the radix fallback.
  const bool stopped = cnt_smem[2] != 0ull;
  const bool overflow = stopped || kp > r.L;
  __syncthreads();
  // Sec. 4.4: the tiny counters add up to N exactly when every key is one
  // of the u sampled keys, i.e. when the column has exactly u distinct keys.
  int path;
  if (d == 3) path = (!overflow && kp == (unsigned long long)r.u) ? 3 : (overflow ? 8 : 7);
  else path = overflow ? 6 : 4;
  if (sc.lead()) {
    r.path = path;
    r.k_distinct = overflow ? 0ull : kp;
    r.n_pairs = stopped ? 0ull : kp;
  }
  if (stopped) {
    // The count stopped: clear the claimed slots; the caller runs the radix sort.
    reset_claimed(p, occ, sc);
    return kColumnRadix;
  }
  if (occ <= (unsigned)kRankPairs) {
    phase_rank_pairs<K>(p, occ, special, smem, sc);
    if (!sc.sync(c, epoch, p.timeout_ns)) return kColumnFailed;
    mark(c, 4, sc);
    reset_claimed(p, occ, sc);
    phase_emit<K>(p, kp, smem, sc);
    return kColumnDone;
  } else {
    int pairs_end = kColumnRadix;   // the radix sort of the pairs, unless the bucket sort ran
    if constexpr (kGrid) {
      if (bucket_sort_fits(p, sc.nparts())) {
        pairs_end = phase_bucket_pairs<K>(p, occ, special, kp, smem, epoch, sc);
        if (pairs_end == kColumnFailed) return kColumnFailed;
      }
    }
    if (pairs_end == kColumnDone) {
      mark(c, 4, sc);
      phase_emit<K>(p, kp, smem, sc);
      return kColumnDone;
    }
  }
  {
    // Gather the claimed slots into pair arrays and reset the table (the
    // bucket sort may have done so already), LSD radix, scan.
    K* ak = reinterpret_cast<K*>(p.pkeys_a);
    const unsigned long long G = sc.gthreads();
    const unsigned long long gt = sc.gthread();
    bool gathered = false;
    if constexpr (kGrid) gathered = bucket_sort_fits(p, sc.nparts());
    if (!gathered) {
      for (unsigned long long i = gt; i < occ; i += G) {
        const unsigned slot = __ldcg(p.claimed + i);
        ak[i] = (K)(long long)__ldcg(p.tkeys + slot);
        p.pvals_a[i] = __ldcg(p.tcounts + slot);
        p.tkeys[slot] = kEmpty64;
        p.tcounts[slot] = 0u;
      }
      if (special && gt == 0) {
        ak[occ] = KeyTraits<K>::min_key();
        p.pvals_a[occ] = (unsigned)special;
      }
      if (!sc.sync(c, epoch, p.timeout_ns)) return kColumnFailed;
    }
    if (!radix_sort<K, true>(p, ak, p.pvals_a, kp, reinterpret_cast<K*>(p.skeys), p.svals,
                             reinterpret_cast<K*>(p.pkeys_b), p.pvals_b, smem, epoch, sc))
      return kColumnFailed;
    if (!grid_scan_counts(p, p.svals, kp, smem, epoch, sc)) return kColumnFailed;
    mark(c, 4, sc);
  }
  phase_emit<K>(p, kp, smem, sc);
  return kColumnDone;
}

// The radix fallback of a column: keys -> out through the tmp buffer.
template <typename K, class S>
__device__ bool column_radix(const Params& p, unsigned char* smem, const S& sc, unsigned& epoch) {
  return radix_sort<K, false>(p, reinterpret_cast<const K*>(p.keys), nullptr, p.n,
                              reinterpret_cast<K*>(p.out), nullptr, reinterpret_cast<K*>(p.tmp),
                              nullptr, smem, epoch, sc);
}

// ---------------------------------------------------------------------------
// N < 2048, one CTA: the sampler statistics are still computed for the
// report, then IsMonotone and a shared-memory bitonic sort.
// ---------------------------------------------------------------------------
template <typename K>
__device__ void small_body(const Params& p, unsigned char* smem) {
  const K* keys = reinterpret_cast<const K*>(p.keys);
  K* out = reinterpret_cast<K*>(p.out);
  Record& r = p.ctrl->rec;
  phase_sample<K>(p, keys, smem);
  const int n = (int)p.n;
  long long* s = reinterpret_cast<long long*>(smem);
  for (int i = threadIdx.x; i < kSmallCap; i += blockDim.x) s[i] = i < n ? (long long)keys[i] : LLONG_MAX;
  __syncthreads();
  int asc = 1;
  for (int i = threadIdx.x; i + 1 < n; i += blockDim.x) asc &= (s[i] <= s[i + 1]);
  const int mono = __syncthreads_and(asc);
  if (threadIdx.x == 0) {
    r.dispatch = mono ? 1 : 2;
    r.path = mono ? 1 : 2;
  }
  if (p.mode == kModeEstimate) return;
  if (!mono) bitonic_sort_pairs(s, nullptr, kSmallCap);
  if (!(mono && (const void*)keys == (const void*)out))
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = (K)s[i];
  __syncthreads();
}

// The N < 2048 kernel needs the sampler's shared memory (kSampleSmem)
// and later the column itself (kSmallCap x 8 B).
constexpr int kSmallSmem = kSampleSmem + 1024;
static_assert(kSmallSmem >= kSmallCap * 8, "small-kernel shared memory");

}  // namespace cafs
