// The CAFS count-and-emit frequency sort on one GB300 (sm_103a).
//
// One cooperative, persistent launch runs the whole pipeline of Sec. 4.1 for
// a column of N >= 2048 keys; phases are separated by a bounded grid barrier:
//
//   0  sampler + Chao1 + dispatcher record          (Alg. 2, Eq. 5, Eq. 6,
//                                                    Alg. 3; CTA 0)
//   1  IsMonotone full scan, only when the 1024 samples ascend (Alg. 3);
//      a sorted column is copied through (bypass)
//   2  count: tiny path (K_hat <= 8, u <= 8: register counters per thread,
//      Sec. 4.4) or main path (per-CTA shared-memory open-addressing table,
//      merged into a global table hashed with Eq. 4, Sec. 4.2); the global
//      table counts distinct keys and raises the overflow guard when they
//      exceed L = C/2 (Eq. 6, Alg. 4)
//   3  the K' (key, count) pairs are sorted by key (Alg. 4): one CTA in shared
//      memory when K' <= 8192, otherwise an LSD radix sort over all CTAs;
//      then an exclusive scan of the counts gives each run's output offset
//   4  emit: every output tile looks up its runs and writes them with 16-byte
//      streaming stores (the paper's fill_n per pair)
//   R  radix fallback (the paper's pdqsort: 2*K_hat > N, or the guard fired):
//      LSD radix sort, 8-bit digits, one-sweep passes with decoupled
//      look-back; passes whose digit is constant are skipped.
//
// Columns with N < 2048 are sorted by a single CTA in shared memory
// (Table 2: "sampling does not amortize").
//
// All device waits (grid barrier, look-back) are bounded by a timeout; a wait
// that runs out records kDevTimeout and the launch ends early.

#include <cstdio>

#include "cafs_device.cuh"
#include "cafs_internal.h"

namespace cafs {

// ---------------------------------------------------------------------------
// Phase 0: sampler, spectrum, Chao1, Eq. 6, provisional dispatch (CTA 0).
// ---------------------------------------------------------------------------
template <typename K>
__device__ void phase_sample(const Params& p, const K* keys, unsigned char* smem) {
  using T = KeyTraits<K>;
  long long* s = reinterpret_cast<long long*>(smem);           // 1024 samples
  int* wcount = reinterpret_cast<int*>(s + kSamples);           // 32 warp counts
  const int t = threadIdx.x;
  const unsigned long long n = p.n;
  const unsigned long long stride = n / kSamples > 0 ? n / kSamples : 1ull;
  const int ns = n < (unsigned long long)kSamples ? (int)n : kSamples;

  long long v = LLONG_MAX;
  if (t < ns) v = (long long)keys[(unsigned long long)t * stride];
  s[t] = v;
  __syncthreads();
  int asc = (t + 1 < ns) ? (s[t] <= s[t + 1]) : 1;
  const int hint = __syncthreads_and(asc);

  // Sort the samples; runs of equal values give the frequency spectrum.
  bitonic_sort_pairs(s, nullptr, kSamples);
  const int start = (t < ns) && (t == 0 || s[t] != s[t - 1]);
  int len = 0;
  if (start) {
    len = 1;
    while (t + len < ns && s[t + len] == s[t]) ++len;
  }
  const int u = __syncthreads_count(start);
  const int f1 = __syncthreads_count(start && len == 1);
  const int f2 = __syncthreads_count(start && len == 2);

  // The u <= 8 distinct sample values, ascending (kept for the tiny path).
  const unsigned ballot = __ballot_sync(0xffffffffu, start);
  if ((t & 31) == 0) wcount[t >> 5] = __popc(ballot);
  __syncthreads();
  Record& r = p.ctrl->rec;
  if (start && u <= kTinyMax) {
    int rank = __popc(ballot & lanemask_lt());
    for (int w = 0; w < (t >> 5); ++w) rank += wcount[w];
    r.tiny_keys[rank] = s[t];
  }
  if (t == 0) {
    const bool saturated = (u == kSamples);
    unsigned long long k_hat = saturated
        ? n
        : (unsigned long long)u + ((unsigned long long)f1 * f1) / (2ull * (f2 + 1));
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
    if (k_hat <= (unsigned long long)kTinyMax && u <= kTinyMax) d = 3;          // TINY
    else if (2ull * k_hat > n) d = 5;                                          // HIGH_ENTROPY
    else d = 4;                                                                // MAIN
    r.dispatch = d;
    r.path = d;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Element iteration over one CTA's contiguous share of a column, with 16-byte
// vector loads on the aligned interior and scalar loads on the ragged ends.
// ---------------------------------------------------------------------------
template <typename K, int U, typename F>
__device__ __forceinline__ void for_each_key(const K* keys, unsigned long long n, F&& f,
                                             const unsigned* abort_flag) {
  using T = KeyTraits<K>;
  using V = typename T::Vec;
  constexpr int VPE = T::kVec;
  const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
  unsigned long long head = ((16u - (addr & 15u)) & 15u) / sizeof(K);
  if (head > n) head = n;
  const unsigned long long nvec = (n - head) / VPE;
  const unsigned long long tail0 = head + nvec * VPE;
  const unsigned nb = gridDim.x, b = blockIdx.x;
  if (b == 0)
    for (unsigned long long i = threadIdx.x; i < head; i += blockDim.x) f(keys[i]);
  if (b == nb - 1)
    for (unsigned long long i = tail0 + threadIdx.x; i < n; i += blockDim.x) f(keys[i]);
  const unsigned long long v0 = nvec * b / nb, v1 = nvec * (b + 1) / nb;
  const V* vp = reinterpret_cast<const V*>(keys + head);
  for (unsigned long long base = v0; base < v1; base += (unsigned long long)kThreads * U) {
    if (abort_flag) {
      unsigned a = 0;
      if ((threadIdx.x & 31) == 0) a = ld_relaxed_u32(abort_flag);
      a = __shfl_sync(0xffffffffu, a, 0);
      if (a) break;
    }
    V buf[U];
    #pragma unroll
    for (int j = 0; j < U; ++j) {
      const unsigned long long v = base + (unsigned long long)j * kThreads + threadIdx.x;
      if (v < v1) buf[j] = __ldcs(vp + v);
    }
    #pragma unroll
    for (int j = 0; j < U; ++j) {
      const unsigned long long v = base + (unsigned long long)j * kThreads + threadIdx.x;
      if (v < v1) {
        K e[VPE];
        unpack(buf[j], e);
        #pragma unroll
        for (int q = 0; q < VPE; ++q) f(e[q]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Phase 1: IsMonotone (Alg. 3) over the whole column; early exit on the
// first descent found by any thread.
// ---------------------------------------------------------------------------
template <typename K>
__device__ void phase_monotone(const Params& p, const K* keys) {
  Ctrl* c = p.ctrl;
  const unsigned long long n = p.n;
  const unsigned long long G = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long gt = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
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
template <typename K>
__device__ void grid_copy(const K* src, K* dst, unsigned long long n) {
  using T = KeyTraits<K>;
  using V = typename T::Vec;
  const unsigned long long G = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long gt = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
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
__device__ __forceinline__ void global_insert(const Params& p, unsigned long long key64,
                                              unsigned inc, int logC, unsigned long long C,
                                              unsigned long long L) {
  Ctrl* c = p.ctrl;
  const unsigned long long mask = C - 1;
  const unsigned long long h = hash_slot(key64, logC);
  for (unsigned long long probe = 0; probe < C; ++probe) {
    const unsigned long long slot = (h + probe) & mask;
    const unsigned long long k = ld_relaxed_u64(p.tkeys + slot);
    if (k == key64) {
      atomicAdd(p.tcounts + slot, inc);
      return;
    }
    if (k == kEmpty64) {
      const unsigned long long old = atomicCAS(p.tkeys + slot, kEmpty64, key64);
      if (old == kEmpty64) {
        const unsigned idx = atomicAdd(&c->occupancy, 1u);
        if (idx < C) p.claimed[idx] = (unsigned)slot;
        atomicAdd(p.tcounts + slot, inc);
        if (idx >= L) atomicExch(&c->overflow, 1u);
        return;
      }
      if (old == key64) {
        atomicAdd(p.tcounts + slot, inc);
        return;
      }
    }
  }
  atomicExch(&c->overflow, 1u);
}

// ---------------------------------------------------------------------------
// Phase 2: count (tiny or main).
// ---------------------------------------------------------------------------
template <typename K>
__device__ void phase_count(const Params& p, const K* keys, unsigned char* smem, bool tiny) {
  using T = KeyTraits<K>;
  Ctrl* c = p.ctrl;
  const Record& r = c->rec;
  const unsigned long long C = r.C, L = r.L;
  const int logC = log2_pow2(C);
  const unsigned long long k_hat = r.k_hat;
  const K kmin = T::min_key();

  // Per-CTA shared table: S slots (power of two) with R privatised counter
  // replicas per slot (lane % R) so that hot keys do not serialise a warp.
  constexpr int kKeyBytes = sizeof(K);
  const int budget = kPipelineSmem - 4096;
  int S = 256;
  while (S < kLocalSlotsMax && (unsigned long long)S < 4ull * k_hat) S <<= 1;
  while (S > 256 && S * (kKeyBytes + 4) > budget) S >>= 1;
  int R = 32;
  while (R > 1 && S * (kKeyBytes + 4 * R) > budget) R >>= 1;
  const bool use_local = tiny || (k_hat <= (unsigned long long)(kLocalSlotsMax / 2));
  const int logS = log2_pow2(S);
  const unsigned limit = S / 2;

  K* lkeys = reinterpret_cast<K*>(smem);
  unsigned* lcnt = reinterpret_cast<unsigned*>(smem + (size_t)S * kKeyBytes);
  unsigned* misc = reinterpret_cast<unsigned*>(smem + (size_t)S * (kKeyBytes + 4 * R));
  unsigned* local_occ = misc;                                          // 1
  unsigned long long* tiny_tot = reinterpret_cast<unsigned long long*>(misc + 2);  // 8
  unsigned long long* red = tiny_tot + kTinyMax;                        // kWarps

  if (use_local) {
    for (int i = threadIdx.x; i < S; i += blockDim.x) lkeys[i] = kmin;
    for (int i = threadIdx.x; i < S * R; i += blockDim.x) lcnt[i] = 0u;
  }
  if (threadIdx.x == 0) *local_occ = 0u;
  if (threadIdx.x < kTinyMax) tiny_tot[threadIdx.x] = 0ull;
  __syncthreads();

  const int nt = tiny ? r.n_tiny : 0;
  K tk[kTinyMax];
  #pragma unroll
  for (int j = 0; j < kTinyMax; ++j) tk[j] = (K)r.tiny_keys[j < nt ? j : 0];
  unsigned tc[kTinyMax];
  #pragma unroll
  for (int j = 0; j < kTinyMax; ++j) tc[j] = 0u;
  unsigned long long special = 0, miss = 0;
  const int lane_rep = (threadIdx.x & 31) & (R - 1);

  auto local_insert = [&](K x) -> bool {
    const unsigned long long ux = (unsigned long long)(typename T::U)x;
    const unsigned long long h = hash_slot(ux, logS);
    bool reserved = false;
    for (int probe = 0; probe < S; ++probe) {
      const int slot = (int)((h + probe) & (unsigned long long)(S - 1));
      const K k = *reinterpret_cast<volatile K*>(lkeys + slot);
      if (k == x) {
        atomicAdd(lcnt + slot * R + lane_rep, 1u);
        return true;
      }
      if (k == kmin) {
        if (!reserved) {
          if (atomicAdd(local_occ, 1u) >= limit) return false;
          reserved = true;
        }
        K old;
        if constexpr (sizeof(K) == 8) {
          old = (K)atomicCAS(reinterpret_cast<unsigned long long*>(lkeys + slot),
                             (unsigned long long)kmin, (unsigned long long)x);
        } else {
          old = (K)atomicCAS(reinterpret_cast<unsigned*>(lkeys + slot), (unsigned)kmin,
                             (unsigned)x);
        }
        if (old == kmin || old == x) {
          atomicAdd(lcnt + slot * R + lane_rep, 1u);
          return true;
        }
      }
    }
    return false;
  };

  auto process = [&](K x) {
    if (tiny) {
      bool hit = false;
      #pragma unroll
      for (int j = 0; j < kTinyMax; ++j) {
        const bool e = (j < nt) && (x == tk[j]);
        tc[j] += e ? 1u : 0u;
        hit |= e;
      }
      if (hit) return;
      ++miss;
    }
    if (x == kmin) {
      ++special;
      return;
    }
    if (use_local && local_insert(x)) return;
    global_insert(p, (unsigned long long)(long long)x, 1u, logC, C, L);
  };

  for_each_key<K, 4>(keys, p.n, process, &c->overflow);
  __syncthreads();

  // Flush the shared table into the global table.
  if (use_local) {
    for (int i = threadIdx.x; i < S; i += blockDim.x) {
      const K k = lkeys[i];
      if (k != kmin) {
        unsigned tot = 0;
        for (int q = 0; q < R; ++q) tot += lcnt[i * R + q];
        if (tot) global_insert(p, (unsigned long long)(long long)k, tot, logC, C, L);
      }
    }
  }
  if (tiny) {
    #pragma unroll
    for (int j = 0; j < kTinyMax; ++j) {
      unsigned v = tc[j];
      v = __reduce_add_sync(0xffffffffu, v);
      if ((threadIdx.x & 31) == 0 && v) atomicAdd(tiny_tot + j, (unsigned long long)v);
    }
  }
  __syncthreads();
  if (tiny && threadIdx.x < nt) {
    const unsigned long long tot = tiny_tot[threadIdx.x];
    const K key = (K)r.tiny_keys[threadIdx.x];
    if (tot) {
      if (key == kmin) special += tot;
      else global_insert(p, (unsigned long long)(long long)key, (unsigned)tot, logC, C, L);
    }
  }
  const unsigned long long bs = block_sum(special, red);
  const unsigned long long bm = block_sum(miss, red);
  if (threadIdx.x == 0) {
    if (bs) atomicAdd(&c->special, bs);
    if (bm) atomicAdd(&c->miss, bm);
  }
}

// Reset the global-table slots claimed in this call (grid-stride).
__device__ void reset_claimed(const Params& p, unsigned occ) {
  const unsigned long long G = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long gt = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (unsigned long long i = gt; i < occ; i += G) {
    const unsigned slot = __ldcg(p.claimed + i);
    p.tkeys[slot] = kEmpty64;
    p.tcounts[slot] = 0u;
  }
}

// ---------------------------------------------------------------------------
// Phase 3a: K' <= kSmallPairs pairs sorted by CTA 0 in shared memory, then
// exclusive scan of the counts.  Pads (key max, count 0) fill up to a power
// of two; zero-count runs are skipped by the emit lookup.
// ---------------------------------------------------------------------------
template <typename K>
__device__ void phase_small_pairs(const Params& p, unsigned occ, unsigned long long special,
                                  unsigned char* smem) {
  using T = KeyTraits<K>;
  Ctrl* c = p.ctrl;
  const unsigned kp = occ + (special ? 1u : 0u);
  const int P = (int)bit_ceil_u64(kp);
  long long* sk = reinterpret_cast<long long*>(smem);
  unsigned* sc = reinterpret_cast<unsigned*>(sk + kSmallPairs);
  unsigned* scratch = sc + kSmallPairs;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    if (i < (int)occ) {
      const unsigned slot = __ldcg(p.claimed + i);
      sk[i] = (long long)__ldcg(p.tkeys + slot);
      sc[i] = __ldcg(p.tcounts + slot);
      p.tkeys[slot] = kEmpty64;
      p.tcounts[slot] = 0u;
    } else if (i == (int)occ && special) {
      sk[i] = (long long)T::min_key();
      sc[i] = (unsigned)special;
    } else {
      sk[i] = LLONG_MAX;
      sc[i] = 0u;
    }
  }
  __syncthreads();
  bitonic_sort_pairs(sk, sc, P);
  K* skeys = reinterpret_cast<K*>(p.skeys);
  unsigned carry = 0;
  for (int base = 0; base < P; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const unsigned v = i < P ? sc[i] : 0u;
    unsigned tot;
    const unsigned ex = block_exclusive_scan(v, scratch, &tot);
    if (i < P) {
      p.offsets[i] = carry + ex;
      skeys[i] = (K)sk[i];
    }
    carry += tot;
  }
  if (threadIdx.x == 0) {
    p.offsets[P] = (unsigned)p.n;
    c->rec.n_pairs = (unsigned long long)P;
  }
}

// ---------------------------------------------------------------------------
// LSD radix sort, 8-bit digits, stable one-sweep passes with decoupled
// look-back across tiles of kRadixTile items (all CTAs).
// ---------------------------------------------------------------------------
template <typename K>
__device__ __forceinline__ unsigned radix_digit(K k, int shift) {
  using T = KeyTraits<K>;
  const typename T::U u = (typename T::U)k ^ T::kSign;
  return (unsigned)(u >> shift) & (kRadixDigits - 1);
}

constexpr unsigned long long kFlagAgg = 1ull, kFlagIncl = 2ull;

template <typename K, bool PAY>
__device__ bool radix_pass(const Params& p, const K* in_k, const unsigned* in_v, K* out_k,
                           unsigned* out_v, unsigned long long n, int pass, unsigned tag,
                           unsigned char* smem) {
  Ctrl* c = p.ctrl;
  const int shift = pass * kRadixBits;
  const unsigned long long ntiles = (n + kRadixTile - 1) / kRadixTile;
  K* stage_k = reinterpret_cast<K*>(smem);
  unsigned* stage_v = reinterpret_cast<unsigned*>(stage_k + kRadixTile);
  unsigned short* wcnt = reinterpret_cast<unsigned short*>(stage_v + (PAY ? kRadixTile : 0));
  unsigned* tile_cnt = reinterpret_cast<unsigned*>(wcnt + kWarps * kRadixDigits);
  unsigned* tile_start = tile_cnt + kRadixDigits;
  unsigned* gbase = tile_start + kRadixDigits;
  unsigned* dstart = gbase + kRadixDigits;
  unsigned* scratch = dstart + kRadixDigits;  // kWarps
  unsigned* s_ticket = scratch + kWarps;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long tagbits = ((unsigned long long)(tag & 0x3FFFFFFFu)) << 34;

  // Global exclusive start of every digit for this pass.
  {
    const unsigned v = threadIdx.x < kRadixDigits ? c->hist[pass][threadIdx.x] : 0u;
    unsigned tot;
    const unsigned ex = block_exclusive_scan(v, scratch, &tot);
    if (threadIdx.x < kRadixDigits) dstart[threadIdx.x] = ex;
  }
  bool ok = true;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) *s_ticket = atomicAdd(&c->tickets[pass], 1u);
    __syncthreads();
    const unsigned long long tile = *s_ticket;
    if (tile >= ntiles) break;
    const unsigned long long base = tile * kRadixTile;
    // zero this warp's digit counters
    for (int d = lane; d < kRadixDigits; d += 32) wcnt[w * kRadixDigits + d] = 0;
    __syncwarp();
    K key[kRadixItems];
    unsigned val[kRadixItems];
    unsigned short rank[kRadixItems];
    unsigned dig[kRadixItems];
    #pragma unroll
    for (int j = 0; j < kRadixItems; ++j) {
      const unsigned long long idx = base + (unsigned long long)w * (32 * kRadixItems) + j * 32 + lane;
      const bool valid = idx < n;
      key[j] = valid ? __ldcg(in_k + idx) : (K)0;
      if constexpr (PAY) val[j] = valid ? __ldcg(in_v + idx) : 0u;
      dig[j] = valid ? radix_digit(key[j], shift) : (unsigned)kRadixDigits;
    }
    #pragma unroll
    for (int j = 0; j < kRadixItems; ++j) {
      const unsigned d = dig[j];
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      unsigned old = 0;
      if (d < (unsigned)kRadixDigits) old = wcnt[w * kRadixDigits + d];
      __syncwarp();
      const int leader = __ffs(peers) - 1;
      if (lane == leader && d < (unsigned)kRadixDigits)
        wcnt[w * kRadixDigits + d] = (unsigned short)(old + __popc(peers));
      __syncwarp();
      rank[j] = (unsigned short)(old + __popc(peers & lanemask_lt()));
    }
    __syncthreads();
    // Per digit: exclusive scan over warps, tile total.
    if (threadIdx.x < kRadixDigits) {
      unsigned run = 0;
      for (int q = 0; q < kWarps; ++q) {
        const unsigned x = wcnt[q * kRadixDigits + threadIdx.x];
        wcnt[q * kRadixDigits + threadIdx.x] = (unsigned short)run;
        run += x;
      }
      tile_cnt[threadIdx.x] = run;
    }
    __syncthreads();
    {
      const unsigned v = threadIdx.x < kRadixDigits ? tile_cnt[threadIdx.x] : 0u;
      unsigned tot;
      const unsigned ex = block_exclusive_scan(v, scratch, &tot);
      if (threadIdx.x < kRadixDigits) tile_start[threadIdx.x] = ex;
    }
    // Decoupled look-back: digit d's exclusive prefix over earlier tiles.
    if (threadIdx.x < kRadixDigits) {
      const int d = threadIdx.x;
      unsigned long long* st = p.lookback + tile * kRadixDigits + d;
      const unsigned agg = tile_cnt[d];
      unsigned excl = 0;
      if (tile == 0) {
        st_release_u64(st, tagbits | (kFlagIncl << 32) | agg);
      } else {
        st_release_u64(st, tagbits | (kFlagAgg << 32) | agg);
        long long look = (long long)tile - 1;
        const unsigned long long t0 = global_timer_ns();
        unsigned it = 0;
        while (look >= 0) {
          const unsigned long long wv = ld_acquire_u64(p.lookback + (unsigned long long)look * kRadixDigits + d);
          const unsigned long long flag = (wv >> 32) & 3ull;
          if ((wv & ~((1ull << 34) - 1)) != tagbits || flag == 0) {
            if ((++it & 63u) == 0 && global_timer_ns() - t0 > p.timeout_ns) {
              atomicExch(&c->rec.status, kDevTimeout);
              break;
            }
            continue;
          }
          excl += (unsigned)(wv & 0xFFFFFFFFull);
          if (flag == kFlagIncl) break;
          --look;
        }
        st_release_u64(st, tagbits | (kFlagIncl << 32) | (unsigned long long)(excl + agg));
      }
      gbase[d] = dstart[d] + excl - tile_start[d];
    }
    __syncthreads();
    // Scatter into shared memory in tile-sorted order.
    #pragma unroll
    for (int j = 0; j < kRadixItems; ++j) {
      const unsigned d = dig[j];
      if (d < (unsigned)kRadixDigits) {
        const unsigned pos = tile_start[d] + wcnt[w * kRadixDigits + d] + rank[j];
        stage_k[pos] = key[j];
        if constexpr (PAY) stage_v[pos] = val[j];
      }
    }
    __syncthreads();
    const unsigned cnt = (unsigned)((n - base) < (unsigned long long)kRadixTile ? (n - base) : kRadixTile);
    for (unsigned i = threadIdx.x; i < cnt; i += blockDim.x) {
      const K k = stage_k[i];
      const unsigned long long dst = (unsigned long long)(unsigned)(gbase[radix_digit(k, shift)] + i);
      __stcg(out_k + dst, k);
      if constexpr (PAY) __stcg(out_v + dst, stage_v[i]);
    }
    if (device_failed(c)) { ok = false; }
  }
  __syncthreads();
  return ok;
}

// Full LSD radix sort src -> dst (tmp as ping-pong), all CTAs.  Returns false
// if a barrier failed (the caller must return).
template <typename K, bool PAY>
__device__ bool radix_sort(const Params& p, const K* src_k, const unsigned* src_v,
                           unsigned long long n, K* dst_k, unsigned* dst_v, K* tmp_k,
                           unsigned* tmp_v, unsigned char* smem, unsigned& epoch,
                           unsigned tag_base) {
  using T = KeyTraits<K>;
  constexpr int NP = T::kPasses;
  Ctrl* c = p.ctrl;
  // Histogram of every digit of every pass.
  unsigned* sh = reinterpret_cast<unsigned*>(smem);
  for (int i = threadIdx.x; i < NP * kRadixDigits; i += blockDim.x) sh[i] = 0u;
  __syncthreads();
  {
    const unsigned long long G = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long gt = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (unsigned long long i = gt; i < n; i += G) {
      const typename T::U u = (typename T::U)__ldcg(src_k + i) ^ T::kSign;
      #pragma unroll
      for (int q = 0; q < NP; ++q) atomicAdd(sh + q * kRadixDigits + ((u >> (q * kRadixBits)) & 0xFF), 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NP * kRadixDigits; i += blockDim.x)
    if (sh[i]) atomicAdd(&c->hist[i / kRadixDigits][i % kRadixDigits], sh[i]);
  if (!grid_sync(c, epoch, p.timeout_ns)) return false;

  // Plan: a pass whose digit is the same for every key changes nothing.
  int active[NP];
  int na = 0;
  for (int q = 0; q < NP; ++q) {
    bool trivial = false;
    for (int d = 0; d < kRadixDigits; ++d)
      if ((unsigned long long)ld_relaxed_u32(&c->hist[q][d]) == n) { trivial = true; break; }
    if (!trivial) active[na++] = q;
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
    const unsigned tag = (p.gen << 4) | ((tag_base + (unsigned)active[a]) & 15u);
    radix_pass<K, PAY>(p, cur_k, cur_v, ok_, ov, n, active[a], tag, smem);
    if (!grid_sync(c, epoch, p.timeout_ns)) return false;
    cur_k = ok_;
    cur_v = ov;
  }
  if ((const void*)cur_k != (const void*)dst_k) {
    grid_copy<K>(cur_k, dst_k, n);
    if constexpr (PAY) {
      const unsigned long long G = (unsigned long long)gridDim.x * blockDim.x;
      const unsigned long long gt = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
      for (unsigned long long i = gt; i < n; i += G) dst_v[i] = __ldcg(cur_v + i);
    }
    if (!grid_sync(c, epoch, p.timeout_ns)) return false;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Scan of the sorted counts (large pair path): offsets[i] = sum of counts
// before i; offsets[kp] = n.  Two levels with one grid barrier.
// ---------------------------------------------------------------------------
__device__ bool grid_scan_counts(const Params& p, const unsigned* vals, unsigned long long kp,
                                 unsigned char* smem, unsigned& epoch) {
  Ctrl* c = p.ctrl;
  unsigned long long* scratch = reinterpret_cast<unsigned long long*>(smem);
  const unsigned b = blockIdx.x, nb = gridDim.x;
  const unsigned long long i0 = kp * b / nb, i1 = kp * (b + 1) / nb;
  unsigned long long s = 0;
  for (unsigned long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) s += __ldcg(vals + i);
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) c->chunk_sums[b] = s;
  if (!grid_sync(c, epoch, p.timeout_ns)) return false;
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
  return grid_sync(c, epoch, p.timeout_ns);
}

// ---------------------------------------------------------------------------
// Phase 4: emit.  Output tiles of kEmitTileVec 16-byte vectors; each CTA
// looks up the first and last run of each of its tiles (binary search on the
// run offsets), stages the tile's runs in shared memory and writes the
// vectors with streaming stores.
// ---------------------------------------------------------------------------
constexpr int kEmitTileVec = 4096;
constexpr int kEmitMaxTilesPerCta = 512;

// Largest j in [lo, hi] with off[j] <= x (off non-decreasing, off[lo] <= x).
__device__ __forceinline__ unsigned long long run_of(const unsigned* off, unsigned long long lo,
                                                     unsigned long long hi, unsigned long long x) {
  while (lo < hi) {
    const unsigned long long mid = (lo + hi + 1) >> 1;
    if ((unsigned long long)__ldcg(off + mid) <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename K>
__device__ void phase_emit(const Params& p, unsigned long long npairs, unsigned char* smem) {
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
  const unsigned nb = gridDim.x, b = blockIdx.x;

  if (b == 0)
    for (unsigned long long i = threadIdx.x; i < head; i += blockDim.x) out[i] = __ldcg(sk + run_of(off, 0, last, i));
  if (b == nb - 1)
    for (unsigned long long i = tail0 + threadIdx.x; i < n; i += blockDim.x) out[i] = __ldcg(sk + run_of(off, 0, last, i));

  const unsigned long long ntile = (nvec + kEmitTileVec - 1) / kEmitTileVec;
  unsigned* tj = reinterpret_cast<unsigned*>(smem);                     // 2 per local tile
  unsigned* soff = tj + 2 * kEmitMaxTilesPerCta;                        // kEmitStagePairs + 1
  K* skey = reinterpret_cast<K*>(soff + kEmitStagePairs + 2);           // kEmitStagePairs
  // skey must be 16-byte aligned for K = long long: soff block is (4096+2)*4 B.
  V* vout = reinterpret_cast<V*>(out + head);

  for (unsigned long long round = 0;; ++round) {
    const unsigned long long first_tile = (unsigned long long)b + round * kEmitMaxTilesPerCta * nb;
    if (first_tile >= ntile) break;
    // Look up the first and last run of up to kEmitMaxTilesPerCta tiles at once.
    for (int q = threadIdx.x; q < 2 * kEmitMaxTilesPerCta; q += blockDim.x) {
      const unsigned long long tile = first_tile + (unsigned long long)(q >> 1) * nb;
      if (tile < ntile) {
        const unsigned long long vb = tile * kEmitTileVec;
        const unsigned long long ve = (vb + kEmitTileVec < nvec) ? vb + kEmitTileVec : nvec;
        const unsigned long long e = (q & 1) ? head + ve * VPE - 1 : head + vb * VPE;
        tj[q] = (unsigned)run_of(off, 0, last, e);
      }
    }
    __syncthreads();
    for (int lt = 0; lt < kEmitMaxTilesPerCta; ++lt) {
      const unsigned long long tile = first_tile + (unsigned long long)lt * nb;
      if (tile >= ntile) break;
      const unsigned long long vb = tile * kEmitTileVec;
      const unsigned long long ve = (vb + kEmitTileVec < nvec) ? vb + kEmitTileVec : nvec;
      const unsigned j0 = tj[2 * lt], j1 = tj[2 * lt + 1];
      const unsigned m = j1 - j0 + 1;
      if (m == 1) {
        const V kv = splat(__ldcg(sk + j0));
        for (unsigned long long v = vb + threadIdx.x; v < ve; v += blockDim.x) __stcs(vout + v, kv);
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
template <typename K>
__global__ void __launch_bounds__(kThreads, 1) pipeline_kernel(Params p) {
  extern __shared__ __align__(16) unsigned char smem[];
  Ctrl* c = p.ctrl;
  const K* keys = reinterpret_cast<const K*>(p.keys);
  K* out = reinterpret_cast<K*>(p.out);
  unsigned epoch = 0;

  if ((p.test_flags & kTestSkipBarrier) && blockIdx.x == 0) return;  // test: never arrive

  if (blockIdx.x == 0) phase_sample<K>(p, keys, smem);
  if (!grid_sync(c, epoch, p.timeout_ns)) return;

  Record& r = c->rec;
  const int hint = r.sample_nondecreasing;
  if (hint) {
    phase_monotone<K>(p, keys);
    if (!grid_sync(c, epoch, p.timeout_ns)) return;
    if (ld_relaxed_u32(&c->inversion) == 0u) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        r.dispatch = 1;   // BYPASS_SORTED
        r.path = 1;
      }
      if (p.mode == kModeSort && (const void*)keys != (const void*)out) grid_copy<K>(keys, out, p.n);
      return;
    }
  }
  if (p.mode == kModeEstimate) return;

  const int d = r.dispatch;
  unsigned occ = 0;
  if (d == 3 || d == 4) {
    phase_count<K>(p, keys, smem, d == 3);
    if (!grid_sync(c, epoch, p.timeout_ns)) return;
    occ = ld_relaxed_u32(&c->occupancy);
    const unsigned long long special = ld_relaxed_u64(&c->special);
    const unsigned long long miss = ld_relaxed_u64(&c->miss);
    const unsigned long long kp = (unsigned long long)occ + (special ? 1ull : 0ull);
    const bool overflow = ld_relaxed_u32(&c->overflow) != 0u || kp > r.L;
    int path;
    if (d == 3) path = (miss == 0) ? 3 : (overflow ? 8 : 7);
    else path = overflow ? 6 : 4;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      r.path = path;
      r.k_distinct = overflow ? 0ull : kp;
    }
    if (!overflow) {
      unsigned long long npairs;
      if (kp <= (unsigned long long)kSmallPairs) {
        if (blockIdx.x == 0) phase_small_pairs<K>(p, occ, special, smem);
        if (!grid_sync(c, epoch, p.timeout_ns)) return;
        npairs = bit_ceil_u64(kp);
      } else {
        // Gather the claimed slots into pair arrays and reset the table.
        K* ak = reinterpret_cast<K*>(p.pkeys_a);
        const unsigned long long G = (unsigned long long)gridDim.x * blockDim.x;
        const unsigned long long gt = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
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
        if (!grid_sync(c, epoch, p.timeout_ns)) return;
        if (!radix_sort<K, true>(p, ak, p.pvals_a, kp, reinterpret_cast<K*>(p.skeys), p.svals,
                                 reinterpret_cast<K*>(p.pkeys_b), p.pvals_b, smem, epoch, 0u))
          return;
        if (!grid_scan_counts(p, p.svals, kp, smem, epoch)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) r.n_pairs = kp;
        npairs = kp;
      }
      phase_emit<K>(p, npairs, smem);
      return;
    }
    // Guard fired: clear the claimed slots, then fall back to radix.
    reset_claimed(p, occ);
  } else if (blockIdx.x == 0 && threadIdx.x == 0) {
    r.path = 5;  // HIGH_ENTROPY_RADIX
  }
  radix_sort<K, false>(p, keys, nullptr, p.n, out, nullptr, reinterpret_cast<K*>(p.tmp), nullptr,
                       smem, epoch, 8u);
}

// ---------------------------------------------------------------------------
// N < 2048: one CTA; the sampler statistics are still computed for the
// report, then IsMonotone and a shared-memory bitonic sort.
// ---------------------------------------------------------------------------
template <typename K>
__global__ void __launch_bounds__(kThreads, 1) small_kernel(Params p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const K* keys = reinterpret_cast<const K*>(p.keys);
  K* out = reinterpret_cast<K*>(p.out);
  Record& r = p.ctrl->rec;
  phase_sample<K>(p, keys, smem);
  const int n = (int)p.n;
  long long* s = reinterpret_cast<long long*>(smem);
  for (int i = threadIdx.x; i < 2 * kThreads; i += blockDim.x) s[i] = i < n ? (long long)keys[i] : LLONG_MAX;
  __syncthreads();
  int asc = 1;
  for (int i = threadIdx.x; i + 1 < n; i += blockDim.x) asc &= (s[i] <= s[i + 1]);
  const int mono = __syncthreads_and(asc);
  if (threadIdx.x == 0) {
    r.dispatch = mono ? 1 : 2;
    r.path = mono ? 1 : 2;
  }
  if (p.mode == kModeEstimate) return;
  if (!mono) bitonic_sort_pairs(s, nullptr, 2 * kThreads);
  if (mono && (const void*)keys == (const void*)out) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = (K)s[i];
}

__global__ void fill_u64_kernel(unsigned long long* p, unsigned long long n, unsigned long long v) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    p[i] = v;
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
cudaError_t prepare_kernels() {
  cudaError_t e;
  e = cudaFuncSetAttribute(pipeline_kernel<int>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPipelineSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(pipeline_kernel<long long>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPipelineSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(small_kernel<int>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kThreads * 8 + 256);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(small_kernel<long long>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kThreads * 8 + 256);
}

cudaError_t pipeline_occupancy(int dtype, int* blocks_per_sm) {
  if (dtype == 0)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, pipeline_kernel<int>, kThreads, kPipelineSmem);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, pipeline_kernel<long long>, kThreads, kPipelineSmem);
}

cudaError_t launch_pipeline(const Params& p, int dtype, int grid, cudaStream_t s) {
  Params copy = p;
  void* args[] = {&copy};
  if (dtype == 0)
    return cudaLaunchCooperativeKernel((const void*)pipeline_kernel<int>, dim3(grid), dim3(kThreads), args, kPipelineSmem, s);
  return cudaLaunchCooperativeKernel((const void*)pipeline_kernel<long long>, dim3(grid), dim3(kThreads), args, kPipelineSmem, s);
}

cudaError_t launch_small(const Params& p, int dtype, cudaStream_t s) {
  const int smem = 2 * kThreads * 8 + 256;
  if (dtype == 0) small_kernel<int><<<1, kThreads, smem, s>>>(p);
  else small_kernel<long long><<<1, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_fill_u64(unsigned long long* ptr, unsigned long long n, unsigned long long v, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  unsigned long long blocks = (n + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  fill_u64_kernel<<<(unsigned)blocks, 256, 0, s>>>(ptr, n, v);
  return cudaGetLastError();
}

}  // namespace cafs
