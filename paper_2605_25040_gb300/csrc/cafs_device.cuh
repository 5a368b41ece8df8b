// Device-side building blocks shared by the pipeline kernels: key traits, the
// multiplicative hash of Eq. 4, memory-ordering helpers, a bounded grid
// barrier, block scans and a shared-memory bitonic sort.
#pragma once

#include <climits>
#include <cstdint>

#include "cafs_internal.h"

namespace cafs {

template <typename K> struct KeyTraits;
template <> struct KeyTraits<int> {
  using U = unsigned;
  using Vec = int4;                       // 16-byte vector of keys
  static constexpr int kVec = 4;
  static constexpr int kCap = 8;          // Eq. 6: keys per 64-byte bucket
  static constexpr int kPasses = 4;       // 8-bit radix digits
  static constexpr U kSign = 0x80000000u;
  __device__ static constexpr int min_key() { return INT_MIN; }
};
template <> struct KeyTraits<long long> {
  using U = unsigned long long;
  using Vec = longlong2;
  static constexpr int kVec = 2;
  static constexpr int kCap = 4;
  static constexpr int kPasses = 8;
  static constexpr U kSign = 0x8000000000000000ull;
  __device__ static constexpr long long min_key() { return LLONG_MIN; }
};

// Eq. 4: multiplier 2^64 / golden ratio.
constexpr unsigned long long kPhi = 0x9E3779B97F4A7C15ull;
// Empty marker of the global table.  Keys equal to the type minimum never
// enter any table (they are counted on the side), so the marker is free.
constexpr unsigned long long kEmpty64 = 0x8000000000000000ull;

// Eq. 4: h(x) = ((x * phi^-1) mod 2^64) >> (64 - log2 M).
__device__ __forceinline__ unsigned long long hash_slot(unsigned long long x, int log2size) {
  return log2size == 0 ? 0ull : ((x * kPhi) >> (64 - log2size));
}
// Eq. 4 with another odd multiplier (a per-call hash seed; which slot a key
// lands in never changes a count, the result or the path).
__device__ __forceinline__ unsigned long long hash_slot_m(unsigned long long x, unsigned long long mult,
                                                          int log2size) {
  return log2size == 0 ? 0ull : ((x * mult) >> (64 - log2size));
}

// Bucket index in a per-CTA shared table of 2^log2size buckets: a 32-bit
// multiplicative hash of the key folded to 32 bits (the same golden-ratio
// multiplier as Eq. 4, 32-bit form).  Which bucket a key lands in never
// changes a count; a 32-bit product costs a third of Eq. 4's 64-bit one.
__device__ __forceinline__ unsigned local_bucket(unsigned x32, int log2size) {
  return (x32 * 0x9E3779B1u) >> (32 - log2size);
}
__device__ __forceinline__ unsigned local_bucket_m(unsigned x32, unsigned mult, int log2size) {
  return (x32 * mult) >> (32 - log2size);
}
__device__ __forceinline__ unsigned fold32(unsigned long long x) { return (unsigned)x ^ (unsigned)(x >> 32); }
__device__ __forceinline__ unsigned fold32(unsigned x) { return x; }

__device__ __forceinline__ void unpack(const int4& v, int* e) {
  e[0] = v.x; e[1] = v.y; e[2] = v.z; e[3] = v.w;
}
__device__ __forceinline__ void unpack(const longlong2& v, long long* e) {
  e[0] = v.x; e[1] = v.y;
}
__device__ __forceinline__ int4 pack(const int* e) { return make_int4(e[0], e[1], e[2], e[3]); }
__device__ __forceinline__ longlong2 pack(const long long* e) { return make_longlong2(e[0], e[1]); }
__device__ __forceinline__ int4 splat(int k) { return make_int4(k, k, k, k); }
__device__ __forceinline__ longlong2 splat(long long k) { return make_longlong2(k, k); }

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ unsigned long long bit_ceil_u64(unsigned long long x) {
  return x <= 1 ? 1ull : (1ull << (64 - __clzll(x - 1)));
}
__device__ __forceinline__ int log2_pow2(unsigned long long x) { return 63 - __clzll(x); }

__device__ __forceinline__ bool device_failed(const Ctrl* c) {
  return ld_relaxed_u32(&c->rec.status) != kDevOk;
}

// --- mbarrier / bulk-copy (TMA engine) helpers ------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's earlier generic-proxy shared-memory accesses before
// its later async-proxy (bulk copy) accesses of the same bytes.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Waits (suspended, up to ~0.1 ms per call) for phase `parity` of `bar`.
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0;
}
// Bulk copy global -> this CTA's shared memory, completion counted in bytes
// on `bar`.  Both addresses 16-byte aligned, `bytes` a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Bounded wait for phase `parity` of an mbarrier; on timeout records
// kDevTimeout and returns false.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          unsigned long long timeout_ns, Ctrl* c) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_timer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_timer_ns() - t0 > timeout_ns) {
      atomicExch(&c->rec.status, kDevTimeout);
      return false;
    }
  }
  return true;
}

// Grid-wide barrier for the cooperative (co-resident) pipeline grid.  The
// wait is bounded by `timeout_ns`; when it runs out the CTA records
// kDevTimeout in the control block and returns false instead of waiting on.
// Every caller returns from the kernel when the barrier reports failure, so
// a lost CTA ends the launch with an error status rather than a hang.
static __device__ __noinline__ bool grid_sync(Ctrl* c, unsigned& epoch, unsigned long long timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned e = epoch;
    __threadfence();
    unsigned arrived = atomicAdd(&c->bar_count, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(&c->bar_count, 0u);
      __threadfence();
      atomicExch(&c->bar_epoch, e + 1u);
    } else {
      unsigned long long t0 = global_timer_ns();
      unsigned it = 0;
      while (ld_acquire_u32(&c->bar_epoch) == e) {
        __nanosleep(40);
        if ((++it & 63u) == 0 && global_timer_ns() - t0 > timeout_ns) {
          atomicExch(&c->rec.status, kDevTimeout);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    epoch = e + 1u;
    if (device_failed(c)) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Block-wide sum of one value per thread (all threads receive the total).
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch /* >= kWarps */) {
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  T t = (l < kWarps) ? scratch[l] : T(0);
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive
// prefix and writes the block total to *total.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* scratch /* >= kWarps */, T* total) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  T x = v;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (l >= o) x += y;
  }
  __syncthreads();
  if (l == 31) scratch[w] = x;
  __syncthreads();
  if (w == 0) {
    T s = (l < kWarps) ? scratch[l] : T(0);
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, o);
      if (l >= o) s += y;
    }
    if (l < kWarps) scratch[l] = s;   // inclusive warp-total prefix
  }
  __syncthreads();
  T warp_base = (w > 0) ? scratch[w - 1] : T(0);
  *total = scratch[kWarps - 1];
  return warp_base + x - v;
}

// In-place ascending bitonic sort of `n` (a power of two) signed 64-bit keys
// with a 32-bit payload, by all threads of the block.
__device__ __forceinline__ void bitonic_sort_pairs(long long* k, unsigned* v, int n) {
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int j = i ^ stride;
        if (j > i) {
          bool up = (i & size) == 0;
          long long a = k[i], b = k[j];
          if ((a > b) == up) {
            k[i] = b; k[j] = a;
            if (v) { unsigned t = v[i]; v[i] = v[j]; v[j] = t; }
          }
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace cafs
