// Stable argsort: the permutation pi of Sec. 3.1's problem statement, with
// equal keys in input order.  The column first goes through the sort's own
// pipeline (Alg. 3: sample, dispatch, count, pair sort and scan, emit), which
// writes the sorted keys; then
//  - count paths (tiny, main): each key's rank among the K' sorted distinct
//    keys (binary search) is a small integer, and one stable LSD radix sort
//    of (rank, input position) pairs -- passes of constant digit skipped, so
//    one pass for K' <= 256, two for K' <= 65536 -- gives pi;
//  - radix paths (2 K_hat > N, guard fired): the LSD radix sorts (key, input
//    position) pairs directly;
//  - a sorted column (bypass): pi is the identity;
//  - N < 2048: one CTA counts, for each key, the keys that precede it.

#include "cafs_argsort.h"
#include "cafs_phases.cuh"

namespace cafs {

// Distinct keys ranked from shared memory (8 B each, 32 KB); more are
// searched in global memory.
constexpr unsigned kArgRankShared = kRankPairs + 1;

// Position of x in the ascending distinct keys sk[0, kp) (x is one of them).
template <typename K>
__device__ __forceinline__ unsigned rank_shared(const K* sk, unsigned kp, K x) {
  unsigned lo = 0, hi = kp;
  while (lo < hi) {
    const unsigned mid = (lo + hi) >> 1;
    if (sk[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
template <typename K>
__device__ __forceinline__ unsigned rank_global(const K* sk, unsigned kp, K x) {
  unsigned lo = 0, hi = kp;
  while (lo < hi) {
    const unsigned mid = (lo + hi) >> 1;
    if (__ldcg(sk + mid) < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// The radix sorts below start from empty digit counts and key bits.
__device__ __forceinline__ void clear_radix_state(Ctrl* c) {
  unsigned* h = &c->hist[0][0];
  for (int i = threadIdx.x; i < 8 * kRadixDigits; i += blockDim.x) h[i] = 0u;
  if (threadIdx.x == 0) {
    c->key_or = 0ull;
    c->key_nor = 0ull;
  }
}

template <typename K>
__global__ void __launch_bounds__(kThreads, 1) argsort_kernel(ArgsortParams ap) {
  extern __shared__ __align__(128) unsigned char smem[];
  const GridScope sc;
  const Params& p = ap.p;
  Ctrl* c = p.ctrl;
  zero_next_ctrl(p);
  mark(c, 0, sc);
  unsigned epoch = 0;
  const int end = column_body<K>(p, smem, sc, epoch);
  const unsigned long long n = p.n;
  const unsigned long long G = sc.gthreads(), gt = sc.gthread();
  const K* keys = reinterpret_cast<const K*>(p.keys);
  if (end == kColumnDone) {
    if (c->rec.path == 1) {
      // sorted input (the bypass): equal keys are already in input order
      for (unsigned long long i = gt; i < n; i += G) ap.perm[i] = (unsigned)i;
    } else {
      // The pair sort finished before the emit (a grid barrier lies between).
      const unsigned kp = (unsigned)c->rec.n_pairs;
      const K* sk = reinterpret_cast<const K*>(p.skeys);
      K* ssk = reinterpret_cast<K*>(smem);
      const bool in_shared = kp <= kArgRankShared;
      __syncthreads();   // the emit's shared memory
      if (in_shared) {
        for (unsigned j = threadIdx.x; j < kp; j += blockDim.x) ssk[j] = __ldcg(sk + j);
        __syncthreads();
      }
      for (unsigned long long i = gt; i < n; i += G) {
        const K x = keys[i];
        ap.rk[i] = in_shared ? rank_shared<K>(ssk, kp, x) : rank_global<K>(sk, kp, x);
        ap.iv[i] = (unsigned)i;
      }
      // the pair radix (K' > 4096) left its digit counts in the control block
      if (blockIdx.x == 0) clear_radix_state(c);
      if (sc.sync(c, epoch, p.timeout_ns))
        radix_sort<int, true>(p, reinterpret_cast<const int*>(ap.rk), ap.iv, n, reinterpret_cast<int*>(ap.rk2),
                              ap.perm, reinterpret_cast<int*>(p.tmp), ap.tv, smem, epoch, sc);
    }
  } else if (end == kColumnRadix) {
    for (unsigned long long i = gt; i < n; i += G) ap.iv[i] = (unsigned)i;
    if (blockIdx.x == 0) clear_radix_state(c);
    if (sc.sync(c, epoch, p.timeout_ns))
      radix_sort<K, true>(p, keys, ap.iv, n, reinterpret_cast<K*>(p.out), ap.perm, reinterpret_cast<K*>(p.tmp),
                          ap.tv, smem, epoch, sc);
  }
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(&c->rec.timeline[5], global_timer_ns());
}

// N < 2048, one CTA: the sort's small-column body (sorted keys, record),
// then pi[#{j : x_j < x_i or (x_j == x_i and j < i)}] = i.
template <typename K>
__global__ void __launch_bounds__(kThreads, 1) small_argsort_kernel(ArgsortParams ap) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Params& p = ap.p;
  zero_next_ctrl(p);
  small_body<K>(p, smem);
  __syncthreads();
  const K* keys = reinterpret_cast<const K*>(p.keys);
  const int n = (int)p.n;
  long long* s = reinterpret_cast<long long*>(smem);
  for (int i = threadIdx.x; i < n; i += blockDim.x) s[i] = (long long)keys[i];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const long long x = s[i];
    unsigned pos = 0;
    for (int j = 0; j < n; ++j) {
      const long long y = s[j];
      pos += (y < x || (y == x && j < i)) ? 1u : 0u;
    }
    ap.perm[pos] = (unsigned)i;
  }
}

cudaError_t prepare_argsort_kernels() {
  cudaError_t e;
  e = cudaFuncSetAttribute(argsort_kernel<int>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPipelineSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(argsort_kernel<long long>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPipelineSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(small_argsort_kernel<int>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmallSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(small_argsort_kernel<long long>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kSmallSmem);
}

cudaError_t argsort_occupancy(int dtype, int* blocks_per_sm) {
  if (dtype == 0)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, argsort_kernel<int>, kThreads, kPipelineSmem);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, argsort_kernel<long long>, kThreads,
                                                       kPipelineSmem);
}

cudaError_t launch_argsort(const ArgsortParams& ap, int dtype, int grid, cudaStream_t s) {
  ArgsortParams copy = ap;
  void* args[] = {&copy};
  if (dtype == 0)
    return cudaLaunchCooperativeKernel((const void*)argsort_kernel<int>, dim3(grid), dim3(kThreads), args,
                                       kPipelineSmem, s);
  return cudaLaunchCooperativeKernel((const void*)argsort_kernel<long long>, dim3(grid), dim3(kThreads), args,
                                     kPipelineSmem, s);
}

cudaError_t launch_small_argsort(const ArgsortParams& ap, int dtype, cudaStream_t s) {
  if (dtype == 0) small_argsort_kernel<int><<<1, kThreads, kSmallSmem, s>>>(ap);
  else small_argsort_kernel<long long><<<1, kThreads, kSmallSmem, s>>>(ap);
  return cudaGetLastError();
}

}  // namespace cafs
