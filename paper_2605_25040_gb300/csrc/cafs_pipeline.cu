// Single-column kernels of the CAFS sort and their host launchers: the
// cooperative persistent pipeline (N >= 2048, the whole grid works on one
// column, phases separated by the bounded grid barrier) and the one-CTA
// kernel for N < 2048.  The phases themselves are in cafs_phases.cuh.

#include "cafs_phases.cuh"

namespace cafs {

// Phase timeline (globaltimer ns): 0 start, 1 sampled, 2 monotone checked,
// 3 counted, 4 pairs sorted and scanned, 5 last CTA finished.
template <typename K>
__global__ void __launch_bounds__(kThreads, 1) pipeline_kernel(Params p) {
  extern __shared__ __align__(128) unsigned char smem[];
  const GridScope sc;
  zero_next_ctrl(p);
  mark(p.ctrl, 0, sc);
  if (!((p.test_flags & kTestSkipBarrier) && blockIdx.x == 0)) {  // test: CTA 0 never arrives
    unsigned epoch = 0;
    if (column_body<K>(p, smem, sc, epoch) == kColumnRadix) column_radix<K>(p, smem, sc, epoch);
  }
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(&p.ctrl->rec.timeline[5], global_timer_ns());
}

// ---------------------------------------------------------------------------
// N < 2048: one CTA.
// ---------------------------------------------------------------------------
template <typename K>
__global__ void __launch_bounds__(kThreads, 1) small_kernel(Params p) {
  extern __shared__ __align__(128) unsigned char smem[];
  zero_next_ctrl(p);
  small_body<K>(p, smem);
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
  e = cudaFuncSetAttribute(small_kernel<int>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmallSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(small_kernel<long long>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmallSmem);
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
  if (dtype == 0) small_kernel<int><<<1, kThreads, kSmallSmem, s>>>(p);
  else small_kernel<long long><<<1, kThreads, kSmallSmem, s>>>(p);
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
