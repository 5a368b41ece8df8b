// Order-preserving maps of unsigned and IEEE-float keys onto signed integers
// of the same width.  The signed order of the image is the unsigned order,
// resp. the totalOrder of IEEE 754, of the keys; equal images are equal bit
// patterns.  Applying a map twice restores the keys.

#include <cstdint>

#include "cafs_transform.h"

namespace cafs {
namespace {

template <typename U>
__device__ __forceinline__ U order_map(U x, int kind) {
  constexpr U kSign = U(1) << (sizeof(U) * 8 - 1);
  if (kind == 1) return x ^ kSign;
  return (x & kSign) ? (x ^ (kSign - 1)) : x;   // negative: larger magnitude sorts first
}

// 16-byte vectors over the aligned body, scalars over the ragged head and tail.
template <typename U>
__global__ void order_map_kernel(const U* src, U* dst, unsigned long long n, unsigned long long head,
                                 unsigned long long nvec, int kind) {
  constexpr int VPE = 16 / sizeof(U);
  const unsigned long long G = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long gt = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const uint4* vs = reinterpret_cast<const uint4*>(src + head);
  uint4* vd = reinterpret_cast<uint4*>(dst + head);
  for (unsigned long long i = gt; i < nvec; i += G) {
    uint4 v = vs[i];
    U e[VPE];
    memcpy(e, &v, 16);
    #pragma unroll
    for (int q = 0; q < VPE; ++q) e[q] = order_map<U>(e[q], kind);
    memcpy(&v, e, 16);
    vd[i] = v;
  }
  for (unsigned long long i = gt; i < head; i += G) dst[i] = order_map<U>(src[i], kind);
  for (unsigned long long i = head + nvec * VPE + gt; i < n; i += G) dst[i] = order_map<U>(src[i], kind);
}

template <typename U>
cudaError_t launch_typed(const void* src, void* dst, unsigned long long n, int kind, cudaStream_t s) {
  constexpr int VPE = 16 / sizeof(U);
  const uintptr_t a = reinterpret_cast<uintptr_t>(src), b = reinterpret_cast<uintptr_t>(dst);
  unsigned long long head = 0, nvec = 0;
  if ((a & 15u) == (b & 15u)) {   // same misalignment: vectors line up for both
    head = ((16u - (a & 15u)) & 15u) / sizeof(U);
    if (head > n) head = n;
    nvec = (n - head) / VPE;
  } else {
    head = n;                     // scalar only
  }
  unsigned long long work = nvec ? nvec : n;
  unsigned long long blocks = (work + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  order_map_kernel<U><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const U*>(src), static_cast<U*>(dst), n, head,
                                                        nvec, kind);
  return cudaGetLastError();
}

}  // namespace

bool key_type_known(cafs_dtype t) { return t >= CAFS_INT32 && t <= CAFS_FLOAT64; }
size_t key_type_width(cafs_dtype t) { return (t == CAFS_INT64 || t == CAFS_UINT64 || t == CAFS_FLOAT64) ? 8 : 4; }
int key_type_base(cafs_dtype t) { return key_type_width(t) == 8 ? 1 : 0; }
int key_type_kind(cafs_dtype t) {
  return (t == CAFS_UINT32 || t == CAFS_UINT64) ? 1 : (t == CAFS_FLOAT32 || t == CAFS_FLOAT64) ? 2 : 0;
}

cudaError_t launch_order_map(const void* src, void* dst, unsigned long long n, int width, int kind,
                             cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (width == 8) return launch_typed<unsigned long long>(src, dst, n, kind, s);
  return launch_typed<unsigned>(src, dst, n, kind, s);
}

}  // namespace cafs
