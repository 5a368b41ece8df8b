// Order-preserving maps of unsigned and IEEE-float keys onto the signed
// integers of the same width (the pipeline sorts signed integers).

#pragma once

#include <cstddef>

#include <cuda_runtime.h>

#include "cafs.h"

namespace cafs {

// The C ABI's key types: known, element width in bytes, the signed type the
// kernels sort (0: int32, 1: int64) and the order map onto it (0: none,
// 1: unsigned, 2: IEEE float).
bool key_type_known(cafs_dtype t);
size_t key_type_width(cafs_dtype t);
int key_type_base(cafs_dtype t);
int key_type_kind(cafs_dtype t);

// Argument checks of one column for entry points that take every key type
// (defined in cafs_api.cu).
cafs_status check_args_typed(const void* keys, size_t n, cafs_dtype dtype, const void* out, bool need_out);

// kind: 1 = unsigned (flip the sign bit), 2 = IEEE float (flip the magnitude
// bits of values whose sign bit is set).  Both maps are their own inverse.
// width: 4 or 8 bytes.  src and dst may be equal (in place).
cudaError_t launch_order_map(const void* src, void* dst, unsigned long long n, int width, int kind,
                             cudaStream_t s);

}  // namespace cafs
