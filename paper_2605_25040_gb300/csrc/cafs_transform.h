// Order-preserving maps of unsigned and IEEE-float keys onto the signed
// integers of the same width (the pipeline sorts signed integers).

#pragma once

#include <cuda_runtime.h>

namespace cafs {

// kind: 1 = unsigned (flip the sign bit), 2 = IEEE float (flip the magnitude
// bits of values whose sign bit is set).  Both maps are their own inverse.
// width: 4 or 8 bytes.  src and dst may be equal (in place).
cudaError_t launch_order_map(const void* src, void* dst, unsigned long long n, int width, int kind,
                             cudaStream_t s);

}  // namespace cafs
