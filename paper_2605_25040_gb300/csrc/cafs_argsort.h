// Stable argsort (the permutation of Sec. 3.1's problem statement) on top of
// the count-and-emit pipeline: device parameters and host launchers.

#pragma once

#include "cafs_internal.h"

namespace cafs {

// One column's argsort: the sort's parameters plus the permutation and
// four scratch arrays of n 32-bit words each.
struct ArgsortParams {
  Params p;            // as for the sort (p.out receives the sorted keys)
  unsigned* perm;      // n: output, perm[j] = input position of the j-th key
  unsigned* rk;        // n: each key's rank among the distinct keys
  unsigned* iv;        // n: input positions (the payload sorted with the ranks)
  unsigned* tv;        // n: payload ping-pong of the radix passes
  unsigned* rk2;       // n: the sorted ranks (not needed afterwards)
};

cudaError_t prepare_argsort_kernels();
cudaError_t argsort_occupancy(int dtype, int* blocks_per_sm);
cudaError_t launch_argsort(const ArgsortParams& ap, int dtype, int grid, cudaStream_t s);
cudaError_t launch_small_argsort(const ArgsortParams& ap, int dtype, cudaStream_t s);

}  // namespace cafs
