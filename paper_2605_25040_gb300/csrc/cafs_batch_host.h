// Host-side pieces of the batched form shared by the batch entry points
// (cafs_batch.cu) and the request server (cafs_server.cu).
#pragma once

#include <cstdint>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "cafs_internal.h"

namespace cafs {

struct Tuning {
  unsigned long long grid_min_n = 0;        // 0: resolved per batch by make_schedule
  unsigned long long defer_min_n = 0;       // 0: resolve_defer() picks it per batch
  unsigned long long cta_table_slots = 0;   // 0: what the longest queue column can need
  unsigned local_slots_max = kLocalSlotsMax;
  unsigned replicas_max = kDefaultReplicasMax;
  unsigned emit_tile_vec = kEmitTileVecDefault;
  unsigned ctas = 0;   // 0: one per SM
};

// Device buffers of one batched launch configuration.
struct BatchBuffers {
  int device = -1;
  int grid = 0;
  SlotLayout gl{}, cl{};
  unsigned char* grid_slot = nullptr;
  unsigned char* cta_slots = nullptr;
  size_t col_cap = 0;
  BatchColumn* d_cols = nullptr;
  unsigned* d_items = nullptr;      // grid items, then queue items
  unsigned* d_deferred = nullptr;
  Record* d_records = nullptr;
  BatchState* d_state = nullptr;    // one per key type
  BatchColumn* h_cols = nullptr;    // pinned staging
  unsigned* h_items = nullptr;
  Record* h_records = nullptr;
  BatchState* h_state = nullptr;
  cudaEvent_t staged = nullptr;     // the last upload from the staging buffers has run
};

struct BatchDevice {
  bool ready = false;
  int grid = 0;   // one CTA per SM (the batched kernel's occupancy)
};

// The columns of one batch, validated and scheduled.
struct Schedule {
  std::vector<BatchColumn> cols;
  // Unsigned and float columns: their keys are mapped into `out` before the
  // launch, the kernels sort those signed images in place, and `out` is
  // mapped back after it.
  struct Mapped {
    const void* keys;
    void* out;
    unsigned long long n;
    cafs_dtype type;
  };
  std::vector<Mapped> mapped;
  std::vector<unsigned> grid_items, cta_items;
  unsigned long long n_max_grid = 0, n_max_cta = 0;
  unsigned long long sum_cta = 0;   // keys in the per-CTA queue
  unsigned n_grid32 = 0, n_cta32 = 0;   // int32 items come first in each list
};

// Validates and converts the public knobs (NULL = defaults).
cafs_status tuning_from(const cafs_batch_tuning* t, Tuning* out);
void tuning_to(const Tuning& d, cafs_batch_tuning* t);
// Validates the columns and orders the work: all-CTA columns, then the
// queue, longest first.  With grid_min_n 0 a column goes to the all-CTA
// stage when one CTA would take more than twice the batch's average work
// per CTA to sort it: n >= max(2^16, 2 * total keys / grid).
cafs_status make_schedule(const cafs_column* cols, size_t ncols, const Tuning& t, int grid, Schedule* s);
unsigned long long resolve_grid_min(const Tuning& t, unsigned long long total_keys, int grid);
// The set-aside threshold of a batch: the knob, or (knob 0) the length at
// which one CTA's radix sort of a column (about 17 passes over its keys)
// would take longer than about twice the queue's average work per CTA.
unsigned long long resolve_defer(const Tuning& t, const Schedule& s, int grid);
// CTAs of a batched launch on `dev` (one per SM); takes the batch lock.
cafs_status batch_grid(int dev, int* grid);
// Grows `b` for the schedule (device current; stream-ordered on s).
cafs_status ensure_batch(BatchBuffers* b, int grid, const Schedule& sc, const Tuning& t, cudaStream_t s);
void free_batch(BatchBuffers* b);
// Copies the schedule's descriptors to the device (asynchronously on s).
cafs_status upload(BatchBuffers* b, const Schedule& sc, cudaStream_t s);
// Launch parameters for the columns of one key type (0 int32, 1 int64).
BatchParams make_params(const BatchBuffers* b, const Schedule& sc, const Tuning& t, int dtype);
// The zeroing memsets and one cooperative launch per key type present.
cafs_status enqueue_batch(const BatchBuffers* b, const Schedule& sc, const Tuning& t, int grid,
                          cudaStream_t s, bool count, unsigned* launched);

}  // namespace cafs
