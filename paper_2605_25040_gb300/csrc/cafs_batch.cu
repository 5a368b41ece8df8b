// Batched form of the CAFS sort: many columns in one persistent cooperative
// launch per key type (the paper sorts one array per call; batching is this
// library's addition and leaves every column's integer result and path
// unchanged).
//
// One CTA per SM.  A launch works in three stages:
//   1  columns with n >= grid_min_n: all CTAs sort them together, one after
//      another, exactly like the single-column pipeline (grid barrier);
//   2  the other columns form a work queue, longest first; each CTA takes
//      whole columns and runs the same phases alone (phases separated by
//      __syncthreads), in its own workspace slot;  a column whose path ends
//      in the radix fallback with n >= defer_min_n is put aside;
//   3  the set-aside columns are radix-sorted by all CTAs together.
// Every wait is bounded, as in the single-column kernels.  A plan records
// the launches (and their zeroing memsets) once in a CUDA graph and replays
// them.

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "cafs_batch_host.h"
#include "cafs_phases.cuh"
#include "cafs_transform.h"

namespace cafs {

// ---------------------------------------------------------------------------
// Device side.
// ---------------------------------------------------------------------------
__device__ __forceinline__ Params column_params(const BatchColumn& col, unsigned char* slot,
                                                const SlotLayout& L, const BatchParams& bp) {
  Params p;
  p.keys = col.keys;
  p.out = col.out;
  p.n = col.n;
  p.ctrl = reinterpret_cast<Ctrl*>(slot + L.ctrl);
  p.ctrl_next = nullptr;
  p.tkeys = reinterpret_cast<unsigned long long*>(slot + L.tkeys);
  p.tcounts = reinterpret_cast<unsigned*>(slot + L.tcounts);
  p.claimed = reinterpret_cast<unsigned*>(slot + L.claimed);
  p.table_cap = L.table_cap;
  p.pkeys_a = slot + L.pka;
  p.pvals_a = reinterpret_cast<unsigned*>(slot + L.pva);
  p.pkeys_b = slot + L.pkb;
  p.pvals_b = reinterpret_cast<unsigned*>(slot + L.pvb);
  p.skeys = slot + L.sk;
  p.svals = reinterpret_cast<unsigned*>(slot + L.sv);
  p.offsets = reinterpret_cast<unsigned*>(slot + L.off);
  p.pair_cap = L.pair_cap;
  p.tmp = slot + L.tmp;
  p.lookback = reinterpret_cast<unsigned long long*>(slot + L.look);
  p.lookback_cap = L.lookback_cap;
  p.sample_keys = reinterpret_cast<long long*>(slot + L.sample);
  p.gen = 0;
  p.mode = kModeSort;
  p.test_flags = 0;
  p.local_slots_max = bp.local_slots_max;
  p.replicas_max = bp.replicas_max;
  p.emit_tile_vec = bp.emit_tile_vec;
  p.local_mult = bp.local_mult;
  p.timeout_ns = bp.timeout_ns;
  p.hash_mult = bp.hash_mult;
  return p;
}

static_assert(sizeof(Record) % 8 == 0, "Record copies as 8-byte words");

// CTA-wide copy of a column's record into the batch's record array.
__device__ __forceinline__ void copy_record(Record* dst, const Record* src) {
  const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(Record) / 8); i += blockDim.x) d[i] = __ldcg(s + i);
}

// CTA-wide reset of everything a column expects to find zero in its control
// block; the grid-barrier words are left alone.
__device__ __forceinline__ void clear_column_state(Ctrl* c) {
  unsigned long long* r = reinterpret_cast<unsigned long long*>(&c->rec);
  for (int i = threadIdx.x; i < (int)(sizeof(Record) / 8); i += blockDim.x) r[i] = 0ull;
  if (threadIdx.x == 0) {
    c->occupancy = 0u;
    c->overflow = 0u;
    c->inversion = 0u;
    c->special = 0ull;
    c->key_or = 0ull;
    c->key_nor = 0ull;
  }
  unsigned* h = &c->hist[0][0];
  for (int i = threadIdx.x; i < 8 * kRadixDigits; i += blockDim.x) h[i] = 0u;
}

__device__ __forceinline__ void note_failure(const BatchParams& bp, const Ctrl* c) {
  if (threadIdx.x == 0) {
    unsigned st = ld_relaxed_u32(&c->rec.status);
    if (st == kDevOk) st = kDevInternal;
    atomicCAS(&bp.state->status, kDevOk, st);
  }
}

template <typename K, class S>
__device__ __forceinline__ int run_body(const Params& p, unsigned char* smem, unsigned& epoch) {
  return column_body<K>(p, smem, S(), epoch);
}
template <typename K, class S>
__device__ __forceinline__ bool run_radix(const Params& p, unsigned char* smem, unsigned& epoch) {
  return column_radix<K>(p, smem, S(), epoch);
}

// Set-aside list entries: a column index, with this bit for a whole column.
constexpr unsigned kDeferWhole = 0x80000000u;

// One launch per key type present in the batch (the bodies of both types in
// one kernel would not fit the 64 registers a 1024-thread CTA can have).
template <typename K>
__global__ void __launch_bounds__(kThreads, 1) batch_kernel(BatchParams bp) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ Params s_p;
  __shared__ unsigned s_item;
  Ctrl* gc = reinterpret_cast<Ctrl*>(bp.grid_slot + bp.grid_layout.ctrl);
  unsigned epoch = 0;

  // Stage 1: long columns, all CTAs together.
  for (unsigned j = 0; j < bp.n_grid; ++j) {
    const unsigned col = __ldg(bp.grid_items + j);
    const BatchColumn cd = bp.cols[col];
    if (threadIdx.x == 0) s_p = column_params(cd, bp.grid_slot, bp.grid_layout, bp);
    __syncthreads();
    int end = run_body<K, GridScope>(s_p, smem, epoch);
    if (end == kColumnRadix) end = run_radix<K, GridScope>(s_p, smem, epoch) ? kColumnDone : kColumnFailed;
    const bool ok = end == kColumnDone && grid_sync(gc, epoch, bp.timeout_ns);
    if (blockIdx.x == 0) {
      copy_record(bp.records + col, &gc->rec);
      if (!ok) note_failure(bp, gc);
    }
    if (!ok) return;
    if (blockIdx.x == 0) clear_column_state(gc);
    if (!grid_sync(gc, epoch, bp.timeout_ns)) return;
  }

  // Stage 2: the work queue, one column per CTA at a time.
  {
    unsigned char* slot = bp.cta_slots + (size_t)blockIdx.x * bp.cta_layout.bytes;
    Ctrl* mc = reinterpret_cast<Ctrl*>(slot + bp.cta_layout.ctrl);
    clear_column_state(mc);
    __syncthreads();
    for (;;) {
      if (threadIdx.x == 0) s_item = atomicAdd(&bp.state->next, 1u);
      __syncthreads();
      const unsigned item = s_item;
      if (item >= bp.n_cta) break;
      const unsigned col = __ldg(bp.cta_items + item);
      const BatchColumn cd = bp.cols[col];
      if (threadIdx.x == 0) s_p = column_params(cd, slot, bp.cta_layout, bp);
      __syncthreads();
      int end = kColumnDone;
      if (cd.n < kSmallN) {
        small_body<K>(s_p, smem);
      } else {
        unsigned local_epoch = 0;
        end = run_body<K, CtaScope>(s_p, smem, local_epoch);
        if (end == kColumnTooBig) {
          // Its Eq. 6 table exceeds this slot's: all CTAs sort it in stage 3.
          if (threadIdx.x == 0) bp.deferred[atomicAdd(&bp.state->ndeferred, 1u)] = col | kDeferWhole;
          end = kColumnDone;
        } else if (end == kColumnRadix) {
          if (cd.n >= bp.defer_min_n) {
            if (threadIdx.x == 0) bp.deferred[atomicAdd(&bp.state->ndeferred, 1u)] = col;
            end = kColumnDone;
          } else {
            end = run_radix<K, CtaScope>(s_p, smem, local_epoch) ? kColumnDone : kColumnFailed;
          }
        }
      }
      __syncthreads();
      copy_record(bp.records + col, &mc->rec);
      if (end == kColumnFailed) note_failure(bp, mc);
      __syncthreads();
      if (end == kColumnFailed) break;   // this CTA takes no more columns
      clear_column_state(mc);
      __syncthreads();
    }
  }

  // Stage 3: set-aside columns, all CTAs together: radix-fallback columns
  // (their record is final) and whole columns whose table was too big for a
  // per-CTA slot (sorted from the start; their record is rewritten).
  if (!grid_sync(gc, epoch, bp.timeout_ns)) return;
  const unsigned nd = ld_relaxed_u32(&bp.state->ndeferred);
  for (unsigned j = 0; j < nd; ++j) {
    const unsigned entry = __ldcg(bp.deferred + j);
    const unsigned col = entry & ~kDeferWhole;
    const BatchColumn cd = bp.cols[col];
    if (threadIdx.x == 0) s_p = column_params(cd, bp.grid_slot, bp.grid_layout, bp);
    __syncthreads();
    bool ok;
    if (entry & kDeferWhole) {
      int end = run_body<K, GridScope>(s_p, smem, epoch);
      if (end == kColumnRadix) end = run_radix<K, GridScope>(s_p, smem, epoch) ? kColumnDone : kColumnFailed;
      ok = (end == kColumnDone) && grid_sync(gc, epoch, bp.timeout_ns);
      if (ok && blockIdx.x == 0) copy_record(bp.records + col, &gc->rec);
    } else {
      ok = run_radix<K, GridScope>(s_p, smem, epoch) && grid_sync(gc, epoch, bp.timeout_ns);
    }
    if (!ok) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned st = ld_relaxed_u32(&gc->rec.status);
        bp.records[col].status = st == kDevOk ? kDevInternal : st;
      }
      if (blockIdx.x == 0) note_failure(bp, gc);
      return;
    }
    if (blockIdx.x == 0) clear_column_state(gc);
    if (!grid_sync(gc, epoch, bp.timeout_ns)) return;
  }
}

// Empties the hash tables of `nslots` slots (key slots to the empty marker,
// counts to zero) in one launch.
__global__ void init_slots_kernel(unsigned char* base, unsigned nslots, SlotLayout L) {
  const unsigned long long per = L.table_cap;
  const unsigned long long total = per * nslots;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long s = i / per, j = i - s * per;
    unsigned char* slot = base + s * L.bytes;
    reinterpret_cast<unsigned long long*>(slot + L.tkeys)[j] = kEmpty64;
    reinterpret_cast<unsigned*>(slot + L.tcounts)[j] = 0u;
  }
}

cudaError_t prepare_batch_kernel() {
  cudaError_t e = cudaFuncSetAttribute(batch_kernel<int>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPipelineSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(batch_kernel<long long>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPipelineSmem);
}

cudaError_t batch_occupancy(int* blocks_per_sm) {
  int a = 0, b = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, batch_kernel<int>, kThreads, kPipelineSmem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batch_kernel<long long>, kThreads, kPipelineSmem);
  *blocks_per_sm = a < b ? a : b;
  return e;
}

cudaError_t launch_batch(const BatchParams& bp, int dtype, int grid, cudaStream_t s) {
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kPipelineSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return dtype == 1 ? cudaLaunchKernelEx(&cfg, batch_kernel<long long>, bp)
                    : cudaLaunchKernelEx(&cfg, batch_kernel<int>, bp);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
namespace {
constexpr unsigned long long align256(unsigned long long x) { return (x + 255) & ~255ull; }
}  // namespace

SlotLayout slot_layout(unsigned long long table_cap, unsigned long long tmp_keys, unsigned parts) {
  SlotLayout L;
  std::memset(&L, 0, sizeof(L));
  L.table_cap = table_cap < 64 ? 64 : table_cap;
  L.pair_cap = pair_capacity(L.table_cap);
  L.lookback_cap = radix_scratch_words(parts ? parts : 1);
  L.n_cap = tmp_keys;
  const unsigned long long pc = L.pair_cap;
  unsigned long long o = 0;
  L.ctrl = o;    o = align256(o + sizeof(Ctrl));
  L.tkeys = o;   o = align256(o + L.table_cap * 8);
  L.tcounts = o; o = align256(o + L.table_cap * 4);
  L.claimed = o; o = align256(o + L.table_cap * 4);
  L.look = o;    o = align256(o + L.lookback_cap * 8);
  L.sample = o;  o = align256(o + (unsigned long long)kSamples * 8);
  const unsigned long long region = o;
  L.pka = o; o = align256(o + pc * 8);
  L.pva = o; o = align256(o + pc * 4);
  L.pkb = o; o = align256(o + pc * 8);
  L.pvb = o; o = align256(o + pc * 4);
  L.sk = o;  o = align256(o + pc * 8);
  L.sv = o;  o = align256(o + pc * 4);
  L.off = o; o = align256(o + (pc + 2) * 4);
  L.tmp = region;
  const unsigned long long tmp_end = align256(region + tmp_keys * 8);
  L.bytes = o > tmp_end ? o : tmp_end;
  return L;
}



cafs_status tuning_from(const cafs_batch_tuning* t, Tuning* out) {
  Tuning d;
  if (t) {
    if (t->reserved != 0) return CAFS_ERR_INVALID_ARGUMENT;
    if (t->grid_min_n) {
      if (t->grid_min_n < kSmallN) return CAFS_ERR_INVALID_ARGUMENT;
      d.grid_min_n = t->grid_min_n;
    }
    if (t->defer_min_n) d.defer_min_n = t->defer_min_n;
    if (t->cta_table_slots) {
      const unsigned long long v = t->cta_table_slots;
      if (v < 64 || (v & (v - 1))) return CAFS_ERR_INVALID_ARGUMENT;
      d.cta_table_slots = v;
    }
    if (t->local_slots_max) {
      const unsigned v = t->local_slots_max;
      if (v < 256 || v > (unsigned)kLocalSlotsMax || (v & (v - 1))) return CAFS_ERR_INVALID_ARGUMENT;
      d.local_slots_max = v;
    }
    if (t->replicas_max) {
      const unsigned v = t->replicas_max;
      if (v > 32 || (v & (v - 1))) return CAFS_ERR_INVALID_ARGUMENT;
      d.replicas_max = v;
    }
    if (t->emit_tile_vec) {
      const unsigned v = t->emit_tile_vec;
      if (v % kThreads || v > kEmitTileVecMax) return CAFS_ERR_INVALID_ARGUMENT;
      d.emit_tile_vec = v;
    }
    d.ctas = t->ctas;
  }
  *out = d;
  return CAFS_OK;
}

void tuning_to(const Tuning& d, cafs_batch_tuning* t) {
  std::memset(t, 0, sizeof(*t));
  t->grid_min_n = d.grid_min_n;
  t->defer_min_n = d.defer_min_n;
  t->cta_table_slots = d.cta_table_slots;
  t->local_slots_max = d.local_slots_max;
  t->replicas_max = d.replicas_max;
  t->emit_tile_vec = d.emit_tile_vec;
  t->ctas = d.ctas;
}


void free_batch(BatchBuffers* b) {
  auto fd = [](auto*& p) { if (p) cudaFree((void*)p); p = nullptr; };
  auto fh = [](auto*& p) { if (p) cudaFreeHost((void*)p); p = nullptr; };
  fd(b->grid_slot); fd(b->cta_slots); fd(b->d_cols); fd(b->d_items); fd(b->d_deferred);
  fd(b->d_records); fd(b->d_state);
  fh(b->h_cols); fh(b->h_items); fh(b->h_records); fh(b->h_state);
  if (b->staged) cudaEventDestroy(b->staged);
  b->staged = nullptr;
  b->col_cap = 0;
  b->gl = SlotLayout{};
  b->cl = SlotLayout{};
}

std::mutex g_batch_mu;
std::map<int, BatchDevice> g_batch_dev;
std::map<std::pair<int, uintptr_t>, BatchBuffers*> g_batch_ws;

cafs_status batch_device(int dev, BatchDevice** out) {
  BatchDevice& d = g_batch_dev[dev];
  if (!d.ready) {
    if (prepare_kernels() != cudaSuccess || prepare_batch_kernel() != cudaSuccess) return CAFS_ERR_CUDA;
    int sms = 0, bps = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CAFS_ERR_CUDA;
    if (batch_occupancy(&bps) != cudaSuccess || bps < 1) return CAFS_ERR_CUDA;
    long long g = (long long)sms * bps;
    if (g > kMaxGrid) g = kMaxGrid;
    d.grid = (int)g;
    d.ready = true;
  }
  *out = &d;
  return CAFS_OK;
}

cafs_status batch_grid(int dev, int* grid) {
  std::lock_guard<std::mutex> lock(g_batch_mu);
  BatchDevice* d = nullptr;
  const cafs_status st = batch_device(dev, &d);
  if (st == CAFS_OK) *grid = d->grid;
  return st;
}


unsigned long long resolve_grid_min(const Tuning& t, unsigned long long total_keys, int grid) {
  if (t.grid_min_n) return t.grid_min_n;
  return std::max(1ull << 16, 2ull * total_keys / (unsigned long long)(grid > 0 ? grid : 1));
}

cafs_status make_schedule(const cafs_column* cols, size_t ncols, const Tuning& t, int grid, Schedule* s) {
  s->cols.clear();
  s->mapped.clear();
  s->grid_items.clear();
  s->cta_items.clear();
  s->n_max_grid = s->n_max_cta = s->sum_cta = 0;
  s->n_grid32 = s->n_cta32 = 0;
  if (ncols && !cols) return CAFS_ERR_INVALID_ARGUMENT;
  if (ncols > 0xFFFFFFF0ull) return CAFS_ERR_TOO_LARGE;
  s->cols.resize(ncols);
  unsigned long long total = 0;
  for (size_t i = 0; i < ncols; ++i) {
    const cafs_column& c = cols[i];
    if (c.reserved != 0) return CAFS_ERR_INVALID_ARGUMENT;
    cafs_status st = check_args_typed(c.keys, c.n, c.dtype, c.out, true);
    if (st != CAFS_OK) return st;
    total += c.n;
  }
  const unsigned long long grid_min = resolve_grid_min(t, total, grid);
  for (size_t i = 0; i < ncols; ++i) {
    const cafs_column& c = cols[i];
    BatchColumn& b = s->cols[i];
    // unsigned and float columns: their signed images are sorted in place in out
    const bool mapped = key_type_kind(c.dtype) != 0 && c.n != 0;
    if (mapped) s->mapped.push_back(Schedule::Mapped{c.keys, c.out, (unsigned long long)c.n, c.dtype});
    b.keys = mapped ? c.out : c.keys;
    b.out = c.out;
    b.n = c.n;
    b.dtype = (unsigned)key_type_base(c.dtype);
    b.pad = 0;
    if (c.n == 0) continue;
    if ((unsigned long long)c.n >= grid_min) {
      s->grid_items.push_back((unsigned)i);
      s->n_max_grid = std::max(s->n_max_grid, (unsigned long long)c.n);
    } else {
      s->cta_items.push_back((unsigned)i);
      s->n_max_cta = std::max(s->n_max_cta, (unsigned long long)c.n);
      s->sum_cta += c.n;
    }
  }
  // int32 columns first (one launch per key type), then longest first
  // within each type: the queue's tail ends with the shortest columns.
  auto order = [&](unsigned a, unsigned b) {
    if (s->cols[a].dtype != s->cols[b].dtype) return s->cols[a].dtype < s->cols[b].dtype;
    return s->cols[a].n > s->cols[b].n;
  };
  std::stable_sort(s->cta_items.begin(), s->cta_items.end(), order);
  std::stable_partition(s->grid_items.begin(), s->grid_items.end(),
                        [&](unsigned a) { return s->cols[a].dtype == 0; });
  s->n_grid32 = (unsigned)std::count_if(s->grid_items.begin(), s->grid_items.end(),
                                        [&](unsigned a) { return s->cols[a].dtype == 0; });
  s->n_cta32 = (unsigned)std::count_if(s->cta_items.begin(), s->cta_items.end(),
                                       [&](unsigned a) { return s->cols[a].dtype == 0; });
  return CAFS_OK;
}

unsigned long long resolve_defer(const Tuning& t, const Schedule& s, int grid) {
  if (t.defer_min_n) return t.defer_min_n;
  const unsigned long long fair = s.sum_cta / (2ull * (unsigned long long)(grid > 0 ? grid : 1));
  return std::max(1ull << 15, fair);
}

// Grows `b` to hold the schedule (call with g_batch_mu held, device current).
cafs_status ensure_batch(BatchBuffers* b, int grid, const Schedule& sc, const Tuning& t,
                         cudaStream_t s) {
  const unsigned long long ncols = sc.cols.size();
  // The all-CTA slot also sorts the set-aside queue columns.
  const unsigned long long n_grid_slot = std::max(sc.n_max_grid, sc.n_max_cta);
  const SlotLayout gl = slot_layout(table_capacity_any(n_grid_slot), n_grid_slot, (unsigned)grid);
  unsigned long long cta_table = table_capacity_any(sc.n_max_cta);
  if (t.cta_table_slots && t.cta_table_slots < cta_table) cta_table = t.cta_table_slots;
  const SlotLayout cl = slot_layout(cta_table, std::min(sc.n_max_cta, resolve_defer(t, sc, grid)), 1);
  const bool grow_grid = !b->grid_slot || gl.bytes > b->gl.bytes || gl.table_cap > b->gl.table_cap ||
                         gl.pair_cap > b->gl.pair_cap || gl.n_cap > b->gl.n_cap ||
                         gl.lookback_cap > b->gl.lookback_cap;
  const bool grow_cta = !b->cta_slots || grid != b->grid || cl.bytes > b->cl.bytes ||
                        cl.table_cap > b->cl.table_cap || cl.pair_cap > b->cl.pair_cap ||
                        cl.n_cap > b->cl.n_cap;
  const bool grow_cols = ncols > b->col_cap || !b->d_state;
  if ((grow_grid || grow_cta || grow_cols) && (b->grid_slot || b->cta_slots || b->d_cols)) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return CAFS_ERR_CUDA;
  }
  if (grow_grid) {
    if (b->grid_slot) cudaFree(b->grid_slot);
    b->grid_slot = nullptr;
    const SlotLayout L = slot_layout(std::max(gl.table_cap, b->gl.table_cap), std::max(gl.n_cap, b->gl.n_cap),
                                     (unsigned)grid);
    if (cudaMalloc((void**)&b->grid_slot, L.bytes) != cudaSuccess) {
      cudaGetLastError();
      b->gl = SlotLayout{};
      return CAFS_ERR_OUT_OF_MEMORY;
    }
    b->gl = L;
    init_slots_kernel<<<1024, 256, 0, s>>>(b->grid_slot, 1u, L);
    if (cudaGetLastError() != cudaSuccess) return CAFS_ERR_CUDA;
    count_launches(1);
  }
  if (grow_cta) {
    if (b->cta_slots) cudaFree(b->cta_slots);
    b->cta_slots = nullptr;
    const bool same = grid == b->grid;
    const SlotLayout L = slot_layout(std::max(cl.table_cap, same ? b->cl.table_cap : 0ull),
                                     std::max(cl.n_cap, same ? b->cl.n_cap : 0ull), 1);
    if (cudaMalloc((void**)&b->cta_slots, L.bytes * (size_t)grid) != cudaSuccess) {
      cudaGetLastError();
      b->cl = SlotLayout{};
      return CAFS_ERR_OUT_OF_MEMORY;
    }
    b->cl = L;
    b->grid = grid;
    init_slots_kernel<<<4096, 256, 0, s>>>(b->cta_slots, (unsigned)grid, L);
    if (cudaGetLastError() != cudaSuccess) return CAFS_ERR_CUDA;
    count_launches(1);
  }
  if (grow_cols) {
    const size_t cap = std::max<size_t>(std::max<size_t>(ncols, 64), b->col_cap);
    auto fd = [](auto*& p) { if (p) cudaFree((void*)p); p = nullptr; };
    auto fh = [](auto*& p) { if (p) cudaFreeHost((void*)p); p = nullptr; };
    fd(b->d_cols); fd(b->d_items); fd(b->d_deferred); fd(b->d_records); fd(b->d_state);
    fh(b->h_cols); fh(b->h_items); fh(b->h_records);
    b->col_cap = 0;
    const bool ok = cudaMalloc((void**)&b->d_cols, cap * sizeof(BatchColumn)) == cudaSuccess &&
                    cudaMalloc((void**)&b->d_items, cap * sizeof(unsigned)) == cudaSuccess &&
                    cudaMalloc((void**)&b->d_deferred, cap * sizeof(unsigned)) == cudaSuccess &&
                    cudaMalloc((void**)&b->d_records, cap * sizeof(Record)) == cudaSuccess &&
                    cudaMalloc((void**)&b->d_state, 2 * sizeof(BatchState)) == cudaSuccess &&
                    cudaMallocHost((void**)&b->h_cols, cap * sizeof(BatchColumn)) == cudaSuccess &&
                    cudaMallocHost((void**)&b->h_items, cap * sizeof(unsigned)) == cudaSuccess &&
                    cudaMallocHost((void**)&b->h_records, cap * sizeof(Record)) == cudaSuccess &&
                    (b->h_state || cudaMallocHost((void**)&b->h_state, 2 * sizeof(BatchState)) == cudaSuccess);
    if (!ok) {
      cudaGetLastError();
      return CAFS_ERR_OUT_OF_MEMORY;
    }
    b->col_cap = cap;
  }
  if (!b->staged && cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming) != cudaSuccess)
    return CAFS_ERR_CUDA;
  return CAFS_OK;
}

// Copies the schedule to the device buffers (asynchronously on s).
cafs_status upload(BatchBuffers* b, const Schedule& sc, cudaStream_t s) {
  const size_t ncols = sc.cols.size();
  const size_t nitems = sc.grid_items.size() + sc.cta_items.size();
  if (ncols > b->col_cap || nitems > ncols) return CAFS_ERR_INTERNAL;
  if (cudaEventSynchronize(b->staged) != cudaSuccess) return CAFS_ERR_CUDA;  // staging free again
  if (ncols) std::memcpy(b->h_cols, sc.cols.data(), ncols * sizeof(BatchColumn));
  if (!sc.grid_items.empty())
    std::memcpy(b->h_items, sc.grid_items.data(), sc.grid_items.size() * sizeof(unsigned));
  if (!sc.cta_items.empty())
    std::memcpy(b->h_items + sc.grid_items.size(), sc.cta_items.data(), sc.cta_items.size() * sizeof(unsigned));
  if (ncols && cudaMemcpyAsync(b->d_cols, b->h_cols, ncols * sizeof(BatchColumn), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return CAFS_ERR_CUDA;
  if (nitems && cudaMemcpyAsync(b->d_items, b->h_items, nitems * sizeof(unsigned), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return CAFS_ERR_CUDA;
  if (cudaEventRecord(b->staged, s) != cudaSuccess) return CAFS_ERR_CUDA;
  return CAFS_OK;
}

BatchParams make_params(const BatchBuffers* b, const Schedule& sc, const Tuning& t, int dtype) {
  BatchParams bp;
  std::memset(&bp, 0, sizeof(bp));
  const size_t ng = sc.grid_items.size(), nq = sc.cta_items.size();
  bp.cols = b->d_cols;
  bp.grid_items = b->d_items + (dtype == 1 ? sc.n_grid32 : 0u);
  bp.cta_items = b->d_items + ng + (dtype == 1 ? sc.n_cta32 : 0u);
  bp.deferred = b->d_deferred;
  bp.records = b->d_records;
  bp.state = b->d_state + dtype;
  bp.grid_slot = b->grid_slot;
  bp.cta_slots = b->cta_slots;
  bp.grid_layout = b->gl;
  bp.cta_layout = b->cl;
  bp.n_grid = dtype == 1 ? (unsigned)ng - sc.n_grid32 : sc.n_grid32;
  bp.n_cta = dtype == 1 ? (unsigned)nq - sc.n_cta32 : sc.n_cta32;
  // A queue column sorted by its own CTA's radix must fit the slot's buffer.
  bp.defer_min_n = std::min(resolve_defer(t, sc, b->grid), b->cl.n_cap + 1);
  bp.local_slots_max = t.local_slots_max;
  bp.replicas_max = t.replicas_max;
  bp.emit_tile_vec = t.emit_tile_vec;
  bp.timeout_ns = wait_timeout_ns();
  next_hash_multipliers(&bp.hash_mult, &bp.local_mult);
  return bp;
}

// The zeroing memsets and the launch (what a plan's graph records).
cafs_status enqueue_batch(const BatchBuffers* b, const Schedule& sc, const Tuning& t, int grid,
                          cudaStream_t s, bool count, unsigned* launched) {
  const size_t ncols = sc.cols.size();
  unsigned nl = 0;
  for (const Schedule::Mapped& m : sc.mapped) {   // signed images of unsigned / float keys
    if (launch_order_map(m.keys, m.out, m.n, (int)key_type_width(m.type), key_type_kind(m.type), s) != cudaSuccess)
      return CAFS_ERR_CUDA;
    ++nl;
  }
  if (cudaMemsetAsync(b->d_state, 0, 2 * sizeof(BatchState), s) != cudaSuccess) return CAFS_ERR_CUDA;
  if (ncols && cudaMemsetAsync(b->d_records, 0, ncols * sizeof(Record), s) != cudaSuccess) return CAFS_ERR_CUDA;
  for (int dtype = 0; dtype < 2; ++dtype) {
    const BatchParams bp = make_params(b, sc, t, dtype);
    if (bp.n_grid == 0 && bp.n_cta == 0) continue;
    // the grid barrier's words start from zero in every launch
    if (cudaMemsetAsync(b->grid_slot + b->gl.ctrl, 0, sizeof(Ctrl), s) != cudaSuccess) return CAFS_ERR_CUDA;
    if (launch_batch(bp, dtype, grid, s) != cudaSuccess) return CAFS_ERR_CUDA;
    ++nl;
  }
  for (const Schedule::Mapped& m : sc.mapped) {   // the sorted images back to keys
    if (launch_order_map(m.out, m.out, m.n, (int)key_type_width(m.type), key_type_kind(m.type), s) != cudaSuccess)
      return CAFS_ERR_CUDA;
    ++nl;
  }
  if (count) count_launches(nl);
  if (launched) *launched = nl;
  return CAFS_OK;
}

// Reads the records back (blocking) and fills the reports.
cafs_status read_reports(BatchBuffers* b, const Schedule& sc, cafs_report* reports, cudaStream_t s) {
  const size_t ncols = sc.cols.size();
  if (ncols && cudaMemcpyAsync(b->h_records, b->d_records, ncols * sizeof(Record), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CAFS_ERR_CUDA;
  if (cudaMemcpyAsync(b->h_state, b->d_state, 2 * sizeof(BatchState), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CAFS_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CAFS_ERR_CUDA;
  BatchState st = b->h_state[0];
  if (st.status == kDevOk) st.status = b->h_state[1].status;
  for (size_t i = 0; i < ncols; ++i) {
    if (sc.cols[i].n == 0) {
      std::memset(&reports[i], 0, sizeof(cafs_report));
      reports[i].path = CAFS_PATH_EMPTY;
      reports[i].est.dispatch = CAFS_PATH_EMPTY;
      continue;
    }
    fill_report(b->h_records[i], &reports[i]);
    if (st.status != kDevOk && reports[i].device_status == CAFS_OK)
      reports[i].device_status = (cafs_status)st.status;
  }
  return CAFS_OK;
}

}  // namespace cafs

using namespace cafs;

struct cafs_batch_plan {
  int device = -1;
  Tuning tuning;
  Schedule sched;
  BatchBuffers buf;
  unsigned launches = 0;   // kernels one replay launches
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::mutex mu;
};

extern "C" {

cafs_status cafs_batch_tuning_default(cafs_batch_tuning* t) {
  if (!t) return CAFS_ERR_INVALID_ARGUMENT;
  tuning_to(Tuning{}, t);
  return CAFS_OK;
}

cafs_status cafs_sort_batch_tuned(const cafs_column* cols, size_t ncols, const cafs_batch_tuning* tuning,
                                  cafs_report* reports, void* stream) {
  Tuning t;
  cafs_status st = tuning_from(tuning, &t);
  if (st != CAFS_OK) return st;
  Schedule sc;
  // Argument errors first, before any CUDA call; then the real schedule.
  if ((st = make_schedule(cols, ncols, t, 1, &sc)) != CAFS_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_batch_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CAFS_ERR_CUDA;
  BatchDevice* d = nullptr;
  if ((st = batch_device(dev, &d)) != CAFS_OK) return st;
  int grid = d->grid;
  if (t.ctas && (int)t.ctas < grid) grid = (int)t.ctas;
  if ((st = make_schedule(cols, ncols, t, grid, &sc)) != CAFS_OK) return st;
  auto key = std::make_pair(dev, reinterpret_cast<uintptr_t>(s));
  BatchBuffers*& b = g_batch_ws[key];
  if (!b) {
    b = new BatchBuffers();
    b->device = dev;
  }
  if ((st = ensure_batch(b, grid, sc, t, s)) != CAFS_OK) return st;
  if ((st = upload(b, sc, s)) != CAFS_OK) return st;
  if ((st = enqueue_batch(b, sc, t, grid, s, true, nullptr)) != CAFS_OK) return st;
  if (reports) return read_reports(b, sc, reports, s);
  return CAFS_OK;
}

cafs_status cafs_sort_batch(const cafs_column* cols, size_t ncols, cafs_report* reports, void* stream) {
  return cafs_sort_batch_tuned(cols, ncols, nullptr, reports, stream);
}

cafs_status cafs_batch_plan_create(const cafs_column* cols, size_t ncols, const cafs_batch_tuning* tuning,
                                   cafs_batch_plan** out) {
  if (!out) return CAFS_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  cafs_batch_plan* pl = new cafs_batch_plan();
  cafs_status st = tuning_from(tuning, &pl->tuning);
  if (st == CAFS_OK) st = make_schedule(cols, ncols, pl->tuning, 1, &pl->sched);
  if (st != CAFS_OK) {
    delete pl;
    return st;
  }
  cudaStream_t s = nullptr;
  auto fail = [&](cafs_status e) {
    if (s) cudaStreamDestroy(s);
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    free_batch(&pl->buf);
    delete pl;
    return e;
  };
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(CAFS_ERR_CUDA);
  pl->device = dev;
  int grid = 0;
  if ((st = batch_grid(dev, &grid)) != CAFS_OK) return fail(st);
  if (pl->tuning.ctas && (int)pl->tuning.ctas < grid) grid = (int)pl->tuning.ctas;
  if ((st = make_schedule(cols, ncols, pl->tuning, grid, &pl->sched)) != CAFS_OK) return fail(st);
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return fail(CAFS_ERR_CUDA);
  if ((st = ensure_batch(&pl->buf, grid, pl->sched, pl->tuning, s)) != CAFS_OK) return fail(st);
  if ((st = upload(&pl->buf, pl->sched, s)) != CAFS_OK) return fail(st);
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(CAFS_ERR_CUDA);

  // Record the memsets and the cooperative launch once.
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(CAFS_ERR_CUDA);
  // (Capturing launches nothing; the launch counter counts the replays.)
  st = enqueue_batch(&pl->buf, pl->sched, pl->tuning, grid, s, false, &pl->launches);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(s, &g);
  pl->graph = g;
  if (st != CAFS_OK || ce != cudaSuccess || !g) {
    cudaGetLastError();
    return fail(st != CAFS_OK ? st : CAFS_ERR_CUDA);
  }
  if (cudaGraphInstantiate(&pl->exec, pl->graph, 0) != cudaSuccess) {
    cudaGetLastError();
    return fail(CAFS_ERR_CUDA);
  }
  cudaStreamDestroy(s);
  pl->buf.grid = grid;
  *out = pl;
  return CAFS_OK;
}

cafs_status cafs_batch_plan_launch(cafs_batch_plan* pl, void* stream) {
  if (!pl) return CAFS_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lock(pl->mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CAFS_ERR_CUDA;
  if (dev != pl->device) return CAFS_ERR_INVALID_ARGUMENT;
  if (cudaGraphLaunch(pl->exec, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return CAFS_ERR_CUDA;
  count_launches(pl->launches);
  return CAFS_OK;
}

cafs_status cafs_batch_plan_reports(cafs_batch_plan* pl, cafs_report* reports, void* stream) {
  if (!pl || (!reports && !pl->sched.cols.empty())) return CAFS_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lock(pl->mu);
  return read_reports(&pl->buf, pl->sched, reports, reinterpret_cast<cudaStream_t>(stream));
}

size_t cafs_batch_plan_columns(const cafs_batch_plan* pl) { return pl ? pl->sched.cols.size() : 0; }

cafs_status cafs_batch_autotune(const cafs_column* cols, size_t ncols, const cafs_batch_tuning* candidates,
                                size_t ncand, int reps, double* ms, size_t* best, void* stream) {
  if (!candidates || ncand == 0 || reps < 1 || !ms || !best) return CAFS_ERR_INVALID_ARGUMENT;
  for (size_t c = 0; c < ncand; ++c) {
    Tuning t;
    cafs_status st = tuning_from(&candidates[c], &t);
    if (st != CAFS_OK) return st;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CAFS_ERR_CUDA;
  cafs_status st = CAFS_OK;
  double best_ms = 0.0;
  std::vector<double> times;
  for (size_t c = 0; c < ncand && st == CAFS_OK; ++c) {
    cafs_batch_plan* pl = nullptr;
    st = cafs_batch_plan_create(cols, ncols, &candidates[c], &pl);
    if (st != CAFS_OK) break;
    times.clear();
    for (int r = 0; r <= reps && st == CAFS_OK; ++r) {   // launch 0 warms up
      if (cudaEventRecord(e0, s) != cudaSuccess) st = CAFS_ERR_CUDA;
      if (st == CAFS_OK) st = cafs_batch_plan_launch(pl, stream);
      if (st == CAFS_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
        st = CAFS_ERR_CUDA;
      float t = 0.f;
      if (st == CAFS_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) st = CAFS_ERR_CUDA;
      if (st == CAFS_OK && r > 0) times.push_back(t);
    }
    cafs_batch_plan_destroy(pl);
    if (st != CAFS_OK) break;
    std::sort(times.begin(), times.end());
    ms[c] = times[times.size() / 2];
    if (c == 0 || ms[c] < best_ms) {
      best_ms = ms[c];
      *best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

void cafs_batch_plan_destroy(cafs_batch_plan* pl) {
  if (!pl) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (pl->device >= 0 && pl->device != cur) cudaSetDevice(pl->device);
  cudaDeviceSynchronize();
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  free_batch(&pl->buf);
  if (pl->device >= 0 && pl->device != cur) cudaSetDevice(cur);
  delete pl;
}

}  // extern "C"
