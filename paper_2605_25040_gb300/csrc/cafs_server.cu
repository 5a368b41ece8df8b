// Served form of the CAFS sort (no counterpart in the paper): a request
// server that admits sort requests as they arrive, by device-memory budget,
// and sorts whatever is admitted together with one batched launch.
//
// Memory: at creation the server reserves its whole budget once -- the
// batched kernel's workspace and one arena for request buffers -- and never
// allocates again.  A request is admitted (FIFO) when its n keys fit in the
// arena; its keys stay resident in that buffer while it is copied in, sorted
// in place and copied out, and the buffer returns to the arena when the
// result is in the caller's host memory.
//
// Pipeline: a scheduler thread takes everything admissible, issues the
// host-to-device copies on a copy stream, then the batched launch on the
// compute stream and the device-to-host copies on a third stream; a
// completion thread waits for each launch's last copy in order, records the
// completion time and frees the buffers.  Copies of the next launch overlap
// the current launch (continuous batching: requests arriving during a
// launch form the next one).

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cafs_batch_host.h"
#include "cafs_transform.h"

namespace cafs {
namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

constexpr unsigned long long kArenaAlign = 256;

// First-fit allocator over [0, size) with coalescing free ranges.
class Arena {
 public:
  void reset(unsigned long long size) {
    free_.clear();
    if (size) free_[0] = size;
    size_ = size;
  }
  // Returns the offset or ~0 when no free range is large enough.
  unsigned long long alloc(unsigned long long bytes) {
    bytes = (bytes + kArenaAlign - 1) & ~(kArenaAlign - 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const unsigned long long off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        return off;
      }
    }
    return ~0ull;
  }
  void release(unsigned long long off, unsigned long long bytes) {
    bytes = (bytes + kArenaAlign - 1) & ~(kArenaAlign - 1);
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  unsigned long long size() const { return size_; }

 private:
  std::map<unsigned long long, unsigned long long> free_;
  unsigned long long size_ = 0;
};

struct Request {
  uint64_t ticket = 0;
  const void* host_in = nullptr;
  void* host_out = nullptr;
  size_t n = 0;
  cafs_dtype dtype = CAFS_INT64;
  unsigned long long bytes = 0;
  unsigned long long off = 0;
  double t_arrival = 0.0;
  double t_done = 0.0;
  bool done = false;
  cafs_report report{};
};

struct Launch {
  std::vector<Request*> reqs;
  cudaEvent_t done = nullptr;
  Record* h_records = nullptr;   // pinned, max_batch entries
  BatchState* h_state = nullptr;  // pinned
};

}  // namespace
}  // namespace cafs

using namespace cafs;

struct cafs_server {
  int device = -1;
  int grid = 0;
  unsigned max_batch = 0;
  unsigned max_inflight = 0;
  unsigned long long max_request_keys = 0;
  Tuning tuning;
  BatchBuffers buf;
  unsigned char* arena_base = nullptr;
  Arena arena;
  cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
  cudaEvent_t ev_in = nullptr, ev_run = nullptr;
  std::vector<Launch*> free_launches;
  std::deque<Launch*> inflight;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, Request*> tickets;
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done, cv_client;
  std::thread sched, completer;
  bool stop = false;
  cafs_status fatal = CAFS_OK;
  // statistics
  uint64_t launches = 0, completed = 0, keys_done = 0;
  size_t peak_arena_used = 0, arena_used = 0;
  unsigned dispatching = 0;   // a launch is being enqueued (scheduler or submitter): one at a time
};

namespace cafs {
namespace {

// One request on an idle server: copy in, the single-column kernel over the
// grid slot's buffers and the record read on the compute stream, the copy
// out on the output stream.  The batched launch adds a schedule upload, its
// own clears, three stages and another cross-stream wait, which at low load
// only add latency.
cafs_status enqueue_solo(cafs_server* sv, Request* r, Launch* L) {
  const BatchBuffers& b = sv->buf;
  const SlotLayout& gl = b.gl;
  unsigned char* slot = b.grid_slot;
  void* d = sv->arena_base + r->off;
  cudaStream_t s = sv->s_run;
  if (cudaMemcpyAsync(d, r->host_in, r->bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return CAFS_ERR_CUDA;
  const int kind = key_type_kind(r->dtype);   // unsigned / float keys: sorted as signed images
  const int width = (int)key_type_width(r->dtype);
  if (kind) {
    if (launch_order_map(d, d, r->n, width, kind, s) != cudaSuccess) return CAFS_ERR_CUDA;
    count_launches(1);
  }
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(slot + gl.ctrl);
  if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s) != cudaSuccess) return CAFS_ERR_CUDA;
  Params p;
  std::memset(&p, 0, sizeof(p));
  p.keys = d;
  p.out = d;
  p.n = r->n;
  p.ctrl = ctrl;
  p.tkeys = reinterpret_cast<unsigned long long*>(slot + gl.tkeys);
  p.tcounts = reinterpret_cast<unsigned*>(slot + gl.tcounts);
  p.claimed = reinterpret_cast<unsigned*>(slot + gl.claimed);
  p.table_cap = gl.table_cap;
  p.pkeys_a = slot + gl.pka;
  p.pvals_a = reinterpret_cast<unsigned*>(slot + gl.pva);
  p.pkeys_b = slot + gl.pkb;
  p.pvals_b = reinterpret_cast<unsigned*>(slot + gl.pvb);
  p.skeys = slot + gl.sk;
  p.svals = reinterpret_cast<unsigned*>(slot + gl.sv);
  p.offsets = reinterpret_cast<unsigned*>(slot + gl.off);
  p.pair_cap = gl.pair_cap;
  p.tmp = slot + gl.tmp;
  p.lookback = reinterpret_cast<unsigned long long*>(slot + gl.look);
  p.lookback_cap = gl.lookback_cap;
  p.sample_keys = reinterpret_cast<long long*>(slot + gl.sample);
  p.mode = kModeSort;
  p.local_slots_max = sv->tuning.local_slots_max;
  p.replicas_max = sv->tuning.replicas_max;
  p.emit_tile_vec = sv->tuning.emit_tile_vec;
  p.timeout_ns = wait_timeout_ns();
  next_hash_multipliers(&p.hash_mult, &p.local_mult);
  const int dtype = key_type_base(r->dtype);
  cudaError_t e;
  if (r->n < kSmallN) {
    e = launch_small(p, dtype, s);
  } else {
    // the same CTA count rule as the single-column entry point, within the
    // grid slot's radix scratch (sized for sv->grid CTAs)
    unsigned long long grid = (r->n + 16383) / 16384;
    if (grid > (unsigned long long)sv->grid) grid = (unsigned long long)sv->grid;
    e = launch_pipeline(p, dtype, (int)grid, s);
  }
  if (e != cudaSuccess) return CAFS_ERR_CUDA;
  count_launches(1);
  if (kind) {
    if (launch_order_map(d, d, r->n, width, kind, s) != cudaSuccess) return CAFS_ERR_CUDA;
    count_launches(1);
  }
  std::memset(L->h_state, 0, 2 * sizeof(BatchState));   // no batch state: both key types OK
  // The copy out goes on its own stream, as in the batched path, so that a
  // batch formed meanwhile does not wait behind it.
  if (cudaMemcpyAsync(L->h_records, &ctrl->rec, sizeof(Record), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaEventRecord(sv->ev_run, s) != cudaSuccess || cudaStreamWaitEvent(sv->s_out, sv->ev_run, 0) != cudaSuccess ||
      cudaMemcpyAsync(r->host_out, d, r->bytes, cudaMemcpyDeviceToHost, sv->s_out) != cudaSuccess ||
      cudaEventRecord(L->done, sv->s_out) != cudaSuccess)
    return CAFS_ERR_CUDA;
  return CAFS_OK;
}

void scheduler_loop(cafs_server* sv) {
  cudaSetDevice(sv->device);
  Schedule sc;
  std::vector<cafs_column> cols;
  for (;;) {
    Launch* L = nullptr;
    std::vector<Request*> batch;
    bool idle = false;   // nothing in flight when this batch was formed
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      for (;;) {
        if (sv->stop) return;
        // one thread enqueues at a time (the launches share streams and events)
        if (!sv->pending.empty() && !sv->free_launches.empty() && sv->dispatching == 0) {
          // Admission by memory budget, first come first served.
          while (!sv->pending.empty() && batch.size() < sv->max_batch) {
            Request* r = sv->pending.front();
            const unsigned long long off = sv->arena.alloc(r->bytes);
            if (off == ~0ull) break;
            r->off = off;
            sv->arena_used += (r->bytes + kArenaAlign - 1) & ~(kArenaAlign - 1);
            sv->peak_arena_used = std::max(sv->peak_arena_used, sv->arena_used);
            sv->pending.pop_front();
            batch.push_back(r);
          }
          if (!batch.empty()) {
            L = sv->free_launches.back();
            sv->free_launches.pop_back();
            idle = sv->inflight.empty();
            sv->dispatching++;
            break;
          }
        }
        sv->cv_sched.wait(lk);
      }
    }
    cafs_status st = CAFS_OK;
    if (idle && batch.size() == 1) {
      st = enqueue_solo(sv, batch[0], L);
      L->reqs.swap(batch);
      {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (st != CAFS_OK && sv->fatal == CAFS_OK) sv->fatal = st;
        sv->inflight.push_back(L);
        sv->launches++;
        sv->dispatching--;
      }
      sv->cv_done.notify_one();
      continue;
    }
    // Copies in, one batched launch, copies out.
    cols.resize(batch.size());
    for (size_t i = 0; i < batch.size(); ++i) {
      Request* r = batch[i];
      void* d = sv->arena_base + r->off;
      if (cudaMemcpyAsync(d, r->host_in, r->bytes, cudaMemcpyHostToDevice, sv->s_in) != cudaSuccess)
        st = CAFS_ERR_CUDA;
      cols[i].keys = d;
      cols[i].out = d;
      cols[i].n = r->n;
      cols[i].dtype = r->dtype;
      cols[i].reserved = 0;
    }
    if (st == CAFS_OK && (cudaEventRecord(sv->ev_in, sv->s_in) != cudaSuccess ||
                          cudaStreamWaitEvent(sv->s_run, sv->ev_in, 0) != cudaSuccess))
      st = CAFS_ERR_CUDA;
    if (st == CAFS_OK) st = make_schedule(cols.data(), cols.size(), sv->tuning, sv->grid, &sc);
    if (st == CAFS_OK) st = upload(&sv->buf, sc, sv->s_run);
    if (st == CAFS_OK) st = enqueue_batch(&sv->buf, sc, sv->tuning, sv->grid, sv->s_run, true, nullptr);
    if (st == CAFS_OK &&
        (cudaMemcpyAsync(L->h_records, sv->buf.d_records, batch.size() * sizeof(Record),
                         cudaMemcpyDeviceToHost, sv->s_run) != cudaSuccess ||
         cudaMemcpyAsync(L->h_state, sv->buf.d_state, 2 * sizeof(BatchState), cudaMemcpyDeviceToHost,
                         sv->s_run) != cudaSuccess ||
         cudaEventRecord(sv->ev_run, sv->s_run) != cudaSuccess ||
         cudaStreamWaitEvent(sv->s_out, sv->ev_run, 0) != cudaSuccess))
      st = CAFS_ERR_CUDA;
    for (Request* r : batch)
      if (st == CAFS_OK && cudaMemcpyAsync(r->host_out, sv->arena_base + r->off, r->bytes,
                                           cudaMemcpyDeviceToHost, sv->s_out) != cudaSuccess)
        st = CAFS_ERR_CUDA;
    if (st == CAFS_OK && cudaEventRecord(L->done, sv->s_out) != cudaSuccess) st = CAFS_ERR_CUDA;
    L->reqs.swap(batch);
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      if (st != CAFS_OK && sv->fatal == CAFS_OK) sv->fatal = st;
      sv->inflight.push_back(L);
      sv->launches++;
      sv->dispatching--;
    }
    sv->cv_done.notify_one();
  }
}

void completion_loop(cafs_server* sv) {
  cudaSetDevice(sv->device);
  for (;;) {
    Launch* L = nullptr;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv_done.wait(lk, [&] { return sv->stop || !sv->inflight.empty(); });
      if (sv->inflight.empty()) return;   // stopping with nothing in flight
      L = sv->inflight.front();
    }
    const bool ok = cudaEventSynchronize(L->done) == cudaSuccess;
    const double t = now_s();
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      BatchState st = L->h_state[0];
      if (st.status == kDevOk) st.status = L->h_state[1].status;
      for (size_t i = 0; i < L->reqs.size(); ++i) {
        Request* r = L->reqs[i];
        fill_report(L->h_records[i], &r->report);
        if (!ok) r->report.device_status = CAFS_ERR_CUDA;
        else if (sv->fatal != CAFS_OK) r->report.device_status = sv->fatal;
        else if (st.status != kDevOk && r->report.device_status == CAFS_OK)
          r->report.device_status = (cafs_status)st.status;
        r->t_done = t;
        r->done = true;
        sv->arena.release(r->off, r->bytes);
        sv->arena_used -= (r->bytes + kArenaAlign - 1) & ~(kArenaAlign - 1);
        sv->completed++;
        sv->keys_done += r->n;
      }
      L->reqs.clear();
      sv->inflight.pop_front();
      sv->free_launches.push_back(L);
      if (!ok && sv->fatal == CAFS_OK) sv->fatal = CAFS_ERR_CUDA;
    }
    sv->cv_sched.notify_one();
    sv->cv_client.notify_all();
  }
}

void destroy_server(cafs_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_sched.notify_all();
  if (sv->sched.joinable()) sv->sched.join();
  // the completion thread drains what is in flight, then stops
  sv->cv_done.notify_all();
  if (sv->completer.joinable()) sv->completer.join();
  if (sv->device >= 0) cudaSetDevice(sv->device);
  for (Launch* L : sv->free_launches) {
    if (L->done) cudaEventDestroy(L->done);
    if (L->h_records) cudaFreeHost(L->h_records);
    if (L->h_state) cudaFreeHost(L->h_state);
    delete L;
  }
  sv->free_launches.clear();
  for (auto& kv : sv->tickets) delete kv.second;
  for (Request* r : sv->pending) {
    if (!sv->tickets.count(r->ticket)) delete r;
  }
  if (sv->ev_in) cudaEventDestroy(sv->ev_in);
  if (sv->ev_run) cudaEventDestroy(sv->ev_run);
  if (sv->s_in) cudaStreamDestroy(sv->s_in);
  if (sv->s_run) cudaStreamDestroy(sv->s_run);
  if (sv->s_out) cudaStreamDestroy(sv->s_out);
  if (sv->arena_base) cudaFree(sv->arena_base);
  free_batch(&sv->buf);
  delete sv;
}

}  // namespace
}  // namespace cafs

extern "C" {

cafs_status cafs_server_config_default(cafs_server_config* cfg) {
  if (!cfg) return CAFS_ERR_INVALID_ARGUMENT;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->max_batch_columns = 1024;
  cfg->max_inflight = 3;
  cfg->max_request_keys = 1ull << 22;
  Tuning t;
  t.cta_table_slots = 1ull << 18;   // larger Eq. 6 tables are set aside
  t.defer_min_n = 1ull << 16;       // fixed, so the per-CTA radix buffers stay small
  tuning_to(t, &cfg->tuning);
  return CAFS_OK;
}

cafs_status cafs_server_create(size_t mem_budget_bytes, const cafs_server_config* cfg_in,
                               cafs_server** out) {
  if (!out) return CAFS_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  cafs_server_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else cafs_server_config_default(&cfg);
  if (cfg.max_batch_columns == 0 || cfg.max_inflight == 0 || cfg.max_request_keys == 0 ||
      cfg.max_request_keys > 0xFFFFFFFFull || cfg.reserved != 0)
    return CAFS_ERR_INVALID_ARGUMENT;
  cafs_server* sv = new cafs_server();
  cafs_status st = tuning_from(&cfg.tuning, &sv->tuning);
  if (st != CAFS_OK) {
    delete sv;
    return st;
  }
  sv->max_batch = cfg.max_batch_columns;
  sv->max_inflight = cfg.max_inflight;
  sv->max_request_keys = cfg.max_request_keys;
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    return CAFS_ERR_CUDA;
  }
  auto fail = [&](cafs_status e) {
    cudaGetLastError();
    destroy_server(sv);
    return e;
  };
  if ((st = batch_grid(sv->device, &sv->grid)) != CAFS_OK) return fail(st);
  if (sv->tuning.ctas && (int)sv->tuning.ctas < sv->grid) sv->grid = (int)sv->tuning.ctas;
  if (cudaStreamCreateWithFlags(&sv->s_in, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&sv->s_run, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&sv->s_out, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&sv->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&sv->ev_run, cudaEventDisableTiming) != cudaSuccess)
    return fail(CAFS_ERR_CUDA);
  // The workspace for the largest admissible batch.
  Schedule worst;
  worst.cols.resize(sv->max_batch);
  const unsigned long long nmax = sv->max_request_keys;
  const unsigned long long gmin = sv->tuning.grid_min_n ? sv->tuning.grid_min_n : nmax + 1;
  if (nmax >= gmin) worst.n_max_grid = nmax;
  worst.n_max_cta = std::min(nmax, gmin - 1);
  if ((st = ensure_batch(&sv->buf, sv->grid, worst, sv->tuning, sv->s_run)) != CAFS_OK) return fail(st);
  if (cudaStreamSynchronize(sv->s_run) != cudaSuccess) return fail(CAFS_ERR_CUDA);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(CAFS_ERR_CUDA);
  const unsigned long long ws = sv->buf.gl.bytes + sv->buf.cl.bytes * (unsigned long long)sv->grid +
                                (unsigned long long)sv->buf.col_cap * (sizeof(BatchColumn) + 2 * sizeof(unsigned) + sizeof(Record));
  if (ws >= mem_budget_bytes) return fail(CAFS_ERR_OUT_OF_MEMORY);
  const unsigned long long arena_bytes = (mem_budget_bytes - ws) & ~(kArenaAlign - 1);
  if (arena_bytes < kArenaAlign || cudaMalloc((void**)&sv->arena_base, arena_bytes) != cudaSuccess)
    return fail(CAFS_ERR_OUT_OF_MEMORY);
  sv->arena.reset(arena_bytes);
  for (unsigned i = 0; i < sv->max_inflight; ++i) {
    Launch* L = new Launch();
    sv->free_launches.push_back(L);
    if (cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void**)&L->h_records, sv->max_batch * sizeof(Record)) != cudaSuccess ||
        cudaMallocHost((void**)&L->h_state, 2 * sizeof(BatchState)) != cudaSuccess)
      return fail(CAFS_ERR_OUT_OF_MEMORY);
  }
  sv->sched = std::thread(scheduler_loop, sv);
  sv->completer = std::thread(completion_loop, sv);
  *out = sv;
  return CAFS_OK;
}

}  // extern "C"

namespace cafs {
namespace {

cafs_status submit_at(cafs_server* sv, const void* host_keys, size_t n, cafs_dtype dtype, void* host_out,
                      double t_arrival, uint64_t* ticket) {
  if (!sv || !ticket) return CAFS_ERR_INVALID_ARGUMENT;
  cafs_status st = check_args_typed(host_keys, n, dtype, host_out, false);
  if (st != CAFS_OK) return st;
  if (n && !host_out) return CAFS_ERR_INVALID_ARGUMENT;
  if ((unsigned long long)n > sv->max_request_keys) return CAFS_ERR_TOO_LARGE;
  const unsigned long long bytes = (unsigned long long)n * key_type_width(dtype);
  if (((bytes + kArenaAlign - 1) & ~(kArenaAlign - 1)) > sv->arena.size()) return CAFS_ERR_TOO_LARGE;
  Launch* direct = nullptr;
  Request* r = new Request();
  r->host_in = host_keys;
  r->host_out = host_out;
  r->n = n;
  r->dtype = dtype;
  r->bytes = bytes;
  r->t_arrival = t_arrival;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->fatal != CAFS_OK) {
      delete r;
      return sv->fatal;
    }
    r->ticket = sv->next_ticket++;
    sv->tickets[r->ticket] = r;
    if (n == 0) {
      r->report.path = CAFS_PATH_EMPTY;
      r->t_done = r->t_arrival;
      r->done = true;
    } else if (sv->pending.empty() && sv->inflight.empty() && sv->dispatching == 0 &&
               !sv->free_launches.empty()) {
      // An idle server: this thread launches the request itself (the
      // scheduler's wake-up would only add latency).
      const unsigned long long off = sv->arena.alloc(r->bytes);
      if (off != ~0ull) {
        r->off = off;
        sv->arena_used += (r->bytes + kArenaAlign - 1) & ~(kArenaAlign - 1);
        sv->peak_arena_used = std::max(sv->peak_arena_used, sv->arena_used);
        direct = sv->free_launches.back();
        sv->free_launches.pop_back();
        sv->dispatching++;
      } else {
        sv->pending.push_back(r);
      }
    } else {
      sv->pending.push_back(r);
    }
    *ticket = r->ticket;
  }
  if (direct) {
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != sv->device) cudaSetDevice(sv->device);
    const cafs_status est = enqueue_solo(sv, r, direct);
    if (prev >= 0 && prev != sv->device) cudaSetDevice(prev);
    direct->reqs.assign(1, r);
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      if (est != CAFS_OK && sv->fatal == CAFS_OK) sv->fatal = est;
      sv->inflight.push_back(direct);
      sv->launches++;
      sv->dispatching--;
    }
    sv->cv_done.notify_one();
    sv->cv_sched.notify_one();   // requests that queued meanwhile
    return CAFS_OK;
  }
  if (n) sv->cv_sched.notify_one();
  else sv->cv_client.notify_all();
  return CAFS_OK;
}

void spin_until(double t) {
  while (now_s() < t) {
  }
}

}  // namespace
}  // namespace cafs

extern "C" {

cafs_status cafs_server_submit(cafs_server* sv, const void* host_keys, size_t n, cafs_dtype dtype,
                               void* host_out, uint64_t* ticket) {
  return submit_at(sv, host_keys, n, dtype, host_out, now_s(), ticket);
}

cafs_status cafs_server_wait(cafs_server* sv, uint64_t ticket, cafs_report* report, double* latency_us) {
  if (!sv) return CAFS_ERR_INVALID_ARGUMENT;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->tickets.find(ticket);
  if (it == sv->tickets.end()) return CAFS_ERR_INVALID_ARGUMENT;
  Request* r = it->second;
  sv->cv_client.wait(lk, [&] { return r->done || sv->fatal != CAFS_OK; });
  if (!r->done) return sv->fatal;
  if (report) *report = r->report;
  if (latency_us) *latency_us = (r->t_done - r->t_arrival) * 1e6;
  sv->tickets.erase(it);
  delete r;
  return CAFS_OK;
}

cafs_status cafs_server_stats(cafs_server* sv, cafs_server_stats_t* out) {
  if (!sv || !out) return CAFS_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(sv->mu);
  std::memset(out, 0, sizeof(*out));
  out->launches = sv->launches;
  out->completed = sv->completed;
  out->keys_done = sv->keys_done;
  out->pending = sv->pending.size();
  out->arena_bytes = sv->arena.size();
  out->arena_peak_bytes = sv->peak_arena_used;
  out->workspace_bytes = sv->buf.gl.bytes + sv->buf.cl.bytes * (unsigned long long)sv->grid;
  return CAFS_OK;
}

void cafs_server_destroy(cafs_server* sv) { destroy_server(sv); }

cafs_status cafs_server_run_trace(cafs_server* sv, const cafs_request* reqs, size_t nreq,
                                  const double* arrival_s, double* latency_us, cafs_report* reports,
                                  double* elapsed_s) {
  if (!sv || (nreq && (!reqs || !arrival_s || !latency_us))) return CAFS_ERR_INVALID_ARGUMENT;
  for (size_t i = 0; i < nreq; ++i) {
    if (reqs[i].reserved != 0 || !(arrival_s[i] >= 0.0) || (i && arrival_s[i] < arrival_s[i - 1]))
      return CAFS_ERR_INVALID_ARGUMENT;
    const cafs_status st = check_args_typed(reqs[i].host_keys, reqs[i].n, reqs[i].dtype, reqs[i].host_out, false);
    if (st != CAFS_OK) return st;
    if (reqs[i].n && !reqs[i].host_out) return CAFS_ERR_INVALID_ARGUMENT;
    if ((unsigned long long)reqs[i].n > sv->max_request_keys) return CAFS_ERR_TOO_LARGE;
  }
  std::vector<uint64_t> tickets(nreq, 0);
  std::vector<size_t> submitted(1, 0);
  std::mutex m;
  std::condition_variable cv;
  cafs_status wait_status = CAFS_OK;
  double t_last = 0.0;
  const double t0 = now_s() + 1e-3;
  // The waiter collects results in submission order while requests arrive.
  std::thread waiter([&] {
    for (size_t i = 0; i < nreq; ++i) {
      {
        std::unique_lock<std::mutex> lk(m);
        cv.wait(lk, [&] { return submitted[0] > i; });
      }
      double lat = 0.0;
      cafs_report rep;
      const cafs_status st = cafs_server_wait(sv, tickets[i], &rep, &lat);
      if (st != CAFS_OK && wait_status == CAFS_OK) wait_status = st;
      latency_us[i] = lat;
      if (reports) reports[i] = rep;
      t_last = now_s();
    }
  });
  cafs_status st = CAFS_OK;
  for (size_t i = 0; i < nreq && st == CAFS_OK; ++i) {
    const double t = t0 + arrival_s[i];
    spin_until(t);
    st = submit_at(sv, reqs[i].host_keys, reqs[i].n, reqs[i].dtype, reqs[i].host_out, t, &tickets[i]);
    {
      std::lock_guard<std::mutex> lk(m);
      if (st == CAFS_OK) submitted[0] = i + 1;
    }
    cv.notify_one();
  }
  if (st != CAFS_OK) {
    // Unblock the waiter: it only waits for what was submitted.
    std::lock_guard<std::mutex> lk(m);
    nreq = submitted[0];
  }
  {
    std::lock_guard<std::mutex> lk(m);
    submitted[0] = nreq;
  }
  cv.notify_one();
  waiter.join();
  if (elapsed_s) *elapsed_s = nreq ? t_last - (t0 + arrival_s[0]) : 0.0;
  return st != CAFS_OK ? st : wait_status;
}

cafs_status cafs_serial_run_trace(const cafs_request* reqs, size_t nreq, const double* arrival_s,
                                  double* latency_us, cafs_report* reports, double* elapsed_s, void* stream) {
  if (nreq && (!reqs || !arrival_s || !latency_us)) return CAFS_ERR_INVALID_ARGUMENT;
  for (size_t i = 0; i < nreq; ++i)
    if (reqs[i].reserved != 0 || !(arrival_s[i] >= 0.0) || (i && arrival_s[i] < arrival_s[i - 1]))
      return CAFS_ERR_INVALID_ARGUMENT;
  const double t0 = now_s() + 1e-3;
  double t_last = t0;
  for (size_t i = 0; i < nreq; ++i) {
    const double t = t0 + arrival_s[i];
    spin_until(t);
    cafs_report rep;
    const cafs_status st = cafs_sort_host(reqs[i].host_keys, reqs[i].n, reqs[i].dtype, reqs[i].host_out,
                                          &rep, stream);
    if (st != CAFS_OK) return st;
    t_last = now_s();
    latency_us[i] = (t_last - t) * 1e6;
    if (reports) reports[i] = rep;
  }
  if (elapsed_s) *elapsed_s = nreq ? t_last - (t0 + arrival_s[0]) : 0.0;
  return CAFS_OK;
}

}  // extern "C"
