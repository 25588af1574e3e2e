// Trigger-style serving loop: continuous batching of arriving events.
//
// The paper runs batches of events through the GPU and notes that transfers, kernels and
// result copies can overlap (Sec. 3, event-level parallelism; streams are future work in
// Sec. 5). Here a host thread owned by the server admits requests into micro-batches and
// keeps up to `slots` micro-batches in flight, each on its own stream with its own device
// buffers: while earlier batches run, new arrivals are gathered into the next free slot, so
// their work overlaps on the device. A micro-batch is launched when it is full or when its
// oldest request has waited flush_ns. Per slot: pinned gather -> H2D -> validate + fused kernel
// (one CTA per event) -> peak packing -> D2H of counts, masks and packed peaks -> event; when
// the event completes the loop copies each request's results into the caller's buffers and
// stamps its completion time. Every wait is bounded: a batch that cannot be enqueued, or has
// not completed after HOUGH_SERVE_BATCH_TIMEOUT_NS, finishes its requests with an error flag
// and no results. The loop keeps a ring of per-batch timestamps and watches the gaps between
// its own passes (and between the submissions of hough_serve_replay) for stalls.
#include <sys/resource.h>
#include <time.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "hough_internal.h"

namespace hgpu {

int make_plan(const hough_params* p, Plan& pl, int acc32);

namespace {

long long now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Resource usage of the calling thread: user and system CPU time (ns), minor page faults,
// voluntary context switches (the thread blocked) and involuntary ones (it was preempted).
struct ThreadUsage {
  long long user_ns = 0, sys_ns = 0, minflt = 0, nvcsw = 0, nivcsw = 0;
};

ThreadUsage thread_usage() {
  ThreadUsage u;
  rusage r;
  if (getrusage(RUSAGE_THREAD, &r) != 0) return u;
  u.user_ns = (long long)r.ru_utime.tv_sec * 1000000000LL + (long long)r.ru_utime.tv_usec * 1000LL;
  u.sys_ns = (long long)r.ru_stime.tv_sec * 1000000000LL + (long long)r.ru_stime.tv_usec * 1000LL;
  u.minflt = r.ru_minflt;
  u.nvcsw = r.ru_nvcsw;
  u.nivcsw = r.ru_nivcsw;
  return u;
}

constexpr long long kStallNs = 1000000;  // a gap above 1 ms between passes is a stall

// Gaps between consecutive ticks of one thread. The thread's resource usage is sampled about once
// a millisecond, so its usage over a stall's window (the gap plus at most 1 ms before it) tells
// what the thread did meanwhile: CPU time near the window means it was busy (system time and
// page faults: in the kernel), near zero that it was not running (voluntary switches: blocked;
// involuntary ones: preempted).
struct StallWatch {
  long long t_last = 0, t_sample = 0;
  ThreadUsage u_sample;
  long long stalls = 0, max_gap = 0, max_at = 0;
  ThreadUsage max_use;  // usage over the longest stall's window
  void start(long long now) {
    t_last = t_sample = now;
    u_sample = thread_usage();
  }
  void tick(long long now) {
    if (now - t_last > kStallNs) {
      ++stalls;
      const long long gap = now - t_last;
      if (gap > max_gap) {
        const ThreadUsage u = thread_usage();
        max_gap = gap;
        max_at = t_last;
        max_use.user_ns = u.user_ns - u_sample.user_ns;
        max_use.sys_ns = u.sys_ns - u_sample.sys_ns;
        max_use.minflt = u.minflt - u_sample.minflt;
        max_use.nvcsw = u.nvcsw - u_sample.nvcsw;
        max_use.nivcsw = u.nivcsw - u_sample.nivcsw;
      }
    }
    t_last = now;
    if (now - t_sample > kStallNs) {
      t_sample = now;
      u_sample = thread_usage();
    }
  }
};

struct Request {
  const int32_t* xy;
  int64_t n_hits;
  int64_t id;
  uint8_t* mask_out;
  hough_peak* peaks_out;
  hough_serve_result* result_out;  // nullable: the result goes here instead of the results ring
  long long t_arrival;             // scheduled arrival (ns, steady clock)
};

// Fixed-capacity FIFO whose storage is allocated and written once at construction, so that
// pushing and popping never allocate or touch a fresh page: on the serving path a page fault
// can block a thread for tens of milliseconds while the kernel compacts or migrates memory.
template <class T>
struct Ring {
  std::vector<T> buf;
  size_t head = 0, count = 0;
  explicit Ring(size_t cap = 1) : buf(cap > 0 ? cap : 1) {}
  bool empty() const { return count == 0; }
  size_t size() const { return count; }
  size_t capacity() const { return buf.size(); }
  T& front() { return buf[head]; }
  void pop_front() {
    head = head + 1 == buf.size() ? 0 : head + 1;
    --count;
  }
  bool push_back(const T& x) {
    if (count == buf.size()) return false;
    size_t at = head + count;
    if (at >= buf.size()) at -= buf.size();
    buf[at] = x;
    ++count;
    return true;
  }
};

// Per-slot carve-up of the device and pinned host buffers.
struct SlotLayout {
  size_t d_xy, d_off, d_npeaks, d_peaks, d_mask, d_nkept, d_status, d_peak_off, d_dense, d_ws, d_total;
  size_t h_xy, h_off, h_npeaks, h_nkept, h_mask, h_peak_off, h_dense, h_status, h_total;
  size_t ws_bytes;
};

bool slot_layout(const hough_serve_config& c, const Plan& pl, SlotLayout& L) {
  const size_t ne = (size_t)c.max_batch_events, nh = (size_t)c.max_batch_hits, mp = (size_t)c.params.max_peaks;
  size_t o = 0;
  auto dt = [&](size_t b) {
    const size_t at = o;
    o = al256(o + (b ? b : 1));
    return at;
  };
  L.d_xy = dt(8 * nh);
  L.d_off = dt(8 * (ne + 1));
  L.d_npeaks = dt(4 * ne);
  L.d_peaks = dt(sizeof(hough_peak) * ne * mp);
  L.d_mask = dt(nh);
  L.d_nkept = dt(4 * ne);
  L.d_status = dt(4 * HOUGH_STATUS_WORDS);
  L.d_peak_off = dt(8 * (ne + 1));
  L.d_dense = dt(sizeof(hough_peak) * ne * mp);
  L.ws_bytes = ws_layout(pl, (long long)ne).total;
  L.d_ws = dt(L.ws_bytes);
  L.d_total = o;
  o = 0;
  L.h_xy = dt(8 * nh);
  L.h_off = dt(8 * (ne + 1));
  L.h_npeaks = dt(4 * ne);
  L.h_nkept = dt(4 * ne);
  L.h_mask = dt(nh);
  L.h_peak_off = dt(8 * (ne + 1));
  L.h_dense = dt(sizeof(hough_peak) * ne * mp);
  L.h_status = dt(4 * HOUGH_STATUS_WORDS);
  L.h_total = o;
  return true;
}

struct Slot {
  char* d = nullptr;
  char* h = nullptr;
  hough_peak* dense_mapped = nullptr;  // device view of the pinned dense-peak area, when mapped
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<Request> reqs;            // capacity max_batch_events, reserved at open
  std::vector<hough_serve_result> out;  // the batch's results, likewise
  bool busy = false;
  bool dead = false;         // retired after a timeout or an unrecoverable error: never reused
  long long t_launch = 0;    // when its batch was enqueued
  long long rec = -1;        // its batch record (ring sequence number)
};

struct Server {
  hough_serve_config cfg;
  Plan plan;
  SlotLayout L;
  TrigTable trig;
  int device = 0;
  std::vector<Slot> slots;
  std::mutex mu;                  // guards pending, results, counters
  std::condition_variable cv;     // wakes drain() waiters
  Ring<Request> pending;          // queue_capacity requests waiting for a slot
  int64_t pending_hits = 0;
  Ring<hough_serve_result> results;  // finished requests not yet polled
  long long outstanding = 0;      // admitted requests whose result has not reached the caller
  std::atomic<bool> running{false};
  std::atomic<bool> draining{false};
  std::atomic<int> error{0};
  long long submitted = 0, completed = 0;
  std::thread loop;
  // tracing: batch records (ring), loop and submitter stall watches, under trace_mu
  std::mutex trace_mu;
  std::vector<hough_serve_batch_record> ring = std::vector<hough_serve_batch_record>(HOUGH_SERVE_RECORDS);
  long long ring_next = 0;
  long long passes = 0, batches = 0;
  StallWatch loop_watch, submit_watch;
  std::atomic<int> inject_failures{0};
};

hough_serve_batch_record& record_at(Server& S, long long seq) { return S.ring[(size_t)(seq % HOUGH_SERVE_RECORDS)]; }

cudaError_t launch_batch(Server& S, Slot& sl) {
  if (S.inject_failures.load() > 0 && S.inject_failures.fetch_sub(1) > 0)
    return cudaErrorLaunchFailure;  // test hook: fail before anything is enqueued
  const SlotLayout& L = S.L;
  const size_t ne = sl.reqs.size();
  int64_t* hoff = (int64_t*)(sl.h + L.h_off);
  int32_t* hxy = (int32_t*)(sl.h + L.h_xy);
  hoff[0] = 0;
  for (size_t i = 0; i < ne; ++i) {
    const Request& r = sl.reqs[i];
    std::memcpy(hxy + 2 * hoff[i], r.xy, 8 * (size_t)r.n_hits);
    hoff[i + 1] = hoff[i] + r.n_hits;
  }
  const int64_t nh = hoff[ne];
  cudaStream_t st = sl.stream;
  cudaError_t e = cudaMemcpyAsync(sl.d + L.d_xy, hxy, 8 * (size_t)nh, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sl.d + L.d_off, hoff, 8 * (ne + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sl.d + L.d_status, 0, 4 * HOUGH_STATUS_WORDS, st);
  if (e != cudaSuccess) return e;
  FusedIO io;
  std::memset(&io, 0, sizeof(io));
  io.xy = (const int2*)(sl.d + L.d_xy);
  io.n_hits = nh;
  io.off = (const long long*)(sl.d + L.d_off);
  io.n_events = (long long)ne;
  io.npeaks = (int*)(sl.d + L.d_npeaks);
  io.peaks = (hough_peak*)(sl.d + L.d_peaks);
  io.mask = (uint8_t*)(sl.d + L.d_mask);
  io.nkept = (int*)(sl.d + L.d_nkept);
  io.status = (int*)(sl.d + L.d_status);
  WsLayout wl = ws_layout(S.plan, (long long)ne);
  char* ws = sl.d + L.d_ws;
  bind_workspace(S.plan, wl, ws, io);
  io.n_items = (long long)ne * S.plan.tiles;
  io.persistent = 0;
  e = launch_prep(io.off, io.n_events, nh, io.status, io.queue, io.tickets, nullptr, st);
  if (e == cudaSuccess) e = launch_fused(S.plan, io, S.trig, (int)io.n_items, st);
  // packed peaks go straight into pinned host memory when it is mapped (only the stored ones
  // cross the link), else into device memory and are copied back whole
  hough_peak* dense = sl.dense_mapped ? sl.dense_mapped : (hough_peak*)(sl.d + L.d_dense);
  if (e == cudaSuccess)
    e = launch_pack_peaks(io.npeaks, io.peaks, io.n_events, S.plan.max_peaks, (long long*)(sl.d + L.d_peak_off),
                          dense, st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(sl.h + L.h_npeaks, io.npeaks, 4 * ne, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h + L.h_nkept, io.nkept, 4 * ne, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && nh) e = cudaMemcpyAsync(sl.h + L.h_mask, io.mask, (size_t)nh, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sl.h + L.h_peak_off, sl.d + L.d_peak_off, 8 * (ne + 1), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && !sl.dense_mapped)
    e = cudaMemcpyAsync(sl.h + L.h_dense, sl.d + L.d_dense, sizeof(hough_peak) * ne * (size_t)S.plan.max_peaks,
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sl.h + L.h_status, io.status, 4 * HOUGH_STATUS_WORDS, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, st);
  return e;
}

// Results of a finished slot into the callers' buffers and the results ring (or each request's
// own result record). Admission keeps room in the ring for every admitted request.
void deliver(Server& S, Slot& sl) {
  std::lock_guard<std::mutex> lk(S.mu);
  for (size_t i = 0; i < sl.reqs.size(); ++i) {
    if (sl.reqs[i].result_out) {
      *sl.reqs[i].result_out = sl.out[i];
      --S.outstanding;
    } else {
      S.results.push_back(sl.out[i]);
    }
  }
  S.completed += (long long)sl.reqs.size();
  S.cv.notify_all();
}

void finish_batch(Server& S, Slot& sl, long long t_done) {
  const SlotLayout& L = S.L;
  const int32_t* npk = (const int32_t*)(sl.h + L.h_npeaks);
  const int32_t* nk = (const int32_t*)(sl.h + L.h_nkept);
  const uint8_t* mask = (const uint8_t*)(sl.h + L.h_mask);
  const int64_t* poff = (const int64_t*)(sl.h + L.h_peak_off);
  const hough_peak* dense = (const hough_peak*)(sl.h + L.h_dense);
  const int32_t flags = *(const int32_t*)(sl.h + L.h_status);  // device flags of the whole micro-batch
  int64_t hit0 = 0;
  sl.out.resize(sl.reqs.size());  // within the capacity reserved at open
  for (size_t i = 0; i < sl.reqs.size(); ++i) {
    const Request& r = sl.reqs[i];
    if (r.mask_out && r.n_hits) std::memcpy(r.mask_out, mask + hit0, (size_t)r.n_hits);
    const int64_t np = poff[i + 1] - poff[i];
    if (r.peaks_out && np) std::memcpy(r.peaks_out, dense + poff[i], sizeof(hough_peak) * (size_t)np);
    hit0 += r.n_hits;
    hough_serve_result& o = sl.out[i];
    o.id = r.id;
    o.status = flags;
    o.npeaks = npk[i];
    o.nkept = nk[i];
    o.reserved = 0;
    o.t_arrival_ns = r.t_arrival;
    o.t_done_ns = t_done;
  }
  deliver(S, sl);
}

// Requests of a batch that produced no results (flag: HOUGH_F_TIMEOUT or HOUGH_F_LAUNCH_FAILED):
// they finish with that status and nothing is copied to their output buffers.
void fail_batch(Server& S, Slot& sl, long long t_done, int32_t flag) {
  sl.out.resize(sl.reqs.size());
  for (size_t i = 0; i < sl.reqs.size(); ++i) {
    hough_serve_result& o = sl.out[i];
    std::memset(&o, 0, sizeof(o));
    o.id = sl.reqs[i].id;
    o.status = flag;
    o.t_arrival_ns = sl.reqs[i].t_arrival;
    o.t_done_ns = t_done;
  }
  deliver(S, sl);
  sl.reqs.clear();
}

// Waits (bounded) until the slot's stream has no work left: true if it drained.
bool drain_slot(Server& S, Slot& sl) {
  const long long t0 = now_ns();
  for (;;) {
    const cudaError_t q = cudaStreamQuery(sl.stream);
    if (q == cudaSuccess) return true;
    if (q != cudaErrorNotReady) {
      note_cuda_error(q);
      S.error.store(HOUGH_ECUDA);
      return false;
    }
    if (now_ns() - t0 > HOUGH_SERVE_BATCH_TIMEOUT_NS) {
      S.error.store(HOUGH_ETIMEDOUT);
      return false;
    }
    std::this_thread::yield();
  }
}

void serve_loop(Server* Sp) {
  Server& S = *Sp;
  cudaSetDevice(S.device);
  {
    std::lock_guard<std::mutex> tk(S.trace_mu);
    S.loop_watch.start(now_ns());
  }
  while (S.running.load(std::memory_order_acquire)) {
    bool progress = false;
    {
      std::lock_guard<std::mutex> tk(S.trace_mu);
      S.loop_watch.tick(now_ns());
      ++S.passes;
    }
    for (Slot& sl : S.slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaSuccess) {
        const long long t_seen = now_ns();
        finish_batch(S, sl, t_seen);
        const long long t_fin = now_ns();
        {
          std::lock_guard<std::mutex> tk(S.trace_mu);
          if (sl.rec >= 0 && sl.rec + HOUGH_SERVE_RECORDS > S.ring_next) {
            record_at(S, sl.rec).t_done_seen = t_seen;
            record_at(S, sl.rec).t_finished = t_fin;
          }
        }
        sl.reqs.clear();
        sl.busy = false;
        progress = true;
      } else if (q != cudaErrorNotReady) {  // the batch failed on the device
        note_cuda_error(q);
        S.error.store(HOUGH_ECUDA);
        fail_batch(S, sl, now_ns(), HOUGH_F_LAUNCH_FAILED);
        sl.busy = false;
        sl.dead = true;
        progress = true;
      } else if (now_ns() - sl.t_launch > HOUGH_SERVE_BATCH_TIMEOUT_NS) {
        // its buffers may still be in use on the device: the slot is retired
        S.error.store(HOUGH_ETIMEDOUT);
        fail_batch(S, sl, now_ns(), HOUGH_F_TIMEOUT);
        sl.busy = false;
        sl.dead = true;
        progress = true;
      }
    }
    Slot* free_slot = nullptr;
    for (Slot& sl : S.slots)
      if (!sl.busy && !sl.dead) {
        free_slot = &sl;
        break;
      }
    if (free_slot) {
      std::unique_lock<std::mutex> lk(S.mu);
      bool go = false;
      if (!S.pending.empty()) {
        const bool full = (int64_t)S.pending.size() >= S.cfg.max_batch_events || S.pending_hits >= S.cfg.max_batch_hits;
        const long long waited = now_ns() - S.pending.front().t_arrival;
        go = full || (S.cfg.flush_ns > 0 && waited >= S.cfg.flush_ns) || S.draining.load();
      }
      if (go) {
        int64_t hits = 0;
        while (!S.pending.empty() && (int64_t)free_slot->reqs.size() < S.cfg.max_batch_events &&
               hits + S.pending.front().n_hits <= S.cfg.max_batch_hits) {
          hits += S.pending.front().n_hits;
          free_slot->reqs.push_back(S.pending.front());
          S.pending.pop_front();
        }
        S.pending_hits -= hits;
        lk.unlock();
        if (!free_slot->reqs.empty()) {
          Slot& sl = *free_slot;
          const long long t_gather = now_ns();
          const cudaError_t e = launch_batch(S, sl);
          const long long t_launched = now_ns();
          if (e != cudaSuccess) {
            // Nothing of this batch may report results: its requests finish with the flag once
            // whatever was enqueued before the failure has drained from the slot's stream.
            note_cuda_error(e);
            if (!drain_slot(S, sl)) sl.dead = true;
            fail_batch(S, sl, now_ns(), HOUGH_F_LAUNCH_FAILED);
          } else {
            sl.busy = true;
            sl.t_launch = t_launched;
            std::lock_guard<std::mutex> tk(S.trace_mu);
            sl.rec = S.ring_next++;
            hough_serve_batch_record& r = record_at(S, sl.rec);
            r.t_gather = t_gather;
            r.t_launched = t_launched;
            r.t_done_seen = 0;
            r.t_finished = 0;
            r.n_events = (int32_t)sl.reqs.size();
            r.slot = (int32_t)(&sl - S.slots.data());
            r.n_hits = 0;
            for (const Request& q : sl.reqs) r.n_hits += q.n_hits;
            ++S.batches;
          }
          progress = true;
        }
      }
    }
    if (!progress) std::this_thread::yield();
  }
}

}  // namespace
}  // namespace hgpu

using namespace hgpu;

extern "C" {

static int serve_sizes(const hough_serve_config* c, SlotLayout& L, Plan& pl) {
  if (!c || c->slots < 1 || c->slots > 64 || c->max_batch_events < 1 || c->max_batch_hits < 1 ||
      c->queue_capacity < 1)
    return HOUGH_EINVAL;
  if (c->max_batch_hits > (int64_t)1 << 31) return HOUGH_EINVAL;
  int rc = make_plan(&c->params, pl, -1);
  if (rc) return rc;
  slot_layout(*c, pl, L);
  return HOUGH_OK;
}

int hough_serve_buffer_sizes(const hough_serve_config* c, size_t* device_bytes, size_t* pinned_bytes) {
  SlotLayout L;
  Plan pl;
  int rc = serve_sizes(c, L, pl);
  if (rc) return rc;
  if (device_bytes) *device_bytes = L.d_total * (size_t)c->slots;
  if (pinned_bytes) *pinned_bytes = L.h_total * (size_t)c->slots;
  return HOUGH_OK;
}

int hough_serve_open(const hough_serve_config* c, void* d_buf, size_t d_bytes, void* h_pinned, size_t h_bytes,
                     void** server) {
  if (!server || !d_buf || !h_pinned || ((uintptr_t)d_buf & 255) || ((uintptr_t)h_pinned & 255))
    return HOUGH_EINVAL;
  *server = nullptr;
  Server* S = new Server();
  int rc = serve_sizes(c, S->L, S->plan);
  if (rc) {
    delete S;
    return rc;
  }
  if (d_bytes < S->L.d_total * (size_t)c->slots || h_bytes < S->L.h_total * (size_t)c->slots) {
    delete S;
    return HOUGH_EWORKSPACE;
  }
  S->cfg = *c;
  // every buffer of the serving path is allocated and touched now, none later
  S->pending = Ring<Request>((size_t)c->queue_capacity);
  S->results = Ring<hough_serve_result>((size_t)c->queue_capacity + (size_t)c->slots * (size_t)c->max_batch_events);
  host_trig(c->params.n_theta, &S->trig);
  cudaGetDevice(&S->device);
  if (fused_max_ctas_per_sm(S->plan) < 1) {  // also sets the kernel's shared-memory limit
    delete S;
    return HOUGH_ESMEM;
  }
  S->slots.resize((size_t)c->slots);
  for (int i = 0; i < c->slots; ++i) {
    Slot& sl = S->slots[i];
    sl.reqs.reserve((size_t)c->max_batch_events);
    sl.out.reserve((size_t)c->max_batch_events);
    sl.d = (char*)d_buf + (size_t)i * S->L.d_total;
    sl.h = (char*)h_pinned + (size_t)i * S->L.h_total;
    void* mapped = nullptr;
    if (cudaHostGetDevicePointer(&mapped, sl.h + S->L.h_dense, 0) == cudaSuccess)
      sl.dense_mapped = (hough_peak*)mapped;
    else
      cudaGetLastError();  // not mapped: copy back instead
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      note_cuda_error(e);
      for (Slot& s2 : S->slots) {
        if (s2.done) cudaEventDestroy(s2.done);
        if (s2.stream) cudaStreamDestroy(s2.stream);
      }
      delete S;
      return HOUGH_ECUDA;
    }
  }
  S->running.store(true);
  S->loop = std::thread(serve_loop, S);
  *server = S;
  return HOUGH_OK;
}

static int submit_at(Server* S, const int32_t* h_xy, int64_t n_hits, int64_t id, uint8_t* h_mask_out,
                     hough_peak* h_peaks_out, hough_serve_result* h_result_out, long long t_arrival) {
  if (n_hits < 0 || (n_hits > 0 && !h_xy)) return HOUGH_EINVAL;
  if (n_hits > S->cfg.max_batch_hits || n_hits > HOUGH_MAX_EVENT_HITS) return HOUGH_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  // admitted only with room for the request in the queue and for its result in the ring
  if ((int64_t)S->pending.size() >= S->cfg.queue_capacity || S->outstanding >= (long long)S->results.capacity())
    return HOUGH_EFULL;
  S->pending.push_back(Request{h_xy, n_hits, id, h_mask_out, h_peaks_out, h_result_out, t_arrival});
  S->pending_hits += n_hits;
  ++S->outstanding;
  ++S->submitted;
  return HOUGH_OK;
}

int hough_serve_submit(void* server, const int32_t* h_xy, int64_t n_hits, int64_t id, uint8_t* h_mask_out,
                       hough_peak* h_peaks_out) {
  if (!server) return HOUGH_EINVAL;
  Server* S = (Server*)server;
  if (S->error.load()) return S->error.load();
  return submit_at(S, h_xy, n_hits, id, h_mask_out, h_peaks_out, nullptr, now_ns());
}

int hough_serve_poll(void* server, hough_serve_result* out, int32_t max_results, int32_t* n_out) {
  if (!server || !n_out || (max_results > 0 && !out)) return HOUGH_EINVAL;
  Server* S = (Server*)server;
  std::lock_guard<std::mutex> lk(S->mu);
  int32_t n = 0;
  while (n < max_results && !S->results.empty()) {
    out[n++] = S->results.front();
    S->results.pop_front();
    --S->outstanding;
  }
  *n_out = n;
  return S->error.load();
}

int hough_serve_drain(void* server, int64_t timeout_ns) {
  if (!server || timeout_ns < 0) return HOUGH_EINVAL;
  Server* S = (Server*)server;
  S->draining.store(true);  // partial micro-batches are launched at once
  std::unique_lock<std::mutex> lk(S->mu);
  const bool ok = S->cv.wait_for(lk, std::chrono::nanoseconds(timeout_ns),
                                 [&] { return S->completed >= S->submitted || S->error.load() != 0; });
  S->draining.store(false);
  if (S->error.load()) return S->error.load();
  return ok ? HOUGH_OK : HOUGH_ETIMEDOUT;
}

int hough_serve_close(void* server) {
  if (!server) return HOUGH_EINVAL;
  Server* S = (Server*)server;
  S->running.store(false);
  if (S->loop.joinable()) S->loop.join();
  for (Slot& sl : S->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  const int err = S->error.load();
  delete S;
  return err;
}

int hough_serve_replay(void* server, const int32_t* h_xy_pool, const int64_t* h_off_pool, int64_t pool_events,
                       const int64_t* arrival_ns, int64_t n_requests, int64_t* t_start_ns, uint8_t* h_mask_out,
                       hough_peak* h_peaks_out, hough_serve_result* h_results_out) {
  if (!server || !h_off_pool || pool_events < 1 || !arrival_ns || n_requests < 0) return HOUGH_EINVAL;
  Server* S = (Server*)server;
  const long long t0 = now_ns();
  if (t_start_ns) *t_start_ns = t0;
  StallWatch w;
  w.start(t0);
  int64_t m = 0;  // request i's mask offset
  int rc = HOUGH_OK;
  for (int64_t i = 0; i < n_requests && rc == HOUGH_OK; ++i) {
    const long long due = t0 + arrival_ns[i];
    long long t;
    while ((t = now_ns()) < due) w.tick(t);
    w.tick(t);
    const int64_t e = i % pool_events, nh = h_off_pool[e + 1] - h_off_pool[e];
    uint8_t* mo = h_mask_out ? h_mask_out + m : nullptr;
    hough_peak* po = h_peaks_out ? h_peaks_out + i * (int64_t)S->cfg.params.max_peaks : nullptr;
    m += nh;
    // admission is refused while the queue is full; retry (for at most 10 s) keeping the
    // scheduled arrival time, so the wait shows up in the latency
    hough_serve_result* ro = h_results_out ? h_results_out + i : nullptr;
    while ((rc = submit_at(S, h_xy_pool + 2 * h_off_pool[e], nh, i, mo, po, ro, due)) == HOUGH_EFULL) {
      if (now_ns() - due > 10000000000LL) {
        rc = HOUGH_ETIMEDOUT;
        break;
      }
      std::this_thread::yield();
    }
  }
  std::lock_guard<std::mutex> tk(S->trace_mu);
  S->submit_watch = w;
  return rc;
}

int hough_serve_trace(void* server, hough_serve_stats* out, hough_serve_batch_record* records, int32_t max_records,
                      int32_t* n_records) {
  if (!server || !out || max_records < 0 || (max_records > 0 && !records)) return HOUGH_EINVAL;
  Server* S = (Server*)server;
  std::lock_guard<std::mutex> tk(S->trace_mu);
  std::memset(out, 0, sizeof(*out));
  out->passes = S->passes;
  out->batches = S->batches;
  out->stall_ns = kStallNs;
  auto put = [](const StallWatch& w, hough_serve_stall* o) {
    o->count = w.stalls;
    o->max_gap_ns = w.max_gap;
    o->max_gap_at = w.max_at;
    o->user_ns = w.max_use.user_ns;
    o->sys_ns = w.max_use.sys_ns;
    o->minor_faults = w.max_use.minflt;
    o->voluntary_switches = w.max_use.nvcsw;
    o->involuntary_switches = w.max_use.nivcsw;
  };
  put(S->loop_watch, &out->loop);
  put(S->submit_watch, &out->submit);
  const long long avail = S->ring_next < HOUGH_SERVE_RECORDS ? S->ring_next : HOUGH_SERVE_RECORDS;
  const long long n = avail < max_records ? avail : max_records;
  for (long long i = 0; i < n; ++i) records[i] = record_at(*S, S->ring_next - n + i);
  if (n_records) *n_records = (int32_t)n;
  return HOUGH_OK;
}

int hough_serve_inject_launch_failures(void* server, int32_t n) {
  if (!server || n < 0) return HOUGH_EINVAL;
  ((Server*)server)->inject_failures.store(n);
  return HOUGH_OK;
}

}  // extern "C"
