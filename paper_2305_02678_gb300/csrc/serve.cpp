// Serving: continuous batching of frames.
//
// nam_submit queues a frame (host arrays, or device arrays with
// NAM_FRAME_DEVICE).  One scheduler thread per context admits queued frames
// in submission order, each once its arrival time has come (so that a paced
// stream does not depend on when its caller gets to run), a stream slot is
// free and the frame's device buffers fit under the HBM budget.  The slot's
// launcher thread then enqueues on the slot's stream the host->device
// copies, one multi-material tensor-core launch over the frame's tiles (each
// tile one material, so every 128-query MMA tile is material-coherent, the
// analogue of the paper's coherent warps, Sec. 7.3) and the device->host
// copy of the RGB; a device frame (the renderer's case) needs no copies.
// Frames on different slots run concurrently on the GPU, and a CUDA call
// that sleeps inside the driver holds up only its own slot.  The scheduler
// observes completion with CUDA events; per-frame latency is finish -
// arrival on the nam_now() clock.  Each frame's device timeline (copies
// begin, kernel begins and ends, copies end) is taken with timing events on
// its stream and mapped onto the nam_now() clock through an anchor event
// recorded while no frame is on the GPU.
#include <cuda_runtime.h>
#ifdef __linux__
#include <sys/prctl.h>
#endif

#include <algorithm>
#include <chrono>
#include <cstring>
#include <memory>

#include "nam_ctx.h"

using namespace nam;

namespace nam {

struct Job {
  nam_ticket ticket = 0;
  nam_frame frame{};
  std::vector<nam_material> mats;
  std::vector<Chunk> chunks;
  uint64_t bytes = 0;
  int nf = 9;
  nam_frame_stats st{};
  bool done = false;
  int slot = -1;
  void* dev = nullptr;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;      // after the RGB copy: the frame is complete
  cudaEvent_t begin = nullptr;     // before the frame's first copy
  cudaEvent_t k_begin = nullptr;   // before its kernel
  cudaEvent_t k_end = nullptr;     // after its kernel
  Job* job = nullptr;        // admitted frame (the scheduler sets and clears it)
  Job* pending = nullptr;    // handed to the slot's launcher thread
  bool launched = false;     // the launcher has enqueued job's work (or failed)
  nam_status launch_status = NAM_OK;
  // pinned staging for the frame's work table: an upload from pageable
  // memory could make the scheduler thread wait for the slot's stream.
  // Allocated with the slot (kTableBytes); a frame that outgrows it gets a
  // larger one and the old one is kept until serving stops, because freeing
  // pinned memory synchronises the device and would stall every frame in
  // flight.
  void* host_tab = nullptr;
  size_t host_tab_bytes = 0;
  std::vector<void*> retired_tabs;
};

// 4 MiB: the work table of a frame of 2^25 queries (262,144 chunks)
constexpr size_t kTableBytes = 4u << 20;

struct ServeState {
  std::mutex mu;                    // guards everything below but the CUDA objects
  std::condition_variable cv;       // wakes the scheduler
  std::unique_ptr<std::condition_variable[]> launcher_cv;  // one per slot
  std::vector<std::thread> launchers;
  std::condition_variable done_cv;  // wakes nam_wait
  std::deque<Job*> queue;
  std::map<nam_ticket, Job*> jobs;
  std::deque<nam_ticket> finished_order;
  std::vector<Slot> slots;
  std::thread thread;
  bool stop = false;
  nam_ticket next_ticket = 1;
  int64_t in_flight = 0, completed = 0, failed = 0, queries_completed = 0;
  uint64_t serving_bytes = 0;
  // the context pool is grown on the submitting thread (slots x the largest
  // frame so far), so that the scheduler's per-frame allocations come from
  // memory the pool already holds: growing it maps new memory and would hold
  // the scheduler thread, and with it every frame in flight
  std::mutex prime_mu;
  cudaStream_t prime_stream = nullptr;
  uint64_t primed_bytes = 0;
  std::deque<double> latencies_ms;
  double first_arrival = -1.0, last_finish = 0.0;
  // device-time anchor: anchor_ev completed at anchor_host_s (nam_now())
  cudaStream_t anchor_stream = nullptr;
  cudaEvent_t anchor_ev = nullptr;
  double anchor_host_s = 0.0;
  bool anchored = false;
};

}  // namespace nam

extern "C" double nam_now(void) {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Record the anchor event on its own (idle) stream and wait for it: the
// host time right after the wait is the anchor's time on the nam_now()
// clock, to within the wait's wake-up latency.  Called with no frame on the
// GPU, so that every frame's events come after the anchor.
static void take_anchor(ServeState* S) {
  S->anchored = false;
  if (cudaEventRecord(S->anchor_ev, S->anchor_stream) != cudaSuccess) return;
  if (cudaEventSynchronize(S->anchor_ev) != cudaSuccess) return;
  S->anchor_host_s = nam_now();
  S->anchored = true;
}

// A completed timing event's time on the nam_now() clock (0 if unknown).
static double device_time(const ServeState* S, cudaEvent_t ev) {
  if (!S->anchored) return 0.0;
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, S->anchor_ev, ev) != cudaSuccess) {
    cudaGetLastError();
    return 0.0;
  }
  return S->anchor_host_s + 1e-3 * (double)ms;
}

static void finish_job(ServeState* S, Job* j, nam_status status) {
  // S->mu held
  j->st.status = status;
  j->st.finish_s = nam_now();
  j->done = true;
  if (status == NAM_OK) {
    S->completed++;
    S->queries_completed += j->frame.n_queries;
    double lat = (j->st.finish_s - j->st.arrival_s) * 1e3;
    S->latencies_ms.push_back(lat);
    if (S->latencies_ms.size() > 4096) S->latencies_ms.pop_front();
    if (S->first_arrival < 0 || j->st.arrival_s < S->first_arrival) S->first_arrival = j->st.arrival_s;
    S->last_finish = std::max(S->last_finish, j->st.finish_s);
  } else {
    S->failed++;
  }
  S->finished_order.push_back(j->ticket);
  while (S->finished_order.size() > 65536) {
    auto it = S->jobs.find(S->finished_order.front());
    if (it != S->jobs.end()) {
      delete it->second;
      S->jobs.erase(it);
    }
    S->finished_order.pop_front();
  }
  S->done_cv.notify_all();
}

// Enqueue one admitted frame on its slot (S->mu not held).  Returns a status.
static nam_status launch_job(nam_ctx* ctx, Slot& slot, Job* j) {
  DeviceGuard g(ctx->device);
  cudaStream_t s = slot.stream;
  const int64_t n = j->frame.n_queries;
  if (ctx->fault_alloc.exchange(false)) return fail(NAM_ERR_OOM, "injected allocation failure");
  cudaError_t e = cudaMallocFromPoolAsync(&j->dev, j->bytes, ctx->pool, s);
  if (e != cudaSuccess) return cuda_fail((int)e, "serving: frame buffers");
  uint8_t* base = (uint8_t*)j->dev;
  const int64_t nfield = j->nf;
  const bool on_device = (j->frame.flags & NAM_FRAME_DEVICE) != 0;
  e = cudaEventRecord(slot.begin, s);
  if (e != cudaSuccess) return cuda_fail((int)e, "serving: event");
  // host frames: query fields, then the RGB, then the work table (int64
  // fields) at the next 16-byte boundary; device frames: the table alone.
  // The table goes first, from the slot's pinned buffer (free: the slot's
  // previous frame has completed)
  float* rgb = on_device ? j->frame.rgb_out : (float*)(base + (size_t)nfield * n * 4);
  uint8_t* tab = on_device ? base : base + (((size_t)nfield * n * 4 + (size_t)n * 12 + 15) / 16 * 16);
  const size_t cb = j->chunks.size() * sizeof(Chunk);
  const size_t pb = j->mats.size() * sizeof(void*);
  const size_t tb = cb + 2 * pb;
  if (tb > slot.host_tab_bytes) {
    void* bigger = nullptr;
    const size_t want = std::max<size_t>(tb * 2, kTableBytes);
    e = cudaMallocHost(&bigger, want);
    if (e != cudaSuccess) return cuda_fail((int)e, "serving: pinned table buffer");
    if (slot.host_tab) slot.retired_tabs.push_back(slot.host_tab);
    slot.host_tab = bigger;
    slot.host_tab_bytes = want;
  }
  uint8_t* host = (uint8_t*)slot.host_tab;
  std::memcpy(host, j->chunks.data(), cb);
  for (size_t k = 0; k < j->mats.size(); ++k) {
    const void* p = j->mats[k]->pyramid;
    const void* w = j->mats[k]->blob;
    std::memcpy(host + cb + k * sizeof(void*), &p, sizeof p);
    std::memcpy(host + cb + pb + k * sizeof(void*), &w, sizeof w);
  }
  e = cudaMemcpyAsync(tab, host, tb, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail((int)e, "serving: table upload");
  const float* src[10] = {j->frame.q.u, j->frame.q.v, j->frame.q.lod, j->frame.q.wix, j->frame.q.wiy,
                          j->frame.q.wiz, j->frame.q.wox, j->frame.q.woy, j->frame.q.woz, j->frame.q.xi};
  float* dst[10] = {nullptr};
  nam_queries dq = j->frame.q;
  if (!on_device) {
    for (int f = 0; f < j->nf; ++f) {
      dst[f] = (float*)(base + (size_t)f * n * 4);
      e = cudaMemcpyAsync(dst[f], src[f], (size_t)n * 4, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return cuda_fail((int)e, "serving: H2D");
    }
    dq = nam_queries{dst[0], dst[1], dst[2], dst[3], dst[4], dst[5], dst[6], dst[7], dst[8], dst[9]};
  }
  LaunchCommon L;
  fill_launch(ctx, j->mats[0], &dq, 0, rgb, j->frame.flags & ~(uint32_t)NAM_FRAME_DEVICE, &L);
  L.chunks = (const Chunk*)tab;
  L.n_chunks = (int32_t)j->chunks.size();
  L.mats.pyramid = (const void* const*)(tab + cb);
  L.mats.weights = (const void* const*)(tab + cb + pb);
  L.mats.nmat = (int32_t)j->mats.size();
  if (ctx->fault_launch.exchange(false)) return fail(NAM_ERR_CUDA, "injected launch failure");
  e = cudaEventRecord(slot.k_begin, s);
  if (e != cudaSuccess) return cuda_fail((int)e, "serving: event");
  int le = launch_material(L, j->mats[0]->desc.precision, s);
  if (le) return cuda_fail(le, "serving: launch");
  e = cudaEventRecord(slot.k_end, s);
  if (e != cudaSuccess) return cuda_fail((int)e, "serving: event");
  if (!on_device) {
    e = cudaMemcpyAsync(j->frame.rgb_out, rgb, (size_t)n * 12, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail((int)e, "serving: D2H");
  }
  cudaFreeAsync(j->dev, s);
  j->dev = nullptr;
  e = cudaEventRecord(slot.done, s);
  if (e != cudaSuccess) return cuda_fail((int)e, "serving: event");
  return NAM_OK;
}

// One launcher thread per slot enqueues its frames' work (launch_job), so
// that a CUDA call that sleeps inside the driver delays only its own frame:
// the scheduler thread never calls into a slot's stream.
static void launcher(nam_ctx* ctx, int k) {
  ServeState* S = ctx->serve;
  Slot& sl = S->slots[k];
  DeviceGuard g(ctx->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    S->launcher_cv[k].wait(lk, [&] { return S->stop || sl.pending != nullptr; });
    if (!sl.pending) break;  // stopping, nothing handed over
    Job* j = sl.pending;
    sl.pending = nullptr;
    lk.unlock();
    j->st.start_s = nam_now();
    nam_status st = launch_job(ctx, sl, j);
    j->st.enqueued_s = nam_now();
    if (st != NAM_OK) {
      if (j->dev) cudaFreeAsync(j->dev, sl.stream);
      j->dev = nullptr;
      cudaStreamSynchronize(sl.stream);
    }
    lk.lock();
    sl.launch_status = st;
    sl.launched = true;
    S->cv.notify_all();
  }
}

static void scheduler(nam_ctx* ctx) {
  ServeState* S = ctx->serve;
  DeviceGuard g(ctx->device);
#ifdef __linux__
  // timed waits wake within a microsecond of their deadline (the default
  // slack of 50 us would delay paced arrivals and completions)
  prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
#endif
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    bool progressed = false;
    // completions (and launches that failed)
    for (Slot& sl : S->slots) {
      if (!sl.job || !sl.launched) continue;
      nam_status st = sl.launch_status;
      cudaError_t q = cudaSuccess;
      if (st == NAM_OK) {
        q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) st = NAM_ERR_CUDA;
      }
      Job* j = sl.job;
      sl.job = nullptr;
      sl.launched = false;
      S->in_flight--;
      budget_release(ctx, j->bytes);
      S->serving_bytes -= j->bytes;
      if (st == NAM_OK) {
        j->st.gpu_begin_s = device_time(S, sl.begin);
        j->st.gpu_kernel_begin_s = device_time(S, sl.k_begin);
        j->st.gpu_kernel_end_s = device_time(S, sl.k_end);
        j->st.gpu_end_s = device_time(S, sl.done);
      }
      finish_job(S, j, st);
      progressed = true;
    }
    if (S->stop && S->in_flight == 0) break;
    // admissions, in submission order, each once its arrival time has come
    double next_arrival = 0.0;
    if (!S->stop && !ctx->fault_stall.load()) {
      for (size_t k = 0; k < S->slots.size(); ++k) {
        Slot& sl = S->slots[k];
        if (sl.job || S->queue.empty()) continue;
        Job* j = S->queue.front();
        const double now = nam_now();
        if (j->st.arrival_s > now) {
          next_arrival = j->st.arrival_s;
          break;
        }
        if (!budget_reserve(ctx, j->bytes)) break;  // head of line waits for memory
        S->queue.pop_front();
        S->serving_bytes += j->bytes;
        j->st.in_flight_at_admit = (int32_t)S->in_flight;
        S->in_flight++;
        j->st.admit_s = now;
        j->st.slot = (int32_t)k;
        sl.job = j;
        sl.pending = j;
        sl.launched = false;
        S->launcher_cv[k].notify_one();
        progressed = true;
      }
    }
    if (progressed) continue;
    const double now = nam_now();
    // idle GPU: refresh the device-time anchor every 10 s (the events'
    // FP32 millisecond offsets stay well below a microsecond)
    if (S->in_flight == 0 && (!S->anchored || now - S->anchor_host_s > 10.0) &&
        (next_arrival == 0.0 || next_arrival - now > 1e-3))
      take_anchor(S);
    double wait_s = S->in_flight ? 20e-6 : 2e-3;
    if (next_arrival > 0.0) wait_s = std::min(wait_s, std::max(next_arrival - nam_now(), 0.0));
    if (wait_s > 0.0) S->cv.wait_for(lk, std::chrono::nanoseconds((int64_t)(wait_s * 1e9)));
  }
}

static nam_status ensure_serving(nam_ctx* ctx) {
  std::lock_guard<std::mutex> lk(ctx->serve_mu);
  if (ctx->serve) return NAM_OK;
  DeviceGuard g(ctx->device);
  ServeState* S = new ServeState();
  S->slots.resize(ctx->serve_streams);
  auto release = [](ServeState* X) {
    for (Slot& x : X->slots) {
      if (x.stream) cudaStreamDestroy(x.stream);
      for (cudaEvent_t ev : {x.done, x.begin, x.k_begin, x.k_end})
        if (ev) cudaEventDestroy(ev);
      if (x.host_tab) cudaFreeHost(x.host_tab);
    }
    if (X->prime_stream) cudaStreamDestroy(X->prime_stream);
    if (X->anchor_stream) cudaStreamDestroy(X->anchor_stream);
    if (X->anchor_ev) cudaEventDestroy(X->anchor_ev);
    delete X;
  };
  cudaError_t e = cudaSuccess;
  for (Slot& sl : S->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&sl.done, &sl.begin, &sl.k_begin, &sl.k_end})
      if (e == cudaSuccess) e = cudaEventCreate(ev);  // timing events
    if (e == cudaSuccess) e = cudaMallocHost(&sl.host_tab, kTableBytes);
    if (e == cudaSuccess) sl.host_tab_bytes = kTableBytes;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->prime_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->anchor_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&S->anchor_ev);
  if (e != cudaSuccess) {
    release(S);
    return cuda_fail((int)e, "serving: stream creation");
  }
  take_anchor(S);
  S->launcher_cv.reset(new std::condition_variable[S->slots.size()]);
  ctx->serve = S;
  for (size_t k = 0; k < S->slots.size(); ++k) S->launchers.emplace_back(launcher, ctx, (int)k);
  S->thread = std::thread(scheduler, ctx);
  return NAM_OK;
}

void nam::serve_stop(nam_ctx* ctx) {
  ServeState* S;
  {
    std::lock_guard<std::mutex> lk(ctx->serve_mu);
    S = ctx->serve;
    if (!S) return;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    while (!S->queue.empty()) {
      Job* j = S->queue.front();
      S->queue.pop_front();
      finish_job(S, j, NAM_ERR_CANCELLED);
    }
  }
  ctx->fault_stall.store(false);
  S->cv.notify_all();
  S->thread.join();  // returns once no frame is in flight
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (size_t k = 0; k < S->slots.size(); ++k) S->launcher_cv[k].notify_all();
  }
  for (std::thread& t : S->launchers) t.join();
  DeviceGuard g(ctx->device);
  for (Slot& sl : S->slots) {
    cudaStreamSynchronize(sl.stream);
    cudaStreamDestroy(sl.stream);
    for (cudaEvent_t ev : {sl.done, sl.begin, sl.k_begin, sl.k_end}) cudaEventDestroy(ev);
    if (sl.host_tab) cudaFreeHost(sl.host_tab);
    for (void* t : sl.retired_tabs) cudaFreeHost(t);
  }
  cudaStreamDestroy(S->prime_stream);
  cudaStreamDestroy(S->anchor_stream);
  cudaEventDestroy(S->anchor_ev);
  for (auto& kv : S->jobs) delete kv.second;
  delete S;
  ctx->serve = nullptr;
}

extern "C" nam_status nam_submit(nam_ctx* ctx, const nam_frame* f, nam_ticket* out) {
  if (!ctx || !f || !out) return fail(NAM_ERR_INVALID_ARG, "nam_submit: NULL argument");
  *out = 0;
  if (f->n_queries <= 0 || f->n_items <= 0 || !f->items || !f->rgb_out)
    return fail(NAM_ERR_INVALID_ARG, "nam_submit: empty frame");
  nam_status st = check_multi(ctx, f->materials, f->n_materials);
  if (st) return st;
  st = check_queries(f->materials[0], &f->q);
  if (st) return st;
  Job* j = new Job();
  j->frame = *f;
  j->mats.assign(f->materials, f->materials + f->n_materials);
  for (int32_t i = 0; i < f->n_items; ++i) {
    const nam_work_item& it = f->items[i];
    if (it.material < 0 || it.material >= f->n_materials || it.count < 0 || it.start < 0 ||
        it.start + it.count > f->n_queries) {
      delete j;
      return fail(NAM_ERR_INVALID_ARG, "nam_submit: bad work item %d", i);
    }
  }
  build_chunks(f->items, f->n_items, &j->chunks);
  j->nf = f->materials[0]->desc.filter == NAM_FILTER_STOCHASTIC ? 10 : 9;
  const int64_t n = f->n_queries;
  // device buffers the frame needs from the pool: a host frame's copy of its
  // query fields and its RGB, and the work table
  const uint64_t io = (f->flags & NAM_FRAME_DEVICE) ? 0 : ((uint64_t)n * 4 * j->nf + (uint64_t)n * 12 + 15) / 16 * 16;
  j->bytes = io + j->chunks.size() * sizeof(Chunk) + 2 * j->mats.size() * sizeof(void*) + 256;
  j->st.submit_s = nam_now();
  j->st.arrival_s = f->arrival_s > 0 ? f->arrival_s : j->st.submit_s;
  j->st.n_queries = n;
  j->st.slot = -1;
  st = ensure_serving(ctx);
  if (st) {
    delete j;
    return st;
  }
  ServeState* S = ctx->serve;
  {
    std::lock_guard<std::mutex> pk(S->prime_mu);
    uint64_t want = (uint64_t)ctx->serve_streams * j->bytes;
    if (ctx->budget) {
      const uint64_t res = ctx->resident.load();
      want = std::min<uint64_t>(want, ctx->budget > res ? ctx->budget - res : 0);
    }
    if (want > S->primed_bytes) {
      DeviceGuard g(ctx->device);
      void* p = nullptr;
      if (cudaMallocFromPoolAsync(&p, want, ctx->pool, S->prime_stream) == cudaSuccess) {
        cudaFreeAsync(p, S->prime_stream);
        if (cudaStreamSynchronize(S->prime_stream) == cudaSuccess) S->primed_bytes = want;
      }
      cudaGetLastError();  // a failed reservation only means the scheduler grows the pool itself
    }
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (ctx->budget) {
      const uint64_t other = ctx->resident.load() - S->serving_bytes;
      if (j->bytes + other > ctx->budget) {
        delete j;
        return fail(NAM_ERR_BUDGET, "nam_submit: frame needs %llu bytes, budget leaves %llu",
                    (unsigned long long)j->bytes, (unsigned long long)(ctx->budget - std::min(other, ctx->budget)));
      }
    }
    if ((int)S->queue.size() >= ctx->serve_queue_depth) {
      delete j;
      return fail(NAM_ERR_BUSY, "nam_submit: admission queue full");
    }
    j->ticket = S->next_ticket++;
    S->jobs[j->ticket] = j;
    S->queue.push_back(j);
    *out = j->ticket;
  }
  S->cv.notify_all();
  return NAM_OK;
}

extern "C" nam_status nam_poll(nam_ctx* ctx, nam_ticket t, int32_t* done, nam_frame_stats* st) {
  if (!ctx || !done) return fail(NAM_ERR_INVALID_ARG, "nam_poll: NULL argument");
  ServeState* S = ctx->serve;
  if (!S) return fail(NAM_ERR_NOT_FOUND, "nam_poll: no frames submitted");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(t);
  if (it == S->jobs.end()) return fail(NAM_ERR_NOT_FOUND, "nam_poll: unknown ticket");
  *done = it->second->done ? 1 : 0;
  if (st) *st = it->second->st;
  return NAM_OK;
}

extern "C" nam_status nam_wait(nam_ctx* ctx, nam_ticket t, uint64_t timeout_ns, nam_frame_stats* st) {
  if (!ctx) return fail(NAM_ERR_INVALID_ARG, "nam_wait: NULL context");
  ServeState* S = ctx->serve;
  if (!S) return fail(NAM_ERR_NOT_FOUND, "nam_wait: no frames submitted");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(t);
  if (it == S->jobs.end()) return fail(NAM_ERR_NOT_FOUND, "nam_wait: unknown ticket");
  Job* j = it->second;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::nanoseconds(timeout_ns ? timeout_ns : ctx->timeout_ns);
  while (!j->done) {
    if (S->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && !j->done)
      return fail(NAM_ERR_TIMEOUT, "nam_wait: ticket %llu not done", (unsigned long long)t);
  }
  if (st) *st = j->st;
  if (j->st.status != NAM_OK) return fail(j->st.status, "frame %llu failed: %s", (unsigned long long)t, nam_status_string(j->st.status));
  return NAM_OK;
}

extern "C" nam_status nam_cancel(nam_ctx* ctx, nam_ticket t) {
  if (!ctx) return fail(NAM_ERR_INVALID_ARG, "nam_cancel: NULL context");
  ServeState* S = ctx->serve;
  if (!S) return fail(NAM_ERR_NOT_FOUND, "nam_cancel: no frames submitted");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(t);
  if (it == S->jobs.end()) return fail(NAM_ERR_NOT_FOUND, "nam_cancel: unknown ticket");
  Job* j = it->second;
  if (j->done) return NAM_OK;
  auto qi = std::find(S->queue.begin(), S->queue.end(), j);
  if (qi == S->queue.end()) return fail(NAM_ERR_BUSY, "nam_cancel: frame already on the GPU");
  S->queue.erase(qi);
  finish_job(S, j, NAM_ERR_CANCELLED);
  return NAM_OK;
}

extern "C" nam_status nam_get_stats(nam_ctx* ctx, nam_stats* out) {
  if (!ctx || !out) return fail(NAM_ERR_INVALID_ARG, "nam_get_stats: NULL argument");
  std::memset(out, 0, sizeof *out);
  out->resident_bytes = ctx->resident.load();
  out->budget_bytes = ctx->budget;
  ServeState* S = ctx->serve;
  if (!S) return NAM_OK;
  std::lock_guard<std::mutex> lk(S->mu);
  out->queued = (int64_t)S->queue.size();
  out->in_flight = S->in_flight;
  out->completed = S->completed;
  out->failed = S->failed;
  out->queries_completed = S->queries_completed;
  if (!S->latencies_ms.empty()) {
    std::vector<double> v(S->latencies_ms.begin(), S->latencies_ms.end());
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
      double pos = p * (v.size() - 1);
      size_t lo = (size_t)pos;
      size_t hi = std::min(lo + 1, v.size() - 1);
      return v[lo] + (v[hi] - v[lo]) * (pos - lo);
    };
    out->p50_latency_ms = pct(0.50);
    out->p99_latency_ms = pct(0.99);
  }
  if (S->last_finish > S->first_arrival && S->first_arrival >= 0)
    out->evals_per_s = S->queries_completed / (S->last_finish - S->first_arrival);
  return NAM_OK;
}

extern "C" nam_status nam_inject_fault(nam_ctx* ctx, int32_t fault) {
  if (!ctx) return fail(NAM_ERR_INVALID_ARG, "NULL context");
  switch (fault) {
    case NAM_FAULT_NONE:
      ctx->fault_alloc = false;
      ctx->fault_launch = false;
      ctx->fault_stall = false;
      break;
    case NAM_FAULT_ALLOC: ctx->fault_alloc = true; break;
    case NAM_FAULT_LAUNCH: ctx->fault_launch = true; break;
    case NAM_FAULT_STALL: ctx->fault_stall = true; break;
    default: return fail(NAM_ERR_INVALID_ARG, "unknown fault %d", fault);
  }
  if (ctx->serve) ctx->serve->cv.notify_all();
  return NAM_OK;
}
