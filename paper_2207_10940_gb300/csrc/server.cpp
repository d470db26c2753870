// Serving loop of the tracking library (include/dri.h, dri_server_*): many
// independent camera streams, each tracked frame by frame as in Sec. IV, share
// one GPU through continuous batching.
//
// Clients submit requests (a frame, with the IMU samples since the stream's
// previous frame) from any thread and poll tickets.  One worker thread owns
// every stream handle: it takes the oldest pending request of each stream (at
// most max_batch streams per tick), uploads them and launches one batched frame
// (dri_track_batch's plan over all the server's streams; streams without a
// request sit the tick out).  One tick is on the GPU at a time: every request
// that arrives while it runs joins the next tick, launched when it completes,
// so a request waits at most for the running tick and its own.  (With a second
// tick launched behind the running one, that tick takes only the few requests
// that came in meanwhile and the rest wait for a third: at the 256-stream
// mixed load p50 / p99 were 40 / 54 ms against 27 / 35 ms.)  A stream is admitted only while the device bytes
// of all admitted streams stay within the HBM budget.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "host.h"

using namespace dri_host;

namespace {

constexpr int kInflight = 1;                 // ticks on the GPU at once
constexpr size_t kSlotOverheadBytes = 65536; // plan table, staging and result head of one slot
constexpr size_t kMaxLatencySamples = 1 << 20;
constexpr size_t kTraceTicks = 1 << 16;      // per-tick timestamps kept (a ring)

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
  dri_stream_s* s;
  double t;
  const float* depth;
  const float* inten;
  size_t pitch;
  int32_t mem_kind;
  std::vector<dri_imu_sample> imu;
  uint64_t ticket;
};

struct Ticket {
  bool done = false;
  int status = DRI_OK;
  dri_track_result res;
  Clock::time_point t_submit;
};

struct TickEntry {
  int slot;
  uint64_t ticket;
  bool init;
  double t0;
};

struct Tick {
  Plan* plan;
  int ring_slot;
  std::vector<TickEntry> entries;
  dri_server_tick trace;                      // done_ms filled when the tick completes
  int ev;                                     // timing events of the tick (-1: none)
};

constexpr int kTickEvents = 4;                // pairs of timing events (ticks in flight + 1)

}  // namespace

struct dri_server_s {
  size_t budget = 0, used = 0;
  int max_batch = 0;
  cudaStream_t stream = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  // admitted streams, in slot order of the plan, and their device bytes
  std::vector<dri_stream_s*> streams;
  std::unordered_map<dri_stream_s*, size_t> cost;
  std::unordered_map<dri_stream_s*, std::deque<Request>> queues;
  std::vector<dri_stream_s*> closing;
  std::vector<dri_stream_s*> closed;
  bool dirty = false;                         // stream set changed since the last plan
  std::vector<dri_stream_s*> plan_key;        // stream list of the current plan
  bool have_tiles = false;                    // rows per thread chosen by the first plan
  int32_t tiles[DRI_MAX_LEVELS] = {};
  int32_t levels = 0, iters[DRI_MAX_LEVELS] = {}, flags = 0;
  int opt = 0;                                // pixel-kernel options (every stream alike)
  std::unordered_map<uint64_t, Ticket> tickets;
  uint64_t next_ticket = 1;
  std::deque<Tick> inflight;
  int64_t pending = 0;
  // statistics since the last reset
  int64_t submitted = 0, completed = 0, failed = 0, ticks = 0, tick_frames = 0;
  std::vector<double> lat_ms;
  Clock::time_point t_first_submit, t_last_done;
  bool any_submit = false;
  // per-tick host timestamps (ms since creation), the last kTraceTicks ticks
  Clock::time_point t_created;
  std::vector<dri_server_tick> trace;
  size_t trace_next = 0;
  int64_t tick_seq = 0;
  cudaEvent_t tev[kTickEvents][2] = {};       // device time of a tick's launch sequence
  int tev_next = 0;
};

namespace {

double since_created(const dri_server_s* S) { return ms_since(S->t_created, Clock::now()); }

// Records a finished tick's timestamps (lock held).
void record_tick(dri_server_s* S, const dri_server_tick& t) {
  if (S->trace.size() < kTraceTicks) {
    S->trace.push_back(t);
  } else {
    S->trace[S->trace_next] = t;
    S->trace_next = (S->trace_next + 1) % kTraceTicks;
  }
}

void finish_ticket(dri_server_s* S, uint64_t id, int status, const dri_track_result* res) {
  auto it = S->tickets.find(id);
  if (it == S->tickets.end()) return;
  Ticket& t = it->second;
  t.done = true;
  t.status = status;
  if (res) t.res = *res;
  else std::memset(&t.res, 0, sizeof(t.res));
  t.res.status = status;
  const Clock::time_point now = Clock::now();
  if (S->lat_ms.size() < kMaxLatencySamples) S->lat_ms.push_back(ms_since(t.t_submit, now));
  S->t_last_done = now;
  S->completed++;
  if (status != DRI_OK) S->failed++;
}

// Completes the oldest in-flight tick (its event has completed).  Called with
// the lock held.
void complete_tick(dri_server_s* S) {
  Tick tk = S->inflight.front();
  S->inflight.pop_front();
  tk.trace.done_ms = since_created(S);
  float ms = -1.f;
  if (tk.ev >= 0 && cudaEventElapsedTime(&ms, S->tev[tk.ev][0], S->tev[tk.ev][1]) != cudaSuccess) {
    cudaGetLastError();
    ms = -1.f;
  }
  tk.trace.device_ms = ms;
  record_tick(S, tk.trace);
  for (const TickEntry& e : tk.entries) {
    dri_stream_s* s = tk.plan->slots[e.slot];
    settle(s, false);                          // this tick's frame has completed
    dri_track_result r;
    const Ctrl* h = ring_head(tk.plan, tk.ring_slot, e.slot);
    fill_result(s, h, &r, e.init, e.t0);
    finish_ticket(S, e.ticket, h->status, &r);
  }
  S->cv_done.notify_all();
}

// Plan over all admitted streams, rebuilt (worker, nothing in flight) when the
// set changed.  The first plan tunes the rows per thread; later ones reuse them.
int current_plan(dri_server_s* S, Plan** out) {
  if (S->dirty || S->plan_key != S->streams) {
    if (S->plan_key.size() > 1) release_batch_plan(S->plan_key);
    S->plan_key = S->streams;
    S->dirty = false;
  }
  std::vector<dri_stream> key(S->plan_key.begin(), S->plan_key.end());
  const int r = batch_plan(key.data(), (int32_t)key.size(), out);
  if (r != DRI_OK) return r;
  if (key.size() > 1 && S->have_tiles) {
    dri_batch_options o;
    dri_batch_get_options(key.data(), (int32_t)key.size(), &o);
    bool same = !o.autotune;
    for (int l = 0; l < S->levels && same; ++l) same = o.rows_per_thread[l] == S->tiles[l];
    if (!same) {
      for (int l = 0; l < DRI_MAX_LEVELS; ++l) o.rows_per_thread[l] = S->tiles[l];
      o.autotune = 0;                 // the plan keeps its default slot groups
      const int rs = dri_batch_set_options(key.data(), (int32_t)key.size(), &o);
      if (rs != DRI_OK) return rs;
    }
  }
  return DRI_OK;
}

void remember_tiles(dri_server_s* S) {
  if (S->have_tiles || S->plan_key.size() < 2) return;
  std::vector<dri_stream> key(S->plan_key.begin(), S->plan_key.end());
  dri_batch_options o;
  if (dri_batch_get_options(key.data(), (int32_t)key.size(), &o) != DRI_OK || o.autotune) return;
  for (int l = 0; l < DRI_MAX_LEVELS; ++l) S->tiles[l] = o.rows_per_thread[l];
  S->have_tiles = true;
}

void worker_main(dri_server_s* S) {
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    // completed ticks
    while (!S->inflight.empty()) {
      const Tick& t = S->inflight.front();
      if (cudaEventQuery(t.plan->ev[t.ring_slot]) != cudaSuccess) break;
      complete_tick(S);
    }
    // streams to close: once nothing of theirs is queued or in flight
    if (!S->closing.empty() && S->inflight.empty()) {
      std::vector<dri_stream_s*> now;
      for (dri_stream_s* s : S->closing)
        if (S->queues[s].empty()) now.push_back(s);
      if (!now.empty()) {
        for (dri_stream_s* s : now) {
          S->closing.erase(std::find(S->closing.begin(), S->closing.end(), s));
          S->streams.erase(std::find(S->streams.begin(), S->streams.end(), s));
          S->queues.erase(s);
          S->used -= S->cost[s];
          S->cost.erase(s);
        }
        const std::vector<dri_stream_s*> old = S->plan_key;
        S->plan_key.clear();
        S->dirty = true;
        lk.unlock();
        if (old.size() > 1) release_batch_plan(old);
        for (dri_stream_s* s : now) dri_destroy_stream(s);
        lk.lock();
        for (dri_stream_s* s : now) S->closed.push_back(s);
        S->cv_done.notify_all();
        continue;
      }
    }
    // a new tick
    const bool plan_change = S->dirty || S->plan_key != S->streams;
    if (S->pending > 0 && (int)S->inflight.size() < kInflight && !(plan_change && !S->inflight.empty())) {
      // oldest request first, one per stream
      std::vector<std::pair<uint64_t, dri_stream_s*>> order;
      for (dri_stream_s* s : S->streams) {
        auto& q = S->queues[s];
        if (!q.empty()) order.push_back({q.front().ticket, s});
      }
      std::sort(order.begin(), order.end());
      if ((int)order.size() > S->max_batch) order.resize(S->max_batch);
      dri_server_tick tr;
      std::memset(&tr, 0, sizeof(tr));
      tr.tick = S->tick_seq++;
      tr.requests = (int32_t)order.size();
      tr.dequeue_ms = since_created(S);
      std::vector<Request> reqs;
      for (auto& o : order) {
        reqs.push_back(std::move(S->queues[o.second].front()));
        S->queues[o.second].pop_front();
        S->pending--;
      }
      Plan* plan = nullptr;
      int rp = current_plan(S, &plan);
      lk.unlock();
      std::vector<int> up(reqs.size(), DRI_OK);
      for (size_t i = 0; i < reqs.size(); ++i) {
        Request& q = reqs[i];
        if (!q.imu.empty()) up[i] = dri_push_imu(q.s, q.imu.data(), q.imu.size());
        if (up[i] == DRI_OK)
          up[i] = dri_upload_frame(q.s, q.t, q.depth, q.inten, q.pitch, q.mem_kind);
      }
      tr.staged_ms = since_created(S);
      std::vector<SlotWork> work;
      std::vector<double> t0;
      int rs = -1;
      int tev = -1;
      if (rp == DRI_OK) {
        work.resize(plan->S);
        t0.resize(plan->S);
        for (int i = 0; i < plan->S; ++i) {
          dri_stream_s* s = plan->slots[i];
          settle(s, false);
          work[i] = plan_slot_work(s);
          t0[i] = s->t_prev;
          if (work[i].mode == kSlotIdle && s->frame_pending) s->frame_pending = false;   // IMU short
        }
        bool any = false;
        for (const SlotWork& w : work) any = any || w.mode != kSlotIdle;
        if (any) {
          tev = S->tev[S->tev_next][0] ? S->tev_next : -1;
          if (tev >= 0) cudaEventRecord(S->tev[tev][0], S->stream);
          rp = plan_launch(plan, work, &rs);
          if (tev >= 0) cudaEventRecord(S->tev[tev][1], S->stream);
          S->tev_next = (S->tev_next + 1) % kTickEvents;
        }
      }
      tr.launched_ms = since_created(S);
      tr.status = rp;
      lk.lock();
      Tick tk{plan, rs, {}, tr, tev};
      for (size_t i = 0; i < reqs.size(); ++i) {
        int slot = -1;
        if (rp == DRI_OK && rs >= 0)
          for (int k = 0; k < plan->S; ++k)
            if (plan->slots[k] == reqs[i].s) slot = k;
        if (up[i] != DRI_OK) {
          finish_ticket(S, reqs[i].ticket, up[i], nullptr);
        } else if (rp != DRI_OK) {
          finish_ticket(S, reqs[i].ticket, rp, nullptr);
        } else if (slot < 0 || work[slot].mode == kSlotIdle) {
          finish_ticket(S, reqs[i].ticket, slot < 0 ? DRI_ENOTREADY : work[slot].status, nullptr);
        } else {
          tk.entries.push_back({slot, reqs[i].ticket, work[slot].mode == kSlotInit, t0[slot]});
        }
      }
      if (!tk.entries.empty()) {
        S->inflight.push_back(tk);
        S->ticks++;
        S->tick_frames += (int64_t)tk.entries.size();
      } else {                                 // nothing on the GPU: done as launched
        tk.trace.done_ms = tk.trace.launched_ms;
        tk.trace.device_ms = 0.0;
        record_tick(S, tk.trace);
      }
      if (rp == DRI_OK && rs >= 0) remember_tiles(S);
      S->cv_done.notify_all();
      continue;
    }
    if (S->stop && S->pending == 0 && S->inflight.empty() && S->closing.empty()) break;
    if (!S->inflight.empty()) {
      cudaEvent_t ev = S->inflight.front().plan->ev[S->inflight.front().ring_slot];
      lk.unlock();
      cudaEventSynchronize(ev);
      lk.lock();
      continue;
    }
    S->cv_work.wait(lk);
  }
}

}  // namespace

extern "C" {

int dri_server_create(size_t hbm_budget_bytes, int32_t max_batch, void* cuda_stream, dri_server* out) {
  if (!out || hbm_budget_bytes == 0 || max_batch < 1 || max_batch > 4096) return DRI_EINVAL;
  *out = nullptr;
  dri_server_s* S = new (std::nothrow) dri_server_s();
  if (!S) return DRI_ENOMEM;
  S->budget = hbm_budget_bytes;
  S->max_batch = max_batch;
  S->stream = (cudaStream_t)cuda_stream;
  S->t_created = Clock::now();
  for (int i = 0; i < kTickEvents; ++i)         // without events the trace reports device_ms -1
    for (int j = 0; j < 2; ++j)
      if (cudaEventCreate(&S->tev[i][j]) != cudaSuccess) {
        cudaGetLastError();
        S->tev[i][j] = nullptr;
      }
  try {
    S->worker = std::thread(worker_main, S);
  } catch (...) {
    delete S;
    return DRI_ENOMEM;
  }
  *out = S;
  return DRI_OK;
}

int dri_server_destroy(dri_server S) {
  if (!S) return DRI_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (dri_stream_s* s : S->streams)
      if (std::find(S->closing.begin(), S->closing.end(), s) == S->closing.end())
        S->closing.push_back(s);
    S->stop = true;
  }
  S->cv_work.notify_all();
  S->worker.join();
  for (int i = 0; i < kTickEvents; ++i)
    for (int j = 0; j < 2; ++j)
      if (S->tev[i][j]) cudaEventDestroy(S->tev[i][j]);
  delete S;
  return DRI_OK;
}

int dri_server_open_stream(dri_server S, const dri_stream_config* cfg, const dri_state* x_init,
                           dri_stream* out) {
  if (!S || !cfg || !x_init || !out) return DRI_EINVAL;
  *out = nullptr;
  size_t ws = 0;
  int r = dri_stream_workspace_bytes(cfg, &ws);
  if (r != DRI_OK) return r;
  const size_t need = ws + kSlotOverheadBytes;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return DRI_EINVAL;
    if (!S->streams.empty()) {
      bool same = cfg->levels == S->levels && cfg->precision_flags == S->flags &&
                  pixel_options(*cfg) == S->opt;
      for (int l = 0; l < cfg->levels && same; ++l) same = cfg->iters[l] == S->iters[l];
      if (!same) return DRI_EINVAL;
    }
    if (S->used + need > S->budget) return DRI_EADMIT;
    S->used += need;                           // reserved while the stream is created
  }
  dri_stream s = nullptr;
  r = dri_create_stream(cfg, x_init, S->stream, nullptr, 0, &s);
  std::lock_guard<std::mutex> lk(S->mu);
  if (r != DRI_OK) {
    S->used -= need;
    return r;
  }
  if (S->streams.empty()) {
    S->levels = cfg->levels;
    S->flags = cfg->precision_flags;
    S->opt = pixel_options(*cfg);
    for (int l = 0; l < DRI_MAX_LEVELS; ++l) S->iters[l] = l < cfg->levels ? cfg->iters[l] : 0;
  }
  S->streams.push_back(s);
  S->cost[s] = need;
  S->queues[s];
  S->dirty = true;
  *out = s;
  return DRI_OK;
}

int dri_server_close_stream(dri_server S, dri_stream s) {
  if (!S || !s) return DRI_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  if (std::find(S->streams.begin(), S->streams.end(), s) == S->streams.end()) return DRI_EINVAL;
  if (std::find(S->closing.begin(), S->closing.end(), s) == S->closing.end()) S->closing.push_back(s);
  S->cv_work.notify_all();
  S->cv_done.wait(lk, [&] {
    return std::find(S->closed.begin(), S->closed.end(), s) != S->closed.end();
  });
  S->closed.erase(std::find(S->closed.begin(), S->closed.end(), s));
  return DRI_OK;
}

int dri_server_submit(dri_server S, dri_stream s, double t, const float* depth,
                      const float* intensity, size_t pitch_bytes, int32_t mem_kind,
                      const dri_imu_sample* imu, size_t n_imu, uint64_t* ticket) {
  if (!S || !s || !depth || !intensity || !ticket || (n_imu && !imu)) return DRI_EINVAL;
  if (mem_kind != DRI_HOST && mem_kind != DRI_DEVICE) return DRI_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop || std::find(S->streams.begin(), S->streams.end(), s) == S->streams.end() ||
      std::find(S->closing.begin(), S->closing.end(), s) != S->closing.end())
    return DRI_EINVAL;
  Request q;
  q.s = s;
  q.t = t;
  q.depth = depth;
  q.inten = intensity;
  q.pitch = pitch_bytes;
  q.mem_kind = mem_kind;
  q.imu.assign(imu, imu + n_imu);
  q.ticket = S->next_ticket++;
  Ticket& tk = S->tickets[q.ticket];
  tk.t_submit = Clock::now();
  if (!S->any_submit) {
    S->any_submit = true;
    S->t_first_submit = tk.t_submit;
  }
  *ticket = q.ticket;
  S->queues[s].push_back(std::move(q));
  S->pending++;
  S->submitted++;
  S->cv_work.notify_all();
  return DRI_OK;
}

int dri_server_poll(dri_server S, uint64_t ticket, dri_track_result* out, int32_t timeout_ms) {
  if (!S) return DRI_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return DRI_EINVAL;
  auto ready = [&] { return S->tickets[ticket].done; };
  if (timeout_ms < 0) S->cv_done.wait(lk, ready);
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return DRI_ETIMEDOUT;
  const Ticket t = S->tickets[ticket];
  S->tickets.erase(ticket);
  if (out) *out = t.res;
  return t.status;
}

int dri_server_stats_read(dri_server S, int32_t reset, dri_server_stats* out) {
  if (!S || !out) return DRI_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->failed = S->failed;
  out->ticks = S->ticks;
  out->mean_batch = S->ticks ? (double)S->tick_frames / S->ticks : 0.0;
  out->streams = (int32_t)S->streams.size();
  out->hbm_used = S->used;
  out->hbm_budget = S->budget;
  if (!S->lat_ms.empty()) {
    std::vector<double> v = S->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = v.back();
  }
  if (S->any_submit && S->completed > 0) {
    const double span = ms_since(S->t_first_submit, S->t_last_done) / 1000.0;
    out->frames_per_s = span > 0 ? (double)S->completed / span : 0.0;
  }
  if (reset) {
    S->submitted = S->completed = S->failed = S->ticks = S->tick_frames = 0;
    S->lat_ms.clear();
    S->any_submit = false;
    S->trace.clear();
    S->trace_next = 0;
  }
  return DRI_OK;
}

int dri_server_trace_read(dri_server S, dri_server_tick* out, int32_t cap, int32_t* n) {
  if (!S || !n || cap < 0 || (cap > 0 && !out)) return DRI_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  const size_t have = S->trace.size();
  const size_t k = std::min(have, (size_t)cap);
  // oldest first: the ring starts at trace_next once it is full
  const size_t first = have < kTraceTicks ? 0 : S->trace_next;
  for (size_t i = 0; i < k; ++i) out[i] = S->trace[(first + (have - k) + i) % have];
  *n = (int32_t)k;
  return DRI_OK;
}

}  // extern "C"
