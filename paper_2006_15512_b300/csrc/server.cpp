// Continuous-batching WMC server over one compiled plan.
//
// Queries (weight vectors) arrive through wmc_submit.  A batcher thread
// forms a wave from what is queued as soon as a wave slot is free: the
// wave's Q is the next power of two >= the count it takes (capped at
// max_batch; padding lanes repeat the last query and are discarded), and it
// takes fewer queries, a power of two of them, rather than pad more than a
// quarter of the lanes (wave_take).  A partial wave starts only when no
// wave is running: while one runs, arrivals accumulate into the next, so
// the wave size grows with the load; a full wave starts in any free slot
// (throughput-bound serving overlaps full waves).  Each
// slot owns a stream and a workspace sized for max_batch, so admission is
// by the plan's workspace bytes: the number of slots is what fits in
// arena_bytes.  Waves on different slots overlap on the device.  A host
// callback on the slot's stream hands the finished wave to a completion
// thread, which publishes per-ticket results and frees the slot.  The query
// index is a pure batch index of every contraction and every per-query
// exponent depends only on that query, so a result does not depend on the
// wave it lands in.
#include <cuda_runtime.h>

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

#include "internal.h"

using namespace wmc;

namespace {

struct Query {
  uint64_t ticket;
  std::vector<double> wp, wn;
  bool negative;
};

struct Slot {
  cudaStream_t stream = nullptr;
  void *ws = nullptr;
  double *d_w = nullptr;          // [2][max_batch][n_vars]
  double *h_w = nullptr;          // pinned staging
  double *d_mant = nullptr;
  int64_t *d_exp = nullptr;
  uint32_t *d_flags = nullptr;
  double *h_mant = nullptr;       // pinned results
  int64_t *h_exp = nullptr;
  uint32_t *h_flags = nullptr;
  std::vector<Query> wave;        // queries of the wave in flight
  int32_t Q = 0;
  int status = WMC_OK;
  bool busy = false;
  int64_t launched_ns = 0;
  // a full wave staged in h_w2 while this slot's wave runs (throughput-
  // bound serving: launched as soon as the slot frees)
  double *h_w2 = nullptr;
  std::vector<Query> next;
  bool staged = false;
};

struct TicketState {
  int status = WMC_PENDING;
  wmc_result res{};
  int64_t done_ns = 0;
};

int64_t mono_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct wmc_server {
  Plan *plan = nullptr;
  wmc_server_opts opts{};
  int32_t n_vars = 0;
  int64_t ws_bytes = 0;              // each slot's workspace
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work;   // batcher: queue or slot changes
  std::condition_variable cv_done;   // waiters: tickets completed
  std::condition_variable cv_comp;   // completion thread
  std::deque<Query> queue;
  std::deque<int> finished;          // slot ids whose wave finished
  std::unordered_map<uint64_t, TicketState> tickets;
  uint64_t next_ticket = 1;
  bool stop = false;
  int in_flight = 0;
  wmc_server_stats_t stats{};
  double sum_q = 0;
  std::thread batcher, completer;
};

static void CUDART_CB on_wave_done(void *arg);

namespace {
struct CbArg {
  wmc_server *srv;
  int slot;
};
}  // namespace

// Weights of `wave` into pinned staging `h` ([2][Q][n_vars]); lanes past the
// wave's queries (Q is the next power of two) repeat its last query.
static int32_t stage_weights(const std::vector<Query> &wave, size_t nv, double *h) {
  const int32_t n = (int32_t)wave.size();
  int32_t Q = 1;
  while (Q < n) Q <<= 1;
  for (int32_t q = 0; q < Q && nv; ++q) {
    const Query &src = wave[(size_t)std::min(q, n - 1)];
    std::memcpy(h + (size_t)q * nv, src.wp.data(), sizeof(double) * nv);
    std::memcpy(h + (size_t)Q * nv + (size_t)q * nv, src.wn.data(), sizeof(double) * nv);
  }
  return Q;
}

// Enqueues the slot's wave (its weights already staged in h_w for sl.Q lanes).
static int submit_wave(wmc_server *srv, int si);

static int launch_wave(wmc_server *srv, int si) {
  Slot &sl = srv->slots[(size_t)si];
  sl.Q = stage_weights(sl.wave, (size_t)srv->n_vars, sl.h_w);
  return submit_wave(srv, si);
}

static int submit_wave(wmc_server *srv, int si) {
  Slot &sl = srv->slots[(size_t)si];
  const size_t nv = (size_t)srv->n_vars;
  const int32_t Q = sl.Q;
  ExecState *st = nullptr;
  int rc = exec_state(*srv->plan, Q, &st);
  if (rc) return rc;
  if (exec_ws_bytes(st) > srv->ws_bytes) {
    set_error("wave of %d needs %lld workspace bytes, slots hold %lld", Q, (long long)exec_ws_bytes(st),
              (long long)srv->ws_bytes);
    return WMC_EPLAN_TOO_BIG;
  }
  if (nv && cudaMemcpyAsync(sl.d_w, sl.h_w, sizeof(double) * 2 * (size_t)Q * nv,
                            cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
    return WMC_ECUDA;
  rc = exec_run_device(*srv->plan, st, sl.d_w, sl.d_w + (size_t)Q * nv, sl.ws, sl.d_mant, sl.d_exp,
                       sl.d_flags, sl.stream);
  if (rc) return rc;
  if (cudaMemcpyAsync(sl.h_mant, sl.d_mant, sizeof(double) * (size_t)Q, cudaMemcpyDeviceToHost, sl.stream) ||
      cudaMemcpyAsync(sl.h_exp, sl.d_exp, sizeof(int64_t) * (size_t)Q, cudaMemcpyDeviceToHost, sl.stream) ||
      cudaMemcpyAsync(sl.h_flags, sl.d_flags, sizeof(uint32_t) * (size_t)Q, cudaMemcpyDeviceToHost, sl.stream))
    return WMC_ECUDA;
  CbArg *arg = new CbArg{srv, si};
  if (cudaLaunchHostFunc(sl.stream, on_wave_done, arg) != cudaSuccess) {
    delete arg;
    return WMC_ECUDA;
  }
  return WMC_OK;
}

static void CUDART_CB on_wave_done(void *p) {
  CbArg *arg = (CbArg *)p;
  wmc_server *srv = arg->srv;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->finished.push_back(arg->slot);
  }
  srv->cv_comp.notify_one();
  delete arg;
}

// How many of the n queued queries the next wave takes.  A wave runs on a
// power-of-two batch, so n queries fill Q = the next power of two >= n
// lanes and the rest repeat the last query.  When that would leave more
// than a quarter of the lanes as padding, the wave takes the largest power
// of two <= n instead and the others wait for the next slot: under load
// the queue is long and every lane does real work; when the queue is short
// (n below 8) the wave takes everything, which keeps the latency of light
// traffic at one walk.
static size_t wave_take(size_t n, size_t max_b) {
  if (n >= max_b) return max_b;
  if (n < 8) return n;
  size_t up = 1, down = 1;
  while (up < n) up <<= 1;
  while (down * 2 <= n) down <<= 1;
  return (up - n) * 4 > up ? down : n;
}

static void batcher_loop(wmc_server *srv) {
  std::unique_lock<std::mutex> lk(srv->mu);
  const size_t max_b = (size_t)srv->opts.max_batch;
  // a partial wave starts only on an idle device (or with partial_overlap):
  // while a wave runs, the queue grows into the next one; a full wave
  // starts in any free slot
  auto may_start = [&] {
    return srv->in_flight == 0 || srv->opts.partial_overlap == 1 || srv->queue.size() >= max_b;
  };
  auto free_slot = [&](bool staged) {
    for (size_t i = 0; i < srv->slots.size(); ++i)
      if (!srv->slots[i].busy && srv->slots[i].staged == staged) return (int)i;
    return -1;
  };
  // the busy slot launched first without a staged wave (expected to free first)
  auto stage_slot = [&] {
    int sk = -1;
    for (size_t i = 0; i < srv->slots.size(); ++i)
      if (srv->slots[i].busy && !srv->slots[i].staged &&
          (sk < 0 || srv->slots[i].launched_ns < srv->slots[(size_t)sk].launched_ns))
        sk = (int)i;
    return sk;
  };
  auto can_launch = [&] { return !srv->queue.empty() && free_slot(false) >= 0 && may_start(); };
  // a full wave queued that cannot start now: staged for a busy slot
  auto can_stage = [&] { return srv->queue.size() >= max_b && !can_launch() && stage_slot() >= 0; };
  for (;;) {
    // every wake-up that returns makes progress (a launch or a staging),
    // so the loop never spins while holding the lock
    srv->cv_work.wait(lk, [&] { return srv->stop || free_slot(true) >= 0 || can_launch() || can_stage(); });
    if (srv->stop) return;
    // a free slot with a staged wave: launch it at once
    const int sj = free_slot(true);
    if (sj >= 0) {
      Slot &sl = srv->slots[(size_t)sj];
      sl.wave = std::move(sl.next);
      sl.next.clear();
      std::swap(sl.h_w, sl.h_w2);
      sl.Q = (int32_t)max_b;
      sl.staged = false;
      sl.busy = true;
      sl.status = WMC_OK;
      sl.launched_ns = mono_ns();
      srv->in_flight++;
      srv->stats.max_in_flight = std::max<int64_t>(srv->stats.max_in_flight, srv->in_flight);
      lk.unlock();
      int rc = submit_wave(srv, sj);
      lk.lock();
      if (rc) {
        sl.status = rc;
        srv->finished.push_back(sj);
        srv->cv_comp.notify_one();
      }
      continue;
    }
    if (!can_launch()) {
      // every slot that could take it is busy and a full wave is queued:
      // stage it for the slot expected to free first
      const int sk = stage_slot();
      if (sk < 0 || srv->queue.size() < max_b) continue;
      Slot &sl = srv->slots[(size_t)sk];
      sl.next.clear();
      for (size_t k = 0; k < max_b; ++k) {
        sl.next.push_back(std::move(srv->queue.front()));
        srv->queue.pop_front();
      }
      lk.unlock();
      stage_weights(sl.next, (size_t)srv->n_vars, sl.h_w2);
      lk.lock();
      sl.staged = true;
      continue;
    }
    // optional short wait for a fuller wave while other waves run
    if (srv->opts.max_wave_wait_us > 0 && srv->queue.size() < max_b && srv->in_flight > 0) {
      srv->cv_work.wait_for(lk, std::chrono::microseconds(srv->opts.max_wave_wait_us),
                            [&] { return srv->stop || srv->queue.size() >= max_b; });
      if (srv->stop) return;
      if (!can_launch()) continue;
    }
    const int si = free_slot(false);
    Slot &sl = srv->slots[(size_t)si];
    sl.wave.clear();
    const size_t take = wave_take(srv->queue.size(), max_b);
    while (sl.wave.size() < take) {
      sl.wave.push_back(std::move(srv->queue.front()));
      srv->queue.pop_front();
    }
    sl.busy = true;
    sl.status = WMC_OK;
    sl.launched_ns = mono_ns();
    srv->in_flight++;
    srv->stats.max_in_flight = std::max<int64_t>(srv->stats.max_in_flight, srv->in_flight);
    lk.unlock();
    int rc = launch_wave(srv, si);
    lk.lock();
    if (rc) {
      // fail only this wave's tickets
      sl.status = rc;
      srv->finished.push_back(si);
      srv->cv_comp.notify_one();
    }
  }
}

static void completer_loop(wmc_server *srv) {
  std::unique_lock<std::mutex> lk(srv->mu);
  for (;;) {
    srv->cv_comp.wait(lk, [&] { return !srv->finished.empty() || (srv->stop && srv->in_flight == 0); });
    if (srv->finished.empty()) return;
    const int si = srv->finished.front();
    srv->finished.pop_front();
    Slot &sl = srv->slots[(size_t)si];
    ExecState *st = nullptr;
    int rc = sl.status;
    if (rc == WMC_OK) {
      cudaError_t e = cudaStreamQuery(sl.stream);
      if (e != cudaSuccess && e != cudaErrorNotReady) rc = WMC_ECUDA;
    }
    if (rc == WMC_OK) rc = exec_state(*srv->plan, sl.Q, &st);
    const int64_t now = mono_ns();
    for (size_t q = 0; q < sl.wave.size(); ++q) {
      auto it = srv->tickets.find(sl.wave[q].ticket);
      if (it == srv->tickets.end()) continue;
      it->second.done_ns = now;
      if (rc == WMC_OK && (sl.h_flags[q] & WMC_FLAG_DEVICE_TIMEOUT)) {
        it->second.status = WMC_ETIMEOUT;
      } else if (rc == WMC_OK) {
        exec_fill_result(st, sl.h_mant[q], sl.h_exp[q], sl.h_flags[q], false, sl.wave[q].negative,
                         &it->second.res);
        it->second.status = WMC_OK;
      } else {
        it->second.status = rc;
      }
    }
    srv->stats.completed += (int64_t)sl.wave.size();
    srv->stats.waves += 1;
    if (rc) srv->stats.failed_waves += 1;
    srv->sum_q += (double)sl.wave.size();
    sl.wave.clear();
    sl.busy = false;
    srv->in_flight--;
    srv->cv_done.notify_all();
    srv->cv_work.notify_one();
  }
}

static void free_slot(Slot &s) {
  if (s.stream) cudaStreamSynchronize(s.stream);
  cudaFree(s.ws); cudaFree(s.d_w); cudaFree(s.d_mant); cudaFree(s.d_exp); cudaFree(s.d_flags);
  cudaFreeHost(s.h_w); cudaFreeHost(s.h_w2); cudaFreeHost(s.h_mant); cudaFreeHost(s.h_exp); cudaFreeHost(s.h_flags);
  if (s.stream) cudaStreamDestroy(s.stream);
  s = Slot();
}

extern "C" int wmc_server_create(wmc_plan_t *cplan, const wmc_server_opts *opts, wmc_server_t **out) {
  if (!cplan || !out) { set_error("NULL argument"); return WMC_EINVAL; }
  *out = nullptr;
  Plan &plan = plan_of(cplan);
  wmc_server_opts o{};
  o.precision = plan.precision;
  o.max_batch = 256;
  o.max_waves = 2;
  if (opts) o = *opts;
  if (o.precision != plan.precision) { set_error("server precision differs from the plan's"); return WMC_EINVAL; }
  if (o.max_batch < 1 || o.max_batch > 1024 || (o.max_batch & (o.max_batch - 1))) {
    set_error("max_batch must be a power of two in [1, 1024]");
    return WMC_EINVAL;
  }
  if (o.max_waves < 1 || o.max_waves > 64) { set_error("max_waves must be in [1, 64]"); return WMC_EINVAL; }
  ExecState *st = nullptr;
  int rc = exec_state(plan, o.max_batch, &st);
  if (rc) return rc;
  const int64_t ws = exec_ws_bytes(st);
  int32_t n_slots = o.max_waves;
  if (o.arena_bytes > 0) n_slots = (int32_t)std::min<int64_t>(n_slots, o.arena_bytes / std::max<int64_t>(ws, 1));
  if (n_slots < 1) {
    set_error("arena_bytes %lld cannot hold one wave (%lld bytes)", (long long)o.arena_bytes, (long long)ws);
    return WMC_EPLAN_TOO_BIG;
  }
  wmc_server *srv = new (std::nothrow) wmc_server();
  if (!srv) { set_error("out of host memory"); return WMC_ENOMEM; }
  srv->plan = &plan;
  srv->opts = o;
  srv->ws_bytes = ws;
  srv->n_vars = plan.n_vars;
  srv->slots.resize((size_t)n_slots);
  const size_t nv = std::max<size_t>((size_t)plan.n_vars, 1);
  const size_t B = (size_t)o.max_batch;
  for (auto &s : srv->slots) {
    bool ok = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc(&s.ws, (size_t)ws) == cudaSuccess &&
              cudaMalloc((void **)&s.d_w, sizeof(double) * 2 * B * nv) == cudaSuccess &&
              cudaMalloc((void **)&s.d_mant, sizeof(double) * B) == cudaSuccess &&
              cudaMalloc((void **)&s.d_exp, sizeof(int64_t) * B) == cudaSuccess &&
              cudaMalloc((void **)&s.d_flags, sizeof(uint32_t) * B) == cudaSuccess &&
              cudaMallocHost((void **)&s.h_w, sizeof(double) * 2 * B * nv) == cudaSuccess &&
              cudaMallocHost((void **)&s.h_w2, sizeof(double) * 2 * B * nv) == cudaSuccess &&
              cudaMallocHost((void **)&s.h_mant, sizeof(double) * B) == cudaSuccess &&
              cudaMallocHost((void **)&s.h_exp, sizeof(int64_t) * B) == cudaSuccess &&
              cudaMallocHost((void **)&s.h_flags, sizeof(uint32_t) * B) == cudaSuccess;
    if (!ok) {
      (void)cudaGetLastError();
      for (auto &t : srv->slots) free_slot(t);
      delete srv;
      set_error("server allocation failed");
      return WMC_ENOMEM;
    }
  }
  // capture every slot's graph for every wave size (powers of two up to
  // max_batch) now, so that no wave waits for a capture later; sizes whose
  // workspace exceeds the slots' are left to fail at their first wave
  for (int32_t Q = 1; Q <= o.max_batch; Q <<= 1) {
    ExecState *st = nullptr;
    if (exec_state(plan, Q, &st)) break;
    if (exec_ws_bytes(st) > ws) continue;
    for (auto &s : srv->slots)
      if (exec_prepare(plan, st, s.ws)) break;
    if (Q == o.max_batch) break;
  }
  (void)cudaGetLastError();
  srv->batcher = std::thread(batcher_loop, srv);
  srv->completer = std::thread(completer_loop, srv);
  *out = srv;
  return WMC_OK;
}

extern "C" int wmc_submit(wmc_server_t *srv, const double *w_pos, const double *w_neg, uint64_t *ticket) {
  if (!srv || !ticket || (srv->n_vars > 0 && (!w_pos || !w_neg))) { set_error("NULL argument"); return WMC_EINVAL; }
  Query q;
  q.wp.assign(w_pos, w_pos + srv->n_vars);
  q.wn.assign(w_neg, w_neg + srv->n_vars);
  q.negative = false;
  for (int32_t i = 0; i < srv->n_vars; ++i) q.negative |= (q.wp[(size_t)i] < 0) | (q.wn[(size_t)i] < 0);
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) { set_error("server is shutting down"); return WMC_ESHUTDOWN; }
    q.ticket = srv->next_ticket++;
    *ticket = q.ticket;
    srv->tickets[q.ticket] = TicketState();
    srv->queue.push_back(std::move(q));
    srv->stats.submitted++;
  }
  srv->cv_work.notify_one();
  return WMC_OK;
}

extern "C" int wmc_submit_many(wmc_server_t *srv, int64_t n, const double *w_pos, const double *w_neg,
                               uint64_t *tickets) {
  if (!srv || n < 0 || (n > 0 && !tickets) || (n > 0 && srv->n_vars > 0 && (!w_pos || !w_neg))) {
    set_error("NULL argument or n < 0");
    return WMC_EINVAL;
  }
  const size_t nv = (size_t)srv->n_vars;
  std::vector<Query> qs((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    Query &q = qs[(size_t)i];
    q.wp.assign(w_pos + (size_t)i * nv, w_pos + (size_t)(i + 1) * nv);
    q.wn.assign(w_neg + (size_t)i * nv, w_neg + (size_t)(i + 1) * nv);
    q.negative = false;
    for (size_t v = 0; v < nv; ++v) q.negative |= (q.wp[v] < 0) | (q.wn[v] < 0);
  }
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) { set_error("server is shutting down"); return WMC_ESHUTDOWN; }
    for (int64_t i = 0; i < n; ++i) {
      Query &q = qs[(size_t)i];
      q.ticket = srv->next_ticket++;
      tickets[i] = q.ticket;
      srv->tickets[q.ticket] = TicketState();
      srv->queue.push_back(std::move(q));
      srv->stats.submitted++;
    }
  }
  srv->cv_work.notify_one();
  return WMC_OK;
}

static int take_result(wmc_server *srv, uint64_t ticket, wmc_result *out, int64_t *done_ns = nullptr) {
  auto it = srv->tickets.find(ticket);
  if (it == srv->tickets.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return WMC_EUNKNOWN_TICKET; }
  if (it->second.status == WMC_PENDING) return WMC_PENDING;
  int st = it->second.status;
  if (st == WMC_OK && out) *out = it->second.res;
  if (done_ns) *done_ns = it->second.done_ns;
  if (st != WMC_OK) set_error("the wave of ticket %llu failed", (unsigned long long)ticket);
  srv->tickets.erase(it);
  return st;
}

extern "C" int wmc_poll(wmc_server_t *srv, uint64_t ticket, wmc_result *out) {
  if (!srv) { set_error("NULL argument"); return WMC_EINVAL; }
  std::lock_guard<std::mutex> lk(srv->mu);
  return take_result(srv, ticket, out);
}

extern "C" int wmc_poll_ex(wmc_server_t *srv, uint64_t ticket, wmc_result *out, int64_t *done_ns) {
  if (!srv) { set_error("NULL argument"); return WMC_EINVAL; }
  std::lock_guard<std::mutex> lk(srv->mu);
  return take_result(srv, ticket, out, done_ns);
}

extern "C" int wmc_wait(wmc_server_t *srv, uint64_t ticket, int64_t timeout_us, wmc_result *out) {
  if (!srv) { set_error("NULL argument"); return WMC_EINVAL; }
  std::unique_lock<std::mutex> lk(srv->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
  for (;;) {
    int rc = take_result(srv, ticket, out);
    if (rc != WMC_PENDING) return rc;
    if (srv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      rc = take_result(srv, ticket, out);
      if (rc == WMC_PENDING) { set_error("timed out waiting for ticket"); return WMC_ETIMEOUT; }
      return rc;
    }
  }
}

extern "C" int wmc_server_stats(wmc_server_t *srv, wmc_server_stats_t *out) {
  if (!srv || !out) { set_error("NULL argument"); return WMC_EINVAL; }
  std::lock_guard<std::mutex> lk(srv->mu);
  *out = srv->stats;
  out->mean_wave_q = srv->stats.waves ? srv->sum_q / (double)srv->stats.waves : 0.0;
  return WMC_OK;
}

extern "C" void wmc_server_destroy(wmc_server_t *srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  if (srv->batcher.joinable()) srv->batcher.join();
  for (auto &s : srv->slots) if (s.stream) cudaStreamSynchronize(s.stream);
  srv->cv_comp.notify_all();
  if (srv->completer.joinable()) srv->completer.join();
  for (auto &s : srv->slots) free_slot(s);
  delete srv;
}
