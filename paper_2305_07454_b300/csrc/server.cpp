// server.cpp — the serving runtime declared in include/cvetl.h: feeds of stream-mode contexts,
// one FIFO request queue, worker slots that run the windows of different feeds at the same
// time on the feeds' own CUDA streams, and admission against a device-memory budget.
//
// Everything here is host code over the public C ABI; the GPU work of a request is the
// stream-mode extract / transform / load (or flush) of its feed's context.
#include <cuda_runtime.h>

#include <time.h>

#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "cvetl.h"

namespace {

int64_t now_ns() {
  timespec t;
  clock_gettime(CLOCK_MONOTONIC, &t);
  return (int64_t)t.tv_sec * 1000000000LL + t.tv_nsec;
}

struct Request {
  uint64_t ticket = 0;
  int32_t feed = 0;
  int32_t kind = 0;  // 0 window, 1 flush
  cvetl_input in{};
  size_t reserve = 0;
  int64_t submit_ns = 0;
};

struct Feed {
  cvetl_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  bool busy = false;
  bool closed = false;   // a flush was submitted
  int64_t queued = 0;    // requests queued or running
  size_t held = 0;       // device bytes of the context after its last request
};

std::string g_server_error;

}  // namespace

struct cvetl_server {
  cvetl_server_config cfg{};
  std::mutex mu;
  std::condition_variable work_cv, done_cv;
  std::deque<Request> queue;
  std::deque<Feed> feeds;  // a deque: a worker's Feed& stays valid while feeds are added
  std::unordered_map<uint64_t, cvetl_ticket_info> done;
  std::unordered_set<uint64_t> live;  // issued and not yet released
  std::vector<std::thread> workers;
  uint64_t next_ticket = 1;
  size_t held = 0;      // sum of the feeds' held bytes
  size_t reserved = 0;  // reservations of the running requests
  int in_flight = 0, peak_in_flight = 0;
  bool stop = false;
  std::string err;
};

namespace {

cvetl_status sfail(cvetl_server* s, cvetl_status st, const char* msg) {
  if (s) s->err = msg;
  else g_server_error = msg;
  return st;
}

// Index of the request to start next, or -1. Called with the lock held.
long pick(cvetl_server* s) {
  std::vector<char> seen(s->feeds.size(), 0);
  for (size_t i = 0; i < s->queue.size(); ++i) {
    const Request& r = s->queue[i];
    Feed& f = s->feeds[r.feed];
    if (f.busy || seen[r.feed]) {  // the feed's earlier request goes first
      seen[r.feed] = 1;
      continue;
    }
    const size_t budget = s->cfg.mem_budget_bytes;
    if (budget == 0 || s->in_flight == 0 || s->held + s->reserved + r.reserve <= budget) return (long)i;
    return -1;  // first come, first served on memory
  }
  return -1;
}

cvetl_status run(Feed& f, const Request& r, std::string& msg) {
  cvetl_status st;
  if (r.kind == 0) {
    st = cvetl_extract(f.ctx, &r.in);
    if (st == CVETL_OK) st = cvetl_transform(f.ctx);
    if (st == CVETL_OK) st = cvetl_load(f.ctx);
  } else {
    st = cvetl_flush(f.ctx);
  }
  if (st == CVETL_OK) {
    cudaError_t e = cudaStreamSynchronize(f.st);
    if (e != cudaSuccess) {
      msg = std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e);
      return CVETL_ECUDA;
    }
  } else {
    msg = cvetl_last_error(f.ctx);
  }
  return st;
}

void worker(cvetl_server* s, int slot) {
  cudaSetDevice(s->cfg.device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    long i = -1;
    s->work_cv.wait(lk, [&] { return (i = pick(s)) >= 0 || (s->stop && s->in_flight == 0); });
    if (i < 0) return;
    Request r = s->queue[(size_t)i];
    s->queue.erase(s->queue.begin() + i);
    Feed& f = s->feeds[r.feed];
    f.busy = true;
    s->reserved += r.reserve;
    s->in_flight += 1;
    if (s->in_flight > s->peak_in_flight) s->peak_in_flight = s->in_flight;
    const int64_t start = now_ns();
    lk.unlock();

    std::string msg;
    cvetl_status st = run(f, r, msg);
    cvetl_stats stats;
    size_t held = f.held;
    if (cvetl_stats_get(f.ctx, &stats) == CVETL_OK) held = (size_t)stats.device_bytes;
    const int64_t end = now_ns();

    lk.lock();
    f.busy = false;
    f.queued -= 1;
    s->reserved -= r.reserve;
    s->in_flight -= 1;
    s->held = s->held - f.held + held;
    f.held = held;
    cvetl_ticket_info info;
    memset(&info, 0, sizeof info);
    info.status = st;
    info.feed = r.feed;
    info.kind = r.kind;
    info.slot = slot;
    info.n = r.kind == 0 ? r.in.n : 0;
    info.submit_ns = r.submit_ns;
    info.start_ns = start;
    info.done_ns = end;
    info.peak_in_flight = s->peak_in_flight;
    snprintf(info.message, sizeof info.message, "%s", msg.c_str());
    s->done[r.ticket] = info;
    s->done_cv.notify_all();
    s->work_cv.notify_all();
  }
}

cvetl_status enqueue(cvetl_server* s, Request&& r, uint64_t* ticket) {
  r.ticket = s->next_ticket++;
  r.submit_ns = now_ns();
  s->feeds[r.feed].queued += 1;
  s->live.insert(r.ticket);
  *ticket = r.ticket;
  s->queue.push_back(r);
  s->work_cv.notify_all();
  return CVETL_OK;
}

}  // namespace

extern "C" {

cvetl_status cvetl_server_create(const cvetl_server_config* cfg, cvetl_server** out) {
  if (!cfg || !out) return sfail(nullptr, CVETL_EINVAL, "cvetl_server_create: NULL argument");
  if (cfg->n_slots < 1 || cfg->n_slots > CVETL_SERVE_MAX_SLOTS)
    return sfail(nullptr, CVETL_EINVAL, "cvetl_server_create: n_slots must be in [1, 64]");
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    cudaGetLastError();
    return sfail(nullptr, CVETL_ECUDA, "cvetl_server_create: the device cannot be used");
  }
  cvetl_server* s = new cvetl_server();
  s->cfg = *cfg;
  for (int i = 0; i < cfg->n_slots; ++i) s->workers.emplace_back(worker, s, i);
  *out = s;
  return CVETL_OK;
}

cvetl_status cvetl_server_add_feed(cvetl_server* s, const cvetl_config* cfg, int32_t* feed) {
  if (!s) return CVETL_EINVAL;
  if (!cfg || !feed) return sfail(s, CVETL_EINVAL, "cvetl_server_add_feed: NULL argument");
  cudaSetDevice(s->cfg.device);
  Feed f;
  if (cudaStreamCreateWithFlags(&f.st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return sfail(s, CVETL_ECUDA, "cvetl_server_add_feed: cudaStreamCreateWithFlags failed");
  }
  cvetl_config c = *cfg;
  c.mode = CVETL_STREAM;
  c.stream = f.st;
  c.device = s->cfg.device;
  c.mem_budget_bytes = 0;  // the server admits by its own budget
  cvetl_status st = cvetl_create(&c, &f.ctx);
  if (st != CVETL_OK) {
    cudaStreamDestroy(f.st);
    return sfail(s, st, cvetl_last_error(nullptr));
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->feeds.push_back(f);
  *feed = (int32_t)(s->feeds.size() - 1);
  return CVETL_OK;
}

cvetl_status cvetl_server_submit(cvetl_server* s, int32_t feed, const cvetl_input* in, uint64_t* ticket) {
  if (!s) return CVETL_EINVAL;
  if (!in || !ticket) return sfail(s, CVETL_EINVAL, "cvetl_server_submit: NULL argument");
  if (in->kind != CVETL_IN_COLUMNS || in->n < 0 || in->n > CVETL_MAX_RECORDS)
    return sfail(s, CVETL_EINVAL, "cvetl_server_submit: a window is binary columns of [0, 2^30) rows");
  std::lock_guard<std::mutex> lk(s->mu);
  if (feed < 0 || (size_t)feed >= s->feeds.size()) return sfail(s, CVETL_EINVAL, "cvetl_server_submit: no such feed");
  if (s->feeds[feed].closed) return sfail(s, CVETL_ESTATE, "cvetl_server_submit: the feed was flushed");
  Request r;
  r.feed = feed;
  r.kind = 0;
  r.in = *in;
  r.reserve = (size_t)in->n * CVETL_SERVE_BYTES_PER_ROW;
  if (s->cfg.mem_budget_bytes && r.reserve > s->cfg.mem_budget_bytes)
    return sfail(s, CVETL_EFULL, "cvetl_server_submit: the window alone exceeds the memory budget");
  return enqueue(s, std::move(r), ticket);
}

cvetl_status cvetl_server_submit_flush(cvetl_server* s, int32_t feed, uint64_t* ticket) {
  if (!s) return CVETL_EINVAL;
  if (!ticket) return sfail(s, CVETL_EINVAL, "cvetl_server_submit_flush: NULL ticket");
  std::lock_guard<std::mutex> lk(s->mu);
  if (feed < 0 || (size_t)feed >= s->feeds.size()) return sfail(s, CVETL_EINVAL, "cvetl_server_submit_flush: no such feed");
  if (s->feeds[feed].closed) return sfail(s, CVETL_ESTATE, "cvetl_server_submit_flush: the feed was flushed");
  s->feeds[feed].closed = true;
  Request r;
  r.feed = feed;
  r.kind = 1;
  return enqueue(s, std::move(r), ticket);
}

cvetl_status cvetl_server_wait(cvetl_server* s, uint64_t ticket, cvetl_ticket_info* info) {
  if (!s) return CVETL_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  if (!s->live.count(ticket)) return sfail(s, CVETL_EINVAL, "cvetl_server_wait: unknown or released ticket");
  s->done_cv.wait(lk, [&] { return s->done.count(ticket) > 0; });
  auto it = s->done.find(ticket);
  cvetl_ticket_info r = it->second;
  s->done.erase(it);
  s->live.erase(ticket);
  if (info) *info = r;
  return (cvetl_status)r.status;
}

cvetl_status cvetl_server_drain(cvetl_server* s) {
  if (!s) return CVETL_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  s->done_cv.wait(lk, [&] { return s->queue.empty() && s->in_flight == 0; });
  return CVETL_OK;
}

cvetl_status cvetl_server_feed(cvetl_server* s, int32_t feed, cvetl_ctx** ctx) {
  if (!s) return CVETL_EINVAL;
  if (!ctx) return sfail(s, CVETL_EINVAL, "cvetl_server_feed: NULL output");
  std::lock_guard<std::mutex> lk(s->mu);
  if (feed < 0 || (size_t)feed >= s->feeds.size()) return sfail(s, CVETL_EINVAL, "cvetl_server_feed: no such feed");
  if (s->feeds[feed].queued) return sfail(s, CVETL_ESTATE, "cvetl_server_feed: the feed has requests queued or running");
  *ctx = s->feeds[feed].ctx;
  return CVETL_OK;
}

cvetl_status cvetl_server_destroy(cvetl_server* s) {
  if (!s) return CVETL_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (const Request& r : s->queue) s->feeds[r.feed].queued -= 1;
    s->queue.clear();
    s->stop = true;
    s->work_cv.notify_all();
  }
  for (auto& t : s->workers) t.join();
  cudaSetDevice(s->cfg.device);
  for (Feed& f : s->feeds) {
    cvetl_destroy(f.ctx);
    cudaStreamDestroy(f.st);
  }
  delete s;
  return CVETL_OK;
}

const char* cvetl_server_last_error(const cvetl_server* s) {
  return s ? s->err.c_str() : g_server_error.c_str();
}

}  // extern "C"
