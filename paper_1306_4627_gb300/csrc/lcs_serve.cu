// Serving: continuous batching of LCS requests that arrive over time (lcs_serve_* in include/lcs.h).
//
// Requests are copied at submit and queued. Worker threads, each with its own context (device buffers and
// stream), take work as soon as they are free, so requests that arrive while others run join the next launch:
//   * one batch worker takes every waiting short length-only request (up to max_batch) and runs them as one
//     persistent batched launch (lcs_batch);
//   * several single-pair workers (lcs_serve_cfg.pair_workers) take long pairs and all traceback requests, one at a
//     time each (lcs_length / lcs_traceback), so their work overlaps on the GPU with the batches and with each
//     other (a single pair's fill occupies only n / 4096 SMs).
// A traceback needs a direction bitmap of about m*n/8 bytes: the server admits it only while the bitmaps of the
// tracebacks in flight fit the HBM budget (it waits otherwise), and refuses one that could never fit at submit.
// Every result is computed by the same exact kernels as a call on its own, so it does not depend on the mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lcs_ctx.h"

namespace {

constexpr uint32_t kPairWorkersDefault = 8;
constexpr uint32_t kPairWorkersMax = 32;

double now_s() {
  using clk = std::chrono::steady_clock;
  return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

struct Req {
  uint64_t ticket = 0;
  std::vector<uint8_t> x, y;
  uint32_t flags = 0;
  uint64_t bitmap = 0;   // device bytes reserved while it runs (tracebacks)
  double t_submit = 0, t_done = 0;
  int status = LCS_PENDING;
  uint64_t length = 0;
  std::vector<uint8_t> lcs;
  bool short_pair = false;
};

// Device bytes a traceback of an m x n pair holds: the direction bitmap plus its per-row scratch and the segment
// walkers' buffers (at most 65536 walkers of 256-row segments), rounded up.
uint64_t traceback_bytes(uint64_t m, uint64_t n) {
  const uint64_t words = n / 32 + 1;
  const uint64_t lanes = (words + 127) / 128 * 128;
  return lanes * ((m + 7) / 8 + 31) * 8 * 4 + (uint64_t)257 * lanes * 8 + 64 * m + (40u << 20);
}

}  // namespace

struct lcs_server {
  int device = 0;
  lcs_serve_cfg cfg{};
  uint64_t budget = 0;
  uint64_t long_cells = 0;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> q_short, q_pair;
  std::unordered_map<uint64_t, Req*> reqs;  // every request until its result is released
  uint64_t next_ticket = 1;
  size_t live = 0;                          // waiting or running
  uint64_t reserved = 0;                    // bitmap bytes of tracebacks in flight
  bool stop = false;

  std::vector<std::thread> threads;
  std::vector<lcs_ctx*> ctxs;

  void finish(Req* r) {
    std::lock_guard<std::mutex> g(mu);
    r->t_done = now_s();
    --live;
    if (r->bitmap) reserved -= r->bitmap;
    cv_done.notify_all();
    cv_work.notify_all();
  }

  void batch_worker(lcs_ctx* c) {
    std::vector<Req*> take;
    std::vector<uint8_t> xs, ys;
    std::vector<uint64_t> xo, yo, out;
    try {
      take.reserve(cfg.max_batch);  // filled under the lock below without allocating
    } catch (...) {
    }
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || !q_short.empty(); });
        if (q_short.empty() && stop) return;
        take.clear();
        const size_t cap = std::min<size_t>(cfg.max_batch, std::max<size_t>(take.capacity(), 1));
        while (!q_short.empty() && take.size() < cap) {
          take.push_back(q_short.front());
          q_short.pop_front();
        }
      }
      int rc = LCS_OK;
      try {
        xs.clear();
        ys.clear();
        xo.assign(1, 0);
        yo.assign(1, 0);
        for (Req* r : take) {
          xs.insert(xs.end(), r->x.begin(), r->x.end());
          ys.insert(ys.end(), r->y.begin(), r->y.end());
          xo.push_back(xs.size());
          yo.push_back(ys.size());
        }
        out.assign(take.size(), 0);
      } catch (...) {
        rc = LCS_ERR_NOMEM;
      }
      if (!rc)
        rc = lcs_batch(c, xs.empty() ? nullptr : xs.data(), xo.data(), ys.empty() ? nullptr : ys.data(), yo.data(),
                       take.size(), out.data());
      for (size_t k = 0; k < take.size(); ++k) {
        take[k]->status = rc;
        take[k]->length = rc == LCS_OK ? out[k] : 0;
        finish(take[k]);
      }
    }
  }

  void pair_worker(lcs_ctx* c) {
    for (;;) {
      Req* r = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] {
          if (stop && q_pair.empty()) return true;
          for (Req* q : q_pair)
            if (!q->bitmap || reserved + q->bitmap <= budget) return true;
          return false;
        });
        if (q_pair.empty() && stop) return;
        for (auto it = q_pair.begin(); it != q_pair.end(); ++it) {
          if (!(*it)->bitmap || reserved + (*it)->bitmap <= budget) {
            r = *it;
            q_pair.erase(it);
            break;
          }
        }
        if (!r) continue;
        reserved += r->bitmap;
      }
      const uint8_t* x = r->x.empty() ? nullptr : r->x.data();
      const uint8_t* y = r->y.empty() ? nullptr : r->y.data();
      if (r->flags & LCS_TRACEBACK) {
        uint64_t len = 0;
        try {
          r->lcs.resize(std::max<size_t>(1, std::min(r->x.size(), r->y.size())));
          r->status = lcs_traceback(c, x, r->x.size(), y, r->y.size(), r->lcs.data(), r->lcs.size(), &len);
        } catch (...) {
          r->status = LCS_ERR_NOMEM;
        }
        r->length = len;
        r->lcs.resize(r->status == LCS_OK ? len : 0);  // shrinking: no allocation
        // give large bitmaps back, so that the budget is what the device actually holds
        if (c->T.cap > (256ull << 20)) {
          cudaSetDevice(c->device);
          cudaStreamSynchronize(c->stream);
          lcs::release(c->T);
        }
      } else {
        uint64_t len = 0;
        r->status = lcs_length(c, x, r->x.size(), y, r->y.size(), &len);
        r->length = len;
      }
      finish(r);
    }
  }
};

static int lcs_serve_create_impl(lcs_ctx* ctx, const lcs_serve_cfg* cfg, lcs_server** out) {
  if (!ctx || !out) return LCS_ERR_INVALID;
  *out = nullptr;
  lcs_server* s = new (std::nothrow) lcs_server();
  if (!s) return LCS_ERR_NOMEM;
  s->device = ctx->device;
  if (cfg) s->cfg = *cfg;
  if (s->cfg.max_queue == 0) s->cfg.max_queue = 65536;
  if (s->cfg.max_batch == 0) s->cfg.max_batch = 4096;
  if (s->cfg.long_pair_cells_log2 == 0) s->cfg.long_pair_cells_log2 = 24;
  if (s->cfg.pair_workers == 0) s->cfg.pair_workers = kPairWorkersDefault;
  s->cfg.pair_workers = std::min(s->cfg.pair_workers, kPairWorkersMax);
  s->long_cells = 1ull << std::min<uint32_t>(s->cfg.long_pair_cells_log2, 62);
  cudaSetDevice(s->device);
  s->budget = s->cfg.hbm_budget_bytes;
  if (s->budget == 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return LCS_ERR_CUDA;
    }
    s->budget = (uint64_t)(free_b * 0.6);
  }
  int rc = LCS_OK;
  try {
    s->ctxs.reserve(1 + s->cfg.pair_workers);
    s->threads.reserve(1 + s->cfg.pair_workers);
    for (uint32_t k = 0; k < 1 + s->cfg.pair_workers && !rc; ++k) {
      lcs_ctx* c = nullptr;
      rc = lcs_ctx_create(s->device, &c);
      if (!rc) s->ctxs.push_back(c);
    }
    if (!rc) {
      s->threads.emplace_back(&lcs_server::batch_worker, s, s->ctxs[0]);
      for (uint32_t k = 0; k < s->cfg.pair_workers; ++k)
        s->threads.emplace_back(&lcs_server::pair_worker, s, s->ctxs[1 + k]);
    }
  } catch (...) {  // a thread that could not start: stop the ones that did
    rc = LCS_ERR_INTERNAL;
  }
  if (rc) {
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->threads) t.join();
    for (lcs_ctx* d : s->ctxs) lcs_ctx_destroy(d);
    delete s;
    return rc;
  }
  *out = s;
  return LCS_OK;
}

extern "C" int lcs_serve_create(lcs_ctx* ctx, const lcs_serve_cfg* cfg, lcs_server** out) {
  try {  // no C++ exception crosses the C boundary
    return lcs_serve_create_impl(ctx, cfg, out);
  } catch (const std::bad_alloc&) {
    return LCS_ERR_NOMEM;
  } catch (...) {
    return LCS_ERR_INTERNAL;
  }
}

static int lcs_serve_submit_impl(lcs_server* s, const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n,
                                uint32_t flags, uint64_t* ticket) {
  if (!s || !ticket || (m && !x) || (n && !y) || (flags & ~LCS_TRACEBACK)) return LCS_ERR_INVALID;
  if (m >= (1ull << 32) || n >= (1ull << 32)) return LCS_ERR_INVALID;
  const bool tb = (flags & LCS_TRACEBACK) != 0;
  const uint64_t need = tb && m && n ? traceback_bytes(m, n) : 0;
  if (need > s->budget) return LCS_ERR_NOMEM;
  std::unique_ptr<Req> owned(new (std::nothrow) Req());
  if (!owned) return LCS_ERR_NOMEM;
  owned->x.assign(x, x + m);  // may throw bad_alloc: the request is freed by owned
  owned->y.assign(y, y + n);
  Req* r = owned.get();
  r->flags = flags;
  r->bitmap = need;
  r->short_pair = !tb && n <= 4096 && m * n < s->long_cells;
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop || s->live >= s->cfg.max_queue) return s->stop ? LCS_ERR_INVALID : LCS_ERR_BUSY;
    r->ticket = s->next_ticket++;
    auto& q = r->short_pair ? s->q_short : s->q_pair;
    s->reqs[r->ticket] = r;
    try {
      q.push_back(r);
    } catch (...) {
      s->reqs.erase(r->ticket);
      throw;
    }
    ++s->live;
    owned.release();  // the server owns the request now
  }
  s->cv_work.notify_all();
  *ticket = r->ticket;
  return LCS_OK;
}

extern "C" int lcs_serve_submit(lcs_server* s, const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n,
                                uint32_t flags, uint64_t* ticket) {
  try {  // no C++ exception crosses the C boundary
    return lcs_serve_submit_impl(s, x, m, y, n, flags, ticket);
  } catch (const std::bad_alloc&) {
    return LCS_ERR_NOMEM;
  } catch (...) {
    return LCS_ERR_INTERNAL;
  }
}

static void fill_result(const Req* r, lcs_result* out) {
  out->status = r->status;
  out->flags = r->flags;
  out->length = r->length;
  out->lcs = (r->flags & LCS_TRACEBACK) && !r->lcs.empty() ? r->lcs.data() : nullptr;
  out->lcs_len = (r->flags & LCS_TRACEBACK) ? r->lcs.size() : 0;
  out->submit_to_done_s = r->t_done - r->t_submit;
}

extern "C" int lcs_serve_poll(lcs_server* s, uint64_t ticket, lcs_result* out) {
  if (!s || !out) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return LCS_ERR_INVALID;
  if (it->second->t_done == 0) return LCS_PENDING;
  fill_result(it->second, out);
  return LCS_OK;
}

extern "C" int lcs_serve_wait(lcs_server* s, uint64_t ticket, double timeout_s, lcs_result* out) {
  if (!s || !out) return LCS_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return LCS_ERR_INVALID;
  Req* r = it->second;
  auto ready = [&] { return r->t_done != 0; };
  if (timeout_s < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    return LCS_PENDING;
  }
  fill_result(r, out);
  return LCS_OK;
}

extern "C" void lcs_result_release(lcs_server* s, uint64_t ticket) {
  if (!s) return;
  Req* r = nullptr;
  {
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || it->second->t_done == 0) return;  // unknown, or still running
    r = it->second;
    s->reqs.erase(it);
  }
  delete r;
}

extern "C" void lcs_serve_destroy(lcs_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->threads) t.join();
  for (lcs_ctx* c : s->ctxs) lcs_ctx_destroy(c);
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
}
