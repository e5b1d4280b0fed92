// Serving: continuous batching of LCS requests that arrive over time (lcs_serve_* in include/lcs.h).
//
// Requests are copied at submit and queued. Worker threads, each with its own context (device buffers and
// stream), take work as soon as they are free, so requests that arrive while others run join the next launch:
//   * two batch workers take every waiting short length-only request (up to max_batch) and run them as one
//     persistent batched launch (lcs_batch), one planning and launching a wave while the other's runs;
//   * several single-pair workers (lcs_serve_cfg.pair_workers) take long pairs and all traceback requests, one at a
//     time each (lcs_length / lcs_traceback), so their work overlaps on the GPU with the batches and with each
//     other (a single pair's fill occupies only n / 4096 SMs).
// A traceback needs a direction bitmap of about m*n/8 bytes: the server admits it only while the bitmaps of the
// tracebacks in flight fit the HBM budget (it waits otherwise), and refuses one that could never fit at submit.
// Every result is computed by the same exact kernels as a call on its own, so it does not depend on the mix.
//
// Nothing is allocated on the device while requests run: every worker's buffers are grown at creation for pairs
// of up to 65536 x 65536 (the batch worker's for its largest wave), and the direction bitmaps of tracebacks come
// from one arena allocated at creation (the HBM budget). Admission of a traceback is a first-fit reservation of its
// bitmap in the arena. (cudaMalloc and cudaFree synchronise the device: a worker that grew a buffer while another
// worker's fill ran stalled every stream, which showed as tail latency even at low load.)
//
// Scheduling is O(1) per event: three FIFO queues (short length-only pairs for the batch worker, long length-only
// pairs and tracebacks for the pair workers), one condition variable per kind of worker, one wake-up per submitted
// request, and a batch wave's results published under one lock. A pair worker takes the older of the two pair
// queues' heads; a traceback head that does not fit the budget yet lets length-only pairs pass it, and the budget
// it waits for is announced when a traceback finishes. (A scan of the whole queue on every wake-up, with every
// worker woken by every event, made the server slower the more workers it had.)
// A length-only pair whose shorter side fits a batch row (and whose longer side is at most 16384) is sent to the
// batch workers with its strings swapped when needed: the LCS length is symmetric in X and Y.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lcs_ctx.h"

namespace lcs {
uint64_t traceback_bitmap_bytes(const lcs_ctx* c, uint64_t m, uint64_t n);
int presize(lcs_ctx* c, uint64_t max_m, uint64_t max_n);
int batch_presize(lcs_ctx* c, uint64_t max_pairs, uint64_t x_bytes, uint64_t y_bytes);
}  // namespace lcs

namespace {

constexpr uint32_t kPairWorkersDefault = 16;
constexpr uint64_t kShortMaxRows = 16384;  // batched pairs have at most this many rows: a wave lasts as long as its
                                           // longest pair's chain of rows (half of them when the pair is split)
constexpr uint32_t kPairWorkersMax = 32;
constexpr uint32_t kBatchWorkers = 2;  // one plans and launches a wave while the other's wave runs

double now_s() {
  using clk = std::chrono::steady_clock;
  return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

constexpr uint64_t kPresizeLen = 65536;       // pair workers: buffers for m, n up to this
constexpr uint64_t kWaveXBytes = 8ull << 20;   // batch waves: at most this many symbols of X in all
constexpr uint64_t kWaveYBytes = 2ull << 20;   // and of Y
constexpr uint64_t kArenaAlign = 256;

struct Req {
  uint64_t ticket = 0;
  std::vector<uint8_t> x, y;
  uint32_t flags = 0;
  uint64_t bitmap = 0;      // arena bytes its direction bitmap needs (tracebacks)
  uint64_t arena_off = 0;   // where they were reserved while it runs
  double t_submit = 0, t_done = 0;
  int status = LCS_PENDING;
  uint64_t length = 0;
  std::vector<uint8_t> lcs;
  bool short_pair = false;
};

// First-fit reservations in the bitmap arena (offsets and sizes in bytes, multiples of kArenaAlign).
struct Arena {
  uint64_t size = 0;
  std::map<uint64_t, uint64_t> free;  // offset -> length of each free range, neighbours coalesced
  void reset(uint64_t bytes) {
    size = bytes;
    free.clear();
    if (bytes) free[0] = bytes;
  }
  bool take(uint64_t len, uint64_t* off) {
    for (auto it = free.begin(); it != free.end(); ++it) {
      if (it->second < len) continue;
      *off = it->first;
      const uint64_t rest = it->second - len, at = it->first + len;
      free.erase(it);
      if (rest) free[at] = rest;
      return true;
    }
    return false;
  }
  void give(uint64_t off, uint64_t len) {
    auto nx = free.lower_bound(off);
    if (nx != free.end() && off + len == nx->first) {  // merge with the range after
      len += nx->second;
      nx = free.erase(nx);
    }
    if (nx != free.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == off) {  // and with the one before
        pv->second += len;
        return;
      }
    }
    free[off] = len;
  }
};

}  // namespace

struct lcs_server {
  int device = 0;
  lcs_serve_cfg cfg{};
  uint64_t budget = 0;      // bytes of the bitmap arena
  uint64_t long_cells = 0;
  void* arena_mem = nullptr;
  Arena arena;

  std::mutex mu;
  std::condition_variable cv_short, cv_pair, cv_done;
  std::deque<Req*> q_short, q_len, q_tb;  // batch worker; pair workers: length-only, traceback
  std::unordered_map<uint64_t, Req*> reqs;  // every request until its result is released
  uint64_t next_ticket = 1;
  size_t live = 0;                          // waiting or running
  uint64_t reserved = 0;                    // bitmap bytes of tracebacks in flight
  bool stop = false;

  std::vector<std::thread> threads;
  std::vector<lcs_ctx*> ctxs;

  void finish(Req* r) {
    bool freed = false;
    {
      std::lock_guard<std::mutex> g(mu);
      r->t_done = now_s();
      --live;
      freed = r->bitmap != 0;
      if (freed) {
        reserved -= r->bitmap;
        arena.give(r->arena_off, r->bitmap);
      }
    }
    cv_done.notify_all();
    if (freed) cv_pair.notify_all();  // a traceback waiting for the budget may fit now
  }

  // The results of one batch wave, published together.
  void finish_wave(const std::vector<Req*>& rs) {
    {
      std::lock_guard<std::mutex> g(mu);
      const double t = now_s();
      for (Req* r : rs) r->t_done = t;
      live -= rs.size();
    }
    cv_done.notify_all();
  }

  // Next request for a pair worker (called with mu held): the older of the two heads, a traceback only when its
  // bitmap fits the budget.
  Req* take_pair() {
    Req* tb = q_tb.empty() ? nullptr : q_tb.front();
    Req* ln = q_len.empty() ? nullptr : q_len.front();
    if (tb && (!ln || tb->ticket < ln->ticket) && (!tb->bitmap || arena.take(tb->bitmap, &tb->arena_off))) {
      q_tb.pop_front();
      reserved += tb->bitmap;
      return tb;
    }
    if (ln) q_len.pop_front();
    return ln;
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
        cv_short.wait(lk, [&] { return stop || !q_short.empty(); });
        if (q_short.empty() && stop) return;
        take.clear();
        const size_t cap = std::min<size_t>(cfg.max_batch, std::max<size_t>(take.capacity(), 1));
        uint64_t bx = 0, by = 0;  // a wave stays within the sizes its buffers were grown for
        while (!q_short.empty() && take.size() < cap) {
          const Req* r = q_short.front();
          if (!take.empty() && (bx + r->x.size() > kWaveXBytes || by + r->y.size() > kWaveYBytes)) break;
          bx += r->x.size();
          by += r->y.size();
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
      }
      finish_wave(take);
    }
  }

  void pair_worker(lcs_ctx* c) {
    for (;;) {
      Req* r = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_pair.wait(lk, [&] { return (r = take_pair()) != nullptr || (stop && q_len.empty() && q_tb.empty()); });
        if (!r) return;  // stopping, nothing left
      }
      const uint8_t* x = r->x.empty() ? nullptr : r->x.data();
      const uint8_t* y = r->y.empty() ? nullptr : r->y.data();
      if (r->flags & LCS_TRACEBACK) {
        uint64_t len = 0;
        // the bitmap is the request's reservation in the arena, lent to the context for this call
        c->T.p = r->bitmap ? static_cast<char*>(arena_mem) + r->arena_off : nullptr;
        c->T.cap = r->bitmap;
        c->T.fixed = true;
        try {
          r->lcs.resize(std::max<size_t>(1, std::min(r->x.size(), r->y.size())));
          r->status = lcs_traceback(c, x, r->x.size(), y, r->y.size(), r->lcs.data(), r->lcs.size(), &len);
        } catch (...) {
          r->status = LCS_ERR_NOMEM;
        }
        if (c->T.overflow) r->status = LCS_ERR_INTERNAL;  // the reservation was too small (a sizing mistake)
        c->T = lcs::DBuf{};
        r->length = len;
        r->lcs.resize(r->status == LCS_OK ? len : 0);  // shrinking: no allocation
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
  int rc = LCS_OK;
  try {
    s->ctxs.reserve(kBatchWorkers + s->cfg.pair_workers);
    s->threads.reserve(kBatchWorkers + s->cfg.pair_workers);
    for (uint32_t k = 0; k < kBatchWorkers + s->cfg.pair_workers && !rc; ++k) {
      lcs_ctx* c = nullptr;
      rc = lcs_ctx_create(s->device, &c);
      if (!rc) {
        c->blocking_wait = true;  // many workers, few host cores: wait for the GPU asleep, not spinning
        s->ctxs.push_back(c);
      }
    }
    // buffers grown now, so that no request allocates: the batch workers' for their largest wave, every pair
    // worker's for pairs of up to 65536 x 65536
    for (uint32_t k = 0; k < kBatchWorkers && !rc; ++k)
      rc = lcs::batch_presize(s->ctxs[k], s->cfg.max_batch, kWaveXBytes, kWaveYBytes);
    for (uint32_t k = kBatchWorkers; k < s->ctxs.size() && !rc; ++k)
      rc = lcs::presize(s->ctxs[k], kPresizeLen, kPresizeLen);
    if (!rc && s->budget == 0) {  // default: the bitmaps of one 65536 x 65536 traceback per pair worker
      size_t free_b = 0, total_b = 0;
      rc = lcs::from_cuda(cudaMemGetInfo(&free_b, &total_b));
      const uint64_t one = lcs::traceback_bitmap_bytes(s->ctxs.back(), kPresizeLen, kPresizeLen);
      s->budget = std::min<uint64_t>((uint64_t)(free_b * 0.6), one * s->cfg.pair_workers);
    }
    s->budget = s->budget / kArenaAlign * kArenaAlign;
    if (!rc && s->budget) rc = lcs::from_cuda(cudaMalloc(&s->arena_mem, s->budget));
    if (!rc) s->arena.reset(s->budget);
    if (!rc) rc = lcs::from_cuda(cudaDeviceSynchronize());  // the buffers are in place before any request
    if (!rc) {
      for (uint32_t k = 0; k < kBatchWorkers; ++k) s->threads.emplace_back(&lcs_server::batch_worker, s, s->ctxs[k]);
      for (uint32_t k = 0; k < s->cfg.pair_workers; ++k)
        s->threads.emplace_back(&lcs_server::pair_worker, s, s->ctxs[kBatchWorkers + k]);
    }
  } catch (...) {  // a thread that could not start: stop the ones that did
    rc = LCS_ERR_INTERNAL;
  }
  if (rc) {
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->stop = true;
    }
    s->cv_short.notify_all();
    s->cv_pair.notify_all();
    for (auto& t : s->threads) t.join();
    for (lcs_ctx* d : s->ctxs) lcs_ctx_destroy(d);
    if (s->arena_mem) cudaFree(s->arena_mem);
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
  const uint64_t bm = tb ? lcs::traceback_bitmap_bytes(s->ctxs.back(), m, n) : 0;
  const uint64_t need = (bm + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
  if (need > s->budget) return LCS_ERR_NOMEM;
  std::unique_ptr<Req> owned(new (std::nothrow) Req());
  if (!owned) return LCS_ERR_NOMEM;
  // a length-only pair whose shorter side fits a batch row goes to the batch worker, longer side as X (rows)
  const bool swap = !tb && m < n && m <= 4096 && m * n < s->long_cells && n <= kShortMaxRows;
  owned->x.assign(swap ? y : x, swap ? y + n : x + m);  // may throw bad_alloc: the request is freed by owned
  owned->y.assign(swap ? x : y, swap ? x + m : y + n);
  Req* r = owned.get();
  r->flags = flags;
  r->bitmap = need;
  r->short_pair = !tb && r->y.size() <= 4096 && r->x.size() <= kShortMaxRows && m * n < s->long_cells;
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop || s->live >= s->cfg.max_queue) return s->stop ? LCS_ERR_INVALID : LCS_ERR_BUSY;
    r->ticket = s->next_ticket++;
    auto& q = r->short_pair ? s->q_short : (tb ? s->q_tb : s->q_len);
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
  if (r->short_pair) s->cv_short.notify_one();
  else s->cv_pair.notify_one();
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
  s->cv_short.notify_all();
  s->cv_pair.notify_all();
  for (auto& t : s->threads) t.join();
  for (lcs_ctx* c : s->ctxs) lcs_ctx_destroy(c);
  if (s->arena_mem) cudaFree(s->arena_mem);
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
}
