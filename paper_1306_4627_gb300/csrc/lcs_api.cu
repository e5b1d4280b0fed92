// C ABI of liblcs.so: contexts, LCS length and traceback for one pair (paper §I.C LCS-length, §I.D Print-LCS).
// Host code only; the kernels live in lcs_prep.cu, lcs_fill.cu and lcs_trace.cu.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "lcs_ctx.h"

int ensure_hstage(lcs_ctx* c, size_t bytes);  // below: the pinned staging area of a context

using namespace lcs;

extern "C" const char* lcs_strerror(int status) {
  switch (status) {
    case LCS_OK: return "ok";
    case LCS_PENDING: return "pending";
    case LCS_ERR_INVALID: return "invalid argument";
    case LCS_ERR_NOMEM: return "out of device memory";
    case LCS_ERR_CAPACITY: return "output buffer too small";
    case LCS_ERR_BUSY: return "queue full";
    case LCS_ERR_TIMEOUT: return "device wait timed out";
    case LCS_ERR_CUDA: return "CUDA error";
    case LCS_ERR_INTERNAL: return "internal consistency check failed";
    default: return "unknown status";
  }
}

namespace lcs {

int from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return LCS_OK;
  cudaGetLastError();  // clear a sticky-free error so the context stays usable
  if (e == cudaErrorMemoryAllocation) return LCS_ERR_NOMEM;
  return LCS_ERR_CUDA;
}

cudaError_t ensure(DBuf& b, size_t bytes) {
  if (bytes <= b.cap) return cudaSuccess;
  if (b.fixed) {  // neither freed nor replaced: the caller sees an allocation failure and the flag tells why
    b.overflow = true;
    return cudaErrorMemoryAllocation;
  }
  if (b.p) {
    cudaError_t e = cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    if (e != cudaSuccess) return e;
  }
  const size_t want = std::max<size_t>(bytes + bytes / 8, 256);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  b.p = p;
  b.cap = want;
  return cudaSuccess;
}

void release(DBuf& b) {
  if (b.fixed) return;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

// Waits for the context's stream: a spin wait by default, or a blocking wait on an event for contexts that set
// blocking_wait (the server's workers), which sleeps instead of spinning.
int wait_stream(lcs_ctx* c) {
  if (!c->blocking_wait) return from_cuda(cudaStreamSynchronize(c->stream));
  int rc = LCS_OK;
  if (!c->wait_ev) rc = from_cuda(cudaEventCreateWithFlags(&c->wait_ev, cudaEventBlockingSync | cudaEventDisableTiming));
  if (!rc) rc = from_cuda(cudaEventRecord(c->wait_ev, c->stream));
  if (!rc) rc = from_cuda(cudaEventSynchronize(c->wait_ev));
  return rc;
}

// Copies the status word back behind the work enqueued on the context's stream, waits for the stream, and returns
// the latched error (clearing it) or LCS_OK.
int fetch_status(lcs_ctx* c) {
  int rc = from_cuda(cudaMemcpyAsync(c->host_tail, (char*)c->small.p + kOffStatus, sizeof(DevStatus),
                                     cudaMemcpyDeviceToHost, c->stream));
  if (!rc) rc = wait_stream(c);
  if (rc) return rc;
  DevStatus h;
  std::memcpy(&h, c->host_tail, sizeof(h));
  if (h.flags == 0) return LCS_OK;
  cudaMemset(c->status(), 0, sizeof(DevStatus));
  return (h.flags & kStatTimeout) ? LCS_ERR_TIMEOUT : LCS_ERR_INTERNAL;
}

// Copies the status word and the result length of the call just enqueued on the context's stream back in one
// transfer, waits for the stream, and returns the latched error (clearing it) or LCS_OK with *len.
int fetch_result(lcs_ctx* c, uint64_t* len) {
  static_assert(kOffOutLen > kOffStatus && kOffOutLen - kOffStatus + 8 <= 8 * sizeof(uint64_t), "layout");
  int rc = from_cuda(cudaMemcpyAsync(c->host_tail, (char*)c->small.p + kOffStatus, kOffOutLen - kOffStatus + 8,
                                     cudaMemcpyDeviceToHost, c->stream));
  if (!rc) rc = wait_stream(c);
  if (rc) return rc;
  DevStatus h;
  std::memcpy(&h, c->host_tail, sizeof(h));
  std::memcpy(len, (const char*)c->host_tail + (kOffOutLen - kOffStatus), 8);
  if (h.flags == 0) return LCS_OK;
  cudaMemset(c->status(), 0, sizeof(DevStatus));
  return (h.flags & kStatTimeout) ? LCS_ERR_TIMEOUT : LCS_ERR_INTERNAL;
}

// Latched device status: returns its error (if any) and clears it. Caller has synchronised the stream.
int take_status(lcs_ctx* c) {
  DevStatus h{};
  if (cudaMemcpy(&h, c->status(), sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return from_cuda(cudaGetLastError());
  if (h.flags == 0) return LCS_OK;
  cudaMemset(c->status(), 0, sizeof(DevStatus));
  if (h.flags & kStatTimeout) return LCS_ERR_TIMEOUT;
  return LCS_ERR_INTERNAL;
}

// Runs one or two fill jobs: one cooperative launch when all their blocks fit on the GPU at once, otherwise each
// job alone, in passes of at most max_coop blocks (the carry slots between passes are complete in memory).
int run_fill(lcs_ctx* c, FillJob* jobs, int njobs, bool traceback, uint32_t B, cudaStream_t st) {
  FillArgs a{};
  a.status = c->status();
  a.spin_limit = c->spin_limit;
  a.variant = traceback ? c->fill_variant_tb : c->fill_variant;
  a.debug_drop = c->debug_drop;
  // traceback segments of fewer than 32 row-blocks need the dense snapshots (every 8 row-blocks); a period past the
  // last row (the table export: no snapshot at all) does not
  a.dense_snap =
      (traceback && jobs[0].snap && jobs[0].snap_rb % 32 != 0 && jobs[0].snap_rb <= jobs[0].R) ? 1u : 0u;
  uint32_t total = 0;
  for (int k = 0; k < njobs; ++k) total += jobs[k].nblocks_total;
  if (total <= (uint32_t)c->max_coop) {
    for (int k = 0; k < njobs; ++k) {
      a.job[k] = jobs[k];
      a.job[k].block0 = 0;
      a.job[k].nblocks = jobs[k].nblocks_total;
    }
    a.njobs = (uint32_t)njobs;
    return from_cuda(launch_fill(a, B, traceback, st));
  }
  for (int k = 0; k < njobs; ++k) {
    for (uint32_t b0 = 0; b0 < jobs[k].nblocks_total; b0 += (uint32_t)c->max_coop) {
      a.job[0] = jobs[k];
      a.job[0].block0 = b0;
      a.job[0].nblocks = std::min<uint32_t>((uint32_t)c->max_coop, jobs[k].nblocks_total - b0);
      a.njobs = 1;
      int rc = from_cuda(launch_fill(a, B, traceback, st));
      if (rc) return rc;
    }
  }
  return LCS_OK;
}

// Geometry of one table: words per row (one extra word catches the carry out of column n), blocks, lanes.
struct Geo {
  uint64_t wq, nblocks, wpad;
};
static Geo geo_for(uint64_t n) {
  Geo g;
  g.wq = n / 32 + 1;
  g.nblocks = (g.wq + kStripeWords - 1) / kStripeWords;
  g.wpad = g.nblocks * kStripeWords;
  return g;
}

// Prepares the alphabet of Y and the context's mask buffers; the masks of Y (forward and, if wanted, reversed) are
// built by the row-offset launch, as the returned job describes.
static int prep_y(lcs_ctx* c, const uint8_t* d_y, uint64_t n, const Geo& g, bool want_rev, PeqJob* pj,
                  cudaStream_t st) {
  int rc = from_cuda(ensure(c->peq_f, (size_t)kSigmaMax * g.wpad * 4));
  if (!rc && want_rev) rc = from_cuda(ensure(c->peq_r, (size_t)kSigmaMax * g.wpad * 4));
  if (rc) return rc;
  *pj = PeqJob{d_y, n, g.wpad, (uint32_t*)c->peq_f.p, want_rev ? (uint32_t*)c->peq_r.p : nullptr};
  return from_cuda(launch_alphabet(d_y, n, c->presence(), c->codemap(), c->sigma(), st));
}

// A small pair in one launch (lcs_small.cu): its stages are all under the fill's marks.
static int run_small(lcs_ctx* c, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n, bool traceback,
                     uint8_t* d_out, uint64_t out_cap, uint64_t* d_out_len, cudaStream_t st) {
  c->mark(0, st);
  c->mark(1, st);
  const int rc = from_cuda(launch_small(d_x, m, d_y, n, traceback, d_out, out_cap, d_out_len, c->status(), st));
  c->mark(2, st);
  c->mark(3, st);
  c->prof_valid = c->prof;
  c->prof_trace = traceback;
  c->prof_blocks = 1;
  c->prof_cells = m * n;
  return rc;
}

// Geometry of a length-only call. Meet in the middle: the top half of the rows forward, the bottom half on the
// reversed strings, at the same time; L = max_j (c[mt, j] + LCS(X[mt+1..m], Y[j+1..n])) (the recurrence read from
// both ends).
struct LenGeo {
  uint32_t B;
  Geo g;
  bool split;
  uint64_t mt, mb, Rf, padr, Rr;
};
static LenGeo len_geo(const lcs_ctx* c, uint64_t m, uint64_t n) {
  LenGeo L;
  L.B = c->fill_B;
  L.g = geo_for(n);
  L.split = m >= 2 * L.B && 2 * L.g.nblocks <= (uint64_t)c->max_coop;
  L.mt = L.split ? L.B * (m / (2 * L.B)) : m;
  L.mb = m - L.mt;
  L.Rf = (L.mt + L.B - 1) / L.B;
  L.padr = L.split ? (L.B - L.mb % L.B) % L.B : 0;
  L.Rr = L.split ? (L.mb + L.padr) / L.B : 0;
  return L;
}

// Every device buffer a length-only call of this geometry uses (grow-only).
static int ensure_len(lcs_ctx* c, const LenGeo& L) {
  const uint32_t B = L.B;
  const Geo& g = L.g;
  int rc = from_cuda(ensure(c->peq_f, (size_t)kSigmaMax * g.wpad * 4));
  if (!rc && L.split) rc = from_cuda(ensure(c->peq_r, (size_t)kSigmaMax * g.wpad * 4));
  if (!rc) rc = from_cuda(ensure(c->xoff_f, (L.Rf + kPadRowblocks + kPadBackRowblocks) * B * 4));
  if (!rc) rc = from_cuda(ensure(c->carry_f, g.nblocks * L.Rf * 4));
  if (!rc) rc = from_cuda(ensure(c->fv_f, g.wpad * 4));
  if (!rc && L.split) rc = from_cuda(ensure(c->xoff_r, (L.Rr + kPadRowblocks + kPadBackRowblocks) * B * 4));
  if (!rc && L.split) rc = from_cuda(ensure(c->carry_r, g.nblocks * L.Rr * 4));
  if (!rc && L.split) rc = from_cuda(ensure(c->fv_r, g.wpad * 4));
  if (!rc && L.split) rc = from_cuda(ensure(c->colsum, (2 * (g.wq + 1) + 4) * 4));
  return rc;
}

int run_length(lcs_ctx* c, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n, uint64_t* d_out,
               cudaStream_t st) {
  if (m == 0 || n == 0) return from_cuda(cudaMemsetAsync(d_out, 0, sizeof(uint64_t), st));
  if (c->small_path && small_pair(m, n)) return run_small(c, d_x, m, d_y, n, false, nullptr, 0, d_out, st);
  const LenGeo LG = len_geo(c, m, n);
  const uint32_t B = LG.B;
  const Geo& g = LG.g;
  const bool split = LG.split;
  const uint64_t mt = LG.mt, mb = LG.mb, Rf = LG.Rf, padr = LG.padr, Rr = LG.Rr;
  c->mark(0, st);
  int rc = ensure_len(c, LG);
  PeqJob pj{};
  if (!rc) rc = prep_y(c, d_y, n, g, split, &pj, st);
  if (rc) return rc;
  {  // row offsets of both tables; the hand-off slots and the length accumulator start at zero
    const XoffJob xj[2] = {{d_x, mt, 0, 0, Rf, (uint32_t*)c->xoff_f.p, nullptr},
                           {d_x + mt, mb, 1, padr, Rr, (uint32_t*)c->xoff_r.p, nullptr}};
    const ZeroSpan zs[3] = {{c->carry_f.p, g.nblocks * Rf * 4}, {c->len_acc(), sizeof(unsigned long long)},
                            {c->carry_r.p, g.nblocks * Rr * 4}};
    rc = from_cuda(launch_xoff(xj, split ? 2 : 1, B, c->codemap(), c->sigma(), zs, split ? 3 : 2, &pj, st));
  }
  if (rc) return rc;
  FillJob jobs[2]{};
  jobs[0].xoff = (const uint32_t*)c->xoff_f.p;
  jobs[0].peq = (const uint32_t*)c->peq_f.p;
  jobs[0].sigma_rows = c->sigma();
  jobs[0].carry = (uint32_t*)c->carry_f.p;
  jobs[0].final_v = split ? (uint32_t*)c->fv_f.p : nullptr;
  jobs[0].len_acc = split ? nullptr : c->len_acc();
  jobs[0].R = Rf;
  jobs[0].wpad = g.wpad;
  jobs[0].nblocks_total = (uint32_t)g.nblocks;
  if (split) {
    jobs[1] = jobs[0];
    jobs[1].xoff = (const uint32_t*)c->xoff_r.p;
    jobs[1].peq = (const uint32_t*)c->peq_r.p;
    jobs[1].carry = (uint32_t*)c->carry_r.p;
    jobs[1].final_v = (uint32_t*)c->fv_r.p;
    jobs[1].len_acc = nullptr;
    jobs[1].R = Rr;
  }
  c->mark(1, st);
  rc = run_fill(c, jobs, split ? 2 : 1, false, B, st);
  c->mark(2, st);
  if (rc) return rc;
  if (split)
    rc = from_cuda(launch_combine((const uint32_t*)c->fv_f.p, (const uint32_t*)c->fv_r.p, n, g.wq,
                                  (uint32_t*)c->colsum.p, (unsigned long long*)d_out, st));
  else
    rc = from_cuda(cudaMemcpyAsync(d_out, c->len_acc(), sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
  c->mark(3, st);
  c->prof_valid = c->prof;
  c->prof_trace = false;
  c->prof_blocks = g.nblocks * (split ? 2 : 1);
  c->prof_cells = m * n;
  return rc;
}

// Geometry of a traceback call. Segments of H rows for the parallel walk, at most kMaxSegments of them. H is a
// multiple of 32 * B (the fill snapshots a lane's word once per 32 steps) or, when that allows more and shorter
// segments, of 8 * B (the fill's dense snapshots, every 8 steps).
struct TbGeo {
  uint32_t B;
  Geo g;
  uint64_t H, S, Rf, padr, Rr, W;
  bool rev;
  size_t t_bytes;  // the direction bitmap
};
static TbGeo tb_geo(const lcs_ctx* c, uint64_t m, uint64_t n) {
  TbGeo T;
  T.B = c->fill_B_tb;
  T.g = geo_for(n);
  const uint64_t unit = 32ull * T.B;
  T.H = unit * ((m + kMaxSegments * unit - 1) / (kMaxSegments * unit));
  // Small pairs take shorter segments, down to 8 row-blocks: a walk is a chain of dependent steps, one or more per
  // row, so its time grows with H, and for a short fill the walks are a large share of the call. The fill then
  // snapshots every 8 row-blocks, which costs it 7-12 % more per step (measured), so larger pairs keep 32.
  const uint64_t unit8 = 8ull * T.B;
  const uint64_t Hd = unit8 * ((m + kMaxSegments * unit8 - 1) / (kMaxSegments * unit8));
  if (c->dense_snap && m <= kDenseSnapMaxRows && m * n <= kDenseSnapMaxCells && Hd < T.H) T.H = Hd;
  T.S = (m + T.H - 1) / T.H;
  T.rev = T.S > 1;
  T.Rf = (m + T.B - 1) / T.B;
  T.padr = T.S * T.H - m;
  T.Rr = T.rev ? (T.S * T.H) / T.B : 0;
  const uint64_t nwarps = T.g.nblocks * kFillWarps;
  T.t_bytes = (size_t)nwarps * (T.Rf + 31) * 32 * T.B * 4;
  // walkers per segment: as many as the corridor can have columns (n + 1), within the budget
  const uint64_t budget = T.H % unit ? kWalkerBudgetDense : kWalkerBudget;  // more segments, as many walkers each
  uint64_t W = std::min<uint64_t>(n + 1, std::min<uint64_t>(kMaxWalkersPerSeg, budget / T.S));
  T.W = std::max<uint64_t>(kWalkers, (W + kWalkers - 1) / kWalkers * kWalkers);
  return T;
}

// Every device buffer a traceback call of this geometry uses (grow-only), the bitmap only when with_T.
static int ensure_tb(lcs_ctx* c, const TbGeo& T, uint64_t m, bool with_T) {
  const uint32_t B = T.B;
  const Geo& g = T.g;
  const uint64_t S = T.S, W = T.W;
  int rc = from_cuda(ensure(c->peq_f, (size_t)kSigmaMax * g.wpad * 4));
  if (!rc && T.rev) rc = from_cuda(ensure(c->peq_r, (size_t)kSigmaMax * g.wpad * 4));
  if (!rc && with_T) rc = from_cuda(ensure(c->T, T.t_bytes));
  if (!rc) rc = from_cuda(ensure(c->xoff_f, (T.Rf + kPadRowblocks + kPadBackRowblocks) * B * 4));
  if (!rc) rc = from_cuda(ensure(c->xcode, m));
  if (!rc) rc = from_cuda(ensure(c->carry_f, g.nblocks * T.Rf * 4));
  if (!rc) rc = from_cuda(ensure(c->snap_f, S * g.wpad * 4));
  if (!rc && T.rev) rc = from_cuda(ensure(c->xoff_r, (T.Rr + kPadRowblocks + kPadBackRowblocks) * B * 4));
  if (!rc && T.rev) rc = from_cuda(ensure(c->carry_r, g.nblocks * T.Rr * 4));
  if (!rc && T.rev) rc = from_cuda(ensure(c->snap_r, S * g.wpad * 4));
  if (!rc) rc = from_cuda(ensure(c->colsum, (S * 2 * (g.wq + 1) + 4) * 4));
  if (!rc) rc = from_cuda(ensure(c->ent, S * W * 4));
  if (!rc) rc = from_cuda(ensure(c->ext, S * W * 4));
  if (!rc) rc = from_cuda(ensure(c->nch, S * W * 4));
  if (!rc) rc = from_cuda(ensure(c->entcnt, S * 4));
  if (!rc) rc = from_cuda(ensure(c->sel, S * 4));
  if (!rc) rc = from_cuda(ensure(c->chars, S * (W + 1) * T.H));
  if (!rc) rc = from_cuda(ensure(c->cmap, S * (g.wq * 32 + 1) * sizeof(uint16_t)));  // n + 1 <= 32 wq entries a row
  if (!rc) rc = from_cuda(ensure(c->wlink, S * W * sizeof(uint16_t)));
  return rc;
}

uint64_t traceback_bitmap_bytes(const lcs_ctx* c, uint64_t m, uint64_t n) {
  if (m == 0 || n == 0 || (c->small_path && small_pair(m, n))) return 0;
  return tb_geo(c, m, n).t_bytes;
}

// Grows every buffer a length-only or traceback call with m <= max_m and n <= max_n uses, except the traceback's
// direction bitmap, so that such calls allocate nothing (the growth keeps a margin for the few shapes whose
// walker buffers exceed those of (max_m, max_n) slightly).
int presize(lcs_ctx* c, uint64_t max_m, uint64_t max_n) {
  c->dense_snap = false;  // the segment geometry of (max_m, max_n) then bounds every smaller call's walker buffers
  int rc = ensure_len(c, len_geo(c, max_m, max_n));
  if (!rc) rc = ensure_tb(c, tb_geo(c, max_m, max_n), max_m, false);
  if (!rc) rc = from_cuda(ensure(c->x, std::max<uint64_t>(max_m, 1)));
  if (!rc) rc = from_cuda(ensure(c->y, std::max<uint64_t>(max_n, 1)));
  if (!rc) rc = from_cuda(ensure(c->out, std::max<uint64_t>(std::min(max_m, max_n), 1)));
  if (!rc) rc = ensure_hstage(c, max_m + max_n);
  return rc;
}

int run_traceback(lcs_ctx* c, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n, uint8_t* d_out,
                  uint64_t out_cap, uint64_t* d_out_len, cudaStream_t st) {
  if (m == 0 || n == 0) return from_cuda(cudaMemsetAsync(d_out_len, 0, sizeof(uint64_t), st));
  if (c->small_path && small_pair(m, n)) return run_small(c, d_x, m, d_y, n, true, d_out, out_cap, d_out_len, st);
  const TbGeo TG = tb_geo(c, m, n);
  const uint32_t B = TG.B;
  const Geo& g = TG.g;
  const uint64_t H = TG.H, S = TG.S, Rf = TG.Rf, padr = TG.padr, Rr = TG.Rr, W = TG.W;
  const bool rev = TG.rev;
  c->mark(0, st);
  int rc = ensure_tb(c, TG, m, true);
  PeqJob pj{};
  if (!rc) rc = prep_y(c, d_y, n, g, rev, &pj, st);
  if (rc) return rc;
  {  // row offsets of both tables; hand-off slots, length accumulator and corridor counts start at zero
    const XoffJob xj[2] = {{d_x, m, 0, 0, Rf, (uint32_t*)c->xoff_f.p, (uint8_t*)c->xcode.p},
                           {d_x, m, 1, padr, Rr, (uint32_t*)c->xoff_r.p, nullptr}};
    const ZeroSpan zs[4] = {{c->carry_f.p, g.nblocks * Rf * 4}, {c->len_acc(), sizeof(unsigned long long)},
                            {c->entcnt.p, S * 4}, {c->carry_r.p, g.nblocks * Rr * 4}};
    rc = from_cuda(launch_xoff(xj, rev ? 2 : 1, B, c->codemap(), c->sigma(), zs, rev ? 4 : 3, &pj, st));
  }
  if (rc) return rc;
  FillJob jobs[2]{};
  jobs[0].xoff = (const uint32_t*)c->xoff_f.p;
  jobs[0].peq = (const uint32_t*)c->peq_f.p;
  jobs[0].sigma_rows = c->sigma();
  jobs[0].carry = (uint32_t*)c->carry_f.p;
  jobs[0].T = (uint32_t*)c->T.p;
  jobs[0].snap = (uint32_t*)c->snap_f.p;
  jobs[0].snap_rb = (uint32_t)(H / B);
  jobs[0].len_acc = c->len_acc();
  jobs[0].R = Rf;
  jobs[0].wpad = g.wpad;
  jobs[0].nblocks_total = (uint32_t)g.nblocks;
  if (rev) {
    jobs[1] = jobs[0];
    jobs[1].xoff = (const uint32_t*)c->xoff_r.p;
    jobs[1].peq = (const uint32_t*)c->peq_r.p;
    jobs[1].carry = (uint32_t*)c->carry_r.p;
    jobs[1].T = nullptr;
    jobs[1].snap = (uint32_t*)c->snap_r.p;
    jobs[1].len_acc = nullptr;
    jobs[1].R = Rr;
  }
  c->mark(1, st);
  rc = run_fill(c, jobs, rev ? 2 : 1, true, B, st);
  c->mark(2, st);
  if (rc) return rc;
  TraceArgs t{};
  t.T = (const uint32_t*)c->T.p;
  t.peq = (const uint32_t*)c->peq_f.p;
  t.xcode = (const uint8_t*)c->xcode.p;
  t.x = d_x;
  t.snapF = (const uint32_t*)c->snap_f.p;
  t.snapR = (const uint32_t*)c->snap_r.p;
  t.L = c->len_acc();
  t.ent = (uint32_t*)c->ent.p;
  t.ent_cnt = (uint32_t*)c->entcnt.p;
  t.ext = (uint32_t*)c->ext.p;
  t.nch = (uint32_t*)c->nch.p;
  t.chars = (uint8_t*)c->chars.p;
  t.sel = (uint32_t*)c->sel.p;
  t.colsum = (uint32_t*)c->colsum.p;
  t.cmap = (uint16_t*)c->cmap.p;
  t.link = (uint16_t*)c->wlink.p;
  t.out = d_out;
  t.out_len = (unsigned long long*)d_out_len;
  t.out_cap = out_cap;
  t.m = m;
  t.n = n;
  t.w = g.wq;
  t.wpad = g.wpad;
  t.R = Rf;
  t.H = H;
  t.S = S;
  t.B = B;
  t.W = (uint32_t)W;
  t.status = c->status();
  rc = from_cuda(launch_traceback(t, st));
  c->mark(3, st);
  c->prof_valid = c->prof;
  c->prof_trace = true;
  c->prof_blocks = g.nblocks * (rev ? 2 : 1);
  c->prof_cells = m * n;
  return rc;
}

// ---- repeated single-pair calls, replayed as a CUDA graph ----------------------------------------------------------
// A single-pair call on the general path enqueues eight launches, one of them cooperative; for short pairs the host's
// cost per launch, not the GPU, sets the pace. When a call repeats the previous call's arguments exactly (a caller
// that reuses its buffers, such as a loop over pairs of one shape, or every host-buffer call of one shape, which
// stages into the context's own buffers), its launches are captured once as a CUDA graph, and this call and every
// further repeat replay the graph with one launch. The graph reads the buffers when it runs, so new strings in the
// same buffers give their own results.

// The arguments of a call and everything its launches take from the context: the fill configuration, the wait limit,
// the test hook, whether stage profiling is on (a profiled call's graph records the stage events) and the address of
// every device buffer.
static std::vector<uint64_t> pair_key(const lcs_ctx* c, bool traceback, const uint8_t* d_x, uint64_t m,
                                      const uint8_t* d_y, uint64_t n, const void* d_out, uint64_t out_cap,
                                      const void* d_out_len) {
  std::vector<uint64_t> k = {traceback ? 1u : 0u, (uint64_t)d_x, m, (uint64_t)d_y, n, (uint64_t)d_out, out_cap,
                             (uint64_t)d_out_len, c->fill_B, c->fill_B_tb, c->fill_variant, c->fill_variant_tb,
                             c->spin_limit, c->debug_drop, (uint64_t)c->max_coop, c->prof ? 1u : 0u};
  const DBuf* bufs[] = {&c->small, &c->xoff_f, &c->xoff_r, &c->xcode, &c->peq_f, &c->peq_r, &c->carry_f, &c->carry_r,
                        &c->fv_f, &c->fv_r, &c->T, &c->snap_f, &c->snap_r, &c->colsum, &c->ent, &c->ext, &c->nch,
                        &c->entcnt, &c->sel, &c->chars, &c->cmap, &c->wlink};
  for (const DBuf* b : bufs) k.push_back((uint64_t)b->p);
  return k;
}

int run_pair(lcs_ctx* c, bool traceback, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n,
             uint8_t* d_out, uint64_t out_cap, uint64_t* d_out_len, cudaStream_t st) {
  auto direct = [&](cudaStream_t s) {
    return traceback ? run_traceback(c, d_x, m, d_y, n, d_out, out_cap, d_out_len, s)
                     : run_length(c, d_x, m, d_y, n, d_out_len, s);
  };
  if (c->pgraph_off || m == 0 || n == 0 || (c->small_path && small_pair(m, n))) return direct(st);
  // every buffer of the call first, so that a capture never allocates
  int rc = traceback ? ensure_tb(c, tb_geo(c, m, n), m, true) : ensure_len(c, len_geo(c, m, n));
  if (rc) return rc;
  std::vector<uint64_t> key = pair_key(c, traceback, d_x, m, d_y, n, d_out, out_cap, d_out_len);
  if (c->pexec && key == c->pkey) {
    rc = from_cuda(cudaGraphLaunch(c->pexec, st));
    if (!rc && c->prof) {  // with profiling on, the graph records the stage events; the call is the captured one
      c->prof_valid = true;
      c->prof_trace = c->pprof_trace;
      c->prof_blocks = c->pprof_blocks;
      c->prof_cells = c->pprof_cells;
    }
    return rc;
  }
  if (key != c->pseen) {  // the first call with these arguments is launched directly
    c->pseen = std::move(key);
    return direct(st);
  }
  if (c->pexec) cudaGraphExecDestroy(c->pexec);
  c->pexec = nullptr;
  c->pkey.clear();
  if (!c->cap_stream) {
    rc = from_cuda(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    if (rc) return rc;
  }
  // the capture records the launches without running them; the graph then runs on st
  rc = from_cuda(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  if (rc) return rc;
  const int rc_run = direct(c->cap_stream);
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(c->cap_stream, &graph);
  cudaGraphExec_t exec = nullptr;
  cudaError_t ei = cudaErrorUnknown;
  if (rc_run == LCS_OK && ec == cudaSuccess && graph) ei = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {  // the launches could not be captured here: every call launches directly from now on
    cudaGetLastError();
    c->pgraph_off = true;
    return direct(st);
  }
  c->pexec = exec;
  c->pkey = std::move(key);
  c->pprof_trace = c->prof_trace;  // what the capture set for the stage profile of this call
  c->pprof_blocks = c->prof_blocks;
  c->pprof_cells = c->prof_cells;
  return from_cuda(cudaGraphLaunch(c->pexec, st));
}

// The full tables of LCS-length (§I.C): the forward fill over all m rows in traceback mode gives the direction
// bitmap; c and b are expanded from it (launch_tables). d_c: (m+1)(n+1) words, d_b: m*n bytes, row-major.
int run_tables(lcs_ctx* c, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n, uint32_t* d_c,
               uint8_t* d_b, cudaStream_t st) {
  if (m == 0 || n == 0) return from_cuda(cudaMemsetAsync(d_c, 0, (m + 1) * (n + 1) * sizeof(uint32_t), st));
  const uint32_t B = c->fill_B_tb;
  const Geo g = geo_for(n);
  const uint64_t Rf = (m + B - 1) / B;
  const uint64_t nwarps = g.nblocks * kFillWarps;
  const size_t t_bytes = (size_t)nwarps * (Rf + 31) * 32 * B * 4;
  PeqJob pj{};
  int rc = prep_y(c, d_y, n, g, false, &pj, st);
  if (!rc) rc = from_cuda(ensure(c->T, t_bytes));
  if (!rc) rc = from_cuda(ensure(c->xoff_f, (Rf + kPadRowblocks + kPadBackRowblocks) * B * 4));
  if (!rc) rc = from_cuda(ensure(c->carry_f, g.nblocks * Rf * 4));
  if (!rc) rc = from_cuda(ensure(c->snap_f, g.wpad * 4));
  if (!rc) rc = from_cuda(ensure(c->colsum, tables_sum_words(m, n) * 4));
  if (rc) return rc;
  {
    const XoffJob xj = {d_x, m, 0, 0, Rf, (uint32_t*)c->xoff_f.p, nullptr};
    const ZeroSpan zs[2] = {{c->carry_f.p, g.nblocks * Rf * 4}, {c->len_acc(), sizeof(unsigned long long)}};
    rc = from_cuda(launch_xoff(&xj, 1, B, c->codemap(), c->sigma(), zs, 2, &pj, st));
  }
  if (rc) return rc;
  FillJob job{};
  job.xoff = (const uint32_t*)c->xoff_f.p;
  job.peq = (const uint32_t*)c->peq_f.p;
  job.sigma_rows = c->sigma();
  job.carry = (uint32_t*)c->carry_f.p;
  job.T = (uint32_t*)c->T.p;
  job.snap = (uint32_t*)c->snap_f.p;  // a snapshot period past the last row: nothing is stored
  job.snap_rb = (uint32_t)(Rf + 1);
  job.len_acc = c->len_acc();
  job.R = Rf;
  job.wpad = g.wpad;
  job.nblocks_total = (uint32_t)g.nblocks;
  rc = run_fill(c, &job, 1, true, B, st);
  if (rc) return rc;
  TraceArgs t{};
  t.T = (const uint32_t*)c->T.p;
  t.x = d_x;
  t.m = m;
  t.n = n;
  t.R = Rf;
  t.B = B;
  return from_cuda(launch_tables(t, d_y, (uint32_t*)c->colsum.p, d_c, d_b, st));
}

}  // namespace lcs

// ---- C ABI -----------------------------------------------------------------------------------------------------

extern "C" int lcs_ctx_create(int device, lcs_ctx** out) {
  if (!out) return LCS_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return LCS_ERR_INVALID;
  }
  lcs_ctx* c = new (std::nothrow) lcs_ctx();
  if (!c) return LCS_ERR_NOMEM;
  c->device = device;
  int rc = from_cuda(cudaSetDevice(device));
  if (!rc) rc = from_cuda(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
  if (!rc) rc = from_cuda(ensure(c->small, kSmallBytes));
  if (!rc) rc = from_cuda(cudaMallocHost((void**)&c->host_tail, 8 * sizeof(uint64_t)));
  if (!rc) rc = from_cuda(cudaMemset(c->small.p, 0, kSmallBytes));
  if (!rc) {
    c->max_coop = fill_max_coop_blocks(device);
    if (c->max_coop <= 0) rc = LCS_ERR_CUDA;
  }
  if (rc) {
    lcs_ctx_destroy(c);
    return rc;
  }
  if (const char* e = getenv("LCS_FILL_B")) c->fill_B = c->fill_B_tb = (atoi(e) == 16) ? 16u : 8u;
  if (const char* e = getenv("LCS_FILL_VARIANT")) c->fill_variant = c->fill_variant_tb = (uint32_t)atoi(e);
  // bounded-wait testing: a short wait limit and a carry hand-off that is never published
  if (const char* e = getenv("LCS_SPIN_LIMIT")) c->spin_limit = (uint32_t)std::max(64, atoi(e));
  if (const char* e = getenv("LCS_DEBUG_DROP_HANDOFF")) c->debug_drop = atoi(e) ? 1u : 0u;
  if (const char* e = getenv("LCS_BATCH_BLOCKS_PER_SM")) c->batch_blocks_per_sm = atoi(e);
  // test hook: small pairs through the general path too
  if (const char* e = getenv("LCS_NO_SMALL_PATH")) c->small_path = atoi(e) == 0;
  // every single-pair call launched directly, never replayed as a graph (for comparisons)
  if (const char* e = getenv("LCS_NO_PAIR_GRAPH")) c->pgraph_off = atoi(e) != 0;
  // traceback segments of at least 32 row-blocks whatever the size (for comparisons)
  if (const char* e = getenv("LCS_NO_DENSE_SNAP")) c->dense_snap = atoi(e) == 0;
  *out = c;
  return LCS_OK;
}

extern "C" void lcs_ctx_destroy(lcs_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  c->release_all();
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->wait_ev) cudaEventDestroy(c->wait_ev);
  if (c->stream) cudaStreamDestroy(c->stream);
  if (c->host_tail) cudaFreeHost(c->host_tail);
  delete c;
}

extern "C" int lcs_ctx_sync(lcs_ctx* c) {
  if (!c) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  cudaSetDevice(c->device);
  int rc = from_cuda(cudaStreamSynchronize(c->stream));
  if (rc) return rc;
  return take_status(c);
}

static cudaStream_t pick(lcs_ctx* c, void* s) { return s ? (cudaStream_t)s : c->stream; }

extern "C" int lcs_ctx_set_profiling(lcs_ctx* c, int enable) {
  if (!c) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  cudaSetDevice(c->device);
  if (enable && !c->ev[0])
    for (auto& e : c->ev) {
      int rc = from_cuda(cudaEventCreate(&e));
      if (rc) return rc;
    }
  c->prof = enable != 0;
  c->prof_valid = false;
  return LCS_OK;
}

extern "C" int lcs_ctx_last_profile(lcs_ctx* c, lcs_profile* out) {
  if (!c || !out) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  if (!c->prof || !c->prof_valid) return LCS_ERR_INVALID;
  cudaSetDevice(c->device);
  int rc = from_cuda(cudaEventSynchronize(c->ev[3]));
  if (rc) return rc;
  float t01 = 0, t12 = 0, t23 = 0, t03 = 0;
  rc = from_cuda(cudaEventElapsedTime(&t01, c->ev[0], c->ev[1]));
  if (!rc) rc = from_cuda(cudaEventElapsedTime(&t12, c->ev[1], c->ev[2]));
  if (!rc) rc = from_cuda(cudaEventElapsedTime(&t23, c->ev[2], c->ev[3]));
  if (!rc) rc = from_cuda(cudaEventElapsedTime(&t03, c->ev[0], c->ev[3]));
  if (rc) return rc;
  out->prep_ms = t01;
  out->fill_ms = t12;
  out->trace_ms = c->prof_trace ? t23 : 0.0;
  out->total_ms = t03;
  out->fill_blocks = c->prof_blocks;
  out->cells = c->prof_cells;
  return LCS_OK;
}

extern "C" int lcs_length_dev(lcs_ctx* c, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n,
                              uint64_t* d_out_len, void* stream) {
  if (!c || !d_out_len || (m && !d_x) || (n && !d_y)) return LCS_ERR_INVALID;
  if (m >= (1ull << 32) || n >= (1ull << 32)) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  cudaSetDevice(c->device);
  return run_pair(c, false, d_x, m, d_y, n, nullptr, 0, d_out_len, pick(c, stream));
}

extern "C" int lcs_traceback_dev(lcs_ctx* c, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n,
                                 uint8_t* d_out, uint64_t out_cap, uint64_t* d_out_len, void* stream) {
  if (!c || !d_out_len || (m && !d_x) || (n && !d_y)) return LCS_ERR_INVALID;
  if (m >= (1ull << 32) || n >= (1ull << 32)) return LCS_ERR_INVALID;
  if (out_cap < std::min(m, n)) return LCS_ERR_CAPACITY;
  if (std::min(m, n) > 0 && !d_out) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  cudaSetDevice(c->device);
  return run_pair(c, true, d_x, m, d_y, n, d_out, out_cap, d_out_len, pick(c, stream));
}

// Copies host inputs into the context's device buffers.
// Grows the pinned host staging area to at least `bytes` (the old contents are not kept). The caller has waited for
// every copy that used it.
int ensure_hstage(lcs_ctx* c, size_t bytes) {
  if (bytes <= c->hstage_cap) return LCS_OK;
  if (c->hstage) cudaFreeHost(c->hstage);
  c->hstage = nullptr;
  c->hstage_cap = 0;
  const size_t want = std::max<size_t>(bytes + bytes / 4, 4096);
  void* p = nullptr;
  const int rc = from_cuda(cudaMallocHost(&p, want));
  if (rc) return rc;
  c->hstage = static_cast<uint8_t*>(p);
  c->hstage_cap = want;
  return LCS_OK;
}

// True when p is page-locked host memory (copies from it run asynchronously without the driver's staging).
bool host_pinned(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

// Copies host inputs into the context's device buffers. Pageable inputs up to kStageBytesMax go through the pinned
// staging area (a host copy, then asynchronous copies); pinned inputs and larger ones are copied directly. The
// previous call on the context has finished (its result was fetched), so the staging area is free.
static int stage_inputs(lcs_ctx* c, const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n) {
  int rc = from_cuda(ensure(c->x, std::max<uint64_t>(m, 1)));
  if (!rc) rc = from_cuda(ensure(c->y, std::max<uint64_t>(n, 1)));
  if (rc) return rc;
  const uint8_t* sx = x;
  const uint8_t* sy = y;
  if (m + n <= kStageBytesMax && !(m && host_pinned(x)) && ensure_hstage(c, m + n) == LCS_OK) {
    if (m) std::memcpy(c->hstage, x, m);
    if (n) std::memcpy(c->hstage + m, y, n);
    sx = c->hstage;
    sy = c->hstage + m;
  }
  if (m) rc = from_cuda(cudaMemcpyAsync(c->x.p, sx, m, cudaMemcpyHostToDevice, c->stream));
  if (!rc && n) rc = from_cuda(cudaMemcpyAsync(c->y.p, sy, n, cudaMemcpyHostToDevice, c->stream));
  return rc;
}

extern "C" int lcs_length(lcs_ctx* c, const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n,
                          uint64_t* out_len) {
  if (!c || !out_len || (m && !x) || (n && !y)) return LCS_ERR_INVALID;
  if (m >= (1ull << 32) || n >= (1ull << 32)) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  cudaSetDevice(c->device);
  *out_len = 0;
  int rc = stage_inputs(c, x, m, y, n);
  if (!rc) rc = run_pair(c, false, (const uint8_t*)c->x.p, m, (const uint8_t*)c->y.p, n, nullptr, 0, c->out_len(), c->stream);
  uint64_t L = 0;
  if (!rc) rc = fetch_result(c, &L);
  if (!rc) *out_len = L;
  return rc;
}

extern "C" int lcs_traceback(lcs_ctx* c, const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n, uint8_t* out,
                             uint64_t out_cap, uint64_t* out_len) {
  if (!c || !out_len || (m && !x) || (n && !y)) return LCS_ERR_INVALID;
  if (m >= (1ull << 32) || n >= (1ull << 32)) return LCS_ERR_INVALID;
  if (out_cap && !out) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  cudaSetDevice(c->device);
  *out_len = 0;
  const uint64_t cap = std::max<uint64_t>(std::min(m, n), 1);
  int rc = stage_inputs(c, x, m, y, n);
  if (!rc) rc = from_cuda(ensure(c->out, cap));
  if (!rc)
    rc = run_pair(c, true, (const uint8_t*)c->x.p, m, (const uint8_t*)c->y.p, n, (uint8_t*)c->out.p, cap,
                  c->out_len(), c->stream);
  // the string (at most min(m, n) bytes) comes back with the status and the length, behind one synchronisation. A
  // copy into pageable memory would go through the CUDA runtime's own staging, synchronously: a pageable destination
  // of up to kStageBytesMax bytes gets the string through the context's page-locked staging area instead (the input
  // copies from it are done by then: stream order; it already holds m + n >= take bytes when they used it)
  const uint64_t take = std::min<uint64_t>(std::min(m, n), out_cap);
  const bool staged = take && take <= kStageBytesMax && !host_pinned(out) && ensure_hstage(c, take) == LCS_OK;
  if (!rc && take)
    rc = from_cuda(cudaMemcpyAsync(staged ? c->hstage : out, c->out.p, take, cudaMemcpyDeviceToHost, c->stream));
  uint64_t L = 0;
  if (!rc) rc = fetch_result(c, &L);
  if (rc) return rc;
  *out_len = L;
  if (L > out_cap) return LCS_ERR_CAPACITY;
  if (staged && L) std::memcpy(out, c->hstage, L);
  return LCS_OK;
}

// Table sizes in bytes; false when they do not fit in 64 bits.
static bool table_bytes(uint64_t m, uint64_t n, uint64_t* cb, uint64_t* bb) {
  if (m >= (1ull << 32) || n >= (1ull << 32) || m > 65535ull * 64) return false;  // row chunks: one grid row each
  const unsigned __int128 cells = (unsigned __int128)(m + 1) * (n + 1);
  if (cells * 4 >= ((unsigned __int128)1 << 63)) return false;
  *cb = (uint64_t)cells * 4;
  *bb = m * n;
  return true;
}

extern "C" int lcs_tables_dev(lcs_ctx* c, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n,
                              uint32_t* d_c, uint8_t* d_b, void* stream) {
  uint64_t cb = 0, bb = 0;
  if (!c || !d_c || (m && !d_x) || (n && !d_y) || !table_bytes(m, n, &cb, &bb) || (bb && !d_b))
    return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  cudaSetDevice(c->device);
  return run_tables(c, d_x, m, d_y, n, d_c, d_b, pick(c, stream));
}

extern "C" int lcs_tables(lcs_ctx* c, const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n, uint32_t* cout,
                          uint8_t* bout) {
  uint64_t cb = 0, bb = 0;
  if (!c || !cout || (m && !x) || (n && !y) || !table_bytes(m, n, &cb, &bb) || (bb && !bout))
    return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  cudaSetDevice(c->device);
  void* dc = nullptr;
  void* db = nullptr;
  int rc = stage_inputs(c, x, m, y, n);
  if (!rc) rc = from_cuda(cudaMalloc(&dc, cb));
  if (!rc && bb) rc = from_cuda(cudaMalloc(&db, bb));
  if (!rc)
    rc = run_tables(c, (const uint8_t*)c->x.p, m, (const uint8_t*)c->y.p, n, (uint32_t*)dc, (uint8_t*)db,
                    c->stream);
  if (!rc) rc = from_cuda(cudaStreamSynchronize(c->stream));
  if (!rc) rc = take_status(c);
  if (!rc) rc = from_cuda(cudaMemcpy(cout, dc, cb, cudaMemcpyDeviceToHost));
  if (!rc && bb) rc = from_cuda(cudaMemcpy(bout, db, bb, cudaMemcpyDeviceToHost));
  if (dc) cudaFree(dc);
  if (db) cudaFree(db);
  return rc;
}

// ---- fill configuration and autotuning -------------------------------------------------------------------------

static bool valid_fill_config(const lcs_fill_config* f) {
  return f && (f->rows_per_step == 8 || f->rows_per_step == 16) && f->vg_select <= 1;
}

extern "C" int lcs_ctx_get_fill_config(lcs_ctx* c, uint32_t mode, lcs_fill_config* out) {
  if (!c || !out || mode > 1) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  out->rows_per_step = mode ? c->fill_B_tb : c->fill_B;
  out->vg_select = (((mode ? c->fill_variant_tb : c->fill_variant) >> 1) & 3u) == 2u ? 1u : 0u;
  return LCS_OK;
}

static void apply_fill_config(lcs_ctx* c, uint32_t mode, const lcs_fill_config* f) {
  const uint32_t var = f->vg_select ? 4u : 0u;  // bits 1-2 = 2: the alternative validation group
  if (mode) {
    c->fill_B_tb = f->rows_per_step;
    c->fill_variant_tb = var;
  } else {
    c->fill_B = f->rows_per_step;
    c->fill_variant = var;
  }
}

extern "C" int lcs_ctx_set_fill_config(lcs_ctx* c, uint32_t mode, const lcs_fill_config* cfg) {
  if (!c || mode > 1 || !valid_fill_config(cfg)) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  apply_fill_config(c, mode, cfg);
  return LCS_OK;
}

// Times every fill configuration on the caller's pair (one untimed call, then the median of three timed calls, each
// bracketed by events on the stream), keeps the fastest for the mode and reports it. Results do not depend on the
// configuration; only the time does.
extern "C" int lcs_ctx_autotune_dev(lcs_ctx* c, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n,
                                    uint32_t mode, void* stream, lcs_fill_config* best, double* best_ms) {
  if (!c || mode > 1 || (m && !d_x) || (n && !d_y)) return LCS_ERR_INVALID;
  if (m >= (1ull << 32) || n >= (1ull << 32)) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  cudaSetDevice(c->device);
  cudaStream_t st = pick(c, stream);
  const lcs_fill_config cand[4] = {{8, 0}, {8, 1}, {16, 0}, {16, 1}};
  lcs_fill_config keep{};
  keep.rows_per_step = mode ? c->fill_B_tb : c->fill_B;
  keep.vg_select = (((mode ? c->fill_variant_tb : c->fill_variant) >> 1) & 3u) == 2u ? 1u : 0u;
  const bool prof = c->prof;
  c->prof = false;
  const uint64_t cap = std::max<uint64_t>(std::min(m, n), 1);
  int rc = mode ? from_cuda(ensure(c->out, cap)) : LCS_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!rc) rc = from_cuda(cudaEventCreate(&e0));
  if (!rc) rc = from_cuda(cudaEventCreate(&e1));
  double bt = 1e300;
  lcs_fill_config bc = keep;
  for (const lcs_fill_config& f : cand) {
    if (rc) break;
    apply_fill_config(c, mode, &f);
    double ts[4];
    for (int k = 0; k < 4 && !rc; ++k) {
      rc = from_cuda(cudaEventRecord(e0, st));
      if (!rc)
        rc = mode ? run_traceback(c, d_x, m, d_y, n, (uint8_t*)c->out.p, cap, c->out_len(), st)
                  : run_length(c, d_x, m, d_y, n, c->out_len(), st);
      if (!rc) rc = from_cuda(cudaEventRecord(e1, st));
      if (!rc) rc = from_cuda(cudaEventSynchronize(e1));
      if (!rc) rc = take_status(c);
      float ms = 0.f;
      if (!rc) rc = from_cuda(cudaEventElapsedTime(&ms, e0, e1));
      ts[k] = ms;
    }
    if (rc) break;
    std::sort(ts + 1, ts + 4);
    if (ts[2] < bt) {
      bt = ts[2];
      bc = f;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->prof = prof;
  apply_fill_config(c, mode, rc ? &keep : &bc);
  if (rc) return rc;
  if (best) *best = bc;
  if (best_ms) *best_ms = bt;
  return LCS_OK;
}
