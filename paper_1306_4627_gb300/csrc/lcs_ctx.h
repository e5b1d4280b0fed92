// The context behind lcs_ctx*: streams, grow-only device buffers and the small control block.
#pragma once

#include <cstdint>
#include <mutex>
#include <vector>

#include "lcs_internal.h"

namespace lcs {

struct DBuf {
  void* p = nullptr;
  size_t cap = 0;
  bool fixed = false;     // memory the buffer does not own (a carved part of a static array): never freed or grown
  bool overflow = false;  // set when a request did not fit a fixed buffer (ensure() then fails instead of growing)
};

cudaError_t ensure(DBuf& b, size_t bytes);
void release(DBuf& b);
int from_cuda(cudaError_t e);
int wait_stream(lcs_ctx* c);   // waits for the context's stream (spin or blocking wait, see lcs_ctx::blocking_wait)
int fetch_status(lcs_ctx* c);  // copies the status word back behind the stream's work, waits, returns its error

// Layout of the small control block (bytes).
constexpr size_t kOffCodemap = 0;      // uint16_t[256]
constexpr size_t kOffPresence = 512;   // uint32_t[8]
constexpr size_t kOffSigma = 544;      // uint32_t
constexpr size_t kOffLenAcc = 552;     // unsigned long long
constexpr size_t kOffStatus = 576;     // DevStatus (16 B)
constexpr size_t kOffOutLen = 608;     // uint64_t
constexpr size_t kOffTicket = 640;     // uint32_t[2] work tickets of the persistent batch kernels
constexpr size_t kSmallBytes = 1024;
constexpr uint64_t kStageBytesMax = 4ull << 20;  // pageable host inputs up to this size go through pinned staging

}  // namespace lcs

struct lcs_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int max_coop = 0;
  uint32_t spin_limit = 1u << 22;
  uint32_t fill_B = 8;        // rows per systolic step of length-only fills (8 or 16)
  uint32_t fill_B_tb = 8;     // rows per systolic step of traceback fills
  uint32_t fill_variant = 0;     // length-only fills: bits 1-2 select the hand-off validation group (see launch_fill)
  uint32_t fill_variant_tb = 0;  // the same for traceback fills
  int b_sms = 0, b_prep_per_sm = 0, b_main_occ = 0;  // batch: SMs and blocks per SM (looked up once)
  int b_main_occ_k[3] = {0, 0, 0};  // batch row kernel: blocks per SM at the stage sizes of 2 / 4 / 8 words per lane
  // batch configuration (lcs_ctx_set_batch_config): words per lane, split height in % of the average rows per
  // resident warp (0 = never split), persistent kernel blocks per SM (0 = one)
  uint32_t batch_k = 4, batch_split_pct = 100;
  int batch_blocks_per_sm = 0;
  uint32_t bk_max = 4;  // the planned batch's largest words per lane
  uint32_t debug_drop = 0;    // test hook (environment LCS_DEBUG_DROP_HANDOFF): a hand-off that never comes
  bool small_path = true;     // small pairs in one launch (lcs_small.cu); environment LCS_NO_SMALL_PATH=1 turns it off
  bool dense_snap = true;     // traceback segments of 8 row-blocks and up (else 32 and up); LCS_NO_DENSE_SNAP=1: off
  // host-buffer calls wait for their stream by a spin (lowest latency) or, when set (the server's workers: many
  // contexts waiting at once on few host cores), by sleeping on an event recorded with blocking synchronisation
  bool blocking_wait = false;
  cudaEvent_t wait_ev = nullptr;
  std::mutex mu;
  lcs::DBuf small, x, y, out;
  lcs::DBuf xoff_f, xoff_r, xcode, peq_f, peq_r, carry_f, carry_r, fv_f, fv_r, T, snap_f, snap_r;
  lcs::DBuf colsum, ent, ext, nch, entcnt, sel, chars, cmap, wlink;
  lcs::DBuf bplan, bsig, bxcode, bpeq, bout, bfv;  // batch: plan, alphabet sizes, codes, masks, lengths, half rows
  // batch: the last plan's launches captured as a CUDA graph, replayed while the same batch is submitted again
  bool bvalid = false;
  uint64_t bptrs[4] = {0, 0, 0, 0};
  std::vector<uint64_t> boffs;  // relative offsets of the planned batch, x and y interleaved
  cudaGraphExec_t bexec = nullptr;
  std::vector<uint64_t> bbig;
  uint64_t bcells = 0, bblocks = 0, bnpairs = 0, bnitems = 0, bnsplit = 0;
  uint64_t bjobs_at = 0, bitems_at = 0, bsplit_at = 0, border_at = 0;  // byte offsets of the plan's parts in bplan
  cudaStream_t cap_stream = nullptr;
  // single-pair calls: the last call's arguments (pseen), and the launches of a call that repeated them captured as a
  // CUDA graph (pexec, for the arguments pkey), replayed while they keep repeating; pgraph_off after a failed capture
  std::vector<uint64_t> pseen, pkey;
  cudaGraphExec_t pexec = nullptr;
  bool pgraph_off = false;
  // pinned host memory: the status word and result length of a call (fetched together), and a staging area for
  // host-buffer calls' inputs and traceback output (copies from pinned memory run asynchronously)
  uint64_t* host_tail = nullptr;  // 8 words
  uint8_t* hstage = nullptr;
  size_t hstage_cap = 0;
  // pinned copy of the last batch plan (uploaded with one asynchronous copy; the event marks that copy's end)
  uint8_t* hplan = nullptr;
  size_t hplan_cap = 0;
  cudaEvent_t hplan_ev = nullptr;
  // stage events of the last profiled call: [0] start, [1] fill start, [2] fill end, [3] end
  bool prof = false, prof_valid = false, prof_trace = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  uint64_t prof_blocks = 0, prof_cells = 0;
  // the same for a call captured into a graph (see run_pair): what the last call replayed reports
  bool pprof_trace = false;
  uint64_t pprof_blocks = 0, pprof_cells = 0;
  void mark(int k, cudaStream_t st) {
    if (!prof) return;
    // inside a stream capture the record becomes a node of the graph, which records the event each time it runs
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
      cudaEventRecordWithFlags(ev[k], st, cudaEventRecordExternal);
    else
      cudaEventRecord(ev[k], st);
  }

  uint16_t* codemap() { return (uint16_t*)((char*)small.p + lcs::kOffCodemap); }
  uint32_t* presence() { return (uint32_t*)((char*)small.p + lcs::kOffPresence); }
  uint32_t* sigma() { return (uint32_t*)((char*)small.p + lcs::kOffSigma); }
  unsigned long long* len_acc() { return (unsigned long long*)((char*)small.p + lcs::kOffLenAcc); }
  lcs::DevStatus* status() { return (lcs::DevStatus*)((char*)small.p + lcs::kOffStatus); }
  uint64_t* out_len() { return (uint64_t*)((char*)small.p + lcs::kOffOutLen); }

  void release_all() {
    if (hstage) cudaFreeHost(hstage);
    hstage = nullptr;
    hstage_cap = 0;
    if (hplan_ev) cudaEventSynchronize(hplan_ev);
    if (hplan) cudaFreeHost(hplan);
    hplan = nullptr;
    hplan_cap = 0;
    if (hplan_ev) cudaEventDestroy(hplan_ev);
    hplan_ev = nullptr;
    if (bexec) cudaGraphExecDestroy(bexec);
    bexec = nullptr;
    bvalid = false;
    if (pexec) cudaGraphExecDestroy(pexec);
    pexec = nullptr;
    pkey.clear();
    pseen.clear();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cap_stream = nullptr;
    lcs::DBuf* all[] = {&small, &x, &y, &out, &xoff_f, &xoff_r, &xcode, &peq_f, &peq_r, &carry_f, &carry_r,
                        &fv_f, &fv_r, &T, &snap_f, &snap_r, &colsum, &ent, &ext, &nch, &entcnt, &sel, &chars, &cmap, &wlink,
                        &bplan, &bsig, &bxcode, &bpeq, &bout, &bfv};
    for (lcs::DBuf* b : all) lcs::release(*b);
  }
};
