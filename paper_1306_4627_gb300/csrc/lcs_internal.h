// Internal declarations shared by the CUDA translation units of liblcs.so.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/lcs.h"

namespace lcs {

// ---- fill kernel geometry ------------------------------------------------------------------------------------
// One fill block = 4 warps (one per SM sub-partition); every lane owns one 32-bit word of the DP row, i.e. 32
// columns of Y. A block therefore covers a stripe of 128 words = 4096 columns.
constexpr int kFillWarps = 4;
constexpr int kFillThreads = kFillWarps * 32;
constexpr int kStripeWords = kFillThreads;
constexpr int kRing = 256;              // slots of the shared-memory carry ring between neighbouring warps
constexpr int kSigmaMax = 257;          // up to 256 byte values present in Y, plus the all-zero row
constexpr int kPadRowblocks = 32;       // zero row-blocks in front of every row-offset array
constexpr int kPadBackRowblocks = 128;  // zero row-blocks behind it (the fill reads up to 95 row-blocks past the end)

// ---- device status word (latched errors) ---------------------------------------------------------------------
constexpr uint32_t kStatTimeout = 1u;   // a bounded spin-wait expired
constexpr uint32_t kStatInternal = 2u;  // internal consistency check failed (e.g. traced length != c[m,n])

struct DevStatus {
  uint32_t flags;   // kStat* bits
  uint32_t abort;   // set together with a timeout: every waiting warp stops waiting
  uint32_t where;   // diagnostic: which wait gave up
  uint32_t pad;
};

// One DP problem for the fill kernel (a forward table, or the table of the reversed strings).
struct FillJob {
  const uint32_t* xoff;     // per padded row: word offset of its symbol's row in the block's shared Peq stripe;
                            // (kPadRowblocks + R + kPadBackRowblocks) * B entries
  const uint32_t* peq;      // match masks [sigma row][wpad], row 'sigma' (the last) all zero
  const uint32_t* sigma_rows;  // device word: rows of peq in use (present symbols + 1)
  uint32_t* carry;          // [nblocks_total][R] hand-off slots, block b's last warp -> block b+1's first warp
  uint32_t* T;              // traceback bitmap (carry-into vectors) or nullptr
  uint32_t* snap;           // V snapshots [k][wpad] at the ends of row-blocks r with (r+1) % snap_rb == 0
  uint32_t* final_v;        // V after the last row [wpad], or nullptr
  unsigned long long* len_acc;  // += popc(~V) over the row (number of zero bits = c[last row, n]), or nullptr
  uint64_t R;               // row-blocks
  uint64_t wpad;            // words per row = lanes of the job (nblocks_total * 128)
  uint32_t snap_rb;         // 0 = no snapshots
  uint32_t nblocks_total;   // blocks of the job over all passes
  uint32_t block0;          // first block of this launch (multi-pass)
  uint32_t nblocks;         // blocks in this launch
};

struct FillArgs {
  FillJob job[2];
  uint32_t njobs;
  DevStatus* status;
  uint32_t spin_limit;      // iterations of a bounded wait before it gives up
  uint32_t variant;         // bit 0: shorter dependent chain per row (same results)
  uint32_t debug_drop;      // test hook: the first warp never hands its carries on (its consumer's wait runs out)
  uint32_t dense_snap;      // traceback: snapshot rows every 8 row-blocks (snap_rb a multiple of 8) instead of 32
};

// ---- traceback segment walkers ---------------------------------------------------------------------------------
constexpr int kWalkers = 32;            // walkers per warp; a segment has W of them (a multiple of 32)
constexpr int kMaxWalkersPerSeg = 1024; // W <= this, and S * W <= kWalkerBudget (kWalkerBudgetDense for segments
constexpr int kWalkerBudget = 65536;    // of fewer than 32 row-blocks, whose snapshots come every 8 row-blocks)
constexpr int kWalkerBudgetDense = 1 << 18;
constexpr uint64_t kDenseSnapMaxRows = 8192;        // traceback pairs with shorter segments: at most this many rows
constexpr uint64_t kDenseSnapMaxCells = 1ull << 24;  // and cells
constexpr int kMaxSegments = 256;

struct TraceArgs {
  const uint32_t* T;        // forward bitmap (carry-into vectors, skewed chunk layout of the fill kernel)
  const uint32_t* peq;      // forward match masks [sigma][wpad]
  const uint8_t* xcode;     // symbol code per row (rows 1..m at index 0..m-1)
  const uint8_t* x;         // the original X (bytes emitted into the LCS)
  const uint32_t* snapF;    // forward V snapshots, index k-1 = row k*H
  const uint32_t* snapR;    // reverse V snapshots, index S-k-1 = forward row k*H
  const unsigned long long* L;  // c[m,n]
  uint32_t* ent;            // [S][W] entry columns of the walkers
  uint32_t* ent_cnt;        // [S] corridor columns found (more than W: the segment may need the fallback walk)
  uint32_t* ext;            // [S][W] exit columns
  uint32_t* nch;            // [S][W] symbols emitted by each walker
  uint8_t* chars;           // [S][W + 1][H] emitted symbols in walk order (slot W: the fallback walk)
  uint32_t* sel;            // [S] selected walker per segment
  uint32_t* colsum;         // scratch [2][S][w+1] word prefix popcounts
  uint16_t* cmap;           // [S][n+1] column -> walker of the segments with more than 32 walkers (k_corr_map)
  uint16_t* link;           // [S][W] walker of segment s - 1 that continues walker k of segment s (k_chain_links)
  uint8_t* out;             // LCS output (capacity out_cap)
  unsigned long long* out_len;
  uint64_t out_cap;
  uint64_t m, n, w, wpad, R, H, S;
  uint32_t B;
  uint32_t W;               // walkers per segment
  DevStatus* status;
};

// Runs set() (a cudaFuncSetAttribute call) once per device and process; done holds one bit per device.
template <typename F>
inline cudaError_t once_per_device_attr(F&& set, std::atomic<uint64_t>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = set();
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// ---- launchers (implemented in the .cu files) ------------------------------------------------------------------
// prep
constexpr uint64_t kAlphabetOneBlock = 1ull << 18;  // Y up to this length: the alphabet in one block, no clearing
constexpr int kMaxZeroSpans = 4;

// The row offsets of one table: x (m symbols, read backwards when reverse) after pad_front zero rows, R row-blocks
// of B rows, kPadRowblocks zero row-blocks in front and kPadBackRowblocks behind; xcode (or nullptr) receives the
// symbol codes of the m rows.
struct XoffJob {
  const uint8_t* x;
  uint64_t m;
  int reverse;
  uint64_t pad_front;
  uint64_t R;
  uint32_t* xoff;
  uint8_t* xcode;
};
struct ZeroSpan {  // device words to clear (bytes a multiple of 4)
  void* p;
  uint64_t bytes;
};

cudaError_t launch_alphabet(const uint8_t* y, uint64_t n, uint32_t* presence8, uint16_t* codemap,
                            uint32_t* sigma_rows, cudaStream_t st);
// The match masks of every symbol row 0..sigma for every word < wpad, over Y into peq_f and, if peq_r is not null,
// over reversed Y into peq_r.
struct PeqJob {
  const uint8_t* y;
  uint64_t n, wpad;
  uint32_t* peq_f;
  uint32_t* peq_r;
};
// The match masks (when peq is not null), the row offsets of up to two jobs and the clearing of up to kMaxZeroSpans
// spans, in one launch (all of it needs only the alphabet).
cudaError_t launch_xoff(const XoffJob* jobs, int njobs, uint32_t B, const uint16_t* codemap,
                        const uint32_t* sigma_rows, const ZeroSpan* zero, int nzero, const PeqJob* peq,
                        cudaStream_t st);
// fill
int fill_max_coop_blocks(int device);
cudaError_t launch_fill(const FillArgs& a, uint32_t B, bool traceback, cudaStream_t st);
size_t fill_smem_bytes();
// step floor probe: clock cycles of one systolic step of B rows (8 or 16) with the fill's row arithmetic and carry
// shuffles only (masks in registers; the two bitmap stores per step in traceback mode), one warp per scheduler
cudaError_t step_floor(uint32_t B, bool traceback, uint32_t steps, double* cycles_per_step);
// One 8-row traceback step with the match masks from source 0..3 (registers, the fill's shared table, bit planes
// with byte-permuted codes, bit planes with expanded row masks); see k_step_floor.
cudaError_t step_masks(uint32_t source, uint32_t steps, double* cycles_per_step);
// length meet-in-the-middle combine: L = n - min_j (pf(j) + pr(n-j))
cudaError_t launch_combine(const uint32_t* vf, const uint32_t* vr, uint64_t n, uint64_t w,
                           uint32_t* colsum, unsigned long long* out_len, cudaStream_t st);
// traceback
cudaError_t launch_traceback(const TraceArgs& t, cudaStream_t st);
// full tables c, b from the forward bitmap (t.T, t.x, t.m, t.n, t.R, t.B); sums holds tables_sum_words words
cudaError_t launch_tables(const TraceArgs& t, const uint8_t* y, uint32_t* sums, uint32_t* c, uint8_t* b,
                          cudaStream_t st);
uint64_t tables_sum_words(uint64_t m, uint64_t n);
// small pairs in one launch (one warp, masks and bitmap in shared memory): length, and the LCS in traceback mode
constexpr uint64_t kSmallMaxRows = 1024;
constexpr uint64_t kSmallMaxCols = 992;  // 31 words, so the row's words and the column-n carry fit one warp
bool small_pair(uint64_t m, uint64_t n);
cudaError_t launch_small(const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n, bool traceback, uint8_t* out,
                         uint64_t out_cap, uint64_t* out_len, DevStatus* status, cudaStream_t st);

}  // namespace lcs
