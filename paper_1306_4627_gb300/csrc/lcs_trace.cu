// Traceback (paper §I.D, Print-LCS) over the 1-bit direction bitmap of the fill kernel, made parallel.
//
// Print-LCS walks from (m, n) towards row 0: DIAG on a match (emit x_i), else UP when c[i-1,j] >= c[i,j-1],
// else LEFT. At row i the walk moves left past LEFT cells to the first column c <= j that is a match or an UP
// cell, then steps to row i-1 (to column c-1 on a match, to c otherwise). That is one word scan per row here.
//
// The rows are cut into S segments of H rows, and every segment is walked at once by its walkers (a warp each when
// the segment has at most 32 of them, a thread each otherwise). Where the true path enters a segment is unknown
// until the segment below is done, but it must lie on an optimal
// path, so it is one of the columns j of the segment's bottom row with c[i,j] + LCS(X[i+1..m], Y[j+1..n]) = c[m,n]
// ("corridor" columns). The prefix lengths c[i,.] come from V snapshots of the forward fill, the suffix lengths
// from V snapshots of the same fill run on the reversed strings. Every corridor column gets a walker; a short
// chain pass then follows the true path from (m, n) segment by segment, picking in each segment the walker whose
// entry is the exit of the segment below (or walking the segment itself when the corridor had more columns than
// walkers). The chosen walkers' symbols are finally copied to the output in order. The result is exactly the walk
// of Print-LCS; only the order of the work differs.
#include <algorithm>
#include <atomic>

#include "lcs_internal.h"

namespace lcs {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint64_t kWarpWalkers = 32;  // corridors of up to this many columns get a warp per walker

// ---- word prefix popcounts of V rows ------------------------------------------------------------------------
// For a V row (bit j-1 of the row = 1 - (c[i,j] - c[i,j-1])), pre[q] = ones among the first 32*q bits, q = 0..w.
// One block (a multiple of 32 threads, at most 1024) does NR rows at once: each thread sums a contiguous run of words
// of every row, the runs' totals are scanned by shuffles within each warp and then over the warps' totals, and each
// thread writes the prefixes of its runs.
template <int NR>
__device__ void block_prefix_popc(const uint32_t* const (&v)[NR], uint64_t w, uint32_t* const (&pre)[NR]) {
  __shared__ uint32_t wsum[NR][32];
  const uint32_t nt = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const uint64_t per = (w + nt - 1) / nt;
  const uint64_t q0 = tid * per, q1 = (q0 + per < w) ? q0 + per : w;
  uint32_t s[NR], incl[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    s[r] = 0;
    for (uint64_t q = q0; q < q1; ++q) s[r] += __popc(v[r][q]);
    incl[r] = s[r];
  }
  for (uint32_t off = 1; off < 32; off <<= 1) {  // inclusive scan of the run totals within the warp
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const uint32_t o = __shfl_up_sync(kFull, incl[r], off);
      if (lane >= off) incl[r] += o;
    }
  }
  if (lane == 31) {
#pragma unroll
    for (int r = 0; r < NR; ++r) wsum[r][wid] = incl[r];
  }
  __syncthreads();
  if (wid == 0) {  // inclusive scan of the warps' totals
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      uint32_t t = lane < nw ? wsum[r][lane] : 0u;
      for (uint32_t off = 1; off < 32; off <<= 1) {
        const uint32_t o = __shfl_up_sync(kFull, t, off);
        if (lane >= off) t += o;
      }
      if (lane < nw) wsum[r][lane] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    uint32_t run = (wid ? wsum[r][wid - 1] : 0u) + incl[r] - s[r];
    for (uint64_t q = q0; q < q1; ++q) {
      pre[r][q] = run;
      run += __popc(v[r][q]);
    }
    if (tid == nt - 1) pre[r][w] = wsum[r][nw - 1];
  }
  __syncthreads();
}

// ones among the first x bits of the row
__device__ __forceinline__ uint32_t ones_prefix(const uint32_t* v, const uint32_t* pre, uint64_t x) {
  const uint64_t q = x >> 5;
  const uint32_t k = (uint32_t)(x & 31);
  return pre[q] + (k ? __popc(v[q] & ((1u << k) - 1u)) : 0u);
}

// ---- meet-in-the-middle length: L = n - min_j (ones_f(j) + ones_r(n - j)) -----------------------------------
__global__ void k_combine_pre(const uint32_t* vf, const uint32_t* vr, uint64_t w, uint32_t* colsum) {
  const uint32_t* const v[1] = {blockIdx.x == 0 ? vf : vr};
  uint32_t* const pre[1] = {colsum + blockIdx.x * (w + 1)};
  block_prefix_popc<1>(v, w, pre);
  if (blockIdx.x == 0 && threadIdx.x == 0) colsum[2 * (w + 1)] = 0xFFFFFFFFu;  // running minimum
}

__global__ void k_combine_min(const uint32_t* vf, const uint32_t* vr, uint64_t n, uint64_t w, uint32_t* colsum) {
  const uint32_t* pf = colsum;
  const uint32_t* pr = colsum + (w + 1);
  uint32_t best = 0xFFFFFFFFu;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= n; j += stride) {
    const uint32_t s = ones_prefix(vf, pf, j) + ones_prefix(vr, pr, n - j);
    best = s < best ? s : best;
  }
  best = __reduce_min_sync(kFull, best);
  if ((threadIdx.x & 31) == 0) atomicMin(colsum + 2 * (w + 1), best);
}

// Rows up to kCombineOneBlockWords words (n < 65536): prefix popcounts, the minimum and the length in one block.
constexpr uint64_t kCombineOneBlockWords = 2048;

__global__ void __launch_bounds__(1024) k_combine_small(const uint32_t* vf, const uint32_t* vr, uint64_t n,
                                                        uint64_t w, unsigned long long* out_len) {
  __shared__ uint32_t pre[2][kCombineOneBlockWords + 1];
  __shared__ uint32_t part[1024];
  __shared__ uint32_t red[32];
  const uint32_t tid = threadIdx.x;
  for (int d = 0; d < 2; ++d) {  // pre[d][q] = ones among the first 32 q bits of the row
    const uint32_t* v = d ? vr : vf;
    const uint64_t per = (w + 1023) / 1024;
    const uint64_t q0 = tid * per, q1 = q0 + per < w ? q0 + per : w;
    uint32_t sum = 0;
    for (uint64_t q = q0; q < q1; ++q) sum += __popc(v[q]);
    part[tid] = sum;
    __syncthreads();
    for (uint32_t off = 1; off < 1024; off <<= 1) {
      const uint32_t add = tid >= off ? part[tid - off] : 0u;
      __syncthreads();
      part[tid] += add;
      __syncthreads();
    }
    uint32_t run = part[tid] - sum;
    for (uint64_t q = q0; q < q1; ++q) {
      pre[d][q] = run;
      run += __popc(v[q]);
    }
    if (tid == 1023) pre[d][w] = part[tid];
    __syncthreads();
  }
  uint32_t best = 0xFFFFFFFFu;
  for (uint64_t j = tid; j <= n; j += 1024) {
    const uint64_t x = n - j;
    const uint32_t of = pre[0][j >> 5] + ((j & 31) ? __popc(vf[j >> 5] & ((1u << (j & 31)) - 1u)) : 0u);
    const uint32_t orr = pre[1][x >> 5] + ((x & 31) ? __popc(vr[x >> 5] & ((1u << (x & 31)) - 1u)) : 0u);
    best = of + orr < best ? of + orr : best;
  }
  best = __reduce_min_sync(kFull, best);
  if ((tid & 31) == 0) red[tid >> 5] = best;
  __syncthreads();
  if (tid < 32) {
    best = __reduce_min_sync(kFull, red[tid]);
    if (tid == 0) *out_len = (unsigned long long)(n - best);
  }
}

__global__ void k_combine_fin(const uint32_t* colsum, uint64_t n, uint64_t w, unsigned long long* out_len) {
  *out_len = (unsigned long long)(n - colsum[2 * (w + 1)]);
}

// ---- corridors -------------------------------------------------------------------------------------------------
// Boundary k (1..S-1) is forward row k*H, the bottom row of segment k-1.
__global__ void k_corr_pre(TraceArgs a) {
  const uint64_t k = blockIdx.x + 1;
  const uint64_t wp1 = a.w + 1;
  const uint32_t* const v[2] = {a.snapF + (k - 1) * a.wpad, a.snapR + (a.S - k - 1) * a.wpad};
  uint32_t* const pre[2] = {a.colsum + (2 * (k - 1)) * wp1, a.colsum + (2 * (k - 1) + 1) * wp1};
  block_prefix_popc<2>(v, a.w, pre);
}

// Thread (q, boundary k): the columns j = 32q .. 32q + 31 (up to n) of the boundary's row. ones_f(j) comes from
// the forward snapshot's word q, ones_r(n - j) from the at most two words of the reverse snapshot that hold the
// positions n - 32q - 31 .. n - 32q, so a thread reads six words for its 32 columns.
__global__ void __launch_bounds__(128) k_corr_cols(TraceArgs a) {
  __shared__ uint32_t wsum[4];
  __shared__ uint32_t base_s;
  const uint64_t k = blockIdx.y + 1;
  const uint64_t wp1 = a.w + 1;
  const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t j0 = q * 32;
  const uint64_t s = k - 1;
  uint32_t hits = 0;  // bit t: column j0 + t is a corridor column
  if (j0 <= a.n) {
    const uint32_t* vf = a.snapF + (k - 1) * a.wpad;
    const uint32_t* vr = a.snapR + (a.S - k - 1) * a.wpad;
    const uint32_t* pf = a.colsum + (2 * (k - 1)) * wp1;
    const uint32_t* pr = a.colsum + (2 * (k - 1) + 1) * wp1;
    const uint32_t target = (uint32_t)(a.n - *a.L);  // c[i,j] + suffix = n - (ones_f + ones_r); optimal at n - L
    const uint32_t bf = pf[q], wf = vf[q];
    const uint64_t xb = a.n - j0;                      // the reverse position of column j0 (the largest)
    const uint64_t qb = xb >> 5;
    const uint64_t qa = xb >= 31 ? (xb - 31) >> 5 : 0; // the word of the smallest position used
    const uint32_t bra = pr[qa], wra = vr[qa];
    // Over the thread's columns, ones_f(j) never falls below its value at j0 (bf) and ones_r(n - j) never below
    // its value at the smallest reverse position used (xa): when even that sum is above the optimum, no column here
    // is on an optimal path (the usual case: a corridor is a few columns of the row).
    const uint32_t ra = (uint32_t)((xb >= 31 ? xb - 31 : 0) & 31);  // xa = that position, in word qa
    if (bf + bra + (ra ? __popc(wra & ((1u << ra) - 1u)) : 0u) <= target) {
      const uint32_t brb = pr[qb], wrb = qb < a.w ? vr[qb] : 0u;
      for (uint32_t t = 0; t < 32; ++t) {
        const uint64_t j = j0 + t;
        if (j > a.n) break;
        const uint64_t x = a.n - j;
        const uint32_t r = (uint32_t)(x & 31);
        const bool inb = (x >> 5) == qb;
        const uint32_t of = bf + (t ? __popc(wf & ((1u << t) - 1u)) : 0u);
        const uint32_t orr = (inb ? brb : bra) + (r ? __popc((inb ? wrb : wra) & ((1u << r) - 1u)) : 0u);
        if (of + orr == target) hits |= 1u << t;
      }
    }
  }
  // Walker slots in column order within the block: a scan of the threads' counts, one reservation per block, so
  // that the walkers of a warp start at neighbouring corridor columns (their paths run together).
  const uint32_t cnt = __popc(hits), lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = cnt;
#pragma unroll
  for (uint32_t off = 1; off < 32; off <<= 1) {
    const uint32_t o = __shfl_up_sync(kFull, incl, off);
    if (lane >= off) incl += o;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t total = wsum[0] + wsum[1] + wsum[2] + wsum[3];
    base_s = total ? atomicAdd(&a.ent_cnt[s], total) : 0u;
  }
  __syncthreads();
  uint32_t slot = base_s + incl - cnt;
  for (uint32_t w = 0; w < wid; ++w) slot += wsum[w];
  for (uint32_t h = hits; h; h &= h - 1, ++slot) {
    const uint64_t j = j0 + (uint32_t)(__ffs(h) - 1);
    if (slot < a.W) {
      a.ent[s * a.W + slot] = (uint32_t)j;
      a.cmap[s * (a.n + 1) + j] = (uint16_t)slot;  // the column -> walker map (see map_lookup)
    }
  }
}

// ---- the walk of one segment -------------------------------------------------------------------------------------
// Direction bit of cell (i, c): bit c%32 of T-frame word c/32 of row i holds c[i,c] - c[i-1,c] (the carry into
// column c+1's bit); 0 = UP, 1 = LEFT on a mismatch. Match bit of (i, c): bit (c-1)%32 of Peq word (c-1)/32.
// Bitmap layout of the fill kernel: warp g's chunk for step t holds, for each of its 32 lanes, the B words of the
// row-block that lane processed at that step (lane l at step t: row-block t - l), as [B/4][32 lanes][4 words].
__device__ __forceinline__ uint32_t t_word(const TraceArgs& a, uint64_t i, uint64_t Q) {
  const uint32_t lb = 31u - __clz(a.B);  // B is a power of two (8 or 16)
  const uint32_t i0 = (uint32_t)(i - 1), b = i0 & (a.B - 1);
  const uint64_t chunk = (Q >> 5) * (a.R + 31) + (i0 >> lb) + (Q & 31);
  return a.T[(chunk << (5 + lb)) + (b >> 2) * 128 + (Q & 31) * 4 + (b & 3)];
}

__device__ __forceinline__ uint32_t p_word(const TraceArgs& a, uint32_t code, int64_t q) {
  return q < 0 ? 0u : __ldg(a.peq + (uint64_t)code * a.wpad + (uint64_t)q);
}

// Walks rows hi..lo+1 from column e; returns the exit column (at row lo); writes emitted symbols to out_chars.
// Requires hi a multiple of B and hi - lo a multiple of kWalkGroup (every segment but the last: H is a multiple of
// 8 B). The rows are taken in aligned groups of kWalkGroup: the bitmap words of a group's rows at one 32-column
// word lie at fixed offsets from one address (the fill's layout below), so the group's bitmap and match-mask words
// at the walk's current word are requested together, with one address computation; the symbol codes and symbols of
// the next group (code in bits 0-7, symbol in bits 8-15) are requested a group ahead. When the walk moves to
// another word inside the group (a diagonal step across the word's edge, or a LEFT run past it), the group's
// remaining rows are requested again at that word.
constexpr int kWalkGroup = 16;

template <int B>
__device__ uint64_t walk_segment(const TraceArgs& a, uint64_t hi, uint64_t lo, uint64_t e, uint8_t* out_chars,
                                 uint32_t* out_cnt) {
  constexpr int kG = kWalkGroup;
  constexpr uint32_t lb = B == 8 ? 3 : 4;
  static_assert(B == 8 || B == 16, "rows per step");
  uint64_t i = hi, j = e;
  uint32_t cnt = 0;
  const uint64_t wp = a.wpad;
  uint32_t cd[kG];  // code | symbol << 8 of the group's rows
#pragma unroll
  for (int k = 0; k < kG; ++k)
    cd[k] = i > lo + (uint64_t)k ? (uint32_t)a.xcode[i - k - 1] | (uint32_t)a.x[i - k - 1] << 8 : 0u;
  while (i > lo && j > 0) {
    uint32_t ncd[kG];
    const bool more = i > lo + kG;
#pragma unroll
    for (int k = 0; k < kG; ++k)
      ncd[k] = more ? (uint32_t)a.xcode[i - kG - k - 1] | (uint32_t)a.x[i - kG - k - 1] << 8 : 0u;
    const uint64_t rb0 = (i >> lb) - 1;  // the row-block of the group's first row, i - 1
    uint32_t done = 0;                   // rows of the group walked
    for (;;) {
      const uint64_t Qg = j >> 5;
      // t_word(i - k, Qg) = tp[off(k)]: row i - 1 - k is row B - 1 - k % B of row-block rb0 - k / B
      const uint32_t* tp = a.T + ((((Qg >> 5) * (a.R + 31) + rb0 + (Qg & 31)) << (5 + lb)) + (Qg & 31) * 4);
      const uint32_t* pp = a.peq + Qg;
      const uint32_t border = Qg ? kFull : ~1u;  // column 0 is the border
      uint32_t pm[kG], ev[kG];  // bit b: a match at column 32 Qg + b; a match or an UP cell there
#pragma unroll
      for (int k = 0; k < kG; ++k) {
        const int bk = B - 1 - (k % B);
        const int off = -((k / B) << (5 + lb)) + (bk >> 2) * 128 + (bk & 3);
        const uint32_t d = tp[off];
        const uint32_t* pr = pp + (uint64_t)(cd[k] & 0xFFu) * wp;
        const uint32_t pa = __ldg(pr), pb = Qg ? __ldg(pr - 1) : 0u;
        pm[k] = (pa << 1) | (pb >> 31);
        ev[k] = (pm[k] | ~d) & border;
      }
      bool again = false;  // the walk moved to another word: request the remaining rows there
#pragma unroll
      for (int k = 0; k < kG; ++k) {
        if (k < (int)done) continue;
        const uint32_t stop = ev[k] & (kFull >> (31u - (uint32_t)(j & 31)));  // columns 32 Qg .. j
        if (!stop) {  // a LEFT run past the word's first column: this row's scan goes on in the previous word
          if (Qg == 0) {
            j = 0;
          } else {
            j = (Qg << 5) - 1;
            again = true;
          }
          break;
        }
        const uint32_t bit = 31u - __clz(stop);
        const uint32_t mt = (pm[k] >> bit) & 1u;  // a match at column c: DIAG; else an UP cell: the walk goes up at c
        if (mt) out_chars[cnt++] = (uint8_t)(cd[k] >> 8);
        j = (Qg << 5) + bit - mt;
        done = (uint32_t)k + 1;
        if (j == 0) break;
        if ((j >> 5) != Qg) {
          again = true;
          break;
        }
      }
      if (!again || done == kG) break;
    }
    i -= kG;
#pragma unroll
    for (int k = 0; k < kG; ++k) cd[k] = ncd[k];
  }
  *out_cnt = cnt;
  return j;
}

// The same walk done by a whole warp (all lanes call it with the same arguments and follow the same path). Each
// round fetches the words of kWalkRounds * 32 rows at the walk's current 32-column word (lane k, slot r: row
// i - 32 r - k), so the loads of all those rows are in flight together. Most rows of a walk step UP at the walk's
// column without a match (nearly all of them for a tall pair, whose path is mostly vertical); such a row changes
// nothing but i. So the warp takes one ballot of "this row's cell at column j is a match or a LEFT cell" over the
// 32 rows of a slot and jumps straight to the first such row; only those rows are worked one by one (their words
// taken from their lane by shuffles). When the walk moves to another word it fetches again from that row. Lane 0
// writes the emitted symbols (when out_chars is not null).
constexpr int kWalkRounds = 4;

__device__ uint64_t walk_segment_warp(const TraceArgs& a, uint64_t hi, uint64_t lo, uint64_t e, uint8_t* out_chars,
                                      uint32_t* out_cnt) {
  const uint32_t lane = threadIdx.x & 31;
  uint64_t i = hi, j = e;
  uint32_t cnt = 0;
  while (i > lo && j > 0) {
    const int64_t Qg = (int64_t)(j >> 5);
    const uint64_t i0 = i;
    uint32_t cd[kWalkRounds], xs[kWalkRounds], dv[kWalkRounds], pm[kWalkRounds];
    bool okr[kWalkRounds];
#pragma unroll
    for (int r = 0; r < kWalkRounds; ++r) {
      const uint64_t off = 32ull * r + lane;  // this lane's row of slot r: i0 - off
      okr[r] = i0 > lo + off;
      cd[r] = okr[r] ? a.xcode[i0 - off - 1] : 0u;
      xs[r] = okr[r] ? a.x[i0 - off - 1] : 0u;
      dv[r] = okr[r] ? t_word(a, i0 - off, (uint64_t)Qg) : 0u;
    }
#pragma unroll
    for (int r = 0; r < kWalkRounds; ++r) {  // bit b of pm: a match at column 32 Qg + b
      const uint32_t pa = okr[r] ? p_word(a, cd[r], Qg) : 0u;
      const uint32_t pb = okr[r] ? p_word(a, cd[r], Qg - 1) : 0u;
      pm[r] = (pa << 1) | (pb >> 31);
    }
    bool leave = false;  // the walk ended, or left the fetched word (same value on every lane)
#pragma unroll
    for (int r = 0; r < kWalkRounds; ++r) {
      if (leave) break;
      // invariant: i = i0 - (32 r + k)
      for (uint32_t k = 0; k < 32;) {
        if (i <= lo || j == 0 || (int64_t)(j >> 5) != Qg) {
          leave = true;
          break;
        }
        const uint32_t bj = (uint32_t)(j & 31);
        // rows past the segment count as events too: the walk stops there
        const bool evl = !okr[r] || (((dv[r] | pm[r]) >> bj) & 1u);
        const uint32_t ev = __ballot_sync(kFull, evl) & (kFull << k);
        if (!ev) {  // every remaining row of the slot steps UP at column j
          i -= 32 - k;
          break;
        }
        const uint32_t kk = (uint32_t)__ffs(ev) - 1;
        i -= kk - k;
        k = kk;
        if (i <= lo) {
          leave = true;
          break;
        }
        const uint32_t code = __shfl_sync(kFull, cd[r], kk), sym = __shfl_sync(kFull, xs[r], kk);
        const uint32_t dk = __shfl_sync(kFull, dv[r], kk), pmk = __shfl_sync(kFull, pm[r], kk);
        if ((pmk >> bj) & 1u) {  // a match at column j: DIAG
          if (out_chars && lane == 0) out_chars[cnt] = (uint8_t)sym;
          ++cnt;
          --j;
        } else {  // a LEFT cell: the first column c < j with a match or an UP cell
          int64_t Q = Qg;
          uint32_t mask = kFull >> (31 - bj), d = dk, pq = pmk, stop = 0;
          for (;;) {
            stop = (pq | ~d) & mask;
            if (Q == 0) stop &= ~1u;  // column 0 is the border
            if (stop || Q == 0) break;
            --Q;
            mask = kFull;
            d = t_word(a, i, (uint64_t)Q);
            pq = (p_word(a, code, Q) << 1) | (p_word(a, code, Q - 1) >> 31);
          }
          if (!stop) {
            j = 0;
            leave = true;
            break;
          }
          const uint32_t bit = 31u - __clz(stop);
          const uint64_t c = ((uint64_t)Q << 5) + bit;
          if ((pq >> bit) & 1u) {
            if (out_chars && lane == 0) out_chars[cnt] = (uint8_t)sym;
            ++cnt;
            j = c - 1;
          } else {
            j = c;
          }
        }
        --i;
        ++k;
      }
    }
  }
  *out_cnt = cnt;
  return j;
}

// Column -> walker map: k_corr_cols writes, for every corridor column j it gives a walker k < W, k at cmap[s][j].
// The rest of the map is never cleared, so a lookup checks its answer: k names the walker entering at column e only
// when k is one of the segment's walkers and that walker's entry is e (the entries of a segment are distinct).
constexpr uint16_t kNoWalker = 0xFFFF;

__device__ __forceinline__ uint16_t map_lookup(const TraceArgs& a, uint64_t s, uint32_t c, uint32_t e) {
  const uint16_t k = a.cmap[s * (a.n + 1) + e];
  return (k < c && a.ent[s * a.W + k] == e) ? k : kNoWalker;
}

// The link of a walker of segment s with exit x: the walker of segment s - 1 whose entry is x, or kNoWalker (none of
// its walkers enters there: its corridor had more columns than walkers). The entries and counts of segments below
// the last are final once the corridor pass is done, so a walker finds its link right after its own walk.
__device__ __forceinline__ uint16_t walker_link(const TraceArgs& a, uint64_t s, uint32_t x) {
  if (s == 0) return kNoWalker;
  const uint32_t cntb = a.ent_cnt[s - 1], cb = cntb < a.W ? cntb : a.W;
  if (cb > kWalkers) return map_lookup(a, s - 1, cb, x);
  uint32_t hit = 0;  // the (at most 32) entries are loaded together, then the first equal one is taken
#pragma unroll
  for (uint32_t kk = 0; kk < kWalkers; ++kk)
    if (kk < cb && a.ent[(s - 1) * a.W + kk] == x) hit |= 1u << kk;
  return hit ? (uint16_t)(__ffs(hit) - 1) : kNoWalker;
}

// The same for a whole warp (all lanes, the same x): lane kk compares entry kk of a narrow segment below.
__device__ __forceinline__ uint16_t walker_link_warp(const TraceArgs& a, uint64_t s, uint32_t x, uint32_t lane) {
  if (s == 0) return kNoWalker;
  const uint32_t cntb = a.ent_cnt[s - 1], cb = cntb < a.W ? cntb : a.W;
  if (cb > kWalkers) return map_lookup(a, s - 1, cb, x);
  const uint32_t b = __ballot_sync(kFull, lane < cb && a.ent[(s - 1) * a.W + lane] == x);
  return b ? (uint16_t)(__ffs(b) - 1) : kNoWalker;
}

// Walkers of segment s. A segment whose corridor has at most gridDim.y columns (the usual case for pairs of similar
// length) gives each walker a whole warp: block (s, k) walks from the k-th corridor column with
// walk_segment_warp, whose lanes fetch 32 rows at a time and follow one path, so a row costs a few dependent
// instructions and no divergence. A wider corridor (tall pairs, hundreds of columns) runs one walker per thread:
// block (s, y), thread t walks from column y * 32 + t (such a segment is never the last, so its rows hi..lo+1 are
// aligned as walk_segment requires). The last segment has one walker, from (m, n); it records that entry for the
// chain pass.
__global__ void k_walk(TraceArgs a) {
  const uint64_t s = blockIdx.x;
  const bool last = s + 1 == a.S;
  const uint32_t found = last ? 1u : a.ent_cnt[s];
  const uint32_t cnt = found < a.W ? found : a.W;
  const uint64_t lo = s * a.H, hi = (s + 1) * a.H < a.m ? (s + 1) * a.H : a.m;
  if (cnt <= gridDim.y) {  // a warp per walker
    const uint32_t k = blockIdx.y;
    if (k >= cnt) return;
    const uint64_t e = last ? a.n : a.ent[s * a.W + k];
    uint32_t nc = 0;
    const uint64_t x = walk_segment_warp(a, hi, lo, e, a.chars + (s * (a.W + 1) + k) * a.H, &nc);
    const uint16_t l = walker_link_warp(a, s, (uint32_t)x, threadIdx.x);
    if (threadIdx.x == 0) {
      if (last) {
        a.ent[s * a.W] = (uint32_t)a.n;
        a.ent_cnt[s] = 1;
      }
      a.ext[s * a.W + k] = (uint32_t)x;
      a.nch[s * a.W + k] = nc;
      a.link[s * a.W + k] = l;
    }
    return;
  }
  const uint32_t k = blockIdx.y * kWalkers + threadIdx.x;  // a thread per walker
  if (k >= cnt) return;
  const uint64_t e = a.ent[s * a.W + k];
  uint32_t nc = 0;
  uint8_t* out = a.chars + (s * (a.W + 1) + k) * a.H;
  const uint64_t x = a.B == 8 ? walk_segment<8>(a, hi, lo, e, out, &nc) : walk_segment<16>(a, hi, lo, e, out, &nc);
  a.ext[s * a.W + k] = (uint32_t)x;
  a.nch[s * a.W + k] = nc;
  a.link[s * a.W + k] = walker_link(a, s, (uint32_t)x);
}

// Follows the true path from (m, n) down the segments: warp 0 follows the walkers' links (k_walk), the first 32 of
// every segment staged in shared memory, from segment S - 1's walker (it starts at (m, n)); where a link is missing
// (the entry is not among the segment's W walkers: more corridor columns than walkers) the warp walks that segment
// itself and looks its exit up among the next segment's walkers, until the path meets a walker again.
constexpr uint32_t kChainThreads = 256;

__device__ __forceinline__ bool chain_lookup(const TraceArgs& a, const uint32_t* ent32, const uint32_t* cnt,
                                             uint64_t s, uint32_t e, uint32_t lane, uint32_t* k_out) {
  const uint32_t c = cnt[s] < a.W ? cnt[s] : a.W;
  if (c <= kWalkers) {
    const bool hit = lane < c && ent32[s * kWalkers + lane] == e;
    const uint32_t b = __ballot_sync(kFull, hit);
    *k_out = b ? (uint32_t)__ffs(b) - 1 : 0u;
    return b != 0;
  }
  const uint16_t k = map_lookup(a, s, c, e);
  *k_out = k;
  return k != kNoWalker;
}

// Shared memory of k_chain: ent32 [S][32] and cnt [S] (words), then link32 [S][32] (16-bit) from a 16-byte boundary.
__host__ __device__ constexpr uint64_t chain_link_offset(uint64_t S) { return (S * kWalkers + S + 3) & ~(uint64_t)3; }

__global__ void __launch_bounds__(kChainThreads) k_chain(TraceArgs a) {
  extern __shared__ uint32_t sm[];
  uint32_t* ent32 = sm;                   // [S][kWalkers]: the first 32 entries of every segment
  uint32_t* cnt = sm + a.S * kWalkers;    // [S]
  uint16_t* link32 = reinterpret_cast<uint16_t*>(sm + chain_link_offset(a.S));  // [S][kWalkers]
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  const uint32_t S = (uint32_t)a.S, W = a.W;
#pragma unroll 8
  for (uint32_t i = tid; i < S * kWalkers; i += kChainThreads) {  // the loads of 8 rounds in flight together
    const uint64_t src = (uint64_t)(i / kWalkers) * W + (i % kWalkers);
    ent32[i] = a.ent[src];
    link32[i] = a.link[src];
  }
  for (uint32_t i = tid; i < S; i += kChainThreads) cnt[i] = a.ent_cnt[i];
  __shared__ int32_t stop_s;
  __shared__ uint32_t stop_k;
  __syncthreads();
  if (tid == 0) {  // thread 0 follows the links from segment S-1's walker (it starts at (m, n)) as far as they go
    int64_t s0 = (int64_t)a.S - 1;
    uint32_t k0 = 0;
    stop_s = -1;
    for (;;) {
      a.sel[s0] = k0;
      if (s0 == 0) break;
      const uint16_t nk = k0 < kWalkers ? link32[s0 * kWalkers + k0] : a.link[s0 * a.W + k0];
      if (nk == kNoWalker) {
        stop_s = (int32_t)s0;
        stop_k = k0;
        break;
      }
      k0 = nk;
      --s0;
    }
  }
  __syncthreads();
  if (tid >= 32 || stop_s < 0) return;
  // warp 0 from the first missing link on
  int64_t s = stop_s;
  uint32_t k = stop_k;
  for (;;) {
    if (lane == 0) a.sel[s] = k;
    if (s == 0) break;
    const uint16_t nk = k < kWalkers ? link32[s * kWalkers + k] : a.link[s * a.W + k];
    if (nk != kNoWalker) {
      k = nk;
      --s;
      continue;
    }
    // no walker of segment s - 1 enters at this exit: walk segments here until the path meets a walker again
    uint64_t e = a.ext[s * a.W + k];
    bool met = false;
    while (!met) {
      --s;
      const uint64_t lo = (uint64_t)s * a.H, hi = ((uint64_t)s + 1) * a.H < a.m ? ((uint64_t)s + 1) * a.H : a.m;
      uint32_t nc = 0;
      e = walk_segment_warp(a, hi, lo, e, a.chars + ((uint64_t)s * (a.W + 1) + a.W) * a.H, &nc);
      if (lane == 0) {
        a.sel[s] = a.W;
        a.ent_cnt[s] = 0x80000000u | nc;  // fallback count, read by k_finalize
      }
      if (s == 0) return;
      met = chain_lookup(a, ent32, cnt, (uint64_t)(s - 1), (uint32_t)e, lane, &k);
    }
    --s;  // the walker k of segment s (now s - 1 of the walked one) continues the path
  }
}

__device__ __forceinline__ uint32_t seg_count(const TraceArgs& a, uint64_t s) {
  const uint32_t k = a.sel[s];
  if (k == a.W) return a.ent_cnt[s] & 0x7FFFFFFFu;
  return a.nch[s * a.W + k];
}

// Block s copies its selected walker's symbols (walk order = reverse output order) to their place in the output.
__global__ void k_finalize(TraceArgs a) {
  __shared__ uint32_t red[32];
  const uint64_t s = blockIdx.x;
  uint32_t before = 0, total = 0;
  for (uint64_t t = threadIdx.x; t < a.S; t += blockDim.x) {
    const uint32_t c = seg_count(a, t);
    total += c;
    if (t < s) before += c;
  }
  before = __reduce_add_sync(kFull, before);
  total = __reduce_add_sync(kFull, total);
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = before;
    red[16 + (threadIdx.x >> 5)] = total;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t b = 0, tt = 0;
    for (uint32_t w = 0; w < blockDim.x / 32; ++w) {
      b += red[w];
      tt += red[16 + w];
    }
    red[0] = b;
    red[16] = tt;
  }
  __syncthreads();
  before = red[0];
  total = red[16];
  const uint32_t k = a.sel[s];
  const uint32_t c = seg_count(a, s);
  const uint8_t* src = a.chars + (s * (a.W + 1) + k) * a.H;
  const bool fits = (uint64_t)before + c <= a.out_cap;  // always true unless the walks were inconsistent
  if (fits)
    for (uint32_t t = threadIdx.x; t < c; t += blockDim.x) a.out[before + c - 1 - t] = src[t];
  if (threadIdx.x == 0 && (!fits || (s == 0 && (unsigned long long)total != *a.L)))
    atomicOr(&a.status->flags, kStatInternal);
  if (s == 0 && threadIdx.x == 0) *a.out_len = total;
}

// ---- the full tables c and b of LCS-length (§I.C) from the forward bitmap ----------------------------------------
// c[i,j] = c[i-1,j] + dv(i,j), where dv(i,j) = c[i,j] - c[i-1,j] is bit j % 32 of T-frame word j / 32 of row i
// (column 0 reads 0). Rows are cut into chunks of kTabChunk rows: the chunk sums of dv per column, their exclusive
// prefix over the chunks (the value of c at each chunk's top row), then every chunk expanded row by row. b[i,j] is
// DIAG when x_i = y_j, else UP when dv(i,j) = 0 (c[i-1,j] >= c[i,j-1]) and LEFT when it is 1.
constexpr uint32_t kTabChunk = 64;

__device__ __forceinline__ uint32_t dv_bit(const TraceArgs& a, uint64_t i, uint64_t j) {
  return (t_word(a, i, j >> 5) >> (j & 31)) & 1u;
}

__global__ void k_tab_sum(TraceArgs a, uint32_t* sums) {
  const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t k = blockIdx.y;
  if (j > a.n) return;
  const uint64_t i0 = k * kTabChunk + 1, i1 = i0 + kTabChunk <= a.m + 1 ? i0 + kTabChunk : a.m + 1;
  uint32_t s = 0;
  for (uint64_t i = i0; i < i1; ++i) s += dv_bit(a, i, j);
  sums[k * (a.n + 1) + j] = s;
}

__global__ void k_tab_scan(uint64_t n, uint64_t chunks, uint32_t* sums) {
  const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j > n) return;
  uint32_t run = 0;
  for (uint64_t k = 0; k < chunks; ++k) {
    const uint32_t t = sums[k * (n + 1) + j];
    sums[k * (n + 1) + j] = run;
    run += t;
  }
}

__global__ void k_tab_expand(TraceArgs a, const uint8_t* y, const uint32_t* sums, uint32_t* c, uint8_t* b) {
  const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t k = blockIdx.y;
  if (j > a.n) return;
  const uint64_t w = a.n + 1;
  if (k == 0) c[j] = 0;  // row 0
  const uint64_t i0 = k * kTabChunk + 1, i1 = i0 + kTabChunk <= a.m + 1 ? i0 + kTabChunk : a.m + 1;
  const uint32_t yj = j > 0 ? y[j - 1] : 0u;
  uint32_t cc = sums[k * w + j];
  for (uint64_t i = i0; i < i1; ++i) {
    const uint32_t d = dv_bit(a, i, j);
    cc += d;
    c[i * w + j] = cc;
    if (j > 0) b[(i - 1) * a.n + (j - 1)] = a.x[i - 1] == yj ? 1u : (d ? 3u : 2u);
  }
}

std::atomic<uint64_t> chain_attr_done{0};

}  // namespace

cudaError_t launch_combine(const uint32_t* vf, const uint32_t* vr, uint64_t n, uint64_t w, uint32_t* colsum,
                           unsigned long long* out_len, cudaStream_t st) {
  if (w <= kCombineOneBlockWords) {  // one launch: the block keeps both prefix arrays in shared memory
    k_combine_small<<<1, 1024, 0, st>>>(vf, vr, n, w, out_len);
    return cudaGetLastError();
  }
  k_combine_pre<<<2, 1024, 0, st>>>(vf, vr, w, colsum);
  uint64_t blocks = (n + 1 + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  k_combine_min<<<(unsigned)blocks, 256, 0, st>>>(vf, vr, n, w, colsum);
  k_combine_fin<<<1, 1, 0, st>>>(colsum, n, w, out_len);
  return cudaGetLastError();
}

// The corridor counts ent_cnt must be zero on entry (the caller clears them with the row offsets).
cudaError_t launch_traceback(const TraceArgs& a, cudaStream_t st) {
  if (a.S > 1) {
    k_corr_pre<<<(unsigned)(a.S - 1), 1024, 0, st>>>(a);
    const uint64_t gx = (a.n / 32 + 1 + 127) / 128;  // one thread per 32-column word
    k_corr_cols<<<dim3((unsigned)gx, (unsigned)(a.S - 1)), 128, 0, st>>>(a);
  }
  // gridDim.y: enough blocks for W walkers of a thread each, and at least kWarpWalkers (a warp per walker)
  const unsigned walk_y = (unsigned)std::max<uint64_t>(a.W / kWalkers, kWarpWalkers);
  k_walk<<<dim3((unsigned)a.S, walk_y), kWalkers, 0, st>>>(a);
  const size_t chain_smem = (size_t)chain_link_offset(a.S) * sizeof(uint32_t) + a.S * kWalkers * sizeof(uint16_t);
  cudaError_t e = once_per_device_attr(
      [] {
        return cudaFuncSetAttribute(
            k_chain, cudaFuncAttributeMaxDynamicSharedMemorySize,
            (int)(chain_link_offset(kMaxSegments) * sizeof(uint32_t) + kMaxSegments * kWalkers * sizeof(uint16_t)));
      },
      chain_attr_done);
  if (e != cudaSuccess) return e;
  k_chain<<<1, kChainThreads, chain_smem, st>>>(a);
  k_finalize<<<(unsigned)a.S, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_tables(const TraceArgs& a, const uint8_t* y, uint32_t* sums, uint32_t* c, uint8_t* b,
                          cudaStream_t st) {
  const uint64_t chunks = (a.m + kTabChunk - 1) / kTabChunk;
  const unsigned gx = (unsigned)((a.n + 1 + 255) / 256);
  k_tab_sum<<<dim3(gx, (unsigned)chunks), 256, 0, st>>>(a, sums);
  k_tab_scan<<<gx, 256, 0, st>>>(a.n, chunks, sums);
  k_tab_expand<<<dim3(gx, (unsigned)chunks), 256, 0, st>>>(a, y, sums, c, b);
  return cudaGetLastError();
}

uint64_t tables_sum_words(uint64_t m, uint64_t n) { return ((m + kTabChunk - 1) / kTabChunk) * (n + 1); }

}  // namespace lcs
