// The LCS table fill (paper §I.C, LCS-length) as a bit-parallel row update on a systolic wavefront.
//
// Row i of the table is represented by the vector V of "no horizontal increase" bits: bit (j-1) of V is
// 1 - (c[i,j] - c[i,j-1]), packed 32 columns per 32-bit word. With P = the match mask of x_i over Y,
//     U = V & P;   S = V + U (one multi-word add, no carry into column 1);   V' = S | (V & ~P)
// turns row i-1 into row i. The carry that leaves column j during the add is c[i,j] - c[i-1,j], so the
// carry-into vector T = S ^ V ^ U of every word is exactly the information that table b of the paper keeps on a
// mismatch (UP when that difference is 0, LEFT when it is 1; a match is always DIAG), at one bit per cell. This
// follows from the recurrence of §I.B-C: with a = c[i-1,j-1], h = c[i-1,j] - a, v = c[i,j-1] - a and M = [x_i = y_j],
// c[i,j] = a + (M | h | v), so c[i,j] - c[i-1,j] = (M | v) & ~h and c[i,j] - c[i,j-1] = (M | h) & ~v; the ripple
// carry of the add computes the first, and the sum bit OR (V & ~P) the complement of the second.
//
// Parallel layout (replaces the paper's split of the table into stripes over 4 OpenMP threads, §II-II.B):
//   * every lane owns one word (32 columns) and keeps V in a register for all m rows;
//   * lanes form a systolic chain along the row: lane l works on row-block r = t - l at step t (B rows per
//     step), takes the B carry bits entering its word from lane l-1 (shuffle), and passes its own B carry-out
//     bits to lane l+1 one step later;
//   * warp w+1 continues the chain of warp w through a shared-memory ring, block b+1 that of block b through
//     self-validating global slots (data bits + a row-block tag, so no separate flag or fence is needed);
//   * all blocks are co-resident (cooperative launch), one block of 4 warps per SM;
//   * every wait is bounded: when it expires the kernel records a timeout in the status word and runs to the end
//     without waiting, so the host gets LCS_ERR_TIMEOUT instead of a hung GPU.
#include <algorithm>

#include "lcs_internal.h"

namespace lcs {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Predicated relaxed store (no branch around it): stores only when pred != 0.
__device__ __forceinline__ void st_relaxed_gpu_if(uint32_t* p, uint32_t v, uint32_t pred) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.relaxed.gpu.global.u32 [%0], %1;\n\t}" ::"l"(p), "r"(v),
      "r"(pred)
      : "memory");
}
// Predicated plain store (no branch around it): stores only when pred != 0.
__device__ __forceinline__ void st_global_if(uint32_t* p, uint32_t v, uint32_t pred) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.u32 [%0], %1;\n\t}" ::"l"(p), "r"(v), "r"(pred)
               : "memory");
}
__device__ __forceinline__ uint32_t lds_vol_u32(uint32_t saddr) {
  uint32_t v;
  asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(v) : "r"(saddr) : "memory");
  return v;
}
__device__ __forceinline__ void sts_vol_u32(uint32_t saddr, uint32_t v) {
  asm volatile("st.volatile.shared.u32 [%0], %1;" ::"r"(saddr), "r"(v) : "memory");
}
__device__ __forceinline__ void sts_vol_u32_if(uint32_t saddr, uint32_t v, uint32_t pred) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.volatile.shared.u32 [%0], %1;\n\t}" ::"r"(saddr),
               "r"(v), "r"(pred)
               : "memory");
}

// Bounded waits. A wait that gives up (its own timeout, or the abort flag raised after another warp's timeout)
// records the timeout in the status word; the warp then stops waiting for the rest of the launch.
__device__ __forceinline__ bool give_up(DevStatus* st, uint32_t it, uint32_t limit, uint32_t where) {
  if (*(volatile uint32_t*)&st->abort) return true;
  if (it >= limit) {
    atomicOr(&st->flags, kStatTimeout);
    atomicExch(&st->where, where);
    atomicExch(&st->abort, 1u);
    return true;
  }
  return false;
}

// Waits (all lanes together) until the consumer of a shared-memory ring has consumed row-blocks below `need`.
__device__ __noinline__ bool spin_ring_space(uint32_t cons_saddr, uint32_t need, DevStatus* st, uint32_t limit) {
  for (uint32_t it = 0;; ++it) {
    const uint32_t c = lds_vol_u32(cons_saddr);
    if ((int32_t)(c - need) >= 0) return true;
    if ((it & 63u) == 63u && give_up(st, it, limit, 3u)) return false;
    __nanosleep(32);
  }
}

template <int B>
__device__ __forceinline__ void load_xo(const uint4* p, uint32_t (&dst)[B]) {
#pragma unroll
  for (int v = 0; v < B / 4; ++v) {
    const uint4 q4 = __ldg(p + v);
    dst[4 * v + 0] = q4.x;
    dst[4 * v + 1] = q4.y;
    dst[4 * v + 2] = q4.z;
    dst[4 * v + 3] = q4.w;
  }
}

// Where a warp's inbound carries come from and where its outbound carries go.
enum : int { kSrcNone = 0, kSrcGlobal = 1, kSrcRing = 2 };
enum : int { kDstNone = 0, kDstGlobal = 1, kDstRing = 2 };

// Constants of one warp.
struct Warp {
  uint32_t peq_lane;   // shared-memory address of this lane's column of the match masks
  uint32_t ring_src;   // shared-memory ring read by lane 0 (row-block r at slot r % kRing)
  uint32_t ring_dst;   // shared-memory ring written by lane 31
  uint32_t cons_self;  // this warp's consumption counter (read by the producer for back-pressure)
  uint32_t cons_next;  // the next warp's consumption counter
  uint32_t xring;     // shared-memory ring of symbol offsets: row-block rb at slot rb % 64 (B words each)
  const uint4* xring_p;  // the same ring, laid out [B/4][64 slots] of 16-byte vectors (bank-conflict free)
  const uint32_t* peq_p;  // this lane's column of the match masks (row s at peq_p[s * kStripeWords])
  const uint32_t* xoff;  // global symbol offsets: row-block rb at xoff + (rb + kPadRowblocks) * B
  const uint32_t* src_g;
  uint32_t* dst_g;
  DevStatus* status;
  uint32_t* snap;     // snapshot rows [k][wpad] (k = (r + 1) / snap_rb - 1), this lane's column
  uint64_t wpad;
  int32_t R;
  uint32_t lane, snap_rb, spin_limit;
  uint32_t cap_k;     // step (mod 32) at which this lane finishes a row-block r with (r + 1) % 32 == 0
  uint32_t hands_on;  // 1 for the lane that hands the warp's carries on (lane 31)
};

// Loop state of one lane, kept in registers across the unrolled steps.
struct Lane {
  uint32_t V;         // the lane's word of the current row vector
  uint32_t cout;      // carry bits produced in the last step (row 0 of the block at bit 31)
  uint32_t cin_a;     // carries for rows 0 .. B/2-1 of this step from lane-1 (top bits), received last step
  uint32_t cin_b;     // carries for rows B/2 .. B-1
  uint32_t win;       // inbound window of the current 32-step block t0 .. t0+31: slot t0 + lane
  uint32_t win_next;  // the next block's window, requested in the middle of the current block
  uint32_t cin0;      // the previous warp's carries for this step's row-block (lane 0's input), taken from the
                      // window one step ahead, or right after a validation at a window or group start
  uint32_t cap;       // V captured at the end of this lane's row-block r with (r + 1) % 32 == 0 in this block
  uint32_t xstage[16];  // symbol offsets of row-block t0 + 34 + lane, staged for the next 32-step boundary
  int32_t nsnap;      // dense snapshots: the next row-block whose end row is snapshotted, and where its word goes
  uint32_t* snp;
  uint4* tp;          // this step's bitmap chunk of the warp, plus this lane's offset
  bool failed;
};

// One row of the update: U = V & P; S = V + U + (carry bit at the top of cw); V' = S | (V & ~P); the carry out of
// the word is shifted into co; T (the carries into every bit) is kept in traceback mode.
template <bool TB>
__device__ __forceinline__ void row1(uint32_t P, uint32_t& V, uint32_t& cw, uint32_t& co, uint32_t& tw) {
  const uint32_t U = V & P;
  uint32_t S;
  asm("add.cc.u32 %0, %0, %0;\n\t"
      "addc.cc.u32 %1, %3, %4;\n\t"
      "addc.u32 %2, %2, %2;"
      : "+r"(cw), "=r"(S), "+r"(co)
      : "r"(V), "r"(U));
  if (TB) tw = S ^ V ^ U;
  V = S | (V & ~P);
}

// The B rows of one step. The carries entering the word come in two halves (rows 0 .. B/2-1 in cin_a, the rest in
// cin_b, each at the top bits); the carries leaving it go to lane+1 in two halves as well, the first right after
// row B/2-1, so that lane+1 has them long before its next step needs them and no shuffle latency sits on the chain
// of rows. Returns the full B carry-out bits (row 0 at bit B-1) in co.
template <int B, bool TB>
__device__ __forceinline__ void rows(const uint32_t (&P)[B], uint32_t& V, uint32_t cin_a, uint32_t cin_b,
                                     uint32_t& co, uint32_t& send_a, uint32_t& send_b, uint32_t (&tw)[B]) {
  constexpr int H = B / 2;
  uint32_t cw = cin_a;
  co = 0;
#pragma unroll
  for (int b = 0; b < H; ++b) row1<TB>(P[b], V, cw, co, tw[b]);
  send_a = __shfl_up_sync(kFull, co << (32 - H), 1);
  cw = cin_b;
#pragma unroll
  for (int b = H; b < B; ++b) row1<TB>(P[b], V, cw, co, tw[b]);
  send_b = __shfl_up_sync(kFull, co << (32 - H), 1);
}

// Symbol offsets of row-block rb from the warp's shared ring (B words). The ring is laid out [B/4][64] in 16-byte
// vectors, so the 32 lanes (consecutive row-blocks) read 32 consecutive vectors: no bank conflicts.
template <int B>
__device__ __forceinline__ void xo_from_ring(const Warp& w, int32_t rb, uint32_t (&dst)[B]) {
  const uint32_t slot = (uint32_t)rb & 63u;
#pragma unroll
  for (int v = 0; v < B / 4; ++v) {
    const uint4 q = w.xring_p[v * 64 + slot];
    dst[4 * v] = q.x;
    dst[4 * v + 1] = q.y;
    dst[4 * v + 2] = q.z;
    dst[4 * v + 3] = q.w;
  }
}

// Match masks of the B rows whose symbol offsets are xo (in words), for this lane's word.
template <int B>
__device__ __forceinline__ void p_from_offsets(const Warp& w, const uint32_t (&xo)[B], uint32_t (&P)[B]) {
#pragma unroll
  for (int b = 0; b < B; ++b) P[b] = w.peq_p[xo[b]];
}

// One step of one warp: lane l updates its word over the B rows of row-block r = t - l, with the match masks pu
// loaded during the previous step. During this step it loads the next step's match masks (from the offsets xa it
// already holds) and the offsets of the step after that, so no step waits on a load. Lane 0 takes the previous
// warp's carries from the block's window (validated once per block), lane 31 hands its own on; the step has no
// branches.
template <int B, bool TB, bool SNAP, bool DS, int SRC, int DST>
__device__ __forceinline__ void fill_step(const Warp& w, Lane& s, int32_t t, const uint32_t (&pu)[B],
                                          const uint32_t (&xa)[B], uint32_t (&pl)[B], uint32_t (&xl)[B]) {
  constexpr uint32_t kTagMask = (1u << (32 - B)) - 1u;
  const uint32_t lane = w.lane;
  const int32_t r = t - (int32_t)lane;
  p_from_offsets<B>(w, xa, pl);
  xo_from_ring<B>(w, r + 2, xl);
  uint32_t cin0 = 0;
  if (SRC != kSrcNone) {  // slot t was read one step ago; read slot t + 1 now, off the path of this step's rows
    cin0 = s.cin0;
    const uint32_t nx = __shfl_sync(kFull, s.win, (t + 1) & 31);
    s.cin0 = t + 1 < w.R ? (nx & ~kTagMask) : 0u;
  }
  // lane 0 takes the previous warp's carries (rows 0 .. B/2-1 at the top of cin0, then the rest)
  const uint32_t cin_a = lane == 0 ? cin0 : s.cin_a;
  const uint32_t cin_b = lane == 0 ? (cin0 << (B / 2)) : s.cin_b;
  uint32_t co, V = s.V;
  uint32_t tw[B];
  rows<B, TB>(pu, V, cin_a, cin_b, co, s.cin_a, s.cin_b, tw);
  s.V = V;
  s.cout = co << (32 - B);
  if (TB) {
#pragma unroll
    for (int v = 0; v < B / 4; ++v) s.tp[v * 32] = make_uint4(tw[4 * v], tw[4 * v + 1], tw[4 * v + 2], tw[4 * v + 3]);
    s.tp += 8 * B;  // 32 lanes x B words = 8 * B uint4 per step
  }
  if (SNAP && !DS) s.cap = (((uint32_t)t & 31u) == w.cap_k) ? V : s.cap;
  if (SNAP && DS) {  // dense: every snapshotted row-block's word stored as it ends (predicated, no branch)
    const uint32_t hit = (r == s.nsnap) & (r < w.R);
    st_global_if(s.snp, V, hit);
    s.snp += hit ? w.wpad : 0u;
    s.nsnap += hit ? (int32_t)w.snap_rb : 0;
  }
  if (DST != kDstNone) {  // lane 31 hands its carries for row-block t - 31 to the next warp
    const uint32_t r31 = (uint32_t)(t - 31);
    const uint32_t v = s.cout | ((r31 + 1u) | 1u) & kTagMask;
    const uint32_t pred = w.hands_on & (t >= 31);
    if (DST == kDstGlobal) st_relaxed_gpu_if(w.dst_g + (int64_t)t - 31, v, pred);
    else sts_vol_u32_if(w.ring_dst + (r31 & (kRing - 1)) * 4u, v, pred);
  }
}

// Loads the symbol offsets of row-block rb (B words) from global memory into registers.
template <int B>
__device__ __forceinline__ void xo_load_global(const Warp& w, int32_t rb, uint32_t* dst) {
  const uint4* p = reinterpret_cast<const uint4*>(w.xoff + (int64_t)(rb + kPadRowblocks) * B);
#pragma unroll
  for (int v = 0; v < B / 4; ++v) {
    const uint4 q = __ldg(p + v);
    dst[4 * v] = q.x;
    dst[4 * v + 1] = q.y;
    dst[4 * v + 2] = q.z;
    dst[4 * v + 3] = q.w;
  }
}
template <int B>
__device__ __forceinline__ void xo_store_ring(const Warp& w, int32_t rb, const uint32_t* src) {
  uint4* ring = const_cast<uint4*>(w.xring_p);
  const uint32_t slot = (uint32_t)rb & 63u;
#pragma unroll
  for (int v = 0; v < B / 4; ++v) ring[v * 64 + slot] = make_uint4(src[4 * v], src[4 * v + 1], src[4 * v + 2], src[4 * v + 3]);
}

// Refill of the symbol-offset ring at a 32-step boundary t0: during steps t0 .. t0+31 the lanes read row-blocks
// t0-29 .. t0+33 (two steps ahead); the 64-slot ring holds t0-30 .. t0+33 after this refill. Row-blocks t0+2 ..
// t0+33 were loaded into registers at the previous boundary; the next 32 are requested now, stored 32 steps later.
template <int B>
__device__ __forceinline__ void xo_refill(const Warp& w, Lane& s, int32_t t0) {
  __syncwarp();
  xo_store_ring<B>(w, t0 + 2 + (int32_t)w.lane, s.xstage);
  __syncwarp();
  xo_load_global<B>(w, t0 + 34 + (int32_t)w.lane, s.xstage);
}

// After the 32-step block starting at t0 (or the shorter last block ending at `end`): store the captured V when its
// row-block r = t0 + cap_k - lane is one whose end row is snapshotted, (r + 1) % snap_rb == 0.
__device__ __forceinline__ void snap_store(const Warp& w, const Lane& s, int32_t t0, int32_t end) {
  const int32_t r = t0 + (int32_t)w.cap_k - (int32_t)w.lane;
  if (t0 + (int32_t)w.cap_k < end && r >= 0 && r < w.R && ((uint32_t)(r + 1) % w.snap_rb) == 0)
    w.snap[(uint64_t)((uint32_t)(r + 1) / w.snap_rb - 1) * w.wpad] = s.cap;
}

// Inbound window slot q (lane-specific) from the previous warp: global slots or the shared ring.
template <int SRC>
__device__ __forceinline__ uint32_t window_load(const Warp& w, int32_t q) {
  if (SRC == kSrcGlobal) return q < w.R ? ld_relaxed_gpu(w.src_g + q) : 0u;
  return lds_vol_u32(w.ring_src + ((uint32_t)q & (kRing - 1)) * 4u);
}

// The previous warp's carries for row-block t from the (validated) window.
template <int B>
__device__ __forceinline__ void take_cin0(const Warp& w, Lane& s, int32_t t) {
  constexpr uint32_t kTagMask = (1u << (32 - B)) - 1u;
  const uint32_t src = __shfl_sync(kFull, s.win, t & 31);
  s.cin0 = t < w.R ? (src & ~kTagMask) : 0u;
}

// Start of a VG-step group at t (t % VG == 0) for a warp fed by a shared-memory ring: lanes t%32 .. t%32+VG-1 of
// the window load the group's VG slots and the warp waits until all of them have arrived (bounded). A group only
// needs the producer VG + 31 steps ahead, so neighbouring warps in a block run close together.
template <int B, int SRC, int VG>
__device__ __forceinline__ void ring_group_wait(const Warp& w, Lane& s, int32_t t) {
  constexpr uint32_t kTagMask = (1u << (32 - B)) - 1u;
  constexpr uint32_t kSel = 32u - VG;  // lane bits that select the group
  const uint32_t lane = w.lane;
  const bool mine = (lane & kSel) == ((uint32_t)t & kSel);
  const int32_t q = (t & ~31) + (int32_t)lane;
  const uint32_t want = ((uint32_t)(q + 1) | 1u) & kTagMask;
  if (mine) s.win = q < w.R ? lds_vol_u32(w.ring_src + ((uint32_t)q & (kRing - 1)) * 4u) : 0u;
  bool ok = !mine || q >= w.R || (s.win & kTagMask) == want;
  if (__all_sync(kFull, ok) || s.failed) return;
  for (uint32_t it = 0;; ++it) {
    if (!ok) {
      s.win = lds_vol_u32(w.ring_src + ((uint32_t)q & (kRing - 1)) * 4u);
      ok = (s.win & kTagMask) == want;
    }
    if (__all_sync(kFull, ok)) return;
    if ((it & 63u) == 63u) {
      const bool quit = __any_sync(kFull, give_up(w.status, it, w.spin_limit, 2u));
      if (quit) {
        s.failed = true;
        return;
      }
    }
    __nanosleep(32);
  }
}

template <int B, int SRC, int VG>
__device__ __forceinline__ void ring_group_validate(const Warp& w, Lane& s, int32_t t) {
  if (SRC != kSrcRing) return;
  ring_group_wait<B, SRC, VG>(w, s, t);
  take_cin0<B>(w, s, t);
}

// Start of the 32-step block t0 for a warp fed by global slots: switch to the window requested in the middle of the
// last block and make sure every slot this block needs has arrived (all lanes together; a bounded wait in the rare
// case one has not).
template <int B, int SRC>
__device__ __forceinline__ void window_wait(const Warp& w, Lane& s, int32_t t0, bool first) {
  constexpr uint32_t kTagMask = (1u << (32 - B)) - 1u;
  if (!first) s.win = s.win_next;
  const int32_t q = t0 + (int32_t)w.lane;
  const uint32_t want = ((uint32_t)(q + 1) | 1u) & kTagMask;
  bool ok = q >= w.R || (s.win & kTagMask) == want;
  if (__all_sync(kFull, ok) || s.failed) return;
  for (uint32_t it = 0;; ++it) {
    if (!ok) {
      s.win = window_load<SRC>(w, q);
      ok = (s.win & kTagMask) == want;
    }
    if (__all_sync(kFull, ok)) return;
    if ((it & 63u) == 63u) {
      const bool quit = __any_sync(kFull, give_up(w.status, it, w.spin_limit, SRC == kSrcGlobal ? 1u : 2u));
      if (quit) {
        s.failed = true;
        return;
      }
    }
    __nanosleep(32);
  }
}

template <int B, int SRC>
__device__ __forceinline__ void window_validate(const Warp& w, Lane& s, int32_t t0, bool first) {
  if (SRC != kSrcGlobal) return;
  window_wait<B, SRC>(w, s, t0, first);
  take_cin0<B>(w, s, t0);
}

// Work at the start of each 32-step block: publish consumption, honour ring back-pressure.
template <int SRC, int DST>
__device__ __forceinline__ void block_start(const Warp& w, Lane& s, int32_t t) {
  if (SRC == kSrcRing) sts_vol_u32(w.cons_self, (uint32_t)t);  // all lanes write the same value
  if (DST == kDstRing && !s.failed) {
    // this block writes row-blocks up to t; they overwrite slot r - kRing, which must be consumed
    const uint32_t need = (uint32_t)(t - (kRing - 64));
    if (t >= kRing - 64 && (int32_t)(lds_vol_u32(w.cons_next) - need) < 0)
      s.failed = !spin_ring_space(w.cons_next, need, w.status, w.spin_limit);
  }
}

template <int B, bool TB, int VG, bool SNAP, bool DS, int SRC, int DST>
__device__ __forceinline__ void warp_loop(const Warp& w, Lane& s) {
  static_assert(VG % 4 == 0 && 32 % VG == 0, "validation group: a multiple of 4 steps that divides 32");
  const int32_t lane = (int32_t)w.lane;
  uint32_t x0[B], x1[B], p0[B], p1[B];
  // ring: row-blocks -30 .. 1 now (block 0 reads -29 .. 33), 2 .. 33 at the first boundary, 34 .. 65 staged
  xo_load_global<B>(w, -30 + lane, s.xstage);
  xo_store_ring<B>(w, -30 + lane, s.xstage);
  xo_load_global<B>(w, 2 + lane, s.xstage);
  xo_load_global<B>(w, -lane, x0);     // step 0's row-block
  xo_load_global<B>(w, 1 - lane, x1);  // step 1's row-block
  __syncwarp();
  p_from_offsets<B>(w, x0, p0);
  if (SRC == kSrcGlobal) s.win = window_load<SRC>(w, lane);
  const int32_t steps = w.R + 31;
  int32_t t = 0;
  // pipeline at an even step t: p0 = masks of step t, x1 = offsets of step t+1
  for (; t + 32 <= steps; t += 32) {
    xo_refill<B>(w, s, t);
    window_validate<B, SRC>(w, s, t, t == 0);
    block_start<SRC, DST>(w, s, t);
#pragma unroll 1
    for (int g = 0; g < 32 / VG; ++g) {
      ring_group_validate<B, SRC, VG>(w, s, t + VG * g);
      // four steps per iteration (VG is a multiple of 4): measured 10-13 % faster than two at 65536^2, while
      // eight or sixteen per iteration were slower (1.86 / 2.47 ms against 1.30 ms for the traceback fill)
#pragma unroll 1
      for (int k = VG * g; k < VG * g + VG; k += 4) {
        fill_step<B, TB, SNAP, DS, SRC, DST>(w, s, t + k, p0, x1, p1, x0);
        fill_step<B, TB, SNAP, DS, SRC, DST>(w, s, t + k + 1, p1, x0, p0, x1);
        fill_step<B, TB, SNAP, DS, SRC, DST>(w, s, t + k + 2, p0, x1, p1, x0);
        fill_step<B, TB, SNAP, DS, SRC, DST>(w, s, t + k + 3, p1, x0, p0, x1);
      }
      if (SRC == kSrcGlobal && VG * g + VG == 16) s.win_next = window_load<SRC>(w, t + 32 + lane);  // next window
    }
    if (SNAP && !DS) snap_store(w, s, t, steps);
  }
  xo_refill<B>(w, s, t);
  window_validate<B, SRC>(w, s, t, t == 0);
  block_start<SRC, DST>(w, s, t);
  const int32_t t_tail = t;
  for (; t + 1 < steps; t += 2) {
    if ((t & (VG - 1)) == 0) ring_group_validate<B, SRC, VG>(w, s, t);
    fill_step<B, TB, SNAP, DS, SRC, DST>(w, s, t, p0, x1, p1, x0);
    fill_step<B, TB, SNAP, DS, SRC, DST>(w, s, t + 1, p1, x0, p0, x1);
  }
  if (t < steps) {
    if ((t & (VG - 1)) == 0) ring_group_validate<B, SRC, VG>(w, s, t);
    fill_step<B, TB, SNAP, DS, SRC, DST>(w, s, t, p0, x1, p1, x0);
  }
  if (SNAP && !DS) snap_store(w, s, t_tail, steps);
}

template <int B, bool TB, int VG, bool SNAP, bool DS>
__device__ __forceinline__ void dispatch(const Warp& w, Lane& s, bool first_warp, bool last_warp, uint32_t wib) {
  if (first_warp) warp_loop<B, TB, VG, SNAP, DS, kSrcNone, kDstRing>(w, s);
  else if (wib == 0) warp_loop<B, TB, VG, SNAP, DS, kSrcGlobal, kDstRing>(w, s);
  else if (wib + 1 < kFillWarps) warp_loop<B, TB, VG, SNAP, DS, kSrcRing, kDstRing>(w, s);
  else if (!last_warp) warp_loop<B, TB, VG, SNAP, DS, kSrcRing, kDstGlobal>(w, s);
  else warp_loop<B, TB, VG, SNAP, DS, kSrcRing, kDstNone>(w, s);
}

// DS: dense snapshots (a traceback's segments shorter than 32 row-blocks), stored as each row-block ends.
template <int B, bool TB, int VG, bool DS>
__global__ void __launch_bounds__(kFillThreads, 1) k_fill(const __grid_constant__ FillArgs a) {
  static_assert(B % 4 == 0 && B >= 4 && B <= 16, "row-block height");
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t bid = blockIdx.x;
  int js = 0;
  if (a.njobs > 1 && bid >= a.job[0].nblocks) {
    bid -= a.job[0].nblocks;
    js = 1;
  }
  const FillJob& J = a.job[js];
  const uint32_t blk = J.block0 + bid;
  const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint32_t sigr = *J.sigma_rows;

  uint32_t* ring = sm;                             // [kFillWarps-1][kRing]: ring w carries warp w -> warp w+1
  uint32_t* cons = sm + (kFillWarps - 1) * kRing;  // [kFillWarps] consumption counters
  uint32_t* xring = cons + 8;                      // [kFillWarps][64][B] symbol-offset rings
  uint32_t* peq_s = xring + kFillWarps * 64 * 16;  // [sigr][kStripeWords]: this block's stripe of the masks
  for (uint32_t i = threadIdx.x; i < (kFillWarps - 1) * kRing + 8; i += kFillThreads) sm[i] = 0;
  const uint64_t col0 = (uint64_t)blk * kStripeWords;
  for (uint32_t i = threadIdx.x; i < sigr * kStripeWords; i += kFillThreads) {
    const uint32_t row = i / kStripeWords, col = i % kStripeWords;
    peq_s[i] = J.peq[(uint64_t)row * J.wpad + col0 + col];
  }
  __syncthreads();

  const uint64_t gw = (uint64_t)blk * kFillWarps + wib;
  const bool first_warp = (gw == 0);
  const bool last_warp = (wib == kFillWarps - 1) && (blk + 1 >= J.nblocks_total);
  Warp w;
  w.lane = lane;
  w.R = (int32_t)J.R;
  w.wpad = J.wpad;
  w.snap_rb = J.snap_rb;
  w.spin_limit = a.spin_limit;
  w.status = a.status;
  w.src_g = (wib == 0 && !first_warp) ? J.carry + (uint64_t)(blk - 1) * J.R : J.carry;
  w.dst_g = J.carry + (uint64_t)blk * J.R;
  w.peq_lane = (uint32_t)__cvta_generic_to_shared(peq_s) + (wib * 32 + lane) * 4u;
  w.xring = (uint32_t)__cvta_generic_to_shared(xring + wib * 64 * B);
  w.xring_p = reinterpret_cast<const uint4*>(xring + wib * 64 * B);
  w.peq_p = peq_s + wib * 32 + lane;
  w.xoff = J.xoff;
  w.ring_src = (uint32_t)__cvta_generic_to_shared(ring + (wib == 0 ? 0 : wib - 1) * kRing);
  w.ring_dst = (uint32_t)__cvta_generic_to_shared(ring + (wib + 1 < kFillWarps ? wib : 0) * kRing);
  w.cons_self = (uint32_t)__cvta_generic_to_shared(cons + wib);
  w.cons_next = (uint32_t)__cvta_generic_to_shared(cons + (wib + 1 < kFillWarps ? wib + 1 : wib));

  Lane s;
  s.V = kFull;
  s.cout = 0;
  s.cin_a = 0;
  s.cin_b = 0;
  s.failed = false;
  s.cap = 0;
  w.snap = J.snap ? J.snap + gw * 32 + lane : nullptr;
  w.cap_k = (lane + 31u) & 31u;
  w.hands_on = (lane == 31 && !(a.debug_drop && gw == 0)) ? 1u : 0u;
  s.win = 0;
  s.win_next = 0;
  s.cin0 = 0;
  s.tp = J.T ? reinterpret_cast<uint4*>(J.T + (gw * (J.R + 31)) * 32 * (uint64_t)B) + lane : nullptr;
  s.nsnap = (int32_t)J.snap_rb - 1;
  s.snp = w.snap;

  if (TB && J.T) {
    dispatch<B, true, VG, true, DS>(w, s, first_warp, last_warp, wib);
  } else if (TB && J.snap) {  // the table of the reversed strings in a traceback launch: snapshots, no bitmap
    dispatch<B, false, VG, true, DS>(w, s, first_warp, last_warp, wib);
  } else if (!DS) {
    dispatch<B, false, VG, false, false>(w, s, first_warp, last_warp, wib);
  }

  if (J.final_v) J.final_v[gw * 32 + lane] = s.V;
  if (J.len_acc) {
    const uint32_t z = __reduce_add_sync(kFull, (uint32_t)__popc(~s.V));
    if (lane == 0 && z) atomicAdd(J.len_acc, (unsigned long long)z);
  }
}

template <int B, bool TB, int VG, bool DS = false>
cudaError_t launch_t(const FillArgs& a, cudaStream_t st) {
  if constexpr (TB && !DS) {
    if (a.dense_snap) return launch_t<B, true, VG, true>(a, st);
  }
  static std::atomic<uint64_t> attr_done{0};  // per template instance: devices whose attribute is set
  auto fn = k_fill<B, TB, VG, DS>;
  const size_t smem = fill_smem_bytes();
  cudaError_t e = once_per_device_attr(
      [&] { return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); }, attr_done);
  if (e != cudaSuccess) return e;
  const unsigned grid = a.job[0].nblocks + (a.njobs > 1 ? a.job[1].nblocks : 0u);
  void* args[] = {const_cast<FillArgs*>(&a)};
  return cudaLaunchCooperativeKernel((const void*)fn, dim3(grid), dim3(kFillThreads), args, smem, st);
}

// ---- step floor probe --------------------------------------------------------------------------------------------
// The fill's step without the work around it: one block of 4 warps (one per SM sub-partition, as in the fill) runs
// `steps` systolic steps of B rows with exactly the fill's row arithmetic (rows<B, TB>: the row updates and the two
// carry shuffles per step) and in traceback mode the fill's two 16-byte bitmap stores per lane and step (into a
// 64-step ring per warp that stays in L2). Each warp times its steps with clock64 after 64 untimed ones.
// MSRC chooses where the rows' match masks come from (lane l works on row-block r = t - l at step t, as in the
// fill; the alphabet has 4 symbols, so Y's codes have two bit planes):
//   kMaskRegs   the masks held in registers (the floor of the row arithmetic);
//   kMaskTable  the fill's way: a shared table of every symbol's mask at the lane's word, read at the row's symbol
//               offset; the B offsets of a row-block come from a shared ring two steps ahead (two 16-byte loads), the
//               masks one step ahead (B loads);
//   kMaskPrmt   formed in registers from the lane's two bit planes of Y's codes: P = ~((pl0 ^ s0) | (pl1 ^ s1)),
//               s0 / s1 all ones where the row's code bit is set, each taken from the sign bit of a byte by one
//               byte permute; the codes of a row-block (bit b of row k at the top of byte k % 4 of word 2b + k / 4)
//               come from a shared ring one step ahead (one 16-byte load);
//   kMaskRows   the same formula with s0 / s1 of every row stored expanded in the ring (four 16-byte loads).
// Index ranges: masks[0..64), cycles[0..4), sink[0..128), tbuf[0 .. 4 warps * 64 slots * 32 lanes * B words) with
// B <= 16; the shared table [4 warps][8 rows][32 lanes] and ring [4 warps][4 vectors][64 slots] (B = 8 when MSRC
// is not kMaskRegs).
enum { kMaskRegs = 0, kMaskTable = 1, kMaskPrmt = 2, kMaskRows = 3 };

__device__ __forceinline__ uint32_t probe_code(const uint32_t* masks, uint32_t slot, uint32_t k) {
  return (masks[(slot + 7 * k) & 63] >> (k + slot % 7)) & 3u;  // the code (0..3) of row k of ring slot `slot`
}

template <int B, bool TB, int MSRC>
__global__ void __launch_bounds__(kFillThreads, 1)
    k_step_floor(const uint32_t* masks, uint32_t steps, unsigned long long* cycles, uint32_t* sink, uint4* tbuf) {
  static_assert(MSRC == kMaskRegs || B == 8, "mask sources other than registers are probed with 8 rows per step");
  __shared__ uint32_t tab_s[kFillWarps][8][32];
  __shared__ uint4 ring_s[kFillWarps][4][64];
  const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint32_t pl0 = masks[lane], pl1 = masks[lane + 32];  // the lane's two bit planes of Y's codes
  if (MSRC != kMaskRegs) {
    for (uint32_t c = 0; c < 8; ++c)  // the mask of code c at the lane's word (rows 4..7: no symbol, zero)
      tab_s[wib][c][lane] = c < 4 ? ~((pl0 ^ (0u - (c & 1u))) | (pl1 ^ (0u - (c >> 1)))) : 0u;
    for (uint32_t sl = lane; sl < 64; sl += 32) {
      uint32_t cd[8];
#pragma unroll
      for (uint32_t k = 0; k < 8; ++k) cd[k] = probe_code(masks, sl, k);
      if (MSRC == kMaskTable) {
        ring_s[wib][0][sl] = make_uint4(cd[0] * 32, cd[1] * 32, cd[2] * 32, cd[3] * 32);
        ring_s[wib][1][sl] = make_uint4(cd[4] * 32, cd[5] * 32, cd[6] * 32, cd[7] * 32);
      } else if (MSRC == kMaskPrmt) {
        uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
        for (uint32_t k = 0; k < 8; ++k)
#pragma unroll
          for (uint32_t b = 0; b < 2; ++b) w[2 * b + k / 4] |= ((cd[k] >> b) & 1u) << (8 * (k % 4) + 7);
        ring_s[wib][0][sl] = make_uint4(w[0], w[1], w[2], w[3]);
      } else {
        uint32_t e[16];
#pragma unroll
        for (uint32_t k = 0; k < 8; ++k) {
          e[k] = 0u - (cd[k] & 1u);
          e[8 + k] = 0u - (cd[k] >> 1);
        }
#pragma unroll
        for (uint32_t v = 0; v < 4; ++v) ring_s[wib][v][sl] = make_uint4(e[4 * v], e[4 * v + 1], e[4 * v + 2], e[4 * v + 3]);
      }
    }
  }
  __syncthreads();
  uint32_t P[B];  // kMaskRegs: the masks; kMaskTable: the next step's masks
#pragma unroll
  for (int b = 0; b < B; ++b) P[b] = masks[(threadIdx.x * B + b) & 63];
  uint32_t xo[B];  // kMaskTable: symbol offsets of the row-block two steps ahead
#pragma unroll
  for (int b = 0; b < B; ++b) xo[b] = 0;
  uint4 c4[4] = {};  // kMaskPrmt / kMaskRows: the codes of the next step's row-block
  const uint32_t* tp_s = &tab_s[wib][0][lane];
  uint32_t V = kFull, cin_a = 0, cin_b = 0, acc = 0;
  uint4* tp = tbuf + (size_t)wib * 64 * 32 * (B / 4) + lane;  // the fill's chunk layout: [B/4][32 lanes] vectors
  long long t0 = 0;
#pragma unroll 1
  for (uint32_t t = 0; t < steps + 64; ++t) {
    if (t == 64) t0 = clock64();
    const uint32_t r = t - lane;
    uint32_t Pu[B];
    if (MSRC == kMaskRegs) {
#pragma unroll
      for (int b = 0; b < B; ++b) Pu[b] = P[b];
    } else if (MSRC == kMaskTable) {
#pragma unroll
      for (int b = 0; b < B; ++b) Pu[b] = P[b];
#pragma unroll
      for (int b = 0; b < B; ++b) P[b] = tp_s[xo[b]];
      const uint4 q0 = ring_s[wib][0][(r + 2) & 63], q1 = ring_s[wib][1][(r + 2) & 63];
      xo[0] = q0.x; xo[1] = q0.y; xo[2] = q0.z; xo[3] = q0.w;
      xo[4] = q1.x; xo[5] = q1.y; xo[6] = q1.z; xo[7] = q1.w;
    } else if (MSRC == kMaskPrmt) {
      const uint32_t w[4] = {c4[0].x, c4[0].y, c4[0].z, c4[0].w};
#pragma unroll
      for (int k = 0; k < B; ++k) {
        const uint32_t sel = 0x8888u + 0x1111u * (uint32_t)(k % 4);  // byte k % 4, its sign bit replicated
        const uint32_t s0 = __byte_perm(w[k / 4], 0u, sel), s1 = __byte_perm(w[2 + k / 4], 0u, sel);
        Pu[k] = ~((pl0 ^ s0) | (pl1 ^ s1));
      }
      c4[0] = ring_s[wib][0][(r + 1) & 63];
    } else {
      const uint32_t e[16] = {c4[0].x, c4[0].y, c4[0].z, c4[0].w, c4[1].x, c4[1].y, c4[1].z, c4[1].w,
                              c4[2].x, c4[2].y, c4[2].z, c4[2].w, c4[3].x, c4[3].y, c4[3].z, c4[3].w};
#pragma unroll
      for (int k = 0; k < B; ++k) Pu[k] = ~((pl0 ^ e[k]) | (pl1 ^ e[8 + k]));
#pragma unroll
      for (int v = 0; v < 4; ++v) c4[v] = ring_s[wib][v][(r + 1) & 63];
    }
    uint32_t co, tw[B];
    rows<B, TB>(Pu, V, cin_a, cin_b, co, cin_a, cin_b, tw);
    acc += co;
    if (TB) {
      uint4* q = tp + (size_t)(t & 63) * 32 * (B / 4);
#pragma unroll
      for (int v = 0; v < B / 4; ++v) q[v * 32] = make_uint4(tw[4 * v], tw[4 * v + 1], tw[4 * v + 2], tw[4 * v + 3]);
    }
  }
  const long long t1 = clock64();
  if (lane == 0) cycles[wib] = (unsigned long long)(t1 - t0);
  sink[threadIdx.x] = V ^ acc;
}

template <int B, bool TB, int MSRC = kMaskRegs>
cudaError_t step_floor_t(uint32_t steps, double* cycles_per_step) {
  uint32_t *masks = nullptr, *sink = nullptr;
  unsigned long long* cyc = nullptr;
  uint4* tbuf = nullptr;
  const size_t tbuf_bytes = (size_t)4 * 64 * 32 * 16 * 4;
  cudaError_t e = cudaMalloc(&masks, 64 * 4);
  if (e == cudaSuccess) e = cudaMalloc(&sink, kFillThreads * 4);
  if (e == cudaSuccess) e = cudaMalloc(&cyc, kFillWarps * 8);
  if (e == cudaSuccess) e = cudaMalloc(&tbuf, tbuf_bytes);
  if (e == cudaSuccess) {
    uint32_t h[64];
    uint64_t z = 0x9E3779B97F4A7C15ull;
    for (int k = 0; k < 64; ++k) {  // fixed pseudo-random masks (splitmix64 outputs)
      z += 0x9E3779B97F4A7C15ull;
      uint64_t v = z;
      v = (v ^ (v >> 30)) * 0xBF58476D1CE4E5B9ull;
      v = (v ^ (v >> 27)) * 0x94D049BB133111EBull;
      h[k] = (uint32_t)(v ^ (v >> 31));
    }
    e = cudaMemcpy(masks, h, sizeof(h), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    k_step_floor<B, TB, MSRC><<<1, kFillThreads>>>(masks, steps, cyc, sink, tbuf);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  unsigned long long hc[kFillWarps] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(hc, cyc, sizeof(hc), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) {
    std::sort(hc, hc + kFillWarps);
    *cycles_per_step = 0.5 * (double)(hc[1] + hc[2]) / (double)steps;  // median of the 4 warps
  }
  cudaFree(masks);
  cudaFree(sink);
  cudaFree(cyc);
  cudaFree(tbuf);
  return e;
}

}  // namespace

size_t fill_smem_bytes() {
  return ((size_t)(kFillWarps - 1) * kRing + 8 + (size_t)kFillWarps * 64 * 16 + (size_t)kSigmaMax * kStripeWords) *
         sizeof(uint32_t);
}

int fill_max_coop_blocks(int device) {
  int sms = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  auto fn = k_fill<8, true, 16, false>;
  const size_t smem = fill_smem_bytes();
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kFillThreads, smem) != cudaSuccess) return 0;
  return sms * per_sm;
}

// B = rows per step (8 or 16); variant bits 1-2 choose the hand-off validation group of ring-fed warps: 2 = the
// larger (32 steps for B = 8, 16 for B = 16), any other value the default (16 / 8). Both give the same results;
// only the pipeline lag and the per-step overhead differ.
template <int B, int VGD, int VGA>
cudaError_t launch_b(const FillArgs& a, bool traceback, cudaStream_t st) {
  const int sel = (a.variant >> 1) & 3;
  if (sel == 2) return traceback ? launch_t<B, true, VGA>(a, st) : launch_t<B, false, VGA>(a, st);
  return traceback ? launch_t<B, true, VGD>(a, st) : launch_t<B, false, VGD>(a, st);
}

cudaError_t launch_fill(const FillArgs& a, uint32_t B, bool traceback, cudaStream_t st) {
  if (B == 8) return launch_b<8, 16, 32>(a, traceback, st);
  if (B == 16) return launch_b<16, 8, 16>(a, traceback, st);
  return cudaErrorInvalidValue;
}

cudaError_t step_floor(uint32_t B, bool traceback, uint32_t steps, double* cycles_per_step) {
  if (B == 8) return traceback ? step_floor_t<8, true>(steps, cycles_per_step) : step_floor_t<8, false>(steps, cycles_per_step);
  if (B == 16) return traceback ? step_floor_t<16, true>(steps, cycles_per_step) : step_floor_t<16, false>(steps, cycles_per_step);
  return cudaErrorInvalidValue;
}

cudaError_t step_masks(uint32_t source, uint32_t steps, double* cycles_per_step) {
  switch (source) {
    case kMaskRegs: return step_floor_t<8, true, kMaskRegs>(steps, cycles_per_step);
    case kMaskTable: return step_floor_t<8, true, kMaskTable>(steps, cycles_per_step);
    case kMaskPrmt: return step_floor_t<8, true, kMaskPrmt>(steps, cycles_per_step);
    case kMaskRows: return step_floor_t<8, true, kMaskRows>(steps, cycles_per_step);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lcs
