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
#include "lcs_internal.h"

namespace lcs {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_gpu(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_vol_shared(const uint32_t* p) { return *(const volatile uint32_t*)p; }
__device__ __forceinline__ void st_vol_shared(uint32_t* p, uint32_t v) { *(volatile uint32_t*)p = v; }

// Slot = carry bits (the top B bits, row 0 of the block at bit 31) | tag (low 32-B bits, never 0).
template <int B>
__device__ __forceinline__ uint32_t slot_tag(uint64_t r) {
  constexpr uint32_t mask = (1u << (32 - B)) - 1u;
  return ((uint32_t)(r + 1) | 1u) & mask;
}

__device__ __noinline__ uint32_t spin_slot(const uint32_t* p, bool global, uint32_t want, uint32_t tmask,
                                           DevStatus* st, uint32_t limit, bool& failed, uint32_t where) {
  uint32_t v = 0;
  for (uint32_t it = 0;; ++it) {
    v = global ? ld_relaxed_gpu(p) : ld_vol_shared(p);
    if ((v & tmask) == want || failed) return v;
    if ((it & 127u) == 127u) {
      if (*(volatile uint32_t*)&st->abort) { failed = true; return v; }
      if (it >= limit) {
        atomicOr(&st->flags, kStatTimeout);
        atomicExch(&st->where, where);
        atomicExch(&st->abort, 1u);
        failed = true;
        return v;
      }
    }
    __nanosleep(64);
  }
}

__device__ __noinline__ void spin_ring_space(const uint32_t* cons, uint64_t r, DevStatus* st, uint32_t limit,
                                             bool& failed) {
  for (uint32_t it = 0;; ++it) {
    const uint32_t c = ld_vol_shared(cons);
    if ((int64_t)r - (int64_t)c < (int64_t)(kRing - 64) || failed) return;
    if ((it & 127u) == 127u) {
      if (*(volatile uint32_t*)&st->abort) { failed = true; return; }
      if (it >= limit) {
        atomicOr(&st->flags, kStatTimeout);
        atomicExch(&st->where, 3u);
        atomicExch(&st->abort, 1u);
        failed = true;
        return;
      }
    }
    __nanosleep(64);
  }
}

template <int B, bool TB>
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

  uint32_t* ring = sm;                       // [kFillWarps-1][kRing]: ring w carries warp w -> warp w+1
  uint32_t* cons = sm + (kFillWarps - 1) * kRing;  // [kFillWarps] consumer progress (row-blocks consumed)
  uint32_t* peq_s = cons + 8;                // [sigr][kStripeWords], this block's stripe of the match masks
  for (uint32_t i = threadIdx.x; i < (kFillWarps - 1) * kRing + 8; i += kFillThreads) sm[i] = 0;
  const uint64_t col0 = (uint64_t)blk * kStripeWords;
  for (uint32_t i = threadIdx.x; i < sigr * kStripeWords; i += kFillThreads) {
    const uint32_t row = i / kStripeWords, col = i % kStripeWords;
    peq_s[i] = J.peq[(uint64_t)row * J.wpad + col0 + col];
  }
  __syncthreads();

  const uint64_t R = J.R;
  const uint64_t gw = (uint64_t)blk * kFillWarps + wib;
  const bool first_warp = (gw == 0);
  const bool src_global = (wib == 0);
  const bool dst_global = (wib == kFillWarps - 1);
  const bool has_consumer = !(dst_global && blk + 1 >= J.nblocks_total);
  const uint32_t* src_g = (src_global && !first_warp) ? J.carry + (uint64_t)(blk - 1) * R : nullptr;
  const uint32_t* src_s = ring + (wib == 0 ? 0 : (wib - 1)) * kRing;
  uint32_t* dst_g = J.carry + (uint64_t)blk * R;
  uint32_t* dst_s = ring + (dst_global ? 0 : wib) * kRing;
  const char* peq_lane = reinterpret_cast<const char*>(peq_s) + (wib * 32 + lane) * 4;
  constexpr uint32_t kTagMask = (1u << (32 - B)) - 1u;
  bool failed = false;

  auto load_slot = [&](uint64_t s) -> uint32_t {
    if (first_warp || s >= R) return 0u;
    return src_global ? ld_relaxed_gpu(src_g + s) : ld_vol_shared(src_s + (s % kRing));
  };
  uint32_t win_cur = load_slot(lane), win_next = load_slot(32 + lane);

  uint64_t next_snap = J.snap_rb ? (uint64_t)J.snap_rb - 1 : ~0ull;  // next row-block whose end is snapshotted
  uint32_t* snap_lane = J.snap ? J.snap + gw * 32 + lane : nullptr;
  uint64_t snap_idx = 0;
  uint32_t V = kFull;
  uint32_t cout_prev = 0;
  const uint64_t steps = R + 31;
  for (uint64_t t = 0; t < steps; ++t) {
    const int64_t r = (int64_t)t - (int64_t)lane;
    // symbol offsets of the B rows of this lane's row-block (the array has zero rows around [0, R))
    const uint4* xo4 = reinterpret_cast<const uint4*>(J.xoff + (uint64_t)(r + kPadRowblocks) * B);
    uint32_t xo[B];
#pragma unroll
    for (int v = 0; v < B / 4; ++v) {
      const uint4 q4 = __ldg(xo4 + v);
      xo[4 * v + 0] = q4.x;
      xo[4 * v + 1] = q4.y;
      xo[4 * v + 2] = q4.z;
      xo[4 * v + 3] = q4.w;
    }
    // carries entering this lane's word: from lane-1's previous step; lane 0 from the previous warp
    uint32_t cin = __shfl_up_sync(kFull, cout_prev, 1);
    const uint32_t wv = __shfl_sync(kFull, win_cur, (int)(t & 31));
    if (lane == 0) {
      cin = 0;
      if (!first_warp && t < R) {
        uint32_t v = wv;
        if ((v & kTagMask) != slot_tag<B>(t)) {
          const uint32_t* p = src_global ? (src_g + t) : (src_s + (t % kRing));
          v = spin_slot(p, src_global, slot_tag<B>(t), kTagMask, a.status, a.spin_limit, failed,
                        src_global ? 1u : 2u);
        }
        cin = v & ~kTagMask;
      }
      if (!src_global && (t & 31) == 0) st_vol_shared(&cons[wib], (uint32_t)t);
    }
    if ((t & 31) == 31) {
      win_cur = win_next;
      win_next = load_slot(t + 33 + lane);
    }
    // B rows of the bit-parallel update; the carry bits enter at the MSB of cw and leave into the LSB of co
    uint32_t cw = cin, co = 0;
    uint32_t tw[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const uint32_t P = *reinterpret_cast<const uint32_t*>(peq_lane + xo[b]);
      const uint32_t U = V & P;
      uint32_t S;
      asm("add.cc.u32 %0, %0, %0;\n\t"
          "addc.cc.u32 %1, %3, %4;\n\t"
          "addc.u32 %2, %2, %2;"
          : "+r"(cw), "=r"(S), "+r"(co)
          : "r"(V), "r"(U));
      if (TB) tw[b] = S ^ V ^ U;
      V = S | (V & ~P);
    }
    cout_prev = co << (32 - B);
    if (TB && J.T) {
      uint4* chunk = reinterpret_cast<uint4*>(J.T + ((gw * (R + 31) + t) * 32) * (uint64_t)B);
#pragma unroll
      for (int v = 0; v < B / 4; ++v)
        chunk[v * 32 + lane] = make_uint4(tw[4 * v], tw[4 * v + 1], tw[4 * v + 2], tw[4 * v + 3]);
    }
    if (snap_lane && r == (int64_t)next_snap) {
      if ((uint64_t)r < R) snap_lane[snap_idx * J.wpad] = V;
      next_snap += J.snap_rb;
      ++snap_idx;
    }
    if (lane == 31 && has_consumer) {
      const int64_t r31 = (int64_t)t - 31;
      if (r31 >= 0 && (uint64_t)r31 < R) {
        const uint32_t v = cout_prev | slot_tag<B>((uint64_t)r31);
        if (dst_global) {
          st_relaxed_gpu(dst_g + r31, v);
        } else {
          if ((r31 & 31) == 0) spin_ring_space(&cons[wib + 1], (uint64_t)r31, a.status, a.spin_limit, failed);
          st_vol_shared(dst_s + ((uint64_t)r31 % kRing), v);
        }
      }
    }
  }
  if (J.final_v) J.final_v[gw * 32 + lane] = V;
  if (J.len_acc) {
    const uint32_t z = __reduce_add_sync(kFull, (uint32_t)__popc(~V));
    if (lane == 0 && z) atomicAdd(J.len_acc, (unsigned long long)z);
  }
}

template <int B, bool TB>
cudaError_t launch_t(const FillArgs& a, cudaStream_t st) {
  auto fn = k_fill<B, TB>;
  const size_t smem = fill_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = a.job[0].nblocks + (a.njobs > 1 ? a.job[1].nblocks : 0u);
  void* args[] = {const_cast<FillArgs*>(&a)};
  return cudaLaunchCooperativeKernel((const void*)fn, dim3(grid), dim3(kFillThreads), args, smem, st);
}

}  // namespace

size_t fill_smem_bytes() {
  return ((size_t)(kFillWarps - 1) * kRing + 8 + (size_t)kSigmaMax * kStripeWords) * sizeof(uint32_t);
}

int fill_max_coop_blocks(int device) {
  int sms = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  auto fn = k_fill<8, true>;
  const size_t smem = fill_smem_bytes();
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kFillThreads, smem) != cudaSuccess) return 0;
  return sms * per_sm;
}

cudaError_t launch_fill(const FillArgs& a, uint32_t B, bool traceback, cudaStream_t st) {
  if (B != 8) return cudaErrorInvalidValue;
  return traceback ? launch_t<8, true>(a, st) : launch_t<8, false>(a, st);
}

}  // namespace lcs
