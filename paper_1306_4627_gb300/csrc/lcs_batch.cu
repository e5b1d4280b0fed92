// lcs_batch: LCS lengths (c[m,n], paper §I.C) of many independent pairs in one persistent launch.
//
// Every pair is a small instance of the same bit-parallel row update as the single-pair fill (U = V & P;
// S = V + U; V' = S | (V & ~P), one 32-column word per register). Here the rows of a pair are processed by a group
// of G lanes of a warp, each lane holding K consecutive words of the row (K = 2, 4 or 8 words per lane):
//   * the add inside a lane ripples through its K words with the carry flag;
//   * the lanes of a group run skewed by one row each (lane g works on row t - g at step t), so the carry out of a
//     lane's 32K bits for a row is shuffled to the next lane, which adds it in the same row one step later;
//   * a warp works on floor(32 / G) pairs of the same shape at once, G = ceil(ceil(n / 32) / K) lanes per pair (so
//     short pairs share a warp and long pairs spread over it).
// The host plans the launch: it buckets pairs by (K, G), orders work items (up to 32 / G pairs each) by decreasing
// rows, and a persistent kernel lets every warp take the next item from an atomic ticket. A pair with many rows is
// split in two jobs that run at the same time, its top half forward and its bottom half on the reversed strings;
// a small kernel then takes L = max_j (c[mt, j] + LCS(X[mt+1..m], Y[j+1..n])) from the two final rows, so the
// longest serial chain of rows in a batch is halved. Words per lane, the height above which a pair is split and the
// resident blocks per SM form the batch configuration, which lcs_ctx_autotune_batch_dev picks by timing.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <new>
#include <vector>

#include "lcs_ctx.h"
#include "lcs_plan.h"

namespace lcs {
int take_status(lcs_ctx* c);
}  // namespace lcs
int ensure_hstage(lcs_ctx* c, size_t bytes);  // lcs_api.cu: pinned staging area of a context
bool host_pinned(const void* p);

namespace {

using namespace lcs;
using namespace lcs_plan;

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr int kBatchWarps = 8;     // warps per block of the persistent kernel
constexpr int kStageRows = 24;     // match-mask rows staged in shared memory per warp (alphabets up to 23 symbols)

struct BatchArgs {
  const uint8_t* xs;
  const uint8_t* ys;
  const BPair* pairs;
  const BJob* jobs;
  const BItem* items;
  uint32_t* sigma;     // per plan pair: symbols present in y (its zero row index)
  uint16_t* xcode;     // per job: the codes of its rows in its pair's alphabet (0..256); 16 zeros at the start
  uint32_t* peq;
  uint32_t* fvbuf;     // final rows of split pairs' jobs, kRowWords words per slot
  uint64_t* out_lens;
  uint32_t* ticket;      // ticket[0]: items of k_batch_main, ticket[1]: pairs of k_batch_prep
  const uint32_t* split;  // plan indices of split pairs
  const uint32_t* prep_order;  // plan indices of all pairs, most prep work first
  uint32_t npairs, nitems, nsplit;
  uint32_t stage_words;  // k_batch_main: words of match-mask stage per warp (dynamic shared memory)
};

// ---- per-pair alphabet, symbol codes and match-mask table (one warp per pair) ------------------------------------
// Strings are read with 16-byte loads where their alignment allows (a forward job's 16-bit codes are placed so
// that a 16-byte group of x maps to a 32-byte group of codes), and y is kept in shared memory for the alphabet
// and the table build.
constexpr uint32_t kMaxBatchCols = kRowWords * 32;  // 4096: the longest y of a batch pair


// One match-mask table (see the comment in k_batch_prep): column j of the table has the code map[y[j]], or
// map[y[n - 1 - j]] for the table over reversed y. The words are independent; four are in flight at a time.
template <int NB>
__device__ __forceinline__ void build_table(uint32_t* tab, const BPair& pr, bool reversed, const uint8_t* ysh,
                                            const uint16_t* map, uint32_t sigma, uint32_t lane) {
  uint32_t flip0[NB];  // for row r = lane: 0 where bit b of r is set, all ones where it is not
#pragma unroll
  for (int b = 0; b < NB; ++b) flip0[b] = ((lane >> b) & 1u) - 1u;
#pragma unroll 4
  for (uint32_t q = 0; q < pr.w; ++q) {
    const uint32_t j = q * 32 + lane;
    const bool in = j < pr.n;
    const uint32_t valid = __ballot_sync(kFull, in);
    const uint32_t code = in ? map[ysh[reversed ? pr.n - 1 - j : j]] : 0u;
    uint32_t pf[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) pf[b] = __ballot_sync(kFull, (code >> b) & 1u);
    if (lane <= sigma) {
      uint32_t mf = valid;
#pragma unroll
      for (int b = 0; b < NB; ++b) mf &= pf[b] ^ flip0[b];
      tab[(uint64_t)lane * pr.w + q] = mf;
    }
    for (uint32_t r = lane + 32; r <= sigma; r += 32) {  // alphabets of more than 31 symbols
      uint32_t mf = valid;
#pragma unroll
      for (int b = 0; b < NB; ++b) mf &= pf[b] ^ (((r >> b) & 1u) - 1u);
      tab[(uint64_t)r * pr.w + q] = mf;
    }
  }
}

template <int NB>
__device__ __noinline__ void build_tables(const BatchArgs& a, const BPair& pr, const uint8_t* ysh, const uint16_t* map,
                                          uint32_t sigma, uint32_t lane) {
  build_table<NB>(a.peq + pr.peq_off, pr, false, ysh, map, sigma, lane);
  if (pr.mt < pr.m) build_table<NB>(a.peq + pr.peqr_off, pr, true, ysh, map, sigma, lane);
}

__global__ void __launch_bounds__(256, 4) k_batch_prep(BatchArgs a) {
  __shared__ uint32_t pres_s[8][8];
  __shared__ uint16_t map_s[8][256];
  __shared__ __align__(16) uint8_t y_s[8][kMaxBatchCols + 16];
  const uint32_t wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* pres = pres_s[wid];
  uint16_t* map = map_s[wid];
  for (;;) {  // persistent: every warp takes the next pair (most work first) from a ticket
    uint32_t it = 0;
    if (lane == 0) it = atomicAdd(a.ticket + 1, 1u);
    it = __shfl_sync(kFull, it, 0);
    if (it >= a.npairs) break;
    const uint32_t p = a.prep_order[it];
    const BPair pr = a.pairs[p];
    // y into shared memory: y[j] at ysh[j], where ysh = y_s + sh places the 16-byte groups of y on 16-byte
    // boundaries of y_s (sh = 16 - (y mod 16), or 0 when y is aligned)
    const uint8_t* y = a.ys + pr.y_off;
    const uint32_t head = (uint32_t)((16u - ((uintptr_t)y & 15u)) & 15u);
    const uint32_t hn = head < pr.n ? head : pr.n;
    uint8_t* ysh = y_s[wid] + ((16u - head) & 15u);
    const uint32_t nvec = (pr.n - hn) >> 4;
    if (lane < hn) ysh[lane] = y[lane];
#pragma unroll 8
    for (uint32_t v = lane; v < nvec; v += 32)
      *reinterpret_cast<uint4*>(ysh + hn + 16 * v) = __ldg(reinterpret_cast<const uint4*>(y + hn + 16 * v));
    {
      const uint32_t j = hn + 16 * nvec + lane;
      if (lane < 16 && j < pr.n) ysh[j] = y[j];
    }
    __syncwarp();
    // presence of each byte value: which 32-value blocks occur, and the OR of the values' low five bits, which is
    // the presence mask itself when a single block occurs (uppercase DNA or protein letters); otherwise one pass per
    // occurring block (few for text alphabets), or one pass with a register per block when more than two occur
    {
      if (lane < 8) pres[lane] = 0;
      uint32_t blocks = 0, low = 0;
      for (uint32_t j = lane; j < pr.n; j += 32) {
        const uint32_t v = ysh[j];
        blocks |= 1u << (v >> 5);
        low |= 1u << (v & 31);
      }
      blocks = __reduce_or_sync(kFull, blocks);
      low = __reduce_or_sync(kFull, low);
      __syncwarp();
      if (__popc(blocks) == 1) {
        if (lane == 0) pres[__ffs(blocks) - 1] = low;
      } else if (__popc(blocks) == 2) {
        for (uint32_t bl = blocks; bl; bl &= bl - 1) {
          const uint32_t hi = __ffs(bl) - 1;
          uint32_t acc = 0;
          for (uint32_t j = lane; j < pr.n; j += 32) {
            const uint32_t v = ysh[j];
            acc |= (v >> 5) == hi ? 1u << (v & 31) : 0u;
          }
          acc = __reduce_or_sync(kFull, acc);
          if (lane == 0) pres[hi] = acc;
        }
      } else {
        uint32_t pl[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (uint32_t j = lane; j < pr.n; j += 32) {
          const uint32_t v = ysh[j], hi = v >> 5, bit = 1u << (v & 31);
#pragma unroll
          for (uint32_t k = 0; k < 8; ++k) pl[k] |= hi == k ? bit : 0u;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const uint32_t v = __reduce_or_sync(kFull, pl[k]);
          if (lane == (uint32_t)k) pres[k] = v;
        }
      }
    }
    __syncwarp();
    // code of a present byte = its rank among the present bytes; absent bytes map to the zero row (sigma)
    uint32_t sigma;
    {
      const uint32_t pk = lane < 8 ? pres[lane] : 0u, cnt = __popc(pk);
      uint32_t incl = cnt;
      for (uint32_t off = 1; off < 8; off <<= 1) {
        const uint32_t o = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += o;
      }
      sigma = __shfl_sync(kFull, incl, 7);
      const uint32_t below_lane = (1u << lane) - 1u;  // lane < 32: bits under this lane's byte within a block
#pragma unroll
      for (uint32_t k = 0; k < 8; ++k) {
        const uint32_t pw = __shfl_sync(kFull, pk, k), base = __shfl_sync(kFull, incl - cnt, k);
        map[k * 32 + lane] = (uint16_t)(((pw >> lane) & 1u) ? base + __popc(pw & below_lane) : sigma);
      }
    }
    if (lane == 0) a.sigma[p] = sigma;
    __syncwarp();
    // codes of the forward job's rows x[0..mt), 16 symbols per load where the alignment of x allows, then of the
    // reverse job's rows x[m-1] down to x[mt]; each list has kCodePadFront zero-row codes before it and
    // kCodePadBack after it, so the main kernel reads the codes of 8 rows without a bounds check
    {
      const uint8_t* x = a.xs + pr.x_off;
      uint16_t* xc = a.xcode + pr.xcf;
      const uint32_t xh0 = (uint32_t)((16u - ((uintptr_t)x & 15u)) & 15u);
      const uint32_t xh = xh0 < pr.mt ? xh0 : pr.mt;
      const uint32_t xv = (pr.mt - xh) >> 4;
      if (lane < xh) xc[lane] = map[x[lane]];
#pragma unroll 4
      for (uint32_t v = lane; v < xv; v += 32) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(x + xh + 16 * v));
        const uint32_t in[4] = {q.x, q.y, q.z, q.w};
        uint32_t o[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          o[2 * k] = (uint32_t)map[in[k] & 0xFF] | ((uint32_t)map[(in[k] >> 8) & 0xFF] << 16);
          o[2 * k + 1] = (uint32_t)map[(in[k] >> 16) & 0xFF] | ((uint32_t)map[in[k] >> 24] << 16);
        }
        uint4* dst = reinterpret_cast<uint4*>(xc + xh + 16 * v);
        dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
        dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
      }
      const uint32_t i = xh + 16 * xv + lane;
      if (lane < 16 && i < pr.mt) xc[i] = map[x[i]];
      xc[(int)lane - (int)kCodePadFront] = (uint16_t)sigma;  // kCodePadFront == 32
      if (lane < kCodePadBack) xc[pr.mt + lane] = (uint16_t)sigma;
      if (pr.mt < pr.m) {  // x[mt + k'] is row rr - 1 - k' of the reverse job; 16-byte loads, 2-byte stores
        uint16_t* xr = a.xcode + pr.xcr;
        const uint32_t rr = pr.m - pr.mt;
        const uint8_t* xb = x + pr.mt;
        const uint32_t rh0 = (uint32_t)((16u - ((uintptr_t)xb & 15u)) & 15u);
        const uint32_t rh = rh0 < rr ? rh0 : rr;
        const uint32_t rv = (rr - rh) >> 4;
        if (lane < rh) xr[rr - 1 - lane] = map[xb[lane]];
#pragma unroll 2
        for (uint32_t v = lane; v < rv; v += 32) {
          const uint4 q = __ldg(reinterpret_cast<const uint4*>(xb + rh + 16 * v));
          const uint32_t in[4] = {q.x, q.y, q.z, q.w};
          uint16_t* dst = xr + (rr - 1 - rh - 16 * v);  // rows dst[0], dst[-1], ..., dst[-15]
#pragma unroll
          for (int k = 0; k < 16; ++k) dst[-k] = map[(in[k >> 2] >> (8 * (k & 3))) & 0xFF];
        }
        const uint32_t kt = rh + 16 * rv + lane;
        if (lane < 16 && kt < rr) xr[rr - 1 - kt] = map[xb[kt]];
        xr[(int)lane - (int)kCodePadFront] = (uint16_t)sigma;
        if (lane < kCodePadBack) xr[rr + lane] = (uint16_t)sigma;
      }
    }
    // The tables, one 32-column word q at a time: lane k holds the code of column 32q + k; ballots of the code's
    // bits give bit planes, and the mask of symbol r is the AND over the planes of the plane (bit b of r set) or
    // its complement (not set), restricted to the columns that exist. Lane r writes row r (rows 0..sigma, 32 rows
    // per pass); row sigma matches no column, since the columns' codes are 0..sigma-1, and comes out zero.
    const uint32_t nb = 32 - __clz(sigma);  // bits of the codes 0..sigma
    switch (nb) {
      case 1: build_tables<1>(a, pr, ysh, map, sigma, lane); break;
      case 2: build_tables<2>(a, pr, ysh, map, sigma, lane); break;
      case 3: build_tables<3>(a, pr, ysh, map, sigma, lane); break;
      case 4: build_tables<4>(a, pr, ysh, map, sigma, lane); break;
      case 5: build_tables<5>(a, pr, ysh, map, sigma, lane); break;
      case 6: build_tables<6>(a, pr, ysh, map, sigma, lane); break;
      case 7: build_tables<7>(a, pr, ysh, map, sigma, lane); break;
      case 8: build_tables<8>(a, pr, ysh, map, sigma, lane); break;
      default: build_tables<9>(a, pr, ysh, map, sigma, lane); break;
    }
    __syncwarp();
  }
}

// ---- the persistent batch kernel --------------------------------------------------------------------------------
// S = V + U + c over the lane's K words (s holds V on entry), c = cin & 1 when take is all ones and 0 when take is 0
// (cin is 0 or 1); cout = carry out of the lane's top bit. One asm block per K keeps the carry flag between the words.
template <int K>
__device__ __forceinline__ void addc_words(const uint32_t (&u)[K], uint32_t cin, uint32_t take, uint32_t (&s)[K],
                                           uint32_t& cout);
template <>
__device__ __forceinline__ void addc_words<2>(const uint32_t (&u)[2], uint32_t cin, uint32_t take, uint32_t (&s)[2],
                                              uint32_t& cout) {
  asm("{\n\t"
      ".reg .u32 t;\n\t"
      "add.cc.u32 t, %3, %6;\n\t"  // carry flag = cin when take = 0xFFFFFFFF, 0 when take = 0
      "addc.cc.u32 %0, %0, %4;\n\t"
      "addc.cc.u32 %1, %1, %5;\n\t"
      "addc.u32 %2, 0, 0;\n\t"
      "}"
      : "+r"(s[0]), "+r"(s[1]), "=r"(cout)
      : "r"(cin), "r"(u[0]), "r"(u[1]), "r"(take));
}
template <>
__device__ __forceinline__ void addc_words<4>(const uint32_t (&u)[4], uint32_t cin, uint32_t take, uint32_t (&s)[4],
                                              uint32_t& cout) {
  asm("{\n\t"
      ".reg .u32 t;\n\t"
      "add.cc.u32 t, %5, %10;\n\t"
      "addc.cc.u32 %0, %0, %6;\n\t"
      "addc.cc.u32 %1, %1, %7;\n\t"
      "addc.cc.u32 %2, %2, %8;\n\t"
      "addc.cc.u32 %3, %3, %9;\n\t"
      "addc.u32 %4, 0, 0;\n\t"
      "}"
      : "+r"(s[0]), "+r"(s[1]), "+r"(s[2]), "+r"(s[3]), "=r"(cout)
      : "r"(cin), "r"(u[0]), "r"(u[1]), "r"(u[2]), "r"(u[3]), "r"(take));
}
template <>
__device__ __forceinline__ void addc_words<8>(const uint32_t (&u)[8], uint32_t cin, uint32_t take, uint32_t (&s)[8],
                                              uint32_t& cout) {
  asm("{\n\t"
      ".reg .u32 t;\n\t"
      "add.cc.u32 t, %9, %18;\n\t"
      "addc.cc.u32 %0, %0, %10;\n\t"
      "addc.cc.u32 %1, %1, %11;\n\t"
      "addc.cc.u32 %2, %2, %12;\n\t"
      "addc.cc.u32 %3, %3, %13;\n\t"
      "addc.cc.u32 %4, %4, %14;\n\t"
      "addc.cc.u32 %5, %5, %15;\n\t"
      "addc.cc.u32 %6, %6, %16;\n\t"
      "addc.cc.u32 %7, %7, %17;\n\t"
      "addc.u32 %8, 0, 0;\n\t"
      "}"
      : "+r"(s[0]), "+r"(s[1]), "+r"(s[2]), "+r"(s[3]), "+r"(s[4]), "+r"(s[5]), "+r"(s[6]), "+r"(s[7]),
        "=r"(cout)
      : "r"(cin), "r"(u[0]), "r"(u[1]), "r"(u[2]), "r"(u[3]), "r"(u[4]), "r"(u[5]), "r"(u[6]), "r"(u[7]),
        "r"(take));
}

// K consecutive words from shared memory (8-byte aligned for K = 2, 16-byte aligned otherwise).
template <int K>
__device__ __forceinline__ void lds_words(const uint32_t* src, uint32_t (&P)[K]) {
  if constexpr (K == 2) {
    const uint2 q = *reinterpret_cast<const uint2*>(src);
    P[0] = q.x;
    P[1] = q.y;
  } else {
#pragma unroll
    for (int h = 0; h < K / 4; ++h) {
      const uint4 q = reinterpret_cast<const uint4*>(src)[h];
      P[4 * h] = q.x;
      P[4 * h + 1] = q.y;
      P[4 * h + 2] = q.z;
      P[4 * h + 3] = q.w;
    }
  }
}
template <int K>
__device__ __forceinline__ void sts_words(uint32_t* dst, const uint32_t (&v)[K]) {
  if constexpr (K == 2) {
    *reinterpret_cast<uint2*>(dst) = make_uint2(v[0], v[1]);
  } else {
#pragma unroll
    for (int h = 0; h < K / 4; ++h)
      reinterpret_cast<uint4*>(dst)[h] = make_uint4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
  }
}

// The rows of one item for one lane. STAGED: the masks come from the warp's shared stage (lane_stage points at this
// lane's K words of row 0; row r is 32K words further), else from the pair's table in L2. The masks of the next step
// are loaded one step ahead, the symbol codes eight steps ahead.
template <int K, bool STAGED>
__device__ __forceinline__ void run_rows(uint32_t (&V)[K], const uint32_t* lane_stage, const uint32_t* peq,
                                         uint64_t tab, uint32_t w, uint32_t w0, bool has, const uint16_t* xp,
                                         uint32_t jend, uint32_t gl, uint32_t take, uint32_t steps) {
  auto load_p = [&](uint32_t code, uint32_t (&P)[K]) {
    if (STAGED) {
      lds_words<K>(lane_stage + code * (32u * K), P);
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const uint32_t q = w0 + k;
        P[k] = (has && q < w) ? __ldg(peq + tab + (uint64_t)code * w + q) : 0u;
      }
    }
  };
  auto codes8 = [&](uint32_t t0, uint32_t (&c)[8]) {
    const uint32_t r0 = min(t0 + kCodePadFront - gl, jend);
#pragma unroll
    for (int b = 0; b < 8; ++b) c[b] = __ldg(xp + r0 + b);
  };
  uint32_t cin = 0;
  uint32_t cq[8], nq[8], P[K], Pn[K];
  codes8(0, cq);
  load_p(cq[0], Pn);
  for (uint32_t t0 = 0; t0 < steps; t0 += 8) {
    codes8(t0 + 8, nq);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
#pragma unroll
      for (int k = 0; k < K; ++k) P[k] = Pn[k];
      load_p(b + 1 < 8 ? cq[b + 1 < 8 ? b + 1 : 0] : nq[0], Pn);  // the next step's masks, one step ahead
      uint32_t U[K], S[K], cout;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        U[k] = V[k] & P[k];
        S[k] = V[k];
      }
      addc_words<K>(U, cin, take, S, cout);
      cin = __shfl_up_sync(kFull, cout, 1);
#pragma unroll
      for (int k = 0; k < K; ++k) V[k] = S[k] | (V[k] & ~P[k]);
    }
#pragma unroll
    for (int b = 0; b < 8; ++b) cq[b] = nq[b];
  }
}

// One work item with K words per lane (K is uniform over the warp: it comes from the item).
template <int K>
__device__ __forceinline__ void run_item(const BatchArgs& a, const BItem& item, uint32_t* stage, uint32_t lane) {
  const uint32_t G = item.G;
  const uint32_t grp = lane / G, gl = lane % G;
  const bool has = grp < item.count;
  BJob job{};
  BPair pr{};
  uint32_t sig = 0;
  if (has) {
    job = a.jobs[item.first + grp];
    pr = a.pairs[job.pair];
    sig = a.sigma[job.pair];
  }
  const uint64_t tab = job.rev ? pr.peqr_off : pr.peq_off;
  // lanes whose group has no job, or whose words lie beyond the pair's row, read the all-zero row / zero words
  const uint32_t w0 = gl * K;  // first word of this lane within its pair's row
  const uint32_t sig_max = __reduce_max_sync(kFull, has ? sig : 0u);
  const bool staged = (sig_max + 1) * 32u * K <= a.stage_words;
  if (staged) {
    // stage rows 0..sig_max: warp-row layout [row][lane * K + k]; rows above a pair's sigma read as zero
    __syncwarp();
    for (uint32_t r = 0; r <= sig_max; ++r) {
      uint32_t v[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const uint32_t q = w0 + k;
        v[k] = (has && r <= sig && q < pr.w) ? a.peq[tab + (uint64_t)r * pr.w + q] : 0u;
      }
      sts_words<K>(&stage[r * 32u * K + lane * K], v);
    }
    __syncwarp();
  }
  // Lane gl of a group works on row t - gl at step t (a skew of one row per lane), so the carry out of its 32K
  // bits for that row reaches lane gl + 1 by one shuffle, in time for the same row at step t + 1. Rows before 0
  // or past the job read the zero-row codes around the job's list: a row without a match leaves V unchanged.
  // xp[r] is the code of row r - kCodePadFront; lanes without a job read the zeros at the start of xcode (code 0,
  // whose staged row is zero for them).
  const uint16_t* xp = has ? a.xcode + (job.rev ? pr.xcr : pr.xcf) - kCodePadFront : a.xcode;
  const uint32_t jend = has ? job.rows + kCodePadFront : 0u;  // rows from here on read the padding only
  const uint32_t take = gl ? kFull : 0u;  // the first lane of a group starts every row without a carry
  const uint32_t steps = (item.rows + G - 1 + 7) & ~7u;
  uint32_t V[K];
#pragma unroll
  for (int k = 0; k < K; ++k) V[k] = kFull;
  if (staged)
    run_rows<K, true>(V, stage + lane * K, a.peq, tab, pr.w, w0, has, xp, jend, gl, take, steps);
  else
    run_rows<K, false>(V, stage + lane * K, a.peq, tab, pr.w, w0, has, xp, jend, gl, take, steps);
  if (has && pr.mt < pr.m) {
    // a split pair: keep the job's final row for the combine kernel (words gl*K .. gl*K+K-1 < kRowWords)
    uint32_t* dst = a.fvbuf + (uint64_t)(pr.fv + job.rev) * kRowWords + w0;
    if constexpr (K == 2) {
      *reinterpret_cast<uint2*>(dst) = make_uint2(V[0], V[1]);
    } else {
#pragma unroll
      for (int h = 0; h < K / 4; ++h)
        reinterpret_cast<uint4*>(dst)[h] = make_uint4(V[4 * h], V[4 * h + 1], V[4 * h + 2], V[4 * h + 3]);
    }
  } else if (has) {
    // c[m, n] = zero bits of V over the pair's n columns (bits past n stay 1): every lane of the group adds its
    // share to the length, which starts at zero
    uint32_t z = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) z += __popc(~V[k]);
    if (z) atomicAdd(reinterpret_cast<unsigned long long*>(a.out_lens + pr.out), (unsigned long long)z);
  }
}

__global__ void __launch_bounds__(kBatchWarps * 32) k_batch_main(BatchArgs a) {
  extern __shared__ __align__(16) uint32_t stage_dyn[];  // [kBatchWarps][stage_words]
  const uint32_t wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* stage = stage_dyn + wid * a.stage_words;
  for (;;) {
    uint32_t it = 0;
    if (lane == 0) it = atomicAdd(a.ticket, 1u);
    it = __shfl_sync(kFull, it, 0);
    if (it >= a.nitems) break;
    const BItem item = a.items[it];
    if (item.K == 8) run_item<8>(a, item, stage, lane);
    else if (item.K == 2) run_item<2>(a, item, stage, lane);
    else run_item<4>(a, item, stage, lane);
  }
}

// Split pairs: L = n - min over j of (ones of the forward row among its first j columns + ones of the reverse row
// among its first n - j columns). One warp per pair, prefix popcounts of the two rows in shared memory.
constexpr int kCW = kRowWords / 32;  // words of a final row per lane in the combine kernel

__global__ void __launch_bounds__(256) k_batch_combine(BatchArgs a) {
  __shared__ uint32_t pre_s[8][2][kRowWords + 1];  // ones among the first 32q columns, q = 0..128
  __shared__ uint32_t row_s[8][2][kRowWords];
  const uint32_t wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t k = blockIdx.x * (blockDim.x >> 5) + wid; k < a.nsplit; k += nwarps) {
    const BPair pr = a.pairs[a.split[k]];
    for (int d = 0; d < 2; ++d) {
      const uint4 v4 = *reinterpret_cast<const uint4*>(a.fvbuf + (uint64_t)(pr.fv + d) * kRowWords + lane * kCW);
      const uint32_t v[kCW] = {v4.x, v4.y, v4.z, v4.w};
      uint32_t c[kCW], sum = 0;
#pragma unroll
      for (int q = 0; q < kCW; ++q) {
        c[q] = __popc(v[q]);
        sum += c[q];
        row_s[wid][d][lane * kCW + q] = v[q];
      }
      uint32_t incl = sum;
      for (uint32_t off = 1; off < 32; off <<= 1) {
        const uint32_t o = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += o;
      }
      uint32_t run = incl - sum;
#pragma unroll
      for (int q = 0; q < kCW; ++q) {
        pre_s[wid][d][lane * kCW + q] = run;
        run += c[q];
      }
      if (lane == 31) pre_s[wid][d][kRowWords] = incl;
    }
    __syncwarp();
    auto ones = [&](int d, uint32_t x) {
      const uint32_t q = x >> 5, r = x & 31;
      return pre_s[wid][d][q] + (r ? __popc(row_s[wid][d][q] & ((1u << r) - 1u)) : 0u);
    };
    uint32_t best = 0xFFFFFFFFu;
    for (uint32_t j = lane; j <= pr.n; j += 32) {
      const uint32_t t = ones(0, j) + ones(1, pr.n - j);
      best = t < best ? t : best;
    }
    best = __reduce_min_sync(kFull, best);
    if (lane == 0) a.out_lens[pr.out] = pr.n - best;
    __syncwarp();
  }
}

}  // namespace

namespace lcs {
int run_length(lcs_ctx* c, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n, uint64_t* d_out,
               cudaStream_t st);

// Shared memory of the persistent row kernel: a stage of kStageRows mask rows of 32 * k_max words per warp.
inline uint32_t stage_words_for(uint32_t k_max) { return (uint32_t)kStageRows * 32u * k_max; }
inline size_t main_smem_bytes(uint32_t k_max) { return (size_t)kBatchWarps * stage_words_for(k_max) * 4u; }
inline int k_index(uint32_t k) { return k >= 8 ? 2 : (k >= 4 ? 1 : 0); }

// Resident blocks of the persistent row kernel per SM: the configured number (one by default: 8 warps, two per
// scheduler), up to the occupancy limit of the plan's stage size. The ALU work of the bulk of the items keeps two
// warps per scheduler busy, and the longest items, whose serial chains of rows end the launch, then share their
// schedulers with one other warp instead of three (measured: 0.180 ms against 0.201 ms with two blocks for the
// 10000-pair workload). The split of long pairs assumes the occupancy limit at 4 words per lane, so that items
// stay short.
static int batch_blocks_per_sm(lcs_ctx* c, int occ) {
  const int want = c->batch_blocks_per_sm > 0 ? c->batch_blocks_per_sm : 1;
  return want < occ ? want : occ;
}

// Device facts the batch launches need, looked up once per context: SMs, prep occupancy, and the row kernel's
// occupancy for each stage size (largest words per lane 2, 4, 8).
static cudaError_t batch_geometry(lcs_ctx* c) {
  if (c->b_sms > 0) return cudaSuccess;
  static std::atomic<uint64_t> attr_done{0};
  cudaError_t e = once_per_device_attr(
      [] {
        return cudaFuncSetAttribute(k_batch_main, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)main_smem_bytes(8));
      },
      attr_done);
  int sms = 0, prep_per_sm = 0, occ[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&prep_per_sm, k_batch_prep, 256, 0);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[i], k_batch_main, kBatchWarps * 32,
                                                      main_smem_bytes(2u << i));
  if (e != cudaSuccess) return e;
  c->b_sms = std::max(sms, 1);
  c->b_prep_per_sm = std::max(prep_per_sm, 1);
  for (int i = 0; i < 3; ++i) c->b_main_occ_k[i] = std::max(occ[i], 1);
  c->b_main_occ = c->b_main_occ_k[1];
  return cudaSuccess;
}

// The launches of a planned batch: zero the outputs, per-pair prep, the persistent kernel, the join of split pairs
// (stage events around them when profiling). Returns the first error.
static cudaError_t batch_launches(lcs_ctx* c, uint64_t* d_out, uint64_t count, const BatchArgs& a, cudaStream_t st,
                                  bool marks) {
  if (marks) c->mark(0, st);
  cudaError_t e = cudaMemsetAsync(d_out, 0, count * sizeof(uint64_t), st);  // empty pairs: length 0
  if (e == cudaSuccess && a.npairs) {
    e = cudaMemsetAsync(a.ticket, 0, 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.xcode, 0, kCodeZeros * sizeof(uint16_t), st);
    if (e != cudaSuccess) return e;
    const uint64_t sms = (uint64_t)c->b_sms;
    const unsigned prep_blocks = (unsigned)std::min<uint64_t>((a.npairs + 7) / 8, sms * c->b_prep_per_sm);
    k_batch_prep<<<prep_blocks, 256, 0, st>>>(a);
    const uint32_t k_max = a.stage_words / (32u * kStageRows);
    // persistent blocks: one wave over the SMs, but no more than the items need (a small batch then starts at
    // once on the SMs that are free instead of waiting for blocks that would find no work)
    const unsigned blocks = (unsigned)std::min<uint64_t>(sms * batch_blocks_per_sm(c, c->b_main_occ_k[k_index(k_max)]),
                                                         (a.nitems + kBatchWarps - 1) / kBatchWarps);
    if (marks) c->mark(1, st);
    k_batch_main<<<blocks, kBatchWarps * 32, main_smem_bytes(k_max), st>>>(a);
    if (a.nsplit) k_batch_combine<<<(unsigned)std::min<uint64_t>((a.nsplit + 7) / 8, sms * 8), 256, 0, st>>>(a);
    if (marks) c->mark(2, st);
    c->bblocks = blocks;
    e = cudaGetLastError();
  } else if (marks) {
    c->mark(1, st);
    c->mark(2, st);
  }
  return e;
}

// Uploads the plan's parts to c->bplan at their byte offsets: packed into the context's pinned plan buffer and sent
// with one asynchronous copy (the previous upload from that buffer is waited for before it is overwritten), or,
// when no pinned buffer can be had, with one copy per part from the host vectors (the runtime stages those).
static int upload_plan(lcs_ctx* c, const Plan& plan, size_t jat, size_t iat, size_t sat, size_t oat,
                       cudaStream_t st) {
  const size_t pb = plan.pairs.size() * sizeof(BPair), jb = plan.jobs.size() * sizeof(BJob),
               ib = plan.items.size() * sizeof(BItem), sb = plan.split.size() * 4, ob = plan.prep_order.size() * 4;
  const size_t total = oat + ob;
  char* base = (char*)c->bplan.p;
  bool pinned = true;
  if (c->hplan_ev) pinned = cudaEventSynchronize(c->hplan_ev) == cudaSuccess;  // the last upload has left hplan
  if (pinned && !c->hplan_ev) pinned = cudaEventCreateWithFlags(&c->hplan_ev, cudaEventDisableTiming) == cudaSuccess;
  if (pinned && total > c->hplan_cap) {
    if (c->hplan) cudaFreeHost(c->hplan);
    c->hplan = nullptr;
    c->hplan_cap = 0;
    void* p = nullptr;
    const size_t want = std::max<size_t>(total + total / 4, 1 << 16);
    if (cudaMallocHost(&p, want) == cudaSuccess) {
      c->hplan = static_cast<uint8_t*>(p);
      c->hplan_cap = want;
    } else {
      cudaGetLastError();  // clear the failed allocation; fall back to pageable copies
      pinned = false;
    }
  }
  if (pinned) {
    std::memcpy(c->hplan, plan.pairs.data(), pb);
    std::memcpy(c->hplan + jat, plan.jobs.data(), jb);
    std::memcpy(c->hplan + iat, plan.items.data(), ib);
    if (sb) std::memcpy(c->hplan + sat, plan.split.data(), sb);
    std::memcpy(c->hplan + oat, plan.prep_order.data(), ob);
    int rc = from_cuda(cudaMemcpyAsync(base, c->hplan, total, cudaMemcpyHostToDevice, st));
    if (!rc) rc = from_cuda(cudaEventRecord(c->hplan_ev, st));
    return rc;
  }
  // (copies from pageable memory: the runtime has staged the data when the call returns)
  int rc = from_cuda(cudaMemcpyAsync(base, plan.pairs.data(), pb, cudaMemcpyHostToDevice, st));
  if (!rc) rc = from_cuda(cudaMemcpyAsync(base + jat, plan.jobs.data(), jb, cudaMemcpyHostToDevice, st));
  if (!rc) rc = from_cuda(cudaMemcpyAsync(base + iat, plan.items.data(), ib, cudaMemcpyHostToDevice, st));
  if (!rc && sb) rc = from_cuda(cudaMemcpyAsync(base + sat, plan.split.data(), sb, cudaMemcpyHostToDevice, st));
  if (!rc) rc = from_cuda(cudaMemcpyAsync(base + oat, plan.prep_order.data(), ob, cudaMemcpyHostToDevice, st));
  return rc;
}

// Grows every buffer a host-buffer batch call (lcs_batch) uses for batches of at most max_pairs pairs with at most
// x_bytes symbols of X and y_bytes of Y in all, every y at most 4096 symbols, so that such calls allocate nothing:
// the plan and its pinned upload buffer, the alphabet sizes, the padded code lists (every pair's list padded at both
// ends and aligned, twice for a split pair), the match-mask tables (at most (256 + 1) * ceil(n / 32) words per pair,
// twice for a split pair: under 17 words per symbol of Y plus 520 per pair), the split pairs' final rows, the
// device copies of the inputs and the lengths, and the pinned staging area.
int batch_presize(lcs_ctx* c, uint64_t max_pairs, uint64_t x_bytes, uint64_t y_bytes) {
  int rc = from_cuda(batch_geometry(c));
  const uint64_t P = std::max<uint64_t>(max_pairs, 1);
  const size_t plan_bytes = P * sizeof(BPair) + 2 * P * sizeof(BJob) + 2 * P * sizeof(BItem) + 2 * P * 4 + 6 * 256;
  const uint64_t codes = kCodeZeros + x_bytes + 2 * P * (kCodePadFront + 15 + kCodePadBack);
  if (!rc) rc = from_cuda(ensure(c->bplan, plan_bytes));
  if (!rc) rc = from_cuda(ensure(c->bsig, P * 4 + 4));
  if (!rc) rc = from_cuda(ensure(c->bxcode, (codes + 16) * 2));
  if (!rc) rc = from_cuda(ensure(c->bpeq, (17 * y_bytes + 520 * P + 4) * 4));
  if (!rc) rc = from_cuda(ensure(c->bfv, ((uint64_t)2 * P * kRowWords + 4) * 4));
  if (!rc) rc = from_cuda(ensure(c->x, std::max<uint64_t>(x_bytes, 1)));
  if (!rc) rc = from_cuda(ensure(c->y, std::max<uint64_t>(y_bytes, 1)));
  if (!rc) rc = from_cuda(ensure(c->bout, P * 8));
  if (!rc) rc = ensure_hstage(c, x_bytes + y_bytes + P * 8 + 8);
  if (!rc && plan_bytes > c->hplan_cap) {
    if (c->hplan_ev) cudaEventSynchronize(c->hplan_ev);
    if (c->hplan) cudaFreeHost(c->hplan);
    c->hplan = nullptr;
    c->hplan_cap = 0;
    void* p = nullptr;
    rc = from_cuda(cudaMallocHost(&p, plan_bytes));
    if (!rc) {
      c->hplan = static_cast<uint8_t*>(p);
      c->hplan_cap = plan_bytes;
    }
  }
  return rc;
}

// Runs a batch whose xs / ys / out_lens are already on the device. The first call of a batch plans it on the host,
// uploads the plan and launches; a later call with the same pairs (same offsets and buffers) reuses the plan, and
// without profiling its launches are captured once as a CUDA graph and replayed.
int run_batch(lcs_ctx* c, const uint8_t* d_xs, const uint8_t* d_ys, const uint64_t* x_off, const uint64_t* y_off,
              uint64_t count, uint64_t* d_out, cudaStream_t st) {
  // the same batch as the last call: same buffers, same count and the same offsets relative to the first
  const uint64_t ptrs[4] = {count, (uint64_t)d_xs, (uint64_t)d_ys, (uint64_t)d_out};
  bool same = c->bvalid && std::memcmp(ptrs, c->bptrs, sizeof(ptrs)) == 0;
  for (uint64_t k = 0; same && k <= count; ++k)
    same = c->boffs[2 * k] == x_off[k] - x_off[0] && c->boffs[2 * k + 1] == y_off[k] - y_off[0];
  int rc = LCS_OK;
  const bool fresh = !same;
  if (fresh) {
    if (c->bexec) cudaGraphExecDestroy(c->bexec);
    c->bexec = nullptr;
    c->bvalid = false;
    Plan plan;
    c->bbig.clear();
    rc = from_cuda(batch_geometry(c));
    if (rc) return rc;
    make_plan(x_off, y_off, count, (uint64_t)c->b_sms * c->b_main_occ * kBatchWarps, c->batch_k, c->batch_split_pct,
              plan, c->bbig);
    c->bk_max = plan.k_max;
    c->bcells = 0;
    for (uint64_t k = 0; k < count; ++k) c->bcells += (x_off[k + 1] - x_off[k]) * (y_off[k + 1] - y_off[k]);
    const size_t pb = plan.pairs.size() * sizeof(BPair), jb = plan.jobs.size() * sizeof(BJob),
                 ib = plan.items.size() * sizeof(BItem), sb = plan.split.size() * 4,
                 ob = plan.prep_order.size() * 4;
    const size_t jat = (pb + 255) & ~(size_t)255, iat = (jat + jb + 255) & ~(size_t)255,
                 sat = (iat + ib + 255) & ~(size_t)255, oat = (sat + sb + 255) & ~(size_t)255;
    if (!plan.pairs.empty()) {
      rc = from_cuda(ensure(c->bplan, oat + ob + 256));
      if (!rc) rc = from_cuda(ensure(c->bsig, plan.pairs.size() * 4 + 4));
      if (!rc) rc = from_cuda(ensure(c->bxcode, (plan.codes + 16) * 2));
      if (!rc) rc = from_cuda(ensure(c->bpeq, plan.peq_words * 4 + 4));
      if (!rc) rc = from_cuda(ensure(c->bfv, ((uint64_t)plan.fv_slots * kRowWords + 4) * 4));
      if (rc) return rc;
      rc = upload_plan(c, plan, jat, iat, sat, oat, st);
      if (rc) return rc;
    }
    c->bnpairs = plan.pairs.size();
    c->bnitems = plan.items.size();
    c->bnsplit = plan.split.size();
    c->bjobs_at = jat;
    c->bitems_at = iat;
    c->bsplit_at = sat;
    c->border_at = oat;
    std::memcpy(c->bptrs, ptrs, sizeof(ptrs));
    c->boffs.resize(2 * (count + 1));
    for (uint64_t k = 0; k <= count; ++k) {
      c->boffs[2 * k] = x_off[k] - x_off[0];
      c->boffs[2 * k + 1] = y_off[k] - y_off[0];
    }
    c->bvalid = true;
  }
  BatchArgs a{};
  a.xs = d_xs;
  a.ys = d_ys;
  a.pairs = (const BPair*)c->bplan.p;
  a.jobs = (const BJob*)((char*)c->bplan.p + c->bjobs_at);
  a.items = (const BItem*)((char*)c->bplan.p + c->bitems_at);
  a.split = (const uint32_t*)((char*)c->bplan.p + c->bsplit_at);
  a.prep_order = (const uint32_t*)((char*)c->bplan.p + c->border_at);
  a.fvbuf = (uint32_t*)c->bfv.p;
  a.sigma = (uint32_t*)c->bsig.p;
  // xcode + xcf is then a multiple of 32 bytes where xs + x_off is a multiple of 16
  a.xcode = (uint16_t*)c->bxcode.p + ((uintptr_t)d_xs & 15u);
  a.peq = (uint32_t*)c->bpeq.p;
  a.out_lens = d_out;
  a.ticket = (uint32_t*)((char*)c->small.p + kOffTicket);
  a.npairs = (uint32_t)c->bnpairs;
  a.nitems = (uint32_t)c->bnitems;
  a.nsplit = (uint32_t)c->bnsplit;
  a.stage_words = stage_words_for(c->bk_max);
  if (c->prof || fresh) {
    rc = from_cuda(batch_launches(c, d_out, count, a, st, c->prof));
  } else {
    if (!c->bexec) {
      if (!c->cap_stream) {
        rc = from_cuda(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        if (rc) return rc;
      }
      // capture: the recorded launches do not run now; the graph runs on st below
      rc = from_cuda(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      if (rc) return rc;
      const cudaError_t le = batch_launches(c, d_out, count, a, c->cap_stream, false);
      cudaGraph_t graph = nullptr;
      rc = from_cuda(cudaStreamEndCapture(c->cap_stream, &graph));
      if (!rc && le != cudaSuccess) rc = from_cuda(le);
      if (!rc) rc = from_cuda(cudaGraphInstantiate(&c->bexec, graph, 0));
      if (graph) cudaGraphDestroy(graph);
      if (rc) {
        c->bexec = nullptr;
        return rc;
      }
    }
    rc = from_cuda(cudaGraphLaunch(c->bexec, st));
  }
  if (rc) return rc;
  // pairs with more than 4096 columns go through the single-pair path
  for (uint64_t k : c->bbig) {
    rc = run_length(c, d_xs + (x_off[k] - x_off[0]), x_off[k + 1] - x_off[k], d_ys + (y_off[k] - y_off[0]),
                    y_off[k + 1] - y_off[k], d_out + k, st);
    if (rc) return rc;
  }
  if (c->prof) {
    c->mark(3, st);
    c->prof_valid = true;
    c->prof_trace = false;
    c->prof_cells = c->bcells;
    c->prof_blocks = c->bblocks;
  }
  return LCS_OK;
}

}  // namespace lcs

static bool offsets_ok(const uint64_t* off, uint64_t count) {
  for (uint64_t k = 0; k < count; ++k)
    if (off[k + 1] < off[k]) return false;
  return true;
}

static int lcs_batch_dev_impl(lcs_ctx* c, const uint8_t* d_xs, const uint64_t* d_x_off, const uint8_t* d_ys,
                             const uint64_t* d_y_off, uint64_t count, uint64_t* d_out_lens, void* stream) {
  if (!c || (count && (!d_x_off || !d_y_off || !d_out_lens))) return LCS_ERR_INVALID;
  if (count == 0) return LCS_OK;
  std::lock_guard<std::mutex> g(c->mu);
  cudaSetDevice(c->device);
  cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
  // the plan is made on the host, so the offsets come back first
  std::vector<uint64_t> xo(count + 1), yo(count + 1);
  int rc = from_cuda(cudaMemcpyAsync(xo.data(), d_x_off, (count + 1) * 8, cudaMemcpyDeviceToHost, st));
  if (!rc) rc = from_cuda(cudaMemcpyAsync(yo.data(), d_y_off, (count + 1) * 8, cudaMemcpyDeviceToHost, st));
  if (!rc) rc = from_cuda(cudaStreamSynchronize(st));
  if (rc) return rc;
  if (!offsets_ok(xo.data(), count) || !offsets_ok(yo.data(), count)) return LCS_ERR_INVALID;
  return run_batch(c, d_xs + xo[0], d_ys + yo[0], xo.data(), yo.data(), count, d_out_lens, st);
}

extern "C" int lcs_batch_dev(lcs_ctx* c, const uint8_t* d_xs, const uint64_t* d_x_off, const uint8_t* d_ys,
                             const uint64_t* d_y_off, uint64_t count, uint64_t* d_out_lens, void* stream) {
  try {  // no C++ exception crosses the C boundary
    return lcs_batch_dev_impl(c, d_xs, d_x_off, d_ys, d_y_off, count, d_out_lens, stream);
  } catch (const std::bad_alloc&) {
    return LCS_ERR_NOMEM;
  } catch (...) {
    return LCS_ERR_INTERNAL;
  }
}

// Device strings and lengths, host offsets: the plan is made from offsets the caller already holds, so nothing is
// copied back and the stream is not waited on; the call returns once the batch is enqueued.
static int lcs_batch_dev_hoff_impl(lcs_ctx* c, const uint8_t* d_xs, const uint64_t* x_off, const uint8_t* d_ys,
                                   const uint64_t* y_off, uint64_t count, uint64_t* d_out_lens, void* stream) {
  if (!c || (count && (!x_off || !y_off || !d_out_lens))) return LCS_ERR_INVALID;
  if (count == 0) return LCS_OK;
  if (!offsets_ok(x_off, count) || !offsets_ok(y_off, count)) return LCS_ERR_INVALID;
  if ((x_off[count] > x_off[0] && !d_xs) || (y_off[count] > y_off[0] && !d_ys)) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  cudaSetDevice(c->device);
  cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
  return run_batch(c, d_xs + x_off[0], d_ys + y_off[0], x_off, y_off, count, d_out_lens, st);
}

extern "C" int lcs_batch_dev_hoff(lcs_ctx* c, const uint8_t* d_xs, const uint64_t* x_off, const uint8_t* d_ys,
                                  const uint64_t* y_off, uint64_t count, uint64_t* d_out_lens, void* stream) {
  try {  // no C++ exception crosses the C boundary
    return lcs_batch_dev_hoff_impl(c, d_xs, x_off, d_ys, y_off, count, d_out_lens, stream);
  } catch (const std::bad_alloc&) {
    return LCS_ERR_NOMEM;
  } catch (...) {
    return LCS_ERR_INTERNAL;
  }
}

// The address at which the current device reads host memory [p, p + bytes) when that range is page-locked and
// mapped into the device's address space (its first and last byte are, at consistent addresses), else nullptr.
static const uint8_t* mapped_view(const uint8_t* p, uint64_t bytes) {
  if (!p || bytes == 0) return nullptr;
  cudaPointerAttributes a{}, b{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaPointerGetAttributes(&b, p + (bytes - 1)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
    return nullptr;
  const uint8_t* d = static_cast<const uint8_t*>(a.devicePointer);
  return static_cast<const uint8_t*>(b.devicePointer) == d + (bytes - 1) ? d : nullptr;
}

static int lcs_batch_impl(lcs_ctx* c, const uint8_t* xs, const uint64_t* x_off, const uint8_t* ys,
                         const uint64_t* y_off, uint64_t count, uint64_t* out_lens) {
  if (!c || (count && (!x_off || !y_off || !out_lens))) return LCS_ERR_INVALID;
  if (count == 0) return LCS_OK;
  if (!offsets_ok(x_off, count) || !offsets_ok(y_off, count)) return LCS_ERR_INVALID;
  const uint64_t nx = x_off[count] - x_off[0], ny = y_off[count] - y_off[0];
  if ((nx && !xs) || (ny && !ys)) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  cudaSetDevice(c->device);
  const uint8_t* sx = xs + x_off[0];
  const uint8_t* sy = ys + y_off[0];
  // Page-locked strings are read where they are: the kernels load them over the host link instead of a copy into
  // device buffers first. The per-pair preparation, the one pass over the strings, then overlaps their transfer
  // (the link moves about 200 GB/s either way on a GB300 node, ~0.1 ms for the 19.4 MB of the 10,000-pair batch).
  const uint8_t* vx = mapped_view(sx, nx);
  const uint8_t* vy = vx ? mapped_view(sy, ny) : nullptr;
  const bool in_place = vx && vy;
  int rc = in_place ? LCS_OK : from_cuda(ensure(c->x, std::max<uint64_t>(nx, 1)));
  if (!rc && !in_place) rc = from_cuda(ensure(c->y, std::max<uint64_t>(ny, 1)));
  if (!rc) rc = from_cuda(ensure(c->bout, count * 8));
  if (rc) return rc;
  // small pageable batches go through the context's pinned staging area (host copies, then asynchronous copies)
  const bool stage = !in_place && nx + ny + count * 8 <= kStageBytesMax && !(nx && host_pinned(sx)) &&
                     ensure_hstage(c, nx + ny + count * 8) == LCS_OK;
  if (stage) {
    if (nx) std::memcpy(c->hstage, sx, nx);
    if (ny) std::memcpy(c->hstage + nx, sy, ny);
    sx = c->hstage;
    sy = c->hstage + nx;
  }
  if (!in_place && nx) rc = from_cuda(cudaMemcpyAsync(c->x.p, sx, nx, cudaMemcpyHostToDevice, c->stream));
  if (!rc && !in_place && ny) rc = from_cuda(cudaMemcpyAsync(c->y.p, sy, ny, cudaMemcpyHostToDevice, c->stream));
  if (!rc)
    rc = run_batch(c, in_place ? vx : (const uint8_t*)c->x.p, in_place ? vy : (const uint8_t*)c->y.p, x_off, y_off,
                   count, (uint64_t*)c->bout.p, c->stream);
  // the lengths come back through page-locked memory (a copy into pageable memory would go through the CUDA
  // runtime's own staging, synchronously): behind the staged strings, or at the start of the staging area when the
  // strings did not use it (nothing of this call reads it then)
  uint64_t* land = stage ? reinterpret_cast<uint64_t*>(c->hstage + ((nx + ny + 7) & ~(uint64_t)7)) : out_lens;
  if (stage && (uint8_t*)(land + count) > c->hstage + c->hstage_cap) land = out_lens;
  if (!rc && !stage && count * 8 <= kStageBytesMax && !host_pinned(out_lens) && ensure_hstage(c, count * 8) == LCS_OK)
    land = reinterpret_cast<uint64_t*>(c->hstage);
  if (!rc) rc = from_cuda(cudaMemcpyAsync(land, c->bout.p, count * 8, cudaMemcpyDeviceToHost, c->stream));
  if (!rc) rc = fetch_status(c);  // the status word behind the lengths, one wait for both
  if (!rc && land != out_lens) std::memcpy(out_lens, land, count * 8);
  return rc;
}

extern "C" int lcs_batch(lcs_ctx* c, const uint8_t* xs, const uint64_t* x_off, const uint8_t* ys,
                         const uint64_t* y_off, uint64_t count, uint64_t* out_lens) {
  try {  // no C++ exception crosses the C boundary
    return lcs_batch_impl(c, xs, x_off, ys, y_off, count, out_lens);
  } catch (const std::bad_alloc&) {
    return LCS_ERR_NOMEM;
  } catch (...) {
    return LCS_ERR_INTERNAL;
  }
}

// ---- batch configuration and autotuning ---------------------------------------------------------------------------

static bool valid_batch_config(const lcs_batch_config* b) {
  return b && (b->words_per_lane == 2 || b->words_per_lane == 4 || b->words_per_lane == 8) && b->split_pct <= 1000 &&
         (b->blocks_per_sm == 1 || b->blocks_per_sm == 2) && b->reserved == 0;
}

static lcs_batch_config current_batch_config(const lcs_ctx* c) {
  lcs_batch_config b{};
  b.words_per_lane = c->batch_k;
  b.split_pct = c->batch_split_pct;
  b.blocks_per_sm = c->batch_blocks_per_sm > 1 ? 2u : 1u;
  return b;
}

static void apply_batch_config(lcs_ctx* c, const lcs_batch_config& b) {
  if (b.words_per_lane != c->batch_k || b.split_pct != c->batch_split_pct) c->bvalid = false;  // re-plan
  if ((int)b.blocks_per_sm != (c->batch_blocks_per_sm > 1 ? 2 : 1)) c->bvalid = false;  // re-capture the launches
  c->batch_k = b.words_per_lane;
  c->batch_split_pct = b.split_pct;
  c->batch_blocks_per_sm = (int)b.blocks_per_sm;
}

extern "C" int lcs_ctx_get_batch_config(lcs_ctx* c, lcs_batch_config* out) {
  if (!c || !out) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  *out = current_batch_config(c);
  return LCS_OK;
}

extern "C" int lcs_ctx_set_batch_config(lcs_ctx* c, const lcs_batch_config* cfg) {
  if (!c || !valid_batch_config(cfg)) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  apply_batch_config(c, *cfg);
  return LCS_OK;
}

static int autotune_batch_impl(lcs_ctx* c, const uint8_t* d_xs, const uint64_t* d_x_off, const uint8_t* d_ys,
                               const uint64_t* d_y_off, uint64_t count, uint64_t* d_out, void* stream,
                               lcs_batch_config* best, double* best_ms) {
  if (!c || (count && (!d_x_off || !d_y_off || !d_out))) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  cudaSetDevice(c->device);
  cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
  const lcs_batch_config keep = current_batch_config(c);
  if (count == 0) {
    if (best) *best = keep;
    if (best_ms) *best_ms = 0.0;
    return LCS_OK;
  }
  std::vector<uint64_t> xo(count + 1), yo(count + 1);
  int rc = from_cuda(cudaMemcpyAsync(xo.data(), d_x_off, (count + 1) * 8, cudaMemcpyDeviceToHost, st));
  if (!rc) rc = from_cuda(cudaMemcpyAsync(yo.data(), d_y_off, (count + 1) * 8, cudaMemcpyDeviceToHost, st));
  if (!rc) rc = from_cuda(cudaStreamSynchronize(st));
  if (rc) return rc;
  if (!offsets_ok(xo.data(), count) || !offsets_ok(yo.data(), count)) return LCS_ERR_INVALID;
  const bool prof = c->prof;
  c->prof = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  rc = from_cuda(cudaEventCreate(&e0));
  if (!rc) rc = from_cuda(cudaEventCreate(&e1));
  std::vector<uint64_t> first(count), now(count);
  bool have_first = false;
  double bt = 1e300;
  lcs_batch_config bc = keep;
  const uint32_t ks[3] = {2, 4, 8}, splits[4] = {50, 100, 200, 0}, bps[2] = {1, 2};
  for (uint32_t k : ks) {
    for (uint32_t sp : splits) {
      for (uint32_t bp : bps) {
        if (rc) break;
        const lcs_batch_config cand{k, sp, bp, 0};
        apply_batch_config(c, cand);
        double ts[5];
        for (int r = 0; r < 5 && !rc; ++r) {  // call 0 plans, call 1 captures the graph; calls 2-4 replay it
          rc = from_cuda(cudaEventRecord(e0, st));
          if (!rc) rc = run_batch(c, d_xs + xo[0], d_ys + yo[0], xo.data(), yo.data(), count, d_out, st);
          if (!rc) rc = from_cuda(cudaEventRecord(e1, st));
          if (!rc) rc = from_cuda(cudaEventSynchronize(e1));
          if (!rc) rc = take_status(c);
          float ms = 0.f;
          if (!rc) rc = from_cuda(cudaEventElapsedTime(&ms, e0, e1));
          ts[r] = ms;
        }
        if (rc) break;
        // every configuration must give the same lengths
        rc = from_cuda(cudaMemcpy((have_first ? now : first).data(), d_out, count * 8, cudaMemcpyDeviceToHost));
        if (rc) break;
        if (have_first && std::memcmp(first.data(), now.data(), count * 8) != 0) {
          rc = LCS_ERR_INTERNAL;
          break;
        }
        have_first = true;
        std::sort(ts + 2, ts + 5);
        if (ts[3] < bt) {
          bt = ts[3];
          bc = cand;
        }
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->prof = prof;
  apply_batch_config(c, rc ? keep : bc);
  if (rc) return rc;
  if (best) *best = bc;
  if (best_ms) *best_ms = bt;
  return LCS_OK;
}

extern "C" int lcs_ctx_autotune_batch_dev(lcs_ctx* c, const uint8_t* d_xs, const uint64_t* d_x_off,
                                          const uint8_t* d_ys, const uint64_t* d_y_off, uint64_t count,
                                          uint64_t* d_out_lens, void* stream, lcs_batch_config* best,
                                          double* best_ms) {
  try {  // no C++ exception crosses the C boundary
    return autotune_batch_impl(c, d_xs, d_x_off, d_ys, d_y_off, count, d_out_lens, stream, best, best_ms);
  } catch (const std::bad_alloc&) {
    return LCS_ERR_NOMEM;
  } catch (...) {
    return LCS_ERR_INTERNAL;
  }
}
