// lcs_batch: LCS lengths (c[m,n], paper §I.C) of many independent pairs in one persistent launch.
//
// Every pair is a small instance of the same bit-parallel row update as the single-pair fill (U = V & P;
// S = V + U; V' = S | (V & ~P), one 32-column word per register). Here the rows of a pair are processed
// row-synchronously by a group of G lanes of a warp, each lane holding K = 4 consecutive words of the row:
//   * the add inside a lane ripples through its 4 words with the carry flag;
//   * the carries between the lanes of a group are resolved per row by a carry-lookahead over warp ballots:
//     with g = "the lane's 128-bit add generates a carry" and p = "it would pass an incoming carry on", the
//     carries into all lanes are ((A + B) ^ A ^ B) for A = g | p, B = g, with the groups' top lanes masked so that
//     no carry crosses from one pair into the next;
//   * a warp works on 32 / G pairs of the same group size at once, G chosen per pair as the smallest power of two
//     with 4 * G words >= ceil(n / 32) (so short pairs share a warp and long pairs spread over it).
// The host plans the launch: it buckets pairs by G, orders work items (up to 32 / G pairs each) by decreasing
// rows, and a persistent kernel lets every warp take the next item from an atomic ticket.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "lcs_ctx.h"

namespace lcs {
int take_status(lcs_ctx* c);
}  // namespace lcs

namespace {

using namespace lcs;

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr int kBK = 4;             // words per lane
constexpr int kWarpWords = 32 * kBK;  // 128 words per warp row
constexpr int kBatchWarps = 8;     // warps per block of the persistent kernel
constexpr int kStageRows = 24;     // match-mask rows staged in shared memory per warp (alphabets up to 23 symbols)

struct BPair {        // one pair of the plan, in processing order
  uint64_t x_off;     // first symbol of x in xs (and its codes in xcode)
  uint64_t y_off;
  uint64_t peq_off;   // word offset of its match-mask table: (sigma + 1) rows of w words
  uint32_t m, n, w;   // rows, columns, words per row (ceil(n / 32))
  uint32_t out;       // index into out_lens
};

struct BItem {        // a warp's unit of work: pairs [first, first + count) of the plan, G lanes each
  uint32_t first, count, G, rows;
};

struct BatchArgs {
  const uint8_t* xs;
  const uint8_t* ys;
  const BPair* pairs;
  const BItem* items;
  uint32_t* sigma;     // per plan pair: symbols present in y (its zero row index)
  uint8_t* xcode;      // per symbol of xs: code in its pair's alphabet
  uint32_t* peq;
  uint64_t* out_lens;
  uint32_t* ticket;
  uint32_t npairs, nitems;
};

// ---- per-pair alphabet, symbol codes and match-mask table (one warp per pair) ------------------------------------
__global__ void __launch_bounds__(256) k_batch_prep(BatchArgs a) {
  __shared__ uint32_t pres_s[8][8];
  __shared__ uint8_t map_s[8][256];
  const uint32_t wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* pres = pres_s[wid];
  uint8_t* map = map_s[wid];
  const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t p = blockIdx.x * (blockDim.x >> 5) + wid; p < a.npairs; p += nwarps) {
    const BPair pr = a.pairs[p];
    if (lane < 8) pres[lane] = 0;
    __syncwarp();
    const uint8_t* y = a.ys + pr.y_off;
    for (uint32_t j = lane; j < pr.n; j += 32) atomicOr(&pres[y[j] >> 5], 1u << (y[j] & 31));
    __syncwarp();
    uint32_t sigma = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) sigma += __popc(pres[k]);
    for (uint32_t b = lane; b < 256; b += 32) {
      uint32_t below = 0;
      for (uint32_t k = 0; k < (b >> 5); ++k) below += __popc(pres[k]);
      below += __popc(pres[b >> 5] & ((1u << (b & 31)) - 1u));
      map[b] = (uint8_t)(((pres[b >> 5] >> (b & 31)) & 1u) ? below : sigma);
    }
    if (lane == 0) a.sigma[p] = sigma;
    __syncwarp();
    uint32_t* tab = a.peq + pr.peq_off;
    const uint64_t words = (uint64_t)(sigma + 1) * pr.w;
    for (uint64_t i = lane; i < words; i += 32) tab[i] = 0;
    __syncwarp();
    for (uint32_t q = 0; q < pr.w; ++q) {
      const uint32_t j = q * 32 + lane;
      const uint32_t code = j < pr.n ? map[y[j]] : 0xFFFFu;
      const uint32_t mask = __match_any_sync(kFull, code);
      if (code != 0xFFFFu && lane == (uint32_t)(__ffs(mask) - 1)) tab[(uint64_t)code * pr.w + q] = mask;
    }
    const uint8_t* x = a.xs + pr.x_off;
    uint8_t* xc = a.xcode + pr.x_off;
    for (uint32_t i = lane; i < pr.m; i += 32) xc[i] = map[x[i]];
    __syncwarp();
  }
}

// ---- the persistent batch kernel --------------------------------------------------------------------------------
__device__ __forceinline__ void add4(const uint32_t (&v)[kBK], const uint32_t (&u)[kBK], uint32_t (&s)[kBK],
                                     uint32_t& gen) {
  asm("add.cc.u32 %0, %5, %9;\n\t"
      "addc.cc.u32 %1, %6, %10;\n\t"
      "addc.cc.u32 %2, %7, %11;\n\t"
      "addc.cc.u32 %3, %8, %12;\n\t"
      "addc.u32 %4, 0, 0;"
      : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(gen)
      : "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(u[0]), "r"(u[1]), "r"(u[2]), "r"(u[3]));
}
__device__ __forceinline__ void inc4(uint32_t (&s)[kBK], uint32_t c) {
  asm("add.cc.u32 %0, %0, %4;\n\t"
      "addc.cc.u32 %1, %1, 0;\n\t"
      "addc.cc.u32 %2, %2, 0;\n\t"
      "addc.u32 %3, %3, 0;"
      : "+r"(s[0]), "+r"(s[1]), "+r"(s[2]), "+r"(s[3])
      : "r"(c));
}

__global__ void __launch_bounds__(kBatchWarps * 32) k_batch_main(BatchArgs a) {
  __shared__ __align__(16) uint32_t stage_s[kBatchWarps][kStageRows * kWarpWords];
  const uint32_t wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* stage = stage_s[wid];
  for (;;) {
    uint32_t it = 0;
    if (lane == 0) it = atomicAdd(a.ticket, 1u);
    it = __shfl_sync(kFull, it, 0);
    if (it >= a.nitems) break;
    const BItem item = a.items[it];
    const uint32_t G = item.G;
    const uint32_t grp = lane / G, gl = lane % G;
    const bool has = grp < item.count;
    BPair pr{};
    uint32_t sig = 0;
    if (has) {
      pr = a.pairs[item.first + grp];
      sig = a.sigma[item.first + grp];
    }
    // lanes whose group has no pair, or whose words lie beyond the pair's row, read the all-zero row / zero words
    const uint32_t w0 = gl * kBK;  // first word of this lane within its pair's row
    uint32_t sig_max = __reduce_max_sync(kFull, has ? sig : 0u);
    const bool staged = sig_max + 1 <= (uint32_t)kStageRows;
    if (staged) {
      // stage rows 0..sig_max: warp-row layout [row][lane * 4 + k]; rows above a pair's sigma read as zero
      __syncwarp();
      for (uint32_t r = 0; r <= sig_max; ++r) {
        uint32_t v[kBK];
#pragma unroll
        for (int k = 0; k < kBK; ++k) {
          const uint32_t q = w0 + k;
          v[k] = (has && r <= sig && q < pr.w) ? a.peq[pr.peq_off + (uint64_t)r * pr.w + q] : 0u;
        }
        *reinterpret_cast<uint4*>(&stage[r * kWarpWords + lane * kBK]) = make_uint4(v[0], v[1], v[2], v[3]);
      }
      __syncwarp();
    }
    // top lanes of the groups: their carries must not reach the next group
    uint32_t top = 0;
    for (uint32_t l = G - 1; l < 32; l += G) top |= 1u << l;
    const uint8_t* xc = a.xcode + pr.x_off;
    const uint32_t zero_code = sig;  // the all-zero row of this pair
    uint32_t V[kBK] = {kFull, kFull, kFull, kFull};
    const uint32_t rows = item.rows;
    // symbol codes are requested 8 rows before they are used (the rows beyond a pair's m read its zero row)
    auto codes8 = [&](uint32_t i0, uint32_t (&c)[8]) {
#pragma unroll
      for (int b = 0; b < 8; ++b) c[b] = (has && i0 + b < pr.m) ? (uint32_t)__ldg(xc + i0 + b) : zero_code;
    };
    uint32_t cq[8], nq[8];
    codes8(0, cq);
    for (uint32_t i0 = 0; i0 < rows; i0 += 8) {
      codes8(i0 + 8, nq);
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        if (i0 + b >= rows) break;  // warp-uniform
        const uint32_t code = cq[b];
        uint32_t P[kBK];
        if (staged) {
          const uint4 q = *reinterpret_cast<const uint4*>(&stage[code * kWarpWords + lane * kBK]);
          P[0] = q.x; P[1] = q.y; P[2] = q.z; P[3] = q.w;
        } else {
#pragma unroll
          for (int k = 0; k < kBK; ++k) {
            const uint32_t q = w0 + k;
            P[k] = (has && q < pr.w) ? __ldg(a.peq + pr.peq_off + (uint64_t)code * pr.w + q) : 0u;
          }
        }
        uint32_t U[kBK], S[kBK], gen;
#pragma unroll
        for (int k = 0; k < kBK; ++k) U[k] = V[k] & P[k];
        add4(V, U, S, gen);
        const uint32_t prop = (S[0] & S[1] & S[2] & S[3]) == kFull;
        const uint32_t Gb = __ballot_sync(kFull, gen), Pb = __ballot_sync(kFull, prop);
        const uint32_t A = (Gb | Pb) & ~top, Bv = Gb & ~top;
        const uint32_t cin = (((A + Bv) ^ A ^ Bv) >> lane) & 1u;
        inc4(S, cin);
#pragma unroll
        for (int k = 0; k < kBK; ++k) V[k] = S[k] | (V[k] & ~P[k]);
      }
#pragma unroll
      for (int b = 0; b < 8; ++b) cq[b] = nq[b];
    }
    // c[m, n] = zero bits of V over the pair's n columns (bits past n stay 1), summed over the group's lanes
    uint32_t z = 0;
#pragma unroll
    for (int k = 0; k < kBK; ++k) z += __popc(~V[k]);
    for (uint32_t off = 1; off < G; off <<= 1) z += __shfl_xor_sync(kFull, z, off);
    if (has && gl == 0) a.out_lens[pr.out] = z;
  }
}

inline uint32_t group_lanes(uint32_t w) {
  uint32_t g = 1;
  while (g < 32 && g * kBK < w) g <<= 1;
  return g;
}

struct Plan {
  std::vector<BPair> pairs;
  std::vector<BItem> items;
  uint64_t peq_words = 0;
};

// Host plan: lengths from the offsets; pairs whose words exceed one warp's 128 (n > 4096) are not handled here.
bool make_plan(const uint64_t* x_off, const uint64_t* y_off, uint64_t count, Plan& plan, std::vector<uint64_t>& big) {
  struct Tmp {
    uint32_t idx, m, n, w, G;
  };
  std::vector<Tmp> t;
  t.reserve(count);
  for (uint64_t k = 0; k < count; ++k) {
    const uint64_t m = x_off[k + 1] - x_off[k], n = y_off[k + 1] - y_off[k];
    if (m == 0 || n == 0) continue;  // length 0, written by the caller
    const uint64_t w = (n + 31) / 32;
    if (w > (uint64_t)kWarpWords || m >= (1ull << 31)) {
      big.push_back(k);
      continue;
    }
    t.push_back({(uint32_t)k, (uint32_t)m, (uint32_t)n, (uint32_t)w, group_lanes((uint32_t)w)});
  }
  // bucket by G; within a bucket, longest rows first (similar m share a warp)
  std::sort(t.begin(), t.end(), [](const Tmp& a, const Tmp& b) {
    if (a.G != b.G) return a.G > b.G;
    return a.m > b.m;
  });
  plan.pairs.resize(t.size());
  uint64_t off = 0;
  for (size_t i = 0; i < t.size(); ++i) {
    BPair& p = plan.pairs[i];
    p.x_off = x_off[t[i].idx] - x_off[0];
    p.y_off = y_off[t[i].idx] - y_off[0];
    p.m = t[i].m;
    p.n = t[i].n;
    p.w = t[i].w;
    p.out = t[i].idx;
    p.peq_off = off;
    off += (uint64_t)(std::min<uint32_t>(256u, t[i].n) + 1) * t[i].w;
  }
  plan.peq_words = off;
  for (size_t i = 0; i < t.size();) {
    const uint32_t G = t[i].G, per = 32 / G;
    size_t j = i;
    uint32_t rows = 0;
    while (j < t.size() && j - i < per && t[j].G == G) {
      rows = std::max(rows, t[j].m);
      ++j;
    }
    plan.items.push_back({(uint32_t)i, (uint32_t)(j - i), G, rows});
    i = j;
  }
  // longest items first (largest rows * words), for balance across the persistent warps
  std::stable_sort(plan.items.begin(), plan.items.end(), [](const BItem& a, const BItem& b) {
    return (uint64_t)a.rows * a.G > (uint64_t)b.rows * b.G;
  });
  return true;
}

}  // namespace

namespace lcs {
int run_length(lcs_ctx* c, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n, uint64_t* d_out,
               cudaStream_t st);

static uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

// The launches of a planned batch: zero the outputs, per-pair prep, the persistent kernel (stage events around
// them when profiling).
static void batch_launches(lcs_ctx* c, uint64_t* d_out, uint64_t count, const BatchArgs& a, cudaStream_t st,
                           bool marks) {
  if (marks) c->mark(0, st);
  cudaMemsetAsync(d_out, 0, count * sizeof(uint64_t), st);  // empty pairs: length 0
  if (a.npairs) {
    cudaMemsetAsync(a.ticket, 0, 4, st);
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const unsigned prep_blocks = (unsigned)std::min<uint64_t>((a.npairs + 7) / 8, (uint64_t)sms * 8);
    k_batch_prep<<<prep_blocks, 256, 0, st>>>(a);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_main, kBatchWarps * 32, 0);
    const unsigned blocks = (unsigned)std::max(1, sms * std::max(per_sm, 1));
    if (marks) c->mark(1, st);
    k_batch_main<<<blocks, kBatchWarps * 32, 0, st>>>(a);
    if (marks) c->mark(2, st);
    c->bblocks = blocks;
  } else if (marks) {
    c->mark(1, st);
    c->mark(2, st);
  }
}

// Runs a batch whose xs / ys / out_lens are already on the device. The first call of a batch plans it on the host
// and uploads the plan; a later call with the same pairs (same offsets and buffers) reuses it. Without profiling
// the launches are captured once as a CUDA graph and replayed.
int run_batch(lcs_ctx* c, const uint8_t* d_xs, const uint8_t* d_ys, const uint64_t* x_off, const uint64_t* y_off,
              uint64_t count, uint64_t* d_out, cudaStream_t st) {
  uint64_t key = 1469598103934665603ull;
  const uint64_t ptrs[4] = {count, (uint64_t)d_xs, (uint64_t)d_ys, (uint64_t)d_out};
  key = fnv1a(key, ptrs, sizeof(ptrs));
  for (uint64_t k = 0; k <= count; ++k) {
    const uint64_t rel[2] = {x_off[k] - x_off[0], y_off[k] - y_off[0]};
    key = fnv1a(key, rel, sizeof(rel));
  }
  int rc = LCS_OK;
  if (key != c->bkey) {
    if (c->bexec) cudaGraphExecDestroy(c->bexec);
    c->bexec = nullptr;
    c->bkey = 0;
    Plan plan;
    c->bbig.clear();
    make_plan(x_off, y_off, count, plan, c->bbig);
    c->bcells = 0;
    for (uint64_t k = 0; k < count; ++k) c->bcells += (x_off[k + 1] - x_off[k]) * (y_off[k + 1] - y_off[k]);
    const size_t pb = plan.pairs.size() * sizeof(BPair), ib = plan.items.size() * sizeof(BItem);
    if (!plan.pairs.empty()) {
      rc = from_cuda(ensure(c->bplan, pb + ib + 256));
      if (!rc) rc = from_cuda(ensure(c->bsig, plan.pairs.size() * 4 + 4));
      if (!rc) rc = from_cuda(ensure(c->bxcode, std::max<uint64_t>(x_off[count] - x_off[0], 1)));
      if (!rc) rc = from_cuda(ensure(c->bpeq, plan.peq_words * 4 + 4));
      if (rc) return rc;
      // (copies from pageable memory: the runtime has staged the data when the call returns)
      rc = from_cuda(cudaMemcpyAsync(c->bplan.p, plan.pairs.data(), pb, cudaMemcpyHostToDevice, st));
      if (!rc) rc = from_cuda(cudaMemcpyAsync((char*)c->bplan.p + pb, plan.items.data(), ib, cudaMemcpyHostToDevice, st));
      if (rc) return rc;
    }
    c->bnpairs = plan.pairs.size();
    c->bnitems = plan.items.size();
    c->bpairs_bytes = pb;
    c->bkey = key;
  }
  BatchArgs a{};
  a.xs = d_xs;
  a.ys = d_ys;
  a.pairs = (const BPair*)c->bplan.p;
  a.items = (const BItem*)((char*)c->bplan.p + c->bpairs_bytes);
  a.sigma = (uint32_t*)c->bsig.p;
  a.xcode = (uint8_t*)c->bxcode.p;
  a.peq = (uint32_t*)c->bpeq.p;
  a.out_lens = d_out;
  a.ticket = (uint32_t*)((char*)c->small.p + kOffTicket);
  a.npairs = (uint32_t)c->bnpairs;
  a.nitems = (uint32_t)c->bnitems;
  if (c->prof) {
    batch_launches(c, d_out, count, a, st, true);
    rc = from_cuda(cudaGetLastError());
  } else {
    if (!c->bexec) {
      if (!c->cap_stream) {
        rc = from_cuda(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        if (rc) return rc;
      }
      // capture: the recorded launches do not run now; the graph runs on st below
      rc = from_cuda(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      if (rc) return rc;
      batch_launches(c, d_out, count, a, c->cap_stream, false);
      cudaGraph_t graph = nullptr;
      rc = from_cuda(cudaStreamEndCapture(c->cap_stream, &graph));
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

extern "C" int lcs_batch_dev(lcs_ctx* c, const uint8_t* d_xs, const uint64_t* d_x_off, const uint8_t* d_ys,
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

extern "C" int lcs_batch(lcs_ctx* c, const uint8_t* xs, const uint64_t* x_off, const uint8_t* ys,
                         const uint64_t* y_off, uint64_t count, uint64_t* out_lens) {
  if (!c || (count && (!x_off || !y_off || !out_lens))) return LCS_ERR_INVALID;
  if (count == 0) return LCS_OK;
  if (!offsets_ok(x_off, count) || !offsets_ok(y_off, count)) return LCS_ERR_INVALID;
  const uint64_t nx = x_off[count] - x_off[0], ny = y_off[count] - y_off[0];
  if ((nx && !xs) || (ny && !ys)) return LCS_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  cudaSetDevice(c->device);
  int rc = from_cuda(ensure(c->x, std::max<uint64_t>(nx, 1)));
  if (!rc) rc = from_cuda(ensure(c->y, std::max<uint64_t>(ny, 1)));
  if (!rc) rc = from_cuda(ensure(c->bout, count * 8));
  if (!rc && nx) rc = from_cuda(cudaMemcpyAsync(c->x.p, xs + x_off[0], nx, cudaMemcpyHostToDevice, c->stream));
  if (!rc && ny) rc = from_cuda(cudaMemcpyAsync(c->y.p, ys + y_off[0], ny, cudaMemcpyHostToDevice, c->stream));
  if (!rc)
    rc = run_batch(c, (const uint8_t*)c->x.p, (const uint8_t*)c->y.p, x_off, y_off, count, (uint64_t*)c->bout.p,
                   c->stream);
  if (!rc) rc = from_cuda(cudaMemcpyAsync(out_lens, c->bout.p, count * 8, cudaMemcpyDeviceToHost, c->stream));
  if (!rc) rc = from_cuda(cudaStreamSynchronize(c->stream));
  if (!rc) rc = take_status(c);
  return rc;
}
