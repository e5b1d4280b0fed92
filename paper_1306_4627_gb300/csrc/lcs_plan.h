// The host-side plan of a batch (lcs_batch*): which pairs run in the persistent kernel, how long pairs are split,
// how jobs are bucketed by words per lane and lanes per pair and packed into warp items, and where every pair's
// symbol codes and match-mask tables go in the batch buffers. Plain structs shared with the kernels (lcs_batch.cu)
// and host code only, so that the plan can be checked without a GPU.
#pragma once

#include <algorithm>
#include <cstdint>
#include <numeric>
#include <vector>

namespace lcs_plan {

constexpr int kRowWords = 128;     // words of the longest row of a batch pair (n <= 4096)

constexpr uint32_t kCodePadFront = 32;  // zero-row codes before a job's list: lanes run up to 31 rows behind
constexpr uint32_t kCodePadBack = 8;    // and after it: the main kernel reads 8 rows at a time
constexpr uint32_t kCodeZeros = 48;     // zeros at the start of xcode, read by lanes without a job (rows 0..39)

struct BPair {        // one pair of the plan
  uint64_t x_off;     // first symbol of x in xs
  uint64_t y_off;
  uint64_t xcf, xcr;  // codes of the forward job's rows (x[0..mt)) and of the reverse job's (x[m-1] down to x[mt])
                      // in xcode, each list between runs of the pair's zero row index
  uint64_t peq_off;   // word offset of its match-mask table: (sigma + 1) rows of w words
  uint64_t peqr_off;  // the table over reversed y (split pairs only)
  uint32_t m, n, w;   // rows, columns, words per row (ceil(n / 32))
  uint32_t out;       // index into out_lens
  uint32_t mt;        // rows of the forward job (m when the pair is not split)
  uint32_t fv;        // split pairs: final rows of the forward / reverse job in slots fv, fv + 1
};

struct BJob {         // the rows of one pair a group of lanes works through
  uint32_t pair, rev, rows, pad;
};

struct BItem {        // a warp's unit of work: jobs [first, first + count), G lanes of K words each
  uint32_t first, count, rows;
  uint16_t G, K;
};

// Lanes per pair: just enough to hold its w words at K per lane (so 32 / G pairs share a warp).
inline uint32_t group_lanes(uint32_t w, uint32_t K) { return w == 0 ? 1u : (w + K - 1) / K; }

// Words per lane of a pair with w words per row: the configured K, or the smallest larger one that fits the row in
// one warp (32 lanes).
inline uint32_t lane_words(uint32_t w, uint32_t k_cfg) {
  uint32_t K = k_cfg;
  while (K < 8 && w > 32 * K) K *= 2;
  return K;
}

struct Plan {
  std::vector<BPair> pairs;
  std::vector<BJob> jobs;
  std::vector<BItem> items;
  std::vector<uint32_t> split;  // plan indices of split pairs
  std::vector<uint32_t> prep_order;  // plan indices, most prep work first
  uint64_t peq_words = 0;
  uint64_t codes = kCodeZeros;  // xcode: zeros, then the jobs' padded code lists
  uint32_t fv_slots = 0;
  uint32_t k_max = 2;  // the largest words per lane of an item (sizes the kernel's mask stage)
};

constexpr uint32_t kSplitMinRows = 256;  // pairs with fewer rows are never split

// Host plan: lengths from the offsets; pairs whose words exceed one warp's 128 (n > 4096) are not handled here.
// A pair is split when its rows exceed both kSplitMinRows and split_pct % of the rows an average resident warp
// works through (the batch's lane-rows spread over `warps`), i.e. when its serial chain would outlast the rest of
// the launch; split_pct = 0 never splits. k_cfg is the configured words per lane.
inline bool make_plan(const uint64_t* x_off, const uint64_t* y_off, uint64_t count, uint64_t warps, uint32_t k_cfg,
               uint32_t split_pct, Plan& plan, std::vector<uint64_t>& big) {
  uint64_t lane_rows = 0;
  for (uint64_t k = 0; k < count; ++k) {
    const uint64_t m = x_off[k + 1] - x_off[k], n = y_off[k + 1] - y_off[k];
    const uint64_t w = (n + 31) / 32;
    if (m && n && w <= (uint64_t)kRowWords) lane_rows += m * group_lanes((uint32_t)w, lane_words((uint32_t)w, k_cfg));
  }
  const uint64_t avg_rows = lane_rows / (32 * std::max<uint64_t>(warps, 1));
  const uint64_t split_rows =
      split_pct ? std::max<uint64_t>(kSplitMinRows, avg_rows * split_pct / 100) : ~(uint64_t)0;
  for (uint64_t k = 0; k < count; ++k) {
    const uint64_t m = x_off[k + 1] - x_off[k], n = y_off[k + 1] - y_off[k];
    if (m == 0 || n == 0) continue;  // length 0, written by the zeroing launch
    const uint64_t w = (n + 31) / 32;
    if (w > (uint64_t)kRowWords || m >= (1ull << 31)) {
      big.push_back(k);
      continue;
    }
    BPair p{};
    p.x_off = x_off[k] - x_off[0];
    p.y_off = y_off[k] - y_off[0];
    p.m = (uint32_t)m;
    p.n = (uint32_t)n;
    p.w = (uint32_t)w;
    p.out = (uint32_t)k;
    const bool split = m > split_rows;
    p.mt = split ? (uint32_t)((m + 1) / 2) : (uint32_t)m;
    const uint64_t tab = ((std::min<uint64_t>(256u, n) + 1) * w + 3) & ~(uint64_t)3;  // whole 16-byte groups
    p.xcf = plan.codes + kCodePadFront + ((p.x_off - plan.codes - kCodePadFront) & 15);  // = x_off modulo 16
    plan.codes = p.xcf + p.mt + kCodePadBack;
    if (split) {
      p.xcr = plan.codes + kCodePadFront;
      plan.codes = p.xcr + (p.m - p.mt) + kCodePadBack;
    }
    p.peq_off = plan.peq_words;
    plan.peq_words += tab;
    if (split) {
      p.peqr_off = plan.peq_words;
      plan.peq_words += tab;
      p.fv = plan.fv_slots;
      plan.fv_slots += 2;
      plan.split.push_back((uint32_t)plan.pairs.size());
    }
    const uint32_t idx = (uint32_t)plan.pairs.size();
    plan.pairs.push_back(p);
    plan.jobs.push_back({idx, 0u, p.mt, 0u});
    if (split) plan.jobs.push_back({idx, 1u, p.m - p.mt, 0u});
  }
  // prep order: the table build (n columns, twice for split pairs) dominates a pair's prep
  plan.prep_order.resize(plan.pairs.size());
  std::iota(plan.prep_order.begin(), plan.prep_order.end(), 0u);
  auto prep_cost = [&](uint32_t k) {
    const BPair& q = plan.pairs[k];
    return (uint64_t)q.n * (q.mt < q.m ? 2 : 1) + q.m / 16;
  };
  std::stable_sort(plan.prep_order.begin(), plan.prep_order.end(),
                   [&](uint32_t u, uint32_t v) { return prep_cost(u) > prep_cost(v); });
  // bucket jobs by (G, K); within a bucket, longest first (similar rows share a warp)
  std::vector<uint32_t> K(plan.jobs.size()), G(plan.jobs.size());
  for (size_t j = 0; j < plan.jobs.size(); ++j) {
    const uint32_t w = plan.pairs[plan.jobs[j].pair].w;
    K[j] = lane_words(w, k_cfg);
    G[j] = group_lanes(w, K[j]);
  }
  std::vector<uint32_t> order(plan.jobs.size());
  std::iota(order.begin(), order.end(), 0u);
  std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
    if (G[a] != G[b]) return G[a] > G[b];
    if (K[a] != K[b]) return K[a] > K[b];
    return plan.jobs[a].rows > plan.jobs[b].rows;
  });
  std::vector<BJob> jobs(order.size());
  std::vector<uint32_t> Ks(order.size()), Gs(order.size());
  for (size_t j = 0; j < order.size(); ++j) {
    jobs[j] = plan.jobs[order[j]];
    Ks[j] = K[order[j]];
    Gs[j] = G[order[j]];
  }
  plan.jobs.swap(jobs);
  for (size_t i = 0; i < plan.jobs.size();) {
    const uint32_t g = Gs[i], kk = Ks[i], per = 32 / g;
    size_t j = i;
    uint32_t rows = 0;
    while (j < plan.jobs.size() && j - i < per && Gs[j] == g && Ks[j] == kk) {
      rows = std::max(rows, plan.jobs[j].rows);
      ++j;
    }
    plan.items.push_back({(uint32_t)i, (uint32_t)(j - i), rows, (uint16_t)g, (uint16_t)kk});
    plan.k_max = std::max(plan.k_max, kk);
    i = j;
  }
  // longest items first: an item holds its warp for rows + G - 1 steps whatever its G (list scheduling by the
  // atomic ticket then approximates longest-processing-time-first over the persistent warps)
  std::stable_sort(plan.items.begin(), plan.items.end(),
                   [](const BItem& a, const BItem& b) { return a.rows + a.G > b.rows + b.G; });
  return true;
}

}  // namespace lcs_plan
