// Host-side checks of the batch plan (paper_1306_4627_gb300/csrc/lcs_plan.h) on seeded random batches: every pair
// lands exactly once (in the plan or on the single-pair list), splits and jobs are consistent, items partition the
// jobs with one shape each and fit a warp, the order rules hold, and the code lists, mask tables and final-row slots
// of different pairs are disjoint and aligned as the kernels assume. Prints "ok <checks>" or the first failure.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <set>
#include <utility>
#include <vector>

#include "lcs_plan.h"

using namespace lcs_plan;

static long g_checks = 0;
static long g_split = 0, g_big = 0, g_empty = 0, g_items_k[9] = {0};  // coverage of the cases above
#define CHECK(cond, ...)                                      \
  do {                                                        \
    ++g_checks;                                               \
    if (!(cond)) {                                            \
      std::fprintf(stderr, "FAILED %s (line %d): ", #cond, __LINE__); \
      std::fprintf(stderr, __VA_ARGS__);                      \
      std::fprintf(stderr, "\n");                             \
      std::exit(1);                                           \
    }                                                         \
  } while (0)

struct Span {
  uint64_t lo, hi;  // [lo, hi)
};

static void check_disjoint(std::vector<Span> v, const char* what) {
  std::sort(v.begin(), v.end(), [](const Span& a, const Span& b) { return a.lo < b.lo; });
  for (size_t k = 1; k < v.size(); ++k) CHECK(v[k - 1].hi <= v[k].lo, "%s overlap at %zu", what, k);
}

static void check_plan(const std::vector<uint64_t>& xo, const std::vector<uint64_t>& yo, uint64_t warps,
                       uint32_t k_cfg, uint32_t split_pct) {
  const uint64_t count = xo.size() - 1;
  Plan plan;
  std::vector<uint64_t> big;
  CHECK(make_plan(xo.data(), yo.data(), count, warps, k_cfg, split_pct, plan, big), "make_plan");
  // every nonempty pair exactly once: in the plan (rows fit one warp) or on the single-pair list
  std::vector<int> seen(count, 0);
  for (uint64_t k : big) {
    CHECK(k < count, "big index");
    const uint64_t m = xo[k + 1] - xo[k], n = yo[k + 1] - yo[k];
    CHECK(m && n && ((n + 31) / 32 > (uint64_t)kRowWords || m >= (1ull << 31)), "pair %llu on the big list",
          (unsigned long long)k);
    ++seen[k];
  }
  for (const BPair& p : plan.pairs) {
    CHECK(p.out < count, "out index");
    ++seen[p.out];
    const uint64_t k = p.out, m = xo[k + 1] - xo[k], n = yo[k + 1] - yo[k];
    CHECK(p.m == m && p.n == n && p.w == (n + 31) / 32 && p.w <= (uint32_t)kRowWords, "pair %llu sizes",
          (unsigned long long)k);
    CHECK(p.x_off == xo[k] - xo[0] && p.y_off == yo[k] - yo[0], "pair %llu offsets", (unsigned long long)k);
    const bool split = p.mt < p.m;
    CHECK(p.mt == (split ? (p.m + 1) / 2 : p.m), "pair %llu split rows", (unsigned long long)k);
    if (split) CHECK(split_pct != 0 && p.m > kSplitMinRows, "pair %llu split without reason", (unsigned long long)k);
  }
  for (uint64_t k = 0; k < count; ++k) {
    const bool empty = xo[k + 1] == xo[k] || yo[k + 1] == yo[k];
    CHECK(seen[k] == (empty ? 0 : 1), "pair %llu seen %d times", (unsigned long long)k, seen[k]);
  }
  // split list and final-row slots
  std::set<uint32_t> fvs;
  uint32_t nsplit = 0;
  for (uint32_t i = 0; i < plan.pairs.size(); ++i) {
    const BPair& p = plan.pairs[i];
    if (p.mt < p.m) {
      CHECK(nsplit < plan.split.size() && plan.split[nsplit] == i, "split list order");
      ++nsplit;
      CHECK(p.fv + 1 < plan.fv_slots, "fv slot range");
      CHECK(fvs.insert(p.fv).second && fvs.insert(p.fv + 1).second, "fv slots shared");
    }
  }
  CHECK(nsplit == plan.split.size(), "split list length");
  g_split += nsplit;
  g_big += (long)big.size();
  for (uint64_t k = 0; k < count; ++k) g_empty += (xo[k + 1] == xo[k] || yo[k + 1] == yo[k]) ? 1 : 0;
  // jobs: one forward job per pair, one reverse job per split pair, rows as planned
  std::map<std::pair<uint32_t, uint32_t>, uint32_t> jobs;
  for (const BJob& j : plan.jobs) {
    CHECK(j.pair < plan.pairs.size() && j.rev <= 1, "job fields");
    const BPair& p = plan.pairs[j.pair];
    CHECK(j.rows == (j.rev ? p.m - p.mt : p.mt) && j.rows > 0, "job rows");
    CHECK(!j.rev || p.mt < p.m, "reverse job of an unsplit pair");
    const uint32_t times = ++jobs[std::make_pair(j.pair, j.rev)];
    CHECK(times == 1, "job twice");
  }
  CHECK(jobs.size() == plan.pairs.size() + plan.split.size(), "job count");
  // items: consecutive job ranges covering all jobs once, one shape (K, G) each, fitting a warp
  uint32_t next = 0, k_max = 2;
  std::vector<std::pair<uint32_t, uint32_t>> ranges;
  for (const BItem& it : plan.items) ranges.push_back({it.first, it.count});
  std::sort(ranges.begin(), ranges.end());
  for (auto& r : ranges) {
    CHECK(r.first == next && r.second > 0, "items do not partition the jobs");
    next += r.second;
  }
  CHECK(next == plan.jobs.size(), "items cover %u of %zu jobs", next, plan.jobs.size());
  for (size_t i = 0; i < plan.items.size(); ++i) {
    const BItem& it = plan.items[i];
    CHECK(it.K == 2 || it.K == 4 || it.K == 8, "item K");
    CHECK(it.K >= k_cfg || it.K == 8, "item K below the configured words per lane");
    CHECK(it.G >= 1 && it.G <= 32 && (uint32_t)it.G * it.count <= 32, "item does not fit a warp");
    uint32_t rows = 0;
    for (uint32_t j = it.first; j < it.first + it.count; ++j) {
      const BPair& p = plan.pairs[plan.jobs[j].pair];
      CHECK(lane_words(p.w, k_cfg) == it.K && group_lanes(p.w, it.K) == it.G, "job shape differs from its item");
      CHECK(p.w <= 32u * it.K, "row does not fit the item's lanes");
      rows = std::max(rows, plan.jobs[j].rows);
    }
    CHECK(it.rows == rows, "item rows");
    if (i) CHECK(plan.items[i - 1].rows + plan.items[i - 1].G >= it.rows + it.G, "items not longest first");
    k_max = std::max<uint32_t>(k_max, it.K);
    ++g_items_k[it.K];
  }
  CHECK(plan.k_max == k_max, "k_max %u, items %u", plan.k_max, k_max);
  // code lists: zeros at the start, each list with its padding inside the buffer, disjoint, forward lists aligned
  // with x modulo 16 (16-byte loads of x map to 32-byte stores of codes)
  std::vector<Span> codes, tabs;
  for (const BPair& p : plan.pairs) {
    CHECK(p.xcf >= kCodeZeros + kCodePadFront, "forward list over the leading zeros");
    CHECK((p.xcf & 15) == (p.x_off & 15), "forward list alignment");
    codes.push_back({p.xcf - kCodePadFront, p.xcf + p.mt + kCodePadBack});
    CHECK(p.xcf + p.mt + kCodePadBack <= plan.codes, "forward list past the buffer");
    if (p.mt < p.m) {
      CHECK(p.xcr >= kCodeZeros + kCodePadFront, "reverse list over the leading zeros");
      codes.push_back({p.xcr - kCodePadFront, p.xcr + (p.m - p.mt) + kCodePadBack});
      CHECK(p.xcr + (p.m - p.mt) + kCodePadBack <= plan.codes, "reverse list past the buffer");
    }
    // mask tables: (sigma + 1) rows of w words for sigma <= min(256, n), 16-byte aligned
    const uint64_t tab = (std::min<uint64_t>(256u, p.n) + 1) * p.w;
    CHECK(p.peq_off % 4 == 0, "table alignment");
    tabs.push_back({p.peq_off, p.peq_off + tab});
    CHECK(p.peq_off + tab <= plan.peq_words, "table past the buffer");
    if (p.mt < p.m) {
      CHECK(p.peqr_off % 4 == 0, "reverse table alignment");
      tabs.push_back({p.peqr_off, p.peqr_off + tab});
      CHECK(p.peqr_off + tab <= plan.peq_words, "reverse table past the buffer");
    }
  }
  check_disjoint(codes, "code lists");
  check_disjoint(tabs, "mask tables");
  // prep order: a permutation, most prep work first
  std::vector<uint32_t> order = plan.prep_order;
  CHECK(order.size() == plan.pairs.size(), "prep order length");
  auto cost = [&](uint32_t k) {
    const BPair& q = plan.pairs[k];
    return (uint64_t)q.n * (q.mt < q.m ? 2 : 1) + q.m / 16;
  };
  for (size_t i = 1; i < order.size(); ++i) CHECK(cost(order[i - 1]) >= cost(order[i]), "prep order");
  std::sort(order.begin(), order.end());
  for (size_t i = 0; i < order.size(); ++i) CHECK(order[i] == i, "prep order is not a permutation");
}

int main() {
  std::mt19937_64 rng(0x13064627);
  auto loguni = [&](double lo, double hi) {
    std::uniform_real_distribution<double> u(std::log(lo), std::log(hi));
    return (uint64_t)std::exp(u(rng));
  };
  int batches = 0;
  for (int b = 0; b < 60; ++b) {
    const uint64_t count = 1 + rng() % (b < 50 ? 300 : 3000);
    std::vector<uint64_t> xo(count + 1), yo(count + 1);
    xo[0] = rng() % 1000;  // offsets need not start at 0
    yo[0] = rng() % 1000;
    for (uint64_t k = 0; k < count; ++k) {
      uint64_t m, n;
      switch (rng() % 6) {
        case 0: m = rng() % 3; n = rng() % 40; break;                   // empty and tiny pairs
        case 1: m = loguni(1, 20000); n = 4096 + rng() % 200; break;    // around the 4096-column limit
        case 2: m = 5000 + rng() % 5000; n = loguni(1, 4096); break;    // tall pairs (split)
        default: m = loguni(1, 4096); n = loguni(1, 4096); break;       // the batch workload's shapes
      }
      xo[k + 1] = xo[k] + m;
      yo[k + 1] = yo[k] + n;
    }
    for (uint32_t k_cfg : {2u, 4u, 8u})
      for (uint32_t pct : {0u, 50u, 100u, 200u})
        for (uint64_t warps : {8ull, 2432ull}) check_plan(xo, yo, warps, k_cfg, pct);
    ++batches;
  }
  CHECK(g_split > 0 && g_big > 0 && g_empty > 0 && g_items_k[2] > 0 && g_items_k[4] > 0 && g_items_k[8] > 0,
        "a case was never exercised (split %ld, big %ld, empty %ld)", g_split, g_big, g_empty);
  std::printf("ok %ld checks over %d batches (split pairs %ld, single-pair path %ld, empty %ld; items with 2/4/8 "
              "words per lane %ld/%ld/%ld)\n",
              g_checks, batches, g_split, g_big, g_empty, g_items_k[2], g_items_k[4], g_items_k[8]);
  return 0;
}
