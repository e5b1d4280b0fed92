// Small pairs in one launch: LCS-length (paper §I.C) and Print-LCS (§I.D) for n <= 992 columns and m <= 1024 rows.
//
// The general path costs eight launches (alphabet, masks with row offsets, the cooperative fill, five traceback
// kernels), which is most of the time of a pair of a few thousand cells. Here one warp does everything, in shared
// memory:
//   * match masks of all 256 byte values over Y, peq[c][q] bit k = [y[32q + k] = c] (absent bytes give zero rows);
//   * the bit-parallel row update (U = V & P; S = V + U + carry; V' = S | (V & ~P)) with lane q holding word q of
//     V; the lanes run one row apart (lane q works on row t - q + 1 at step t), so the carry out of lane q's word
//     reaches lane q + 1 by one shuffle in time for the same row one step later;
//   * in traceback mode, the carry-into vector T = S ^ V ^ U of every word and row (bit b of word Q of row i is
//     c[i, 32Q + b] - c[i-1, 32Q + b]: 0 = UP, 1 = LEFT on a mismatch), then Print-LCS's walk from (m, n) by one lane,
//     the same word scan per row as the segment walkers of the general path.
// c[m, n] = the zero bits of V after row m.
#include "lcs_internal.h"

namespace lcs {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kMaskWords = 256 * 32;  // peq: 256 byte values x 32 words

__global__ void __launch_bounds__(32, 1)
    k_small(const uint8_t* __restrict__ x, uint32_t m, const uint8_t* __restrict__ y, uint32_t n, uint32_t tw,
            int traceback, uint8_t* out, uint64_t out_cap, unsigned long long* out_len, DevStatus* status) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* peq = sm;                // peq[c * 32 + q]
  uint32_t* T = sm + kMaskWords;     // T[(i - 1) * tw + q], rows 1..m, words 0..tw-1
  const uint32_t lane = threadIdx.x;
  const uint32_t w = (n + 31) / 32;  // <= 31

  uint4* p4 = reinterpret_cast<uint4*>(peq);
  for (uint32_t k = lane; k < kMaskWords / 4; k += 32) p4[k] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
  if (lane < w) {  // lane q sets the bits of word q only: no two lanes write the same word
    for (uint32_t k = 0; k < 32; ++k) {
      const uint32_t j = lane * 32 + k;
      if (j < n) peq[(uint32_t)y[j] * 32 + lane] |= 1u << k;
    }
  }
  __syncwarp();

  // the mask of this lane's word for row i (1-based); 0 outside rows 1..m and beyond the row's words, which leaves
  // V unchanged and sends no carry
  auto mask_of = [&](int64_t i) -> uint32_t {
    return (i >= 1 && i <= (int64_t)m && lane < w) ? peq[(uint32_t)x[i - 1] * 32 + lane] : 0u;
  };
  uint32_t V = kFull, cout = 0;
  uint32_t P = mask_of(1 - (int64_t)lane);
  const uint32_t steps = m + w;  // lane w (when 32 | n) records the carry out of the row for column n
  for (uint32_t t = 0; t < steps; ++t) {
    const int64_t i = (int64_t)t - (int64_t)lane + 1;
    const uint32_t Pn = mask_of(i + 1);
    const uint32_t cin = __shfl_up_sync(kFull, cout, 1);
    const uint32_t c0 = lane ? cin : 0u;  // no carry into column 1
    const uint32_t U = V & P;
    uint32_t S, co;
    asm("{\n\t"
        ".reg .u32 t;\n\t"
        "add.cc.u32 t, %3, 0xFFFFFFFF;\n\t"  // carry flag = c0 (0 or 1)
        "addc.cc.u32 %0, %2, %4;\n\t"        // S = V + U + c0
        "addc.u32 %1, 0, 0;\n\t"             // carry out of the word
        "}"
        : "=r"(S), "=r"(co)
        : "r"(V), "r"(c0), "r"(U));
    if (traceback && i >= 1 && i <= (int64_t)m && lane < tw) T[(uint32_t)(i - 1) * tw + lane] = S ^ V ^ U;
    V = S | (V & ~P);
    cout = co;
    P = Pn;
  }
  const uint32_t L = __reduce_add_sync(kFull, lane < w ? (uint32_t)__popc(~V) : 0u);
  __syncwarp();
  if (lane != 0) return;
  if (traceback) {
    uint32_t i = m, j = n, cnt = 0;
    const bool write = L <= out_cap;
    while (i > 0 && j > 0) {
      const uint32_t cx = x[i - 1];
      uint32_t Q = j >> 5;
      uint32_t mask = kFull >> (31 - (j & 31));
      uint32_t pm = 0, stop = 0;
      for (;;) {
        const uint32_t d = T[(i - 1) * tw + Q];
        const uint32_t pa = Q < w ? peq[cx * 32 + Q] : 0u;
        const uint32_t pb = Q >= 1 ? peq[cx * 32 + Q - 1] : 0u;
        pm = (pa << 1) | (pb >> 31);  // bit b: x_i = y at column 32Q + b
        stop = (pm | ~d) & mask;      // a match or an UP cell ends the move left
        if (Q == 0) stop &= ~1u;      // column 0 is the border
        if (stop || Q == 0) break;
        --Q;
        mask = kFull;
      }
      if (!stop) break;  // the walk reached column 0
      const uint32_t bit = 31u - __clz(stop);
      const uint32_t c = (Q << 5) + bit;
      if ((pm >> bit) & 1u) {
        if (write && cnt < L) out[L - 1 - cnt] = x[i - 1];
        ++cnt;
        j = c - 1;
      } else {
        j = c;
      }
      --i;
    }
    if (cnt != L) atomicOr(&status->flags, kStatInternal);
  }
  *out_len = L;
}

}  // namespace

bool small_pair(uint64_t m, uint64_t n) { return m >= 1 && n >= 1 && m <= kSmallMaxRows && n <= kSmallMaxCols; }

cudaError_t launch_small(const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n, bool traceback, uint8_t* out,
                         uint64_t out_cap, uint64_t* out_len, DevStatus* status, cudaStream_t st) {
  static std::atomic<uint64_t> attr_done{0};
  const uint32_t w = (uint32_t)((n + 31) / 32);
  const uint32_t tw = (n % 32 == 0) ? w + 1 : w;  // word w holds c[i, n] - c[i-1, n] when 32 divides n
  const size_t smem = (size_t)kMaskWords * 4 + (traceback ? (size_t)m * tw * 4 : 0);
  cudaError_t e = once_per_device_attr(
      [] {
        return cudaFuncSetAttribute(k_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)((size_t)kMaskWords * 4 + (size_t)kSmallMaxRows * 32 * 4));
      },
      attr_done);
  if (e != cudaSuccess) return e;
  k_small<<<1, 32, smem, st>>>(x, (uint32_t)m, y, (uint32_t)n, tw, traceback ? 1 : 0, out, out_cap,
                               reinterpret_cast<unsigned long long*>(out_len), status);
  return cudaGetLastError();
}

}  // namespace lcs
