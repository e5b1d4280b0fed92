// Input staging for the fill kernel: the alphabet of Y, per-row symbol offsets for X, and the per-symbol match
// masks Peq (bit k of word q of row s is set when y_{32q+k+1} is symbol s). The match masks realise the test
// x_i = y_j of LCS-length (paper §I.C, its line "if x_i = y_j") for 32 columns at a time.
#include "lcs_internal.h"

namespace lcs {

namespace {

__global__ void k_presence(const uint8_t* __restrict__ y, uint64_t n, uint32_t* __restrict__ presence8) {
  __shared__ uint32_t bits[8];
  if (threadIdx.x < 8) bits[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    const uint32_t v = y[j];
    atomicOr(&bits[v >> 5], 1u << (v & 31));
  }
  __syncthreads();
  if (threadIdx.x < 8 && bits[threadIdx.x]) atomicOr(&presence8[threadIdx.x], bits[threadIdx.x]);
}

// code of a present byte = its rank among present bytes; an absent byte maps to the all-zero row (index sigma).
__global__ void k_codemap(const uint32_t* __restrict__ presence8, uint16_t* __restrict__ codemap,
                          uint32_t* __restrict__ sigma_rows) {
  const uint32_t b = threadIdx.x;  // 256 threads
  uint32_t below = 0, total = 0;
  for (int k = 0; k < 8; ++k) {
    const uint32_t p = presence8[k];
    total += __popc(p);
    if ((uint32_t)k < (b >> 5)) below += __popc(p);
  }
  below += __popc(presence8[b >> 5] & ((1u << (b & 31)) - 1u));
  const bool present = (presence8[b >> 5] >> (b & 31)) & 1u;
  codemap[b] = (uint16_t)(present ? below : total);
  if (b == 0) *sigma_rows = total + 1;
}

__global__ void k_xoff(const uint8_t* __restrict__ x, uint64_t m, int reverse, uint64_t pad_front, uint64_t total,
                       uint32_t B, const uint16_t* __restrict__ codemap, const uint32_t* __restrict__ sigma_rows,
                       uint32_t* __restrict__ xoff, uint8_t* __restrict__ xcode) {
  const uint32_t zero_code = *sigma_rows - 1;
  const uint64_t front = (uint64_t)kPadRowblocks * B + pad_front;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += stride) {
    uint32_t code = zero_code;
    if (p >= front && p - front < m) {
      const uint64_t i = p - front;
      code = codemap[x[reverse ? (m - 1 - i) : i]];
      if (xcode) xcode[i] = (uint8_t)code;
    }
    xoff[p] = code * (uint32_t)kStripeWords;  // word offset of the symbol's row in a block's match-mask stripe
  }
}

// One warp per 32-column word q: lanes holding the same symbol find each other with __match_any_sync and the lowest
// of them writes the word's mask for that symbol. Words and symbols not written stay zero (the array is zeroed).
__global__ void k_peq(const uint8_t* __restrict__ y, uint64_t n, int reverse, uint64_t wpad,
                      const uint16_t* __restrict__ codemap, uint32_t* __restrict__ peq) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t nwords = (n + 31) >> 5;
  for (uint64_t q = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nwords; q += warps) {
    const uint64_t c = q * 32 + lane + 1;  // 1-based column
    uint32_t code = 0xFFFFu;
    if (c <= n) code = codemap[y[reverse ? (n - c) : (c - 1)]];
    const uint32_t mask = __match_any_sync(0xFFFFFFFFu, code);
    if (code != 0xFFFFu && lane == (uint32_t)(__ffs(mask) - 1)) peq[(uint64_t)code * wpad + q] = mask;
  }
}

inline unsigned grid_for(uint64_t items, unsigned threads, unsigned cap = 4096) {
  uint64_t g = (items + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

}  // namespace

cudaError_t launch_alphabet(const uint8_t* y, uint64_t n, uint32_t* presence8, uint16_t* codemap,
                            uint32_t* sigma_rows, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(presence8, 0, 8 * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  if (n > 0) k_presence<<<grid_for(n, 256, 1024), 256, 0, st>>>(y, n, presence8);
  k_codemap<<<1, 256, 0, st>>>(presence8, codemap, sigma_rows);
  return cudaGetLastError();
}

cudaError_t launch_xoff(const uint8_t* x, uint64_t m, bool reverse, uint64_t pad_front, uint64_t R, uint32_t B,
                        const uint16_t* codemap, const uint32_t* sigma_rows, uint32_t* xoff, uint8_t* xcode,
                        cudaStream_t st) {
  const uint64_t total = (R + (uint64_t)kPadRowblocks + kPadBackRowblocks) * B;
  k_xoff<<<grid_for(total, 256), 256, 0, st>>>(x, m, reverse ? 1 : 0, pad_front, total, B, codemap, sigma_rows,
                                               xoff, xcode);
  return cudaGetLastError();
}

cudaError_t launch_peq(const uint8_t* y, uint64_t n, bool reverse, uint64_t wpad, const uint16_t* codemap,
                       uint32_t* peq, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(peq, 0, (size_t)kSigmaMax * wpad * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  if (n == 0) return cudaSuccess;
  const uint64_t nwords = (n + 31) >> 5;
  k_peq<<<grid_for(nwords * 32, 256), 256, 0, st>>>(y, n, reverse ? 1 : 0, wpad, codemap, peq);
  return cudaGetLastError();
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st) { return cudaMemsetAsync(p, 0, bytes, st); }

}  // namespace lcs
