// Input staging for the fill kernel: the alphabet of Y, per-row symbol offsets for X, and the per-symbol match
// masks Peq (bit k of word q of row s is set when y_{32q+k+1} is symbol s). The match masks realise the test
// x_i = y_j of LCS-length (paper §I.C, its line "if x_i = y_j") for 32 columns at a time.
//
// A call is two launches (the host side of a call, not the GPU, bounds small pairs and busy servers): the alphabet
// in one block, then one launch that writes the masks of both directions (every word: nothing to clear first) and
// the row offsets of both directions, and clears the call's scratch words.
#include <algorithm>

#include "lcs_internal.h"

namespace lcs {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

// ---- alphabet --------------------------------------------------------------------------------------------------
// Presence of each byte value: per thread a 256-bit set in registers, OR-reduced per warp, then per block.
__device__ __forceinline__ void add_byte(uint32_t (&pl)[8], uint32_t v) {
  const uint32_t hi = v >> 5, bit = 1u << (v & 31);
#pragma unroll
  for (uint32_t k = 0; k < 8; ++k) pl[k] |= hi == k ? bit : 0u;
}

// Calls f(byte) for every byte of y this thread owns (16-byte loads for the aligned middle).
template <typename F>
__device__ __forceinline__ void for_my_bytes(const uint8_t* y, uint64_t n, F&& f) {
  const uint64_t head = (16u - ((uintptr_t)y & 15u)) & 15u;
  const uint64_t h = head < n ? head : n;
  if (threadIdx.x < h) f((uint32_t)y[threadIdx.x]);
  const uint64_t nv = (n - h) >> 4;
  const uint4* yv = reinterpret_cast<const uint4*>(y + h);
  for (uint64_t v = threadIdx.x; v < nv; v += blockDim.x) {
    const uint4 q = __ldg(yv + v);
    const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 16; ++k) f((w4[k >> 2] >> (8 * (k & 3))) & 0xFFu);
  }
  const uint64_t t = h + 16 * nv + threadIdx.x;
  if (threadIdx.x < 16 && t < n) f((uint32_t)y[t]);
}

// One block (small and medium n): presence, then the code of a present byte = its rank among present bytes; an
// absent byte maps to the all-zero row (index sigma). The first pass finds which 32-value blocks occur and the OR of
// the bytes' low five bits, which is the presence itself when one block occurs (DNA, protein letters); otherwise one
// more pass per occurring block when there are two (text alphabets), else one pass with a register per block.
__global__ void __launch_bounds__(1024) k_alphabet(const uint8_t* __restrict__ y, uint64_t n,
                                                   uint16_t* __restrict__ codemap, uint32_t* __restrict__ sigma_rows) {
  __shared__ uint32_t bits[8];
  __shared__ uint32_t blocks_s, low_s;
  if (threadIdx.x < 8) bits[threadIdx.x] = 0;
  if (threadIdx.x == 0) blocks_s = low_s = 0;
  __syncthreads();
  uint32_t blocks = 0, low = 0;
  for_my_bytes(y, n, [&](uint32_t v) {
    blocks |= 1u << (v >> 5);
    low |= 1u << (v & 31);
  });
  blocks = __reduce_or_sync(kFull, blocks);
  low = __reduce_or_sync(kFull, low);
  if ((threadIdx.x & 31) == 0 && blocks) atomicOr(&blocks_s, blocks);
  if ((threadIdx.x & 31) == 0 && low) atomicOr(&low_s, low);
  __syncthreads();
  const uint32_t all = blocks_s;
  if (__popc(all) == 1) {
    if (threadIdx.x == 0) bits[__ffs(all) - 1] = low_s;
  } else if (__popc(all) == 2) {
    for (uint32_t bl = all; bl; bl &= bl - 1) {
      const uint32_t hi = __ffs(bl) - 1;
      uint32_t acc = 0;
      for_my_bytes(y, n, [&](uint32_t v) { acc |= (v >> 5) == hi ? 1u << (v & 31) : 0u; });
      acc = __reduce_or_sync(kFull, acc);
      if ((threadIdx.x & 31) == 0 && acc) atomicOr(&bits[hi], acc);
    }
  } else {
    uint32_t pl[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for_my_bytes(y, n, [&](uint32_t v) { add_byte(pl, v); });
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t v = __reduce_or_sync(kFull, pl[k]);
      if ((threadIdx.x & 31) == 0 && v) atomicOr(&bits[k], v);
    }
  }
  __syncthreads();
  if (threadIdx.x < 256) {
    const uint32_t b = threadIdx.x;
    uint32_t below = 0, total = 0;
    for (int k = 0; k < 8; ++k) {
      total += __popc(bits[k]);
      if ((uint32_t)k < (b >> 5)) below += __popc(bits[k]);
    }
    below += __popc(bits[b >> 5] & ((1u << (b & 31)) - 1u));
    const bool present = (bits[b >> 5] >> (b & 31)) & 1u;
    codemap[b] = (uint16_t)(present ? below : total);
    if (b == 0) *sigma_rows = total + 1;
  }
}

// Large n: the presence over many blocks (after a clear of presence8), then the codes.
__global__ void k_presence(const uint8_t* __restrict__ y, uint64_t n, uint32_t* __restrict__ presence8) {
  __shared__ uint32_t bits[8];
  if (threadIdx.x < 8) bits[threadIdx.x] = 0;
  __syncthreads();
  uint32_t pl[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) add_byte(pl, y[j]);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t v = __reduce_or_sync(kFull, pl[k]);
    if ((threadIdx.x & 31) == 0 && v) atomicOr(&bits[k], v);
  }
  __syncthreads();
  if (threadIdx.x < 8 && bits[threadIdx.x]) atomicOr(&presence8[threadIdx.x], bits[threadIdx.x]);
}

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

// ---- row offsets and scratch clearing -------------------------------------------------------------------------
struct XoffArgs {
  XoffJob job[2];
  ZeroSpan zero[kMaxZeroSpans];
  PeqJob peq;
  uint32_t njobs, nzero, npeq, B;
  const uint16_t* codemap;
  const uint32_t* sigma_rows;
};

__device__ void peq_slice(const PeqJob& P, bool rev, const uint16_t* __restrict__ codemap,
                          const uint32_t* __restrict__ sigma_rows);

// blockIdx.y < npeq: the match masks over Y (0) or reversed Y (1); then the row offsets of each job; the last y slice
// clears the spans.
__global__ void k_xoff(const __grid_constant__ XoffArgs a) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.y < a.npeq) {
    peq_slice(a.peq, blockIdx.y == 1, a.codemap, a.sigma_rows);
    return;
  }
  const uint32_t yj = blockIdx.y - a.npeq;
  if (yj < a.njobs) {
    const XoffJob& J = a.job[yj];
    const uint32_t zero_code = *a.sigma_rows - 1;
    const uint64_t front = (uint64_t)kPadRowblocks * a.B + J.pad_front;
    const uint64_t total = (J.R + (uint64_t)kPadRowblocks + kPadBackRowblocks) * a.B;
    for (uint64_t p = i0; p < total; p += stride) {
      uint32_t code = zero_code;
      if (p >= front && p - front < J.m) {
        const uint64_t i = p - front;
        code = a.codemap[J.x[J.reverse ? (J.m - 1 - i) : i]];
        if (J.xcode) J.xcode[i] = (uint8_t)code;
      }
      J.xoff[p] = code * (uint32_t)kStripeWords;  // word offset of the symbol's row in a block's mask stripe
    }
  } else {
    for (uint32_t z = 0; z < a.nzero; ++z) {
      uint32_t* p = static_cast<uint32_t*>(a.zero[z].p);
      const uint64_t words = a.zero[z].bytes / 4;
      for (uint64_t k = i0; k < words; k += stride) p[k] = 0;
    }
  }
}

// ---- match masks -----------------------------------------------------------------------------------------------
// One warp per 32-column word q (every word of the padded row, q < wpad): lane k holds the code of column
// 32q + k + 1; ballots of the code's bits give bit planes, and the mask of symbol r is the AND over the planes of
// the plane (bit b of r set) or its complement (not set), restricted to the columns that exist. Lane r writes
// row r (32 rows per pass up to sigma). Row sigma, the zero row, matches no column and comes out zero, and so do
// the words past the end of Y, so nothing needs clearing first. rev: the masks over reversed Y.
__device__ void peq_slice(const PeqJob& P, bool rev, const uint16_t* __restrict__ codemap,
                          const uint32_t* __restrict__ sigma_rows) {
  const uint8_t* __restrict__ y = P.y;
  const uint64_t n = P.n, wpad = P.wpad;
  const uint32_t lane = threadIdx.x & 31;
  uint32_t* peq = rev ? P.peq_r : P.peq_f;
  const uint32_t sigma = *sigma_rows - 1;
  const uint32_t nb = 32 - __clz(sigma);  // bits of the codes 0..sigma
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t q = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < wpad; q += warps) {
    const uint64_t c = q * 32 + lane + 1;  // 1-based column
    const bool in = c <= n;
    const uint32_t code = in ? codemap[y[rev ? (n - c) : (c - 1)]] : 0u;
    const uint32_t valid = __ballot_sync(kFull, in);
    uint32_t pf[9];
#pragma unroll
    for (uint32_t b = 0; b < 9; ++b) pf[b] = b < nb ? __ballot_sync(kFull, (code >> b) & 1u) : 0u;
    for (uint32_t r = lane; r <= sigma; r += 32) {
      uint32_t mk = valid;
#pragma unroll
      for (uint32_t b = 0; b < 9; ++b)
        if (b < nb) mk &= pf[b] ^ (((r >> b) & 1u) - 1u);
      peq[(uint64_t)r * wpad + q] = mk;
    }
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
  if (n <= kAlphabetOneBlock) {
    k_alphabet<<<1, 1024, 0, st>>>(y, n, codemap, sigma_rows);
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(presence8, 0, 8 * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  k_presence<<<grid_for(n, 256, 1024), 256, 0, st>>>(y, n, presence8);
  k_codemap<<<1, 256, 0, st>>>(presence8, codemap, sigma_rows);
  return cudaGetLastError();
}

cudaError_t launch_xoff(const XoffJob* jobs, int njobs, uint32_t B, const uint16_t* codemap,
                        const uint32_t* sigma_rows, const ZeroSpan* zero, int nzero, const PeqJob* peq,
                        cudaStream_t st) {
  if (njobs < 0 || njobs > 2 || nzero < 0 || nzero > kMaxZeroSpans) return cudaErrorInvalidValue;
  XoffArgs a{};
  uint64_t most = 1;
  unsigned gx = 1;
  if (peq) {
    a.peq = *peq;
    a.npeq = peq->peq_r ? 2u : 1u;
    gx = grid_for(peq->wpad * 32, 256);  // a warp per word
  }
  for (int k = 0; k < njobs; ++k) {
    a.job[k] = jobs[k];
    const uint64_t total = (jobs[k].R + (uint64_t)kPadRowblocks + kPadBackRowblocks) * B;
    most = total > most ? total : most;
  }
  for (int z = 0; z < nzero; ++z) {
    a.zero[z] = zero[z];
    most = zero[z].bytes / 4 > most ? zero[z].bytes / 4 : most;
  }
  a.njobs = (uint32_t)njobs;
  a.nzero = (uint32_t)nzero;
  a.B = B;
  a.codemap = codemap;
  a.sigma_rows = sigma_rows;
  gx = std::max(gx, grid_for(most, 256));
  k_xoff<<<dim3(gx, a.npeq + (unsigned)njobs + 1), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace lcs
