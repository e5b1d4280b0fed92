// Measurements of the ceilings the table fill is compared against (no counterpart in the paper, which times its
// method only; §II.A EXEC_TIME). Two probes, both behind the C ABI (include/lcs.h):
//
//   * lcs_probe_int_rate: the INT32 throughput of the whole GPU for the instruction sequence of one row update of
//     one 32-column word (§I.C recurrence in bit-parallel form: U = V & P; the carry-in shift, S = V + U + carry and
//     the carry collection as one add.cc / addc.cc / addc chain; V' = S | (V & ~P)), optionally with the traceback's
//     T = S ^ V ^ U, or plain three-input logic operations. Every thread runs four independent chains, every SM
//     holds as many blocks as fit, so nothing but the integer pipes bounds the rate. It is the ALU roofline of the
//     fill: the most row updates per second this GPU can execute.
//   * lcs_probe_step_floor (lcs_fill.cu): the dependency floor of one systolic step of the fill.
//   * lcs_probe_step_masks (lcs_fill.cu): the same step with its match masks from the fill's shared table or formed
//     in registers from bit planes of Y's codes, to weigh the two ways of supplying them.
#include <algorithm>
#include <vector>

#include "lcs_internal.h"

namespace lcs {
namespace {

constexpr int kChains = 4;       // independent chains per thread
constexpr int kRateThreads = 256;

// MIX 0: the row update (5 instructions per chain and iteration); MIX 1: plus T = S ^ V ^ U, which becomes the next
// iteration's mask (6); MIX 2: one three-input XOR per chain (1).
template <int MIX>
__global__ void __launch_bounds__(kRateThreads) k_int_rate(const uint32_t* in, uint32_t iters,
                                                          unsigned long long* cyc, uint32_t* sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t V[kChains], P[kChains], cw[kChains], co[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    V[k] = in[(tid * kChains + k) & 1023];
    P[k] = in[(tid * kChains + k + 512) & 1023];
    cw[k] = V[k] ^ P[k];
    co[k] = 0;
  }
  __syncthreads();
  const long long t0 = clock64();
#pragma unroll 1
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if (MIX == 2) {
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(V[k]) : "r"(P[k]), "r"(cw[k]));
      } else {
        uint32_t U, S;
        asm volatile(
            "and.b32 %3, %4, %5;\n\t"
            "add.cc.u32 %0, %0, %0;\n\t"
            "addc.cc.u32 %2, %4, %3;\n\t"
            "addc.u32 %1, %1, %1;\n\t"
            : "+r"(cw[k]), "+r"(co[k]), "=&r"(S), "=&r"(U)
            : "r"(V[k]), "r"(P[k]));
        if (MIX == 1) {
          uint32_t T;
          asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(T) : "r"(S), "r"(V[k]), "r"(U));
          asm volatile("lop3.b32 %0, %1, %0, %2, 0xF4;" : "+r"(V[k]) : "r"(S), "r"(P[k]));
          P[k] = T;
        } else {
          asm volatile("lop3.b32 %0, %1, %0, %2, 0xF4;" : "+r"(V[k]) : "r"(S), "r"(P[k]));
        }
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) cyc[blockIdx.x] = (unsigned long long)(t1 - t0);
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc ^= V[k] ^ co[k] ^ P[k];
  sink[tid] = acc;
}

template <int MIX>
int int_rate_t(int device, uint32_t iters, lcs_int_rate* out) {
  constexpr double kOps = MIX == 2 ? 1.0 : (MIX == 1 ? 6.0 : 5.0);
  int sms = 0, per_sm = 0;
  if (cudaSetDevice(device) != cudaSuccess) return LCS_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0)
    return LCS_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_int_rate<MIX>, kRateThreads, 0) != cudaSuccess ||
      per_sm <= 0)
    return LCS_ERR_CUDA;
  const uint32_t grid = (uint32_t)(sms * per_sm);  // one wave: every block resident at once
  uint32_t *in = nullptr, *sink = nullptr;
  unsigned long long* cyc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&in, 1024 * 4);
  if (e == cudaSuccess) e = cudaMalloc(&sink, (size_t)grid * kRateThreads * 4);
  if (e == cudaSuccess) e = cudaMalloc(&cyc, (size_t)grid * 8);
  if (e == cudaSuccess) e = cudaMemset(in, 0x5A, 1024 * 4);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  std::vector<unsigned long long> hc(grid, 0);
  if (e == cudaSuccess) {
    k_int_rate<MIX><<<grid, kRateThreads>>>(in, iters / 8 + 1, cyc, sink);  // warm-up (clocks ramp, code loads)
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0);
  if (e == cudaSuccess) {
    k_int_rate<MIX><<<grid, kRateThreads>>>(in, iters, cyc, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaMemcpy(hc.data(), cyc, (size_t)grid * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && ms > 0.f) {
    const double ops = (double)grid * kRateThreads * (double)iters * kChains * kOps;
    const unsigned long long cmax = *std::max_element(hc.begin(), hc.end());
    out->ops_per_s = ops / (ms * 1e-3);
    out->ops_per_clk_sm = cmax ? ops / (double)sms / (double)cmax : 0.0;
    out->sm_clock_mhz = cmax ? (double)cmax / (ms * 1e-3) / 1e6 : 0.0;
    out->kernel_ms = ms;
    out->sms = sms;
    out->blocks_per_sm = per_sm;
    out->ops_per_chain = (uint32_t)kOps;
    out->threads = grid * kRateThreads;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(in);
  cudaFree(sink);
  cudaFree(cyc);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LCS_ERR_CUDA;
  }
  return ms > 0.f ? LCS_OK : LCS_ERR_INTERNAL;
}

}  // namespace
}  // namespace lcs

extern "C" int lcs_probe_int_rate(int device, uint32_t mix, uint32_t iters, lcs_int_rate* out) {
  if (!out || mix > 2 || iters == 0) return LCS_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return LCS_ERR_INVALID;
  }
  *out = lcs_int_rate{};
  if (mix == 0) return lcs::int_rate_t<0>(device, iters, out);
  if (mix == 1) return lcs::int_rate_t<1>(device, iters, out);
  return lcs::int_rate_t<2>(device, iters, out);
}

extern "C" int lcs_probe_step_floor(int device, uint32_t rows_per_step, int traceback, uint32_t steps,
                                    double* cycles_per_step) {
  if (!cycles_per_step || (rows_per_step != 8 && rows_per_step != 16) || steps == 0 || steps > (1u << 24))
    return LCS_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return LCS_ERR_INVALID;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return LCS_ERR_CUDA;
  }
  const cudaError_t e = lcs::step_floor(rows_per_step, traceback != 0, steps, cycles_per_step);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LCS_ERR_CUDA;
  }
  return LCS_OK;
}

extern "C" int lcs_probe_step_masks(int device, uint32_t source, uint32_t steps, double* cycles_per_step) {
  if (!cycles_per_step || source > 3 || steps == 0 || steps > (1u << 24)) return LCS_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return LCS_ERR_INVALID;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return LCS_ERR_CUDA;
  }
  const cudaError_t e = lcs::step_masks(source, steps, cycles_per_step);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LCS_ERR_CUDA;
  }
  return LCS_OK;
}
