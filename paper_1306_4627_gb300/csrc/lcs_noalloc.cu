// lcs_length_noalloc: the LCS length of two device strings computed entirely in a fixed, statically reserved
// scratch region of device memory, for callers that must not allocate device memory themselves or through this
// library (see include/lcs.h).
//
// The scratch is one file-scope __device__ array. Host code cannot use the array's name as a device address (on
// the host it only names a stand-in object), so the first call on each device looks the real address up with
// cudaGetSymbolAddress while that device is current, and carves the per-call buffers out of it. Every call on a
// device shares the array and leaves its contents behind; the length path clears everything that must start at
// zero (carry slots, length accumulator) before each use, and the status word is cleared whenever it reports an
// error. Calls are serialised per device on the host and each call waits for its own work (also when it fails after
// enqueueing part of it), so two calls of this entry point never overlap on the GPU; work that the caller enqueues
// on other streams while a call runs must not touch the array (nothing outside this file can).
//
// The carved buffers are marked fixed: the length path's grow-only ensure() never frees or replaces them. A request
// that did not fit one (a sizing mistake in carve()) fails the call with LCS_ERR_INTERNAL instead of allocating.
#include <mutex>
#include <functional>
#include <new>

#include "lcs_ctx.h"

namespace lcs {
int run_length(lcs_ctx* c, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n, uint64_t* d_out,
               cudaStream_t st);
}  // namespace lcs

namespace {

constexpr uint64_t kMaxLen = 65536;               // largest m and n accepted
constexpr size_t kScratchBytes = 6815744;         // 6.5 MiB, held by every GPU that loads the library
constexpr uint32_t kRowsPerStep = 8;              // the fill geometry this scratch layout is sized for

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceSlot {
  std::once_flag once;
  std::mutex mu;
  lcs_ctx* ctx = nullptr;
  int rc = LCS_OK;
};
constexpr int kMaxDevices = 64;
DeviceSlot g_slots[kMaxDevices];

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Carves the buffers the length path uses at m, n <= kMaxLen out of the scratch array (base = its device address).
// Each capacity is the largest size the length path asks for in that range, so it never needs to grow one.
int carve(lcs_ctx* c, unsigned char* base) {
  const uint64_t wq = kMaxLen / 32 + 1;
  const uint64_t nblocks = (wq + lcs::kStripeWords - 1) / lcs::kStripeWords;
  const uint64_t wpad = nblocks * lcs::kStripeWords;
  const uint64_t R = (kMaxLen + kRowsPerStep - 1) / kRowsPerStep;  // rows of one table, without the split
  const size_t peq = (size_t)lcs::kSigmaMax * wpad * 4;
  const size_t xoff = (size_t)(R + lcs::kPadRowblocks + lcs::kPadBackRowblocks) * kRowsPerStep * 4;
  const size_t carry = (size_t)nblocks * R * 4;
  const size_t fv = (size_t)wpad * 4;
  const size_t colsum = (size_t)(2 * (wq + 1) + 4) * 4;
  struct Part {
    lcs::DBuf* b;
    size_t bytes;
  } parts[] = {{&c->small, lcs::kSmallBytes}, {&c->peq_f, peq}, {&c->peq_r, peq},   {&c->xoff_f, xoff},
               {&c->xoff_r, xoff},            {&c->carry_f, carry}, {&c->carry_r, carry}, {&c->fv_f, fv},
               {&c->fv_r, fv},                {&c->colsum, colsum}};
  size_t off = 0;
  for (auto& p : parts) {
    const size_t sz = align256(p.bytes);
    if (off + sz > kScratchBytes) return LCS_ERR_INTERNAL;
    p.b->p = base + off;
    p.b->cap = sz;
    p.b->fixed = true;
    off += sz;
  }
  return LCS_OK;
}

// True when a request did not fit one of the carved buffers during the last call (clears the flags).
bool carved_overflow(lcs_ctx* c) {
  lcs::DBuf* all[] = {&c->small, &c->peq_f, &c->peq_r, &c->xoff_f, &c->xoff_r,
                      &c->carry_f, &c->carry_r, &c->fv_f, &c->fv_r, &c->colsum};
  bool any = false;
  for (lcs::DBuf* b : all) {
    any = any || b->overflow;
    b->overflow = false;
  }
  return any;
}

// Reads the status word on the call's own stream (one copy into host stack memory, one wait for that stream) and
// clears it when it holds an error.
int status_on_stream(lcs_ctx* c, cudaStream_t st) {
  lcs::DevStatus h{};
  int rc = lcs::from_cuda(cudaMemcpyAsync(&h, c->status(), sizeof(h), cudaMemcpyDeviceToHost, st));
  if (!rc) rc = lcs::from_cuda(cudaStreamSynchronize(st));
  if (rc) return rc;
  if (h.flags == 0) return LCS_OK;
  cudaMemsetAsync(c->status(), 0, sizeof(lcs::DevStatus), st);
  cudaStreamSynchronize(st);
  return (h.flags & lcs::kStatTimeout) ? LCS_ERR_TIMEOUT : LCS_ERR_INTERNAL;
}

void setup(DeviceSlot& slot, int device) {
  void* base = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&base, g_scratch);  // the device's address of the array
  if (e != cudaSuccess || !base) {
    cudaGetLastError();
    slot.rc = LCS_ERR_CUDA;
    return;
  }
  lcs_ctx* c = new (std::nothrow) lcs_ctx();
  if (!c) {
    slot.rc = LCS_ERR_INTERNAL;
    return;
  }
  c->device = device;
  c->fill_B = kRowsPerStep;
  c->max_coop = lcs::fill_max_coop_blocks(device);
  if (c->max_coop <= 0) {
    delete c;
    slot.rc = LCS_ERR_CUDA;
    return;
  }
  slot.rc = carve(c, static_cast<unsigned char*>(base));
  if (slot.rc != LCS_OK) {
    delete c;
    return;
  }
  slot.ctx = c;
}

}  // namespace

extern "C" int lcs_length_noalloc(const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n,
                                  uint64_t* d_out_len, void* stream) {
  if (!d_out_len || (m && !d_x) || (n && !d_y)) return LCS_ERR_INVALID;
  if (m > kMaxLen || n > kMaxLen) return LCS_ERR_INVALID;
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) {
    cudaGetLastError();
    return LCS_ERR_CUDA;
  }
  DeviceSlot& slot = g_slots[device];
  std::call_once(slot.once, setup, std::ref(slot), device);  // first call on this device, with it current
  if (slot.rc != LCS_OK) return slot.rc;
  std::lock_guard<std::mutex> g(slot.mu);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = lcs::run_length(slot.ctx, d_x, m, d_y, n, d_out_len, st);
  if (rc) {
    // part of the call may be enqueued already: let it finish before the next call can use the array
    cudaStreamSynchronize(st);
    cudaGetLastError();
    return carved_overflow(slot.ctx) ? LCS_ERR_INTERNAL : rc;
  }
  return status_on_stream(slot.ctx, st);
}
