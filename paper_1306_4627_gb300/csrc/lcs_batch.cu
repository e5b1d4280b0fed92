// lcs_batch: LCS lengths of many independent pairs.
#include <algorithm>
#include <mutex>
#include <vector>

#include "lcs_ctx.h"

using namespace lcs;

namespace lcs {
int run_length(lcs_ctx* c, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n, uint64_t* d_out,
               cudaStream_t st);
int take_status(lcs_ctx* c);
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
  std::vector<uint64_t> xo(count + 1), yo(count + 1);
  int rc = from_cuda(cudaMemcpyAsync(xo.data(), d_x_off, (count + 1) * 8, cudaMemcpyDeviceToHost, st));
  if (!rc) rc = from_cuda(cudaMemcpyAsync(yo.data(), d_y_off, (count + 1) * 8, cudaMemcpyDeviceToHost, st));
  if (!rc) rc = from_cuda(cudaStreamSynchronize(st));
  if (rc) return rc;
  if (!offsets_ok(xo.data(), count) || !offsets_ok(yo.data(), count)) return LCS_ERR_INVALID;
  for (uint64_t k = 0; k < count && !rc; ++k)
    rc = run_length(c, d_xs + xo[k], xo[k + 1] - xo[k], d_ys + yo[k], yo[k + 1] - yo[k], d_out_lens + k, st);
  return rc;
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
  DBuf outs;
  if (!rc) rc = from_cuda(ensure(outs, count * 8));
  if (!rc && nx) rc = from_cuda(cudaMemcpyAsync(c->x.p, xs + x_off[0], nx, cudaMemcpyHostToDevice, c->stream));
  if (!rc && ny) rc = from_cuda(cudaMemcpyAsync(c->y.p, ys + y_off[0], ny, cudaMemcpyHostToDevice, c->stream));
  const uint8_t* dx = (const uint8_t*)c->x.p;
  const uint8_t* dy = (const uint8_t*)c->y.p;
  for (uint64_t k = 0; k < count && !rc; ++k)
    rc = run_length(c, dx + (x_off[k] - x_off[0]), x_off[k + 1] - x_off[k], dy + (y_off[k] - y_off[0]),
                    y_off[k + 1] - y_off[k], (uint64_t*)outs.p + k, c->stream);
  if (!rc) rc = from_cuda(cudaMemcpyAsync(out_lens, outs.p, count * 8, cudaMemcpyDeviceToHost, c->stream));
  if (!rc) rc = from_cuda(cudaStreamSynchronize(c->stream));
  if (!rc) rc = take_status(c);
  release(outs);
  return rc;
}
