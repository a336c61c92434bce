// Model update of a full-waveform-inversion loop.
//
// The paper names full-waveform inversion as a user of the propagator (Sec. I
// and IV-B) without giving an update rule; this is the normalised
// steepest-descent step that such a loop takes once the shot gradients have
// been summed:
//     alpha = step * max|m| / max|g|,   m <- clamp(m - alpha g, m_min, m_max),
// so that the largest change of one step is `step` times the model's scale.
// Two kernels: one pass for max|m|, max|g| and the count of non-finite
// gradient values (non-negative floats order like their bit patterns, so
// unsigned atomicMax gives the float maximum), one elementwise pass.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "fd_aux.h"
#include "fd_runtime.h"

namespace fd {
namespace {

__global__ void k_absmax2(const float* __restrict__ m, const float* __restrict__ g, size_t n,
                          unsigned int* out) {
  float am = 0.0f, ag = 0.0f;
  int bad = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    if (!isfinite(gi)) {
      ++bad;
      continue;
    }
    am = fmaxf(am, fabsf(m[i]));
    ag = fmaxf(ag, fabsf(gi));
  }
  for (int o = 16; o > 0; o >>= 1) {
    am = fmaxf(am, __shfl_down_sync(0xffffffffu, am, o));
    ag = fmaxf(ag, __shfl_down_sync(0xffffffffu, ag, o));
    bad += __shfl_down_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out + 0, __float_as_uint(am));
    atomicMax(out + 1, __float_as_uint(ag));
    if (bad) atomicAdd(out + 2, static_cast<unsigned int>(bad));
  }
}

__global__ void k_descent(float* __restrict__ m, const float* __restrict__ g, size_t n,
                          float alpha, float lo, float hi) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    m[i] = fminf(fmaxf(fmaf(-alpha, g[i], m[i]), lo), hi);
}

int blocks_for(size_t n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = (n + 255) / 256;
  return int(std::max<size_t>(1, std::min<size_t>(want, size_t(std::max(1, sms)) * 8)));
}

}  // namespace
}  // namespace fd

using namespace fd;

extern "C" fd_status fd_descent_step(int64_t n, float* m, const float* grad, double step,
                                     double m_min, double m_max, void* stream,
                                     double* alpha_out) {
  clear_error();
  if (alpha_out) *alpha_out = 0.0;
  if (n < 0) return fail(FD_ERR_ARG, "n must be >= 0");
  if (n == 0) return FD_OK;
  if (!m || !grad) return fail(FD_ERR_ARG, "null argument");
  if (!(step >= 0.0) || !(m_min <= m_max))
    return fail(FD_ERR_ARG, "need step >= 0 and m_min <= m_max");
  if (!is_device_ptr(m) || !is_device_ptr(grad))
    return fail(FD_ERR_ARG, "fd_descent_step takes device arrays only");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned int* scratch = nullptr;
  cudaError_t e = dev_alloc(reinterpret_cast<void**>(&scratch), 4 * sizeof(unsigned int));
  if (e) return cuda_fail(e, "update scratch allocation");
  unsigned int h[4] = {0, 0, 0, 0};
  const int nb = blocks_for(size_t(n));
  e = cudaMemsetAsync(scratch, 0, sizeof(h), s);
  if (!e) {
    k_absmax2<<<nb, 256, 0, s>>>(m, grad, size_t(n), scratch);
    count_launch();
    e = cudaGetLastError();
  }
  if (!e) e = cudaMemcpyAsync(h, scratch, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaStreamSynchronize(s);
  fd_status st = FD_OK;
  if (e) {
    st = cuda_fail(e, "gradient maxima");
  } else if (h[2]) {
    st = fail(FD_ERR_NONFINITE, "%u gradient values are NaN or Inf", h[2]);
  } else {
    float mmax, gmax;
    memcpy(&mmax, &h[0], 4);
    memcpy(&gmax, &h[1], 4);
    const double alpha = gmax > 0.0f ? step * double(mmax) / double(gmax) : 0.0;
    if (alpha > 0.0) {
      k_descent<<<nb, 256, 0, s>>>(m, grad, size_t(n), float(alpha), float(m_min),
                                   float(m_max));
      count_launch();
      e = cudaGetLastError();
      if (!e) e = cudaStreamSynchronize(s);
      if (e) st = cuda_fail(e, "model update");
    }
    if (!st && alpha_out) *alpha_out = alpha;
  }
  cudaFree(scratch);
  return st;
}
