// Learned stencil coefficients: a 4 -> 64 -> 64 -> 8 network (FP32) that maps
// local, scale-free inputs to space-order-8 weights, with hand-written
// inference, training (fused forward + loss + backward) and Adam kernels, and
// the sampling kernels that turn fine-grid runs of the propagator into
// training samples.  The paper has no learned component; the construction
// follows the learned-discretisation idea of Bar-Sinai et al. (PNAS 2019).
//
// Inputs per cell: x = [v dt / h, h / 10 m, dt / 1 ms, f / 10 Hz].
// Outputs o_1..o_8 -> s_j = (o_j + o_{j+4}) / 2, c_j = cT_j (1 + tanh(s_j)/2),
// c_0 = -2 sum_j c_j (symmetric, zero row sum; an all-zero output layer gives
// the Taylor weights cT).  Sample: x[4], T[4] (T_j = sum of the six neighbours
// at distance j minus 6 u), target y, weight w; prediction p = sum_j c_j T_j;
// loss L = (1/n) sum w (p - y)^2.
// Parameters (5000 floats): W1[64][4] b1[64] W2[64][64] b2[64] W3[8][64] b3[8].
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fd_aux.h"
#include "fd_mlp.h"
#include "fd_runtime.h"

using namespace fd;

namespace {

constexpr int H = 64, NIN = 4, NOUT = 8, RL = 4;
constexpr int OW1 = 0, OB1 = OW1 + H * NIN, OW2 = OB1 + H, OB2 = OW2 + H * H,
              OW3 = OB2 + H, OB3 = OW3 + NOUT * H, NPARAM = OB3 + NOUT;
static_assert(NPARAM == FD_MLP_NPARAM, "parameter layout");
constexpr int SAMPLE = FD_MLP_SAMPLE;  // x[4] T[4] y w
constexpr int CHUNK = 128;            // samples per block iteration = threads
constexpr int LD = H + 1;             // padded row of the activation tiles

struct TaylorC {
  float c[RL + 1];
};

__device__ __forceinline__ void load_params(float* sp, const float* __restrict__ p) {
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) sp[i] = p[i];
}

// o = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for one sample; h1 kept.
__device__ __forceinline__ void net_forward(const float* sp, const float x[NIN], float h1[H],
                                            float o[NOUT]) {
#pragma unroll
  for (int i = 0; i < H; ++i) {
    float z = sp[OB1 + i];
#pragma unroll
    for (int c = 0; c < NIN; ++c) z = fmaf(sp[OW1 + i * NIN + c], x[c], z);
    h1[i] = fmaxf(z, 0.0f);
  }
#pragma unroll
  for (int o_ = 0; o_ < NOUT; ++o_) o[o_] = sp[OB3 + o_];
  for (int k = 0; k < H; ++k) {
    float z = sp[OB2 + k];
#pragma unroll
    for (int i = 0; i < H; ++i) z = fmaf(sp[OW2 + k * H + i], h1[i], z);
    const float h2 = fmaxf(z, 0.0f);
#pragma unroll
    for (int o_ = 0; o_ < NOUT; ++o_) o[o_] = fmaf(sp[OW3 + o_ * H + k], h2, o[o_]);
  }
}

__device__ __forceinline__ void coef_from_out(const float o[NOUT], const TaylorC& t,
                                              float c[RL], float th[RL]) {
#pragma unroll
  for (int j = 0; j < RL; ++j) {
    th[j] = tanhf(0.5f * (o[j] + o[j + RL]));
    c[j] = t.c[j + 1] * (1.0f + 0.5f * th[j]);
  }
}

// ---------------------------------------------------------------------------
// inference on feature rows: coef[n][4]
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_mlp_coef_rows(const float* __restrict__ params,
                                                      const float* __restrict__ feat, int n,
                                                      TaylorC t, float* __restrict__ coef) {
  __shared__ float sp[NPARAM];
  load_params(sp, params);
  __syncthreads();
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    float x[NIN], h1[H], o[NOUT], c[RL], th[RL];
#pragma unroll
    for (int q = 0; q < NIN; ++q) x[q] = feat[size_t(s) * NIN + q];
    net_forward(sp, x, h1, o);
    coef_from_out(o, t, c, th);
#pragma unroll
    for (int j = 0; j < RL; ++j) coef[size_t(s) * RL + j] = c[j];
  }
}

// inference on every padded cell of a grid: x0 = v dt / h = sqrt(A h^2/h^2) =
// sqrt(A) because A = dt^2 v^2 / h^2; coefficient field j at coef + j*ncell
__global__ void __launch_bounds__(128) k_mlp_coef_grid(const float* __restrict__ params,
                                                      const float* __restrict__ A,
                                                      size_t ncell, int pitch, int Nx,
                                                      float x1, float x2, float x3,
                                                      TaylorC t, float* __restrict__ coef) {
  __shared__ float sp[NPARAM];
  load_params(sp, params);
  __syncthreads();
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < ncell;
       i += size_t(gridDim.x) * blockDim.x) {
    float c[RL], th[RL];
    if (int(i % pitch) >= Nx) {
#pragma unroll
      for (int j = 0; j < RL; ++j) c[j] = t.c[j + 1];
    } else {
      float x[NIN] = {sqrtf(A[i]), x1, x2, x3}, h1[H], o[NOUT];
      net_forward(sp, x, h1, o);
      coef_from_out(o, t, c, th);
    }
#pragma unroll
    for (int j = 0; j < RL; ++j) coef[j * ncell + i] = c[j];
  }
}

// ---------------------------------------------------------------------------
// training: fused forward, loss and backward over chunks of 128 samples; the
// weight gradients are contractions over the chunk done from shared memory and
// accumulated per thread, then added to the global gradient once per block
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CHUNK, 1)
    k_mlp_grad(const float* __restrict__ params, const float* __restrict__ samples, int n,
               float inv_n, TaylorC t, float* __restrict__ grad, double* __restrict__ loss) {
  extern __shared__ float sm[];
  float* sp = sm;                       // NPARAM
  float* H1 = sp + NPARAM;              // [CHUNK][LD]  h1, later read for dW2
  float* H2 = H1 + CHUNK * LD;          // [CHUNK][LD]  h2, then dz2
  float* D1 = H2 + CHUNK * LD;          // [CHUNK][LD]  dz1
  float* DO = D1 + CHUNK * LD;          // [CHUNK][NOUT]
  float* XS = DO + CHUNK * NOUT;        // [CHUNK][NIN]
  const int tid = threadIdx.x;
  load_params(sp, params);

  // per-thread ownership of gradient entries
  const int k2 = tid & 63, half = tid >> 6;        // dW2[k2][32 half + q]
  const int o3 = tid >> 4, kb3 = (tid & 15) * 4;   // dW3[o3][kb3 + q]
  const int i1 = tid >> 1, cb1 = (tid & 1) * 2;    // dW1[i1][cb1 + q]
  float a2[32], a3[4], a1[2], ab1 = 0.f, ab2 = 0.f, ab3 = 0.f;
#pragma unroll
  for (int q = 0; q < 32; ++q) a2[q] = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) a3[q] = 0.f;
  a1[0] = a1[1] = 0.f;
  double lsum = 0.0;
  __syncthreads();

  for (int base = blockIdx.x * CHUNK; base < n; base += gridDim.x * CHUNK) {
    const int s = base + tid;
    const bool ok = s < n;
    float x[NIN], T[RL], y = 0.f, w = 0.f;
#pragma unroll
    for (int q = 0; q < NIN; ++q) x[q] = ok ? samples[size_t(s) * SAMPLE + q] : 0.f;
#pragma unroll
    for (int q = 0; q < RL; ++q) T[q] = ok ? samples[size_t(s) * SAMPLE + NIN + q] : 0.f;
    if (ok) {
      y = samples[size_t(s) * SAMPLE + NIN + RL];
      w = samples[size_t(s) * SAMPLE + NIN + RL + 1];
    }
    // forward, keeping h1 and h2 rows in shared memory
    float h1[H], o[NOUT];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      float z = sp[OB1 + i];
#pragma unroll
      for (int c = 0; c < NIN; ++c) z = fmaf(sp[OW1 + i * NIN + c], x[c], z);
      h1[i] = fmaxf(z, 0.0f);
      H1[tid * LD + i] = h1[i];
    }
#pragma unroll
    for (int o_ = 0; o_ < NOUT; ++o_) o[o_] = sp[OB3 + o_];
    for (int k = 0; k < H; ++k) {
      float z = sp[OB2 + k];
#pragma unroll
      for (int i = 0; i < H; ++i) z = fmaf(sp[OW2 + k * H + i], h1[i], z);
      const float h2 = fmaxf(z, 0.0f);
      H2[tid * LD + k] = h2;
#pragma unroll
      for (int o_ = 0; o_ < NOUT; ++o_) o[o_] = fmaf(sp[OW3 + o_ * H + k], h2, o[o_]);
    }
    // loss and dL/do
    float c[RL], th[RL];
    coef_from_out(o, t, c, th);
    float p = 0.f;
#pragma unroll
    for (int j = 0; j < RL; ++j) p = fmaf(c[j], T[j], p);
    const float r = p - y;
    lsum += double(w) * double(r) * double(r);
    const float dp = 2.0f * w * r * inv_n;
#pragma unroll
    for (int j = 0; j < RL; ++j) {
      const float ds = dp * T[j] * t.c[j + 1] * 0.5f * (1.0f - th[j] * th[j]);
      DO[tid * NOUT + j] = 0.5f * ds;
      DO[tid * NOUT + j + RL] = 0.5f * ds;
    }
#pragma unroll
    for (int q = 0; q < NIN; ++q) XS[tid * NIN + q] = x[q];
    __syncthreads();

    // dW3 and db3 over the chunk
    for (int ss = 0; ss < CHUNK; ++ss) {
      const float d = DO[ss * NOUT + o3];
#pragma unroll
      for (int q = 0; q < 4; ++q) a3[q] = fmaf(d, H2[ss * LD + kb3 + q], a3[q]);
      if (tid < NOUT) ab3 += DO[ss * NOUT + tid];
    }
    __syncthreads();

    // own sample: dz2 (into the H2 row), dh1, dz1
    float dh1[H];
#pragma unroll
    for (int i = 0; i < H; ++i) dh1[i] = 0.f;
    for (int k = 0; k < H; ++k) {
      float g = 0.f;
#pragma unroll
      for (int o_ = 0; o_ < NOUT; ++o_) g = fmaf(sp[OW3 + o_ * H + k], DO[tid * NOUT + o_], g);
      const float dz2 = H2[tid * LD + k] > 0.f ? g : 0.f;
      H2[tid * LD + k] = dz2;
#pragma unroll
      for (int i = 0; i < H; ++i) dh1[i] = fmaf(sp[OW2 + k * H + i], dz2, dh1[i]);
    }
#pragma unroll
    for (int i = 0; i < H; ++i) D1[tid * LD + i] = h1[i] > 0.f ? dh1[i] : 0.f;
    __syncthreads();

    // dW2, dW1 and the hidden biases over the chunk
    for (int ss = 0; ss < CHUNK; ++ss) {
      const float d2 = H2[ss * LD + k2];
#pragma unroll
      for (int q = 0; q < 32; ++q) a2[q] = fmaf(d2, H1[ss * LD + 32 * half + q], a2[q]);
      const float d1 = D1[ss * LD + i1];
      a1[0] = fmaf(d1, XS[ss * NIN + cb1], a1[0]);
      a1[1] = fmaf(d1, XS[ss * NIN + cb1 + 1], a1[1]);
      if (tid < H) {
        ab1 += D1[ss * LD + tid];
        ab2 += H2[ss * LD + tid];
      }
    }
    __syncthreads();
  }

#pragma unroll
  for (int q = 0; q < 32; ++q) atomicAdd(&grad[OW2 + k2 * H + 32 * half + q], a2[q]);
#pragma unroll
  for (int q = 0; q < 4; ++q) atomicAdd(&grad[OW3 + o3 * H + kb3 + q], a3[q]);
  atomicAdd(&grad[OW1 + i1 * NIN + cb1], a1[0]);
  atomicAdd(&grad[OW1 + i1 * NIN + cb1 + 1], a1[1]);
  if (tid < H) {
    atomicAdd(&grad[OB1 + tid], ab1);
    atomicAdd(&grad[OB2 + tid], ab2);
  }
  if (tid < NOUT) atomicAdd(&grad[OB3 + tid], ab3);
  // block sum of the loss
  for (int off = 16; off > 0; off >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, off);
  if ((tid & 31) == 0) atomicAdd(loss, lsum * double(inv_n));
}

constexpr size_t GRAD_SMEM = sizeof(float) * (NPARAM + 3 * CHUNK * LD + CHUNK * NOUT + CHUNK * NIN);

// Adam (Kingma & Ba, ICLR 2015) with bias correction; step t >= 1.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Stencil values of sampled cells: out[n][1 + 6 rad] = centre, then for
// j = 1..rad the neighbours at -j s and +j s along x, y and z (s = stride);
// cells are padded (x, y, z) indices, outside the grid reads as 0.
__global__ void k_sample_stencil(const float* __restrict__ u, int Nx, int Ny, int Nz, int pitch,
                                 const int* __restrict__ cells, int n, int stride, int rad,
                                 float* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int x = cells[3 * s], y = cells[3 * s + 1], z = cells[3 * s + 2];
  auto at = [&](int xx, int yy, int zz) -> float {
    if (xx < 0 || yy < 0 || zz < 0 || xx >= Nx || yy >= Ny || zz >= Nz) return 0.0f;
    return u[(size_t(zz) * Ny + yy) * pitch + xx];
  };
  const int w = 1 + 6 * rad;
  float* o = out + size_t(s) * w;
  o[0] = at(x, y, z);
  for (int j = 1; j <= rad; ++j) {
    const int d = j * stride;
    o[6 * (j - 1) + 1] = at(x - d, y, z);
    o[6 * (j - 1) + 2] = at(x + d, y, z);
    o[6 * (j - 1) + 3] = at(x, y - d, z);
    o[6 * (j - 1) + 4] = at(x, y + d, z);
    o[6 * (j - 1) + 5] = at(x, y, z - d);
    o[6 * (j - 1) + 6] = at(x, y, z + d);
  }
}

// Training samples from three stencil snapshots at coarse times t-dt, t,
// t+dt: T_j = sum of the six values at distance j - 6 u, target
// y = (u+ - 2u + u-) / C^2 with C = v dt / h, so that the coarse update
// u+ = 2u - u- + C^2 sum_j c_j T_j reproduces the fine solution; weight
// w = 1 / (scale + mean of the squared stencil values).
__global__ void k_make_samples(const float* __restrict__ prev, const float* __restrict__ cur,
                               const float* __restrict__ next, const float* __restrict__ vel,
                               int n, float h, float dt, float f, float scale,
                               float* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int w = 1 + 6 * RL;
  const float* c = cur + size_t(s) * w;
  const float u = c[0];
  float* o = out + size_t(s) * SAMPLE;
  const float C = vel[s] * dt / h;
  o[0] = C;
  o[1] = h / 10.0f;
  o[2] = dt / 1.0f;
  o[3] = f / 10.0f;
  float ms = u * u;
  for (int j = 1; j <= RL; ++j) {
    float sum = 0.f;
    for (int q = 1; q <= 6; ++q) {
      const float v = c[6 * (j - 1) + q];
      sum += v;
      ms += v * v;
    }
    o[NIN + j - 1] = sum - 6.0f * u;
  }
  o[NIN + RL] = (next[size_t(s) * w] - 2.0f * u + prev[size_t(s) * w]) / (C * C);
  o[NIN + RL + 1] = 1.0f / (scale + ms / float(w));
}

TaylorC taylor_c() {
  TaylorC t;
  double c[RL + 1], sum = 0.0;
  for (int j = 1; j <= RL; ++j) {
    double ratio = 1.0;
    for (int k = 1; k <= j; ++k) ratio *= double(RL - k + 1) / double(RL + k);
    c[j] = ((j & 1) ? 2.0 : -2.0) * ratio / (double(j) * j);
    sum += c[j];
  }
  c[0] = -2.0 * sum;
  for (int j = 0; j <= RL; ++j) t.c[j] = float(c[j]);
  return t;
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

}  // namespace

struct fd_mlp_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  float* p = nullptr;   // params
  float* g = nullptr;   // gradient
  float* m = nullptr;   // Adam first moment
  float* v = nullptr;   // Adam second moment
  double* loss = nullptr;
  int t = 0;            // Adam step count
  DevBuf stage, stage2;
};

namespace fd {

fd_status mlp_grid_coefficients(fd_mlp net, const float* A, size_t ncell, int pitch, int Nx,
                                double h, double dt, double f_hz, float* coef,
                                cudaStream_t s) {
  const TaylorC t = taylor_c();
  const int grid = std::max(1, std::min<int>(sm_count() * 8, int((ncell + 127) / 128)));
  k_mlp_coef_grid<<<grid, 128, 0, s>>>(net->p, A, ncell, pitch, Nx, float(h / 10.0),
                                       float(dt / 1.0), float(f_hz / 10.0), t, coef);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e) return cuda_fail(e, "learned coefficient inference");
  return FD_OK;
}

}  // namespace fd

extern "C" {

fd_status fd_mlp_create(int32_t device, const float* params, fd_mlp* out) {
  clear_error();
  if (!out) return fail(FD_ERR_ARG, "null argument");
  *out = nullptr;
  cudaError_t e = cudaSetDevice(device);
  if (e) return cuda_fail(e, "cudaSetDevice");
  fd_mlp net = new fd_mlp_s();
  net->device = device;
  fd_status st = FD_OK;
  e = cudaStreamCreateWithFlags(&net->stream, cudaStreamDefault);  // see fd_create_grid
  float** bufs[4] = {&net->p, &net->g, &net->m, &net->v};
  for (int i = 0; i < 4 && !e; ++i) e = dev_alloc(reinterpret_cast<void**>(bufs[i]), NPARAM * 4);
  if (!e) e = dev_alloc(reinterpret_cast<void**>(&net->loss), 16);
  if (!e) {
    for (int i = 0; i < 4 && !e; ++i) e = cudaMemsetAsync(*bufs[i], 0, NPARAM * 4, net->stream);
    if (!e && params) e = cudaMemcpyAsync(net->p, params, NPARAM * 4, cudaMemcpyDefault,
                                          net->stream);
    if (!e) e = cudaStreamSynchronize(net->stream);
  }
  if (e) st = cuda_fail(e, "network allocation");
  if (st) {
    fd_mlp_destroy(net);
    return st;
  }
  *out = net;
  return FD_OK;
}

fd_status fd_mlp_destroy(fd_mlp net) {
  if (!net) return FD_OK;
  cudaSetDevice(net->device);
  if (net->stream) cudaStreamSynchronize(net->stream);
  for (float* p : {net->p, net->g, net->m, net->v})
    if (p) cudaFree(p);
  if (net->loss) cudaFree(net->loss);
  net->stage.release();
  net->stage2.release();
  if (net->stream) cudaStreamDestroy(net->stream);
  delete net;
  return FD_OK;
}

fd_status fd_mlp_get_params(fd_mlp net, float* out) {
  clear_error();
  if (!net || !out) return fail(FD_ERR_ARG, "null argument");
  cudaSetDevice(net->device);
  cudaError_t e = cudaMemcpyAsync(out, net->p, NPARAM * 4, cudaMemcpyDefault, net->stream);
  if (!e) e = cudaStreamSynchronize(net->stream);
  if (e) return cuda_fail(e, "parameter read");
  return FD_OK;
}

fd_status fd_mlp_set_params(fd_mlp net, const float* in) {
  clear_error();
  if (!net || !in) return fail(FD_ERR_ARG, "null argument");
  cudaSetDevice(net->device);
  cudaError_t e = cudaMemcpyAsync(net->p, in, NPARAM * 4, cudaMemcpyDefault, net->stream);
  if (!e) e = cudaMemsetAsync(net->m, 0, NPARAM * 4, net->stream);
  if (!e) e = cudaMemsetAsync(net->v, 0, NPARAM * 4, net->stream);
  if (!e) e = cudaStreamSynchronize(net->stream);
  if (e) return cuda_fail(e, "parameter write");
  net->t = 0;
  return FD_OK;
}

static fd_status mlp_grad_device(fd_mlp net, int64_t n, const float* dsamples, double* loss) {
  cudaError_t e = cudaMemsetAsync(net->g, 0, NPARAM * 4, net->stream);
  if (!e) e = cudaMemsetAsync(net->loss, 0, sizeof(double), net->stream);
  if (e) return cuda_fail(e, "gradient reset");
  if (n > 0) {
    static bool attr = false;
    if (!attr) {
      e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               int(GRAD_SMEM));
      if (e) return cuda_fail(e, "kernel attribute");
      attr = true;
    }
    const int blocks = int(std::min<int64_t>(sm_count(), (n + CHUNK - 1) / CHUNK));
    k_mlp_grad<<<blocks, CHUNK, GRAD_SMEM, net->stream>>>(net->p, dsamples, int(n),
                                                          float(1.0 / double(n)), taylor_c(),
                                                          net->g, net->loss);
    count_launch();
    if ((e = cudaGetLastError())) return cuda_fail(e, "training kernel");
  }
  if (loss) {
    e = cudaMemcpyAsync(loss, net->loss, sizeof(double), cudaMemcpyDeviceToHost, net->stream);
    if (!e) e = cudaStreamSynchronize(net->stream);
    if (e) return cuda_fail(e, "loss read");
  }
  return FD_OK;
}

fd_status fd_mlp_loss_grad(fd_mlp net, int64_t n, const float* samples, double* loss,
                           float* grad_out) {
  clear_error();
  if (!net || (n > 0 && !samples)) return fail(FD_ERR_ARG, "null argument");
  if (n < 0 || n > INT32_MAX) return fail(FD_ERR_ARG, "bad sample count");
  cudaSetDevice(net->device);
  const float* d = samples;
  if (n > 0 && !is_device_ptr(samples)) {
    cudaError_t e = net->stage.ensure(size_t(n) * SAMPLE * 4);
    if (!e) e = cudaMemcpyAsync(net->stage.p, samples, size_t(n) * SAMPLE * 4,
                                cudaMemcpyHostToDevice, net->stream);
    if (e) return cuda_fail(e, "sample upload");
    d = static_cast<const float*>(net->stage.p);
  }
  fd_status st = mlp_grad_device(net, n, d, loss);
  if (st) return st;
  if (grad_out) {
    cudaError_t e = cudaMemcpyAsync(grad_out, net->g, NPARAM * 4, cudaMemcpyDefault, net->stream);
    if (!e) e = cudaStreamSynchronize(net->stream);
    if (e) return cuda_fail(e, "gradient read");
  }
  return FD_OK;
}

static fd_status adam_device(fd_mlp net, float lr) {
  net->t += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = float(1.0 - pow(0.9, net->t)), c2 = float(1.0 - pow(0.999, net->t));
  k_adam<<<(NPARAM + 255) / 256, 256, 0, net->stream>>>(net->p, net->g, net->m, net->v, NPARAM,
                                                       lr, b1, b2, eps, c1, c2);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e) return cuda_fail(e, "adam");
  return FD_OK;
}

fd_status fd_mlp_adam_step(fd_mlp net, float lr) {
  clear_error();
  if (!net || !(lr > 0.f)) return fail(FD_ERR_ARG, "bad argument");
  cudaSetDevice(net->device);
  fd_status st = adam_device(net, lr);
  if (st) return st;
  cudaError_t e = cudaStreamSynchronize(net->stream);
  if (e) return cuda_fail(e, "adam");
  return FD_OK;
}

fd_status fd_mlp_train(fd_mlp net, int64_t n, const float* samples, int32_t epochs,
                       int32_t batch, float lr, double* loss_out) {
  clear_error();
  if (!net || !samples || n <= 0 || epochs < 0 || batch <= 0 || !(lr > 0.f))
    return fail(FD_ERR_ARG, "bad argument");
  cudaSetDevice(net->device);
  const float* d = samples;
  if (!is_device_ptr(samples)) {
    cudaError_t e = net->stage.ensure(size_t(n) * SAMPLE * 4);
    if (!e) e = cudaMemcpyAsync(net->stage.p, samples, size_t(n) * SAMPLE * 4,
                                cudaMemcpyHostToDevice, net->stream);
    if (e) return cuda_fail(e, "sample upload");
    d = static_cast<const float*>(net->stage.p);
  }
  fd_status st;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int64_t b0 = 0; b0 < n; b0 += batch) {
      const int64_t nb = std::min<int64_t>(batch, n - b0);
      if ((st = mlp_grad_device(net, nb, d + size_t(b0) * SAMPLE, nullptr))) return st;
      if ((st = adam_device(net, lr))) return st;
    }
  }
  if (loss_out) {
    // loss of the whole set with the final parameters
    double total = 0.0;
    for (int64_t b0 = 0; b0 < n; b0 += (int64_t(1) << 24)) {
      const int64_t nb = std::min<int64_t>(int64_t(1) << 24, n - b0);
      double l = 0.0;
      if ((st = mlp_grad_device(net, nb, d + size_t(b0) * SAMPLE, &l))) return st;
      total += l * double(nb);
    }
    *loss_out = total / double(n);
  }
  cudaError_t e = cudaStreamSynchronize(net->stream);
  if (e) return cuda_fail(e, "training");
  return FD_OK;
}

fd_status fd_mlp_coefficients(fd_mlp net, int64_t n, const float* features, float* coef_out) {
  clear_error();
  if (!net || (n > 0 && (!features || !coef_out))) return fail(FD_ERR_ARG, "null argument");
  cudaSetDevice(net->device);
  if (n == 0) return FD_OK;
  const float* fin = features;
  float* cout = coef_out;
  cudaError_t e = cudaSuccess;
  if (!is_device_ptr(features)) {
    e = net->stage.ensure(size_t(n) * NIN * 4);
    if (!e) e = cudaMemcpyAsync(net->stage.p, features, size_t(n) * NIN * 4,
                                cudaMemcpyHostToDevice, net->stream);
    fin = static_cast<const float*>(net->stage.p);
  }
  const bool host_out = !is_device_ptr(coef_out);
  if (!e && host_out) {
    e = net->stage2.ensure(size_t(n) * RL * 4);
    cout = static_cast<float*>(net->stage2.p);
  }
  if (e) return cuda_fail(e, "staging");
  const int grid = int(std::min<int64_t>(sm_count() * 8, (n + 127) / 128));
  k_mlp_coef_rows<<<grid, 128, 0, net->stream>>>(net->p, fin, int(n), taylor_c(), cout);
  count_launch();
  if ((e = cudaGetLastError())) return cuda_fail(e, "inference");
  if (host_out)
    e = cudaMemcpyAsync(coef_out, cout, size_t(n) * RL * 4, cudaMemcpyDeviceToHost, net->stream);
  if (!e) e = cudaStreamSynchronize(net->stream);
  if (e) return cuda_fail(e, "inference");
  return FD_OK;
}

fd_status fd_sample_stencil(fd_grid g, int32_t n, const int32_t* cells, int32_t stride,
                            int32_t radius, float* out) {
  clear_error();
  if (!g || (n > 0 && (!cells || !out)) || n < 0 || stride < 1 || radius < 0 || radius > 8)
    return fail(FD_ERR_ARG, "bad argument");
  if (n == 0) return FD_OK;
  cudaSetDevice(g->d.device);
  const size_t w = 1 + 6 * size_t(radius);
  cudaError_t e = g->stage_aux.ensure(size_t(n) * 3 * 4 + 256 + size_t(n) * w * 4);
  if (e) return cuda_fail(e, "staging");
  int* dcells = static_cast<int*>(g->stage_aux.p);
  float* dout = reinterpret_cast<float*>(static_cast<char*>(g->stage_aux.p) +
                                         ((size_t(n) * 12 + 255) / 256) * 256);
  e = cudaMemcpyAsync(dcells, cells, size_t(n) * 12, cudaMemcpyDefault, g->stream);
  if (e) return cuda_fail(e, "cell upload");
  float* target = is_device_ptr(out) ? out : dout;
  k_sample_stencil<<<(n + 127) / 128, 128, 0, g->stream>>>(g->F.u[g->F.cur], g->Nx, g->Ny, g->Nz,
                                                          g->pitch, dcells, n, stride, radius,
                                                          target);
  count_launch();
  if ((e = cudaGetLastError())) return cuda_fail(e, "stencil sampling");
  if (target != out)
    e = cudaMemcpyAsync(out, target, size_t(n) * w * 4, cudaMemcpyDeviceToHost, g->stream);
  if (!e) e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_fail(e, "stencil sampling");
  return FD_OK;
}

fd_status fd_mlp_make_samples(int32_t n, const float* prev, const float* cur, const float* next,
                              const float* vel, double h, double dt, double f_hz, double scale,
                              float* out) {
  clear_error();
  if (n < 0 || (n > 0 && (!prev || !cur || !next || !vel || !out)))
    return fail(FD_ERR_ARG, "bad argument");
  if (n == 0) return FD_OK;
  for (const void* p : {(const void*)prev, (const void*)cur, (const void*)next,
                        (const void*)vel, (const void*)out})
    if (!is_device_ptr(p)) return fail(FD_ERR_ARG, "fd_mlp_make_samples takes device arrays");
  k_make_samples<<<(n + 127) / 128, 128>>>(prev, cur, next, vel, n, float(h), float(dt),
                                           float(f_hz), float(scale), out);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (!e) e = cudaDeviceSynchronize();
  if (e) return cuda_fail(e, "sample assembly");
  return FD_OK;
}

}  // extern "C"
