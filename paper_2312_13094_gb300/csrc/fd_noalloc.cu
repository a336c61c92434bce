// Forward modelling without any device allocation.
//
// Some callers cannot allocate device memory at the time they want a forward
// run: code that runs while another framework owns the memory pool and has
// forbidden new cudaMalloc calls, processes that must keep a fixed device
// footprint, or callers inside a region where an allocation would synchronise
// the device.  fd_forward_noalloc serves them: the wavefields, the model term,
// the source/receiver tables, the launch descriptor and the error words all
// live in one file-scope __device__ array of FD_NOALLOC_MAX_BYTES, which every
// GPU that loads this module keeps until the process exits.  The caller still
// passes its inputs (model, wavelet) and output (receivers) in device memory.
//
// The array's name is only a host-side stand-in in host code; its device
// address is looked up with cudaGetSymbolAddress (with the call's device
// current) on every call whose stream is not being captured, so an address
// made stale by a cudaDeviceReset of the caller is replaced; a call made while
// its stream is being captured reuses the address of the device's last call,
// which is why the first call on a device should come before any stream
// capture.  All calls share the one array and leave the last call's contents
// behind; everything that must start at zero is cleared by the call, and calls
// that overlap on the GPU (other threads, other streams) race on the array.
#include <string.h>

#include <algorithm>
#include <mutex>

#include "fd_runtime.h"

namespace fd {
fd_status make_map(CUtensorMap* m, const float* base, int Nx, int Ny, int Nz, int pitch, int bx,
                   int by);
void fd_weights(int R, double* c);
double cfl_limit(const double* c, int R);
}  // namespace fd

using namespace fd;

static __device__ __align__(256) unsigned char fd_noalloc_scratch[FD_NOALLOC_MAX_BYTES];

namespace {

std::mutex g_mu;
void* g_addr[64] = {};  // device address of the array, per device ordinal

size_t round256(size_t b) { return (std::max<size_t>(b, 16) + 255) / 256 * 256; }

}  // namespace

extern "C" fd_status fd_forward_noalloc(const fd_grid_desc* d, const float* model, int32_t kind,
                                        const fd_points* src, const float* wavelet,
                                        const fd_points* rec, float* rec_out) {
  clear_error();
  if (!d || !model) return fail(FD_ERR_ARG, "null argument");
  if (d->device < 0 || d->device >= 64) return fail(FD_ERR_ARG, "bad device ordinal");
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) return fail(FD_ERR_ARG, "grid sizes must be positive");
  if (!(d->h > 0.0) || !(d->dt > 0.0)) return fail(FD_ERR_ARG, "h and dt must be positive");
  if (d->space_order < 2 || d->space_order > 16 || (d->space_order & 1))
    return fail(FD_ERR_ARG, "space_order must be even, 2..16");
  if (d->nbl < 0 || d->nt < 0) return fail(FD_ERR_ARG, "nbl and nt must be >= 0");
  const int nsrc = src ? src->n : 0, nrec = rec ? rec->n : 0;
  if ((nsrc && (!src->xyz || !wavelet)) || (nrec && (!rec->xyz || !rec_out)))
    return fail(FD_ERR_ARG, "points given without their data array");
  cudaError_t e = cudaSetDevice(d->device);
  if (e) return cuda_fail(e, "cudaSetDevice");
  // inputs and outputs must already be on the device: there is no room to
  // stage host arrays without allocating
  if (!is_device_ptr(model) || (nsrc && !is_device_ptr(wavelet)) ||
      (nrec && !is_device_ptr(rec_out)))
    return fail(FD_ERR_ARG, "fd_forward_noalloc takes device arrays only");

  std::lock_guard<std::mutex> lock(g_mu);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(static_cast<cudaStream_t>(d->stream), &cap);
  if (e) return cuda_fail(e, "stream capture query");
  if (cap == cudaStreamCaptureStatusNone || !g_addr[d->device]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, fd_noalloc_scratch);
    if (e) return cuda_fail(e, "scratch symbol address");
    g_addr[d->device] = p;
  }
  unsigned char* base = static_cast<unsigned char*>(g_addr[d->device]);

  // a grid object on the stack whose buffers all point into the array
  fd_grid_s g;
  g.d = *d;
  g.R = d->space_order / 2;
  g.Nx = d->nx + 2 * d->nbl;
  g.Ny = d->ny + 2 * d->nbl;
  g.Nz = d->nz + 2 * d->nbl;
  if (g.Ny > 65535 || g.Nz > 65535) return fail(FD_ERR_ARG, "padded grid too large");
  g.pitch = (g.Nx + 31) / 32 * 32;
  g.ncell = size_t(g.pitch) * g.Ny * g.Nz;
  fd_weights(g.R, g.c);
  g.cfl = cfl_limit(g.c, g.R);
  g.spin_limit = default_spin_limit();
  g.no_graph = true;  // instantiating a graph allocates
  g.stream = static_cast<cudaStream_t>(d->stream);
  set_shape(&g, default_shape(g.R, g.Nx, g.Ny, g.Nz));
  const size_t ntiles = size_t(g.tiles_x) * g.tiles_y;
  const size_t field = round256(g.ncell * 4);
  const size_t sizes[8] = {round256(256),                                  // error words
                           round256((ntiles + 1) * 4),                     // inj_start
                           round256(size_t(std::max(8 * nsrc, 1)) * sizeof(InjEntry)),
                           round256((ntiles + 1) * 4),                     // rec_start
                           round256(size_t(std::max(nrec, 1)) * sizeof(RecEntry)),
                           round256(2 * (sizeof(ShotDesc) + 256)),  // descriptors
                           0, 0};
  size_t need = 3 * field;
  for (size_t s : sizes) need += s;
  if (need > size_t(FD_NOALLOC_MAX_BYTES))
    return fail(FD_ERR_ARG,
                "grid needs %zu bytes of scratch, above the %d-byte limit of fd_forward_noalloc",
                need, FD_NOALLOC_MAX_BYTES);
  size_t off = 0;
  auto take = [&](size_t b) {
    unsigned char* p = base + off;
    off += b;
    return p;
  };
  g.F.u[0] = reinterpret_cast<float*>(take(field));
  g.F.u[1] = reinterpret_cast<float*>(take(field));
  g.A = reinterpret_cast<float*>(take(field));
  g.d_err = reinterpret_cast<int32_t*>(take(sizes[0]));
  DevBuf* bufs[5] = {&g.tab.inj_start, &g.tab.inj, &g.tab.rec_start, &g.tab.recs, &g.desc};
  for (int i = 0; i < 5; ++i) {
    bufs[i]->cap = sizes[i + 1];
    bufs[i]->p = take(sizes[i + 1]);
  }
  fd_status st = build_maps(&g);
  if (!st) {
    e = cudaMemsetAsync(g.d_err, 0, 256, g.stream);
    if (e) st = cuda_fail(e, "error word reset");
  }
  // set_model clears both wavefields; fd_forward clears them again
  if (!st) st = fd_set_model(&g, model, kind);
  if (!st) st = fd_forward(&g, src, wavelet, rec, rec_out, nullptr);
  // the stack grid owns nothing: detach every pointer before it goes away
  for (int i = 0; i < 5; ++i) {
    bufs[i]->p = nullptr;
    bufs[i]->cap = 0;
  }
  return st;
}
