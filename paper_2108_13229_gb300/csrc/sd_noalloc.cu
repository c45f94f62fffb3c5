// sd_noalloc.cu -- y = A x for the coupled operator without any allocation.
//
// Some callers cannot allocate device memory at the moment they need the
// operator: code that runs inside a framework owning a fixed memory pool
// (allocation would bypass or exhaust it), real-time loops where a
// cudaMalloc would stall every stream on the device, or library code that
// is not allowed to create handles.  sd_apply needs a handle, and a handle
// allocates all its buffers in sd_create.  sd_apply_noalloc does the same
// work -- permeability packing, TPFA / interface coefficients, padded input,
// the operator kernel, unpacking -- with every intermediate array carved out
// of one file-scope device array of fixed size, so it calls no cudaMalloc,
// cudaFree or allocating library routine.
#include "../../include/sd.h"
#include "sd_internal.cuh"

#include <cmath>
#include <mutex>

using namespace sdk;

namespace {

// Working storage of sd_apply_noalloc, in doubles: enough for
// n = SD_NOALLOC_MAX_N (6 MiB).  Every GPU that loads this library holds it
// until the process exits.
const long long kScratchDoubles = 786432;
static __device__ __align__(256) double sd_noalloc_scratch[kScratchDoubles];

const int kMaxDevices = 64;
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {nullptr};

long long align32(long long v) { return (v + 31) / 32 * 32; }

// Device address of the scratch array on the current device.  The array's
// name in host code is only a stand-in for the symbol, so the address is
// looked up once per device (with that device current) and cached.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SD_E_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, sd_noalloc_scratch);
    if (e != cudaSuccess || !p) return SD_E_CUDA;
    g_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_ptr[dev];
  return SD_OK;
}

// True for device memory of device `dev` (or managed memory).  The kernels
// run on the current device and dereference the pointers directly, so memory
// of another GPU is refused rather than read across devices.  A failing
// attribute query (no usable device) is the only error it clears; an error
// pending from the caller's own work does not make the query fail, so it
// stays pending for the check that follows.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" int sd_apply_noalloc(const sd_grid* grid, double mu, const double* K, double alpha_bj, double dt,
                                const double* x, double* y, void* stream) {
  if (!grid || grid->nx != grid->ny || grid->nx < 2) return SD_E_INVAL;
  const int n = grid->nx;
  if (n > SD_NOALLOC_MAX_N) return SD_E_INVAL;
  if (!(mu > 0) || !(alpha_bj > 0) || !(dt > 0) || !std::isfinite(mu) || !std::isfinite(alpha_bj) ||
      !std::isfinite(dt))
    return SD_E_INVAL;
  int dev = 0;
  if (!K || !x || !y || cudaGetDevice(&dev) != cudaSuccess || !on_device(K, dev) || !on_device(x, dev) ||
      !on_device(y, dev))
    return SD_E_INVAL;
  // an error left pending by earlier work is not this call's to report or to
  // clear: refuse to run on top of it
  if (cudaPeekAtLastError() != cudaSuccess) return SD_E_CUDA;
  const Geom g = make_geom(n);
  // carve the scratch array: padded K, coefficients, padded x and y
  const long long oK = 0;
  const long long ow = oK + align32((long long)n * g.P);
  const long long org = ow + align32(n + 1);
  const long long oTx = org + align32(n + 1);
  const long long oTy = oTx + align32((long long)n * g.P);
  const long long ox = oTy + align32((long long)(n + 1) * g.P);
  const long long oy = ox + align32(g.len);
  const long long end = oy + align32(g.len);
  if (end > kScratchDoubles) return SD_E_INVAL;
  double* base = nullptr;
  const int rc = scratch_address(&base);
  if (rc != SD_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // every scratch entry that the operator reads is written first in this
  // call, so the previous call's contents never leak into the result
  // nothing was pending at entry, so an error seen after a launch is that
  // launch's own
  launch_pack_K(K, n, base + oK, g.P, s);
  launch_setup_coef<double>(base + oK, n, n, g.P, mu, alpha_bj, 0, 0, 0, n, n, 0, base + ow, base + org, base + oTx,
                            base + oTy, s);
  launch_pack(g, x, base + ox, s);
  if (cudaGetLastError() != cudaSuccess) return SD_E_CUDA;
  Coef<double> c;
  c.n = n;
  c.nx = n;  // the square geometry
  c.iw = 0;
  c.cx = n;
  c.P = g.P;
  c.lat = 0;  // Dirichlet free-flow sides (the SD_BC_MMS operator)
  c.h = g.h;
  c.mu = mu;
  c.cm = g.h * g.h / dt;
  c.w = base + ow;
  c.rg = base + org;
  c.Tx = base + oTx;
  c.Ty = base + oTy;
  finish_coef(c);
  launch_apply_full(c, base + ox, nullptr, base + oy, s);
  launch_unpack(g, base + oy, y, s);
  return cudaGetLastError() == cudaSuccess ? SD_OK : SD_E_CUDA;
}
