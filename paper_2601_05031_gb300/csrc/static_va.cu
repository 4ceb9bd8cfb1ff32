// Volume and area of a phase field with no device allocation.
//
// Some callers of this library cannot allocate device memory at all: code
// that runs inside a CUDA stream capture (graph capture rejects cudaMalloc),
// code behind a device-memory pool whose owner forbids outside allocations,
// or a host process that only holds a pre-mapped buffer.  This entry point
// serves them: its scratch (one pair of FP64 partial sums per (y, z) row) is
// a file-scope __device__ array, sized for at most kStaticMaxRows rows, that
// every device which loads the library keeps until the process exits.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress while that device is current; later calls reuse it.
// Every call shares the array and leaves its partial sums in it.  Each call
// overwrites all the rows it uses before reading them, so nothing needs
// clearing, but two calls whose kernels overlap on a GPU (different streams)
// race on the array.
#include <mutex>

#include "internal.h"

namespace vsv {

constexpr int kStaticMaxRows = 65536;     // ny * nz rows; 1 MiB of scratch
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) double g_static_rows[2 * kStaticMaxRows];

namespace {

__device__ __forceinline__ int st_mirror(int j, int n) {
  return j < 0 ? -1 - j : (j >= n ? 2 * n - 1 - j : j);
}
__device__ __forceinline__ int st_wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// One block per (y, z) row: FP64 sums over x of phi and of the area density
// 3/(2 sqrt2) [eps/2 |grad phi|^2 + (phi^2 - 1)^2 / (4 eps)] (central
// differences, periodic x, mirror y, mirror or periodic z).
__global__ void k_static_rows(const double* __restrict__ phi, int nx, int ny, int nz, int zper,
                              double inv_h, double eps, double* rows) {
  const int row = blockIdx.x;
  const int j = row % ny, k = row / ny;
  const double hih = 0.5 * inv_h, he = 0.5 * eps, q = 0.25 / eps;
  const double ca = 3.0 / (2.0 * 1.4142135623730951);
  auto at = [&](int i, int jj, int kk) {
    i = st_wrap(i, nx);
    jj = st_mirror(jj, ny);
    kk = zper ? st_wrap(kk, nz) : st_mirror(kk, nz);
    return phi[((long long)kk * ny + jj) * nx + i];
  };
  double sp = 0.0, sa = 0.0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const double f = at(i, j, k);
    const double gx = (at(i + 1, j, k) - at(i - 1, j, k)) * hih;
    const double gy = (at(i, j + 1, k) - at(i, j - 1, k)) * hih;
    const double gz = (at(i, j, k + 1) - at(i, j, k - 1)) * hih;
    const double w = f * f - 1.0;
    sp += f;
    sa += ca * (he * (gx * gx + gy * gy + gz * gz) + w * w * q);
  }
  sp = block_sum(sp);
  sa = block_sum(sa);
  if (threadIdx.x == 0) {
    rows[2 * row] = sp;
    rows[2 * row + 1] = sa;
  }
}

// Fixed-order total of the row sums: out[0] = V = h^3/2 (N - sum phi),
// out[1] = A = h^3 sum(density).
__global__ void k_static_total(const double* rows, int nrows, long long ncells, double h3,
                               double* out) {
  double sp = 0.0, sa = 0.0;
  for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
    sp += rows[2 * r];
    sa += rows[2 * r + 1];
  }
  sp = block_sum(sp);
  sa = block_sum(sa);
  if (threadIdx.x == 0) {
    out[0] = 0.5 * h3 * ((double)ncells - sp);
    out[1] = h3 * sa;
  }
}

std::mutex g_static_mutex;
double* g_static_ptr[kStaticMaxDevices] = {};

// True if p is device (or managed) memory of device dev: a pointer into
// another GPU's memory, or host memory, would make the kernels read through
// an address this device may not map.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();   // the query's own error (an unknown pointer), not a launch's
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

}  // namespace vsv

extern "C" vsv_status vsv_volume_area_static(const double* phi, int nx, int ny, int nz, double h,
                                              double eps, int z_periodic, double* out,
                                              void* cuda_stream) {
  using namespace vsv;
  if (!phi || !out || nx < 1 || ny < 1 || nz < 1 || !(h > 0) || !(eps > 0)) return VSV_EINVAL;
  if ((long long)ny * nz > kStaticMaxRows) return VSV_EINVAL;   // beyond the static scratch
  // an error left pending by earlier work is reported, not cleared: it
  // belongs to its owner
  if (cudaPeekAtLastError() != cudaSuccess) return VSV_ECUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return VSV_ECUDA;
  if (!on_device(phi, dev) || !on_device(out, dev)) return VSV_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (s) {
    int sdev = -1;
    if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) return VSV_ECUDA;
    if (sdev != dev) return VSV_EINVAL;
  }
  double* rows = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[dev]) {
      void* p = nullptr;
      // host code only ever sees a stand-in for the array: its device address
      // comes from the runtime, per device, with that device current
      if (cudaGetSymbolAddress(&p, g_static_rows) != cudaSuccess || !p) return VSV_ECUDA;
      g_static_ptr[dev] = (double*)p;
    }
    rows = g_static_ptr[dev];
  }
  const int nrows = ny * nz;
  k_static_rows<<<nrows, kBlock, 0, s>>>(phi, nx, ny, nz, z_periodic ? 1 : 0, 1.0 / h, eps, rows);
  if (cudaGetLastError() != cudaSuccess) return VSV_ECUDA;
  k_static_total<<<1, kBlock, 0, s>>>(rows, nrows, (long long)nx * ny * nz, h * h * h, out);
  return cudaGetLastError() == cudaSuccess ? VSV_OK : VSV_ECUDA;
}
