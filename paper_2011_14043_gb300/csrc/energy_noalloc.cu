// Field energy without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need
// the energy: code running inside a framework whose caching allocator has
// reserved the device's memory (a cudaMalloc there can fail or force the
// framework to release its pool), or a stepping loop where the implicit
// device-wide synchronisation of cudaMalloc/cudaFree is not acceptable.
// fdtd_energy_noalloc serves them: the caller passes the six field arrays
// and a device output word; the per-plane partial sums live in the fixed
// file-scope array below, which every GPU that loads the library holds until
// the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Each call overwrites exactly the partials it then reads, so no
// clearing is needed; two calls whose kernels overlap on the GPU (different
// streams, or different host threads) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/fdtd.h"

namespace {

constexpr int kMaxPlanes = 4097;  // planes per component: nz + 1 <= 4097
constexpr int kMaxDevices = 64;

// 6 components x kMaxPlanes per-plane sums of weight * value^2 (192 KiB).
static __device__ __align__(256) double g_energy_scratch[6 * kMaxPlanes];

constexpr double kC0 = 299792458.0;
constexpr double kMu0 = 1.25663706212e-6;

std::mutex g_mu;
double* g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of g_energy_scratch on the current device.  The host-side
// name is only a stand-in, so the address is looked up once per device with
// that device current, then cached.  The cache assumes the device's context
// lives as long as the process: after cudaDeviceReset (or a reset of the
// primary context) the module is loaded again and the cached address may no
// longer be valid, so this entry point must not be used after such a reset.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FDTD_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_energy_scratch);
    if (e != cudaSuccess || !p) {
      fprintf(stderr, "fdtd_energy_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
      return FDTD_ERR_CUDA;
    }
    g_scratch_dev[dev] = (double*)p;
  }
  *out = g_scratch_dev[dev];
  return FDTD_OK;
}

template <typename T>
struct Fields6 {
  const T* f[6];
  int sx[6], sy[6], sz[6];
  double w[6];  // eps or mu of each component
};

// Block (k, c) sums w_c * v^2 over plane k of component c (compact layout)
// into partial[c][k].  Fixed thread-to-element assignment and a fixed tree:
// the result is deterministic.
template <typename T>
__global__ void plane_sumsq_kernel(const Fields6<T> F, double* partial) {
  const int k = blockIdx.x;
  const int c = blockIdx.y;
  if (k >= F.sz[c]) return;
  const long long n = (long long)F.sx[c] * F.sy[c];
  const T* p = F.f[c] + (long long)k * n;
  double acc = 0.0;
  for (long long g = threadIdx.x; g < n; g += blockDim.x) {
    const double v = (double)p[g];
    acc += v * v;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) partial[c * kMaxPlanes + k] = F.w[c] * v;
  }
}

// One block: sum the partials written by plane_sumsq_kernel, in a fixed order.
template <typename T>
__global__ void plane_total_kernel(const Fields6<T> F, const double* partial, double scale, double* out) {
  double acc = 0.0;
  for (int c = 0; c < 6; ++c)
    for (int k = threadIdx.x; k < F.sz[c]; k += blockDim.x) acc += partial[c * kMaxPlanes + k];
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) out[0] = scale * v;
  }
}

template <typename T>
int run(int nx, int ny, int nz, double dv, double eps_r, double mu_r, const void* const* fields,
        double* out_device, cudaStream_t stream) {
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  Fields6<T> F;
  const int ext[6][3] = {{nx, ny + 1, nz + 1}, {nx + 1, ny, nz + 1}, {nx + 1, ny + 1, nz},
                         {nx + 1, ny, nz},     {nx, ny + 1, nz},     {nx, ny, nz + 1}};
  const double eps0 = 1.0 / (kMu0 * kC0 * kC0);
  for (int c = 0; c < 6; ++c) {
    F.f[c] = (const T*)fields[c];
    F.sx[c] = ext[c][0];
    F.sy[c] = ext[c][1];
    F.sz[c] = ext[c][2];
    F.w[c] = c < 3 ? eps0 * eps_r : kMu0 * mu_r;
  }
  // An error left pending by someone else is reported, not taken over: it
  // stays pending for its owner, and nothing is launched.
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess) {
    fprintf(stderr, "fdtd_energy_noalloc: a CUDA error is already pending (%s); nothing launched\n",
            cudaGetErrorString(pending));
    return FDTD_ERR_CUDA;
  }
  plane_sumsq_kernel<T><<<dim3((unsigned)(nz + 1), 6), 256, 0, stream>>>(F, scratch);
  if (cudaGetLastError() != cudaSuccess) return FDTD_ERR_CUDA;
  plane_total_kernel<T><<<1, 256, 0, stream>>>(F, scratch, 0.5 * dv, out_device);
  return cudaGetLastError() == cudaSuccess ? FDTD_OK : FDTD_ERR_CUDA;
}

}  // namespace

extern "C" int fdtd_energy_noalloc(int nx, int ny, int nz, double dx, double dy, double dz, double eps_r,
                                   double mu_r, int precision, const void* const* fields, double* out_device,
                                   void* stream) {
  if (!fields || !out_device) return FDTD_ERR_INVALID_ARG;
  for (int c = 0; c < 6; ++c)
    if (!fields[c]) return FDTD_ERR_INVALID_ARG;
  if (nx < 1 || ny < 1 || nz < 1) return FDTD_ERR_INVALID_ARG;
  if (nz + 1 > kMaxPlanes) {
    fprintf(stderr, "fdtd_energy_noalloc: nz = %d exceeds the fixed scratch of %d planes (nz <= %d)\n", nz,
            kMaxPlanes, kMaxPlanes - 1);
    return FDTD_ERR_INVALID_ARG;
  }
  if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !std::isfinite(dx * dy * dz)) return FDTD_ERR_INVALID_ARG;
  if (!(eps_r > 0) || !(mu_r > 0) || !std::isfinite(eps_r) || !std::isfinite(mu_r)) return FDTD_ERR_INVALID_ARG;
  const double dv = dx * dy * dz;
  if (precision == FDTD_F64)
    return run<double>(nx, ny, nz, dv, eps_r, mu_r, fields, out_device, (cudaStream_t)stream);
  if (precision == FDTD_F32)
    return run<float>(nx, ny, nz, dv, eps_r, mu_r, fields, out_device, (cudaStream_t)stream);
  return FDTD_ERR_INVALID_ARG;
}
