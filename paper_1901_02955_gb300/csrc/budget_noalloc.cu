// budget_noalloc.cu -- domain budget without any allocation by the library.
//
// snap_budget_compute needs a context, whose creation allocates device memory for the state
// copies and for the per-block partial sums of the reduction. Some callers cannot allocate:
// code that runs where cudaMalloc is forbidden or unavailable (inside a host callback or a
// tightly memory-budgeted serving process with a fixed pool that must not grow, or a
// framework that owns every byte of device memory and hands out only pre-sized tensors).
// For them this unit offers snap_budget_noalloc: the same two-pass deterministic FP64
// reduction, with its partial sums kept in a fixed file-scope device array instead of
// memory the library allocates. The caller passes the state and the output buffer.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/snap.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1024;                    // partial rows
constexpr int kMaxOut = SNAP_MAX_FIELDS + 1;        // field totals + energy with potential
// 1024 x 25 doubles = 200 KiB, held by every device that loads this library until exit.
static __device__ __align__(256) double g_budget_scratch[kMaxBlocks * kMaxOut];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Per-block partial sums in a fixed order (first pass). The state is in the caller's layout:
// nfields planes of ncell values, the first nmass of them densities, the last the total
// energy rho e; level k of cell c is c / plane.
template <class R>
__global__ void __launch_bounds__(kThreads)
    budget_static_kernel(const R *Y, int nfields, int nmass, long long ncell, long long plane,
                         double dz, double grav, double vol, double *partials) {
  __shared__ double red[kMaxOut][kThreads / 32];
  const int no = nfields + 1;
  double s[kMaxOut];
#pragma unroll
  for (int o = 0; o < kMaxOut; ++o) s[o] = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const double z = (double(c / plane) + 0.5) * dz;
    double rho = 0.0;
#pragma unroll
    for (int v = 0; v < kMaxOut - 1; ++v) {
      if (v < nfields) {
        const double y = double(Y[v * ncell + c]);
        s[v] += y;
        if (v < nmass) rho += y;
      }
    }
    s[kMaxOut - 1] += double(Y[(long long)(nfields - 1) * ncell + c]) + rho * grav * z;
  }
#pragma unroll
  for (int o = 0; o < kMaxOut; ++o) {
    double v = s[o];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[o][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < no; o += blockDim.x) {
    const int src = o < nfields ? o : kMaxOut - 1;
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[src][w];
    partials[(long long)blockIdx.x * no + o] = t * vol;
  }
}

// Second pass: sum the partial rows in block order (deterministic).
__global__ void budget_static_finish(const double *partials, int nblocks, int no, double *out) {
  for (int o = threadIdx.x; o < no; o += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partials[(long long)b * no + o];
    out[o] = t;
  }
}

// Device address of the scratch array for the current device. Outside stream capture it is
// looked up on every call: the address belongs to the module loaded into the device's current
// context, and a context that was destroyed and created again (cudaDeviceReset, or the primary
// context released by its last user) loads the module anew, possibly elsewhere. During capture
// no lookup is made (it may have to load the module, which capture forbids); the address of
// the last call outside capture on this device is used, and a capture with no such call fails.
cudaError_t scratch_for_current_device(cudaStream_t s, double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (cap == cudaStreamCaptureStatusNone) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_budget_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double *>(p);
  } else if (!g_scratch_ptr[dev]) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int snap_budget_noalloc(const void *Y, int dtype, int nx, int ny, int nz,
                                   int nfields, int n_mass_fields, double dx, double dy,
                                   double dz, double grav, double *out, void *stream) {
  if (!Y || !out || nx < 1 || ny < 1 || nz < 1) return SNAP_EINVAL;
  if (dtype != SNAP_F64 && dtype != SNAP_F32) return SNAP_EINVAL;
  if (nfields < 2 || nfields > SNAP_MAX_FIELDS) return SNAP_EINVAL;  // scratch row limit
  if (n_mass_fields < 1 || n_mass_fields >= nfields) return SNAP_EINVAL;
  if (!(dx > 0) || !(dz > 0) || (ny > 1 && !(dy > 0))) return SNAP_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // an error left pending by earlier work of the caller is reported, not consumed: it stays
  // for its owner to read, and this call launches nothing
  if (cudaPeekAtLastError() != cudaSuccess) return SNAP_ECUDA;
  double *partials = nullptr;
  if (scratch_for_current_device(s, &partials) != cudaSuccess) return SNAP_ECUDA;
  const long long ncell = (long long)nx * ny * nz;
  const long long plane = (long long)nx * ny;
  long long nb = (ncell + kThreads - 1) / kThreads;
  const int nblocks = int(nb < 1 ? 1 : (nb > kMaxBlocks ? kMaxBlocks : nb));
  const double vol = dx * (ny > 1 ? dy : 1.0) * dz;
  if (dtype == SNAP_F32)
    budget_static_kernel<float><<<nblocks, kThreads, 0, s>>>(
        (const float *)Y, nfields, n_mass_fields, ncell, plane, dz, grav, vol, partials);
  else
    budget_static_kernel<double><<<nblocks, kThreads, 0, s>>>(
        (const double *)Y, nfields, n_mass_fields, ncell, plane, dz, grav, vol, partials);
  budget_static_finish<<<1, 32, 0, s>>>(partials, nblocks, nfields + 1, out);
  // no error was pending before the launches, so one read here is this call's own
  return cudaGetLastError() == cudaSuccess ? SNAP_OK : SNAP_ECUDA;
}
