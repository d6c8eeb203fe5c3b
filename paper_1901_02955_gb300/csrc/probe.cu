// probe.cu -- arithmetic-throughput probe of the device (a measurement aid, not part of the
// scheme): register-resident chains of fused multiply-adds, eight independent chains per
// thread, a grid of eight 256-thread blocks per SM. The stage kernels are bound by arithmetic
// issue, so their roofline is quoted against the FP32 fused multiply-add rate; this measures
// that rate (and the FP64 one) on the device and clocks at hand, next to the nominal figure.
// It also holds the arithmetic self-checks: the stage kernels' FP64 reciprocal and WENO5
// reconstruction run on caller-given arguments, for tests against IEEE division and the
// textbook formula.
#include <cuda_runtime.h>

#include "../../include/snap.h"
#include "snap_stage.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

template <class R>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(R *out, int iters, R b, R c) {
  R a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = R(threadIdx.x + k) * R(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  R s = R(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == R(-12345.0)) out[blockIdx.x] = s;  // keeps the chains live; never true
}

template <class R>
int probe(double *tflops, cudaStream_t s) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SNAP_ECUDA;
  const int blocks = nsm * 8;
  const int iters = sizeof(R) == 4 ? 4096 : 256;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return SNAP_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SNAP_ECUDA;
  }
  const R b = R(0.9999999), c = R(1e-7);
  float best = 1e30f;
  int rc = SNAP_OK;
  for (int rep = 0; rep < 6 && rc == SNAP_OK; ++rep) {  // the first launches warm up
    cudaEventRecord(e0, s);
    fma_probe_kernel<R><<<blocks, kThreads, 0, s>>>(nullptr, iters, b, c);
    cudaEventRecord(e1, s);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = SNAP_ECUDA;
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep >= 2 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SNAP_OK) return rc;
  const double flops = 2.0 * kChains * 4.0 * iters * double(blocks) * kThreads;
  *tflops = flops / (double(best) * 1e-3) / 1e12;
  return SNAP_OK;
}

__global__ void rcp64_kernel(const double *x, double *y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    y[2 * i] = snap::Ar<double>::rcp(x[i]);
    y[2 * i + 1] = 1.0 / x[i];
  }
}

template <class R>
__global__ void weno_kernel(const R *win, R *out, long long n, R eps) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const R *q = win + 5 * i;
    R qm, qp;
    snap::weno5_pair<R>(q[0], q[1], q[2], q[3], q[4], eps, qm, qp);
    out[2 * i] = qm;
    out[2 * i + 1] = qp;
  }
}

// windows 2p and 2p + 1 as the two lanes of the packed form
__global__ void weno_packed_kernel(const float *win, float *out, long long npair, float eps) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npair;
       p += (long long)gridDim.x * blockDim.x) {
    const float *q = win + 10 * p, *r = q + 5;
    float2 qm, qp;
    snap::weno5_pair2(make_float2(q[0], r[0]), make_float2(q[1], r[1]), make_float2(q[2], r[2]),
                      make_float2(q[3], r[3]), make_float2(q[4], r[4]), eps, qm, qp);
    out[4 * p] = qm.x;
    out[4 * p + 1] = qp.x;
    out[4 * p + 2] = qm.y;
    out[4 * p + 3] = qp.y;
  }
}

int grid_for(long long n) {
  const long long g = (n + kThreads - 1) / kThreads;
  return int(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

}  // namespace

extern "C" int snap_check_rcp64(const double *x, double *y, long long n, void *stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return SNAP_EINVAL;
  if (n == 0) return SNAP_OK;
  rcp64_kernel<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(x, y, n);
  return cudaGetLastError() == cudaSuccess ? SNAP_OK : SNAP_ECUDA;
}

extern "C" int snap_check_weno(int dtype, int packed, const void *win, void *out, long long n,
                               double eps, void *stream) {
  if (n < 0 || (n > 0 && (!win || !out)) || (dtype != SNAP_F32 && dtype != SNAP_F64) ||
      (packed && (dtype != SNAP_F32 || n % 2)))
    return SNAP_EINVAL;
  if (n == 0) return SNAP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (packed)
    weno_packed_kernel<<<grid_for(n / 2), kThreads, 0, s>>>((const float *)win, (float *)out,
                                                            n / 2, float(eps));
  else if (dtype == SNAP_F32)
    weno_kernel<float><<<grid_for(n), kThreads, 0, s>>>((const float *)win, (float *)out, n,
                                                        float(eps));
  else
    weno_kernel<double><<<grid_for(n), kThreads, 0, s>>>((const double *)win, (double *)out, n,
                                                         eps);
  return cudaGetLastError() == cudaSuccess ? SNAP_OK : SNAP_ECUDA;
}

extern "C" int snap_probe_fma(int dtype, double *tflops, void *stream) {
  if (!tflops || (dtype != SNAP_F32 && dtype != SNAP_F64)) return SNAP_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  return dtype == SNAP_F32 ? probe<float>(tflops, s) : probe<double>(tflops, s);
}
