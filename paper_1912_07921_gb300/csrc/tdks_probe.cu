// Arithmetic-rate probe: the FP64 (and FP32) fused multiply-add throughput of the current
// GPU, measured with the library's own kernel.  The complex128 path spends most of its time
// in FP64 adds and FMAs (GB300 runs FP64 at a small fraction of its FP32 rate), so its
// roofline is min(HBM bandwidth, FP64 instruction rate); this probe measures the second.
//
// Each thread runs 8 independent FMA chains x <- x a + b (a just below 1, so nothing
// overflows or becomes subnormal) for `iters` iterations; enough warps per SM keep the
// pipe busy despite each chain's latency.  The sums are written out so nothing is removed.
#include <cuda_runtime.h>

#include <string>

#include "tdks_system.h"

using namespace tdks_host;

namespace {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) fma_probe_kernel(T *out, int iters, T a, T b) {
  T x[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; c++) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; c++) s += x[c];
  out[blockIdx.x * (long)blockDim.x + threadIdx.x] = s;
}

template <typename T>
int probe(int blocks, int iters, double *fma_per_s) {
  T *buf = nullptr;
  CU(cudaMalloc((void **)&buf, sizeof(T) * (size_t)blocks * PROBE_THREADS));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = TDKS_OK;
  float ms = 0.f;
  do {
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      rc = fail(TDKS_EDEVICE, "cudaEventCreate failed");
      break;
    }
    const T a = (T)0.9999999, b = (T)1e-7;
    fma_probe_kernel<T><<<blocks, PROBE_THREADS>>>(buf, iters / 8, a, b);  // warm-up
    cudaEventRecord(e0);
    fma_probe_kernel<T><<<blocks, PROBE_THREADS>>>(buf, iters, a, b);
    cudaEventRecord(e1);
    const cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      rc = fail(TDKS_EDEVICE, std::string("FMA probe: ") + cudaGetErrorString(e));
      break;
    }
    cudaEventElapsedTime(&ms, e0, e1);
  } while (false);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (rc) return rc;
  *fma_per_s = (double)blocks * PROBE_THREADS * (double)iters * PROBE_CHAINS / (ms * 1e-3);
  return TDKS_OK;
}

}  // namespace

extern "C" int tdks_fma_rate(int prec, double *fma_per_s) {
  if (!fma_per_s) return fail(TDKS_EINVAL, "fma_per_s is NULL");
  if (prec != TDKS_C128 && prec != TDKS_C64) return fail(TDKS_EINVAL, "bad precision");
  int dev = 0, sms = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = 8 * sms;  // 64 warps per SM
  return prec == TDKS_C128 ? probe<double>(blocks, 2048, fma_per_s) : probe<float>(blocks, 65536, fma_per_s);
}
