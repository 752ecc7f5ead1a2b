// Measurement of the binary64 fused multiply-add rate of this GPU
// (pcg_fp64_fma_rate). The binary64 PCG iteration is bound by the FP64 pipe
// on this part rather than by HBM, so its roofline is taken against this
// measured rate, not against a figure derived from clocks and unit counts.
//
// Every thread runs NCH independent FMA chains a <- a * m + c (m < 1, c > 0:
// each chain converges to c / (1 - m), no overflow, no subnormals); NCH chains
// per thread and many resident warps per SM hide the FMA latency, so the pipe
// issue rate is what is measured. The chains' sum is stored only if it equals a
// value it cannot reach, which keeps the arithmetic live without a store per
// thread.
#include <cuda_runtime.h>

#include <string>

#include "handle.cuh"

using namespace pcg;

namespace {

constexpr int NCH = 8;        // independent chains per thread
constexpr int UNROLL = 16;    // FMA steps per chain per loop trip
constexpr int THREADS = 256;

__global__ void __launch_bounds__(THREADS) k_dfma_rate(double *sink, int trips, double m, double c) {
  double a[NCH];
#pragma unroll
  for (int k = 0; k < NCH; ++k) a[k] = 1e-3 * (double)(threadIdx.x + k);
  for (int t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u)
#pragma unroll
      for (int k = 0; k < NCH; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < NCH; ++k) s += a[k];
  if (s == -1.0) sink[blockIdx.x] = s;   // never true: the chains stay positive
}

}  // namespace

extern "C" int pcg_fp64_fma_rate(int32_t launches, double *tflops, double *ms_per_launch, void *cuda_stream) {
  if (!tflops || launches <= 0) { set_error("invalid arguments"); return PCG_EINVAL; }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0, per_sm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma_rate, THREADS, 0));
  if (per_sm < 1) { set_error("measurement kernel does not fit on an SM"); return PCG_ECUDA; }
  const int blocks = nsm * per_sm;            // one full wave of resident blocks
  const int trips = 256;                      // about 15 ms per launch at 0.6e12 FMA/s
  double *sink = nullptr;
  CK(cudaMalloc(&sink, sizeof(double) * blocks));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = PCG_OK;
  auto fail = [&](cudaError_t e) {
    set_error(std::string("FP64 rate measurement: ") + cudaGetErrorString(e));
    rc = PCG_ECUDA;
  };
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_dfma_rate<<<blocks, THREADS, 0, s>>>(sink, trips, 0.999, 1e-3);   // warm-up
    note_launches(1);
    e = cudaEventRecord(e0, s);
  }
  for (int l = 0; e == cudaSuccess && l < launches; ++l) {
    k_dfma_rate<<<blocks, THREADS, 0, s>>>(sink, trips, 0.999, 1e-3);
    note_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e != cudaSuccess) fail(e);
  if (rc == PCG_OK) {
    const double fma_per_launch = (double)blocks * THREADS * trips * UNROLL * NCH;
    const double sec = ms * 1e-3 / launches;
    *tflops = 2.0 * fma_per_launch / sec / 1e12;
    if (ms_per_launch) *ms_per_launch = ms / launches;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return rc;
}
