// Pipe-rate probes: the FP64 and FP32 fused multiply-add rates of the current
// GPU, measured by kernels that do nothing else.  The benchmark divides its
// kernels' algorithmic flop rates by these (its roofline is the FP64 pipe for
// the FP64 path and the FP32 pipe for the mixed form's FP32 stages).
//
// Each thread runs ACC independent multiply-add chains (enough to cover the
// pipes' latency with several warps per scheduler), INNER multiply-adds per
// chain per loop trip; one block per SM slot, several blocks per SM.  The
// chains' values stay bounded (x <- x * a + b with |a| < 1), and the result
// is stored only when a data-dependent test that never holds passes, so the
// compiler keeps every operation.
#include <cstdio>
#include <string>

#include "hydro_internal.cuh"

namespace {

constexpr int ACC = 8;
constexpr int INNER = 16;
constexpr int PROBE_THREADS = 256;

template <typename R>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(int trips, R a, R b, R* __restrict__ sink) {
  // each chain has its own multiplier: with one multiplier register shared by
  // every chain the FP64 rate measured 8 % lower (register-operand reuse)
  R x[ACC], m[ACC];
#pragma unroll
  for (int k = 0; k < ACC; k++) {
    x[k] = R(threadIdx.x + k) * R(1e-3);
    m[k] = a - R(k) * R(1e-5);
  }
  for (int t = 0; t < trips; t++) {
#pragma unroll
    for (int i = 0; i < INNER; i++) {
#pragma unroll
      for (int k = 0; k < ACC; k++) x[k] = fma(x[k], m[k], b);
    }
  }
  R s = R(0);
#pragma unroll
  for (int k = 0; k < ACC; k++) s += x[k];
  if (s == R(-12345.0) && sink) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int fail(int code, const std::string& msg) {
  hydro::set_last_error(msg);
  return code;
}

template <typename R>
int time_probe(cudaStream_t s, int blocks, int trips, double* flops_per_s) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return fail(HYDRO_ERR_CUDA, std::string("hydro_measure_peaks: ") + cudaGetErrorString(e));
  // warm-up (clocks up), then the timed launch
  k_fma_probe<R><<<blocks, PROBE_THREADS, 0, s>>>(trips / 4 + 1, R(0.999), R(1e-4), nullptr);
  e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    k_fma_probe<R><<<blocks, PROBE_THREADS, 0, s>>>(trips, R(0.999), R(1e-4), nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(HYDRO_ERR_CUDA, std::string("hydro_measure_peaks: ") + cudaGetErrorString(e));
  const double fl = 2.0 * ACC * INNER * (double)trips * PROBE_THREADS * blocks;
  *flops_per_s = fl / (ms * 1e-3);
  return HYDRO_OK;
}

}  // namespace

extern "C" int hydro_measure_peaks(double* fp64_flops_per_s, double* fp32_flops_per_s, int* sms, void* stream) {
  if (!fp64_flops_per_s || !fp32_flops_per_s || !sms) return fail(HYDRO_ERR_INVALID, "null argument");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  int nsm = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(HYDRO_ERR_CUDA, std::string("hydro_measure_peaks: ") + cudaGetErrorString(e));
  *sms = nsm;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // 8 blocks of 256 threads per SM (64 warps: the SM's limit); trip counts
  // sized for roughly 100-200 ms per launch at the pipes' nominal rates
  const int blocks = 8 * nsm;
  int rc = time_probe<double>(s, blocks, 4096, fp64_flops_per_s);
  if (rc) return rc;
  return time_probe<float>(s, blocks, 131072, fp32_flops_per_s);
}
