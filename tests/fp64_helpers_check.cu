// Checks the device arithmetic helpers of fp64_fast.cuh on the GPU against
// IEEE operations: the bit-pattern sign tests, comparisons, min/max, exact
// halving and doubling, the |x| > 2|y| test, the integer FP64 -> FP32 rounding (against
// the conversion instruction, where it does not defer to it) and the
// integer-pipe product (against the FP64 multiply) bit for bit, on
// patterns drawn over every
// exponent (subnormals, the range edges, zero and both signs included); the
// Newton-refined reciprocal, reciprocal square root and square root within
// their stated error over normal arguments.  Prints one line per check and
// exits non-zero on any mismatch.  Built and run by test_gpu_fp64_helpers.py.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "fp64_fast.cuh"

using namespace hydro;

enum { BAD_HALF, BAD_CMP, BAD_RCP, BAD_SQRT, BAD_RSQRT, BAD_NARROW, BAD_IMUL, NBAD };

__device__ double ulp_of(double r) { return ldexp(1.0, ilogb(r) - 52); }

__global__ void check_bits(const double* x, const double* y, int n, unsigned long long* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = x[i], c = y[i];
  const double h = half_of<double>(a), r = __dmul_rn(0.5, a);
  if (!(__double_as_longlong(h) == __double_as_longlong(r) || (isnan(h) && isnan(r)))) atomicAdd(&bad[BAD_HALF], 1ull);
  const double w = twice_of<double>(a), v2 = __dmul_rn(2.0, a);
  if (!(__double_as_longlong(w) == __double_as_longlong(v2) || (isnan(w) && isnan(v2)))) atomicAdd(&bad[BAD_HALF], 1ull);
  {  // the integer-pipe product: bitwise the IEEE one wherever it does not
     // defer, and deferring exactly where an operand is subnormal, infinite
     // or NaN (zero excepted) or the product is not normal or zero
    unsigned defer = 0u;
    const double p = imul_rn(a, c, defer), q = __dmul_rn(a, c);
    if (!defer && __double_as_longlong(p) != __double_as_longlong(q)) atomicAdd(&bad[BAD_IMUL], 1ull);
    const auto normal = [](double v) { return fabs(v) >= 0x1p-1022 && isfinite(v); };
    const bool zero_op = (a == 0.0 && isfinite(c)) || (c == 0.0 && isfinite(a));
    const double m = fabs(q);
    // a product rounded up to the smallest normal from below it is deferred too
    const bool fast = zero_op || (normal(a) && normal(c) && (isinf(q) ? false : m >= 0x1p-1022));
    if (fast && defer && !(m < 0x1p-1021)) atomicAdd(&bad[BAD_IMUL], 1ull);
    if (!fast && !defer && !isinf(q)) atomicAdd(&bad[BAD_IMUL], 1ull);
  }
  bool rare;
  const unsigned nb = narrow_bits(a, rare);
  if (!rare && nb != __float_as_uint(__double2float_rn(a))) atomicAdd(&bad[BAD_NARROW], 1ull);
  // what it defers: FP32 subnormal results, |x| >= 2^128, infinities and NaN, and nothing else
  const double m = fabs(a);
  const bool expect_rare = isnan(a) || m >= 0x1p128 || (m >= 0x1p-150 && m < 0x1p-126);
  if (rare != expect_rare) atomicAdd(&bad[BAD_NARROW], 1ull);
  if (!isfinite(a) || !isfinite(c)) return;
  bool e = abs_gt_twice<double>(a, c) != (fabs(a) > __dmul_rn(2.0, fabs(c)));
  e |= is_pos<double>(a) != (a > 0.0);
  e |= is_neg<double>(a) != (a < 0.0);
  e |= same_sign<double>(a, c) != ((a > 0.0 && c > 0.0) || (a < 0.0 && c < 0.0));
  e |= opp_sign<double>(a, c) != ((a > 0.0 && c < 0.0) || (a < 0.0 && c > 0.0));
  if (!(a == 0.0 && c == 0.0)) {  // the bit-pattern order puts -0.0 below +0.0
    e |= dgt<double>(a, c) != (a > c);
    e |= dmin<double>(a, c) != fmin(a, c);
    e |= dmax<double>(a, c) != fmax(a, c);
  }
  if (e) atomicAdd(&bad[BAD_CMP], 1ull);
}

// x > 0 normal: reciprocal and square root within 2 ulp of the correctly
// rounded results; 1/sqrt(x) within 2^-51.5 relative, from the residual
// y^2 x - 1 formed with an exact square.  The largest errors in units of 1e-3
// ulp (resp. of 2^-53) are kept in worst[].
__global__ void check_refined(const double* x, int n, unsigned long long* bad, unsigned long long* worst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = x[i];
  const double rr = __drcp_rn(a), er = fabs(nr_rcp(a) - rr) / ulp_of(rr);
  const double sr = __dsqrt_rn(a), es = fabs(nr_sqrt(a) - sr) / ulp_of(sr);
  const double y = nr_rsqrt(a);
  const double t = y * y, tl = fma(y, y, -t);
  const double res = fma(a, t, -1.0) + a * tl;  // y^2 a - 1
  const double eq = fabs(0.5 * res) * 9007199254740992.0;  // relative error of y in units of 2^-53
  if (!(er <= 2.0)) atomicAdd(&bad[BAD_RCP], 1ull);
  if (!(es <= 2.0)) atomicAdd(&bad[BAD_SQRT], 1ull);
  if (!(eq <= 2.83)) atomicAdd(&bad[BAD_RSQRT], 1ull);
  atomicMax(&worst[0], (unsigned long long)(er * 1000.0));
  atomicMax(&worst[1], (unsigned long long)(es * 1000.0));
  atomicMax(&worst[2], (unsigned long long)(eq * 1000.0));
}

// Throughput of the products (informational; printed, not asserted): chains
// of FP64 multiplies by the instruction and on the integer pipe, FP64
// multiply-add chains alone, and the same multiply-adds interleaved with
// integer-pipe products (one vote per iteration for the recomputation).
constexpr int RATE_ITER = 2048, RATE_CH = 8;

template <bool INTEGER>
__global__ void k_rate_mul(double* out, double c, double d) {
  double x[RATE_CH];
  for (int j = 0; j < RATE_CH; j++) x[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  unsigned bad = 0u;
  for (int i = 0; i < RATE_ITER; i++) {
    const double m = (i & 1) ? c : d;
#pragma unroll
    for (int j = 0; j < RATE_CH; j++) x[j] = INTEGER ? imul_rn(x[j], m, bad) : __dmul_rn(x[j], m);
  }
  double s = bad ? 1.0 : 0.0;
  for (int j = 0; j < RATE_CH; j++) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int NM>
__global__ void k_rate_mix(double* out, double c, double d) {
  double y[RATE_CH], x[NM > 0 ? NM : 1];
  for (int j = 0; j < RATE_CH; j++) y[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  for (int j = 0; j < NM; j++) x[j] = 1.0 + 2e-3 * (threadIdx.x + j);
  for (int i = 0; i < RATE_ITER; i++) {
#pragma unroll
    for (int j = 0; j < RATE_CH; j++) y[j] = fma(y[j], c, -d * 1e-9);
    if constexpr (NM > 0) {
      const double m = (i & 1) ? c : d;
      unsigned bad = 0u;
      double xn[NM];
#pragma unroll
      for (int j = 0; j < NM; j++) xn[j] = imul_rn(x[j], m, bad);
      if (__any_sync(0xffffffffu, bad != 0u)) {
#pragma unroll
        for (int j = 0; j < NM; j++) xn[j] = dmul_insn(x[j], m);
      }
#pragma unroll
      for (int j = 0; j < NM; j++) x[j] = xn[j];
    }
  }
  double s = 0.0;
  for (int j = 0; j < RATE_CH; j++) s += y[j];
  for (int j = 0; j < NM; j++) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

static double from_pattern(uint64_t b) {
  double d;
  std::memcpy(&d, &b, 8);
  return d;
}

int main() {
  std::mt19937_64 g(20070521);
  std::vector<double> x, y;
  const uint64_t edges[] = {0, 1, 2, 3, 5, 0x000fffffffffffffull, 0x000ffffffffffffeull, 0x0010000000000000ull,
                            0x0010000000000001ull, 0x001fffffffffffffull, 0x0020000000000000ull,
                            0x0020000000000001ull, 0x3ff0000000000000ull, 0x7fdfffffffffffffull,
                            0x7fe0000000000000ull, 0x7fefffffffffffffull, 0x7ff0000000000000ull,
                            0x7ff8000000000000ull, 0x0000000100000000ull, 0x00000000ffffffffull,
                            0x0000000080000001ull, 0x0000000180000000ull};
  for (uint64_t p : edges)
    for (uint64_t q : edges)
      for (uint64_t sp : {0ull, 1ull << 63})
        for (uint64_t sq : {0ull, 1ull << 63}) {
          x.push_back(from_pattern(p | sp));
          y.push_back(from_pattern(q | sq));
        }
  for (int i = 0; i < (1 << 22); i++) {
    uint64_t p = g(), q = g();
    const uint64_t ep = g() % 2048;
    uint64_t eq = (i % 4 == 0) ? g() % 8 : (i % 4 == 1) ? (ep ? ep - 1 : 0) : g() % 2048;  // tiny y; |x| near 2|y|
    p = (p & 0x800fffffffffffffull) | (ep << 52);
    q = (q & 0x800fffffffffffffull) | (eq << 52);
    if (i % 8 == 3) q = (q & 0xfff0000000000000ull) | (p & 0x000fffffffffffffull);  // |x| == 2|y| exactly
    if (i % 16 == 5) p = (p & 0x8000000000000000ull) | (g() % 0x0020000000000000ull);  // subnormal or smallest normal x
    x.push_back(from_pattern(p));
    y.push_back(from_pattern(q));
  }
  // patterns around the FP32 range for the narrowing: exponents 2^-163 .. 2^137,
  // with the dropped 29 mantissa bits at and next to the rounding tie
  for (int i = 0; i < (1 << 21); i++) {
    const uint64_t e = 860 + g() % 301;
    uint64_t mant = g() & 0x000fffffffffffffull;
    if (i % 4 == 1) mant = (mant & ~0x1fffffffull) | 0x10000000ull;                    // a tie
    if (i % 4 == 2) mant = (mant & ~0x1fffffffull) | (0x10000000ull + (g() % 3) - 1);  // next to it
    if (i % 8 == 3) mant |= 0x000fffffe0000000ull;                                     // all ones above: carry
    x.push_back(from_pattern((g() & (1ull << 63)) | (e << 52) | mant));
    y.push_back(from_pattern(g()));
  }
  // products near the ends of the normal range, exact products and rounding
  // ties: exponent pairs summing to about the bias and to its extremes
  for (int i = 0; i < (1 << 21); i++) {
    const uint64_t ea = 1 + g() % 2046;
    const int64_t target = (i % 3 == 0) ? 1023 : (i % 3 == 1) ? 1 : 2046;  // product exponent near 0, the bottom, the top
    int64_t eb = target - (int64_t)ea + 1023 + (int64_t)(g() % 5) - 2;
    if (eb < 0) eb = 0;
    if (eb > 2047) eb = 2047;
    uint64_t ma = g() & 0x000fffffffffffffull, mb = g() & 0x000fffffffffffffull;
    if (i % 4 == 1) mb &= 0x000ff00000000000ull;  // short significand: exact products and ties
    if (i % 8 == 5) ma = 0x000fffffffffffffull;   // all ones: carries through the rounding
    x.push_back(from_pattern((g() & (1ull << 63)) | (ea << 52) | ma));
    y.push_back(from_pattern((g() & (1ull << 63)) | ((uint64_t)eb << 52) | mb));
  }
  // normal positive arguments for the refined operations, 2^-1000 .. 2^1000
  std::vector<double> z(1 << 22);
  for (double& v : z) v = from_pattern(((uint64_t)(23 + g() % 2001) << 52) | (g() & 0x000fffffffffffffull));

  const int n = (int)x.size(), nz = (int)z.size();
  double *dx, *dy, *dz;
  unsigned long long *dbad, *dworst;
  cudaMalloc(&dx, n * sizeof(double));
  cudaMalloc(&dy, n * sizeof(double));
  cudaMalloc(&dz, nz * sizeof(double));
  cudaMalloc(&dbad, NBAD * sizeof(unsigned long long));
  cudaMalloc(&dworst, 3 * sizeof(unsigned long long));
  cudaMemcpy(dx, x.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(dy, y.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(dz, z.data(), nz * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemset(dbad, 0, NBAD * sizeof(unsigned long long));
  cudaMemset(dworst, 0, 3 * sizeof(unsigned long long));
  check_bits<<<(n + 255) / 256, 256>>>(dx, dy, n, dbad);
  check_refined<<<(nz + 255) / 256, 256>>>(dz, nz, dbad, dworst);
  const cudaError_t err = cudaDeviceSynchronize();
  unsigned long long bad[NBAD] = {}, worst[3] = {};
  cudaMemcpy(bad, dbad, sizeof(bad), cudaMemcpyDeviceToHost);
  cudaMemcpy(worst, dworst, sizeof(worst), cudaMemcpyDeviceToHost);
  std::printf("cuda %s\n", cudaGetErrorString(err));
  std::printf("bit-pattern cases %d: half_of / twice_of mismatches %llu, comparison mismatches %llu, narrowing mismatches %llu, "
              "integer-product mismatches %llu\n",
              n, bad[BAD_HALF], bad[BAD_CMP], bad[BAD_NARROW], bad[BAD_IMUL]);
  std::printf("refined cases %d: rcp > 2 ulp %llu (max %.3f), sqrt > 2 ulp %llu (max %.3f), rsqrt > 2^-51.5 %llu "
              "(max %.3f x 2^-53)\n",
              nz, bad[BAD_RCP], worst[0] / 1000.0, bad[BAD_SQRT], worst[1] / 1000.0, bad[BAD_RSQRT],
              worst[2] / 1000.0);
  {  // product throughput, 8 blocks of 256 threads per SM
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const int blocks = 8 * sms, threads = 256, nt = blocks * threads;
    double *r1, *r2;
    cudaMalloc(&r1, nt * sizeof(double));
    cudaMalloc(&r2, nt * sizeof(double));
    const double c = 1.0 + 0x1p-30, d = 1.0 / c;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto rate = [&](const char* name, auto launch, double ops) {
      launch();
      cudaEventRecord(e0);
      for (int r = 0; r < 5; r++) launch();
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      std::printf("rate %-34s %.3f ms, %.3f G lane-ops/s per SM\n", name, ms / 5, ops * nt / (ms / 5 * 1e-3) / sms / 1e9);
    };
    rate("FP64 multiply chains", [&] { k_rate_mul<false><<<blocks, threads>>>(r1, c, d); }, (double)RATE_ITER * RATE_CH);
    rate("integer-pipe product chains", [&] { k_rate_mul<true><<<blocks, threads>>>(r2, c, d); },
         (double)RATE_ITER * RATE_CH);
    rate("FP64 multiply-add chains", [&] { k_rate_mix<0><<<blocks, threads>>>(r1, c, d); }, (double)RATE_ITER * RATE_CH);
    rate("multiply-adds + 4 integer products", [&] { k_rate_mix<4><<<blocks, threads>>>(r1, c, d); },
         (double)RATE_ITER * (RATE_CH + 4));
    rate("multiply-adds + 8 integer products", [&] { k_rate_mix<8><<<blocks, threads>>>(r1, c, d); },
         (double)RATE_ITER * (RATE_CH + 8));
    k_rate_mul<false><<<blocks, threads>>>(r1, c, d);
    k_rate_mul<true><<<blocks, threads>>>(r2, c, d);
    std::vector<double> h1(nt), h2(nt);
    cudaMemcpy(h1.data(), r1, nt * sizeof(double), cudaMemcpyDeviceToHost);
    cudaMemcpy(h2.data(), r2, nt * sizeof(double), cudaMemcpyDeviceToHost);
    long nd = 0;
    for (int i = 0; i < nt; i++) nd += h1[i] != h2[i];
    std::printf("chained products (2048 per chain): %ld of %d results differ\n", nd, nt);
    if (nd) bad[BAD_IMUL] += (unsigned long long)nd;
    cudaFree(r1);
    cudaFree(r2);
  }
  bool ok = err == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
  for (unsigned long long b : bad) ok = ok && b == 0;
  std::printf("%s\n", ok ? "PASS" : "FAIL");
  return ok ? 0 : 1;
}
