// Allocation-free variant of the CFL time-step reduction.
//
// hydro_compute_dt works on a handle whose scratch buffer the caller has to
// allocate (about 136 doubles per ghosted zone).  Some callers cannot allocate
// device memory at the point where they need a time step: a process that
// hands all device memory to its own pool at start-up and permits no further
// allocation, or a latency-critical loop that cannot pay for cudaMalloc /
// cudaFree, which may stall or synchronise the device.
// hydro_compute_dt_noalloc serves them: the caller
// passes only the state (input) and the dt array (output); the reduction's
// scratch -- a copy of the box table and one max-signal-speed slot per box --
// lives in the file-scope device array below, which every GPU that loads the
// library holds until the process exits.
#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "hydro_internal.cuh"

namespace {

struct DtBox {
  int n[3];
  int pad;
  long long pitch, plane, vs, state_off;
  double idx[3];
  double gamma;
  double cfl;
};

struct DtScratch {
  DtBox boxes[HYDRO_NOALLOC_MAX_BOXES];
  unsigned long long smax[HYDRO_NOALLOC_MAX_BOXES];  // non-negative double bits
};

// The whole scratch of this entry point (about 96 KB per device).
static __device__ __align__(256) DtScratch g_dt_scratch;

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
DtScratch* g_scratch_addr[MAX_DEVICES] = {nullptr};

int fail(int code, const std::string& msg) {
  hydro::set_last_error(msg);
  return code;
}

// Device address of g_dt_scratch for the current device, looked up once per
// device (with that device current) and cached.
int scratch_for_current_device(DtScratch** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(HYDRO_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= MAX_DEVICES) return fail(HYDRO_ERR_INVALID, "device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dt_scratch);
    if (e != cudaSuccess || !p)
      return fail(HYDRO_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<DtScratch*>(p);
  }
  *out = g_scratch_addr[dev];
  return HYDRO_OK;
}

__global__ void __launch_bounds__(256) k_dt_speed(DtScratch* __restrict__ scr, const double* __restrict__ state) {
  const int bi = blockIdx.y;
  const DtBox& b = scr->boxes[bi];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long N = (long long)b.n[0] * b.n[1] * b.n[2];
  unsigned long long sbits = 0ull;
  if (t < N) {
    const long long r = t / b.n[0];
    const int i = (int)(t - r * b.n[0]);
    const int k = (int)(r / b.n[1]);
    const int j = (int)(r - (long long)k * b.n[1]);
    const long long Z = b.state_off + (i + HYDRO_NG) + (j + HYDRO_NG) * b.pitch + (k + HYDRO_NG) * b.plane;
    double rho = state[Z];
    if (rho < hydro::SMALL_DENS) rho = hydro::SMALL_DENS;
    const double ir = 1.0 / rho;
    const double u = state[Z + b.vs] * ir, v = state[Z + 2 * b.vs] * ir, w = state[Z + 3 * b.vs] * ir;
    double p = (b.gamma - 1.0) * (state[Z + 4 * b.vs] - 0.5 * rho * (u * u + v * v + w * w));
    if (p < hydro::SMALL_PRES) p = hydro::SMALL_PRES;
    const double cs = sqrt(b.gamma * p * ir);
    const double s = fmax(fmax((fabs(u) + cs) * b.idx[0], (fabs(v) + cs) * b.idx[1]), (fabs(w) + cs) * b.idx[2]);
    sbits = (unsigned long long)__double_as_longlong(s);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, sbits, off);
    sbits = o > sbits ? o : sbits;
  }
  if ((threadIdx.x & 31) == 0 && sbits) atomicMax(&scr->smax[bi], sbits);
}

__global__ void k_dt_finish(const DtScratch* __restrict__ scr, int nboxes, double* __restrict__ dt) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nboxes; b += gridDim.x * blockDim.x)
    dt[b] = scr->boxes[b].cfl / __longlong_as_double((long long)scr->smax[b]);
}

}  // namespace

extern "C" int hydro_compute_dt_noalloc(const hydro_box_desc* d, int nboxes, const double* state_dev,
                                        double* dt_dev, void* stream) {
  if (!d || !state_dev || !dt_dev) return fail(HYDRO_ERR_INVALID, "null argument");
  if (nboxes <= 0 || nboxes > HYDRO_NOALLOC_MAX_BOXES) {
    char buf[128];
    snprintf(buf, sizeof buf, "hydro_compute_dt_noalloc: nboxes = %d, must be in [1, %d]", nboxes,
             HYDRO_NOALLOC_MAX_BOXES);
    return fail(HYDRO_ERR_INVALID, buf);
  }
  // Validates the descriptors and gives each box's place in the state buffer.
  size_t sb = 0, wb = 0;
  if (hydro_workspace_size(d, nboxes, &sb, &wb) != HYDRO_OK) return HYDRO_ERR_INVALID;
  std::vector<DtBox> table(nboxes);
  long long maxN = 0;
  for (int i = 0; i < nboxes; i++) {
    hydro_layout lay;
    if (hydro_box_layout(d, nboxes, i, &lay) != HYDRO_OK) return HYDRO_ERR_INVALID;
    DtBox& b = table[i];
    memset(&b, 0, sizeof b);
    b.n[0] = d[i].nx;
    b.n[1] = d[i].ny;
    b.n[2] = d[i].nz;
    b.pitch = lay.pitch;
    b.plane = lay.plane;
    b.vs = lay.var_stride;
    b.state_off = lay.offset;
    b.idx[0] = 1.0 / d[i].dx;
    b.idx[1] = 1.0 / d[i].dy;
    b.idx[2] = 1.0 / d[i].dz;
    b.gamma = d[i].gamma;
    b.cfl = d[i].cfl;
    maxN = std::max(maxN, (long long)d[i].nx * d[i].ny * d[i].nz);
  }
  DtScratch* scr = nullptr;
  int rc = scratch_for_current_device(&scr);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The box table goes into the static scratch; the per-box maxima start at zero.
  char* base = reinterpret_cast<char*>(scr);
  cudaError_t e = cudaMemcpyAsync(base + offsetof(DtScratch, boxes), table.data(), sizeof(DtBox) * nboxes,
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(base + offsetof(DtScratch, smax), 0, sizeof(unsigned long long) * nboxes, s);
  if (e == cudaSuccess) {
    const dim3 grid((unsigned)((maxN + 255) / 256), (unsigned)nboxes);
    k_dt_speed<<<grid, 256, 0, s>>>(scr, state_dev);
    k_dt_finish<<<(nboxes + 255) / 256, 256, 0, s>>>(scr, nboxes, dt_dev);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return fail(HYDRO_ERR_CUDA, std::string("hydro_compute_dt_noalloc: ") + cudaGetErrorString(e));
  return HYDRO_OK;
}
