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
// scratch -- a copy of the box table, a block-to-box table and one
// max-signal-speed slot per box -- lives in the file-scope device array below,
// which every GPU that loads the library holds until the process exits.
//
// The signal speeds come from the same device function as the primitive
// stage of a handle (prim_zone.cuh), so under the default limiter the time
// steps equal hydro_compute_dt's bit for bit.
#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "prim_zone.cuh"

namespace {

struct DtBox {
  int n[3];
  int pad;
  long long pitch, plane, vs, state_off;
  double idx[3];
  double gamma;
  double gm1;  // gamma - 1
  double cfl;
};

// Blocks one box gets at most; a larger box is covered by a grid-stride loop,
// so one big box does not make every small box of the call launch as many
// blocks as it does.
constexpr int MAX_BLOCKS_PER_BOX = 2048;
constexpr int DT_THREADS = 256;

struct DtScratch {
  DtBox boxes[HYDRO_NOALLOC_MAX_BOXES];
  int start[HYDRO_NOALLOC_MAX_BOXES + 1];  // first block of each box; start[nboxes] = blocks
  int pad[3];
  unsigned long long smax[HYDRO_NOALLOC_MAX_BOXES];  // non-negative double bits
};

// The whole scratch of this entry point (about 100 KB per device).
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

// One block: find its box in the block-to-box table, then walk the box's
// interior zones with a stride of the box's blocks.
__global__ void __launch_bounds__(DT_THREADS) k_dt_speed(DtScratch* __restrict__ scr, int nboxes,
                                                         const double* __restrict__ state) {
  const int blk = blockIdx.x;
  int lo = 0, hi = nboxes;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (scr->start[mid] <= blk) lo = mid;
    else hi = mid;
  }
  const int bi = lo;
  const DtBox& b = scr->boxes[bi];
  const long long nblk = scr->start[bi + 1] - scr->start[bi];
  const long long N = (long long)b.n[0] * b.n[1] * b.n[2];
  unsigned long long sbits = 0ull;
  for (long long t = (long long)(blk - scr->start[bi]) * DT_THREADS + threadIdx.x; t < N; t += nblk * DT_THREADS) {
    const long long r = t / b.n[0];
    const int i = (int)(t - r * b.n[0]);
    const int k = (int)(r / b.n[1]);
    const int j = (int)(r - (long long)k * b.n[1]);
    const long long Z = b.state_off + (i + HYDRO_NG) + (j + HYDRO_NG) * b.pitch + (k + HYDRO_NG) * b.plane;
    const hydro::PrimZone z = hydro::prim_zone(state[Z], state[Z + b.vs], state[Z + 2 * b.vs],
                                               state[Z + 3 * b.vs], state[Z + 4 * b.vs], b.gamma, b.gm1);
    const unsigned long long s = (unsigned long long)__double_as_longlong(hydro::signal_rate(z.u, z.v, z.w, z.cs, b.idx));
    sbits = s > sbits ? s : sbits;  // non-negative doubles order like their bit patterns
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
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The box table below is copied from host memory that lives only for this
  // call; a graph captured here would keep a pointer to it.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess)
    return fail(HYDRO_ERR_CUDA, std::string("hydro_compute_dt_noalloc: cudaStreamIsCapturing: ") +
                                    cudaGetErrorString(e));
  if (cap != cudaStreamCaptureStatusNone)
    return fail(HYDRO_ERR_INVALID,
                "hydro_compute_dt_noalloc: the stream is being captured; the call copies its box table from "
                "host memory that does not outlive it, so it runs only outside stream capture");
  // Validates the descriptors and gives each box's place in the state buffer.
  std::vector<hydro_layout> lay(nboxes);
  if (hydro::box_layouts(d, nboxes, lay.data()) != HYDRO_OK) return HYDRO_ERR_INVALID;
  // The box table and the block-to-box table, as one host image of the head
  // of the static scratch.
  const size_t head = offsetof(DtScratch, pad);
  std::vector<char> image(head, 0);
  DtBox* table = reinterpret_cast<DtBox*>(image.data() + offsetof(DtScratch, boxes));
  int* start = reinterpret_cast<int*>(image.data() + offsetof(DtScratch, start));
  long long blocks = 0;
  for (int i = 0; i < nboxes; i++) {
    DtBox& b = table[i];
    b.n[0] = d[i].nx;
    b.n[1] = d[i].ny;
    b.n[2] = d[i].nz;
    b.pitch = lay[i].pitch;
    b.plane = lay[i].plane;
    b.vs = lay[i].var_stride;
    b.state_off = lay[i].offset;
    b.idx[0] = 1.0 / d[i].dx;
    b.idx[1] = 1.0 / d[i].dy;
    b.idx[2] = 1.0 / d[i].dz;
    b.gamma = d[i].gamma;
    b.gm1 = d[i].gamma - 1.0;
    b.cfl = d[i].cfl;
    const long long n = (long long)d[i].nx * d[i].ny * d[i].nz;
    start[i] = (int)blocks;
    blocks += std::min<long long>((n + DT_THREADS - 1) / DT_THREADS, MAX_BLOCKS_PER_BOX);
  }
  start[nboxes] = (int)blocks;
  DtScratch* scr = nullptr;
  int rc = scratch_for_current_device(&scr);
  if (rc) return rc;
  // The tables go into the static scratch (pageable source: the copy is
  // staged before cudaMemcpyAsync returns); the per-box maxima start at zero.
  char* base = reinterpret_cast<char*>(scr);
  e = cudaMemcpyAsync(base + offsetof(DtScratch, boxes), table, sizeof(DtBox) * nboxes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + offsetof(DtScratch, start), start, sizeof(int) * (nboxes + 1),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(base + offsetof(DtScratch, smax), 0, sizeof(unsigned long long) * nboxes, s);
  if (e == cudaSuccess) {
    k_dt_speed<<<(unsigned)blocks, DT_THREADS, 0, s>>>(scr, nboxes, state_dev);
    k_dt_finish<<<(nboxes + 255) / 256, 256, 0, s>>>(scr, nboxes, dt_dev);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return fail(HYDRO_ERR_CUDA, std::string("hydro_compute_dt_noalloc: ") + cudaGetErrorString(e));
  return HYDRO_OK;
}
