// Stage kernels of the unsplit PPM/CTU update, one kernel per stage with the
// intermediates in HBM scratch.
//
// Design for GB300: the update costs thousands of floating-point operations
// per zone and GB300's FP64 pipe is narrow, while HBM bandwidth is plentiful.
// So every quantity is computed once and parked in HBM rather than recomputed
// by neighbouring threads: the stage kernels read their stencil from scratch
// fields laid out like the state (x fastest, coalesced across a warp).  For
// FP32 boxes, where the stages are bound by memory traffic instead, four
// line kernels (listed below) fuse several stages along one axis and keep the
// stencil in registers.
//
// Precision.  The state, the dt reduction and the flux-divergence update are
// always FP64.  The reconstruction, tracing, CTU corrections and Riemann
// solves (the templated stage kernels, compute type R) run in FP64 for
// HYDRO_FP64 boxes and in FP32 for HYDRO_MIXED boxes, whose scratch fields are
// FP32 (half the bytes).  Each face flux is a single value used by both
// neighbours, so the FP64 update conserves mass, momentum and energy to FP64
// round-off in both forms.
//
// Stages (paper §3: limited slopes from neighbours, then a polynomial
// reconstruction; the published methods are cited per stage):
//   k_fill       ghost zones from the boundary conditions (x, then y, then z)
//   k_prim       conserved -> primitive + EOS (FP64); per-box max signal speed;
//                1/c and c/rho for the FP64 tracing
//   k_dt         dt = cfl / max((|u_d|+c)/dx_d)
//   k_flatten    CW84 §4 shock flattening coefficient (max over directions)
//   k_slopes     CW84 limited slopes, once per zone and axis (none for CS08)
//   k_trace      PPM parabolas (CW84 or CS08 limiter) + characteristic
//                tracing -> face states
//   k_riemann    normal fluxes F0_d on the extended face region (HLLC or the
//                two-shock solver, as for every Riemann solve below)
//   k_ctu1       3D CTU stage 1: dt/(3dx_e) transverse corrections + solves
//   k_ctu2       3D CTU stage 2: dt/(2dx) corrections + solves -> final fluxes
//   k_update     conservative flux-divergence update (FP64) + physicality flag
// FP32 boxes (unless line fusion is switched off) replace the middle stages:
//   k_line_x     slopes + trace + normal solve along x, one warp per x-line
//   k_line_yz    the same along y or z, threads walking a column segment
//   k_ctu1_line  CTU stage 1, zone-wise: each zone's flux differences loaded
//                once for both of its faces
//   k_ctu2_line  CTU stage 2, zone-wise in the same way
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fp64_fast.cuh"
#include "hydro_internal.cuh"
#include "prim_zone.cuh"

namespace hydro {
namespace {

// slot m of the normal frame of axis D -> x,y,z component (0 rho, 1..3 velocity/momentum, 4 p/E)
template <int D>
__device__ __forceinline__ constexpr int comp(int m) {
  return (m == 0 || m == 4) ? m : 1 + (D + m - 1) % 3;
}

template <typename R>
__device__ __forceinline__ bool box_uses(const DevBox& b);
template <>
__device__ __forceinline__ bool box_uses<double>(const DevBox& b) { return b.precision == HYDRO_FP64; }
template <>
__device__ __forceinline__ bool box_uses<float>(const DevBox& b) { return b.precision == HYDRO_MIXED; }

// Per-box constants in the compute type: FP64 kernels read the doubles, FP32
// kernels the float copies (a double->float conversion occupies the FP64 pipe).
template <typename R>
struct Consts;
template <>
struct Consts<double> {
  // FP64 edge states keep their conserved form in HBM (FP64 arithmetic is the
  // scarce resource); FP32 ones rebuild it where they are read (HBM traffic is)
  static constexpr bool STORE_CONSERVED = true;
  // a corrected state's 1/rho comes from the 1/sqrt(rho) the Riemann solver
  // needs (saves FP64 instructions; in FP32 the extra live register costs
  // more occupancy than the reciprocal it saves)
  static constexpr bool SHARE_RSQRT = true;
  // FP64 instructions are the scarce resource: an instruction that a warp
  // issues with only some lanes active costs as much as a full one, so the
  // limiter selects operands instead of branching, and the tracing skips a
  // wave's block only when no lane of the warp needs it
  static constexpr bool FP_BOUND = true;
  // the primitive conversion stores 1/c and c/rho for the tracing, which
  // reads them for each of the three axes instead of forming two reciprocals
  static constexpr bool PRIM_RECIPROCALS = true;
  static __device__ __forceinline__ double gamma(const DevBox& b) { return b.gamma; }
  static __device__ __forceinline__ double igm1(const DevBox& b) { return b.igm1; }
  static __device__ __forceinline__ double gm1(const DevBox& b) { return b.gm1; }
  // dt/dx, dt/(3 dx) and dt/(2 dx), formed once per step by the time-step kernel
  static __device__ __forceinline__ double dtdx(const DevBox&, const BoxRt& r, int d) { return r.dtdx[d]; }
  static __device__ __forceinline__ double dtdx3(const DevBox&, const BoxRt& r, int d) { return r.dtdx3[d]; }
  static __device__ __forceinline__ double dtdx2(const DevBox&, const BoxRt& r, int d) { return r.dtdx2[d]; }
};
template <>
struct Consts<float> {
  static constexpr bool STORE_CONSERVED = false;
  static constexpr bool SHARE_RSQRT = false;
  static constexpr bool FP_BOUND = false;
  static constexpr bool PRIM_RECIPROCALS = false;
  static __device__ __forceinline__ float gamma(const DevBox& b) { return b.gamma_f; }
  static __device__ __forceinline__ float igm1(const DevBox& b) { return b.igm1_f; }
  static __device__ __forceinline__ float gm1(const DevBox& b) { return b.gamma_f - 1.0f; }
  static __device__ __forceinline__ float dtdx(const DevBox&, const BoxRt& r, int d) { return r.dtdx_f[d]; }
  static __device__ __forceinline__ float dtdx3(const DevBox&, const BoxRt& r, int d) {
    return r.dtdx_f[d] * float(1.0 / 3.0);
  }
  static __device__ __forceinline__ float dtdx2(const DevBox&, const BoxRt& r, int d) { return 0.5f * r.dtdx_f[d]; }
};

template <typename R>
__device__ __forceinline__ R* fields(unsigned char* work, const DevBox& b) {
  return reinterpret_cast<R*>(work + b.work_off);
}

// Whether c holds on any active lane of the warp (FP_BOUND types; else c
// itself): a block guarded by it is skipped when no lane needs it, also where
// the compiler predicates the block rather than branching around it.
template <typename R>
__device__ __forceinline__ bool any_in_warp(bool c) {
  if constexpr (Consts<R>::FP_BOUND) return __any_sync(__activemask(), c);
  return c;
}

__device__ __forceinline__ long long zone(const DevBox& b, int i, int j, int k) {
  return (long long)(i + NG) + (long long)(j + NG) * b.s[1] + (long long)(k + NG) * b.s[2];
}

// linear thread index -> zone of the region lo[a] .. lo[a]+ext[a]-1 (x fastest).
// Regions of fewer than 2^32 zones (every box up to about 1600^3) divide in
// 32 bits -- a 64-bit integer division is a long software sequence, and this
// runs once per thread of every stage; the test is uniform over a block.
__device__ __forceinline__ bool decode(long long t, const int* lo, const int* ext, int* c) {
  const unsigned long long vol = (unsigned long long)ext[0] * (unsigned)ext[1] * (unsigned)ext[2];
  if ((unsigned long long)t >= vol) return false;
  if (vol <= 0xffffffffull) {
    const unsigned tt = (unsigned)t, e0 = (unsigned)ext[0], e1 = (unsigned)ext[1];
    const unsigned r = tt / e0;
    c[0] = lo[0] + (int)(tt - r * e0);
    const unsigned k = r / e1;
    c[1] = lo[1] + (int)(r - k * e1);
    c[2] = lo[2] + (int)k;
  } else {
    const long long r = t / ext[0];
    c[0] = lo[0] + (int)(t - r * ext[0]);
    const long long k = r / ext[1];
    c[1] = lo[1] + (int)(r - k * ext[1]);
    c[2] = lo[2] + (int)k;
  }
  return true;
}

// Device view of a work table: block -> (box, axis) and the thread's index in
// the item's region (binary search over the item start blocks).
struct TableView {
  const int* start;
  const int* item;
  int nitems;
};

__device__ __forceinline__ int locate(const TableView& w, int* z, long long* t) {
  const int blk = blockIdx.x;
  int lo = 0, hi = w.nitems;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(w.start + mid) <= blk) lo = mid;
    else hi = mid;
  }
  const int code = __ldg(w.item + lo);
  *z = code & 7;
  *t = (long long)(blk - __ldg(w.start + lo)) * blockDim.x + threadIdx.x;
  return code >> 3;
}

#define LOCATE(tv)                  \
  int z_;                           \
  long long t_;                     \
  const int bi = locate(tv, &z_, &t_); \
  const DevBox& b = boxes[bi];

// The same for block `blk` of the table (a stage body run by a stage kernel
// with blk = blockIdx.x, or by the persistent kernel for the block it took).
__device__ __forceinline__ int locate_at(const TableView& w, int blk, int* z, long long* t) {
  int lo = 0, hi = w.nitems;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(w.start + mid) <= blk) lo = mid;
    else hi = mid;
  }
  const int code = __ldg(w.item + lo);
  *z = code & 7;
  *t = (long long)(blk - __ldg(w.start + lo)) * blockDim.x + threadIdx.x;
  return code >> 3;
}

#define LOCATE_AT(tv, blk)                    \
  int z_;                                     \
  long long t_;                               \
  const int bi = locate_at(tv, blk, &z_, &t_); \
  const DevBox& b = boxes[bi];

// ----------------------------------------------------------------- ghost fill
template <int D>
__device__ __forceinline__ void body_fill(const TableView& tv, const int blk_, const DevBox* boxes, double* state) {
  LOCATE_AT(tv, blk_)
  int lo[3], ext[3], c[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    if (a == D) { lo[a] = 0; ext[a] = 2 * NG; }
    else if (a < D) { lo[a] = -NG; ext[a] = b.n[a] + 2 * NG; }
    else { lo[a] = 0; ext[a] = b.n[a]; }
  }
  if (!decode(t_, lo, ext, c)) return;
  const int l = c[D], n = b.n[D];
  const int side = l < NG ? 0 : 1;
  const int m = side == 0 ? NG - l : l - NG + 1;  // depth 1..NG
  const int nb1 = b.nbr1[2 * D + side];
  double* U = state + b.state_off;
  if (nb1 > 0) {
    // a neighbouring box of the same domain: copy its interior layer at depth m
    // (its extents across D equal this box's, its strides may differ)
    const DevBox& o = boxes[nb1 - 1];
    const int src = side == 0 ? o.n[D] - m : m - 1;
    c[D] = side == 0 ? -m : n - 1 + m;
    const long long zg = zone(b, c[0], c[1], c[2]);
    c[D] = src;
    const long long zs = zone(o, c[0], c[1], c[2]);
    const double* S = state + o.state_off;
#pragma unroll
    for (int v = 0; v < 5; v++) U[v * b.vs + zg] = S[v * o.vs + zs];
    return;
  }
  const int bc = b.bc[2 * D + side];
  int src;
  if (bc == HYDRO_BC_PERIODIC) src = side == 0 ? n - m : m - 1;
  else if (bc == HYDRO_BC_OUTFLOW) src = side == 0 ? 0 : n - 1;
  else src = side == 0 ? m - 1 : n - m;
  c[D] = side == 0 ? -m : n - 1 + m;
  const long long zg = zone(b, c[0], c[1], c[2]);
  c[D] = src;
  const long long zs = zone(b, c[0], c[1], c[2]);
#pragma unroll
  for (int v = 0; v < 5; v++) {
    double val = U[v * b.vs + zs];
    if (bc == HYDRO_BC_REFLECT && v == 1 + D) val = -val;
    U[v * b.vs + zg] = val;
  }
}

// out-of-line copy for the persistent kernel
template <int D>
__device__ __noinline__ void b_fill(const TableView& tv, const int blk_, const DevBox* boxes, double* state) {
  body_fill<D>(tv, blk_, boxes, state);
}

template <int D>
__global__ void __launch_bounds__(256) k_fill(TableView tv, const DevBox* __restrict__ boxes, double* __restrict__ state) {
  body_fill<D>(tv, blockIdx.x, boxes, state);
}

// ------------------------------------------------- conserved -> primitive, dt
// FP64 arithmetic for every box (the dt reduction needs it); the primitive
// fields are stored in the box's compute type, and for FP64 boxes also 1/c
// and c/rho, which the tracing reads on each axis.
// EXACT (used under the CS08 limiter, whose branches are not continuous in
// their inputs): the primitive state with correctly rounded divides and square
// root and no fused multiply-adds, u = U1 / rho, ..., p = (gamma - 1)(E -
// (rho / 2)(u^2 + v^2 + w^2)), c = sqrt(gamma p / rho), in that order, so that
// the limiter's decisions are reproducible on any IEEE machine.  Otherwise one
// refined reciprocal (1/rho) and one refined reciprocal square root, of c^2,
// which is 1/c and gives c = c^2 (1/c).
template <bool EXACT>
__device__ __forceinline__ void body_prim(const TableView& tv, const int blk_, const DevBox* boxes, const double* state, unsigned char* work, BoxRt* rt) {
  LOCATE_AT(tv, blk_)
  int lo[3] = {-NG, -NG, -NG};
  int ext[3] = {b.n[0] + 2 * NG, b.n[1] + 2 * NG, b.n[2] + 2 * NG};
  int c[3];
  unsigned long long sbits = 0ull;
  if (decode(t_, lo, ext, c)) {
    const long long Z = zone(b, c[0], c[1], c[2]);
    const long long vs = b.vs;
    const double* U = state + b.state_off;
    double rho = U[Z];
    double u, v, w, p, cs, ir = 0.0, ic = 0.0;
    if constexpr (EXACT) {
      if (dgt(SMALL_DENS, rho)) rho = SMALL_DENS;
      u = __ddiv_rn(U[vs + Z], rho);
      v = __ddiv_rn(U[2 * vs + Z], rho);
      w = __ddiv_rn(U[3 * vs + Z], rho);
      const double uu = __dadd_rn(__dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)), __dmul_rn(w, w));
      const double kin = __dmul_rn(__dmul_rn(0.5, rho), uu);
      p = __dmul_rn(b.gm1, __dsub_rn(U[4 * vs + Z], kin));
      if (dgt(SMALL_PRES, p)) p = SMALL_PRES;
      cs = __dsqrt_rn(__ddiv_rn(__dmul_rn(b.gamma, p), rho));
    } else {
      const PrimZone pz = prim_zone(rho, U[vs + Z], U[2 * vs + Z], U[3 * vs + Z], U[4 * vs + Z], b.gamma, b.gm1);
      rho = pz.rho;
      u = pz.u;
      v = pz.v;
      w = pz.w;
      p = pz.p;
      cs = pz.cs;
      ir = pz.ir;
      ic = pz.ic;
    }
    if (b.precision == HYDRO_FP64) {
      double* W = fields<double>(work, b);
      W[Z] = rho;
      W[vs + Z] = u;
      W[2 * vs + Z] = v;
      W[3 * vs + Z] = w;
      W[4 * vs + Z] = p;
      W[FLD_C * vs + Z] = cs;
      if constexpr (EXACT) {
        ic = nr_rcp(cs);
        ir = nr_rcp(rho);
      }
      W[FLD_IC * vs + Z] = ic;
      W[FLD_CR * vs + Z] = cs * ir;
    } else if constexpr (EXACT) {  // conversion instructions (this form is bound by its IEEE divides)
      float* W = fields<float>(work, b);
      W[Z] = (float)rho;
      W[vs + Z] = (float)u;
      W[2 * vs + Z] = (float)v;
      W[3 * vs + Z] = (float)w;
      W[4 * vs + Z] = (float)p;
      W[FLD_C * vs + Z] = (float)cs;
    } else {
      // rounded to FP32 on the integer pipe (bitwise the conversion); a warp
      // converts with the instruction only where a lane holds a value outside
      // the normal FP32 range (other than a zero-bound one)
      float* W = fields<float>(work, b);
      const double q[6] = {rho, u, v, w, p, cs};
      unsigned r[6], defer = 0u;
#pragma unroll
      for (int m = 0; m < 6; m++) {
        bool x;
        r[m] = narrow_bits(q[m], x);
        defer |= (unsigned)x << m;
      }
      if (__any_sync(__activemask(), defer != 0u)) {
#pragma unroll
        for (int m = 0; m < 6; m++)
          if ((defer >> m) & 1u) r[m] = __float_as_uint(__double2float_rn(q[m]));
      }
      const int slot[6] = {0, 1, 2, 3, 4, FLD_C};
#pragma unroll
      for (int m = 0; m < 6; m++) W[slot[m] * vs + Z] = __uint_as_float(r[m]);
    }
    if (c[0] >= 0 && c[0] < b.n[0] && c[1] >= 0 && c[1] < b.n[1] && c[2] >= 0 && c[2] < b.n[2]) {
      const double s = signal_rate(u, v, w, cs, b.idx);
      sbits = (unsigned long long)__double_as_longlong(s);
    }
  }
  // non-negative doubles order like their bit patterns: reduce as integers,
  // in 32-bit halves
  unsigned hs = (unsigned)(sbits >> 32), ls = (unsigned)sbits;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned ho = __shfl_xor_sync(0xffffffffu, hs, off), lo = __shfl_xor_sync(0xffffffffu, ls, off);
    if (ho > hs || (ho == hs && lo > ls)) {
      hs = ho;
      ls = lo;
    }
  }
  if ((threadIdx.x & 31) == 0 && (hs | ls)) atomicMax(&rt[bi].smax, ((unsigned long long)hs << 32) | ls);
}

// out-of-line copy for the persistent kernel
template <bool EXACT>
__device__ __noinline__ void b_prim(const TableView& tv, const int blk_, const DevBox* boxes, const double* state, unsigned char* work, BoxRt* rt) {
  body_prim<EXACT>(tv, blk_, boxes, state, work, rt);
}

template <bool EXACT>
__global__ void __launch_bounds__(256) k_prim(TableView tv, const DevBox* __restrict__ boxes, const double* __restrict__ state, unsigned char* __restrict__ work, BoxRt* __restrict__ rt) {
  body_prim<EXACT>(tv, blockIdx.x, boxes, state, work, rt);
}

// dt/dx per axis in both compute types and the FP64 transverse-correction
// factors of the step, formed once per box
__device__ __forceinline__ void set_factors(BoxRt& r, double dt, const double* idx) {
  for (int a = 0; a < 3; a++) {
    const double f = __dmul_rn(dt, idx[a]);
    r.dtdx[a] = f;
    r.dtdx3[a] = __dmul_rn(f, 1.0 / 3.0);
    r.dtdx2[a] = __dmul_rn(0.5, f);
    r.dtdx_f[a] = (float)f;
  }
}

// The time step of box b: dt_in[b] if given, else cfl / (largest signal rate,
// reduced by the primitive stage); the reduction slot is cleared for the
// next step.
__device__ __noinline__ void b_dt_box(const DevBox* boxes, BoxRt* rt, int b, const double* dt_in, double* dt_out,
                                      int advance) {
  const double smax = __longlong_as_double((long long)rt[b].smax);
  const double dt = dt_in ? dt_in[b] : boxes[b].cfl / smax;
  rt[b].smax = 0ull;
  rt[b].dt = dt;
  set_factors(rt[b], dt, boxes[b].idx);
  if (dt_out) dt_out[b] = dt;
  if (advance) {
    rt[b].time += dt;
    rt[b].steps += 1u;
  }
}

__global__ void k_dt(const DevBox* __restrict__ boxes, BoxRt* __restrict__ rt, int nboxes,
                     const double* __restrict__ dt_in, double* __restrict__ dt_out, int advance) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nboxes; b += gridDim.x * blockDim.x) {
    if (boxes[b].n[0] == 0) continue;  // a free slot of a server plan
    b_dt_box(boxes, rt, b, dt_in, dt_out, advance);
  }
}

// One dt for all boxes of a domain (an AMR level advanced together): the
// minimum over boxes of cfl_b / smax_b.  One block.
__global__ void __launch_bounds__(256) k_dt_shared(const DevBox* __restrict__ boxes, BoxRt* __restrict__ rt,
                                                   int nboxes, double* __restrict__ dt_out, int advance) {
  __shared__ double red[256];
  double m = HUGE_VAL;
  for (int b = threadIdx.x; b < nboxes; b += blockDim.x) {
    if (boxes[b].n[0] == 0) continue;
    m = fmin(m, boxes[b].cfl / __longlong_as_double((long long)rt[b].smax));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  const double dt = red[0];
  for (int b = threadIdx.x; b < nboxes; b += blockDim.x) {
    if (boxes[b].n[0] == 0) continue;
    rt[b].smax = 0ull;
    rt[b].dt = dt;
    set_factors(rt[b], dt, boxes[b].idx);
    if (dt_out) dt_out[b] = dt;
    if (advance) {
      rt[b].time += dt;
      rt[b].steps += 1u;
    }
  }
}

// CS08's branches (interface in bounds, zone or neighbour at an extremum,
// second differences of one sign) are not continuous in their inputs: a
// one-ulp change can move an edge value by the size of the limited
// curvature.  So every quantity a branch depends on (the interface values
// included) is formed with single IEEE operations (no contraction into fused
// multiply-adds) in the order the method writes them, and equal inputs give
// bitwise equal decisions on any IEEE machine.
__device__ __forceinline__ double ie_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ie_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float ie_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float ie_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double ie_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float ie_div(float a, float b) { return __fdiv_rn(a, b); }
// a single rounded product by a multiplication policy: the policy's FP64
// product (correctly rounded, never fused), the FP32 intrinsic
template <typename M>
__device__ __forceinline__ double ie_mul(double a, double b, M& mul) { return mul(a, b); }
template <typename M>
__device__ __forceinline__ float ie_mul(float a, float b, M&) { return __fmul_rn(a, b); }

// ---------------------------------------------------------------- flattening
// CW84's shock test |dp1| / min(p) > eps, a discontinuous decision.  FP64: the
// same decision as the correctly rounded quotient compared with eps, without
// a divide wherever the answer is clear: d = a - eps m from one multiply-add
// has the exact sign of a/m - eps, and when |d| > 2^-48 a the quotient lies
// more than 2^-48 (relative) away from eps, farther than its rounding can
// move it; within that band (rare) the warp forms the quotient itself.
// FP32 (mixed precision): the product form a > eps m.
template <typename R>
__device__ __forceinline__ bool flat_shock(R a, R m) {
  if constexpr (Consts<R>::FP_BOUND) {
    const R d = fma(-R(FLAT_EPS), m, a);
    const bool near = !dgt(R(fabs(d)), a * R(0x1p-48));
    bool r = is_pos(d);
    if (any_in_warp<R>(near)) {
      if (near) r = ie_div(a, m) > R(FLAT_EPS);
    }
    return r;
  } else {
    return dgt(a, R(FLAT_EPS) * m);
  }
}

template <typename R>
// (comparisons and min/max through the helpers: exact, and off the FP64 pipe;
// the ratio dp1/dp2 only enters the clamped linear part, so the refined
// reciprocal's rounding moves the coefficient by rounding alone)
__device__ __forceinline__ R flat_tilde(const R* __restrict__ p, const R* __restrict__ un, long long Z, long long s) {
  const R pp = p[Z + s], pm = p[Z - s];
  const R dp1 = pp - pm;
  if (!flat_shock(R(fabs(dp1)), dmin(pp, pm)) || !is_pos(un[Z - s] - un[Z + s])) return R(0);
  const R dp2 = p[Z + 2 * s] - p[Z - 2 * s];
  if (!is_pos(fabs(dp2))) return R(0);
  return dmin(R(1), dmax(R(0), R(FLAT_OMEGA2) * (dp1 * nr_rcp(dp2) - R(FLAT_OMEGA1))));
}

template <typename R>
__device__ __forceinline__ void body_flatten(const TableView& tv, const int blk_, const DevBox* boxes, unsigned char* work) {
  LOCATE_AT(tv, blk_)
  if (!box_uses<R>(b)) return;
  int lo[3] = {-1, -1, -1}, ext[3] = {b.n[0] + 2, b.n[1] + 2, b.n[2] + 2}, c[3];
  if (!decode(t_, lo, ext, c)) return;
  const long long Z = zone(b, c[0], c[1], c[2]);
  R* W = fields<R>(work, b);
  const R* p = W + 4 * b.vs;
  R f = R(0);
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const R* un = W + (1 + d) * b.vs;
    const long long s = b.s[d];
    const long long sh = is_nonneg(p[Z + s] - p[Z - s]) ? s : -s;
    f = dmax(f, dmax(flat_tilde(p, un, Z, s), flat_tilde(p, un, Z - sh, s)));
  }
  W[FLD_CHI * b.vs + Z] = f;
}

// out-of-line copy for the persistent kernel
template <typename R>
__device__ __noinline__ void b_flatten(const TableView& tv, const int blk_, const DevBox* boxes, unsigned char* work) {
  body_flatten<R>(tv, blk_, boxes, work);
}

template <typename R>
__global__ void __launch_bounds__(256) k_flatten(TableView tv, const DevBox* __restrict__ boxes, unsigned char* __restrict__ work) {
  body_flatten<R>(tv, blockIdx.x, boxes, work);
}

// ------------------------------------------------------------- PPM + tracing
// van Leer limited slope at a0 (CW84 eq. 1.8); the sign test and the minimum
// run on the integer pipe (magnitudes order like their bit patterns).
template <typename R>
__device__ __forceinline__ R vl_slope(R am, R a0, R ap) {
  const R dl = a0 - am, dr = ap - a0;
  if (!same_sign(dl, dr)) return R(0);
  const R dc = R(0.5) * (ap - am);
  auto m = dbits(fabs(dc));
  m = min(m, dbits(R(2) * fabs(dl)));
  m = min(m, dbits(R(2) * fabs(dr)));
  return copysign(from_bits(m), dc);
}

template <>
__device__ __forceinline__ float vl_slope<float>(float am, float a0, float ap) {
  const float dl = a0 - am, dr = ap - a0;
  if (!same_sign(dl, dr)) return 0.0f;
  const float dc = 0.5f * (ap - am);
  return copysignf(fminf(fabsf(dc), fminf(2.0f * fabsf(dl), 2.0f * fabsf(dr))), dc);
}

// FP64 form: the halving and doublings are exponent changes of the bit
// patterns and the sign tests and minimum are integer comparisons, all on
// 32-bit halves (a double's sign, exponent and top mantissa bits sit in its
// high word), so the FP64 pipe only sees the three subtractions.  A changed
// exponent is exact only while the number and its result stay normal;
// differences near the subnormal range (numerical tails ahead of a front decay
// that far) or the overflow threshold take the multiplies instead.
__device__ __forceinline__ bool hw_nonzero(int hi, int lo) { return ((hi & 0x7fffffff) | lo) != 0; }

template <>
__device__ __forceinline__ double vl_slope<double>(double am, double a0, double ap) {
  const double dl = a0 - am, dr = ap - a0;
  const int hl = __double2hiint(dl), ll = __double2loint(dl);
  const int hr = __double2hiint(dr), lr = __double2loint(dr);
  if ((hl ^ hr) < 0 || !hw_nonzero(hl, ll) || !hw_nonzero(hr, lr)) return 0.0;  // not of one sign
  const double sum = ap - am;
  const int hc = __double2hiint(sum), lc = __double2loint(sum);
  const int ec = (hc >> 20) & 0x7ff, el = (hl >> 20) & 0x7ff, er = (hr >> 20) & 0x7ff;
  if (ec < 2 || el < 1 || er < 1 || el > 0x7fd || er > 0x7fd) {
    const double dc = 0.5 * sum;
    return copysign(fmin(fabs(dc), fmin(2.0 * fabs(dl), 2.0 * fabs(dr))), dc);
  }
  constexpr int ONE_EXP = 1 << 20;
  // magnitudes as (high, low) pairs: |sum|/2, 2|dl|, 2|dr|; the smallest wins
  unsigned mh = (unsigned)((hc & 0x7fffffff) - ONE_EXP), ml = (unsigned)lc;
  const unsigned h2 = (unsigned)((hl & 0x7fffffff) + ONE_EXP), l2 = (unsigned)ll;
  if (h2 < mh || (h2 == mh && l2 < ml)) { mh = h2; ml = l2; }
  const unsigned h3 = (unsigned)((hr & 0x7fffffff) + ONE_EXP), l3 = (unsigned)lr;
  if (h3 < mh || (h3 == mh && l3 < ml)) { mh = h3; ml = l3; }
  return __hiloint2double((int)(mh | ((unsigned)hc & 0x80000000u)), (int)ml);  // sign of ap - am
}

// The FP64 slope from its differences dl = a0 - am, dr = ap - a0 and
// sum = ap - am when every exponent involved is in the range where the
// halving and doublings are exponent changes: integer selections only, no
// branch (0 for a zone that is not monotone).
__device__ __forceinline__ double vl_slope_normal(double dl, double dr, double sum) {
  const int hl = __double2hiint(dl), ll = __double2loint(dl);
  const int hr = __double2hiint(dr), lr = __double2loint(dr);
  const int hc = __double2hiint(sum), lc = __double2loint(sum);
  const bool mono = ((hl ^ hr) >= 0) & hw_nonzero(hl, ll) & hw_nonzero(hr, lr);
  constexpr int ONE_EXP = 1 << 20;
  unsigned mh = (unsigned)((hc & 0x7fffffff) - ONE_EXP), ml = (unsigned)lc;
  const unsigned h2 = (unsigned)((hl & 0x7fffffff) + ONE_EXP), l2 = (unsigned)ll;
  const bool t2 = (h2 < mh) | ((h2 == mh) & (l2 < ml));
  mh = t2 ? h2 : mh;
  ml = t2 ? l2 : ml;
  const unsigned h3 = (unsigned)((hr & 0x7fffffff) + ONE_EXP), l3 = (unsigned)lr;
  const bool t3 = (h3 < mh) | ((h3 == mh) & (l3 < ml));
  mh = t3 ? h3 : mh;
  ml = t3 ? l3 : ml;
  return __hiloint2double(mono ? (int)(mh | ((unsigned)hc & 0x80000000u)) : 0, mono ? (int)ml : 0);
}

// Whether a monotone zone's differences leave that exponent range.
__device__ __forceinline__ bool vl_slope_odd(double dl, double dr, double sum) {
  const int hl = __double2hiint(dl), hr = __double2hiint(dr), hc = __double2hiint(sum);
  const bool mono = ((hl ^ hr) >= 0) & hw_nonzero(hl, __double2loint(dl)) & hw_nonzero(hr, __double2loint(dr));
  const int ec = (hc >> 20) & 0x7ff, el = (hl >> 20) & 0x7ff, er = (hr >> 20) & 0x7ff;
  return mono & ((ec < 2) | (el < 1) | (er < 1) | (el > 0x7fd) | (er > 0x7fd));
}

// Limited slopes of the five normal-frame variables of axis D, once per zone
// of [-2, n_D+1] along D and [-1, n] across it.  FP64: per variable the three
// differences first, then one warp-wide choice between the integer-only
// selection and vl_slope (for a warp with a difference near the subnormal or
// overflow range), so that no lane's early exit splits the warp.
template <typename R, int D>
__device__ __forceinline__ void slopes_zone(const DevBox& b, R* __restrict__ W, long long Z) {
  const long long vs = b.vs, s = b.s[D];
  if constexpr (Consts<R>::FP_BOUND) {
#pragma unroll
    for (int m = 0; m < 5; m++) {
      const R* a = W + comp<D>(m) * vs + Z;
      const R am = a[-s], a0 = a[0], ap = a[s];
      const R dl = a0 - am, dr = ap - a0, sum = ap - am;
      R* out = W + (FLD_DQ + 5 * D + m) * vs + Z;
      if (any_in_warp<R>(vl_slope_odd(dl, dr, sum)))
        *out = vl_slope(am, a0, ap);
      else
        *out = vl_slope_normal(dl, dr, sum);
    }
  } else {
#pragma unroll
    for (int m = 0; m < 5; m++) {
      const R* a = W + comp<D>(m) * vs + Z;
      W[(FLD_DQ + 5 * D + m) * vs + Z] = vl_slope(a[-s], a[0], a[s]);
    }
  }
}

// ---------------------------------------- Colella & Sekora (2008) limiter
// Curvature bound of CS08 (C = 1.25).
constexpr double CS_C = 1.25;


// second difference a - 2 b + c, as (a - 2 b) + c (the doubling exact)
template <typename R>
__device__ __forceinline__ R ie_d2(R a, R b, R c) { return ie_add(ie_sub(a, twice_of(b)), c); }

// CS08's limited second difference: when d2 and the neighbouring second
// differences o[] all share a sign, the smallest of |d2| and C |o|, with the
// sign of d2; else zero.
template <typename R, int NO, typename M>
__device__ __forceinline__ R cs_limited_d2(R d2, const R* o, M& mul) {
  R m = fabs(d2);
#pragma unroll
  for (int k = 0; k < NO; k++) {
    if (!same_sign(d2, o[k])) return R(0);
    m = dmin(m, ie_mul(R(CS_C), fabs(o[k]), mul));
  }
  return copysign(m, d2);
}

// Value at the face between zones a0 and a1 (neighbours am, a2): the
// 4th-order interpolant 7/12 (a0 + a1) - 1/12 (am + a2), rebuilt as
// (a0 + a1)/2 - d2_lim/6 from the limited second difference d2 = 3 (a0 - 2v + a1)
// when it does not lie between a0 and a1 (CS08 §2.1; the division by 6 is a
// correctly rounded divide, taken only on that branch).
template <typename R, typename M>
__device__ __forceinline__ R cs_interface(R am, R a0, R a1, R a2, M& mul) {
  R v = ie_sub(ie_mul(R(7.0 / 12.0), ie_add(a0, a1), mul), ie_mul(R(1.0 / 12.0), ie_add(am, a2), mul));
  if (opp_sign(ie_sub(v, a0), ie_sub(a1, v))) {
    const R d2 = ie_mul(R(3), ie_add(ie_sub(a0, twice_of(v)), a1), mul);
    const R o[2] = {ie_d2(am, a0, a1), ie_d2(a0, a1, a2)};
    v = ie_sub(half_of(ie_add(a0, a1)), ie_div(cs_limited_d2<R, 2>(d2, o, mul), R(6)));
  }
  return v;
}

// Interface values of the five normal-frame variables of axis D at the low
// face of each zone of [-2, n_D+1] along D and [-1, n] across it (stored in
// the slope fields, which CS08 does not use).
// (FP64: the products on the integer pipe, the five interfaces redone with
// the FP64 multiply in a lane that flagged -- the same bits)
template <typename R, int D>
__device__ __forceinline__ void cs_faces_zone(const DevBox& b, R* __restrict__ W, long long Z) {
  const long long vs = b.vs, s = b.s[D];
  R v[5];
  IntMul im;
#pragma unroll
  for (int m = 0; m < 5; m++) {
    const R* a = W + comp<D>(m) * vs + Z;
    v[m] = cs_interface(a[-2 * s], a[-s], a[0], a[s], im);
  }
  if constexpr (Consts<R>::FP_BOUND) {
    if (__any_sync(__activemask(), im.bad != 0u)) {
      if (im.bad) {
        InsnMul nm;
#pragma unroll
        for (int m = 0; m < 5; m++) {
          const R* a = W + comp<D>(m) * vs + Z;
          v[m] = cs_interface(a[-2 * s], a[-s], a[0], a[s], nm);
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 5; m++) W[(FLD_DQ + 5 * D + m) * vs + Z] = v[m];
}

// Parabola of zone value a0 (neighbours amm, am, ap, app) between the
// interface values L, Rt: CS08's limiter (§2.2) -- at an extremum of the zone
// or of a neighbour the parabola keeps its shape with its curvature
// 6 (L + Rt - 2 a0) limited by the neighbouring second differences, else the
// CW84 overshoot rule -- then flattening by f.  What a branch reads is formed
// with single IEEE operations, as for cs_interface; the edge values the
// branches then produce feed only continuous stages and take the fast path
// (approximate reciprocal, fused multiply-adds).
template <typename R, bool BLEND = true, typename M>
__device__ __forceinline__ void cs_parabola(R amm, R am, R a0, R ap, R app, R f, R& L, R& Rt, M& mul) {
  const R dL = ie_sub(L, a0), dR = ie_sub(Rt, a0);
  if (!same_sign(dR, ie_sub(a0, L)) || !same_sign(ie_sub(ap, a0), ie_sub(a0, am))) {
    const R d2 = ie_mul(R(6), ie_sub(ie_add(L, Rt), twice_of(a0)), mul);
    const R o[3] = {ie_d2(amm, am, a0), ie_d2(am, a0, ap), ie_d2(a0, ap, app)};
    const R lim = cs_limited_d2<R, 3>(d2, o, mul);
    if (is_pos(fabs(lim))) {
      // lim / d2 in (0, 1]; a true divide when d2 is too small for the
      // approximate reciprocal (subnormal range)
      const R sc = fabs(d2) > R(1e-30) ? lim * nr_rcp(d2) : lim / d2;
      L = a0 + dL * sc;
      Rt = a0 + dR * sc;
    } else {
      L = a0;
      Rt = a0;
    }
  } else if (!dgt(twice_of(fabs(dL)), fabs(dR))) {
    Rt = a0 - R(2) * dL;
  } else if (!dgt(twice_of(fabs(dR)), fabs(dL))) {
    L = a0 - R(2) * dR;
  }
  if (BLEND && is_pos(f)) {
    L = fma(f, a0, (R(1) - f) * L);
    Rt = fma(f, a0, (R(1) - f) * Rt);
  }
}

// Slope stage: van Leer slopes (CW84) or CS08 interface values, per zone.
template <typename R, int LIM>
__device__ __forceinline__ void body_slopes(const TableView& tv, const int blk_, const DevBox* boxes, unsigned char* work) {
  LOCATE_AT(tv, blk_)
  if (!box_uses<R>(b)) return;
  const int d = z_;
  int lo[3] = {-1, -1, -1}, ext[3] = {b.n[0] + 2, b.n[1] + 2, b.n[2] + 2}, c[3];
  lo[d] = -2;
  ext[d] = b.n[d] + 4;
  if (!decode(t_, lo, ext, c)) return;
  const long long Z = zone(b, c[0], c[1], c[2]);
  R* W = fields<R>(work, b);
  if constexpr (LIM == HYDRO_LIMITER_CS08) {
    switch (d) {
      case 0: cs_faces_zone<R, 0>(b, W, Z); break;
      case 1: cs_faces_zone<R, 1>(b, W, Z); break;
      default: cs_faces_zone<R, 2>(b, W, Z); break;
    }
  } else {
    switch (d) {
      case 0: slopes_zone<R, 0>(b, W, Z); break;
      case 1: slopes_zone<R, 1>(b, W, Z); break;
      default: slopes_zone<R, 2>(b, W, Z); break;
    }
  }
}

// out-of-line copy for the persistent kernel
template <typename R, int LIM>
__device__ __noinline__ void b_slopes(const TableView& tv, const int blk_, const DevBox* boxes, unsigned char* work) {
  body_slopes<R, LIM>(tv, blk_, boxes, work);
}

template <typename R, int LIM>
__global__ void __launch_bounds__(256) k_slopes(TableView tv, const DevBox* __restrict__ boxes, unsigned char* __restrict__ work) {
  body_slopes<R, LIM>(tv, blockIdx.x, boxes, work);
}

// Parabola of zone value a0 with neighbours am1, ap1 and limited slopes
// dm1, d0, dp1: interface values (CW84 eq. 1.6), monotonicity limiter
// (eq. 1.10) with its tests on the integer pipe, then flattening by f.
// 4th-order value at the face between zones of values am1, a0 and limited
// slopes dm1, d0 (CW84 eq. 1.6), as (am1 + a0)/2 - (d0 - dm1)/6 with the
// halving exact (on the integer pipe in FP64).
template <typename R>
__device__ __forceinline__ R ppm_face(R am1, R a0, R dm1, R d0) {
  return fma(dm1 - d0, R(1.0 / 6.0), half_of(am1 + a0));
}

// CW84 monotonicity limiter of the parabola of zone value a0 between face
// values L, Rt, then the flattening blend with coefficient f.
// With x = a0 - L and y = Rt - a0 of one sign, CW84's overshoot tests
// dA (a0 - (L + Rt)/2) > dA^2/6 and -dA^2/6 > dA (a0 - (L + Rt)/2), dA = x + y,
// are |x| > 2|y| and |y| > 2|x|; each replaced edge equals the old one on the
// boundary of its test, so the limiter is continuous there.
template <typename R, bool BLEND = true>
__device__ __forceinline__ void cw84_limit(R a0, R f, R& L, R& Rt) {
  const R x = a0 - L, y = Rt - a0;
  if constexpr (Consts<R>::FP_BOUND) {
    // one multiply-add, a0 - 2y or a0 + 2x, for whichever edge is replaced
    const bool ss = same_sign(y, x);
    const bool cl = ss & abs_gt_twice(x, y), cr = ss & !cl & abs_gt_twice(y, x);
    const R t = fma(cl ? R(-2) : R(2), cl ? y : x, a0);
    L = ss ? (cl ? t : L) : a0;
    Rt = ss ? (cr ? t : Rt) : a0;
  } else if (!same_sign(y, x)) {
    L = a0;
    Rt = a0;
  } else if (abs_gt_twice(x, y)) {
    L = a0 - R(2) * y;
  } else if (abs_gt_twice(y, x)) {
    Rt = a0 + R(2) * x;
  }
  if (BLEND && is_pos(f)) {
    L = fma(f, a0, (R(1) - f) * L);
    Rt = fma(f, a0, (R(1) - f) * Rt);
  }
}

template <typename R, bool BLEND = true>
__device__ __forceinline__ void parabola(R am1, R a0, R ap1, R dm1, R d0, R dp1, R f, R& L, R& Rt) {
  L = ppm_face(am1, a0, dm1, d0);
  Rt = ppm_face(a0, ap1, d0, dp1);
  cw84_limit<R, BLEND>(a0, f, L, Rt);
}

// Conserved momenta (normal frame) and total energy of an edge state q, the
// products taken by a multiplication policy.
template <typename R, typename M>
__device__ __forceinline__ void conserved_m(const R* q, R igm1, R* u, M& mul) {
  u[0] = mul(q[0], q[1]);
  u[1] = mul(q[0], q[2]);
  u[2] = mul(q[0], q[3]);
  u[3] = fma(half_of(q[0]), fma(q[3], q[3], fma(q[2], q[2], mul(q[1], q[1]))), mul(q[4], igm1));
}

// Conserved momenta (normal frame) and total energy of a traced edge state,
// stored once so that the Riemann and CTU stages need not rebuild them.
template <typename R, int D>
__device__ __forceinline__ void store_conserved(R* __restrict__ W, long long vs, long long Z, int base, const R* q,
                                                R igm1) {
  W[(base + 4 * D + 0) * vs + Z] = q[0] * q[1];
  W[(base + 4 * D + 1) * vs + Z] = q[0] * q[2];
  W[(base + 4 * D + 2) * vs + Z] = q[0] * q[3];
  W[(base + 4 * D + 3) * vs + Z] = q[4] * igm1 + half_of(q[0]) * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
}

// Characteristic tracing of one zone along one axis (Miller & Colella 2002
// style, R4): zone values a0, limited parabola edges aL, aR of the five
// normal-frame variables (and their dA = aR - aL, c6), zone sound speed cs
// with ic = 1/c and cr = c/rho, dt/dx.  trace_side<1> forms the right-edge
// state (the left state of the zone's high face), trace_side<0> the
// left-edge state, with the products that are not an addend of a fused
// multiply-add taken by a multiplication policy.  Every product is written
// either as a policy multiply or as an explicit fma(), so that the compiler
// has no multiply-add to fuse by choice: the per-stage kernel and the
// persistent kernel's copy of this body then round alike (with products left
// to contraction, the two copies differed by an ulp in a few zones of a long
// Sedov run).
//
// The parabola's dA = aR - aL and a6 = 6 (a0 - (aL + aR)/2) (CW84 §1); the
// factor 6 of a6 is carried by h2 below, so c6 holds a6 / 6.  For a wave of
// speed lambda, sigma = |lambda| dt/dx, the average of the parabola over the
// wave's domain of dependence at an edge is edge -+ h1 (dA -+ h2 c6) with
// h1 = sigma / 2 and h2 = 6 (1 - 2 sigma / 3) = 6 - 4 sigma.
template <typename R>
__device__ __forceinline__ void parabola_coeffs(const R* a0, const R* aL, const R* aR, R* dA, R* c6) {
#pragma unroll
  for (int m = 0; m < 5; m++) {
    dA[m] = aR[m] - aL[m];
    c6[m] = a0[m] - half_of(aL[m] + aR[m]);
  }
}

template <int SIDE, typename R, typename M>
__device__ __forceinline__ void trace_side(const R* a0, const R* aL, const R* aR, const R* dA, const R* c6, R cs, R ic,
                                           R cr, R dtdx, R* out, M& mul) {
  const R rho = a0[0], u = a0[1];
  const R rc = mul(rho, half_of(ic));  // rho / 2c
  const R ic2 = mul(ic, ic);           // 1 / c^2
  const R i2c2 = half_of(ic2);         // 1 / 2c^2
  const R c2 = mul(cs, cs);
  const R lm = u - cs, lp = u + cs;
  const R hdt = half_of(dtdx), fdt = mul(R(4), dtdx);
  if constexpr (SIDE == 1) {
    // right edge: waves with lambda > 0; the fastest (u+c) supplies the reference state
    if (is_pos(lp)) {
      R h1 = mul(lp, hdt), h2 = fma(-lp, fdt, R(6));
      R ref[5];
#pragma unroll
      for (int m = 0; m < 5; m++) ref[m] = fma(-h1, fma(-h2, c6[m], dA[m]), aR[m]);
      R bm = R(0), b0 = R(0);
      out[2] = ref[2];
      out[3] = ref[3];
      const bool wm = is_pos(lm), w0 = is_pos(u);
      if (any_in_warp<R>(wm)) {
        h1 = mul(lm, hdt); h2 = fma(-lm, fdt, R(6));
        const R du = ref[1] - fma(-h1, fma(-h2, c6[1], dA[1]), aR[1]);
        const R dp = ref[4] - fma(-h1, fma(-h2, c6[4], dA[4]), aR[4]);
        if (wm) bm = fma(i2c2, dp, mul(-rc, du));
      }
      if (any_in_warp<R>(w0)) {
        h1 = mul(u, hdt); h2 = fma(-u, fdt, R(6));
        const R dr = ref[0] - fma(-h1, fma(-h2, c6[0], dA[0]), aR[0]);
        const R dp = ref[4] - fma(-h1, fma(-h2, c6[4], dA[4]), aR[4]);
        if (w0) {
          b0 = fma(-ic2, dp, dr);
          out[2] = fma(-h1, fma(-h2, c6[2], dA[2]), aR[2]);
          out[3] = fma(-h1, fma(-h2, c6[3], dA[3]), aR[3]);
        }
      }
      out[0] = ref[0] - (bm + b0);
      out[1] = fma(cr, bm, ref[1]);
      out[4] = fma(-c2, bm, ref[4]);
    } else {
#pragma unroll
      for (int m = 0; m < 5; m++) out[m] = a0[m];
    }
    if (dgt(R(SMALL_DENS), out[0])) out[0] = R(SMALL_DENS);
    if (dgt(R(SMALL_PRES), out[4])) out[4] = R(SMALL_PRES);
  } else {
    // left edge: waves with lambda < 0; the fastest (u-c) supplies the reference state
    if (is_neg(lm)) {
      R h1 = mul(-lm, hdt), h2 = fma(lm, fdt, R(6));
      R ref[5];
#pragma unroll
      for (int m = 0; m < 5; m++) ref[m] = fma(h1, fma(h2, c6[m], dA[m]), aL[m]);
      R bp = R(0), b0 = R(0);
      out[2] = ref[2];
      out[3] = ref[3];
      const bool wp = is_neg(lp), w0 = is_neg(u);
      if (any_in_warp<R>(wp)) {
        h1 = mul(-lp, hdt); h2 = fma(lp, fdt, R(6));
        const R du = ref[1] - fma(h1, fma(h2, c6[1], dA[1]), aL[1]);
        const R dp = ref[4] - fma(h1, fma(h2, c6[4], dA[4]), aL[4]);
        if (wp) bp = fma(i2c2, dp, mul(rc, du));
      }
      if (any_in_warp<R>(w0)) {
        h1 = mul(-u, hdt); h2 = fma(u, fdt, R(6));
        const R dr = ref[0] - fma(h1, fma(h2, c6[0], dA[0]), aL[0]);
        const R dp = ref[4] - fma(h1, fma(h2, c6[4], dA[4]), aL[4]);
        if (w0) {
          b0 = fma(-ic2, dp, dr);
          out[2] = fma(h1, fma(h2, c6[2], dA[2]), aL[2]);
          out[3] = fma(h1, fma(h2, c6[3], dA[3]), aL[3]);
        }
      }
      out[0] = ref[0] - (b0 + bp);
      out[1] = fma(-cr, bp, ref[1]);
      out[4] = fma(-c2, bp, ref[4]);
    } else {
#pragma unroll
      for (int m = 0; m < 5; m++) out[m] = a0[m];
    }
    if (dgt(R(SMALL_DENS), out[0])) out[0] = R(SMALL_DENS);
    if (dgt(R(SMALL_PRES), out[4])) out[4] = R(SMALL_PRES);
  }
}

// Both edge states in turn, handed to sink(side, q[5]) as soon as each is
// formed (plain products: the FP32 kernels and the form that forms 1/c here).
template <typename R, typename Sink>
__device__ __forceinline__ void trace_edges(const R* a0, const R* aL, const R* aR, R cs, R ic, R cr, R dtdx,
                                            Sink&& sink) {
  R dA[5], c6[5], out[5];
  parabola_coeffs(a0, aL, aR, dA, c6);
  PlainMul pm;
  trace_side<1>(a0, aL, aR, dA, c6, cs, ic, cr, dtdx, out, pm);
  sink(1, out);
  trace_side<0>(a0, aL, aR, dA, c6, cs, ic, cr, dtdx, out, pm);
  sink(0, out);
}

// The same with 1/c and c/rho formed here.
template <typename R, typename Sink>
__device__ __forceinline__ void trace_edges(const R* a0, const R* aL, const R* aR, R cs, R dtdx, Sink&& sink) {
  trace_edges(a0, aL, aR, cs, nr_rcp(cs), cs * nr_rcp(a0[0]), dtdx, sink);
}

// The limited parabolas (edges aL, aR) of the five normal-frame variables
// of zone Z along D, flattened by f when BLEND.
template <typename R, int D, int LIM, bool BLEND, typename M>
__device__ __forceinline__ void zone_parabolas_m(const R* __restrict__ W, long long vs, long long s, long long Z, R f,
                                                 R* a0, R* aL, R* aR, M& mul) {
#pragma unroll
  for (int m = 0; m < 5; m++) {
    const R* a = W + comp<D>(m) * vs + Z;
    const R* dq = W + (FLD_DQ + 5 * D + m) * vs + Z;
    a0[m] = a[0];
    if constexpr (LIM == HYDRO_LIMITER_CS08) {
      aL[m] = dq[0];
      aR[m] = dq[s];
      cs_parabola<R, BLEND>(a[-2 * s], a[-s], a[0], a[s], a[2 * s], f, aL[m], aR[m], mul);
    } else {
      parabola<R, BLEND>(a[-s], a[0], a[s], dq[-s], dq[0], dq[s], f, aL[m], aR[m]);
    }
  }
}

// (FP64 CS08: the limiter's products on the integer pipe, the five parabolas
// redone with the FP64 multiply in a lane that flagged -- the same bits)
template <typename R, int D, int LIM, bool BLEND>
__device__ __forceinline__ void zone_parabolas(const R* __restrict__ W, long long vs, long long s, long long Z, R f,
                                               R* a0, R* aL, R* aR) {
  IntMul im;
  zone_parabolas_m<R, D, LIM, BLEND>(W, vs, s, Z, f, a0, aL, aR, im);
  if constexpr (Consts<R>::FP_BOUND && LIM == HYDRO_LIMITER_CS08) {
    if (__any_sync(__activemask(), im.bad != 0u)) {
      if (im.bad) {
        InsnMul nm;
        zone_parabolas_m<R, D, LIM, BLEND>(W, vs, s, Z, f, a0, aL, aR, nm);
      }
    }
  }
}

// One FP64 edge state of a zone along D (and its conserved form) formed with
// integer-pipe products, recomputed with the FP64 multiply in a lane that
// flagged, and stored.
template <int SIDE, bool IM, typename R>
__device__ __forceinline__ void trace_store_side(R* __restrict__ W, long long vs, long long Z, int D, const R* a0,
                                                 const R* aL, const R* aR, const R* dA, const R* c6, R cs, R ic, R cr,
                                                 R dtdx, R igm1) {
  R out[5], u[4];
  IntMul im;
  if constexpr (IM) {
    trace_side<SIDE>(a0, aL, aR, dA, c6, cs, ic, cr, dtdx, out, im);
    conserved_m(out, igm1, u, im);
  } else {  // the FP64 multiply throughout (the same bits)
    PlainMul pm;
    trace_side<SIDE>(a0, aL, aR, dA, c6, cs, ic, cr, dtdx, out, pm);
    conserved_m(out, igm1, u, pm);
  }
  if (IM && __any_sync(__activemask(), im.bad != 0u)) {
    if (im.bad) {
      InsnMul nm;
      trace_side<SIDE>(a0, aL, aR, dA, c6, cs, ic, cr, dtdx, out, nm);
      conserved_m(out, igm1, u, nm);
    }
  }
#pragma unroll
  for (int m = 0; m < 5; m++) W[((SIDE ? FLD_QP : FLD_QM) + 5 * D + m) * vs + Z] = out[m];
#pragma unroll
  for (int j = 0; j < 4; j++) W[((SIDE ? FLD_UP : FLD_UM) + 4 * D + j) * vs + Z] = u[j];
}

template <typename R, int D, int LIM, bool IM = true>
__device__ __forceinline__ void trace_zone(const DevBox& b, R* __restrict__ W, long long Z, R dtdx) {
  const long long vs = b.vs, s = b.s[D];
  const R igm1 = Consts<R>::igm1(b);
  const R f = W[FLD_CHI * vs + Z];
  R a0[5], aL[5], aR[5];
  // FP64: a warp none of whose zones is flattened takes the copy without the
  // flattening blend (the compiler predicates a blend guarded per zone, which
  // then issues in every zone)
  if (Consts<R>::FP_BOUND && !any_in_warp<R>(is_pos(f)))
    zone_parabolas<R, D, LIM, false>(W, vs, s, Z, f, a0, aL, aR);
  else
    zone_parabolas<R, D, LIM, true>(W, vs, s, Z, f, a0, aL, aR);
  const R cs = W[FLD_C * vs + Z];
  auto sink = [&](int side, const R* out) {
#pragma unroll
    for (int m = 0; m < 5; m++) W[((side ? FLD_QP : FLD_QM) + 5 * D + m) * vs + Z] = out[m];
    if constexpr (Consts<R>::STORE_CONSERVED) store_conserved<R, D>(W, vs, Z, side ? FLD_UP : FLD_UM, out, igm1);
  };
  if constexpr (Consts<R>::PRIM_RECIPROCALS) {
    // FP64: each edge state and its conserved form with the products on the
    // integer pipe; a warp with a flagged lane redoes that side with the FP64
    // multiply (the same bits) before it is stored (IM = false: the FP64
    // multiply throughout, the persistent kernel's bodies)
    const R ic = W[FLD_IC * vs + Z], cr = W[FLD_CR * vs + Z];
    R dA[5], c6[5];
    parabola_coeffs(a0, aL, aR, dA, c6);
    trace_store_side<1, IM>(W, vs, Z, D, a0, aL, aR, dA, c6, cs, ic, cr, dtdx, igm1);
    trace_store_side<0, IM>(W, vs, Z, D, a0, aL, aR, dA, c6, cs, ic, cr, dtdx, igm1);
  } else {
    trace_edges(a0, aL, aR, cs, dtdx, sink);
  }
}

template <typename R, int LIM, bool IM = true>
__device__ __forceinline__ void body_trace(const TableView& tv, const int blk_, const DevBox* boxes, const BoxRt* rt, unsigned char* work) {
  LOCATE_AT(tv, blk_)
  if (!box_uses<R>(b)) return;
  int lo[3] = {-1, -1, -1}, ext[3] = {b.n[0] + 2, b.n[1] + 2, b.n[2] + 2}, c[3];
  if (!decode(t_, lo, ext, c)) return;
  const long long Z = zone(b, c[0], c[1], c[2]);
  R* W = fields<R>(work, b);
  const BoxRt& r = rt[bi];
  switch (z_) {
    case 0: trace_zone<R, 0, LIM, IM>(b, W, Z, Consts<R>::dtdx(b, r, 0)); break;
    case 1: trace_zone<R, 1, LIM, IM>(b, W, Z, Consts<R>::dtdx(b, r, 1)); break;
    default: trace_zone<R, 2, LIM, IM>(b, W, Z, Consts<R>::dtdx(b, r, 2)); break;
  }
}

// out-of-line copy for the persistent kernel (FP64 multiply instruction)
template <typename R, int LIM>
__device__ __noinline__ void b_trace(const TableView& tv, const int blk_, const DevBox* boxes, const BoxRt* rt, unsigned char* work) {
  body_trace<R, LIM, false>(tv, blk_, boxes, rt, work);
}

// Registers capped at 128 (4 blocks of 128 threads per SM): the integer-pipe
// products of the FP64 tracing want 154, and with that many the kernel was
// measured 8 % slower (12.29 against 11.28 ms at 256^3; 112 registers: 11.45).
template <typename R, int LIM>
__global__ void __maxnreg__(128) k_trace(
    TableView tv, const DevBox* __restrict__ boxes, const BoxRt* __restrict__ rt, unsigned char* __restrict__ work) {
  body_trace<R, LIM>(tv, blockIdx.x, boxes, rt, work);
}

// ----------------------------------------------------------------------- HLLC
// Normal-frame states (rho, u_n, u_t1, u_t2, p) with their total energies
// El, Er -> normal-frame flux.
// Toro, Spruce & Speares 1994 with Roe-averaged bounds (Batten et al. 1997),
// Davis bounds when the Roe sound speed is not real.  Only the star state on
// the side of the contact that contains x/t = 0 is formed, as the change
// S_K (U*_K - U_K) of that side's flux written without 1/rho_K.  All square
// roots and reciprocals come from two reciprocal square roots per side
// (1/sqrt(rho), which gives sqrt(rho), and 1/sqrt(gamma p), which gives
// c = sqrt(gamma p) / sqrt(rho)), one square root (Roe sound speed) and three
// reciprocals; wave-speed min/max and sign tests run on the integer pipe in
// FP64.
template <typename R, typename M>
__device__ __forceinline__ void hllc_body(const R* L, R El, R rsl, const R* Rs, R Er, R rsr, R gamma, R gm1, R* F,
                                          M& mul) {
  const R rl = L[0], ul = L[1], vl = L[2], wl = L[3], pl = L[4];
  const R rr = Rs[0], ur = Rs[1], vr = Rs[2], wr = Rs[3], pr = Rs[4];
  // 1/sqrt(rho) of each side: from the caller where SHARE_RSQRT holds
  if constexpr (!Consts<R>::SHARE_RSQRT) {
    rsl = nr_rsqrt(rl);
    rsr = nr_rsqrt(rr);
  }
  // mul(): the products that are not an addend of a fused multiply-add
  const R sl = mul(rl, rsl), sr = mul(rr, rsr);  // sqrt(rho)
  const R gpl = mul(gamma, pl), gpr = mul(gamma, pr);
  const R cl = mul(mul(gpl, nr_rsqrt(gpl, mul)), rsl), cr = mul(mul(gpr, nr_rsqrt(gpr, mul)), rsr);
  const R iw = nr_rcp(sl + sr);
  const R wgr = mul(sr, iw);  // Roe weight of the right state; the left one is 1 - wgr
  const R ut = ul + wgr * (ur - ul);
  const R vt = vl + wgr * (vr - vl);
  const R wt = wl + wgr * (wr - wl);
  // Roe enthalpy: sum of w_K (E_K + p_K) / rho_K = sum of (E_K + p_K) / sqrt(rho_K), times iw
  const R hl = El + pl, hr = Er + pr;
  const R Ht = mul(mul(hl, rsl) + hr * rsr, iw);
  const R ct2 = mul(gm1, Ht - half_of(mul(ut, ut) + vt * vt + wt * wt));
  R SL, SR;
  if (is_pos(ct2)) {
    const R ct = nr_sqrt(ct2, mul);
    SL = dmin(ul - cl, ut - ct);
    SR = dmax(ur + cr, ut + ct);
  } else {
    SL = dmin(ul - cl, ur - cr);
    SR = dmax(ul + cl, ur + cr);
  }
  const R ml = mul(rl, SL - ul), mr = mul(rr, SR - ur);
  const R Ss = mul(pr - pl + ml * ul - mr * ur, nr_rcp(ml - mr));
  const bool left = is_nonneg(Ss);
  const R rK = left ? rl : rr, uK = left ? ul : ur, vK = left ? vl : vr, wK = left ? wl : wr;
  const R pK = left ? pl : pr, SK = left ? SL : SR;
  const R mu = mul(rK, uK), hK = left ? hl : hr;
  F[0] = mu;
  F[1] = mu * uK + pK;
  F[4] = mul(hK, uK);
  const bool supersonic = left ? is_nonneg(SL) : !is_pos(SR);
  if (!supersonic) {
    // F += S_K (U*_K - U_K) with U*_K = rho_K phi (1, S*, v_K, w_K,
    // E_K / rho_K + (S* - u_K)(S* + p_K / (rho_K (S_K - u_K)))),
    // phi = (S_K - u_K) / (S_K - S*) = 1 + g, g = (S* - u_K) / (S_K - S*):
    // U*_K - U_K = (rho_K g, rho_K (phi S* - u_K), ., .,
    //               g (E_K + p_K) + rho_K phi S* (S* - u_K))
    const R dsu = Ss - uK;
    const R g = mul(dsu, nr_rcp(SK - Ss));
    const R phi = R(1) + g;
    const R srk = mul(SK, rK);
    F[0] += srk * g;
    F[1] += srk * (phi * Ss - uK);
    F[4] += SK * (mul(g, hK) + mul(mul(rK, phi), Ss) * dsu);
  }
  // the upwind side's star and outer states share its transverse velocity, so
  // the transverse momentum fluxes are the mass flux times that velocity
  F[2] = mul(F[0], vK);
  F[3] = mul(F[0], wK);
}

// FP64: the products on the integer pipe (IntMul); a warp in which a lane's
// operands fell outside its range recomputes that lane with the FP64 multiply
// (the same bits: both are correctly rounded).  IM = false: the FP64 multiply
// throughout, the same bits again.
template <typename R, bool IM = true>
__device__ __forceinline__ void hllc(const R* L, R El, R rsl, const R* Rs, R Er, R rsr, R gamma, R gm1, R* F) {
  if constexpr (!IM) {
    PlainMul pm;
    hllc_body(L, El, rsl, Rs, Er, rsr, gamma, gm1, F, pm);
    return;
  }
  IntMul im;
  hllc_body(L, El, rsl, Rs, Er, rsr, gamma, gm1, F, im);
  if constexpr (Consts<R>::FP_BOUND) {
    if (__any_sync(__activemask(), im.bad != 0u)) {
      if (im.bad) {
        InsnMul nm;
        hllc_body(L, El, rsl, Rs, Er, rsr, gamma, gm1, F, nm);
      }
    }
  }
}

// ------------------------------------------------- two-shock Riemann solver
// Colella & Glaz (1985) two-shock approximation on normal-frame states
// (rho, u_n, u_t1, u_t2, p) -> normal-frame Godunov flux.  Both nonlinear
// waves follow their shock Hugoniot: across the wave of side K the velocity
// changes by (p - p_K) / W_K(p), W_K^2 = rho_K ((gamma+1)/2 p + (gamma-1)/2 p_K).
// p* solves the velocity balance by Newton's method from the acoustic guess
// (floored at the pressure floor; stops when a step is at most TOL p*, at
// most MAXIT steps), u* is the mean of the two sides' star velocities, the
// star density follows the Hugoniot, 1/rho* = 1/rho_K - (p* - p_K)/W_K^2.
// The state at x/t = 0 is taken on the side of the contact that holds it
// (u* = 0: left), across a shock by its speed, across a rarefaction by
// linear interpolation in x/t between head and tail.
template <typename R>
struct TwoShock;
template <>
struct TwoShock<double> {
  static constexpr double TOL = 1e-12;
  static constexpr int MAXIT = 40;
};
template <>
struct TwoShock<float> {
  static constexpr float TOL = 2e-6f;
  static constexpr int MAXIT = 20;
};

template <typename R, typename M>
__device__ __forceinline__ void two_shock_body(const R* L, const R* Rs, R gamma, R igm1, R* F, M& mul) {
  // mul(): the products that are not an addend of a fused multiply-add
  const R rl = L[0], ul = L[1], pl = L[4];
  const R rr = Rs[0], ur = Rs[1], pr = Rs[4];
  const R hp = half_of(gamma + R(1)), hm = half_of(gamma - R(1));
  const R al = mul(rl, hp), bl = mul(mul(rl, hm), pl);  // W_L^2 = al p + bl
  const R ar = mul(rr, hp), br = mul(mul(rr, hm), pr);
  const R Cl = nr_sqrt(mul(mul(gamma, pl), rl), mul), Cr = nr_sqrt(mul(mul(gamma, pr), rr), mul);  // impedances
  R p = mul(mul(Cr, pl) + Cl * pr + mul(Cl, Cr) * (ul - ur), nr_rcp(Cl + Cr));
  p = dmax(p, R(SMALL_PRES));
  for (int it = 0; it < TwoShock<R>::MAXIT; it++) {
    const R iwl = nr_rsqrt(al * p + bl, mul), iwr = nr_rsqrt(ar * p + br, mul);  // 1 / W
    const R dpl = p - pl, dpr = p - pr;
    const R f = dpl * iwl + mul(dpr, iwr) + (ur - ul);
    // d/dp (p - p_K) / W_K = (1 - (p - p_K) (a_K / 2) / W_K^2) / W_K
    const R dl = mul(R(1) - mul(mul(dpl, half_of(al)), iwl) * iwl, iwl);
    const R dr = mul(R(1) - mul(mul(dpr, half_of(ar)), iwr) * iwr, iwr);
    const R pn = dmax(p - f * nr_rcp(dl + dr), R(SMALL_PRES));
    const R step = fabs(pn - p);
    p = pn;
    if (!dgt(step, mul(R(TwoShock<R>::TOL), p))) break;
  }
  const R iwl = nr_rsqrt(al * p + bl, mul), iwr = nr_rsqrt(ar * p + br, mul);
  const R us = half_of((ul - (p - pl) * iwl) + (ur + (p - pr) * iwr));
  const bool left = is_nonneg(us);
  const R rk = left ? rl : rr, uk = left ? ul : ur, pk = left ? pl : pr;
  const R vk = left ? L[2] : Rs[2], wk = left ? L[3] : Rs[3];
  const R iwk = left ? iwl : iwr, w2k = left ? al * p + bl : ar * p + br;
  const R suk = left ? uk : -uk;  // the side's wave moves with u - c (left) or u + c (right)
  const R irk = nr_rcp(rk);
  const R irs = irk - mul(p - pk, iwk) * iwk;  // 1 / rho*
  // speeds of the side's wave head and tail relative to x/t = 0, positive
  // while they are on the side's own half
  R head, tail;
  if (dgt(p, pk)) {
    head = mul(w2k, iwk) * irk - suk;  // shock: |S - u_K| = W_K / rho_K
    tail = head;
  } else {
    const R gpk = mul(mul(gamma, pk), irk), gps = mul(mul(gamma, p), irs);
    head = mul(gpk, nr_rsqrt(gpk, mul)) - suk;
    tail = mul(gps, nr_rsqrt(gps, mul)) - (left ? us : -us);
  }
  R q0, q1, q4;
  if (!is_pos(head)) {
    q0 = rk; q1 = uk; q4 = pk;            // the wave has left x/t = 0 behind
  } else if (is_nonneg(tail)) {
    q0 = nr_rcp(irs); q1 = us; q4 = p;    // star state
  } else {
    const R a = mul(head, nr_rcp(head - tail));  // x/t = 0 inside the fan
    q0 = mul(R(1) - a, rk) + a * nr_rcp(irs);
    q1 = mul(R(1) - a, uk) + a * us;
    q4 = mul(R(1) - a, pk) + a * p;
  }
  const R mu = mul(q0, q1);
  const R E = mul(q4, igm1) + half_of(q0) * (mul(q1, q1) + vk * vk + wk * wk);
  F[0] = mu;
  F[1] = mu * q1 + q4;
  F[2] = mul(mu, vk);
  F[3] = mul(mu, wk);
  F[4] = mul(E + q4, q1);
}

// FP64 products on the integer pipe, recomputed with the FP64 multiply in a
// flagged lane, as for HLLC (IM = false: the FP64 multiply throughout).
template <typename R, bool IM = true>
__device__ __forceinline__ void two_shock(const R* L, const R* Rs, R gamma, R igm1, R* F) {
  if constexpr (!IM) {
    PlainMul pm;
    two_shock_body(L, Rs, gamma, igm1, F, pm);
    return;
  }
  IntMul im;
  two_shock_body(L, Rs, gamma, igm1, F, im);
  if constexpr (Consts<R>::FP_BOUND) {
    if (__any_sync(__activemask(), im.bad != 0u)) {
      if (im.bad) {
        InsnMul nm;
        two_shock_body(L, Rs, gamma, igm1, F, nm);
      }
    }
  }
}

// The handle's Riemann solver.  El, Er: total energies of the states and rsl,
// rsr their 1/sqrt(rho) (HLLC uses them; the two-shock flux is built from the
// sampled state alone).
template <typename R, int RS, bool IM = true>
__device__ __forceinline__ void riemann(const R* L, R El, R rsl, const R* Rs, R Er, R rsr, R gamma, R gm1, R igm1,
                                        R* F) {
  if constexpr (RS == HYDRO_RIEMANN_TWO_SHOCK) two_shock<R, IM>(L, Rs, gamma, igm1, F);
  else hllc<R, IM>(L, El, rsl, Rs, Er, rsr, gamma, gm1, F);
}

template <typename R>
__device__ __forceinline__ void conserved_of(const R* q, R igm1, R* u) {
  u[0] = q[0] * q[1];
  u[1] = q[0] * q[2];
  u[2] = q[0] * q[3];
  u[3] = q[4] * igm1 + half_of(q[0]) * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
}

// The two states of the D-face at zone Z: primitive q (5) and conserved
// momenta + energy u (4) of the left (zone Z - s_D) and right (zone Z) sides;
// the conserved form is loaded (FP64) or rebuilt from q (FP32).
template <typename R, int D>
__device__ __forceinline__ void load_face_states(const R* __restrict__ W, long long vs, long long Z, long long sD,
                                                 R igm1, R* qL, R* uL, R* qR, R* uR) {
#pragma unroll
  for (int m = 0; m < 5; m++) {
    qL[m] = W[(FLD_QP + 5 * D + m) * vs + Z - sD];
    qR[m] = W[(FLD_QM + 5 * D + m) * vs + Z];
  }
  if constexpr (Consts<R>::STORE_CONSERVED) {
#pragma unroll
    for (int j = 0; j < 4; j++) {
      uL[j] = W[(FLD_UP + 4 * D + j) * vs + Z - sD];
      uR[j] = W[(FLD_UM + 4 * D + j) * vs + Z];
    }
  } else {
    conserved_of(qL, igm1, uL);
    conserved_of(qR, igm1, uR);
  }
}

template <typename R, int D>
__device__ __forceinline__ void store_flux(R* __restrict__ dst, long long vs, long long Z, const R* Fn) {
#pragma unroll
  for (int m = 0; m < 5; m++) dst[comp<D>(m) * vs + Z] = Fn[m];
}

template <typename R, int D, int RS, bool IM = true>
__device__ __forceinline__ void riemann_face(const DevBox& b, R* __restrict__ W, long long Z) {
  R qL[5], qR[5], uL[4], uR[4], Fn[5];
  load_face_states<R, D>(W, b.vs, Z, b.s[D], Consts<R>::igm1(b), qL, uL, qR, uR);
  const bool own = RS == HYDRO_RIEMANN_HLLC && Consts<R>::SHARE_RSQRT;
  const R rsl = own ? nr_rsqrt(qL[0]) : R(0);
  const R rsr = own ? nr_rsqrt(qR[0]) : R(0);
  riemann<R, RS, IM>(qL, uL[3], rsl, qR, uR[3], rsr, Consts<R>::gamma(b), Consts<R>::gm1(b), Consts<R>::igm1(b), Fn);
  store_flux<R, D>(W + (FLD_F0 + 5 * D) * b.vs, b.vs, Z, Fn);
}

template <typename R, int RS, bool IM = true>
__device__ __forceinline__ void body_riemann(const TableView& tv, const int blk_, const DevBox* boxes, unsigned char* work) {
  LOCATE_AT(tv, blk_)
  if (!box_uses<R>(b)) return;
  const int d = z_;
  int lo[3] = {-1, -1, -1}, ext[3] = {b.n[0] + 2, b.n[1] + 2, b.n[2] + 2}, c[3];
  lo[d] = 0;
  ext[d] = b.n[d] + 1;
  if (!decode(t_, lo, ext, c)) return;
  const long long Z = zone(b, c[0], c[1], c[2]);
  R* W = fields<R>(work, b);
  switch (d) {
    case 0: riemann_face<R, 0, RS, IM>(b, W, Z); break;
    case 1: riemann_face<R, 1, RS, IM>(b, W, Z); break;
    default: riemann_face<R, 2, RS, IM>(b, W, Z); break;
  }
}

// out-of-line copy for the persistent kernel (FP64 products by the multiply
// instruction: the integer-pipe ones were measured slower there)
template <typename R, int RS>
__device__ __noinline__ void b_riemann(const TableView& tv, const int blk_, const DevBox* boxes, unsigned char* work) {
  body_riemann<R, RS, false>(tv, blk_, boxes, work);
}

// Registers capped at 80 (more resident warps, some spills): the FP64 solver
// took 5.61 instead of 5.80 ms at 256^3 against the 100 the compiler takes
// uncapped (96: 5.78 ms).
template <typename R, int RS>
__global__ void __maxnreg__(80) k_riemann(
    TableView tv, const DevBox* __restrict__ boxes, unsigned char* __restrict__ work) {
  body_riemann<R, RS>(tv, blockIdx.x, boxes, work);
}

// ------------------------------------------------------------ CTU corrections
// Face state of zone Z (primitive q and conserved momenta + energy u, normal
// frame of D) minus fac_t * (flux difference across zone Z along stride s_t)
// for each term t, back to primitive.  A result with rho <= 0 or p <= 0 keeps
// the uncorrected state.  Returns the total energy of the state that is kept
// and, in rs, 1/sqrt(rho) of it where SHARE_RSQRT holds: one reciprocal square
// root gives both the 1/rho of the conversion (its square) and what the
// Riemann solver needs (else rs is 0 and the solver forms its own).
// Flux differences across zone Z along stride st[t] of the fluxes Fb[t], per
// normal-frame variable m: dlt[t][m].
template <typename R, int D, int NT>
__device__ __forceinline__ void flux_deltas(const R* const* Fb, const long long* st, long long vs, long long Z,
                                            R (*dlt)[5]) {
#pragma unroll
  for (int m = 0; m < 5; m++) {
    const long long off = comp<D>(m) * vs + Z;
#pragma unroll
    for (int t = 0; t < NT; t++) dlt[t][m] = Fb[t][off + st[t]] - Fb[t][off];
  }
}

// The correction itself, from the flux differences (see correct).
template <typename R, int NT, typename M>
__device__ __forceinline__ R correct_body(R* q, const R* u, const R (*dlt)[5], const R* fac, R gm1, R igm1, R& rs,
                                          M& mul) {
  R U[5] = {q[0], u[0], u[1], u[2], u[3]};
#pragma unroll
  for (int m = 0; m < 5; m++) {
#pragma unroll
    for (int t = 0; t < NT; t++) U[m] = U[m] - fac[t] * dlt[t][m];
  }
  if (is_pos(U[0])) {
    const R r = Consts<R>::SHARE_RSQRT ? nr_rsqrt(U[0], mul) : R(0);
    const R ir = Consts<R>::SHARE_RSQRT ? mul(r, r) : nr_rcp(U[0]);
    const R uu = mul(U[1], ir), v = mul(U[2], ir), w = mul(U[3], ir);
    const R kin = half_of(mul(U[1], uu) + U[2] * v + U[3] * w);
    const R p = mul(gm1, U[4] - kin);
    if (is_pos(p)) {
      q[0] = U[0];
      q[1] = uu;
      q[2] = v;
      q[3] = w;
      rs = r;
      if (dgt(R(SMALL_PRES), p)) {  // floored pressure: the energy follows it
        q[4] = R(SMALL_PRES);
        return q[4] * igm1 + kin;
      }
      q[4] = p;
      return U[4];
    }
  }
  rs = Consts<R>::SHARE_RSQRT ? nr_rsqrt(q[0], mul) : R(0);
  return u[3];
}

// FP64 products on the integer pipe, as in hllc: a lane flagged there redoes
// its correction from the uncorrected state with the FP64 multiply.
template <typename R, int NT, bool IM = true>
__device__ __forceinline__ R correct_by(R* q, const R* u, const R (*dlt)[5], const R* fac, R gm1, R igm1, R& rs) {
  if constexpr (!IM) {
    PlainMul pm;
    return correct_body<R, NT>(q, u, dlt, fac, gm1, igm1, rs, pm);
  } else if constexpr (Consts<R>::FP_BOUND) {
    R qc[5] = {q[0], q[1], q[2], q[3], q[4]};
    IntMul im;
    R E = correct_body<R, NT>(qc, u, dlt, fac, gm1, igm1, rs, im);
    if (__any_sync(__activemask(), im.bad != 0u)) {
      if (im.bad) {
#pragma unroll
        for (int m = 0; m < 5; m++) qc[m] = q[m];
        InsnMul nm;
        E = correct_body<R, NT>(qc, u, dlt, fac, gm1, igm1, rs, nm);
      }
    }
#pragma unroll
    for (int m = 0; m < 5; m++) q[m] = qc[m];
    return E;
  } else {
    IntMul im;
    return correct_body<R, NT>(q, u, dlt, fac, gm1, igm1, rs, im);
  }
}

template <typename R, int D, int NT, bool IM = true>
__device__ __forceinline__ R correct(R* q, const R* u, const R* const* Fb, const long long* st, const R* fac,
                                     long long vs, long long Z, R gm1, R igm1, R& rs) {
  R dlt[NT][5];
  flux_deltas<R, D, NT>(Fb, st, vs, Z, dlt);
  return correct_by<R, NT, IM>(q, u, dlt, fac, gm1, igm1, rs);
}

constexpr int pair_slot(int d, int e) { return 2 * d + (e > d ? e - 1 : e); }

// Stage 1 of the corner transport: the D-face at zone Z corrected by the
// flux difference along one transverse axis T (the ordered pair (D, T)), for
// each T in {E, F} the face carries: the face's two states are loaded once
// for both pairs.
template <typename R, int D, int T, int RS, bool IM = true>
__device__ __forceinline__ void ctu1_pair(const DevBox& b, R* __restrict__ W, long long Z, const BoxRt& rt,
                                          const R* qL0, const R* uL, const R* qR0, const R* uR) {
  const long long vs = b.vs, sD = b.s[D];
  const R gamma = Consts<R>::gamma(b), gm1 = Consts<R>::gm1(b), igm1 = Consts<R>::igm1(b);
  R qL[5], qR[5], Fn[5];
#pragma unroll
  for (int m = 0; m < 5; m++) {
    qL[m] = qL0[m];
    qR[m] = qR0[m];
  }
  const R* Fb[1] = {W + (FLD_F0 + 5 * T) * vs};
  const long long st[1] = {b.s[T]};
  const R fac[1] = {Consts<R>::dtdx3(b, rt, T)};
  R rsl, rsr;
  const R EL = correct<R, D, 1, IM>(qL, uL, Fb, st, fac, vs, Z - sD, gm1, igm1, rsl);
  const R ER = correct<R, D, 1, IM>(qR, uR, Fb, st, fac, vs, Z, gm1, igm1, rsr);
  riemann<R, RS, IM>(qL, EL, rsl, qR, ER, rsr, gamma, gm1, igm1, Fn);
  store_flux<R, D>(W + (FLD_F1 + 5 * pair_slot(D, T)) * vs, vs, Z, Fn);
}

// One thread per D-face and transverse axis T (the ordered pair (D, T), work
// item z = its pair slot): faces [0, n_D] along D, [0, n_T) along T and
// [-1, n] along the remaining axis.  (Both pairs of a face in one thread load
// its two states once, but with the products on the integer pipe the kernel
// is bound by latency rather than by its loads: one pair per thread, more
// threads with fewer registers, measured 3.6 % faster.)
template <typename R, int D, int T, int RS, bool IM>
__device__ __forceinline__ void ctu1_one_pair(const DevBox& b, R* __restrict__ W, long long t, const BoxRt& rt) {
  constexpr int U = 3 - D - T;
  int lo[3], ext[3], c[3];
  lo[D] = 0;
  ext[D] = b.n[D] + 1;
  lo[T] = 0;
  ext[T] = b.n[T];
  lo[U] = -1;
  ext[U] = b.n[U] + 2;
  if (!decode(t, lo, ext, c)) return;
  const long long Z = zone(b, c[0], c[1], c[2]);
  R qL[5], qR[5], uL[4], uR[4];
  load_face_states<R, D>(W, b.vs, Z, b.s[D], Consts<R>::igm1(b), qL, uL, qR, uR);
  ctu1_pair<R, D, T, RS, IM>(b, W, Z, rt, qL, uL, qR, uR);
}
template <typename R, int RS, bool IM = true>
__device__ __forceinline__ void body_ctu1(const TableView& tv, const int blk_, const DevBox* boxes, const BoxRt* rt, unsigned char* work) {
  LOCATE_AT(tv, blk_)
  if (!box_uses<R>(b)) return;
  R* W = fields<R>(work, b);
  const BoxRt& rtb = rt[bi];
  switch (z_) {
    case 0: ctu1_one_pair<R, 0, 1, RS, IM>(b, W, t_, rtb); break;
    case 1: ctu1_one_pair<R, 0, 2, RS, IM>(b, W, t_, rtb); break;
    case 2: ctu1_one_pair<R, 1, 0, RS, IM>(b, W, t_, rtb); break;
    case 3: ctu1_one_pair<R, 1, 2, RS, IM>(b, W, t_, rtb); break;
    case 4: ctu1_one_pair<R, 2, 0, RS, IM>(b, W, t_, rtb); break;
    default: ctu1_one_pair<R, 2, 1, RS, IM>(b, W, t_, rtb); break;
  }
}

// out-of-line copy for the persistent kernel
template <typename R, int RS>
__device__ __noinline__ void b_ctu1(const TableView& tv, const int blk_, const DevBox* boxes, const BoxRt* rt, unsigned char* work) {
  body_ctu1<R, RS, false>(tv, blk_, boxes, rt, work);
}

template <typename R, int RS>
__global__ void __launch_bounds__(256) k_ctu1(TableView tv, const DevBox* __restrict__ boxes, const BoxRt* __restrict__ rt, unsigned char* __restrict__ work) {
  body_ctu1<R, RS>(tv, blockIdx.x, boxes, rt, work);
}

template <typename R, int D, int RS, bool IM = true>
__device__ __forceinline__ void ctu2_face(const DevBox& b, R* __restrict__ W, long long Z, const BoxRt& rt,
                                          bool wall) {
  constexpr int E = (D + 1) % 3, F = (D + 2) % 3;
  const long long vs = b.vs, sD = b.s[D];
  const R gamma = Consts<R>::gamma(b), gm1 = Consts<R>::gm1(b), igm1 = Consts<R>::igm1(b);
  R qL[5], qR[5], uL[4], uR[4], Fn[5];
  load_face_states<R, D>(W, vs, Z, sD, igm1, qL, uL, qR, uR);
  const R* Fb[2] = {W + (FLD_F1 + 5 * pair_slot(E, F)) * vs, W + (FLD_F1 + 5 * pair_slot(F, E)) * vs};
  const long long st[2] = {b.s[E], b.s[F]};
  const R fac[2] = {Consts<R>::dtdx2(b, rt, E), Consts<R>::dtdx2(b, rt, F)};
  R rsl, rsr;
  const R EL = correct<R, D, 2, IM>(qL, uL, Fb, st, fac, vs, Z - sD, gm1, igm1, rsl);
  const R ER = correct<R, D, 2, IM>(qR, uR, Fb, st, fac, vs, Z, gm1, igm1, rsr);
  riemann<R, RS, IM>(qL, EL, rsl, qR, ER, rsr, gamma, gm1, igm1, Fn);
  if (wall) {
    // a reflecting face is impermeable: only the normal momentum flux (the wall pressure) remains
    Fn[0] = R(0);
    Fn[2] = R(0);
    Fn[3] = R(0);
    Fn[4] = R(0);
  }
  store_flux<R, D>(W + (FLD_F + 5 * D) * vs, vs, Z, Fn);
}

template <typename R, int RS, bool IM = true>
__device__ __forceinline__ void body_ctu2(const TableView& tv, const int blk_, const DevBox* boxes, const BoxRt* rt, unsigned char* work) {
  LOCATE_AT(tv, blk_)
  if (!box_uses<R>(b)) return;
  const int d = z_;
  int lo[3] = {0, 0, 0}, ext[3] = {b.n[0], b.n[1], b.n[2]}, c[3];
  ext[d] = b.n[d] + 1;
  if (!decode(t_, lo, ext, c)) return;
  const long long Z = zone(b, c[0], c[1], c[2]);
  R* W = fields<R>(work, b);
  const BoxRt& r = rt[bi];
  const bool wall = (c[d] == 0 && b.bc[2 * d] == HYDRO_BC_REFLECT && b.nbr1[2 * d] == 0) ||
                    (c[d] == b.n[d] && b.bc[2 * d + 1] == HYDRO_BC_REFLECT && b.nbr1[2 * d + 1] == 0);
  switch (d) {
    case 0: ctu2_face<R, 0, RS, IM>(b, W, Z, r, wall); break;
    case 1: ctu2_face<R, 1, RS, IM>(b, W, Z, r, wall); break;
    default: ctu2_face<R, 2, RS, IM>(b, W, Z, r, wall); break;
  }
}

// out-of-line copy for the persistent kernel
template <typename R, int RS>
__device__ __noinline__ void b_ctu2(const TableView& tv, const int blk_, const DevBox* boxes, const BoxRt* rt, unsigned char* work) {
  body_ctu2<R, RS, false>(tv, blk_, boxes, rt, work);
}

// Registers capped at 80, as for k_riemann (9.73 -> 9.51 ms at 256^3).
template <typename R, int RS>
__global__ void __maxnreg__(80) k_ctu2(
    TableView tv, const DevBox* __restrict__ boxes, const BoxRt* __restrict__ rt, unsigned char* __restrict__ work) {
  body_ctu2<R, RS>(tv, blockIdx.x, boxes, rt, work);
}

// ---------------------------------------------------------- fused line stage
// Slopes, parabolas, tracing and the normal Riemann solve of one axis depend
// only on the zones of one line along that axis, so one kernel does all four
// with the line's values in registers: it reads the primitive state, sound
// speed and flattening coefficient once and writes only the traced edge states
// and the normal fluxes (no slope fields, no second read of the edge states).
// The arithmetic is the staged kernels' own (vl_slope, parabola, trace_edges,
// the Riemann solver), CW84 limiter only.

// Edge states of zone Z (normal frame of D) and, for FP64, their conserved form.
template <typename R, int D>
__device__ __forceinline__ void line_store_edges(R* __restrict__ W, long long vs, long long Z, const R* qm,
                                                 const R* qp, R igm1) {
#pragma unroll
  for (int m = 0; m < 5; m++) {
    W[(FLD_QM + 5 * D + m) * vs + Z] = qm[m];
    W[(FLD_QP + 5 * D + m) * vs + Z] = qp[m];
  }
  if constexpr (Consts<R>::STORE_CONSERVED) {
    store_conserved<R, D>(W, vs, Z, FLD_UM, qm, igm1);
    store_conserved<R, D>(W, vs, Z, FLD_UP, qp, igm1);
  }
}

// Flux through the D-face between left state qL and right state qR, stored at
// zone Z (the face's high-side zone).
template <typename R, int D, int RS>
__device__ __forceinline__ void line_normal_flux(const DevBox& b, R* __restrict__ W, long long Z, const R* qL,
                                                 const R* qR) {
  const R gamma = Consts<R>::gamma(b), gm1 = Consts<R>::gm1(b), igm1 = Consts<R>::igm1(b);
  R uL[4], uR[4], Fn[5];
  conserved_of(qL, igm1, uL);
  conserved_of(qR, igm1, uR);
  const bool own = RS == HYDRO_RIEMANN_HLLC && Consts<R>::SHARE_RSQRT;
  const R rsl = own ? nr_rsqrt(qL[0]) : R(0);
  const R rsr = own ? nr_rsqrt(qR[0]) : R(0);
  riemann<R, RS>(qL, uL[3], rsl, qR, uR[3], rsr, gamma, gm1, igm1, Fn);
  store_flux<R, D>(W + (FLD_F0 + 5 * D) * b.vs, b.vs, Z, Fn);
}

// x lines: a warp holds 32 consecutive zones of one row, one per lane, and
// gets each neighbour's value, slope and right-edge state by shuffle.  Lane l
// of warp w in the row holds zone i = -1 + 27 w + l - 3; lanes 3..29 store
// their zone's edge states (zones -1 .. n_x) and the flux through its low
// face (faces 0 .. n_x), so consecutive warps tile the row.
template <typename R, int RS>
__device__ __forceinline__ void line_x(const DevBox& b, R* __restrict__ W, long long t, R dtdx) {
  const int nx = b.n[0], ny2 = b.n[1] + 2;
  const int wpr = (nx + 2 + LINE_X_OUT - 1) / LINE_X_OUT;
  const long long per_row = (long long)wpr * 32;
  if (t >= per_row * ny2 * (b.n[2] + 2)) return;  // whole warps only: per_row is a multiple of 32
  const long long row = t / per_row;
  const int rem = (int)(t - row * per_row);
  const int lane = rem & 31;
  const int i = -1 + LINE_X_OUT * (rem >> 5) + lane - 3;
  const int j = (int)(row % ny2) - 1, k = (int)(row / ny2) - 1;
  const long long vs = b.vs;
  const long long Z = zone(b, min(i, nx + 3), j, k);  // lanes past the row's end load its last ghost
  R a[5], dq[5], am[5], ap[5];
#pragma unroll
  for (int m = 0; m < 5; m++) a[m] = W[comp<0>(m) * vs + Z];
  const R f = W[FLD_CHI * vs + Z], cs = W[FLD_C * vs + Z];
#pragma unroll
  for (int m = 0; m < 5; m++) {
    am[m] = __shfl_up_sync(0xffffffffu, a[m], 1);
    ap[m] = __shfl_down_sync(0xffffffffu, a[m], 1);
    dq[m] = vl_slope(am[m], a[m], ap[m]);
  }
  R aL[5], aR[5];
#pragma unroll
  for (int m = 0; m < 5; m++) {
    // this lane's low face; the high face is the next lane's low face
    aL[m] = ppm_face(am[m], a[m], __shfl_up_sync(0xffffffffu, dq[m], 1), dq[m]);
    aR[m] = __shfl_down_sync(0xffffffffu, aL[m], 1);
    cw84_limit(a[m], f, aL[m], aR[m]);
  }
  R qm[5], qp[5];
  trace_edges(a, aL, aR, cs, dtdx, [&](int side, const R* out) {
#pragma unroll
    for (int m = 0; m < 5; m++) (side ? qp : qm)[m] = out[m];
  });
  R ql[5];
#pragma unroll
  for (int m = 0; m < 5; m++) ql[m] = __shfl_up_sync(0xffffffffu, qp[m], 1);
  if (lane < 3 || lane > 29 || i > nx) return;
  line_store_edges<R, 0>(W, vs, Z, qm, qp, Consts<R>::igm1(b));
  if (i >= 0) line_normal_flux<R, 0, RS>(b, W, Z, ql, qm);
}

// y and z lines: a thread walks a segment of LINE_SEG zones of one column
// along D (threads of a warp hold consecutive x, so every load and store is
// coalesced).  Between zones it keeps only the values of zones j and j+1, the
// slope of zone j, the value at the zone's low face (the previous zone's high
// face) and the previous zone's right-edge state; the walk starts one zone
// early so that the first face has its left state.
template <typename R, int D, int RS>
__device__ __forceinline__ void line_walk(const DevBox& b, R* __restrict__ W, long long t, R dtdx) {
  constexpr int E = D == 1 ? 2 : 1;  // the transverse axis other than x
  const int nx2 = b.n[0] + 2, ne2 = b.n[E] + 2, nd = b.n[D];
  const int nseg = (nd + 2 + LINE_SEG - 1) / LINE_SEG;
  if (t >= (long long)nx2 * ne2 * nseg) return;
  const long long rest = t / nx2;
  int c[3];
  c[0] = (int)(t - rest * nx2) - 1;
  c[E] = (int)(rest % ne2) - 1;
  const int js = -1 + (int)(rest / ne2) * LINE_SEG;
  const int je = min(js + LINE_SEG, nd + 1);  // traced zones [js, je), within [-1, n_D]
  c[D] = js - 1;
  const long long vs = b.vs, sD = b.s[D];
  long long Z = zone(b, c[0], c[1], c[2]);  // zone js - 1, the first one traced
  const R igm1 = Consts<R>::igm1(b);
  R q0[5], q1[5], q2[5], d0[5], fl[5], qprev[5];
#pragma unroll
  for (int m = 0; m < 5; m++) {
    const R* a = W + comp<D>(m) * vs + Z;
    const R qa = a[-2 * sD], qb = a[-sD];  // zones js-3, js-2 (at least the last ghost)
    q0[m] = a[0];
    q1[m] = a[sD];
    q2[m] = a[2 * sD];
    const R db = vl_slope(qa, qb, q0[m]);
    d0[m] = vl_slope(qb, q0[m], q1[m]);
    fl[m] = ppm_face(qb, q0[m], db, d0[m]);
  }
#pragma unroll 1
  for (int jz = js - 1; jz < je; jz++, Z += sD) {
    const R f = W[FLD_CHI * vs + Z], cs = W[FLD_C * vs + Z];
    R a0[5], aL[5], aR[5];
#pragma unroll
    for (int m = 0; m < 5; m++) {
      const R d1 = vl_slope(q0[m], q1[m], q2[m]);  // slope of zone jz+1
      a0[m] = q0[m];
      aL[m] = fl[m];
      aR[m] = ppm_face(q0[m], q1[m], d0[m], d1);
      fl[m] = aR[m];  // the next zone's low face, before this zone's limiter
      cw84_limit(a0[m], f, aL[m], aR[m]);
      d0[m] = d1;
      q0[m] = q1[m];
      q1[m] = q2[m];
    }
    R qm[5], qp[5];
    trace_edges(a0, aL, aR, cs, dtdx, [&](int side, const R* out) {
#pragma unroll
      for (int m = 0; m < 5; m++) (side ? qp : qm)[m] = out[m];
    });
    if (jz >= js) {
      line_store_edges<R, D>(W, vs, Z, qm, qp, igm1);
      if (jz >= 0) line_normal_flux<R, D, RS>(b, W, Z, qprev, qm);
    }
#pragma unroll
    for (int m = 0; m < 5; m++) qprev[m] = qp[m];
    if (jz + 1 < je) {  // zone jz+3: at most n_D + 2
#pragma unroll
      for (int m = 0; m < 5; m++) q2[m] = W[comp<D>(m) * vs + Z + 3 * sD];
    }
  }
}

// Two kernels: the x lines need a third of the registers of the column walks
// (no stencil window), so they run at twice the occupancy on their own.
template <typename R, int RS>
__device__ __forceinline__ void body_line_x(const TableView& tv, const int blk_, const DevBox* boxes, const BoxRt* rt, unsigned char* work) {
  LOCATE_AT(tv, blk_)
  if (!box_uses<R>(b)) return;
  line_x<R, RS>(b, fields<R>(work, b), t_, Consts<R>::dtdx(b, rt[bi], 0));
}

// out-of-line copy for the persistent kernel
template <typename R, int RS>
__device__ __noinline__ void b_line_x(const TableView& tv, const int blk_, const DevBox* boxes, const BoxRt* rt, unsigned char* work) {
  body_line_x<R, RS>(tv, blk_, boxes, rt, work);
}

template <typename R, int RS>
__global__ void __launch_bounds__(256) k_line_x(TableView tv, const DevBox* __restrict__ boxes, const BoxRt* __restrict__ rt, unsigned char* __restrict__ work) {
  body_line_x<R, RS>(tv, blockIdx.x, boxes, rt, work);
}

template <typename R, int RS>
__device__ __forceinline__ void body_line_yz(const TableView& tv, const int blk_, const DevBox* boxes, const BoxRt* rt, unsigned char* work) {
  LOCATE_AT(tv, blk_)
  if (!box_uses<R>(b)) return;
  R* W = fields<R>(work, b);
  if (z_ == 0) line_walk<R, 1, RS>(b, W, t_, Consts<R>::dtdx(b, rt[bi], 1));
  else line_walk<R, 2, RS>(b, W, t_, Consts<R>::dtdx(b, rt[bi], 2));
}

// out-of-line copy for the persistent kernel
template <typename R, int RS>
__device__ __noinline__ void b_line_yz(const TableView& tv, const int blk_, const DevBox* boxes, const BoxRt* rt, unsigned char* work) {
  body_line_yz<R, RS>(tv, blk_, boxes, rt, work);
}

template <typename R, int RS>
__global__ void __launch_bounds__(256) k_line_yz(TableView tv, const DevBox* __restrict__ boxes, const BoxRt* __restrict__ rt, unsigned char* __restrict__ work) {
  body_line_yz<R, RS>(tv, blockIdx.x, boxes, rt, work);
}

// ------------------------------------------------ CTU stage 2 along lines
// The final correction of a zone's two D-edge states uses the same flux
// differences across the zone (of the once-corrected fluxes along the two
// transverse axes), so a thread that owns zones rather than faces loads them
// once for both edges and hands the corrected right-edge state on to the next
// face (FP32 boxes; same arithmetic as k_ctu2).

// Zone Z's two D-edge states (raw) and the flux differences across the zone
// that stage 2 corrects them with.
template <typename R, int D>
struct Ctu2Zone {
  R qm[5], qp[5], dlt[2][5];
};

template <typename R, int D>
__device__ __forceinline__ void ctu2_load(const DevBox& b, const R* __restrict__ W, long long Z, Ctu2Zone<R, D>& z) {
  constexpr int E = (D + 1) % 3, F = (D + 2) % 3;
  const long long vs = b.vs;
#pragma unroll
  for (int m = 0; m < 5; m++) {
    z.qm[m] = W[(FLD_QM + 5 * D + m) * vs + Z];
    z.qp[m] = W[(FLD_QP + 5 * D + m) * vs + Z];
  }
  const R* Fb[2] = {W + (FLD_F1 + 5 * pair_slot(E, F)) * vs, W + (FLD_F1 + 5 * pair_slot(F, E)) * vs};
  const long long st[2] = {b.s[E], b.s[F]};
  flux_deltas<R, D, 2>(Fb, st, vs, Z, z.dlt);
}

// Both edge states of a loaded zone corrected by stage 2 (in place), with
// their energies and 1/sqrt(rho).  FP32 boxes only (conserved form rebuilt).
template <typename R, int D>
__device__ __forceinline__ void ctu2_correct(const DevBox& b, Ctu2Zone<R, D>& z, const R* fac, R& Em, R& rsm,
                                             R& Ep, R& rsp) {
  static_assert(!Consts<R>::STORE_CONSERVED, "zone-wise stage 2 runs for FP32 boxes");
  const R gamma = Consts<R>::gamma(b), gm1 = Consts<R>::gm1(b), igm1 = Consts<R>::igm1(b);
  R um[4], up[4];
  conserved_of(z.qm, igm1, um);
  conserved_of(z.qp, igm1, up);
  Em = correct_by<R, 2>(z.qm, um, z.dlt, fac, gm1, igm1, rsm);
  Ep = correct_by<R, 2>(z.qp, up, z.dlt, fac, gm1, igm1, rsp);
}

// Final flux through the low D-face of zone Z from the corrected states.
template <typename R, int D, int RS>
__device__ __forceinline__ void ctu2_flux(const DevBox& b, R* __restrict__ W, long long Z, int face, R* qL, R EL,
                                          R rsl, R* qR, R ER, R rsr) {
  R Fn[5];
  riemann<R, RS>(qL, EL, rsl, qR, ER, rsr, Consts<R>::gamma(b), Consts<R>::gm1(b), Consts<R>::igm1(b), Fn);
  const bool wall = (face == 0 && b.bc[2 * D] == HYDRO_BC_REFLECT && b.nbr1[2 * D] == 0) ||
                    (face == b.n[D] && b.bc[2 * D + 1] == HYDRO_BC_REFLECT && b.nbr1[2 * D + 1] == 0);
  if (wall) {  // impermeable: only the normal momentum flux (the wall pressure) remains
    Fn[0] = R(0);
    Fn[2] = R(0);
    Fn[3] = R(0);
    Fn[4] = R(0);
  }
  store_flux<R, D>(W + (FLD_F + 5 * D) * b.vs, b.vs, Z, Fn);
}

// x faces: lane l of warp w in an interior row owns zone i = -1 + 31 w + l and,
// for l >= 1, the face at its low side (faces 0 .. n_x); the left state comes
// from lane l-1 by shuffle.
template <typename R, int RS>
__device__ __forceinline__ void ctu2_x(const DevBox& b, R* __restrict__ W, long long t, const BoxRt& rt) {
  const int nx = b.n[0], ny = b.n[1];
  const int wpr = (nx + 1 + 30) / 31;
  const long long per_row = (long long)wpr * 32;
  if (t >= per_row * ny * b.n[2]) return;  // whole warps only
  const long long row = t / per_row;
  const int rem = (int)(t - row * per_row);
  const int lane = rem & 31;
  const int i = -1 + 31 * (rem >> 5) + lane;
  const long long Z = zone(b, min(i, nx), (int)(row % ny), (int)(row / ny));
  const R fac[2] = {Consts<R>::dtdx2(b, rt, 1), Consts<R>::dtdx2(b, rt, 2)};
  Ctu2Zone<R, 0> z;
  R Em, Ep, rsm, rsp;
  ctu2_load<R, 0>(b, W, Z, z);
  ctu2_correct<R, 0>(b, z, fac, Em, rsm, Ep, rsp);
  R ql[5];
#pragma unroll
  for (int m = 0; m < 5; m++) ql[m] = __shfl_up_sync(0xffffffffu, z.qp[m], 1);
  const R El = __shfl_up_sync(0xffffffffu, Ep, 1), rsl = __shfl_up_sync(0xffffffffu, rsp, 1);
  if (lane == 0 || i > nx) return;
  ctu2_flux<R, 0, RS>(b, W, Z, i, ql, El, rsl, z.qm, Em, rsm);
}

// y and z faces: a thread walks LINE_SEG faces of one interior column.
template <typename R, int D, int RS>
__device__ __forceinline__ void ctu2_walk(const DevBox& b, R* __restrict__ W, long long t, const BoxRt& rt) {
  constexpr int O = D == 1 ? 2 : 1;  // the transverse axis other than x
  constexpr int E = (D + 1) % 3, F = (D + 2) % 3;
  const int nx = b.n[0], no = b.n[O], nd = b.n[D];
  const int nseg = (nd + 1 + LINE_SEG - 1) / LINE_SEG;
  if (t >= (long long)nx * no * nseg) return;
  const long long rest = t / nx;
  int c[3];
  c[0] = (int)(t - rest * nx);
  c[O] = (int)(rest % no);
  const int fs = (int)(rest / no) * LINE_SEG;
  const int fe = min(fs + LINE_SEG, nd + 1);  // faces [fs, fe), within [0, n_D]
  c[D] = fs - 1;
  const long long sD = b.s[D];
  long long Z = zone(b, c[0], c[1], c[2]);
  const R fac[2] = {Consts<R>::dtdx2(b, rt, E), Consts<R>::dtdx2(b, rt, F)};
  Ctu2Zone<R, D> z;
  R ql[5] = {}, El = R(0), rsl = R(0);
  ctu2_load<R, D>(b, W, Z, z);
  // every zone, the one before the first face included, goes through the same
  // code: a face's two states are then computed by the same instructions
  // whichever segment or box holds the face (periodic faces 0 and n agree
  // bitwise, and so do the faces where boxes of one domain meet)
#pragma unroll 1
  for (int f = fs - 1; f < fe; f++, Z += sD) {  // zone f
    R Em, rsm, Ep, rsp;
    ctu2_correct<R, D>(b, z, fac, Em, rsm, Ep, rsp);
    if (f >= fs) ctu2_flux<R, D, RS>(b, W, Z, f, ql, El, rsl, z.qm, Em, rsm);
#pragma unroll
    for (int m = 0; m < 5; m++) ql[m] = z.qp[m];
    El = Ep;
    rsl = rsp;
    if (f + 1 < fe) ctu2_load<R, D>(b, W, Z + sD, z);  // zone f+1, at most n_D
  }
}

template <typename R, int RS>
__device__ __forceinline__ void body_ctu2_line(const TableView& tv, const int blk_, const DevBox* boxes, const BoxRt* rt, unsigned char* work) {
  LOCATE_AT(tv, blk_)
  if (!box_uses<R>(b)) return;
  R* W = fields<R>(work, b);
  switch (z_) {
    case 0: ctu2_x<R, RS>(b, W, t_, rt[bi]); break;
    case 1: ctu2_walk<R, 1, RS>(b, W, t_, rt[bi]); break;
    default: ctu2_walk<R, 2, RS>(b, W, t_, rt[bi]); break;
  }
}

// out-of-line copy for the persistent kernel
template <typename R, int RS>
__device__ __noinline__ void b_ctu2_line(const TableView& tv, const int blk_, const DevBox* boxes, const BoxRt* rt, unsigned char* work) {
  body_ctu2_line<R, RS>(tv, blk_, boxes, rt, work);
}

template <typename R, int RS>
__global__ void __launch_bounds__(256) k_ctu2_line(TableView tv, const DevBox* __restrict__ boxes, const BoxRt* __restrict__ rt, unsigned char* __restrict__ work) {
  body_ctu2_line<R, RS>(tv, blockIdx.x, boxes, rt, work);
}

// ------------------------------------------------ CTU stage 1 along lines
// Stage 1 corrects each D-edge state of a zone along one transverse axis T
// (the ordered pair (D, T)) with the flux differences across the zone along
// T; the zone's two edge states share them.  Zone-wise, as stage 2, one pair
// per thread.

// Zone Z's two D-edge states (raw) and the flux differences across the zone
// along T, then both states corrected along T (FP32 boxes).
template <typename R, int D, int T>
struct Ctu1Zone {
  R qm[5], qp[5], dlt[1][5];
};

template <typename R, int D, int T>
__device__ __forceinline__ void ctu1_load(const DevBox& b, const R* __restrict__ W, long long Z,
                                          Ctu1Zone<R, D, T>& z) {
  const long long vs = b.vs;
#pragma unroll
  for (int m = 0; m < 5; m++) {
    z.qm[m] = W[(FLD_QM + 5 * D + m) * vs + Z];
    z.qp[m] = W[(FLD_QP + 5 * D + m) * vs + Z];
  }
  const R* Fb[1] = {W + (FLD_F0 + 5 * T) * vs};
  const long long st[1] = {b.s[T]};
  flux_deltas<R, D, 1>(Fb, st, vs, Z, z.dlt);
}

template <typename R, int D, int T>
__device__ __forceinline__ void ctu1_correct(const DevBox& b, Ctu1Zone<R, D, T>& z, R fac, R& Em, R& rsm, R& Ep,
                                             R& rsp) {
  static_assert(!Consts<R>::STORE_CONSERVED, "zone-wise stage 1 runs for FP32 boxes");
  const R gamma = Consts<R>::gamma(b), gm1 = Consts<R>::gm1(b), igm1 = Consts<R>::igm1(b);
  R um[4], up[4];
  conserved_of(z.qm, igm1, um);
  conserved_of(z.qp, igm1, up);
  const R f1[1] = {fac};
  Em = correct_by<R, 1>(z.qm, um, z.dlt, f1, gm1, igm1, rsm);
  Ep = correct_by<R, 1>(z.qp, up, z.dlt, f1, gm1, igm1, rsp);
}

template <typename R, int D, int T, int RS>
__device__ __forceinline__ void ctu1_store(const DevBox& b, R* __restrict__ W, long long Z, R* qL, R EL, R rsl,
                                           R* qR, R ER, R rsr) {
  R Fn[5];
  riemann<R, RS>(qL, EL, rsl, qR, ER, rsr, Consts<R>::gamma(b), Consts<R>::gm1(b), Consts<R>::igm1(b), Fn);
  store_flux<R, D>(W + (FLD_F1 + 5 * pair_slot(D, T)) * b.vs, b.vs, Z, Fn);
}

// x faces of pair (x, T): lane l of warp w in a row owns zone i = -1 + 31 w + l
// and, for l >= 1, the face at its low side (faces 0 .. n_x); rows cover T in
// [0, n_T) and the remaining axis in [-1, n].
template <typename R, int T, int RS>
__device__ __forceinline__ void ctu1_x(const DevBox& b, R* __restrict__ W, long long t, const BoxRt& rt) {
  constexpr int U = 3 - T;  // the axis other than x and T
  int lo[3], ext[3];
  lo[T] = 0;
  ext[T] = b.n[T];
  lo[U] = -1;
  ext[U] = b.n[U] + 2;
  const int nx = b.n[0];
  const int wpr = (nx + 1 + 30) / 31;
  const long long per_row = (long long)wpr * 32;
  if (t >= per_row * ext[1] * ext[2]) return;  // whole warps only
  const long long row = t / per_row;
  const int rem = (int)(t - row * per_row);
  const int lane = rem & 31;
  const int i = -1 + 31 * (rem >> 5) + lane;
  const int j = lo[1] + (int)(row % ext[1]), k = lo[2] + (int)(row / ext[1]);
  const long long Z = zone(b, min(i, nx), j, k);
  Ctu1Zone<R, 0, T> z;
  R ql[5], Em, Ep, rsm, rsp;
  ctu1_load<R, 0, T>(b, W, Z, z);
  ctu1_correct<R, 0, T>(b, z, Consts<R>::dtdx3(b, rt, T), Em, rsm, Ep, rsp);
#pragma unroll
  for (int m = 0; m < 5; m++) ql[m] = __shfl_up_sync(0xffffffffu, z.qp[m], 1);
  const R El = __shfl_up_sync(0xffffffffu, Ep, 1), rsl = __shfl_up_sync(0xffffffffu, rsp, 1);
  if (lane == 0 || i > nx) return;
  ctu1_store<R, 0, T, RS>(b, W, Z, ql, El, rsl, z.qm, Em, rsm);
}

// y and z faces of pair (D, T): a thread walks LINE_SEG faces of one column
// (x and the other transverse axis: T in [0, n_T), the remaining one in
// [-1, n]); every zone goes through the same code, the one before the first
// face included.
template <typename R, int D, int T, int RS>
__device__ __forceinline__ void ctu1_walk(const DevBox& b, R* __restrict__ W, long long t, const BoxRt& rt) {
  constexpr int O = D == 1 ? 2 : 1;  // the transverse axis other than x
  constexpr int U = 3 - D - T;       // the transverse axis other than T
  int lo[3], ext[3];
  lo[T] = 0;
  ext[T] = b.n[T];
  lo[U] = -1;
  ext[U] = b.n[U] + 2;
  const int nd = b.n[D];
  const int nseg = (nd + 1 + LINE_SEG - 1) / LINE_SEG;
  if (t >= (long long)ext[0] * ext[O] * nseg) return;
  const long long rest = t / ext[0];
  int c[3];
  c[0] = lo[0] + (int)(t - rest * ext[0]);
  c[O] = lo[O] + (int)(rest % ext[O]);
  const int fs = (int)(rest / ext[O]) * LINE_SEG;
  const int fe = min(fs + LINE_SEG, nd + 1);  // faces [fs, fe), within [0, n_D]
  c[D] = fs - 1;
  const long long sD = b.s[D];
  long long Z = zone(b, c[0], c[1], c[2]);
  const R fac = Consts<R>::dtdx3(b, rt, T);
  Ctu1Zone<R, D, T> z;
  R ql[5] = {}, El = R(0), rsl = R(0);
  ctu1_load<R, D, T>(b, W, Z, z);
#pragma unroll 1
  for (int f = fs - 1; f < fe; f++, Z += sD) {  // zone f
    R Em, Ep, rsm, rsp;
    ctu1_correct<R, D, T>(b, z, fac, Em, rsm, Ep, rsp);
    if (f >= fs) ctu1_store<R, D, T, RS>(b, W, Z, ql, El, rsl, z.qm, Em, rsm);
#pragma unroll
    for (int m = 0; m < 5; m++) ql[m] = z.qp[m];
    El = Ep;
    rsl = rsp;
    if (f + 1 < fe) ctu1_load<R, D, T>(b, W, Z + sD, z);  // zone f+1, at most n_D
  }
}

// work item z = pair slot (xy xz yx yz zx zy)
template <typename R, int RS>
__device__ __forceinline__ void body_ctu1_line(const TableView& tv, const int blk_, const DevBox* boxes, const BoxRt* rt, unsigned char* work) {
  LOCATE_AT(tv, blk_)
  if (!box_uses<R>(b)) return;
  R* W = fields<R>(work, b);
  switch (z_) {
    case 0: ctu1_x<R, 1, RS>(b, W, t_, rt[bi]); break;
    case 1: ctu1_x<R, 2, RS>(b, W, t_, rt[bi]); break;
    case 2: ctu1_walk<R, 1, 0, RS>(b, W, t_, rt[bi]); break;
    case 3: ctu1_walk<R, 1, 2, RS>(b, W, t_, rt[bi]); break;
    case 4: ctu1_walk<R, 2, 0, RS>(b, W, t_, rt[bi]); break;
    default: ctu1_walk<R, 2, 1, RS>(b, W, t_, rt[bi]); break;
  }
}

// out-of-line copy for the persistent kernel
template <typename R, int RS>
__device__ __noinline__ void b_ctu1_line(const TableView& tv, const int blk_, const DevBox* boxes, const BoxRt* rt, unsigned char* work) {
  body_ctu1_line<R, RS>(tv, blk_, boxes, rt, work);
}

template <typename R, int RS>
__global__ void __launch_bounds__(256) k_ctu1_line(TableView tv, const DevBox* __restrict__ boxes, const BoxRt* __restrict__ rt, unsigned char* __restrict__ work) {
  body_ctu1_line<R, RS>(tv, blockIdx.x, boxes, rt, work);
}

// --------------------------------------------------------------------- update
// FP32 -> FP64 on the integer pipe (the conversion instruction would occupy
// the FP64 pipe): exact for normal floats; zero, subnormal floats (below
// 1.2e-38) give zero.  Both neighbours of a face widen its flux identically,
// so conservation is untouched.
__device__ __forceinline__ double widen(float x) {
  const unsigned int f = __float_as_uint(x);
  const unsigned int sign = f & 0x80000000u;
  if ((f & 0x7f800000u) == 0u) return __hiloint2double((int)sign, 0);
  // exponent rebias 127 -> 1023 (+896) and mantissa 23 -> 52 bits, in 32-bit halves
  const unsigned int hi = sign | (((f & 0x7fffffffu) >> 3) + (896u << 20));
  return __hiloint2double((int)hi, (int)(f << 29));
}
__device__ __forceinline__ double widen(double x) { return x; }

// FP64 for every box; the fluxes are read in the box's compute type.
template <typename R>
__device__ __forceinline__ void update_zone(const DevBox& b, double* __restrict__ U, const R* __restrict__ W,
                                            long long Z, const double* dtdx, double* nu) {
  const long long vs = b.vs;
#pragma unroll
  for (int v = 0; v < 5; v++) {
    double val = U[v * vs + Z];
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const R* F = W + (FLD_F + 5 * d + v) * vs;
      val = val - dtdx[d] * (widen(F[Z + b.s[d]]) - widen(F[Z]));
    }
    nu[v] = val;
    U[v * vs + Z] = val;
  }
}

// skip_mixed: FP32 boxes are updated by the fused tile stage
__device__ __forceinline__ void body_update(const TableView& tv, const int blk_, const DevBox* boxes, BoxRt* rt, double* state, unsigned char* work, int skip_mixed) {
  LOCATE_AT(tv, blk_)
  if (skip_mixed && b.precision == HYDRO_MIXED) return;
  int lo[3] = {0, 0, 0}, ext[3] = {b.n[0], b.n[1], b.n[2]}, c[3];
  if (!decode(t_, lo, ext, c)) return;
  const long long Z = zone(b, c[0], c[1], c[2]);
  double* U = state + b.state_off;
  const double dtdx[3] = {rt[bi].dtdx[0], rt[bi].dtdx[1], rt[bi].dtdx[2]};
  double nu[5];
  if (b.precision == HYDRO_FP64) update_zone(b, U, fields<double>(work, b), Z, dtdx, nu);
  else update_zone(b, U, fields<float>(work, b), Z, dtdx, nu);
  // rho > 0 and p = (gamma - 1)(E - |m|^2 / (2 rho)) > 0, i.e. rho E > |m|^2 / 2:
  // no reciprocal; a NaN fails the tests.  One fused multiply-add forms
  // rho E - |m|^2 / 2, half of 2 rho E - |m|^2 and so of its sign (the
  // halving is exact for |m|^2 >= 2^-1021; the two differ only where the
  // difference underflows).
  const double m2 = nu[1] * nu[1] + nu[2] * nu[2] + nu[3] * nu[3];
  const double e2 = fma(nu[0], nu[4], -half_of(m2));
  if (!is_pos(nu[0]) || !pos_not_nan(e2)) atomicOr(&rt[bi].status, STATUS_NONPHYSICAL);
}

// out-of-line copy for the persistent kernel
__device__ __noinline__ void b_update(const TableView& tv, const int blk_, const DevBox* boxes, BoxRt* rt, double* state, unsigned char* work, int skip_mixed) {
  body_update(tv, blk_, boxes, rt, state, work, skip_mixed);
}

// one block per SM stated, as for the tracing (52 registers against 32: 7 % faster)
__global__ void __launch_bounds__(256, 1) k_update(TableView tv, const DevBox* __restrict__ boxes, BoxRt* __restrict__ rt, double* __restrict__ state, unsigned char* __restrict__ work, int skip_mixed) {
  body_update(tv, blockIdx.x, boxes, rt, state, work, skip_mixed);
}

// ---------------------------------------------------------- fused tile stage
// For FP32 boxes under the CW84 limiter, one kernel does what the line, CTU
// and update kernels do, with every traced state and flux of the step kept
// on chip.  A block advances a tile of TILE_X x TY interior zone columns of
// one box over a segment of z-planes, marching in z.  At plane p it stages
// the primitive state of the plane (with a three-zone halo) in shared memory,
// traces plane p along x, y and z, forms plane p's normal fluxes and the
// stage-1 fluxes through its low z-face, then stage 1 in the plane and the
// final fluxes of plane p-1, and applies the FP64 update to plane p-2.  A
// thread owns one zone column of the tile with its one-zone halo (32 x (TY+2)
// columns: a warp covers a row, lane l the zone x0 - 1 + l), keeps the z
// stencil of its column in registers and exchanges in-plane neighbours
// through shared memory and warp shuffles.  Each state and flux is formed by
// the same functions from the same operands as in the line kernels and the
// zone-wise CTU kernels, so the results are bitwise the same; the halo costs
// (TY + 2) x 32 / (TY x 30) times the zone work and 3 planes of pipeline
// warm-up per segment.
constexpr int TILE_X = 30;

template <int TY>
struct TileShape {
  static constexpr int NR = 32 * (TY + 2);  // threads = traced zones of a plane
  static constexpr int QX = 36;             // staged zones along x: -3 .. 32
  static constexpr int NQ = QX * (TY + 6);  // staged zones of a plane
  // shared-memory layout (floats)
  static constexpr int O_Q = 0;                 // q[5][NQ] of the plane being traced
  static constexpr int O_C = O_Q + 5 * NQ;      // c[NR]
  static constexpr int O_CHI = O_C + NR;        // chi[NR]
  static constexpr int O_TX = O_CHI + NR;       // x-traced qm[5], qp[5]: [2 plane parities][10][NR]
  static constexpr int O_TY = O_TX + 20 * NR;   // y-traced, likewise
  static constexpr int O_TZ = O_TY + 20 * NR;   // z-traced, likewise (a thread's own column)
  static constexpr int O_F0X = O_TZ + 20 * NR;  // normal fluxes [2][5][NR], conserved x,y,z components
  static constexpr int O_F0Y = O_F0X + 10 * NR;
  static constexpr int O_F0Z = O_F0Y + 10 * NR;  // by face parity
  static constexpr int O_FZX = O_F0Z + 10 * NR;  // stage-1 z-face fluxes F^{z|x}, F^{z|y}: [2][5][NR]
  static constexpr int O_FZY = O_FZX + 10 * NR;
  static constexpr int O_F1 = O_FZY + 10 * NR;   // stage-1 in-plane fluxes [4][5][NR]: x|y, x|z, y|x, y|z
  static constexpr int O_EX = O_F1 + 20 * NR;    // y exchange of corrected right-edge states: [2][7][NR]
  static constexpr int O_FX = O_EX + 14 * NR;    // final x and y fluxes of the previous plane [5][NR] each
  static constexpr int O_FY = O_FX + 5 * NR;
  static constexpr int TOTAL = O_FY + 5 * NR;
  static constexpr size_t BYTES = TOTAL * sizeof(float);
};

// A corrected edge state: primitive q, total energy and 1/sqrt(rho) (0 in FP32).
struct EdgeF {
  float q[5];
  float E, rs;
};

// An edge state q (raw, normal frame of D) corrected by NT flux differences
// dlt with factors fac, as ctu1_correct / ctu2_correct correct each edge.
template <int NT>
__device__ __forceinline__ EdgeF tile_correct1(const float* q, const float (*dlt)[5], const float* fac, float gamma,
                                               float igm1) {
  EdgeF e;
  float u[4];
  const float gm1 = gamma - 1.0f;
#pragma unroll
  for (int m = 0; m < 5; m++) e.q[m] = q[m];
  conserved_of(e.q, igm1, u);
  e.E = correct_by<float, NT>(e.q, u, dlt, fac, gm1, igm1, e.rs);
  return e;
}

// Both edge states of a zone corrected by the same flux differences.
template <int NT>
__device__ __forceinline__ void tile_correct(const float* qm, const float* qp, const float (*dlt)[5], const float* fac,
                                             float gamma, float igm1, EdgeF& em, EdgeF& ep) {
  em = tile_correct1<NT>(qm, dlt, fac, gamma, igm1);
  ep = tile_correct1<NT>(qp, dlt, fac, gamma, igm1);
}

// Riemann flux between two corrected states, in the normal frame of D.
template <int RS>
__device__ __forceinline__ void tile_flux(const EdgeF& l, const EdgeF& r, float gamma, float igm1, float* Fn) {
  const float gm1 = gamma - 1.0f;
  riemann<float, RS>(l.q, l.E, l.rs, r.q, r.E, r.rs, gamma, gm1, igm1, Fn);
}

// Flux difference across a zone for the normal frame of D: F[comp<D>(m)] at
// the high face minus the low face.
template <int D>
__device__ __forceinline__ void tile_delta(const float* F, int NRr, int lo, int hi, float* d) {
#pragma unroll
  for (int m = 0; m < 5; m++) d[m] = F[comp<D>(m) * NRr + hi] - F[comp<D>(m) * NRr + lo];
}

template <int D>
__device__ __forceinline__ void tile_store(float* F, int NRr, int at, const float* Fn) {
#pragma unroll
  for (int m = 0; m < 5; m++) F[comp<D>(m) * NRr + at] = Fn[m];
}

// Shuffle a corrected state from the lane below.
__device__ __forceinline__ EdgeF shfl_up_edge(const EdgeF& e) {
  EdgeF o;
#pragma unroll
  for (int m = 0; m < 5; m++) o.q[m] = __shfl_up_sync(0xffffffffu, e.q[m], 1);
  o.E = __shfl_up_sync(0xffffffffu, e.E, 1);
  o.rs = __shfl_up_sync(0xffffffffu, e.rs, 1);
  return o;
}

__device__ __forceinline__ void put_edge(float* X, int NRr, int at, const EdgeF& e) {
#pragma unroll
  for (int m = 0; m < 5; m++) X[m * NRr + at] = e.q[m];
  X[5 * NRr + at] = e.E;
  X[6 * NRr + at] = e.rs;
}

__device__ __forceinline__ EdgeF get_edge(const float* X, int NRr, int at) {
  EdgeF e;
#pragma unroll
  for (int m = 0; m < 5; m++) e.q[m] = X[m * NRr + at];
  e.E = X[5 * NRr + at];
  e.rs = X[6 * NRr + at];
  return e;
}

// The PPM parabola of zone 0 of a line a[-2..2] (stride 1 in the array passed):
// van Leer slopes of zones -1, 0, 1, interface values, CW84 limiter with
// flattening f; as the line kernels form it.
__device__ __forceinline__ void tile_parabola(float am2, float am1, float a0, float ap1, float ap2, float f, float& aL,
                                              float& aR) {
  const float dm1 = vl_slope(am2, am1, a0), d0 = vl_slope(am1, a0, ap1), dp1 = vl_slope(a0, ap1, ap2);
  aL = ppm_face(am1, a0, dm1, d0);
  aR = ppm_face(a0, ap1, d0, dp1);
  cw84_limit(a0, f, aL, aR);
}

// Reflecting face of the box (impermeable: only the normal momentum flux
// remains), as ctu2_flux decides it.
template <int D>
__device__ __forceinline__ void tile_wall(const DevBox& b, int face, float* Fn) {
  const bool wall = (face == 0 && b.bc[2 * D] == HYDRO_BC_REFLECT && b.nbr1[2 * D] == 0) ||
                    (face == b.n[D] && b.bc[2 * D + 1] == HYDRO_BC_REFLECT && b.nbr1[2 * D + 1] == 0);
  if (wall) {
    Fn[0] = 0.0f;
    Fn[2] = 0.0f;
    Fn[3] = 0.0f;
    Fn[4] = 0.0f;
  }
}

template <int TY, int RS>
__global__ void __launch_bounds__(TileShape<TY>::NR, 1)
    k_tile(TableView tv, const DevBox* __restrict__ boxes, BoxRt* __restrict__ rt, double* __restrict__ state,
           unsigned char* __restrict__ work, int seg_len) {
  using T = TileShape<TY>;
  constexpr int NR = T::NR, NQ = T::NQ;
  extern __shared__ float sm[];
  LOCATE(tv)
  if (!box_uses<float>(b)) return;
  const int nx = b.n[0], ny = b.n[1], nz = b.n[2];
  const int ntx = (nx + TILE_X - 1) / TILE_X, nty = (ny + TY - 1) / TY, nseg = (nz + seg_len - 1) / seg_len;
  const int vb = (int)(t_ / NR);
  if (vb >= ntx * nty * nseg) return;  // whole blocks only
  const int tx = vb % ntx, ty = (vb / ntx) % nty, seg = vb / (ntx * nty);
  const int x0 = tx * TILE_X, y0 = ty * TY, z0 = seg * seg_len, z1 = min(z0 + seg_len, nz);
  const int t = threadIdx.x, lane = t & 31;
  const int ci = lane - 1, cj = (t >> 5) - 1;
  const int gx = x0 + ci, gy = y0 + cj;
  // a traced zone of the box; a zone of the tile's interior (and of the box);
  // the low x- or y-face of this zone is one of the box's faces
  const bool in_x = gx >= -1 && gx <= nx, in_y = gy >= -1 && gy <= ny;
  const bool int_x = ci >= 0 && ci < TILE_X && gx < nx, int_y = cj >= 0 && cj < TY && gy < ny;
  const bool fc_x = ci >= 0 && gx <= nx, fc_y = cj >= 0 && gy <= ny;
  const long long vs = b.vs;
  float* W = fields<float>(work, b);
  double* U = state + b.state_off;
  const BoxRt& r = rt[bi];
  const float gamma = b.gamma_f, gm1 = gamma - 1.0f, igm1 = b.igm1_f;
  const float dtdx[3] = {r.dtdx_f[0], r.dtdx_f[1], r.dtdx_f[2]};
  const double dtdx64[3] = {r.dt * b.idx[0], r.dt * b.idx[1], r.dt * b.idx[2]};
  const float fac1[3] = {dtdx[0] * float(1.0 / 3.0), dtdx[1] * float(1.0 / 3.0), dtdx[2] * float(1.0 / 3.0)};
  float* sQ = sm + T::O_Q;
  float* sC = sm + T::O_C;
  float* sChi = sm + T::O_CHI;
  // zone of the state/fields at (x, y, k), with x and y clamped into the ghosted box
  auto zat = [&](int x, int y, int k) {
    return zone(b, min(max(x, -NG), nx + NG - 1), min(max(y, -NG), ny + NG - 1), k);
  };
  const long long Zc = zat(gx, gy, 0) - (long long)NG * b.s[2];  // this column at k = 0 is Zc + (k+NG) s_z
  const long long sz = b.s[2];

  // z stencil of this column, as line_walk keeps it: zone values of the next
  // three planes, the slope of the next plane and the value at its low face
  float q0[5], q1[5], q2[5], d0[5], fl[5];
  {
    const int k = z0 - 1;  // the first plane traced
    const long long Z = Zc + (long long)(k + NG) * sz;
#pragma unroll
    for (int m = 0; m < 5; m++) {
      const float* a = W + comp<2>(m) * vs + Z;
      const float qa = a[-2 * sz], qb = a[-sz];
      q0[m] = a[0];
      q1[m] = a[sz];
      q2[m] = a[2 * sz];
      const float db = vl_slope(qa, qb, q0[m]);
      d0[m] = vl_slope(qb, q0[m], q1[m]);
      fl[m] = ppm_face(qb, q0[m], db, d0[m]);
    }
  }
  EdgeF zfin;                         // U^{z,fin} right edge of the plane before the one being finished
  float fz_prev[5] = {0, 0, 0, 0, 0};  // final flux through the low z-face of the plane before
  zfin.E = zfin.rs = 0.0f;
#pragma unroll
  for (int m = 0; m < 5; m++) zfin.q[m] = 0.0f;

#pragma unroll 1
  for (int p = z0 - 1; p <= z1 + 1; p++) {
    const bool trace = p <= z1;
    const int cur = p & 1, prv = cur ^ 1;
    float* tx_c = sm + T::O_TX + cur * 10 * NR;
    float* tx_p = sm + T::O_TX + prv * 10 * NR;
    float* ty_c = sm + T::O_TY + cur * 10 * NR;
    float* ty_p = sm + T::O_TY + prv * 10 * NR;
    float* tz_c = sm + T::O_TZ + cur * 10 * NR;
    float* tz_p = sm + T::O_TZ + prv * 10 * NR;
    float* f0x_c = sm + T::O_F0X + cur * 5 * NR;
    float* f0x_p = sm + T::O_F0X + prv * 5 * NR;
    float* f0y_c = sm + T::O_F0Y + cur * 5 * NR;
    float* f0y_p = sm + T::O_F0Y + prv * 5 * NR;
    float* f0z_c = sm + T::O_F0Z + cur * 5 * NR;
    float* f0z_p = sm + T::O_F0Z + prv * 5 * NR;
    float* fzx_c = sm + T::O_FZX + cur * 5 * NR;
    float* fzx_p = sm + T::O_FZX + prv * 5 * NR;
    float* fzy_c = sm + T::O_FZY + cur * 5 * NR;
    float* fzy_p = sm + T::O_FZY + prv * 5 * NR;
    float* sF1 = sm + T::O_F1;
    float* ex0 = sm + T::O_EX;
    float* ex1 = sm + T::O_EX + 7 * NR;
    float* sFX = sm + T::O_FX;
    float* sFY = sm + T::O_FY;

    // state of the plane the update reaches this step, requested early
    const int pu = p - 2;
    const bool upd = pu >= z0 && pu < z1 && int_x && int_y;
    double uo[5];
    const long long Zu = Zc + (long long)(pu + NG) * sz;
    if (upd) {
#pragma unroll
      for (int v = 0; v < 5; v++) uo[v] = U[v * vs + Zu];
    }

    // 1. stage plane p: primitive state with a three-zone halo, c and chi
    if (trace) {
      for (int e = t; e < NQ; e += NR) {
        const int qi = e % T::QX - 3, qj = e / T::QX - 3;
        const long long Z = zat(x0 + qi, y0 + qj, p);
#pragma unroll
        for (int m = 0; m < 5; m++) sQ[m * NQ + e] = W[m * vs + Z];
      }
      const long long Z = Zc + (long long)(p + NG) * sz;
      sC[t] = W[FLD_C * vs + Z];
      sChi[t] = W[FLD_CHI * vs + Z];
    }
    __syncthreads();

    // 2. trace plane p along x, y (from the staged plane) and z (column registers)
    if (trace) {
      const float cs = sC[t], f = sChi[t];
      const int e0 = (cj + 3) * T::QX + (ci + 3);
      const float rho = sQ[e0];
      const float ic = nr_rcp(cs), cr = cs * nr_rcp(rho);
      float a0[5], aL[5], aR[5];
#pragma unroll
      for (int m = 0; m < 5; m++) {
        const float* a = sQ + comp<0>(m) * NQ + e0;
        a0[m] = a[0];
        tile_parabola(a[-2], a[-1], a[0], a[1], a[2], f, aL[m], aR[m]);
      }
      trace_edges(a0, aL, aR, cs, ic, cr, dtdx[0], [&](int side, const float* out) {
#pragma unroll
        for (int m = 0; m < 5; m++) tx_c[(side * 5 + m) * NR + t] = out[m];
      });
#pragma unroll
      for (int m = 0; m < 5; m++) {
        const float* a = sQ + comp<1>(m) * NQ + e0;
        a0[m] = a[0];
        tile_parabola(a[-2 * T::QX], a[-T::QX], a[0], a[T::QX], a[2 * T::QX], f, aL[m], aR[m]);
      }
      trace_edges(a0, aL, aR, cs, ic, cr, dtdx[1], [&](int side, const float* out) {
#pragma unroll
        for (int m = 0; m < 5; m++) ty_c[(side * 5 + m) * NR + t] = out[m];
      });
#pragma unroll
      for (int m = 0; m < 5; m++) {
        const float d1 = vl_slope(q0[m], q1[m], q2[m]);
        a0[m] = q0[m];
        aL[m] = fl[m];
        aR[m] = ppm_face(q0[m], q1[m], d0[m], d1);
        fl[m] = aR[m];
        cw84_limit(a0[m], f, aL[m], aR[m]);
        d0[m] = d1;
        q0[m] = q1[m];
        q1[m] = q2[m];
      }
      trace_edges(a0, aL, aR, cs, ic, cr, dtdx[2], [&](int side, const float* out) {
#pragma unroll
        for (int m = 0; m < 5; m++) tz_c[(side * 5 + m) * NR + t] = out[m];
      });
      if (p + 1 <= z1) {  // the plane three ahead, for the next plane's stencil
        const long long Z = Zc + (long long)(p + 3 + NG) * sz;
#pragma unroll
        for (int m = 0; m < 5; m++) q2[m] = W[comp<2>(m) * vs + Z];
      }
    }
    __syncthreads();

    // 3. normal fluxes of plane p: x- and y-faces at the zone's low side, and
    // the z-face between planes p-1 and p
    if (trace) {
      float qL[5], qR[5], uL[4], uR[4], Fn[5];
      if (fc_x && in_y) {
#pragma unroll
        for (int m = 0; m < 5; m++) {
          qL[m] = tx_c[(5 + m) * NR + t - 1];
          qR[m] = tx_c[m * NR + t];
        }
        conserved_of(qL, igm1, uL);
        conserved_of(qR, igm1, uR);
        riemann<float, RS>(qL, uL[3], 0.0f, qR, uR[3], 0.0f, gamma, gm1, igm1, Fn);
        tile_store<0>(f0x_c, NR, t, Fn);
      }
      if (fc_y && in_x) {
#pragma unroll
        for (int m = 0; m < 5; m++) {
          qL[m] = ty_c[(5 + m) * NR + t - 32];
          qR[m] = ty_c[m * NR + t];
        }
        conserved_of(qL, igm1, uL);
        conserved_of(qR, igm1, uR);
        riemann<float, RS>(qL, uL[3], 0.0f, qR, uR[3], 0.0f, gamma, gm1, igm1, Fn);
        tile_store<1>(f0y_c, NR, t, Fn);
      }
      if (p >= z0 && in_x && in_y) {
#pragma unroll
        for (int m = 0; m < 5; m++) {
          qL[m] = tz_p[(5 + m) * NR + t];
          qR[m] = tz_c[m * NR + t];
        }
        conserved_of(qL, igm1, uL);
        conserved_of(qR, igm1, uR);
        riemann<float, RS>(qL, uL[3], 0.0f, qR, uR[3], 0.0f, gamma, gm1, igm1, Fn);
        tile_store<2>(f0z_c, NR, t, Fn);
      }
    }
    __syncthreads();

    // 4. stage 1 through z-face p: F^{z|x} and F^{z|y}, from the left edge of
    // plane p and the right edge of plane p-1, each corrected by the flux
    // differences across its own zone
    if (trace && p >= z0) {
      float dl[1][5], Fn[5], qm[5], qpp[5];
#pragma unroll
      for (int m = 0; m < 5; m++) {
        qm[m] = tz_c[m * NR + t];
        qpp[m] = tz_p[(5 + m) * NR + t];
      }
      if (int_x && in_y) {
        const float fac[1] = {fac1[0]};
        tile_delta<2>(f0x_c, NR, t, t + 1, dl[0]);
        const EdgeF em = tile_correct1<1>(qm, dl, fac, gamma, igm1);
        tile_delta<2>(f0x_p, NR, t, t + 1, dl[0]);
        const EdgeF lp = tile_correct1<1>(qpp, dl, fac, gamma, igm1);
        tile_flux<RS>(lp, em, gamma, igm1, Fn);
        tile_store<2>(fzx_c, NR, t, Fn);
      }
      if (in_x && int_y) {
        const float fac[1] = {fac1[1]};
        tile_delta<2>(f0y_c, NR, t, t + 32, dl[0]);
        const EdgeF em = tile_correct1<1>(qm, dl, fac, gamma, igm1);
        tile_delta<2>(f0y_p, NR, t, t + 32, dl[0]);
        const EdgeF lp = tile_correct1<1>(qpp, dl, fac, gamma, igm1);
        tile_flux<RS>(lp, em, gamma, igm1, Fn);
        tile_store<2>(fzy_c, NR, t, Fn);
      }
    }

    // 5. stage 1 in plane p-1: x|y, x|z (x-faces, neighbours by shuffle),
    // y|x, y|z (y-faces, neighbours through shared memory)
    const int pm = p - 1;
    if (p >= z0) {
      const bool mid = pm >= z0 && pm < z1;
      float dl[1][5], Fn[5], qm[5], qp[5];
      EdgeF em, ep;
#pragma unroll
      for (int m = 0; m < 5; m++) {
        qm[m] = tx_p[m * NR + t];
        qp[m] = tx_p[(5 + m) * NR + t];
      }
      {  // x|y
        const float fac[1] = {fac1[1]};
        tile_delta<0>(f0y_p, NR, t, t + 32, dl[0]);
        tile_correct<1>(qm, qp, dl, fac, gamma, igm1, em, ep);
        const EdgeF lp = shfl_up_edge(ep);
        if (fc_x && int_y) {
          tile_flux<RS>(lp, em, gamma, igm1, Fn);
          tile_store<0>(sF1 + 0 * 5 * NR, NR, t, Fn);
        }
      }
      if (mid) {  // x|z
        const float fac[1] = {fac1[2]};
#pragma unroll
        for (int m = 0; m < 5; m++)
          dl[0][m] = f0z_c[comp<0>(m) * NR + t] - f0z_p[comp<0>(m) * NR + t];
        tile_correct<1>(qm, qp, dl, fac, gamma, igm1, em, ep);
        const EdgeF lp = shfl_up_edge(ep);
        if (fc_x && in_y) {
          tile_flux<RS>(lp, em, gamma, igm1, Fn);
          tile_store<0>(sF1 + 1 * 5 * NR, NR, t, Fn);
        }
      }
#pragma unroll
      for (int m = 0; m < 5; m++) {
        qm[m] = ty_p[m * NR + t];
        qp[m] = ty_p[(5 + m) * NR + t];
      }
      EdgeF ymx, ymz;
      {  // y|x: corrected states; the right edge goes to the zone above
        const float fac[1] = {fac1[0]};
        tile_delta<1>(f0x_p, NR, t, t + 1, dl[0]);
        tile_correct<1>(qm, qp, dl, fac, gamma, igm1, ymx, ep);
        put_edge(ex0, NR, t, ep);
      }
      if (mid) {  // y|z
        const float fac[1] = {fac1[2]};
#pragma unroll
        for (int m = 0; m < 5; m++)
          dl[0][m] = f0z_c[comp<1>(m) * NR + t] - f0z_p[comp<1>(m) * NR + t];
        tile_correct<1>(qm, qp, dl, fac, gamma, igm1, ymz, ep);
        put_edge(ex1, NR, t, ep);
      }
      __syncthreads();
      if (fc_y && int_x) {
        const EdgeF lp = get_edge(ex0, NR, t - 32);
        tile_flux<RS>(lp, ymx, gamma, igm1, Fn);
        tile_store<1>(sF1 + 2 * 5 * NR, NR, t, Fn);
      }
      if (mid && fc_y && in_x) {
        const EdgeF lp = get_edge(ex1, NR, t - 32);
        tile_flux<RS>(lp, ymz, gamma, igm1, Fn);
        tile_store<1>(sF1 + 3 * 5 * NR, NR, t, Fn);
      }
    }
    __syncthreads();

    // 6. stage 2 of plane p-1 along z: U^{z,fin}, and the final flux through
    // its low z-face
    float fz_new[5] = {0, 0, 0, 0, 0};
    if (p >= z0 && int_x && int_y) {
      float dl[2][5], qm[5], qp[5];
      const float fac[2] = {0.5f * dtdx[0], 0.5f * dtdx[1]};
      tile_delta<2>(sF1 + 0 * 5 * NR, NR, t, t + 1, dl[0]);
      tile_delta<2>(sF1 + 2 * 5 * NR, NR, t, t + 32, dl[1]);
#pragma unroll
      for (int m = 0; m < 5; m++) {
        qm[m] = tz_p[m * NR + t];
        qp[m] = tz_p[(5 + m) * NR + t];
      }
      EdgeF em, ep;
      tile_correct<2>(qm, qp, dl, fac, gamma, igm1, em, ep);
      if (pm >= z0) {
        float Fn[5];
        tile_flux<RS>(zfin, em, gamma, igm1, Fn);
        tile_wall<2>(b, pm, Fn);
#pragma unroll
        for (int m = 0; m < 5; m++) fz_new[comp<2>(m)] = Fn[m];
      }
      zfin = ep;
    }

    // 7. FP64 update of plane p-2 (the order of update_zone)
    if (upd) {
      double nu[5];
#pragma unroll
      for (int v = 0; v < 5; v++) {
        double val = uo[v];
        val = val - dtdx64[0] * (widen(sFX[v * NR + t + 1]) - widen(sFX[v * NR + t]));
        val = val - dtdx64[1] * (widen(sFY[v * NR + t + 32]) - widen(sFY[v * NR + t]));
        val = val - dtdx64[2] * (widen(fz_new[v]) - widen(fz_prev[v]));
        nu[v] = val;
        U[v * vs + Zu] = val;
      }
      const double m2 = nu[1] * nu[1] + nu[2] * nu[2] + nu[3] * nu[3];
      const double e2 = 2.0 * nu[0] * nu[4] - m2;
      if (!is_pos(nu[0]) || !is_pos(e2) || e2 != e2) atomicOr(&rt[bi].status, STATUS_NONPHYSICAL);
    }
    if (pm >= z0) {
#pragma unroll
      for (int v = 0; v < 5; v++) fz_prev[v] = fz_new[v];
    }
    __syncthreads();

    // 8. stage 2 of plane p-1 along x and y: the final fluxes through the
    // zone's low x- and y-faces
    if (pm >= z0 && pm < z1) {
      float dl[2][5], Fn[5], qm[5], qp[5];
      EdgeF em, ep;
#pragma unroll
      for (int m = 0; m < 5; m++) {
        qm[m] = tx_p[m * NR + t];
        qp[m] = tx_p[(5 + m) * NR + t];
      }
      {
        const float fac[2] = {0.5f * dtdx[1], 0.5f * dtdx[2]};
        tile_delta<0>(sF1 + 3 * 5 * NR, NR, t, t + 32, dl[0]);
#pragma unroll
        for (int m = 0; m < 5; m++) dl[1][m] = fzy_c[comp<0>(m) * NR + t] - fzy_p[comp<0>(m) * NR + t];
        tile_correct<2>(qm, qp, dl, fac, gamma, igm1, em, ep);
        const EdgeF lp = shfl_up_edge(ep);
        if (fc_x && int_y) {
          tile_flux<RS>(lp, em, gamma, igm1, Fn);
          tile_wall<0>(b, gx, Fn);
          tile_store<0>(sFX, NR, t, Fn);
        }
      }
#pragma unroll
      for (int m = 0; m < 5; m++) {
        qm[m] = ty_p[m * NR + t];
        qp[m] = ty_p[(5 + m) * NR + t];
      }
      {
        const float fac[2] = {0.5f * dtdx[2], 0.5f * dtdx[0]};
#pragma unroll
        for (int m = 0; m < 5; m++) dl[0][m] = fzx_c[comp<1>(m) * NR + t] - fzx_p[comp<1>(m) * NR + t];
        tile_delta<1>(sF1 + 1 * 5 * NR, NR, t, t + 1, dl[1]);
        tile_correct<2>(qm, qp, dl, fac, gamma, igm1, em, ep);
        put_edge(ex0, NR, t, ep);
      }
      __syncthreads();
      if (fc_y && int_x) {
        const EdgeF lp = get_edge(ex0, NR, t - 32);
        tile_flux<RS>(lp, em, gamma, igm1, Fn);
        tile_wall<1>(b, gy, Fn);
        tile_store<1>(sFY, NR, t, Fn);
      }
    }
    __syncthreads();
  }
}


// ------------------------------------------------------------ persistent form
// One launch advances every box by K steps.  Its blocks take work blocks from
// a queue ordered by step, then stage, then table order (box by box); the
// body of a work block is the stage kernel's own (the b_* functions, compiled
// once and called by both forms, so the results are bitwise the same).  A work
// block of stage s of box b waits until the box's done count reaches the
// number of its blocks in every stage before s (earlier steps included):
// every such block was taken from the queue before this one by a block that
// is running, so the wait ends without any assumption about how many blocks
// are resident.  A wait polls at most spin_limit times; then the kernel
// records HYDRO_ERR_TIMEOUT, and every block leaves at its next queue access or
// poll.  A block takes PERSIST_CHUNK consecutive work blocks per queue access
// and runs them in order, publishing each as it finishes (a later one may wait
// for an earlier one of the same chunk).  Completion is published with a
// fence and an atomic add after the block's barrier; a waiter's thread 0
// acquires the count and its block's barrier orders the reads after it.
struct PersistArgs {
  TableView tv[NPSTAGES];
  long long prefix[NPSTAGES + 1];  // work blocks of one step before each stage
  const DevBox* boxes;
  BoxRt* rt;
  double* state;
  unsigned char* work;
  PersistHead* head;
  unsigned long long* done;
  const long long* need;
  const double* dt_in;
  long long nsteps;
  long long spin_limit;
  int stall_box;
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// SLOTS: which compute types the handle holds (1 FP64, 2 FP32, 3 both); a
// kernel that calls only one type's stage bodies needs fewer registers.
template <int LIM, int RS, int SLOTS>
__global__ void __launch_bounds__(PERSIST_THREADS) k_persist(const __grid_constant__ PersistArgs a) {
  __shared__ long long s_base;
  __shared__ int s_stage, s_box, s_blk, s_item, s_ok;
  const long long per_step = a.prefix[NPSTAGES];
  const long long total = per_step * a.nsteps;
  int last_st = -1, last_i = 0;  // thread 0: the table item found last (work blocks come in order)
  for (;;) {
    // take PERSIST_CHUNK consecutive work blocks (one queue access)
    if (threadIdx.x == 0) {
      long long base = -1;
      if (ld_relaxed_i32(&a.head->err) == 0) {
        const unsigned long long q = atomicAdd(&a.head->queue, (unsigned long long)PERSIST_CHUNK);
        if ((long long)q < total) base = (long long)q;
      }
      s_base = base;
    }
    __syncthreads();
    const long long base = s_base;
    if (base < 0) return;
    const long long end = min(base + PERSIST_CHUNK, total);
    for (long long it = base; it < end; it++) {
      if (threadIdx.x == 0) {
        const long long step = it / per_step, r = it - step * per_step;
        int st = 0;
        while (a.prefix[st + 1] <= r) st++;
        const int blk = (int)(r - a.prefix[st]);
        const TableView& w = a.tv[st];
        int i;
        if (st == last_st && __ldg(w.start + last_i) <= blk) {
          i = last_i;  // the chunk's blocks are consecutive: walk forward from the last item
          while (__ldg(w.start + i + 1) <= blk) i++;
        } else {
          int lo = 0, hi = w.nitems;
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(w.start + mid) <= blk) lo = mid;
            else hi = mid;
          }
          i = lo;
        }
        last_st = st;
        last_i = i;
        const int box = __ldg(w.item + i) >> 3;
        long long need = step * a.need[box * (NPSTAGES + 1) + NPSTAGES] + a.need[box * (NPSTAGES + 1) + st];
        if (box == a.stall_box && st == PS_FILL_Y) need += 1;  // a count nothing will reach
        int ok = 1;
        long long polls = 0;
        while ((long long)ld_acquire_u64(a.done + box) < need) {
          if (++polls > a.spin_limit || ld_relaxed_i32(&a.head->err) != 0) {
            atomicCAS(&a.head->err, 0, HYDRO_ERR_TIMEOUT);
            ok = 0;
            break;
          }
          __nanosleep(128);
        }
        s_stage = st;
        s_box = box;
        s_blk = blk;
        s_item = i;
        s_ok = ok;
      }
      __syncthreads();  // with the acquire above: the box's earlier results are visible to the block
      if (!s_ok) return;
      const int st = s_stage, bx = s_box, vb = s_blk;
      // a one-item view of the table: the body's own search is then trivial
      const TableView tv{a.tv[st].start + s_item, a.tv[st].item + s_item, 1};
      constexpr bool D = (SLOTS & 1) != 0, F = (SLOTS & 2) != 0;
      switch (st) {
        case PS_FILL_X: b_fill<0>(tv, vb, a.boxes, a.state); break;
        case PS_FILL_Y: b_fill<1>(tv, vb, a.boxes, a.state); break;
        case PS_FILL_Z: b_fill<2>(tv, vb, a.boxes, a.state); break;
        case PS_PRIM: b_prim<LIM == HYDRO_LIMITER_CS08>(tv, vb, a.boxes, a.state, a.work, a.rt); break;
        case PS_DT:
          if (threadIdx.x == 0) b_dt_box(a.boxes, a.rt, bx, a.dt_in, nullptr, 1);
          break;
        case PS_FLATTEN_D: if constexpr (D) b_flatten<double>(tv, vb, a.boxes, a.work); break;
        case PS_FLATTEN_F: if constexpr (F) b_flatten<float>(tv, vb, a.boxes, a.work); break;
        case PS_SLOPES_D: if constexpr (D) b_slopes<double, LIM>(tv, vb, a.boxes, a.work); break;
        case PS_SLOPES_F: if constexpr (F) b_slopes<float, LIM>(tv, vb, a.boxes, a.work); break;
        case PS_TRACE_D: if constexpr (D) b_trace<double, LIM>(tv, vb, a.boxes, a.rt, a.work); break;
        case PS_TRACE_F: if constexpr (F) b_trace<float, LIM>(tv, vb, a.boxes, a.rt, a.work); break;
        case PS_LINE_X: if constexpr (F) b_line_x<float, RS>(tv, vb, a.boxes, a.rt, a.work); break;
        case PS_LINE_YZ: if constexpr (F) b_line_yz<float, RS>(tv, vb, a.boxes, a.rt, a.work); break;
        case PS_RIEMANN_D: if constexpr (D) b_riemann<double, RS>(tv, vb, a.boxes, a.work); break;
        case PS_RIEMANN_F: if constexpr (F) b_riemann<float, RS>(tv, vb, a.boxes, a.work); break;
        case PS_CTU1_D: if constexpr (D) b_ctu1<double, RS>(tv, vb, a.boxes, a.rt, a.work); break;
        case PS_CTU1_F: if constexpr (F) b_ctu1<float, RS>(tv, vb, a.boxes, a.rt, a.work); break;
        case PS_CTU1_LINE: if constexpr (F) b_ctu1_line<float, RS>(tv, vb, a.boxes, a.rt, a.work); break;
        case PS_CTU2_D: if constexpr (D) b_ctu2<double, RS>(tv, vb, a.boxes, a.rt, a.work); break;
        case PS_CTU2_F: if constexpr (F) b_ctu2<float, RS>(tv, vb, a.boxes, a.rt, a.work); break;
        case PS_CTU2_LINE: if constexpr (F) b_ctu2_line<float, RS>(tv, vb, a.boxes, a.rt, a.work); break;
        default: b_update(tv, vb, a.boxes, a.rt, a.state, a.work, 0); break;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();  // the block's writes before the count that publishes them
        atomicAdd(a.done + bx, 1ull);
      }
    }
  }
}

// ----------------------------------------------------- host staging transfers
__global__ void __launch_bounds__(256) k_scatter(TableView tv, const DevBox* __restrict__ boxes,
                                                 double* __restrict__ state, const double* __restrict__ stage) {
  LOCATE(tv)
  int lo[3] = {0, 0, 0}, ext[3] = {b.n[0], b.n[1], b.n[2]}, c[3];
  if (!decode(t_, lo, ext, c)) return;
  const long long Z = zone(b, c[0], c[1], c[2]);
  const long long N = (long long)b.n[0] * b.n[1] * b.n[2];
  const long long src = b.stage_off + ((long long)c[2] * b.n[1] + c[1]) * b.n[0] + c[0];
#pragma unroll
  for (int v = 0; v < 5; v++) state[b.state_off + v * b.vs + Z] = stage[src + v * N];
}

__global__ void __launch_bounds__(256) k_gather(TableView tv, const DevBox* __restrict__ boxes,
                                                const double* __restrict__ state, double* __restrict__ stage) {
  LOCATE(tv)
  int lo[3] = {0, 0, 0}, ext[3] = {b.n[0], b.n[1], b.n[2]}, c[3];
  if (!decode(t_, lo, ext, c)) return;
  const long long Z = zone(b, c[0], c[1], c[2]);
  const long long N = (long long)b.n[0] * b.n[1] * b.n[2];
  const long long dst = b.stage_off + ((long long)c[2] * b.n[1] + c[1]) * b.n[0] + c[0];
#pragma unroll
  for (int v = 0; v < 5; v++) stage[dst + v * N] = state[b.state_off + v * b.vs + Z];
}

}  // namespace

const char* const STAGE_NAMES[NSTAGES] = {"fill_ghosts", "prim", "dt", "flatten", "slopes", "trace",
                                           "riemann", "ctu1", "ctu2", "tile", "update"};

const char* const TABLE_NAMES[NTABLES] = {"fill_x", "fill_y", "fill_z", "prim", "update", "flatten",
                                           "slopes", "trace", "riemann", "ctu1", "ctu2", "line_x", "line_yz",
                                           "ctu2_line", "ctu1_line", "tile"};

int default_tpb(int table) {
  switch (table) {
    case TB_TRACE:
    case TB_LINE_X:
    case TB_LINE_YZ:
    case TB_CTU2_LINE:
    case TB_CTU1_LINE:
    case TB_RIEMANN:
    case TB_CTU1:
    case TB_CTU2:
    case TB_FLATTEN:
      return 128;
    default:
      return 256;
  }
}

// Threads of work item (box d, axis or pair z) of a table: the region the
// matching kernel decodes.
long long item_volume(const hydro_box_desc& d, int table, int z) {
  const long long n[3] = {d.nx, d.ny, d.nz};
  const long long g2 = 2 * NG;
  switch (table) {
    case TB_FILL_X: return g2 * n[1] * n[2];
    case TB_FILL_Y: return (n[0] + g2) * g2 * n[2];
    case TB_FILL_Z: return (n[0] + g2) * (n[1] + g2) * g2;
    case TB_PRIM: return (n[0] + g2) * (n[1] + g2) * (n[2] + g2);
    case TB_UPDATE: return n[0] * n[1] * n[2];
    case TB_FLATTEN:
    case TB_TRACE: return (n[0] + 2) * (n[1] + 2) * (n[2] + 2);
    case TB_SLOPES: return (n[z] + 4) * (n[(z + 1) % 3] + 2) * (n[(z + 2) % 3] + 2);
    case TB_RIEMANN: return (n[z] + 1) * (n[(z + 1) % 3] + 2) * (n[(z + 2) % 3] + 2);
    case TB_CTU1: {  // z = pair slot of (D, T)
      const int dd = z / 2, r = z % 2, tt = r < dd ? r : r + 1, uu = 3 - dd - tt;
      return (n[dd] + 1) * n[tt] * (n[uu] + 2);
    }
    case TB_CTU2: return (n[z] + 1) * n[(z + 1) % 3] * n[(z + 2) % 3];
    case TB_LINE_X: return (n[1] + 2) * (n[2] + 2) * ((n[0] + 2 + LINE_X_OUT - 1) / LINE_X_OUT) * 32;
    case TB_LINE_YZ: {
      const int dd = z + 1;  // walk axis: y, then z
      return (n[0] + 2) * (n[dd == 1 ? 2 : 1] + 2) * ((n[dd] + 2 + LINE_SEG - 1) / LINE_SEG);
    }
    case TB_CTU2_LINE:
      if (z == 0) return n[1] * n[2] * ((n[0] + 1 + 30) / 31) * 32;
      return n[0] * n[z == 1 ? 2 : 1] * ((n[z] + 1 + LINE_SEG - 1) / LINE_SEG);
    case TB_CTU1_LINE: {
      const int dd = z / 2, r = z % 2;  // pair slot -> (D, T)
      const int tt = r == 0 ? (dd == 0 ? 1 : 0) : (dd == 2 ? 1 : 2);
      const int uu = 3 - dd - tt;
      long long ext[3];
      ext[tt] = n[tt];
      ext[uu] = n[uu] + 2;
      if (dd == 0) return ext[1] * ext[2] * ((n[0] + 1 + 30) / 31) * 32;
      return ext[0] * ext[dd == 1 ? 2 : 1] * ((n[dd] + 1 + LINE_SEG - 1) / LINE_SEG);
    }
    default: return 0;
  }
}

int build_table(const Plan& p, int table, int slot, int tpb, int order, int* start, int* item) {
  struct It {
    int code;
    int blocks;
  };
  std::vector<It> items;
  for (int b = 0; b < p.nboxes; b++) {
    if (!p.boxes[b].active) continue;
    const hydro_box_desc& d = p.boxes[b].d;
    if (TABLE_PER_PRECISION[table] && (d.precision == HYDRO_MIXED) != (slot == 1)) continue;
    if (table == TB_TILE) {  // one block per tile and z-segment
      items.push_back({b * 8, (int)tile_blocks(d, p.tile_ty, p.tile_seg)});
      continue;
    }
    for (int z = 0; z < TABLE_ZDIM[table]; z++) {
      const long long v = item_volume(d, table, z);
      items.push_back({b * 8 + z, (int)((v + tpb - 1) / tpb)});
    }
  }
  if (order == 1)
    std::stable_sort(items.begin(), items.end(), [](const It& a, const It& c) { return a.blocks > c.blocks; });
  int acc = 0;
  for (size_t i = 0; i < items.size(); i++) {
    start[i] = acc;
    item[i] = items[i].code;
    acc += items[i].blocks;
  }
  start[items.size()] = acc;
  return (int)items.size();
}

namespace {

TableView view(const WorkTable& w) { return TableView{w.start, w.item, w.nitems}; }

// Launches kernel `k` over table w, if it has work.
template <typename... A, typename... P>
int launch(void (*k)(TableView, A...), const WorkTable& w, cudaStream_t s, P... args) {
  if (w.nitems == 0) return 0;
  k<<<w.blocks, w.tpb, 0, s>>>(view(w), args...);
  return 1;
}

// Launches the compute-type-R kernel of a per-precision table over w with the
// handle's method variant; returns 1 if it had work.
template <typename R>
int launch_typed(const Plan& p, int table, const WorkTable& w, cudaStream_t s) {
  const BoxRt* rt = p.rt;
  const bool cs = p.limiter == HYDRO_LIMITER_CS08;
  const bool ts = p.riemann == HYDRO_RIEMANN_TWO_SHOCK;
  switch (table) {
    case TB_FLATTEN: return launch(k_flatten<R>, w, s, p.dboxes, p.work);
    case TB_SLOPES:
      return cs ? launch(k_slopes<R, HYDRO_LIMITER_CS08>, w, s, p.dboxes, p.work)
                : launch(k_slopes<R, HYDRO_LIMITER_CW84>, w, s, p.dboxes, p.work);
    case TB_TRACE:
      return cs ? launch(k_trace<R, HYDRO_LIMITER_CS08>, w, s, p.dboxes, rt, p.work)
                : launch(k_trace<R, HYDRO_LIMITER_CW84>, w, s, p.dboxes, rt, p.work);
    case TB_RIEMANN:
      return ts ? launch(k_riemann<R, HYDRO_RIEMANN_TWO_SHOCK>, w, s, p.dboxes, p.work)
                : launch(k_riemann<R, HYDRO_RIEMANN_HLLC>, w, s, p.dboxes, p.work);
    case TB_CTU1:
      return ts ? launch(k_ctu1<R, HYDRO_RIEMANN_TWO_SHOCK>, w, s, p.dboxes, rt, p.work)
                : launch(k_ctu1<R, HYDRO_RIEMANN_HLLC>, w, s, p.dboxes, rt, p.work);
    case TB_CTU2:
      return ts ? launch(k_ctu2<R, HYDRO_RIEMANN_TWO_SHOCK>, w, s, p.dboxes, rt, p.work)
                : launch(k_ctu2<R, HYDRO_RIEMANN_HLLC>, w, s, p.dboxes, rt, p.work);
    case TB_LINE_X:
    case TB_LINE_YZ:
    case TB_CTU2_LINE:
    case TB_CTU1_LINE:
      // the line kernels exist for FP32 boxes only (LINE_FUSED_SLOT)
      if constexpr (Consts<R>::STORE_CONSERVED) {
        return 0;
      } else {
        if (table == TB_LINE_X)
          return ts ? launch(k_line_x<R, HYDRO_RIEMANN_TWO_SHOCK>, w, s, p.dboxes, rt, p.work)
                    : launch(k_line_x<R, HYDRO_RIEMANN_HLLC>, w, s, p.dboxes, rt, p.work);
        if (table == TB_LINE_YZ)
          return ts ? launch(k_line_yz<R, HYDRO_RIEMANN_TWO_SHOCK>, w, s, p.dboxes, rt, p.work)
                    : launch(k_line_yz<R, HYDRO_RIEMANN_HLLC>, w, s, p.dboxes, rt, p.work);
        if (table == TB_CTU1_LINE)
          return ts ? launch(k_ctu1_line<R, HYDRO_RIEMANN_TWO_SHOCK>, w, s, p.dboxes, rt, p.work)
                    : launch(k_ctu1_line<R, HYDRO_RIEMANN_HLLC>, w, s, p.dboxes, rt, p.work);
        return ts ? launch(k_ctu2_line<R, HYDRO_RIEMANN_TWO_SHOCK>, w, s, p.dboxes, rt, p.work)
                  : launch(k_ctu2_line<R, HYDRO_RIEMANN_HLLC>, w, s, p.dboxes, rt, p.work);
      }
    default: return 0;
  }
}

// Stage table of one compute type, with the line kernels standing in where
// they apply: the fused line stage for slopes (nothing), tracing (the x and
// y/z line kernels) and the normal Riemann solves (nothing), and the zone-wise
// CTU stages for the face-wise ones.
template <typename R>
int launch_slot(const Plan& p, int table, int slot, cudaStream_t s) {
  if (tile_fused(p, slot) &&
      (table == TB_SLOPES || table == TB_TRACE || table == TB_RIEMANN || table == TB_CTU1 || table == TB_CTU2))
    return 0;
  if (line_fused(p, slot)) {
    if (table == TB_SLOPES || table == TB_RIEMANN) return 0;
    if (table == TB_TRACE)
      return launch_typed<R>(p, TB_LINE_X, p.tab[TB_LINE_X][slot], s) +
             launch_typed<R>(p, TB_LINE_YZ, p.tab[TB_LINE_YZ][slot], s);
    if (table == TB_CTU1) return launch_typed<R>(p, TB_CTU1_LINE, p.tab[TB_CTU1_LINE][slot], s);
    if (table == TB_CTU2) return launch_typed<R>(p, TB_CTU2_LINE, p.tab[TB_CTU2_LINE][slot], s);
  }
  return launch_typed<R>(p, table, p.tab[table][slot], s);
}

// The fused tile stage for FP32 boxes, if the plan runs it.
template <int TY, int RS>
int launch_tile_kernel(const Plan& p, const WorkTable& w, cudaStream_t s) {
  if (w.nitems == 0) return 0;
  const int seg = p.tile_seg > 0 ? p.tile_seg : (1 << 30);
  k_tile<TY, RS><<<w.blocks, TileShape<TY>::NR, TileShape<TY>::BYTES, s>>>(view(w), p.dboxes, p.rt, p.state, p.work,
                                                                          seg);
  return 1;
}

int launch_tiles(const Plan& p, cudaStream_t s) {
  if (!tile_fused(p, 1)) return 0;
  const WorkTable& w = p.tab[TB_TILE][1];
  const bool ts = p.riemann == HYDRO_RIEMANN_TWO_SHOCK;
  if (p.tile_ty == TILE_TYS[0])
    return ts ? launch_tile_kernel<TILE_TYS[0], HYDRO_RIEMANN_TWO_SHOCK>(p, w, s)
              : launch_tile_kernel<TILE_TYS[0], HYDRO_RIEMANN_HLLC>(p, w, s);
  return ts ? launch_tile_kernel<TILE_TYS[1], HYDRO_RIEMANN_TWO_SHOCK>(p, w, s)
            : launch_tile_kernel<TILE_TYS[1], HYDRO_RIEMANN_HLLC>(p, w, s);
}

// Both compute types of a per-precision table.
int launch_both(const Plan& p, int table, cudaStream_t s) {
  return launch_slot<double>(p, table, 0, s) + launch_slot<float>(p, table, 1, s);
}

}  // namespace

cudaError_t launch_stage(const Plan& p, Stage st, cudaStream_t stream, const double* dt_in, double* dt_out,
                         int advance, int* launched) {
  int n = 0;
  const auto& T = p.tab;
  switch (st) {
    case ST_FILL:
      n += launch(k_fill<0>, T[TB_FILL_X][0], stream, p.dboxes, p.state);
      n += launch(k_fill<1>, T[TB_FILL_Y][0], stream, p.dboxes, p.state);
      n += launch(k_fill<2>, T[TB_FILL_Z][0], stream, p.dboxes, p.state);
      break;
    case ST_PRIM:
      if (p.limiter == HYDRO_LIMITER_CS08)
        n += launch(k_prim<true>, T[TB_PRIM][0], stream, p.dboxes, (const double*)p.state, p.work, p.rt);
      else
        n += launch(k_prim<false>, T[TB_PRIM][0], stream, p.dboxes, (const double*)p.state, p.work, p.rt);
      break;
    case ST_DT:
      if (p.shared_dt && !dt_in)
        k_dt_shared<<<1, 256, 0, stream>>>(p.dboxes, p.rt, p.nboxes, dt_out, advance);
      else
        k_dt<<<(p.nboxes + 255) / 256, 256, 0, stream>>>(p.dboxes, p.rt, p.nboxes, dt_in, dt_out, advance);
      n = 1;
      break;
    case ST_FLATTEN: n += launch_both(p, TB_FLATTEN, stream); break;
    case ST_SLOPES: n += launch_both(p, TB_SLOPES, stream); break;
    case ST_TRACE: n += launch_both(p, TB_TRACE, stream); break;
    case ST_RIEMANN: n += launch_both(p, TB_RIEMANN, stream); break;
    case ST_CTU1: n += launch_both(p, TB_CTU1, stream); break;
    case ST_CTU2: n += launch_both(p, TB_CTU2, stream); break;
    case ST_TILE:
      n += launch_tiles(p, stream);
      break;
    case ST_UPDATE:
      n += launch(k_update, T[TB_UPDATE][0], stream, p.dboxes, p.rt, p.state, p.work, tile_fused(p, 1) ? 1 : 0);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  if (launched) *launched = n;
  return cudaGetLastError();
}

cudaError_t launch_table(const Plan& p, int table, int slot, cudaStream_t stream) {
  const WorkTable& w = p.tab[table][slot];
  switch (table) {
    case TB_FILL_X: launch(k_fill<0>, w, stream, p.dboxes, p.state); break;
    case TB_FILL_Y: launch(k_fill<1>, w, stream, p.dboxes, p.state); break;
    case TB_FILL_Z: launch(k_fill<2>, w, stream, p.dboxes, p.state); break;
    case TB_PRIM:
      if (p.limiter == HYDRO_LIMITER_CS08) launch(k_prim<true>, w, stream, p.dboxes, (const double*)p.state, p.work, p.rt);
      else launch(k_prim<false>, w, stream, p.dboxes, (const double*)p.state, p.work, p.rt);
      break;
    case TB_FLATTEN:
    case TB_SLOPES:
    case TB_TRACE:
    case TB_RIEMANN:
    case TB_CTU1:
    case TB_CTU2:
    case TB_LINE_X:
    case TB_LINE_YZ:
    case TB_CTU2_LINE:
    case TB_CTU1_LINE:
      if (slot == 0) launch_typed<double>(p, table, w, stream);
      else launch_typed<float>(p, table, w, stream);
      break;
    case TB_TILE:  // updates the state: the autotuner saves and restores it around this
      launch_tiles(p, stream);
      break;
    default:
      return cudaErrorInvalidValue;  // the update changes the state and is not relaunched
  }
  return cudaGetLastError();
}

void persist_stage_table(int st, int* table, int* slot) {
  static const int T[NPSTAGES] = {TB_FILL_X,  TB_FILL_Y,  TB_FILL_Z,    TB_PRIM,      -1,          TB_FLATTEN,
                                  TB_FLATTEN, TB_SLOPES,  TB_SLOPES,    TB_TRACE,     TB_TRACE,    TB_LINE_X,
                                  TB_LINE_YZ, TB_RIEMANN, TB_RIEMANN,   TB_CTU1,      TB_CTU1,     TB_CTU1_LINE,
                                  TB_CTU2,    TB_CTU2,    TB_CTU2_LINE, TB_UPDATE};
  static const int S[NPSTAGES] = {0, 0, 0, 0, 0, 0, 1, 0, 1, 0, 1, 1, 1, 0, 1, 0, 1, 1, 0, 1, 1, 0};
  *table = T[st];
  *slot = S[st];
}

bool persist_stage_runs(const Plan& p, int st) {
  int t, sl;
  persist_stage_table(st, &t, &sl);
  if (t < 0) return true;  // the per-box dt
  const bool line = t == TB_LINE_X || t == TB_LINE_YZ || t == TB_CTU1_LINE || t == TB_CTU2_LINE;
  const bool replaced = t == TB_SLOPES || t == TB_TRACE || t == TB_RIEMANN || t == TB_CTU1 || t == TB_CTU2;
  if (line) return line_fused(p, sl);
  if (replaced) return !line_fused(p, sl);
  return true;
}

namespace {
// The persistent kernel for the plan's method and compute types.
template <int LIM, int RS>
void (*persist_kernel_m(int slots))(PersistArgs) {
  if (slots == 1) return k_persist<LIM, RS, 1>;
  if (slots == 2) return k_persist<LIM, RS, 2>;
  return k_persist<LIM, RS, 3>;
}

void (*persist_kernel(const Plan& p))(PersistArgs) {
  const int slots = (p.has_fp64 ? 1 : 0) | (p.has_mixed ? 2 : 0);
  const bool cs = p.limiter == HYDRO_LIMITER_CS08, ts = p.riemann == HYDRO_RIEMANN_TWO_SHOCK;
  if (cs) return ts ? persist_kernel_m<HYDRO_LIMITER_CS08, HYDRO_RIEMANN_TWO_SHOCK>(slots)
                    : persist_kernel_m<HYDRO_LIMITER_CS08, HYDRO_RIEMANN_HLLC>(slots);
  return ts ? persist_kernel_m<HYDRO_LIMITER_CW84, HYDRO_RIEMANN_TWO_SHOCK>(slots)
            : persist_kernel_m<HYDRO_LIMITER_CW84, HYDRO_RIEMANN_HLLC>(slots);
}
}  // namespace

cudaError_t persist_occupancy(const Plan& p, int* n) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, persist_kernel(p), PERSIST_THREADS, 0);
}

cudaError_t launch_persistent(const Plan& p, const double* dt_in, int nsteps, cudaStream_t stream) {
  PersistArgs a;
  memset(&a, 0, sizeof a);
  long long acc = 0;
  for (int st = 0; st < NPSTAGES; st++) {
    a.prefix[st] = acc;
    int t, sl;
    persist_stage_table(st, &t, &sl);
    if (t < 0) {
      a.tv[st] = TableView{p.p_dt_start, p.p_dt_item, p.p_dt_items};
      acc += p.p_dt_items;
    } else if (persist_stage_runs(p, st) && p.tab[t][sl].nitems > 0) {
      a.tv[st] = view(p.tab[t][sl]);
      acc += p.tab[t][sl].blocks;
    } else {
      a.tv[st] = TableView{nullptr, nullptr, 0};
    }
  }
  a.prefix[NPSTAGES] = acc;
  a.boxes = p.dboxes;
  a.rt = p.rt;
  a.state = p.state;
  a.work = p.work;
  a.head = p.p_head;
  a.done = p.p_done;
  a.need = p.p_need;
  a.dt_in = dt_in;
  a.nsteps = nsteps;
  a.spin_limit = p.spin_limit;
  a.stall_box = p.stall_box;
  persist_kernel(p)<<<dim3(p.persist_grid), dim3(PERSIST_THREADS), 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t prepare_tile_kernels() {
  static cudaError_t done = cudaErrorNotReady;
  if (done == cudaSuccess) return done;
  cudaError_t e = cudaFuncSetAttribute(k_tile<TILE_TYS[0], HYDRO_RIEMANN_HLLC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)TileShape<TILE_TYS[0]>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tile<TILE_TYS[0], HYDRO_RIEMANN_TWO_SHOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TileShape<TILE_TYS[0]>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tile<TILE_TYS[1], HYDRO_RIEMANN_HLLC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TileShape<TILE_TYS[1]>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tile<TILE_TYS[1], HYDRO_RIEMANN_TWO_SHOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TileShape<TILE_TYS[1]>::BYTES);
  done = e;
  return e;
}

cudaError_t launch_scatter(const Plan& p, const double* stage, cudaStream_t stream) {
  launch(k_scatter, p.tab[TB_UPDATE][0], stream, p.dboxes, p.state, stage);
  return cudaGetLastError();
}

cudaError_t launch_gather(const Plan& p, double* stage, cudaStream_t stream) {
  launch(k_gather, p.tab[TB_UPDATE][0], stream, p.dboxes, (const double*)p.state, stage);
  return cudaGetLastError();
}

}  // namespace hydro
