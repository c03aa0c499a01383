// Conserved -> primitive conversion of one zone in FP64 and the zone's
// largest signal rate, shared by the primitive stage (k_prim) and the
// allocation-free time step, so that both form bitwise the same speeds.
//
// rho is floored at SMALL_DENS, u = m / rho from one refined reciprocal,
// p = (gamma - 1)(E - rho/2 |u|^2) floored at SMALL_PRES, and one refined
// reciprocal square root of c^2 = gamma p / rho gives 1/c and c = c^2 (1/c).
// gm1 = gamma - 1 (the box's stored difference, the same double).  The
// products are formed on the integer pipe (imul_rn, bitwise __dmul_rn).
#pragma once

#include "fp64_fast.cuh"
#include "hydro_internal.cuh"

namespace hydro {

struct PrimZone {
  double rho, u, v, w, p, cs;
  double ir;  // 1 / rho
  double ic;  // 1 / c
};

template <typename M>
__device__ __forceinline__ PrimZone prim_zone_m(double rho, double mx, double my, double mz, double E, double gamma,
                                                double gm1, M& mul) {
  // every operation written out with its rounding (fused where the product
  // feeds a sum), so that no kernel that inlines this can contract it
  // differently from another; the products are taken by a multiplication
  // policy (all of them correctly rounded)
  PrimZone z;
  if (dgt(SMALL_DENS, rho)) rho = SMALL_DENS;
  z.rho = rho;
  z.ir = nr_rcp(rho);
  z.u = mul(mx, z.ir);
  z.v = mul(my, z.ir);
  z.w = mul(mz, z.ir);
  const double uu = __fma_rn(z.w, z.w, __fma_rn(z.v, z.v, mul(z.u, z.u)));
  double p = mul(gm1, __fma_rn(-half_of(rho), uu, E));  // -rho/2 exactly
  if (dgt(SMALL_PRES, p)) p = SMALL_PRES;
  z.p = p;
  const double c2 = mul(mul(gamma, p), z.ir);
  z.ic = nr_rsqrt(c2, mul);
  z.cs = mul(c2, z.ic);
  return z;
}

// The products on the integer pipe; a warp with a flagged lane redoes that
// lane's conversion with the FP64 multiply (the same bits).
__device__ __forceinline__ PrimZone prim_zone(double rho, double mx, double my, double mz, double E,
                                              double gamma, double gm1) {
  IntMul im;
  PrimZone z = prim_zone_m(rho, mx, my, mz, E, gamma, gm1, im);
  if (__any_sync(__activemask(), im.bad != 0u)) {
    if (im.bad) {
      InsnMul nm;
      z = prim_zone_m(rho, mx, my, mz, E, gamma, gm1, nm);
    }
  }
  return z;
}

// max over the axes d of (|u_d| + c) / dx_d, given idx[d] = 1 / dx_d.  With
// one 1/dx for all axes (cubic zones) it is (max_d |u_d| + c) / dx: rounded
// addition and multiplication by a positive number are non-decreasing, so
// taking the maximum first gives the same double, for one addition and one
// multiplication instead of three each (the test and the maximum of the
// magnitudes run on the integer pipe).
__device__ __forceinline__ bool same_double(double a, double b) {
  return ((__double2hiint(a) ^ __double2hiint(b)) | (__double2loint(a) ^ __double2loint(b))) == 0;
}
__device__ __forceinline__ double signal_rate(double u, double v, double w, double cs, const double* idx) {
  if (same_double(idx[0], idx[1]) & same_double(idx[1], idx[2]))
    return __dmul_rn(__dadd_rn(dmax(dmax(fabs(u), fabs(v)), fabs(w)), cs), idx[0]);
  return dmax(dmax(__dmul_rn(__dadd_rn(fabs(u), cs), idx[0]), __dmul_rn(__dadd_rn(fabs(v), cs), idx[1])),
              __dmul_rn(__dadd_rn(fabs(w), cs), idx[2]));
}

}  // namespace hydro
