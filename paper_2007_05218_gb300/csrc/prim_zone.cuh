// Conserved -> primitive conversion of one zone in FP64 and the zone's
// largest signal rate, shared by the primitive stage (k_prim) and the
// allocation-free time step, so that both form bitwise the same speeds.
//
// rho is floored at SMALL_DENS, u = m / rho from one refined reciprocal,
// p = (gamma - 1)(E - rho/2 |u|^2) floored at SMALL_PRES, and one refined
// reciprocal square root of c^2 = gamma p / rho gives 1/c and c = c^2 (1/c).
#pragma once

#include "fp64_fast.cuh"
#include "hydro_internal.cuh"

namespace hydro {

struct PrimZone {
  double rho, u, v, w, p, cs;
  double ir;  // 1 / rho
  double ic;  // 1 / c
};

__device__ __forceinline__ PrimZone prim_zone(double rho, double mx, double my, double mz, double E,
                                              double gamma) {
  PrimZone z;
  if (dgt(SMALL_DENS, rho)) rho = SMALL_DENS;
  z.rho = rho;
  z.ir = nr_rcp(rho);
  z.u = mx * z.ir;
  z.v = my * z.ir;
  z.w = mz * z.ir;
  double p = (gamma - 1.0) * (E - 0.5 * rho * (z.u * z.u + z.v * z.v + z.w * z.w));
  if (dgt(SMALL_PRES, p)) p = SMALL_PRES;
  z.p = p;
  const double c2 = gamma * p * z.ir;
  z.ic = nr_rsqrt(c2);
  z.cs = c2 * z.ic;
  return z;
}

// max over the axes d of (|u_d| + c) / dx_d, given idx[d] = 1 / dx_d
__device__ __forceinline__ double signal_rate(double u, double v, double w, double cs, const double* idx) {
  return dmax(dmax((fabs(u) + cs) * idx[0], (fabs(v) + cs) * idx[1]), (fabs(w) + cs) * idx[2]);
}

}  // namespace hydro
