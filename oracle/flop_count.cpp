/*
 * ORACLE TOOLING -- TEST INFRASTRUCTURE ONLY.
 *
 * Counts the floating-point operations of the oracle's stages by compiling
 * hydro_oracle.cpp unchanged with `double` replaced by a counting number type.
 * The counts define the algorithmic FP64 work per unit (zone, zone-direction
 * or face) of each stage of the method, which the benchmark divides by the
 * measured kernel time for its roofline.  Operations counted: add/sub, mul,
 * div, sqrt (the flops), plus comparisons and min/max separately.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

struct OpCounts {
  long long add, mul, div, sqrt, cmp, minmax;
};
static OpCounts g_ops;

struct cd {
  double v;
  cd() = default;
  cd(double x) : v(x) {}
  cd& operator+=(cd o) { g_ops.add++; v += o.v; return *this; }
  cd& operator-=(cd o) { g_ops.add++; v -= o.v; return *this; }
  cd operator-() const { return cd(-v); }
};
static inline cd operator+(cd a, cd b) { g_ops.add++; return cd(a.v + b.v); }
static inline cd operator-(cd a, cd b) { g_ops.add++; return cd(a.v - b.v); }
static inline cd operator*(cd a, cd b) { g_ops.mul++; return cd(a.v * b.v); }
static inline cd operator/(cd a, cd b) { g_ops.div++; return cd(a.v / b.v); }
static inline bool operator<(cd a, cd b) { g_ops.cmp++; return a.v < b.v; }
static inline bool operator>(cd a, cd b) { g_ops.cmp++; return a.v > b.v; }
static inline bool operator<=(cd a, cd b) { g_ops.cmp++; return a.v <= b.v; }
static inline bool operator>=(cd a, cd b) { g_ops.cmp++; return a.v >= b.v; }
static inline bool operator==(cd a, cd b) { g_ops.cmp++; return a.v == b.v; }
static inline bool operator!=(cd a, cd b) { g_ops.cmp++; return a.v != b.v; }
static inline cd sqrt(cd a) { g_ops.sqrt++; return cd(::sqrt(a.v)); }
static inline cd fabs(cd a) { return cd(::fabs(a.v)); }
static inline cd copysign(cd a, cd b) { return cd(::copysign(a.v, b.v)); }
static inline cd fmin(cd a, cd b) { g_ops.minmax++; return cd(::fmin(a.v, b.v)); }
static inline cd fmax(cd a, cd b) { g_ops.minmax++; return cd(::fmax(a.v, b.v)); }

#define double cd
#include "hydro_oracle.cpp"
#undef double

namespace {
OpCounts diff(const OpCounts& a, const OpCounts& b) {
  OpCounts d = {a.add - b.add, a.mul - b.mul, a.div - b.div, a.sqrt - b.sqrt, a.cmp - b.cmp,
                a.minmax - b.minmax};
  return d;
}
void put(long long* out, const OpCounts& c) {
  out[0] = c.add; out[1] = c.mul; out[2] = c.div; out[3] = c.sqrt; out[4] = c.cmp; out[5] = c.minmax;
}
}  // namespace

extern "C" {

/* Runs one oracle step (ghosts of U already filled) with the given dt and
 * writes, per stage (prim, dt, flatten, trace, riemann, ctu1, ctu2, update,
 * slopes), out[stage*6 + (add, mul, div, sqrt, cmp, minmax)] and units[stage]:
 * zones, zone-directions or faces the stage processed.  "trace" is the
 * interface values plus the zone parabolas and tracing; "slopes" the limited
 * slopes (per zone and axis of the slope region, five variables). */
int oracle_count_step(int nx, int ny, int nz, const double* dx, double gamma, double cfl, const int* bc,
                      const double* U_in, double dt_in, long long* out, long long* units) {
  ob_box b;
  b.nx = nx; b.ny = ny; b.nz = nz; b.ng = 4;
  for (int a = 0; a < 3; a++) b.dx[a] = cd(dx[a]);
  b.gamma = cd(gamma);
  b.cfl = cd(cfl);
  for (int f = 0; f < 6; f++) b.bc[f] = bc[f];
  b.limiter = 0;
  b.riemann = 0;
  if (!box_ok(&b)) return -1;
  Grid G(&b);
  cd* U = (cd*)calloc((size_t)5 * G.size, sizeof(cd));
  cd* W = (cd*)calloc((size_t)W_NFIELDS * G.size, sizeof(cd));
  for (long i = 0; i < 5 * G.size; i++) U[i] = cd(U_in[i]);
  cd dt(dt_in);
  const int n[3] = {nx, ny, nz};
  OpCounts s0 = g_ops;
  cons_to_prim_all(&b, G, U, W + (long)W_Q * G.size, W + (long)W_C * G.size);
  OpCounts s1 = g_ops;
  (void)compute_dt(&b, G, U);
  OpCounts s2 = g_ops;
  flatten_all(G, W + (long)W_Q * G.size, W + (long)W_CHI * G.size);
  OpCounts s3 = g_ops;
  /* trace_all, with the slopes counted apart from interfaces + zone tracing */
  cd* slope = (cd*)calloc((size_t)5 * G.size, sizeof(cd));
  cd* face = (cd*)calloc((size_t)5 * G.size, sizeof(cd));
  OpCounts sl = {0, 0, 0, 0, 0, 0};
  for (int d = 0; d < 3; d++) {
    OpCounts a = g_ops;
    limited_slopes_dir(G, d, W, slope);
    OpCounts bb = g_ops;
    OpCounts dd = diff(bb, a);
    sl.add += dd.add; sl.mul += dd.mul; sl.div += dd.div; sl.sqrt += dd.sqrt; sl.cmp += dd.cmp;
    sl.minmax += dd.minmax;
    interface_values_dir(G, d, W, slope, face);
    trace_zones_dir(&b, G, d, dt, W, face);
  }
  free(slope);
  free(face);
  OpCounts s4 = g_ops;
  OpCounts tr = diff(s4, s3); /* interface values + zone tracing: trace_all minus the slopes */
  tr.add -= sl.add; tr.mul -= sl.mul; tr.div -= sl.div; tr.sqrt -= sl.sqrt; tr.cmp -= sl.cmp;
  tr.minmax -= sl.minmax;
  normal_fluxes(&b, G, W);
  OpCounts s5 = g_ops;
  ctu_stage1(&b, G, dt, W);
  OpCounts s6 = g_ops;
  ctu_stage2(&b, G, dt, W);
  OpCounts s7 = g_ops;
  int ok = update(&b, G, dt, U, W);
  OpCounts s8 = g_ops;
  put(out + 0, diff(s1, s0));
  put(out + 6, diff(s2, s1));
  put(out + 12, diff(s3, s2));
  put(out + 18, tr);
  put(out + 24, diff(s5, s4));
  put(out + 30, diff(s6, s5));
  put(out + 36, diff(s7, s6));
  put(out + 42, diff(s8, s7));
  put(out + 48, sl);
  long long ext = (long long)(nx + 2) * (ny + 2) * (nz + 2);
  long long interior = (long long)nx * ny * nz;
  units[0] = G.size;
  units[1] = interior;
  units[2] = ext;
  units[3] = 3 * ext;
  units[4] = 0;
  units[5] = 0;
  units[6] = 0;
  for (int d = 0; d < 3; d++) {
    int e = (d + 1) % 3, f = (d + 2) % 3;
    units[4] += (long long)(n[d] + 1) * (n[e] + 2) * (n[f] + 2);
    units[5] += (long long)(n[d] + 1) * n[e] * (n[f] + 2) + (long long)(n[d] + 1) * n[f] * (n[e] + 2);
    units[6] += (long long)(n[d] + 1) * n[e] * n[f];
  }
  units[7] = interior;
  units[8] = 0;
  for (int d = 0; d < 3; d++) units[8] += (long long)(n[d] + 4) * (n[(d + 1) % 3] + 2) * (n[(d + 2) % 3] + 2);
  free(U);
  free(W);
  return ok ? 0 : -3;
}

}  /* extern "C" */
