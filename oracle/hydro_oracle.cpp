/*
 * ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct FP64 CPU implementation of one unsplit
 * PPM Godunov update of the 3D Euler equations for an ideal gamma-law gas
 * on a box with ghost zones.  Only the tests, the smoke check and the timed
 * CPU baseline of the benchmark may call it.  It shares no code, header,
 * table or constant with the CUDA library, and never runs on its behalf.
 *
 * What the paper fixes.  §3 ("Porting to GPUs") describes the core stencil:
 * limited slopes from neighbouring zones, then a polynomial reconstruction of
 * the fluid state.  §4 says the hydro is close to the one in Cholla, and §4.A
 * that the blast-wave test couples hydro and equation of state.  The paper
 * gives no formulas, so each stage below restates the published method it
 * names (Colella & Woodward 1984 = CW84; Colella 1990 and Saltzman 1994 for
 * the corner-transport-upwind (CTU) corrections; Toro, Spruce & Speares 1994
 * and Batten et al. 1997 for HLLC; Miller & Colella 2002 for characteristic
 * tracing).  The constants and readings listed here are choices:
 *
 *   R1  floors: small_dens = small_pres = 1e-12, applied to primitive copies only.
 *   R2  flattening (CW84 §4): eps = 0.33, omega1 = 0.75, omega2 = 10;
 *       f_i = max(ft_i, ft_{i-s}), s = sign(p_{i+1}-p_{i-1}) (+1 on a tie);
 *       one coefficient per zone = max over the three directions.
 *   R3  PPM (CW84 eqs. 1.6-1.10): van Leer limited slopes, 4th-order
 *       interface values, CW84 monotonicity limiter, then flattening blend.
 *       Slopes are stored per zone and interface values per face, so every
 *       quantity of the method is computed once (the operation counts of
 *       flop_count.cpp are then the method's algorithmic work).
 *   R4  tracing: reference state = integral of the parabola under the fastest
 *       wave moving toward the edge (zone value if none), characteristic
 *       projection with zone-centred rho and c; waves with lambda == 0 excluded.
 *   R5  HLLC with Roe-averaged (Batten) wave-speed bounds, Davis bounds when
 *       the Roe sound speed squared is <= 0; S* == 0 takes the left star state.
 *   R6  3D CTU: stage 1 corrections with factor dt/(3 dx_e), stage 2 with
 *       dt/(2 dx_e); corrections in conserved variables; a corrected state
 *       with rho <= 0 or p <= 0 reverts to the uncorrected one.
 *   R7  dt = cfl * min over interior zones and directions of dx_d/(|u_d|+c),
 *       computed from the state before the step.
 *   R8  ghost fill in the order x, y, z (later directions span the earlier
 *       directions' ghosts, so edges and corners are filled).
 *   R11 the final flux through a reflecting face carries no mass, energy or
 *       tangential momentum (the wall is impermeable; only the normal
 *       momentum flux, the wall pressure, is kept).
 *   R13 limiter variant (box field limiter = 1): Colella & Sekora 2008 (CS08).
 *       Interface values are the 4th-order interpolant of the four nearest
 *       zone values; one that does not lie between its two zone values is
 *       rebuilt from a limited second difference (CS08 §2.1).  The zone
 *       parabola is then limited by CS08's extremum test (zone or its
 *       neighbours at an extremum: curvature limited by the neighbouring
 *       second differences, edges scaled toward the zone value), else by the
 *       CW84 overshoot rule; C = 1.25; flattening blends afterwards as in R3.
 *       No van Leer slopes are formed.
 *   R14 Riemann variant (box field riemann = 1): two-shock approximation
 *       (Colella & Glaz 1985): both nonlinear waves follow their shock
 *       Hugoniot, p* is the root of the two-shock velocity balance found by
 *       Newton's method from the acoustic guess (floor small_pres; stop when
 *       the step is at most 1e-12 p*, at most 40 steps); u* is the mean of
 *       the two sides' star velocities; star densities come from the
 *       Hugoniot; the state at x/t = 0 is sampled on the side of the contact
 *       that holds it (u* = 0 takes the left side), across a shock by its
 *       speed, across a rarefaction by linear interpolation in x/t between
 *       the head and tail states; the flux is the Euler flux of that state.
 *
 * Layout: every field is a [k][j][i] array over the ghosted box
 * (nx+2g)(ny+2g)(nz+2g), i fastest, no padding.  Conserved state
 * U = (rho, rho u, rho v, rho w, E); primitive q = (rho, u, v, w, p).
 *
 * Build with -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {
typedef struct {
  int nx, ny, nz;   /* interior zones per axis */
  int ng;           /* ghost zones per side */
  double dx[3];     /* zone widths */
  double gamma;     /* ratio of specific heats */
  double cfl;       /* Courant number */
  int bc[6];        /* xlo,xhi,ylo,yhi,zlo,zhi: 0 periodic, 1 outflow, 2 reflect */
  int limiter;      /* 0 CW84 (R3), 1 Colella-Sekora (R13) */
  int riemann;      /* 0 HLLC (R5), 1 two-shock (R14) */
} ob_box;
}

enum { OB_PERIODIC = 0, OB_OUTFLOW = 1, OB_REFLECT = 2 };

static const double SMALL_DENS = 1e-12;
static const double SMALL_PRES = 1e-12;
static const double FLAT_EPS = 0.33;
static const double FLAT_OMEGA1 = 0.75;
static const double FLAT_OMEGA2 = 10.0;

/* Test instrumentation (no effect on any result).  Branch-hit counters: how
 * often a step took each guard branch of the method, so that a test can show
 * that a case really exercises it.  The wall switch turns R11 off, which a
 * test uses to show that R11 changes FP64 results by rounding alone. */
enum {
  OB_HIT_PRIM_DENS_FLOOR = 0,  /* a2: rho < small_dens on a primitive copy */
  OB_HIT_PRIM_PRES_FLOOR,      /* a2: p < small_pres */
  OB_HIT_TRACE_DENS_FLOOR,     /* a5: traced rho < small_dens */
  OB_HIT_TRACE_PRES_FLOOR,     /* a5: traced p < small_pres */
  OB_HIT_DAVIS,                /* a9: Roe sound speed squared <= 0 (Davis bounds) */
  OB_HIT_REVERT_STAGE1,        /* a7: corrected state with rho <= 0 or p <= 0 kept uncorrected */
  OB_HIT_REVERT_STAGE2,        /* a8: the same in stage 2 */
  OB_HIT_CORRECTED_PRES_FLOOR, /* a7/a8: 0 < corrected p < small_pres */
  OB_NHITS
};
static long g_hits[OB_NHITS];
static int g_wall_r11 = 1;

static void hit(int k) {
#pragma omp atomic
  g_hits[k]++;
}

/* ------------------------------------------------------------------ grid */
struct Grid {
  int n[3];
  int g;
  int e[3];      /* extents with ghosts */
  long s[3];     /* strides */
  long size;
  explicit Grid(const ob_box* b) {
    n[0] = b->nx; n[1] = b->ny; n[2] = b->nz; g = b->ng;
    for (int d = 0; d < 3; d++) e[d] = n[d] + 2 * g;
    s[0] = 1; s[1] = e[0]; s[2] = (long)e[0] * e[1];
    size = s[2] * e[2];
  }
  long at(int i, int j, int k) const {
    return (long)(i + g) * s[0] + (long)(j + g) * s[1] + (long)(k + g) * s[2];
  }
};

/* slot m of the normal frame for direction d -> component of q or U
 * m: 0 density, 1 normal velocity, 2 and 3 transverse velocities, 4 pressure/energy */
static int comp(int d, int m) {
  if (m == 0 || m == 4) return m;
  return 1 + (d + (m - 1)) % 3;
}

static int box_ok(const ob_box* b) {
  if (b->ng < 4) return 0;
  if (b->nx < 4 || b->ny < 4 || b->nz < 4) return 0;
  for (int a = 0; a < 3; a++) {
    int lo = b->bc[2 * a], hi = b->bc[2 * a + 1];
    if (lo < 0 || lo > 2 || hi < 0 || hi > 2) return 0;
    if ((lo == OB_PERIODIC) != (hi == OB_PERIODIC)) return 0;
    if (!(b->dx[a] > 0.0)) return 0;
  }
  if (b->limiter < 0 || b->limiter > 1 || b->riemann < 0 || b->riemann > 1) return 0;
  return b->gamma > 1.0 && b->cfl > 0.0;
}

/* ------------------------------------------------------- a1: ghost fill (R8) */
static void fill_ghosts(const ob_box* b, const Grid& G, double* U) {
  for (int d = 0; d < 3; d++) {
    int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    /* transverse ranges: axes before d are extended (already filled), later ones interior */
    int lo1 = t1 < d ? -G.g : 0, hi1 = t1 < d ? G.n[t1] + G.g : G.n[t1];
    int lo2 = t2 < d ? -G.g : 0, hi2 = t2 < d ? G.n[t2] + G.g : G.n[t2];
    int n = G.n[d];
    for (int a = lo1; a < hi1; a++) {
      for (int c = lo2; c < hi2; c++) {
        for (int side = 0; side < 2; side++) {
          int bc = b->bc[2 * d + side];
          for (int m = 1; m <= G.g; m++) {
            int gi = side == 0 ? -m : n - 1 + m;
            int si;
            if (bc == OB_PERIODIC) si = side == 0 ? n - m : m - 1;
            else if (bc == OB_OUTFLOW) si = side == 0 ? 0 : n - 1;
            else si = side == 0 ? m - 1 : n - m;
            int idx_g[3], idx_s[3];
            idx_g[d] = gi; idx_s[d] = si;
            idx_g[t1] = a; idx_s[t1] = a;
            idx_g[t2] = c; idx_s[t2] = c;
            long zg = G.at(idx_g[0], idx_g[1], idx_g[2]);
            long zs = G.at(idx_s[0], idx_s[1], idx_s[2]);
            for (int v = 0; v < 5; v++) {
              double val = U[v * G.size + zs];
              if (bc == OB_REFLECT && v == 1 + d) val = -val;
              U[v * G.size + zg] = val;
            }
          }
        }
      }
    }
  }
}

/* ---------------------------------------------------- a2: conserved -> primitive */
static void cons_to_prim_zone(const double* U, long Z, long N, double gamma, double* q, double* c) {
  double rho = U[Z];
  if (rho < SMALL_DENS) {
    rho = SMALL_DENS;
    hit(OB_HIT_PRIM_DENS_FLOOR);
  }
  double u = U[N + Z] / rho;
  double v = U[2 * N + Z] / rho;
  double w = U[3 * N + Z] / rho;
  double kin = 0.5 * rho * (u * u + v * v + w * w);
  double p = (gamma - 1.0) * (U[4 * N + Z] - kin);
  if (p < SMALL_PRES) {
    p = SMALL_PRES;
    hit(OB_HIT_PRIM_PRES_FLOOR);
  }
  q[Z] = rho; q[N + Z] = u; q[2 * N + Z] = v; q[3 * N + Z] = w; q[4 * N + Z] = p;
  c[Z] = sqrt(gamma * p / rho);
}

static void cons_to_prim_all(const ob_box* b, const Grid& G, const double* U, double* q, double* c) {
#pragma omp parallel for schedule(static)
  for (long Z = 0; Z < G.size; Z++) cons_to_prim_zone(U, Z, G.size, b->gamma, q, c);
}

/* --------------------------------------------------------------- a11: dt (R7) */
static double compute_dt(const ob_box* b, const Grid& G, const double* U) {
  double dtmin = HUGE_VAL;
  for (int k = 0; k < G.n[2]; k++)
    for (int j = 0; j < G.n[1]; j++)
      for (int i = 0; i < G.n[0]; i++) {
        long Z = G.at(i, j, k);
        double rho = U[Z];
        if (rho < SMALL_DENS) rho = SMALL_DENS;
        double u[3];
        for (int d = 0; d < 3; d++) u[d] = U[(1 + d) * G.size + Z] / rho;
        double kin = 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double p = (b->gamma - 1.0) * (U[4 * G.size + Z] - kin);
        if (p < SMALL_PRES) p = SMALL_PRES;
        double cs = sqrt(b->gamma * p / rho);
        for (int d = 0; d < 3; d++) {
          double t = b->dx[d] / (fabs(u[d]) + cs);
          if (t < dtmin) dtmin = t;
        }
      }
  return b->cfl * dtmin;
}

/* ------------------------------------------------------- a3: flattening (R2) */
/* CW84 §4: shock indicator ft at zone Z along stride s (p pressure, un normal velocity) */
static double flat_tilde(const double* p, const double* un, long Z, long s) {
  double dp1 = p[Z + s] - p[Z - s];
  double dp2 = p[Z + 2 * s] - p[Z - 2 * s];
  double pmin = fmin(p[Z + s], p[Z - s]);
  int shock = fabs(dp1) / pmin > FLAT_EPS && un[Z - s] - un[Z + s] > 0.0;
  if (!shock) return 0.0;
  if (dp2 == 0.0) return 0.0;
  double r = FLAT_OMEGA2 * (dp1 / dp2 - FLAT_OMEGA1);
  return fmax(0.0, fmin(1.0, r));
}

static double flat_dir(const double* p, const double* un, long Z, long s) {
  double dp1 = p[Z + s] - p[Z - s];
  long sh = dp1 >= 0.0 ? s : -s;
  return fmax(flat_tilde(p, un, Z, s), flat_tilde(p, un, Z - sh, s));
}

static void flatten_all(const Grid& G, const double* q, double* chi) {
  const double* p = q + 4 * G.size;
#pragma omp parallel for schedule(static)
  for (int k = -1; k <= G.n[2]; k++)
    for (int j = -1; j <= G.n[1]; j++)
      for (int i = -1; i <= G.n[0]; i++) {
        long Z = G.at(i, j, k);
        double f = 0.0;
        for (int d = 0; d < 3; d++) f = fmax(f, flat_dir(p, q + (1 + d) * G.size, Z, G.s[d]));
        chi[Z] = f;
      }
}

/* ---------------------------------------------------------- a4: PPM (R3) */
/* van Leer limited slope at the middle of (am, a0, ap): CW84 eq. 1.8 */
static double limited_slope(double am, double a0, double ap) {
  double dl = a0 - am, dr = ap - a0;
  if (dl * dr > 0.0) {
    double dc = 0.5 * (ap - am);
    double m = fmin(fabs(dc), fmin(2.0 * fabs(dl), 2.0 * fabs(dr)));
    return copysign(m, dc);
  }
  return 0.0;
}

/* 4th-order value at the interface between zones Z-s and Z (CW84 eq. 1.6),
 * from zone values a and limited slopes dm */
static double interface_value(const double* a, const double* dm, long Z, long s) {
  return a[Z - s] + 0.5 * (a[Z] - a[Z - s]) - (dm[Z] - dm[Z - s]) / 6.0;
}

/* Parabola of zone value a0 between interface values (L, R): CW84 monotonicity
 * limiter (eq. 1.10), then a_{L,R} <- f a0 + (1-f) a_{L,R} (CW84 §4). */
static void limit_parabola(double a0, double f, double* aL, double* aR) {
  double L = *aL, R = *aR;
  if ((R - a0) * (a0 - L) <= 0.0) {
    L = a0;
    R = a0;
  } else {
    double dA = R - L;
    double mid = a0 - 0.5 * (L + R);
    if (dA * mid > dA * dA / 6.0) {
      L = 3.0 * a0 - 2.0 * R;
    } else if (-(dA * dA) / 6.0 > dA * mid) {
      R = 3.0 * a0 - 2.0 * L;
    }
  }
  *aL = f * a0 + (1.0 - f) * L;
  *aR = f * a0 + (1.0 - f) * R;
}

/* ------------------------------------------- a4 variant: CS08 limiter (R13) */
static const double CS_C = 1.25;

/* CS08's limited second difference: when d2 and every neighbouring second
 * difference share a sign, the smallest of |d2| and C |others|, with the sign
 * of d2; otherwise zero. */
static double cs_limited_d2(double d2, const double* others, int n) {
  double m = fabs(d2);
  for (int k = 0; k < n; k++) {
    if (!(d2 * others[k] > 0.0)) return 0.0;
    m = fmin(m, CS_C * fabs(others[k]));
  }
  return copysign(m, d2);
}

/* Value at the interface between zones Z-s and Z (CS08 §2.1): the 4th-order
 * interpolant, rebuilt from a limited second difference when it is not
 * between the two zone values. */
static double cs_interface(const double* a, long Z, long s) {
  double am = a[Z - 2 * s], a0 = a[Z - s], a1 = a[Z], a2 = a[Z + s];
  double v = 7.0 / 12.0 * (a0 + a1) - 1.0 / 12.0 * (am + a2);
  if ((v - a0) * (a1 - v) < 0.0) {
    double d2 = 3.0 * (a0 - 2.0 * v + a1);
    double nb[2] = {am - 2.0 * a0 + a1, a0 - 2.0 * a1 + a2};
    v = 0.5 * (a0 + a1) - cs_limited_d2(d2, nb, 2) / 6.0;
  }
  return v;
}

/* Parabola of zone Z of line a (stride s) between interface values (L, R):
 * CS08's limiter (§2.2), then the flattening blend of R3. */
static void cs_limit_parabola(const double* a, long Z, long s, double f, double* aL, double* aR) {
  double a0 = a[Z], L = *aL, R = *aR;
  double am = a[Z - s], ap = a[Z + s];
  if ((R - a0) * (a0 - L) <= 0.0 || (ap - a0) * (a0 - am) <= 0.0) {
    /* an extremum in the zone or at a neighbour: keep the parabola's shape,
     * with its curvature limited by the second differences around it */
    double d2 = 6.0 * (L + R - 2.0 * a0);
    double nb[3] = {a[Z - 2 * s] - 2.0 * am + a0, am - 2.0 * a0 + ap, a0 - 2.0 * ap + a[Z + 2 * s]};
    double lim = cs_limited_d2(d2, nb, 3);
    if (d2 != 0.0) {
      L = a0 + (L - a0) * (lim / d2);
      R = a0 + (R - a0) * (lim / d2);
    } else {
      L = a0;
      R = a0;
    }
  } else if (fabs(R - a0) >= 2.0 * fabs(L - a0)) {
    R = a0 - 2.0 * (L - a0);
  } else if (fabs(L - a0) >= 2.0 * fabs(R - a0)) {
    L = a0 - 2.0 * (R - a0);
  }
  *aL = f * a0 + (1.0 - f) * L;
  *aR = f * a0 + (1.0 - f) * R;
}

/* -------------------------------------------- a5: characteristic tracing (R4) */
/* Average of the parabola over the part of the zone swept by a wave of
 * Courant number sig toward the right edge (Iplus) or the left edge (Iminus). */
static double i_plus(double aL, double aR, double a0, double sig) {
  double dA = aR - aL, a6 = 6.0 * (a0 - 0.5 * (aL + aR));
  return aR - 0.5 * sig * (dA - (1.0 - 2.0 * sig / 3.0) * a6);
}
static double i_minus(double aL, double aR, double a0, double sig) {
  double dA = aR - aL, a6 = 6.0 * (a0 - 0.5 * (aL + aR));
  return aL + 0.5 * sig * (dA + (1.0 - 2.0 * sig / 3.0) * a6);
}

/* Trace zone Z along stride s.  qn[m] points at the normal-frame field m
 * (rho, u_n, u_t1, u_t2, p) and face[m] at its interface values (value at the
 * low face of each zone).  Writes the left-edge state qm[5] (the right state
 * of the low face) and the right-edge state qp[5] (the left state of the high
 * face), both in the normal frame. */
static void trace_zone(const double* const qn[5], const double* const face[5], const double* c, double f,
                       long Z, long s, double dtdx, int limiter, double* qm, double* qp) {
  double aL[5], aR[5], a0[5];
  for (int m = 0; m < 5; m++) {
    a0[m] = qn[m][Z];
    aL[m] = face[m][Z];
    aR[m] = face[m][Z + s];
    if (limiter == 1) cs_limit_parabola(qn[m], Z, s, f, &aL[m], &aR[m]);
    else limit_parabola(a0[m], f, &aL[m], &aR[m]);
  }
  double rho = a0[0], u = a0[1], cs = c[Z];
  double lam[3] = {u - cs, u, u + cs};

  for (int side = 0; side < 2; side++) {
    /* side 0: right edge (toward +s, waves with lambda > 0); side 1: left edge.
     * The fastest wave toward the edge supplies the reference state; its own
     * amplitude is zero by construction and is not formed. */
    double ref[5];
    int fast = side == 0 ? 2 : 0;
    int reaches_fast = side == 0 ? lam[2] > 0.0 : lam[0] < 0.0;
    for (int m = 0; m < 5; m++) {
      if (reaches_fast) {
        double sig = fabs(lam[fast]) * dtdx;
        ref[m] = side == 0 ? i_plus(aL[m], aR[m], a0[m], sig) : i_minus(aL[m], aR[m], a0[m], sig);
      } else {
        ref[m] = a0[m];
      }
    }
    double beta[3] = {0.0, 0.0, 0.0};
    double out[5];
    out[2] = ref[2];
    out[3] = ref[3];
    for (int w = 0; w < 3; w++) {
      if (w == fast) continue;
      int reaches = side == 0 ? lam[w] > 0.0 : lam[w] < 0.0;
      if (!reaches) continue;
      double sig = fabs(lam[w]) * dtdx;
      /* integrals of the variables this wave's amplitude uses */
      const int acoustic[2] = {1, 4}, entropy[4] = {0, 4, 2, 3};
      const int* vars = w == 1 ? entropy : acoustic;
      int nv = w == 1 ? 4 : 2;
      double I[5];
      for (int k = 0; k < nv; k++) {
        int m = vars[k];
        I[m] = side == 0 ? i_plus(aL[m], aR[m], a0[m], sig) : i_minus(aL[m], aR[m], a0[m], sig);
      }
      if (w == 0) {
        double du = ref[1] - I[1], dp = ref[4] - I[4];
        beta[w] = -rho / (2.0 * cs) * du + dp / (2.0 * cs * cs);
      } else if (w == 2) {
        double du = ref[1] - I[1], dp = ref[4] - I[4];
        beta[w] = rho / (2.0 * cs) * du + dp / (2.0 * cs * cs);
      } else {
        double dr = ref[0] - I[0], dp = ref[4] - I[4];
        beta[w] = dr - dp / (cs * cs);
        out[2] = I[2];
        out[3] = I[3];
      }
    }
    out[0] = ref[0] - (beta[0] + beta[1] + beta[2]);
    out[1] = ref[1] - (cs / rho) * (beta[2] - beta[0]);
    out[4] = ref[4] - cs * cs * (beta[0] + beta[2]);
    if (out[0] < SMALL_DENS) {
      out[0] = SMALL_DENS;
      hit(OB_HIT_TRACE_DENS_FLOOR);
    }
    if (out[4] < SMALL_PRES) {
      out[4] = SMALL_PRES;
      hit(OB_HIT_TRACE_PRES_FLOOR);
    }
    double* dst = side == 0 ? qp : qm;
    for (int m = 0; m < 5; m++) dst[m] = out[m];
  }
}

/* --------------------------------------------------------- a9: HLLC (R5) */
/* Normal-frame states L, R = (rho, u_n, u_t1, u_t2, p) -> normal-frame flux F. */
static void hllc_normal(const double* L, const double* R, double gamma, double* F) {
  double rl = L[0], ul = L[1], vl = L[2], wl = L[3], pl = L[4];
  double rr = R[0], ur = R[1], vr = R[2], wr = R[3], pr = R[4];
  double El = pl / (gamma - 1.0) + 0.5 * rl * (ul * ul + vl * vl + wl * wl);
  double Er = pr / (gamma - 1.0) + 0.5 * rr * (ur * ur + vr * vr + wr * wr);
  double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
  double Hl = (El + pl) / rl, Hr = (Er + pr) / rr;
  double sl = sqrt(rl), sr = sqrt(rr);
  double ut = (sl * ul + sr * ur) / (sl + sr);
  double vt = (sl * vl + sr * vr) / (sl + sr);
  double wt = (sl * wl + sr * wr) / (sl + sr);
  double Ht = (sl * Hl + sr * Hr) / (sl + sr);
  double ct2 = (gamma - 1.0) * (Ht - 0.5 * (ut * ut + vt * vt + wt * wt));
  double SL, SR;
  if (ct2 > 0.0) {
    double ct = sqrt(ct2);
    SL = fmin(ul - cl, ut - ct);
    SR = fmax(ur + cr, ut + ct);
  } else {
    SL = fmin(ul - cl, ur - cr);
    SR = fmax(ul + cl, ur + cr);
    hit(OB_HIT_DAVIS);
  }
  double Ss = (pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur)) / (rl * (SL - ul) - rr * (SR - ur));

  if (SL >= 0.0 || (SR > 0.0 && Ss >= 0.0)) {
    double FL[5] = {rl * ul, rl * ul * ul + pl, rl * ul * vl, rl * ul * wl, (El + pl) * ul};
    if (SL >= 0.0) {
      for (int m = 0; m < 5; m++) F[m] = FL[m];
      return;
    }
    double Ul[5] = {rl, rl * ul, rl * vl, rl * wl, El};
    double fac = rl * (SL - ul) / (SL - Ss);
    double Us[5] = {fac, fac * Ss, fac * vl, fac * wl,
                    fac * (El / rl + (Ss - ul) * (Ss + pl / (rl * (SL - ul))))};
    for (int m = 0; m < 5; m++) F[m] = FL[m] + SL * (Us[m] - Ul[m]);
    return;
  }
  double FR[5] = {rr * ur, rr * ur * ur + pr, rr * ur * vr, rr * ur * wr, (Er + pr) * ur};
  if (SR <= 0.0) {
    for (int m = 0; m < 5; m++) F[m] = FR[m];
    return;
  }
  double Ur[5] = {rr, rr * ur, rr * vr, rr * wr, Er};
  double fac = rr * (SR - ur) / (SR - Ss);
  double Us[5] = {fac, fac * Ss, fac * vr, fac * wr,
                  fac * (Er / rr + (Ss - ur) * (Ss + pr / (rr * (SR - ur))))};
  for (int m = 0; m < 5; m++) F[m] = FR[m] + SR * (Us[m] - Ur[m]);
}

/* ------------------------------------ a9 variant: two-shock solver (R14) */
static const double TS_TOL = 1e-12;
static const int TS_MAXIT = 40;

/* Lagrangian speed (mass flux) of a shock from state (rho, p) to pressure ps:
 * W^2 = rho ((gamma+1)/2 ps + (gamma-1)/2 p) (Rankine-Hugoniot). */
static double shock_w(double rho, double p, double ps, double gamma) {
  return sqrt(rho * (0.5 * (gamma + 1.0) * ps + 0.5 * (gamma - 1.0) * p));
}

/* Star pressure and velocity of the two-shock approximation; returns the
 * number of Newton steps taken.  The velocity change across the wave of side
 * K is (p - p_K) / W_K(p); p* balances u_L - that of L with u_R + that of R. */
static int two_shock_star(const double* L, const double* R, double gamma, double* ps, double* us) {
  double rl = L[0], ul = L[1], pl = L[4], rr = R[0], ur = R[1], pr = R[4];
  double Cl = sqrt(gamma * pl * rl), Cr = sqrt(gamma * pr * rr);
  double p = (Cr * pl + Cl * pr + Cl * Cr * (ul - ur)) / (Cl + Cr);
  if (p < SMALL_PRES) p = SMALL_PRES;
  int it = 0;
  while (it < TS_MAXIT) {
    double Wl = shock_w(rl, pl, p, gamma), Wr = shock_w(rr, pr, p, gamma);
    double f = (p - pl) / Wl + (p - pr) / Wr + (ur - ul);
    /* d/dp of (p - p_K)/W_K(p) = (1 - (p - p_K) dW_K/dp / W_K) / W_K, dW_K/dp = rho_K (gamma+1) / (4 W_K) */
    double dl = (1.0 - (p - pl) * rl * (gamma + 1.0) / (4.0 * Wl * Wl)) / Wl;
    double dr = (1.0 - (p - pr) * rr * (gamma + 1.0) / (4.0 * Wr * Wr)) / Wr;
    double pn = p - f / (dl + dr);
    if (pn < SMALL_PRES) pn = SMALL_PRES;
    it++;
    double step = fabs(pn - p);
    p = pn;
    if (step <= TS_TOL * p) break;
  }
  double Wl = shock_w(rl, pl, p, gamma), Wr = shock_w(rr, pr, p, gamma);
  *ps = p;
  *us = 0.5 * ((ul - (p - pl) / Wl) + (ur + (p - pr) / Wr));
  return it;
}

/* State at x/t = 0 of the two-shock solution (normal frame). */
static void two_shock_state(const double* L, const double* R, double gamma, double* q) {
  double ps, us;
  two_shock_star(L, R, gamma, &ps, &us);
  int left = us >= 0.0;
  const double* K = left ? L : R;
  double sgn = left ? 1.0 : -1.0;   /* the side's wave moves with u - sgn c */
  double rk = K[0], uk = K[1], pk = K[4];
  double Wk = shock_w(rk, pk, ps, gamma);
  double rs = 1.0 / (1.0 / rk - (ps - pk) / (Wk * Wk));  /* Hugoniot: [1/rho] = -[p]/W^2 */
  double star[5] = {rs, us, K[2], K[3], ps};
  double outer[5] = {rk, uk, K[2], K[3], pk};
  /* speeds of the side's wave as seen from the interface, positive when
   * the wave is on the side's own half (moving away from x/t = 0) */
  double head, tail;
  if (ps > pk) {
    head = tail = Wk / rk - sgn * uk;   /* shock: |S - u_K| = W_K / rho_K */
  } else {
    head = sqrt(gamma * pk / rk) - sgn * uk;
    tail = sqrt(gamma * ps / rs) - sgn * us;
  }
  if (head <= 0.0) {
    for (int m = 0; m < 5; m++) q[m] = outer[m];   /* the wave has left x/t = 0 behind */
  } else if (tail >= 0.0) {
    for (int m = 0; m < 5; m++) q[m] = star[m];
  } else {
    /* x/t = 0 inside the fan: linear in x/t between head and tail */
    double a = head / (head - tail);
    for (int m = 0; m < 5; m++) q[m] = (1.0 - a) * outer[m] + a * star[m];
  }
}

static void euler_flux(const double* q, double gamma, double* F) {
  double r = q[0], u = q[1], v = q[2], w = q[3], p = q[4];
  double E = p / (gamma - 1.0) + 0.5 * r * (u * u + v * v + w * w);
  F[0] = r * u;
  F[1] = r * u * u + p;
  F[2] = r * u * v;
  F[3] = r * u * w;
  F[4] = (E + p) * u;
}

static void two_shock_normal(const double* L, const double* R, double gamma, double* F) {
  double q[5];
  two_shock_state(L, R, gamma, q);
  euler_flux(q, gamma, F);
}

/* The box's Riemann solver across a face normal to d, states and flux in
 * x,y,z components. */
static void riemann_xyz(int solver, int d, const double* qL, const double* qR, double gamma, double* F) {
  double L[5], R[5], Fn[5];
  for (int m = 0; m < 5; m++) {
    L[m] = qL[comp(d, m)];
    R[m] = qR[comp(d, m)];
  }
  if (solver == 1) two_shock_normal(L, R, gamma, Fn);
  else hllc_normal(L, R, gamma, Fn);
  for (int m = 0; m < 5; m++) F[comp(d, m)] = Fn[m];
}

/* ------------------------------------------------ helpers for the CTU stages */
static void prim_to_cons(const double* q, double gamma, double* U) {
  U[0] = q[0];
  U[1] = q[0] * q[1];
  U[2] = q[0] * q[2];
  U[3] = q[0] * q[3];
  U[4] = q[4] / (gamma - 1.0) + 0.5 * q[0] * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
}

/* returns 0 (and leaves q alone) when the state has rho <= 0 or p <= 0 (R6) */
static int cons_to_prim_checked(const double* U, double gamma, double* q) {
  if (!(U[0] > 0.0)) return 0;
  double u = U[1] / U[0], v = U[2] / U[0], w = U[3] / U[0];
  double p = (gamma - 1.0) * (U[4] - 0.5 * U[0] * (u * u + v * v + w * w));
  if (!(p > 0.0)) return 0;
  q[0] = U[0]; q[1] = u; q[2] = v; q[3] = w;
  if (p < SMALL_PRES) {
    p = SMALL_PRES;
    hit(OB_HIT_CORRECTED_PRES_FLOOR);
  }
  q[4] = p;
  return 1;
}

/* ------------------------------------------------------------- workspace */
/* field order (each G.size doubles): q[5], c, chi, qm[3][5], qp[3][5],
 * F0[3][5], F1[6][5] (pairs xy,xz,yx,yz,zx,zy), F[3][5] -> 97 fields */
enum {
  W_Q = 0, W_C = 5, W_CHI = 6, W_QM = 7, W_QP = 22, W_F0 = 37, W_F1 = 52, W_F = 82, W_NFIELDS = 97
};
static int pair_index(int d, int e) {
  /* (0,1)->0 (0,2)->1 (1,0)->2 (1,2)->3 (2,0)->4 (2,1)->5 */
  return 2 * d + (e > d ? e - 1 : e);
}

/* state of a d-face side, stored per zone in the normal frame, back to x,y,z */
static void load_state(const double* W, long N, int base, int d, long Z, double* q) {
  for (int m = 0; m < 5; m++) q[comp(d, m)] = W[(long)(base + 5 * d + m) * N + Z];
}

/* ------------------------------------------------------------- one step */
/* a4: limited slopes of the five normal-frame variables of axis d on zones
 * [-2, n_d+1] along d and [-1, n] across it (stored per zone: the CPU
 * structure the paper's §3 describes) */
static void limited_slopes_dir(const Grid& G, int d, const double* W, double* slope) {
  long N = G.size, s = G.s[d];
  const double* qn[5];
  for (int m = 0; m < 5; m++) qn[m] = W + (long)(W_Q + comp(d, m)) * N;
  int lo[3] = {-1, -1, -1}, hi[3] = {G.n[0], G.n[1], G.n[2]};
  lo[d] = -2;
  hi[d] = G.n[d] + 1;
#pragma omp parallel for schedule(static)
  for (int k = lo[2]; k <= hi[2]; k++)
    for (int j = lo[1]; j <= hi[1]; j++)
      for (int i = lo[0]; i <= hi[0]; i++) {
        long Z = G.at(i, j, k);
        for (int m = 0; m < 5; m++) slope[(long)m * N + Z] = limited_slope(qn[m][Z - s], qn[m][Z], qn[m][Z + s]);
      }
}

/* a4: interface values on the faces [-1, n_d+1] of axis d (one per face);
 * slope is NULL under the CS08 limiter (R13) */
static void interface_values_dir(const Grid& G, int d, const double* W, const double* slope, double* face) {
  long N = G.size, s = G.s[d];
  const double* qn[5];
  for (int m = 0; m < 5; m++) qn[m] = W + (long)(W_Q + comp(d, m)) * N;
  int lo[3] = {-1, -1, -1}, hi[3] = {G.n[0], G.n[1], G.n[2]};
  hi[d] = G.n[d] + 1;
#pragma omp parallel for schedule(static)
  for (int k = lo[2]; k <= hi[2]; k++)
    for (int j = lo[1]; j <= hi[1]; j++)
      for (int i = lo[0]; i <= hi[0]; i++) {
        long Z = G.at(i, j, k);
        for (int m = 0; m < 5; m++)
          face[(long)m * N + Z] = slope ? interface_value(qn[m], slope + (long)m * N, Z, s) : cs_interface(qn[m], Z, s);
      }
}

/* a4 + a5: per zone of [-1, n]^3 the limited parabolas of axis d and the
 * traced edge states */
static void trace_zones_dir(const ob_box* b, const Grid& G, int d, double dt, double* W, const double* face) {
  long N = G.size, s = G.s[d];
  double dtdx = dt / b->dx[d];
  const double* qn[5];
  const double* fc[5];
  for (int m = 0; m < 5; m++) {
    qn[m] = W + (long)(W_Q + comp(d, m)) * N;
    fc[m] = face + (long)m * N;
  }
#pragma omp parallel for schedule(static)
  for (int k = -1; k <= G.n[2]; k++)
    for (int j = -1; j <= G.n[1]; j++)
      for (int i = -1; i <= G.n[0]; i++) {
        long Z = G.at(i, j, k);
        double qm[5], qp[5];
        trace_zone(qn, fc, W + (long)W_C * N, W[(long)W_CHI * N + Z], Z, s, dtdx, b->limiter, qm, qp);
        for (int m = 0; m < 5; m++) {
          W[(long)(W_QM + 5 * d + m) * N + Z] = qm[m];
          W[(long)(W_QP + 5 * d + m) * N + Z] = qp[m];
        }
      }
}

static void trace_all(const ob_box* b, const Grid& G, double dt, double* W) {
  double* slope = (double*)calloc((size_t)5 * G.size, sizeof(double));
  double* face = (double*)calloc((size_t)5 * G.size, sizeof(double));
  for (int d = 0; d < 3; d++) {
    if (b->limiter == 1) {
      interface_values_dir(G, d, W, NULL, face);
    } else {
      limited_slopes_dir(G, d, W, slope);
      interface_values_dir(G, d, W, slope, face);
    }
    trace_zones_dir(b, G, d, dt, W, face);
  }
  free(slope);
  free(face);
}

/* loop bounds for faces normal to d: normal index lo..n_d, transverse per mode */
static void face_range(const Grid& G, int d, const int* tlo, const int* thi, int* lo, int* hi) {
  for (int a = 0; a < 3; a++) {
    if (a == d) { lo[a] = 0; hi[a] = G.n[a]; }
    else { lo[a] = tlo[a]; hi[a] = thi[a]; }
  }
}

static void normal_fluxes(const ob_box* b, const Grid& G, double* W) {
  long N = G.size;
  for (int d = 0; d < 3; d++) {
    int tlo[3] = {-1, -1, -1}, thi[3] = {G.n[0], G.n[1], G.n[2]}, lo[3], hi[3];
    face_range(G, d, tlo, thi, lo, hi);
#pragma omp parallel for schedule(static)
    for (int k = lo[2]; k <= hi[2]; k++)
      for (int j = lo[1]; j <= hi[1]; j++)
        for (int i = lo[0]; i <= hi[0]; i++) {
          long Z = G.at(i, j, k);
          double qL[5], qR[5], F[5];
          load_state(W, N, W_QP, d, Z - G.s[d], qL);
          load_state(W, N, W_QM, d, Z, qR);
          riemann_xyz(b->riemann, d, qL, qR, b->gamma, F);
          for (int v = 0; v < 5; v++) W[(long)(W_F0 + 5 * d + v) * N + Z] = F[v];
        }
  }
}

/* conserved correction of a face state belonging to zone Z */
static void corrected_state(const ob_box* b, const double* qin, int nterms, const double* fac,
                            const double* const* Fs, const long* s, long Z, long N, double* qout) {
  double U[5];
  prim_to_cons(qin, b->gamma, U);
  for (int v = 0; v < 5; v++) {
    double val = U[v];
    for (int t = 0; t < nterms; t++) val = val - fac[t] * (Fs[t][v * N + Z + s[t]] - Fs[t][v * N + Z]);
    U[v] = val;
  }
  for (int v = 0; v < 5; v++) qout[v] = qin[v];
  if (!cons_to_prim_checked(U, b->gamma, qout)) hit(nterms == 1 ? OB_HIT_REVERT_STAGE1 : OB_HIT_REVERT_STAGE2);
}

static void ctu_stage1(const ob_box* b, const Grid& G, double dt, double* W) {
  long N = G.size;
  for (int d = 0; d < 3; d++)
    for (int e = 0; e < 3; e++) {
      if (e == d) continue;
      int f = 3 - d - e;
      int tlo[3], thi[3], lo[3], hi[3];
      tlo[e] = 0; thi[e] = G.n[e] - 1;
      tlo[f] = -1; thi[f] = G.n[f];
      face_range(G, d, tlo, thi, lo, hi);
      double fac = dt / (3.0 * b->dx[e]);
      const double* Fe = W + (long)(W_F0 + 5 * e) * N;
      long se = G.s[e];
      double* out = W + (long)(W_F1 + 5 * pair_index(d, e)) * N;
#pragma omp parallel for schedule(static)
      for (int k = lo[2]; k <= hi[2]; k++)
        for (int j = lo[1]; j <= hi[1]; j++)
          for (int i = lo[0]; i <= hi[0]; i++) {
            long Z = G.at(i, j, k);
            long ZL = Z - G.s[d];
            double qL0[5], qR0[5], qL[5], qR[5], F[5];
            load_state(W, N, W_QP, d, ZL, qL0);
            load_state(W, N, W_QM, d, Z, qR0);
            corrected_state(b, qL0, 1, &fac, &Fe, &se, ZL, N, qL);
            corrected_state(b, qR0, 1, &fac, &Fe, &se, Z, N, qR);
            riemann_xyz(b->riemann, d, qL, qR, b->gamma, F);
            for (int v = 0; v < 5; v++) out[v * N + Z] = F[v];
          }
    }
}

static void ctu_stage2(const ob_box* b, const Grid& G, double dt, double* W) {
  long N = G.size;
  for (int d = 0; d < 3; d++) {
    int e = (d + 1) % 3, f = (d + 2) % 3;
    int tlo[3] = {0, 0, 0}, thi[3] = {G.n[0] - 1, G.n[1] - 1, G.n[2] - 1}, lo[3], hi[3];
    face_range(G, d, tlo, thi, lo, hi);
    double fac[2] = {dt / (2.0 * b->dx[e]), dt / (2.0 * b->dx[f])};
    const double* Fs[2] = {W + (long)(W_F1 + 5 * pair_index(e, f)) * N,
                           W + (long)(W_F1 + 5 * pair_index(f, e)) * N};
    long s[2] = {G.s[e], G.s[f]};
    double* out = W + (long)(W_F + 5 * d) * N;
#pragma omp parallel for schedule(static)
    for (int k = lo[2]; k <= hi[2]; k++)
      for (int j = lo[1]; j <= hi[1]; j++)
        for (int i = lo[0]; i <= hi[0]; i++) {
          long Z = G.at(i, j, k);
          long ZL = Z - G.s[d];
          double qL0[5], qR0[5], qL[5], qR[5], F[5];
          load_state(W, N, W_QP, d, ZL, qL0);
          load_state(W, N, W_QM, d, Z, qR0);
          corrected_state(b, qL0, 2, fac, Fs, s, ZL, N, qL);
          corrected_state(b, qR0, 2, fac, Fs, s, Z, N, qR);
          riemann_xyz(b->riemann, d, qL, qR, b->gamma, F);
          /* R11: a reflecting face is impermeable -- no mass, energy or
           * tangential momentum crosses it, only the pressure force acts */
          int face = d == 0 ? i : (d == 1 ? j : k);
          if (g_wall_r11 &&
              ((face == 0 && b->bc[2 * d] == OB_REFLECT) || (face == G.n[d] && b->bc[2 * d + 1] == OB_REFLECT))) {
            for (int v = 0; v < 5; v++)
              if (v != 1 + d) F[v] = 0.0;
          }
          for (int v = 0; v < 5; v++) out[v * N + Z] = F[v];
        }
  }
}

/* a10: conservative update of the interior; returns 0 when a zone is nonphysical */
static int update(const ob_box* b, const Grid& G, double dt, double* U, const double* W) {
  long N = G.size;
  double dtdx[3];
  for (int d = 0; d < 3; d++) dtdx[d] = dt / b->dx[d];
  int ok = 1;
#pragma omp parallel for schedule(static) reduction(&& : ok)
  for (int k = 0; k < G.n[2]; k++)
    for (int j = 0; j < G.n[1]; j++)
      for (int i = 0; i < G.n[0]; i++) {
        long Z = G.at(i, j, k);
        for (int v = 0; v < 5; v++) {
          double val = U[v * N + Z];
          for (int d = 0; d < 3; d++) {
            const double* F = W + (long)(W_F + 5 * d + v) * N;
            val = val - dtdx[d] * (F[Z + G.s[d]] - F[Z]);
          }
          U[v * N + Z] = val;
        }
        double rho = U[Z];
        double kin = 0.5 * (U[N + Z] * U[N + Z] + U[2 * N + Z] * U[2 * N + Z] + U[3 * N + Z] * U[3 * N + Z]) / rho;
        double p = (b->gamma - 1.0) * (U[4 * N + Z] - kin);
        if (!(rho > 0.0) || !(p > 0.0) || p != p) ok = 0;
      }
  return ok;
}

static int step_impl(const ob_box* b, double* U, double dt, double* W) {
  Grid G(b);
  cons_to_prim_all(b, G, U, W + (long)W_Q * G.size, W + (long)W_C * G.size);
  flatten_all(G, W + (long)W_Q * G.size, W + (long)W_CHI * G.size);
  trace_all(b, G, dt, W);
  normal_fluxes(b, G, W);
  ctu_stage1(b, G, dt, W);
  ctu_stage2(b, G, dt, W);
  return update(b, G, dt, U, W);
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
  omp_set_num_threads(nthreads > 0 ? nthreads : 1);
#else
  (void)nthreads;
#endif
}

/* ============================================================ exported API
 * Return codes: 0 ok, -1 invalid box, -3 nonphysical state after an update. */
extern "C" {

int oracle_nfields(void) { return W_NFIELDS; }

int oracle_fill_ghosts(const ob_box* b, double* U) {
  if (!box_ok(b)) return -1;
  Grid G(b);
  fill_ghosts(b, G, U);
  return 0;
}

int oracle_compute_dt(const ob_box* b, const double* U, double* dt) {
  if (!box_ok(b)) return -1;
  Grid G(b);
  *dt = compute_dt(b, G, U);
  return 0;
}

int oracle_prim(const ob_box* b, const double* U, double* q, double* c) {
  if (!box_ok(b)) return -1;
  Grid G(b);
  cons_to_prim_all(b, G, U, q, c);
  return 0;
}

/* One update with a given dt; the ghost zones of U must already be filled.
 * work: NULL, or W_NFIELDS * Ng doubles that receive every intermediate. */
int oracle_step(const ob_box* b, double* U, double dt, double* work, int nthreads) {
  if (!box_ok(b)) return -1;
  set_threads(nthreads);
  Grid G(b);
  double* W = work;
  if (!W) W = (double*)calloc((size_t)W_NFIELDS * G.size, sizeof(double));
  if (!W) return -2;
  int ok = step_impl(b, U, dt, W);
  if (!work) free(W);
  return ok ? 0 : -3;
}

/* nsteps of: fill ghosts, dt from the state, update.  dts[s] receives each dt
 * (may be NULL); *t receives the sum. */
int oracle_run(const ob_box* b, double* U, int nsteps, double* dts, double* t, int nthreads) {
  if (!box_ok(b) || nsteps < 0) return -1;
  set_threads(nthreads);
  Grid G(b);
  double* W = (double*)calloc((size_t)W_NFIELDS * G.size, sizeof(double));
  if (!W) return -2;
  double time = 0.0;
  int rc = 0;
  for (int s = 0; s < nsteps; s++) {
    fill_ghosts(b, G, U);
    double dt = compute_dt(b, G, U);
    if (dts) dts[s] = dt;
    if (!step_impl(b, U, dt, W)) { rc = -3; time += dt; break; }
    time += dt;
  }
  fill_ghosts(b, G, U);
  free(W);
  if (t) *t = time;
  return rc;
}

/* Stage-level entry points for unit tests --------------------------------- */

/* HLLC flux across a face normal to d for x,y,z primitive states */
void oracle_hllc(int d, const double* qL, const double* qR, double gamma, double* F) {
  riemann_xyz(0, d, qL, qR, gamma, F);
}

/* Two-shock solver on normal-frame states L, R = (rho, u_n, u_t1, u_t2, p):
 * star pressure and velocity ps_us[2], the state at x/t = 0 (q[5]) and its
 * flux (F[5]); returns the number of Newton steps. */
int oracle_two_shock(const double* L, const double* R, double gamma, double* ps_us, double* q, double* F) {
  int it = two_shock_star(L, R, gamma, &ps_us[0], &ps_us[1]);
  two_shock_state(L, R, gamma, q);
  euler_flux(q, gamma, F);
  return it;
}

/* CS08 parabola of a 1D line a[n] with flattening chi[n]; zones 2..n-3 are written */
void oracle_ppm_line_cs(const double* a, const double* chi, int n, double* aL, double* aR) {
  for (long i = 2; i < n - 2; i++) {
    aL[i] = cs_interface(a, i, 1);
    aR[i] = cs_interface(a, i + 1, 1);
    cs_limit_parabola(a, i, 1, chi[i], &aL[i], &aR[i]);
  }
}

/* PPM parabola of a 1D line a[n] with flattening chi[n]; zones 2..n-3 are written */
void oracle_ppm_line(const double* a, const double* chi, int n, double* aL, double* aR) {
  double* dm = (double*)calloc((size_t)n, sizeof(double));
  for (long i = 1; i < n - 1; i++) dm[i] = limited_slope(a[i - 1], a[i], a[i + 1]);
  for (long i = 2; i < n - 2; i++) {
    aL[i] = interface_value(a, dm, i, 1);
    aR[i] = interface_value(a, dm, i + 1, 1);
    limit_parabola(a[i], chi[i], &aL[i], &aR[i]);
  }
  free(dm);
}

/* limited slope of (am, a0, ap) */
double oracle_limited_slope(double am, double a0, double ap) { return limited_slope(am, a0, ap); }

/* tracing of a 1D line: q[5][n] normal-frame primitive, c[n], chi[n];
 * zones 2..n-3 get qm[5][n], qp[5][n] */
void oracle_trace_line(const double* q, const double* c, const double* chi, int n, double dtdx,
                       double* qm, double* qp) {
  const double* qn[5];
  const double* fc[5];
  double* dm = (double*)calloc((size_t)n, sizeof(double));
  double* face = (double*)calloc((size_t)5 * n, sizeof(double));
  for (int m = 0; m < 5; m++) {
    qn[m] = q + (long)m * n;
    fc[m] = face + (long)m * n;
    for (long i = 1; i < n - 1; i++) dm[i] = limited_slope(qn[m][i - 1], qn[m][i], qn[m][i + 1]);
    for (long i = 2; i < n - 1; i++) face[(long)m * n + i] = interface_value(qn[m], dm, i, 1);
  }
  for (long i = 2; i < n - 2; i++) {
    double a[5], bq[5];
    trace_zone(qn, fc, c, chi[i], i, 1, dtdx, 0, a, bq);
    for (int m = 0; m < 5; m++) {
      qm[(long)m * n + i] = a[m];
      qp[(long)m * n + i] = bq[m];
    }
  }
  free(dm);
  free(face);
}

/* Test instrumentation: branch-hit counters (OB_HIT_*, copied into out[0..n-1]
 * and cleared when reset != 0) and the R11 switch (1 on, the default; 0 off).
 * Neither changes what a step computes while R11 is on. */
int oracle_branch_hits(long* out, int n, int reset) {
  for (int k = 0; k < n && k < OB_NHITS; k++) out[k] = g_hits[k];
  if (reset)
    for (int k = 0; k < OB_NHITS; k++) g_hits[k] = 0;
  return OB_NHITS;
}

void oracle_set_wall_r11(int on) { g_wall_r11 = on ? 1 : 0; }

/* flattening coefficient of a 1D line along x: p[n], u[n]; zones 3..n-4 written */
void oracle_flatten_line(const double* p, const double* u, int n, double* f) {
  for (long i = 3; i < n - 3; i++) f[i] = flat_dir(p, u, i, 1);
}

}  /* extern "C" */
