/*
 * ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * Exact solution of the 1D Riemann problem for an ideal gamma-law gas,
 * following the method of Toro, "Riemann Solvers and Numerical Methods for
 * Fluid Dynamics", ch. 4: Newton iteration on the star pressure p* with the
 * shock/rarefaction pressure functions f_K, then sampling of the
 * self-similar solution at S = x/t.  It pins the whole hydro scheme on shock
 * tubes (the Sod problem along each axis).
 */
#include <math.h>

namespace {

struct Side {
  double rho, u, p, c;
};

/* pressure function f_K(p) and its derivative (Toro §4.2-4.3) */
void pressure_function(double p, const Side& K, double gamma, double* f, double* df) {
  if (p > K.p) {
    double A = 2.0 / ((gamma + 1.0) * K.rho);
    double B = (gamma - 1.0) / (gamma + 1.0) * K.p;
    double root = sqrt(A / (p + B));
    *f = (p - K.p) * root;
    *df = root * (1.0 - 0.5 * (p - K.p) / (B + p));
  } else {
    double ratio = p / K.p;
    *f = 2.0 * K.c / (gamma - 1.0) * (pow(ratio, (gamma - 1.0) / (2.0 * gamma)) - 1.0);
    *df = pow(ratio, -(gamma + 1.0) / (2.0 * gamma)) / (K.rho * K.c);
  }
}

int star_state(const Side& L, const Side& R, double gamma, double* pstar, double* ustar) {
  double du = R.u - L.u;
  if (2.0 / (gamma - 1.0) * (L.c + R.c) <= du) return -1; /* vacuum generated */
  /* starting guess: primitive-variable linearisation, kept positive */
  double p = 0.5 * (L.p + R.p) - 0.125 * du * (L.rho + R.rho) * (L.c + R.c);
  if (p < 1e-10) p = 1e-10;
  for (int it = 0; it < 200; it++) {
    double fl, dfl, fr, dfr;
    pressure_function(p, L, gamma, &fl, &dfl);
    pressure_function(p, R, gamma, &fr, &dfr);
    double pn = p - (fl + fr + du) / (dfl + dfr);
    if (pn < 1e-14) pn = 1e-14;
    double change = 2.0 * fabs(pn - p) / (pn + p);
    p = pn;
    if (change < 1e-15) break;
  }
  double fl, dfl, fr, dfr;
  pressure_function(p, L, gamma, &fl, &dfl);
  pressure_function(p, R, gamma, &fr, &dfr);
  *pstar = p;
  *ustar = 0.5 * (L.u + R.u) + 0.5 * (fr - fl);
  return 0;
}

/* sample the solution at S = x/t (Toro §4.5) */
void sample(const Side& L, const Side& R, double gamma, double ps, double us, double S,
            double* rho, double* u, double* p) {
  double g1 = (gamma - 1.0) / (2.0 * gamma);
  double g2 = (gamma + 1.0) / (2.0 * gamma);
  double gr = (gamma - 1.0) / (gamma + 1.0);
  if (S <= us) {
    if (ps > L.p) { /* left shock */
      double SL = L.u - L.c * sqrt(g2 * ps / L.p + g1);
      if (S <= SL) { *rho = L.rho; *u = L.u; *p = L.p; return; }
      *rho = L.rho * (ps / L.p + gr) / (gr * ps / L.p + 1.0);
      *u = us; *p = ps;
      return;
    }
    double SHL = L.u - L.c; /* left rarefaction */
    if (S <= SHL) { *rho = L.rho; *u = L.u; *p = L.p; return; }
    double cml = L.c * pow(ps / L.p, g1);
    double STL = us - cml;
    if (S > STL) { *rho = L.rho * pow(ps / L.p, 1.0 / gamma); *u = us; *p = ps; return; }
    double base = 2.0 / (gamma + 1.0) + (gamma - 1.0) / ((gamma + 1.0) * L.c) * (L.u - S);
    *rho = L.rho * pow(base, 2.0 / (gamma - 1.0));
    *u = 2.0 / (gamma + 1.0) * (L.c + 0.5 * (gamma - 1.0) * L.u + S);
    *p = L.p * pow(base, 2.0 * gamma / (gamma - 1.0));
    return;
  }
  if (ps > R.p) { /* right shock */
    double SR = R.u + R.c * sqrt(g2 * ps / R.p + g1);
    if (S >= SR) { *rho = R.rho; *u = R.u; *p = R.p; return; }
    *rho = R.rho * (ps / R.p + gr) / (gr * ps / R.p + 1.0);
    *u = us; *p = ps;
    return;
  }
  double SHR = R.u + R.c; /* right rarefaction */
  if (S >= SHR) { *rho = R.rho; *u = R.u; *p = R.p; return; }
  double cmr = R.c * pow(ps / R.p, g1);
  double STR = us + cmr;
  if (S < STR) { *rho = R.rho * pow(ps / R.p, 1.0 / gamma); *u = us; *p = ps; return; }
  double base = 2.0 / (gamma + 1.0) - (gamma - 1.0) / ((gamma + 1.0) * R.c) * (R.u - S);
  *rho = R.rho * pow(base, 2.0 / (gamma - 1.0));
  *u = 2.0 / (gamma + 1.0) * (-R.c + 0.5 * (gamma - 1.0) * R.u + S);
  *p = R.p * pow(base, 2.0 * gamma / (gamma - 1.0));
}

Side make_side(double rho, double u, double p, double gamma) {
  Side s;
  s.rho = rho; s.u = u; s.p = p; s.c = sqrt(gamma * p / rho);
  return s;
}

}  // namespace

extern "C" {

/* star pressure and velocity; returns -1 if the data generate vacuum */
int oracle_riemann_star(double rl, double ul, double pl, double rr, double ur, double pr,
                        double gamma, double* pstar, double* ustar) {
  Side L = make_side(rl, ul, pl, gamma), R = make_side(rr, ur, pr, gamma);
  return star_state(L, R, gamma, pstar, ustar);
}

/* exact (rho, u, p) at n similarity coordinates S[i] = x/t */
int oracle_riemann_sample(double rl, double ul, double pl, double rr, double ur, double pr,
                          double gamma, const double* S, int n, double* rho, double* u, double* p) {
  Side L = make_side(rl, ul, pl, gamma), R = make_side(rr, ur, pr, gamma);
  double ps, us;
  if (star_state(L, R, gamma, &ps, &us) != 0) return -1;
  for (int i = 0; i < n; i++) sample(L, R, gamma, ps, us, S[i], &rho[i], &u[i], &p[i]);
  return 0;
}

}  /* extern "C" */
