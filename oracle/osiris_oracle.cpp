/*
 * Serial FP64 CPU oracle for backward ray tracing of null geodesics in Kerr
 * space-time, following Velasquez-Cadavid et al., "OSIRIS: A New Code for Ray
 * Tracing Around Compact Objects" (arXiv:2202.00086).
 *
 * TEST INFRASTRUCTURE. This library exists only to check the CUDA path. The
 * test suite, the smoke check and the benchmark's CPU-baseline leg are the
 * only code allowed to load it. It shares no source, header, table or helper
 * with the CUDA library, and the CUDA library never calls it.
 *
 * What it computes, one pixel at a time, in plain double precision:
 *   1. initial momenta from the image-plane point (x, y) seen by a zero
 *      angular momentum observer at (r0, theta0)      -- Sec. 2.3, Eq. momentums
 *   2. Hamilton's equations in the paper's component form, with the Kerr
 *      contravariant metric and its r- and theta-derivatives written out
 *                                                      -- Sec. 2.1, Eqs. edm/ligH
 *                                                         and the explicit list
 *                                                         of t', r', ..., p_theta'
 *      on the Kerr metric in Boyer-Lindquist form      -- Sec. 4.3, Eq. Kerr
 *      or on the q-metric                                -- Appendix A, Eq. q-metric
 *      for null (H = 0) or time-like (H = -1/2) geodesics
 *   3. adaptive Runge-Kutta Cash-Karp 4(5) steps        -- Sec. 3.1 (RKCK45)
 *      or Dormand-Prince 5(4) steps                      -- Sec. 3.1 (RKDP45)
 *   4. the Hamiltonian-constraint error |H| at every accepted point
 *                                                      -- Sec. 3.1, Error = |H_num|
 *   5. termination on the horizon buffer, the celestial sphere, or the
 *      equatorial thin disk, each located by bisection of the last step
 *                                                      -- Sec. 4.1, Sec. 5
 *   6. observables: checkerboard cell of the celestial sphere, or the disk
 *      redshift g and observed intensity g^3 I_em     -- Sec. 4.1, Sec. 5
 *
 * Readings of points the paper leaves open (all listed in the design notes):
 *   - P^t = 1 at the observer, p_t = -E with E = 1/A_t + x g_tphi/(r0 sqrt(g_phph)),
 *     p_r < 0 (ingoing); pixel centres x_i = x_min + (i + 1/2)(x_max - x_min)/nx.
 *   - error norm: max over (r, theta, phi, p_r, p_theta) of
 *     |y5 - y4| / (tol (1 + max(|y_n|, |y_{n+1}|))); t is carried but not
 *     controlled. Accept when the norm is <= 1.
 *   - step factor: accept -> min(5, max(0.2, 0.9 err^-1/5));
 *                  reject -> max(0.1, 0.9 err^-1/4); first step 0.01 r0;
 *     every attempt limited to 0.1 r at its start.
 *   - after an accepted step the checks run in this order: equatorial crossing
 *     (disk mode), r < r_cap (captured), r > r_esc (escaped). A crossing is
 *     located by 52 bisections of the step length, re-stepping from the start
 *     of the step each time; the state at the upper end of the final bracket
 *     is the terminal state. A disk crossing outside [r_in, r_out] does not
 *     stop the ray; integration continues from the end of the accepted step.
 *   - redshift g = nu_obs / nu_em with nu_obs = P^t = 1 at the observer and
 *     nu_em = u^t (E - Omega L) for a Keplerian disk Omega = M^1/2 /(r^3/2 + a M^1/2)
 *     or a disk of constant l0 = -u_phi/u_t (the printed Omega of Sec. 5 has
 *     g_phph l0 where l0 = -u_phi/u_t gives g_tt l0); intensity I = g^3 r^-2.
 */

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

constexpr double kPi = 3.14159265358979323846;

// Ray fates. The numeric values are part of the library interface.
enum Status : int {
  kNone = 0,
  kCaptured = 1,
  kEscaped = 2,
  kDisk = 3,
  kMaxStep = 4,
  kError = 5,
};

enum SpacetimeKind { kKerr = 0, kQMetric = 1 };

struct Spacetime {
  double M;          // mass (the paper sets M = 1; M = 0 gives flat space)
  double a;          // Kerr spin parameter a = J / M
  int kind = kKerr;  // kKerr or kQMetric (Appendix A)
  double q = 0.0;    // quadrupole parameter of the q-metric
};

// ---------------------------------------------------------------------------
// Metric (Sec. 4.3, Eq. Kerr). Index order 0 = t, 1 = r, 2 = theta, 3 = phi.
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// q-metric (Appendix A, Eq. q-metric): static, axisymmetric, diagonal. The
// paper prints it with signature (+,-,-,-); with the (-,+,+,+) signature of
// Sec. 1 and f = 1 - 2m/r, X = 1 + m^2 sin^2 / (r^2 - 2 m r), k = q (2 + q):
//   g_tt = -f^(1+q),  g_rr = f^(-1-q) X^-k,  g_thth = f^-q r^2 X^-k,
//   g_phph = f^-q r^2 sin^2.   q = 0 is Schwarzschild.
// ---------------------------------------------------------------------------
void qmetric_cov(const Spacetime& S, double r, double th, double g[4][4]) {
  const double m = S.M, q = S.q, k = q * (2.0 + q);
  const double s = std::sin(th);
  const double f = 1.0 - 2.0 * m / r;
  const double X = 1.0 + m * m * s * s / (r * r - 2.0 * m * r);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) g[i][j] = 0.0;
  g[0][0] = -std::pow(f, 1.0 + q);
  g[1][1] = std::pow(f, -1.0 - q) * std::pow(X, -k);
  g[2][2] = std::pow(f, -q) * r * r * std::pow(X, -k);
  g[3][3] = std::pow(f, -q) * r * r * s * s;
}

void qmetric_con(const Spacetime& S, double r, double th, double gi[4][4]) {
  double g[4][4];
  qmetric_cov(S, r, th, g);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) gi[i][j] = 0.0;
  for (int i = 0; i < 4; ++i) gi[i][i] = 1.0 / g[i][i];
}

// r- and theta-derivatives of the diagonal g^{mu mu} of the q-metric, by the
// product and power rules:
//   g^tt = -f^(-1-q), g^rr = f^(1+q) X^k, g^thth = f^q X^k / r^2,
//   g^phph = f^q / (r^2 sin^2), with f_r = 2m/r^2, X_r = -m^2 sin^2 (2r - 2m)/(r^2 - 2mr)^2,
//   X_th = 2 m^2 sin cos / (r^2 - 2mr).
void qmetric_con_derivs(const Spacetime& S, double r, double th, double dr[4][4],
                        double dth[4][4]) {
  const double m = S.M, q = S.q, k = q * (2.0 + q);
  const double s = std::sin(th), c = std::cos(th);
  const double f = 1.0 - 2.0 * m / r;
  const double f_r = 2.0 * m / (r * r);
  const double D = r * r - 2.0 * m * r;
  const double X = 1.0 + m * m * s * s / D;
  const double X_r = -m * m * s * s * (2.0 * r - 2.0 * m) / (D * D);
  const double X_th = 2.0 * m * m * s * c / D;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      dr[i][j] = 0.0;
      dth[i][j] = 0.0;
    }
  const double fq = std::pow(f, q), Xk = std::pow(X, k);
  const double dfq = q * std::pow(f, q - 1.0) * f_r;  // d(f^q)/dr
  const double dXk_r = k * std::pow(X, k - 1.0) * X_r;
  const double dXk_th = k * std::pow(X, k - 1.0) * X_th;
  dr[0][0] = (1.0 + q) * std::pow(f, -2.0 - q) * f_r;
  dr[1][1] = (1.0 + q) * fq * f_r * Xk + std::pow(f, 1.0 + q) * dXk_r;
  dr[2][2] = (dfq * Xk + fq * dXk_r) / (r * r) - 2.0 * fq * Xk / (r * r * r);
  dr[3][3] = dfq / (r * r * s * s) - 2.0 * fq / (r * r * r * s * s);
  dth[1][1] = std::pow(f, 1.0 + q) * dXk_th;
  dth[2][2] = fq * dXk_th / (r * r);
  dth[3][3] = fq / (r * r) * (-2.0 * c / (s * s * s));
}

void metric_cov_kerr(const Spacetime& S, double r, double th, double g[4][4]);
void metric_con_kerr(const Spacetime& S, double r, double th, double gi[4][4]);
void metric_con_derivs_kerr(const Spacetime& S, double r, double th, double dr[4][4],
                            double dth[4][4]);

void metric_cov(const Spacetime& S, double r, double th, double g[4][4]) {
  if (S.kind == kQMetric)
    qmetric_cov(S, r, th, g);
  else
    metric_cov_kerr(S, r, th, g);
}

void metric_con(const Spacetime& S, double r, double th, double gi[4][4]) {
  if (S.kind == kQMetric)
    qmetric_con(S, r, th, gi);
  else
    metric_con_kerr(S, r, th, gi);
}

void metric_con_derivs(const Spacetime& S, double r, double th, double dr[4][4],
                       double dth[4][4]) {
  if (S.kind == kQMetric)
    qmetric_con_derivs(S, r, th, dr, dth);
  else
    metric_con_derivs_kerr(S, r, th, dr, dth);
}

// Covariant components g_{mu nu} of the Kerr line element.
void metric_cov_kerr(const Spacetime& S, double r, double th, double g[4][4]) {
  const double M = S.M, a = S.a;
  const double s = std::sin(th), c = std::cos(th);
  const double Sigma = r * r + a * a * c * c;
  const double Delta = r * r - 2.0 * M * r + a * a;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) g[i][j] = 0.0;
  g[0][0] = -(1.0 - 2.0 * M * r / Sigma);
  // The line element's -(4 M r a sin^2 / Sigma) dt (x) dphi term is the sum of
  // the two equal off-diagonal components.
  g[0][3] = -2.0 * M * r * a * s * s / Sigma;
  g[3][0] = g[0][3];
  g[1][1] = Sigma / Delta;
  g[2][2] = Sigma;
  g[3][3] = s * s * (r * r + a * a + 2.0 * M * r * a * a * s * s / Sigma);
}

// Contravariant components g^{mu nu}: the inverse of metric_cov, in closed form.
//   g^tt = -[(r^2+a^2)^2 - a^2 Delta sin^2] / (Sigma Delta)
//   g^tphi = -2 M a r / (Sigma Delta)
//   g^phph = (Delta - a^2 sin^2) / (Sigma Delta sin^2)
//   g^rr = Delta / Sigma,  g^thth = 1 / Sigma
void metric_con_kerr(const Spacetime& S, double r, double th, double gi[4][4]) {
  const double M = S.M, a = S.a;
  const double s = std::sin(th), c = std::cos(th);
  const double s2 = s * s;
  const double Sigma = r * r + a * a * c * c;
  const double Delta = r * r - 2.0 * M * r + a * a;
  const double D = Sigma * Delta;
  const double A = (r * r + a * a) * (r * r + a * a) - a * a * Delta * s2;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) gi[i][j] = 0.0;
  gi[0][0] = -A / D;
  gi[0][3] = -2.0 * M * a * r / D;
  gi[3][0] = gi[0][3];
  gi[1][1] = Delta / Sigma;
  gi[2][2] = 1.0 / Sigma;
  gi[3][3] = (Delta - a * a * s2) / (D * s2);
}

// Partial derivatives of g^{mu nu} with respect to r (dr) and theta (dth),
// obtained by differentiating the closed forms above by hand with the
// quotient rule.
void metric_con_derivs_kerr(const Spacetime& S, double r, double th, double dr[4][4],
                            double dth[4][4]) {
  const double M = S.M, a = S.a;
  const double s = std::sin(th), c = std::cos(th);
  const double s2 = s * s;
  const double Sigma = r * r + a * a * c * c;
  const double Delta = r * r - 2.0 * M * r + a * a;
  const double D = Sigma * Delta;
  const double A = (r * r + a * a) * (r * r + a * a) - a * a * Delta * s2;
  const double B = Delta - a * a * s2;  // numerator of g^phph
  const double C = D * s2;              // denominator of g^phph

  // r-derivatives of the building blocks.
  const double Sigma_r = 2.0 * r;
  const double Delta_r = 2.0 * r - 2.0 * M;
  const double D_r = Sigma_r * Delta + Sigma * Delta_r;
  const double A_r = 4.0 * r * (r * r + a * a) - a * a * s2 * Delta_r;
  const double B_r = Delta_r;
  const double C_r = D_r * s2;

  // theta-derivatives of the building blocks (Delta does not depend on theta).
  const double Sigma_th = -2.0 * a * a * s * c;
  const double s2_th = 2.0 * s * c;
  const double D_th = Sigma_th * Delta;
  const double A_th = -a * a * Delta * s2_th;
  const double B_th = -a * a * s2_th;
  const double C_th = D_th * s2 + D * s2_th;

  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      dr[i][j] = 0.0;
      dth[i][j] = 0.0;
    }

  dr[0][0] = -(A_r * D - A * D_r) / (D * D);
  dr[0][3] = -2.0 * M * a * (D - r * D_r) / (D * D);
  dr[3][0] = dr[0][3];
  dr[1][1] = (Delta_r * Sigma - Delta * Sigma_r) / (Sigma * Sigma);
  dr[2][2] = -Sigma_r / (Sigma * Sigma);
  dr[3][3] = (B_r * C - B * C_r) / (C * C);

  dth[0][0] = -(A_th * D - A * D_th) / (D * D);
  dth[0][3] = 2.0 * M * a * r * D_th / (D * D);
  dth[3][0] = dth[0][3];
  dth[1][1] = -Delta * Sigma_th / (Sigma * Sigma);
  dth[2][2] = -Sigma_th / (Sigma * Sigma);
  dth[3][3] = (B_th * C - B * C_th) / (C * C);
}

// ---------------------------------------------------------------------------
// Hamiltonian and equations of motion (Sec. 2.1).
// State vector: y = (t, r, theta, phi, p_r, p_theta); p_t = -E and p_phi = L
// are constants of motion (their equations of motion are zero).
// ---------------------------------------------------------------------------

enum { Y_T = 0, Y_R = 1, Y_TH = 2, Y_PH = 3, Y_PR = 4, Y_PTH = 5, NY = 6 };

struct Ray {
  double E;  // -p_t
  double L;  // p_phi
};

// H = 1/2 g^{mu nu} p_mu p_nu (Eq. ligH).
double hamiltonian(const Spacetime& S, const Ray& R, const double y[NY]) {
  double gi[4][4];
  metric_con(S, y[Y_R], y[Y_TH], gi);
  const double pt = -R.E, pr = y[Y_PR], pth = y[Y_PTH], pph = R.L;
  return 0.5 * (gi[0][0] * pt * pt + 2.0 * gi[0][3] * pt * pph + gi[1][1] * pr * pr +
                gi[2][2] * pth * pth + gi[3][3] * pph * pph);
}

// Carter constant Q = p_theta^2 + cos^2 theta (L^2 / sin^2 theta - a^2 E^2);
// used only as a diagnostic (it is conserved by the exact flow).
double carter(const Spacetime& S, const Ray& R, const double y[NY]) {
  const double s = std::sin(y[Y_TH]), c = std::cos(y[Y_TH]);
  return y[Y_PTH] * y[Y_PTH] + c * c * (R.L * R.L / (s * s) - S.a * S.a * R.E * R.E);
}

// The explicit motion equations of Sec. 2.1, term by term.
void rhs(const Spacetime& S, const Ray& R, const double y[NY], double dy[NY]) {
  double gi[4][4], dr[4][4], dth[4][4];
  metric_con(S, y[Y_R], y[Y_TH], gi);
  metric_con_derivs(S, y[Y_R], y[Y_TH], dr, dth);
  const double pt = -R.E, pr = y[Y_PR], pth = y[Y_PTH], pph = R.L;

  dy[Y_T] = gi[0][0] * pt + gi[0][3] * pph;
  dy[Y_R] = gi[1][1] * pr;
  dy[Y_TH] = gi[2][2] * pth;
  dy[Y_PH] = gi[0][3] * pt + gi[3][3] * pph;
  dy[Y_PR] = (-pt * pt * dr[0][0] - 2.0 * pt * pph * dr[0][3] - pr * pr * dr[1][1] -
              pth * pth * dr[2][2] - pph * pph * dr[3][3]) /
             2.0;
  dy[Y_PTH] = (-pt * pt * dth[0][0] - pr * pr * dth[1][1] - pth * pth * dth[2][2] -
               pph * (2.0 * pt * dth[0][3] + pph * dth[3][3])) /
              2.0;
}

// ---------------------------------------------------------------------------
// Runge-Kutta Cash-Karp 4(5) (Sec. 3.1; Cash & Karp 1990).
// ---------------------------------------------------------------------------

struct Tableau {
  int stages;    // 6 (Cash-Karp) or 7 (Dormand-Prince)
  double c[7];
  double a[7][7];
  double b5[7];  // fifth-order weights (the solution that is propagated)
  double b4[7];  // embedded fourth-order weights
};

Tableau make_cash_karp() {
  Tableau T;
  std::memset(&T, 0, sizeof(T));
  T.stages = 6;
  T.c[0] = 0.0;
  T.c[1] = 1.0 / 5.0;
  T.c[2] = 3.0 / 10.0;
  T.c[3] = 3.0 / 5.0;
  T.c[4] = 1.0;
  T.c[5] = 7.0 / 8.0;

  T.a[1][0] = 1.0 / 5.0;

  T.a[2][0] = 3.0 / 40.0;
  T.a[2][1] = 9.0 / 40.0;

  T.a[3][0] = 3.0 / 10.0;
  T.a[3][1] = -9.0 / 10.0;
  T.a[3][2] = 6.0 / 5.0;

  T.a[4][0] = -11.0 / 54.0;
  T.a[4][1] = 5.0 / 2.0;
  T.a[4][2] = -70.0 / 27.0;
  T.a[4][3] = 35.0 / 27.0;

  T.a[5][0] = 1631.0 / 55296.0;
  T.a[5][1] = 175.0 / 512.0;
  T.a[5][2] = 575.0 / 13824.0;
  T.a[5][3] = 44275.0 / 110592.0;
  T.a[5][4] = 253.0 / 4096.0;

  T.b5[0] = 37.0 / 378.0;
  T.b5[1] = 0.0;
  T.b5[2] = 250.0 / 621.0;
  T.b5[3] = 125.0 / 594.0;
  T.b5[4] = 0.0;
  T.b5[5] = 512.0 / 1771.0;

  T.b4[0] = 2825.0 / 27648.0;
  T.b4[1] = 0.0;
  T.b4[2] = 18575.0 / 48384.0;
  T.b4[3] = 13525.0 / 55296.0;
  T.b4[4] = 277.0 / 14336.0;
  T.b4[5] = 1.0 / 4.0;
  return T;
}

// Dormand & Prince (1980) 5(4), the RKDP45 scheme of Sec. 3.1: seven stages,
// the last evaluated at the fifth-order solution (first same as last), so a
// step costs six new evaluations.
Tableau make_dormand_prince() {
  Tableau T;
  std::memset(&T, 0, sizeof(T));
  T.stages = 7;
  T.c[0] = 0.0;
  T.c[1] = 1.0 / 5.0;
  T.c[2] = 3.0 / 10.0;
  T.c[3] = 4.0 / 5.0;
  T.c[4] = 8.0 / 9.0;
  T.c[5] = 1.0;
  T.c[6] = 1.0;

  T.a[1][0] = 1.0 / 5.0;

  T.a[2][0] = 3.0 / 40.0;
  T.a[2][1] = 9.0 / 40.0;

  T.a[3][0] = 44.0 / 45.0;
  T.a[3][1] = -56.0 / 15.0;
  T.a[3][2] = 32.0 / 9.0;

  T.a[4][0] = 19372.0 / 6561.0;
  T.a[4][1] = -25360.0 / 2187.0;
  T.a[4][2] = 64448.0 / 6561.0;
  T.a[4][3] = -212.0 / 729.0;

  T.a[5][0] = 9017.0 / 3168.0;
  T.a[5][1] = -355.0 / 33.0;
  T.a[5][2] = 46732.0 / 5247.0;
  T.a[5][3] = 49.0 / 176.0;
  T.a[5][4] = -5103.0 / 18656.0;

  T.a[6][0] = 35.0 / 384.0;
  T.a[6][1] = 0.0;
  T.a[6][2] = 500.0 / 1113.0;
  T.a[6][3] = 125.0 / 192.0;
  T.a[6][4] = -2187.0 / 6784.0;
  T.a[6][5] = 11.0 / 84.0;

  for (int j = 0; j < 7; ++j) T.b5[j] = T.a[6][j];  // b5 = last row, b5[6] = 0

  T.b4[0] = 5179.0 / 57600.0;
  T.b4[1] = 0.0;
  T.b4[2] = 7571.0 / 16695.0;
  T.b4[3] = 393.0 / 640.0;
  T.b4[4] = -92097.0 / 339200.0;
  T.b4[5] = 187.0 / 2100.0;
  T.b4[6] = 1.0 / 40.0;
  return T;
}

const Tableau kCK = make_cash_karp();
const Tableau kDP = make_dormand_prince();

enum Integrator { kRKCK45 = 0, kRKDP45 = 1 };

const Tableau& tableau(int integrator) { return integrator == kRKDP45 ? kDP : kCK; }

// One embedded Runge-Kutta step of length h from y with tableau T: y5 is the
// fifth-order result and delta = y5 - y4 the embedded error estimate. Every
// stage is evaluated here (the first-same-as-last saving of Dormand-Prince is
// an optimisation that does not change the result).
void rk_step(const Tableau& T, const Spacetime& S, const Ray& R, const double y[NY], double h,
             double y5[NY], double delta[NY]) {
  double k[7][NY];
  double yi[NY];
  for (int stage = 0; stage < T.stages; ++stage) {
    for (int n = 0; n < NY; ++n) {
      double acc = 0.0;
      for (int j = 0; j < stage; ++j) acc += T.a[stage][j] * k[j][n];
      yi[n] = y[n] + h * acc;
    }
    rhs(S, R, yi, k[stage]);
  }
  for (int n = 0; n < NY; ++n) {
    double s5 = 0.0, sd = 0.0;
    for (int j = 0; j < T.stages; ++j) {
      s5 += T.b5[j] * k[j][n];
      sd += (T.b5[j] - T.b4[j]) * k[j][n];
    }
    y5[n] = y[n] + h * s5;
    delta[n] = h * sd;
  }
}

// ---------------------------------------------------------------------------
// Camera: image-plane point -> initial data (Sec. 2.3).
// ---------------------------------------------------------------------------

struct Camera {
  Spacetime S;
  double r0;       // observer radius
  double th0;      // observer polar angle (inclination)
  double x_min, x_max, y_min, y_max;
  int nx, ny;
};

// Initial state for the image-plane point (x, y): the observer's frame has
// P^t = 1, and the tetrad of the matrix Lambda gives
//   p_theta = y sqrt(g_thth) / r0,   L = -x sqrt(g_phph) / r0,
//   E = 1/A_t + x g_tphi / (r0 sqrt(g_phph)),
//   p_r = -sqrt(g_rr (1 - (y/r0)^2 - (x/r0)^2))        (ingoing ray),
//   A_t = sqrt(g_phph / (g_tphi^2 - g_tt g_phph)),
// at t = 0, r = r0, theta = theta0, phi = 0.
void init_ray(const Camera& cam, double x, double y, Ray* R, double st[NY]) {
  double g[4][4];
  metric_cov(cam.S, cam.r0, cam.th0, g);
  const double gtt = g[0][0], gtph = g[0][3], grr = g[1][1], gthth = g[2][2], gphph = g[3][3];
  const double At = std::sqrt(gphph / (gtph * gtph - gtt * gphph));
  const double r0 = cam.r0;
  const double Ptheta = y / r0;  // P^theta / P^t with P^t = 1
  const double Pphi = -x / r0;   // P^phi / P^t
  R->E = 1.0 / At + x * gtph / (r0 * std::sqrt(gphph));
  R->L = -x * std::sqrt(gphph) / r0;
  st[Y_T] = 0.0;
  st[Y_R] = r0;
  st[Y_TH] = cam.th0;
  st[Y_PH] = 0.0;
  st[Y_PTH] = y * std::sqrt(gthth) / r0;
  st[Y_PR] = -std::sqrt(grr * (1.0 - Ptheta * Ptheta - Pphi * Pphi));
}

double pixel_x(const Camera& cam, int64_t i) {
  return cam.x_min + (static_cast<double>(i) + 0.5) * (cam.x_max - cam.x_min) / cam.nx;
}
double pixel_y(const Camera& cam, int64_t j) {
  return cam.y_min + (static_cast<double>(j) + 0.5) * (cam.y_max - cam.y_min) / cam.ny;
}

// ---------------------------------------------------------------------------
// Integration of one ray.
// ---------------------------------------------------------------------------

struct Options {
  int integrator;        // kRKCK45 or kRKDP45
  double tol;            // per-step error tolerance
  int64_t max_steps;     // cap on accepted + rejected attempts
  double r_cap_factor;   // captured when r < r_cap_factor * r_H
  double r_esc_factor;   // escaped when r > r_esc_factor * r0
  int disk;              // 1: stop on the equatorial disk r_in <= r <= r_out
  double r_in, r_out;
  double cell_deg;       // checkerboard cell size on the celestial sphere
  double cell_phase_deg; // longitude offset of the checkerboard
  int disk_model;        // kKeplerian or kConstantL
  double l0;             // specific angular momentum of the constant-l0 disk
  double mass2;          // 0: null geodesics (H = 0); 1: time-like (H = -1/2), Sec. 2.1
};

struct Result {
  int status;
  double y[NY];  // terminal state
  double E, L;
  double max_abs_H;
  int64_t accepted, rejected, bisection_steps;
  int cell_i, cell_j, parity;
  double g, intensity, r_hit;
  double carter0, max_carter_drift;
};

// Inner stopping surface scale: the Kerr event horizon r_H = M + sqrt(M^2 - a^2)
// (Sec. 4.3), or the singular surface r = 2m of the q-metric (Appendix A).
double horizon_radius(const Spacetime& S) {
  if (S.kind == kQMetric) return 2.0 * S.M;
  return S.M + std::sqrt(S.M * S.M - S.a * S.a);
}

// Which side of the stopping surface a state lies on.
enum Surface { kEquator, kCapture, kEscape };

double surface_function(Surface kind, const double y[NY], double r_cap, double r_esc) {
  switch (kind) {
    case kEquator: return std::cos(y[Y_TH]);
    case kCapture: return y[Y_R] - r_cap;
    default: return y[Y_R] - r_esc;
  }
}

// Bisection of the last step length (Sec. 4.1 stopping surfaces; the disk of
// Sec. 5): the root of F(step(y, h')) for h' in [0, h] is bracketed and
// halved 52 times. Returns the upper end of the bracket and the state there.
double bisect_step(const Tableau& T, const Spacetime& S, const Ray& R, const double y[NY],
                   double h, Surface kind, double r_cap, double r_esc, double y_out[NY],
                   int64_t* n_steps) {
  double lo = 0.0, hi = h;
  const bool start_positive = surface_function(kind, y, r_cap, r_esc) > 0.0;
  double ytry[NY], dtry[NY];
  for (int it = 0; it < 52; ++it) {
    const double mid = 0.5 * (lo + hi);
    rk_step(T, S, R, y, mid, ytry, dtry);
    ++*n_steps;
    const double f = surface_function(kind, ytry, r_cap, r_esc);
    if ((f > 0.0) == start_positive && f != 0.0)
      lo = mid;
    else
      hi = mid;
  }
  rk_step(T, S, R, y, hi, y_out, dtry);
  ++*n_steps;
  return hi;
}

bool crosses_equator(const double y0[NY], const double y1[NY]) {
  const double c0 = std::cos(y0[Y_TH]), c1 = std::cos(y1[Y_TH]);
  return (c0 > 0.0 && c1 <= 0.0) || (c0 < 0.0 && c1 >= 0.0);
}

enum DiskModel { kKeplerian = 0, kConstantL = 1 };

// Redshift and intensity at the disk point r (Sec. 5). The gas moves on
// circular orbits with angular velocity Omega:
//   Keplerian:               Omega = M^1/2 / (r^3/2 + a M^1/2)
//   constant specific angular momentum l0 = -u_phi / u_t (Sec. 5):
//                            Omega = -(g_tphi + l0 g_tt) / (g_phph + l0 g_tphi)
// u^t follows from g_ab u^a u^b = -1 (Eq. norm) in the equatorial plane,
// g = 1 / (u^t (E - Omega L)) and I = g^3 r^-2. Where no timelike orbit with
// that Omega exists (the normalisation has no real solution), g = I = 0.
void disk_observables(const Spacetime& S, const Ray& R, double r, int model, double l0,
                      double* g_out, double* I_out) {
  double g[4][4];
  metric_cov(S, r, 0.5 * kPi, g);
  double Omega;
  if (model == kConstantL) {
    Omega = -(g[0][3] + l0 * g[0][0]) / (g[3][3] + l0 * g[0][3]);
  } else {
    const double sqM = std::sqrt(S.M);
    Omega = sqM / (std::pow(r, 1.5) + S.a * sqM);
  }
  const double norm = -g[0][0] - 2.0 * Omega * g[0][3] - Omega * Omega * g[3][3];
  if (!(norm > 0.0)) {
    *g_out = 0.0;
    *I_out = 0.0;
    return;
  }
  const double ut = 1.0 / std::sqrt(norm);
  const double redshift = 1.0 / (ut * (R.E - Omega * R.L));
  *g_out = redshift;
  *I_out = redshift * redshift * redshift / (r * r);
}

// Celestial-sphere cell of an escaped ray: theta folded into [0, pi] (with
// phi moved by pi when the fold happens), phi wrapped into [0, 2 pi) after the
// checkerboard phase is added.
void sky_cell(const Options& o, double th, double ph, int* ci, int* cj, int* parity) {
  const double two_pi = 2.0 * kPi;
  double t = std::fmod(th, two_pi);
  if (t < 0.0) t += two_pi;
  double p = ph;
  if (t > kPi) {
    t = two_pi - t;
    p += kPi;
  }
  const double cell = o.cell_deg * kPi / 180.0;
  const double phase = o.cell_phase_deg * kPi / 180.0;
  double q = std::fmod(p + phase, two_pi);
  if (q < 0.0) q += two_pi;
  const int n_th = static_cast<int>(std::ceil(180.0 / o.cell_deg - 1e-9));
  const int n_ph = static_cast<int>(std::ceil(360.0 / o.cell_deg - 1e-9));
  int i = static_cast<int>(std::floor(t / cell));
  int j = static_cast<int>(std::floor(q / cell));
  if (i > n_th - 1) i = n_th - 1;
  if (i < 0) i = 0;
  j = ((j % n_ph) + n_ph) % n_ph;
  *ci = i;
  *cj = j;
  *parity = (i + j) & 1;
}

Result integrate(const Spacetime& S, const Ray& R, const double y_init[NY], double r0,
                 const Options& o) {
  Result out;
  std::memset(&out, 0, sizeof(out));
  out.E = R.E;
  out.L = R.L;
  out.status = kNone;
  out.cell_i = out.cell_j = -1;
  out.parity = 0;
  out.g = out.intensity = out.r_hit = 0.0;

  const double r_cap = o.r_cap_factor * horizon_radius(S);
  const double r_esc = o.r_esc_factor * r0;
  const Tableau& T = tableau(o.integrator);

  double y[NY];
  std::memcpy(y, y_init, sizeof(y));
  double h = 0.01 * r0;
  // Error = |H_num - H| (Sec. 3.1) with H = -mass2 / 2 on the mass shell
  const double H_shell = -0.5 * o.mass2;
  double max_H = std::fabs(hamiltonian(S, R, y) - H_shell);
  const double Q0 = carter(S, R, y);
  double max_dQ = 0.0;
  double y5[NY], delta[NY], yfin[NY];
  int64_t acc = 0, rej = 0, bis = 0;

  // Components under error control: r, theta, phi, p_r, p_theta.
  const int controlled[5] = {Y_R, Y_TH, Y_PH, Y_PR, Y_PTH};

  while (true) {
    if (acc + rej >= o.max_steps) {
      out.status = kMaxStep;
      std::memcpy(yfin, y, sizeof(y));
      break;
    }
    const double hs = std::min(h, 0.1 * y[Y_R]);
    rk_step(T, S, R, y, hs, y5, delta);

    double err = 0.0;
    for (int m = 0; m < 5; ++m) {
      const int n = controlled[m];
      const double scale = o.tol * (1.0 + std::max(std::fabs(y[n]), std::fabs(y5[n])));
      err = std::max(err, std::fabs(delta[n]) / scale);
    }
    if (!std::isfinite(err)) {
      out.status = kError;
      std::memcpy(yfin, y, sizeof(y));
      break;
    }

    if (err <= 1.0) {
      ++acc;
      const double grow = (err == 0.0) ? 5.0 : 0.9 * std::pow(err, -0.2);
      h = hs * std::min(5.0, std::max(0.2, grow));

      if (o.disk && crosses_equator(y, y5)) {
        double yc[NY];
        bisect_step(T, S, R, y, hs, kEquator, r_cap, r_esc, yc, &bis);
        if (yc[Y_R] >= o.r_in && yc[Y_R] <= o.r_out) {
          out.status = kDisk;
          std::memcpy(yfin, yc, sizeof(yc));
          break;
        }
      }
      if (y5[Y_R] < r_cap) {
        bisect_step(T, S, R, y, hs, kCapture, r_cap, r_esc, yfin, &bis);
        out.status = kCaptured;
        break;
      }
      if (y5[Y_R] > r_esc) {
        bisect_step(T, S, R, y, hs, kEscape, r_cap, r_esc, yfin, &bis);
        out.status = kEscaped;
        break;
      }
      std::memcpy(y, y5, sizeof(y));
      max_H = std::max(max_H, std::fabs(hamiltonian(S, R, y) - H_shell));
      max_dQ = std::max(max_dQ, std::fabs(carter(S, R, y) - Q0));
    } else {
      ++rej;
      const double shrink = 0.9 * std::pow(err, -0.25);
      h = hs * std::max(0.1, shrink);
    }
  }

  if (out.status != kError) {
    max_H = std::max(max_H, std::fabs(hamiltonian(S, R, yfin) - H_shell));
    max_dQ = std::max(max_dQ, std::fabs(carter(S, R, yfin) - Q0));
  }
  std::memcpy(out.y, yfin, sizeof(yfin));
  out.max_abs_H = max_H;
  out.accepted = acc;
  out.rejected = rej;
  out.bisection_steps = bis;
  out.carter0 = Q0;
  out.max_carter_drift = max_dQ;

  if (out.status == kEscaped) {
    sky_cell(o, yfin[Y_TH], yfin[Y_PH], &out.cell_i, &out.cell_j, &out.parity);
  } else if (out.status == kDisk) {
    out.r_hit = yfin[Y_R];
    disk_observables(S, R, yfin[Y_R], o.disk_model, o.l0, &out.g, &out.intensity);
  }
  return out;
}

}  // namespace

// ===========================================================================
// C interface (loaded with ctypes by the test suite and the benchmark's CPU
// baseline leg).
// ===========================================================================

extern "C" {

// Per-ray outputs; any pointer may be NULL. Arrays hold `count` entries.
struct oracle_outputs {
  int32_t* status;
  double* t;
  double* r;
  double* theta;
  double* phi;
  double* p_r;
  double* p_theta;
  double* E;
  double* L;
  double* max_abs_H;
  int64_t* accepted;
  int64_t* rejected;
  int64_t* bisection_steps;
  int32_t* cell_i;
  int32_t* cell_j;
  int32_t* parity;
  double* g;
  double* intensity;
  double* r_hit;
  double* carter0;
  double* max_carter_drift;
};

struct oracle_options {
  double tol;
  int64_t max_steps;
  double r_cap_factor;
  double r_esc_factor;
  int32_t disk;
  double r_in;
  double r_out;
  double cell_deg;
  double cell_phase_deg;
  int32_t integrator;  // 0 = Cash-Karp 4(5), 1 = Dormand-Prince 5(4)
  int32_t disk_model;  // 0 = Keplerian, 1 = constant specific angular momentum l0
  double l0;
  int32_t spacetime;   // 0 = Kerr (parameter a), 1 = q-metric (parameter q)
  double q;
  double mass2;        // 0 = null, 1 = time-like
};

static void store(const Result& R, oracle_outputs* o, int64_t k) {
  if (o->status) o->status[k] = R.status;
  if (o->t) o->t[k] = R.y[Y_T];
  if (o->r) o->r[k] = R.y[Y_R];
  if (o->theta) o->theta[k] = R.y[Y_TH];
  if (o->phi) o->phi[k] = R.y[Y_PH];
  if (o->p_r) o->p_r[k] = R.y[Y_PR];
  if (o->p_theta) o->p_theta[k] = R.y[Y_PTH];
  if (o->E) o->E[k] = R.E;
  if (o->L) o->L[k] = R.L;
  if (o->max_abs_H) o->max_abs_H[k] = R.max_abs_H;
  if (o->accepted) o->accepted[k] = R.accepted;
  if (o->rejected) o->rejected[k] = R.rejected;
  if (o->bisection_steps) o->bisection_steps[k] = R.bisection_steps;
  if (o->cell_i) o->cell_i[k] = R.cell_i;
  if (o->cell_j) o->cell_j[k] = R.cell_j;
  if (o->parity) o->parity[k] = R.parity;
  if (o->g) o->g[k] = R.g;
  if (o->intensity) o->intensity[k] = R.intensity;
  if (o->r_hit) o->r_hit[k] = R.r_hit;
  if (o->carter0) o->carter0[k] = R.carter0;
  if (o->max_carter_drift) o->max_carter_drift[k] = R.max_carter_drift;
}

static Options to_options(const oracle_options* oo) {
  Options o;
  o.integrator = oo->integrator;
  o.tol = oo->tol;
  o.max_steps = oo->max_steps;
  o.r_cap_factor = oo->r_cap_factor;
  o.r_esc_factor = oo->r_esc_factor;
  o.disk = oo->disk;
  o.r_in = oo->r_in;
  o.r_out = oo->r_out;
  o.cell_deg = oo->cell_deg;
  o.cell_phase_deg = oo->cell_phase_deg;
  o.disk_model = oo->disk_model;
  o.l0 = oo->l0;
  o.mass2 = oo->mass2;
  return o;
}

// Trace the pixels with linear indices idx[0..count) (index = j * nx + i) of
// the camera; results go to slot k of every output array. Work is spread over
// `nthreads` threads in chunks of 64 pixels; each ray is integrated serially.
int oracle_trace_pixels(double M, double a, double r0, double incl_deg, double x_min,
                        double x_max, double y_min, double y_max, int32_t nx, int32_t ny,
                        const oracle_options* opts, const int64_t* idx, int64_t count,
                        int32_t nthreads, oracle_outputs* out) {
  Camera cam;
  cam.S.M = M;
  cam.S.a = a;
  cam.S.kind = opts->spacetime;
  cam.S.q = opts->q;
  cam.r0 = r0;
  cam.th0 = incl_deg * kPi / 180.0;
  cam.x_min = x_min;
  cam.x_max = x_max;
  cam.y_min = y_min;
  cam.y_max = y_max;
  cam.nx = nx;
  cam.ny = ny;
  const Options o = to_options(opts);

  std::atomic<int64_t> next(0);
  auto worker = [&]() {
    while (true) {
      const int64_t k0 = next.fetch_add(64);
      if (k0 >= count) break;
      const int64_t k1 = std::min<int64_t>(count, k0 + 64);
      for (int64_t k = k0; k < k1; ++k) {
        const int64_t pix = idx ? idx[k] : k;
        const int64_t i = pix % nx, j = pix / nx;
        Ray R;
        double y0[NY];
        init_ray(cam, pixel_x(cam, i), pixel_y(cam, j), &R, y0);
        const Result res = integrate(cam.S, R, y0, r0, o);
        store(res, out, k);
      }
    }
  };
  const int nt = std::max(1, nthreads);
  if (nt == 1) {
    worker();
  } else {
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
    for (auto& th : pool) th.join();
  }
  return 0;
}

// Trace rays from explicit initial data: state rows (t, r, theta, phi, p_r,
// p_theta) and constants E, L; r0 sets the escape radius r_esc_factor * r0.
int oracle_trace_states(double M, double a, double r0, const oracle_options* opts,
                        const double* states, const double* E, const double* L, int64_t count,
                        oracle_outputs* out) {
  Spacetime S{M, a, opts->spacetime, opts->q};
  const Options o = to_options(opts);
  for (int64_t k = 0; k < count; ++k) {
    Ray R{E[k], L[k]};
    const Result res = integrate(S, R, states + NY * k, r0, o);
    store(res, out, k);
  }
  return 0;
}

// Initial data of one image-plane point: out = (t, r, theta, phi, p_r,
// p_theta, E, L).
void oracle_init_ray(double M, double a, double r0, double incl_deg, double x, double y,
                     double* out8) {
  Camera cam;
  std::memset(&cam, 0, sizeof(cam));
  cam.S.M = M;
  cam.S.a = a;
  cam.r0 = r0;
  cam.th0 = incl_deg * kPi / 180.0;
  Ray R;
  double st[NY];
  init_ray(cam, x, y, &R, st);
  for (int n = 0; n < NY; ++n) out8[n] = st[n];
  out8[6] = R.E;
  out8[7] = R.L;
}

// Metric functions for either space-time: kind 0 = Kerr (a), 1 = q-metric (q).
void oracle_metric_sp(int32_t kind, double M, double a, double q, double r, double th,
                      double* cov16, double* con16, double* dr16, double* dth16) {
  const Spacetime S{M, a, kind, q};
  double g[4][4], gi[4][4], dr[4][4], dth[4][4];
  metric_cov(S, r, th, g);
  metric_con(S, r, th, gi);
  metric_con_derivs(S, r, th, dr, dth);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      cov16[4 * i + j] = g[i][j];
      con16[4 * i + j] = gi[i][j];
      dr16[4 * i + j] = dr[i][j];
      dth16[4 * i + j] = dth[i][j];
    }
}

double oracle_hamiltonian_sp(int32_t kind, double M, double a, double q, const double* y6,
                             double E, double L) {
  return hamiltonian(Spacetime{M, a, kind, q}, Ray{E, L}, y6);
}

void oracle_rhs_sp(int32_t kind, double M, double a, double q, const double* y6, double E,
                   double L, double* dy6) {
  rhs(Spacetime{M, a, kind, q}, Ray{E, L}, y6, dy6);
}

void oracle_init_ray_sp(int32_t kind, double M, double a, double q, double r0, double incl_deg,
                        double x, double y, double* out8) {
  Camera cam;
  std::memset(&cam, 0, sizeof(cam));
  cam.S = Spacetime{M, a, kind, q};
  cam.r0 = r0;
  cam.th0 = incl_deg * kPi / 180.0;
  Ray R;
  double st[NY];
  init_ray(cam, x, y, &R, st);
  for (int n = 0; n < NY; ++n) out8[n] = st[n];
  out8[6] = R.E;
  out8[7] = R.L;
}

void oracle_metric_cov(double M, double a, double r, double th, double* g16) {
  double g[4][4];
  metric_cov(Spacetime{M, a}, r, th, g);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) g16[4 * i + j] = g[i][j];
}

void oracle_metric_con(double M, double a, double r, double th, double* g16) {
  double g[4][4];
  metric_con(Spacetime{M, a}, r, th, g);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) g16[4 * i + j] = g[i][j];
}

void oracle_metric_con_derivs(double M, double a, double r, double th, double* dr16,
                              double* dth16) {
  double dr[4][4], dth[4][4];
  metric_con_derivs(Spacetime{M, a}, r, th, dr, dth);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      dr16[4 * i + j] = dr[i][j];
      dth16[4 * i + j] = dth[i][j];
    }
}

double oracle_hamiltonian(double M, double a, const double* y6, double E, double L) {
  return hamiltonian(Spacetime{M, a}, Ray{E, L}, y6);
}

void oracle_rhs(double M, double a, const double* y6, double E, double L, double* dy6) {
  rhs(Spacetime{M, a}, Ray{E, L}, y6, dy6);
}

void oracle_ck_step(double M, double a, const double* y6, double E, double L, double h,
                    double* y5_out, double* delta_out) {
  rk_step(kCK, Spacetime{M, a}, Ray{E, L}, y6, h, y5_out, delta_out);
}

void oracle_rk_step(int32_t integrator, double M, double a, const double* y6, double E, double L,
                    double h, double* y5_out, double* delta_out) {
  rk_step(tableau(integrator), Spacetime{M, a}, Ray{E, L}, y6, h, y5_out, delta_out);
}

// Cash-Karp tableau: c[6], a[36] (row-major, lower triangular), b5[6], b4[6].
void oracle_ck_tableau(double* c, double* a, double* b5, double* b4) {
  for (int i = 0; i < 6; ++i) {
    c[i] = kCK.c[i];
    b5[i] = kCK.b5[i];
    b4[i] = kCK.b4[i];
    for (int j = 0; j < 6; ++j) a[6 * i + j] = kCK.a[i][j];
  }
}

// Tableau of an integrator: c[7], a[49] (row-major), b5[7], b4[7]; returns the
// number of stages (unused entries are zero).
int32_t oracle_tableau(int32_t integrator, double* c, double* a, double* b5, double* b4) {
  const Tableau& T = tableau(integrator);
  for (int i = 0; i < 7; ++i) {
    c[i] = T.c[i];
    b5[i] = T.b5[i];
    b4[i] = T.b4[i];
    for (int j = 0; j < 7; ++j) a[7 * i + j] = T.a[i][j];
  }
  return T.stages;
}

void oracle_disk_observables(double M, double a, double r, double E, double L, double* g,
                             double* I) {
  disk_observables(Spacetime{M, a}, Ray{E, L}, r, kKeplerian, 0.0, g, I);
}

void oracle_disk_observables_l0(double M, double a, double r, double E, double L, double l0,
                                double* g, double* I) {
  disk_observables(Spacetime{M, a}, Ray{E, L}, r, kConstantL, l0, g, I);
}

// Radius of the innermost stable circular prograde orbit (Bardeen, Press &
// Teukolsky 1972), used for the inner disk edge r_in = r_isco(a).
double oracle_isco(double M, double a) {
  const double chi = a / M;
  const double z1 = 1.0 + std::cbrt(1.0 - chi * chi) * (std::cbrt(1.0 + chi) + std::cbrt(1.0 - chi));
  const double z2 = std::sqrt(3.0 * chi * chi + z1 * z1);
  return M * (3.0 + z2 - std::sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2)));
}

}  // extern "C"
