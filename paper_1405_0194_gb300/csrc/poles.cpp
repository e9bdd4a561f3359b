// Pole expansion of the Fermi-Dirac function (Sec. II.A, Eq. polerho) and of
// the band-energy and grand-potential functions that share its shifts (Eq.
// gammaF). The paper refers the construction to Lin, Lu, Ying and E (2009);
// this is that contour-quadrature construction written from the mathematics:
//
//  * f(x) = 2/(1+exp(beta x)) has its singularities at x = i pi (2j+1)/beta;
//    xi = x^2 + m, m = (pi/beta)^2, sends them to (-inf, 0] and the spectrum
//    [-dE, dE] to [m, M], M = dE^2 + m.
//  * xi(t) = sqrt(mM) (1/k + sn t)/(1/k - sn t), k = (sqrt(M/m)-1)/(sqrt(M/m)+1),
//    maps the line Im t = K'/2 onto a closed curve around [m, M] avoiding
//    (-inf, 0] (Hale, Higham and Trefethen 2008).
//  * The two square roots x = +-sqrt(xi - m) trace a contour around the
//    spectrum that passes between the Matsubara points +-i pi/beta; the
//    N-point trapezoidal rule in t on the Cauchy integral of F gives 2N poles
//    in conjugate pairs, folded into P = N poles of the form Im sum w/(x - z).
//
// Jacobi elliptic functions and complete elliptic integrals are computed here
// by the arithmetic-geometric mean with the descending Landen recursion
// (Abramowitz and Stegun 16.4 and 17.6); complex arguments use the addition
// theorem with Jacobi's imaginary transformation (A&S 16.21.2-16.21.4).
#include <cmath>
#include <complex>
#include <vector>

#include "../../include/pexsi_gb300.h"

namespace pexsi {
namespace {

using cd = std::complex<double>;
constexpr double kPi = 3.14159265358979323846;

// Arithmetic-geometric mean of (1, b).
double agm1(double b) {
  double a = 1.0;
  for (int it = 0; it < 64 && std::fabs(a - b) > 1e-16 * a; ++it) {
    double an = 0.5 * (a + b);
    b = std::sqrt(a * b);
    a = an;
  }
  return 0.5 * (a + b);
}

// sn, cn, dn of a real argument u for parameter m, its complement mc = 1 - m
// supplied separately so that m near 1 keeps full relative accuracy (A&S
// 16.4: AGM scale with a_0 = 1, b_0 = sqrt(mc), c_0 = sqrt(m); phi_N =
// 2^N a_N u; phi_{n-1} = (phi_n + asin(c_n/a_n sin phi_n))/2).
void sncndn(double u, double m, double mc, double& sn, double& cn, double& dn) {
  double a[40], c[40];
  a[0] = 1.0;
  c[0] = std::sqrt(m);
  double b = std::sqrt(mc);
  int N = 0;
  while (N < 38 && std::fabs(c[N]) > 1e-16 * a[N]) {
    double an = 0.5 * (a[N] + b);
    double cn_ = 0.5 * (a[N] - b);
    b = std::sqrt(a[N] * b);
    ++N;
    a[N] = an;
    c[N] = cn_;
  }
  double phi = std::ldexp(a[N] * u, N);
  for (int k = N; k >= 1; --k) phi = 0.5 * (phi + std::asin(c[k] / a[k] * std::sin(phi)));
  sn = std::sin(phi);
  cn = std::cos(phi);
  dn = std::sqrt(mc + m * cn * cn);  // dn^2 = 1 - m sn^2, positive for real u
}

// Complex argument u = x + i y (A&S 16.21.2-4).
void sncndn(cd u, double m, double mc, cd& sn, cd& cn, cd& dn) {
  double s, c, d, s1, c1, d1;
  sncndn(u.real(), m, mc, s, c, d);
  sncndn(u.imag(), mc, m, s1, c1, d1);
  double den = c1 * c1 + m * s * s * s1 * s1;
  sn = cd(s * d1, c * d * s1 * c1) / den;
  cn = cd(c * c1, -s * d * s1 * d1) / den;
  dn = cd(d * c1 * d1, -m * s * c * s1) / den;
}

// log(1 + w) for |w| <= 1 without loss for small w (w/(u-1) correction).
cd log1p_c(cd w) {
  cd u = 1.0 + w;
  if (u == cd(1.0, 0.0)) return w;
  return std::log(u) * w / (u - 1.0);
}

cd fermi(cd x, double beta) {
  cd bx = beta * x;
  if (bx.real() >= 0) {
    cd e = std::exp(-bx);
    return 2.0 * e / (1.0 + e);
  }
  return 2.0 / (1.0 + std::exp(bx));
}

cd grand(cd x, double beta) {
  cd bx = beta * x;
  cd l = bx.real() >= 0 ? log1p_c(std::exp(-bx)) : -bx + log1p_c(std::exp(bx));
  return -(2.0 / beta) * l;
}

// d/dmu of f(eps - mu) at x = eps - mu: (beta/2) f (2 - f); its weights give
// Gamma^d, whose trace with S is N'(mu) (Sec. II.C).
cd dfermi(cd x, double beta) {
  cd f = fermi(x, beta);
  return 0.5 * beta * f * (2.0 - f);
}

}  // namespace

int pole_table(double beta, double delta_e, int P, double mu, std::vector<cd>& z, std::vector<cd>& w_rho,
               std::vector<cd>& w_E, std::vector<cd>& w_F, std::vector<cd>* w_d) {
  if (!(beta > 0) || !(delta_e > 0) || P < 2 || (P & 1)) return PEXSI_ERR_INVALID_ARG;
  const int N = P;
  const double m = (kPi / beta) * (kPi / beta);
  const double M = delta_e * delta_e + m;
  const double q = std::sqrt(M / m);
  const double k = (q - 1.0) / (q + 1.0);
  const double ksq = k * k;
  const double kc2 = 4.0 * q / ((q + 1.0) * (q + 1.0));  // 1 - k^2
  const double K = kPi / (2.0 * agm1(std::sqrt(kc2)));   // K(k^2)
  const double Kp = kPi / (2.0 * agm1(k));               // K(1 - k^2)
  const double h = 4.0 * K / N;
  const double root = std::sqrt(m * M);
  std::vector<cd> xs(N), cs(N);
  for (int j = 0; j < N; ++j) {
    cd t(-K + (j + 0.5) * h, 0.5 * Kp);
    cd sn, cn, dn;
    sncndn(t, ksq, kc2, sn, cn, dn);
    cd xi = root * (1.0 / k + sn) / (1.0 / k - sn);
    cd dxi = root * (2.0 / k) * cn * dn / ((1.0 / k - sn) * (1.0 / k - sn));
    cd x = std::sqrt(xi - m);
    // increasing t runs clockwise around [m, M]; the Cauchy integral is
    // taken counter-clockwise, hence the minus sign
    xs[j] = x;
    cs[j] = -h * dxi / (cd(0.0, 4.0 * kPi) * x);
  }
  z.clear(); w_rho.clear(); w_E.clear(); w_F.clear();
  if (w_d) w_d->clear();
  // poles at +x_j (residue -c_j F(x_j)) then at -x_j (residue +c_j F(-x_j));
  // keep the upper half-plane member of each conjugate pair, weight 2 i r
  for (int side = 0; side < 2; ++side) {
    for (int j = 0; j < N; ++j) {
      cd y = side == 0 ? xs[j] : -xs[j];
      if (!(y.imag() > 0)) continue;
      double sgn = side == 0 ? -1.0 : 1.0;
      cd two_i(0.0, 2.0);
      cd f = fermi(y, beta);
      z.push_back(y + mu);
      w_rho.push_back(two_i * sgn * cs[j] * f);
      w_E.push_back(two_i * sgn * cs[j] * (y + mu) * f);
      w_F.push_back(two_i * sgn * cs[j] * grand(y, beta));
      if (w_d) w_d->push_back(two_i * sgn * cs[j] * dfermi(y, beta));
    }
  }
  if (int(z.size()) != P) return PEXSI_ERR_INTERNAL;
  return PEXSI_OK;
}

}  // namespace pexsi
