// Pole rules for the Fermi-projector expansion (Sec. 3.1, eqs. FOP and dFOP), host FP64.
//
// Conformal rule: the strip 0 < Im u < K' (period 4K) is mapped by s = sn(u; k) onto the
// plane minus the slits [-1, 1] and [1/k, +inf] U [-inf, -1/k]; the Moebius map
// M(s) = (alpha s + beta)/(s + 1/k) sends -1 -> a, 1 -> b, -1/k -> inf and (given k from
// ((1+k)/(1-k))^2 = (c-a)/(c-b), matching cross ratios) 1/k -> c.  The contour is the image
// of Im u = K'/2 and the trapezoid rule with P nodes gives z_j = M(sn(u_j)) and
// w_j = -h M'(s_j) cn(u_j) dn(u_j) / (2 pi i) for the expansion sum_j w_j (H - z_j)^-1,
// with the orientation fixed so that the filter is +1 on [a, b].
//
// Jacobi functions of real argument by the arithmetic-geometric mean and descending Landen
// recursion (Abramowitz & Stegun 16.4); complex argument t + i y from the addition theorem
// and Jacobi's imaginary transformation; K(k) = pi / (2 AGM(1, k')).
#include <cmath>
#include <complex>
#include <vector>

#include "omm.h"

namespace {

using cd = std::complex<double>;
const double kPi = 3.14159265358979323846264338327950288;

double agm(double a, double b) {
  for (int i = 0; i < 64; ++i) {
    const double an = 0.5 * (a + b), bn = std::sqrt(a * b);
    a = an;
    b = bn;
    if (std::fabs(a - b) <= 1e-17 * a) break;
  }
  return 0.5 * (a + b);
}

// K from the complementary parameter mp = 1 - m (accurate for m close to 1)
double ellip_k_from_mp(double mp) { return kPi / (2.0 * agm(1.0, std::sqrt(mp))); }

// sn, cn, dn of real u with parameter m = k^2 (0 <= m < 1), complementary mp = 1 - m
void jacobi_real(double u, double m, double mp, double& sn, double& cn, double& dn) {
  double a[40], c[40];
  a[0] = 1.0;
  double b = std::sqrt(mp);
  c[0] = std::sqrt(m);
  int nn = 0;
  for (int i = 1; i < 40; ++i) {
    a[i] = 0.5 * (a[i - 1] + b);
    c[i] = 0.5 * (a[i - 1] - b);
    b = std::sqrt(a[i - 1] * b);
    nn = i;
    if (std::fabs(c[i]) <= 1e-17 * a[i]) break;
  }
  double phi = std::ldexp(1.0, nn) * a[nn] * u;
  for (int i = nn; i >= 1; --i) phi = 0.5 * (phi + std::asin(c[i] / a[i] * std::sin(phi)));
  sn = std::sin(phi);
  cn = std::cos(phi);
  // dn^2 = 1 - m sn^2 = mp + m cn^2: a sum of two non-negative terms (no cancellation,
  // and no 0/0 at u = K where the Landen quotient cos(phi0)/cos(phi1 - phi0) degenerates)
  dn = std::sqrt(mp + m * cn * cn);
}

void jacobi_complex(double t, double y, double m, double mp, cd& sn, cd& cn, cd& dn) {
  double s1, c1, d1, s2, c2, d2;
  jacobi_real(t, m, mp, s1, c1, d1);
  jacobi_real(y, mp, m, s2, c2, d2);
  const cd S(0.0, s2 / c2);
  const double C = 1.0 / c2, D = d2 / c2;
  const cd den = 1.0 - m * s1 * s1 * S * S;
  sn = (s1 * C * D + S * c1 * d1) / den;
  cn = (c1 * C - s1 * S * d1 * D) / den;
  dn = (d1 * D - m * s1 * S * c1 * C) / den;
}

}  // namespace

extern "C" omm_status omm_poles_circle(double center, double radius, int P, double* z, double* w) {
  if (!z || !w || P < 1 || !(radius > 0.0)) return OMM_EINVAL;
  for (int j = 0; j < P; ++j) {
    const double th = kPi * (2.0 * j + 1.0) / P;
    const cd e(std::cos(th), std::sin(th));
    const cd zz = center + radius * e;
    const cd ww = -radius * e / (double)P;
    z[2 * j] = zz.real();
    z[2 * j + 1] = zz.imag();
    w[2 * j] = ww.real();
    w[2 * j + 1] = ww.imag();
  }
  return OMM_OK;
}

extern "C" omm_status omm_poles_fermi(double a, double b, double c, int P, double* z, double* w) {
  if (!z || !w || P < 2 || (P % 2) != 0 || !(a < b) || !(b < c)) return OMM_EINVAL;
  const double chi = (c - a) / (c - b);
  const double rchi = std::sqrt(chi);
  const double k = (rchi - 1.0) / (rchi + 1.0);
  const double mp = 4.0 * rchi / ((rchi + 1.0) * (rchi + 1.0));   // k'^2
  const double m = k * k;
  const double K = ellip_k_from_mp(mp);
  const double Kp = ellip_k_from_mp(m);
  const double kappa = 1.0 / k;
  const double alpha = 0.5 * (b * (kappa + 1.0) - a * (kappa - 1.0));
  const double beta = 0.5 * (b * (kappa + 1.0) + a * (kappa - 1.0));
  const double h = 4.0 * K / P;
  std::vector<cd> zz(P), ww(P);
  for (int j = 0; j < P; ++j) {
    const double t = -2.0 * K + (j + 0.5) * h;
    cd sn, cn, dn;
    jacobi_complex(t, 0.5 * Kp, m, mp, sn, cn, dn);
    const cd den = sn + kappa;
    zz[j] = (alpha * sn + beta) / den;
    const cd dzdu = (alpha * kappa - beta) / (den * den) * cn * dn;
    ww[j] = -h * dzdu / cd(0.0, 2.0 * kPi);
  }
  // orientation: the filter must be +1 at the centre of [a, b]
  const double mid = 0.5 * (a + b);
  cd r(0.0, 0.0);
  for (int j = 0; j < P; ++j) r += ww[j] / (mid - zz[j]);
  const double sgn = r.real() < 0.0 ? -1.0 : 1.0;
  for (int j = 0; j < P; ++j) {
    z[2 * j] = zz[j].real();
    z[2 * j + 1] = zz[j].imag();
    w[2 * j] = sgn * ww[j].real();
    w[2 * j + 1] = sgn * ww[j].imag();
  }
  return OMM_OK;
}
