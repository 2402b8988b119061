// Window-convolved model (Sec. 6.2): Wigner 9j symbols, the masked three-point multipoles
// (Eq. zetaMask) with the integral constraint (Eq. IC), and the Hankel transforms between
// three-point and bispectrum multipoles (Eq. HankelTransform, Eq. masked_bispectrum).  Host
// FP64 code on small (r1, r2) and (k1, k2) grids.  The C ABI is declared in include/bisp.h.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/bisp.h"
#include "internal.h"

namespace {

constexpr int LMAX_MODEL = 8;

bisp_status bad(bisp_status st, const std::string& msg) {
  bisp::set_last_error(msg);
  return st;
}

double lfac(int n) { return std::lgamma((double)n + 1.0); }

bool triangle(int a, int b, int c) { return c >= std::abs(a - b) && c <= a + b; }

// Racah's Delta(a b c) = sqrt((a+b-c)! (a-b+c)! (-a+b+c)! / (a+b+c+1)!), as a logarithm
double log_delta(int a, int b, int c) {
  return 0.5 * (lfac(a + b - c) + lfac(a - b + c) + lfac(-a + b + c) - lfac(a + b + c + 1));
}

// 6j symbol {a b c; d e f} by Racah's single-sum formula
double wigner6j(int a, int b, int c, int d, int e, int f) {
  if (!triangle(a, b, c) || !triangle(a, e, f) || !triangle(d, b, f) || !triangle(d, e, c)) return 0.0;
  const double ld = log_delta(a, b, c) + log_delta(a, e, f) + log_delta(d, b, f) + log_delta(d, e, c);
  const int t0 = std::max(std::max(a + b + c, a + e + f), std::max(d + b + f, d + e + c));
  const int t1 = std::min(std::min(a + b + d + e, a + c + d + f), b + c + e + f);
  double s = 0.0;
  for (int t = t0; t <= t1; ++t) {
    const double lg = lfac(t + 1) - lfac(t - a - b - c) - lfac(t - a - e - f) - lfac(t - d - b - f) -
                      lfac(t - d - e - c) - lfac(a + b + d + e - t) - lfac(a + c + d + f - t) - lfac(b + c + e + f - t);
    s += ((t & 1) ? -1.0 : 1.0) * std::exp(lg + ld);
  }
  return s;
}

// 9j symbol as the sum over x of three 6j symbols:
// {j1 j2 j3; j4 j5 j6; j7 j8 j9} = sum_x (-1)^{2x} (2x+1) {j1 j4 j7; j8 j9 x} {j2 j5 j8; j4 x j6} {j3 j6 j9; x j1 j2}
double wigner9j(const int* j) {
  const int xlo = std::max(std::max(std::abs(j[0] - j[8]), std::abs(j[3] - j[7])), std::abs(j[1] - j[5]));
  const int xhi = std::min(std::min(j[0] + j[8], j[3] + j[7]), j[1] + j[5]);
  double s = 0.0;
  for (int x = xlo; x <= xhi; ++x)
    s += (2.0 * x + 1.0) * wigner6j(j[0], j[3], j[6], j[7], j[8], x) * wigner6j(j[1], j[4], j[7], j[3], x, j[5]) *
         wigner6j(j[2], j[5], j[8], x, j[0], j[1]);
  return s;
}

// H_{abc} = 3j(a b c; 0 0 0) in closed form: zero unless a+b+c = 2g is even and the triangle
// rule holds; (-1)^g sqrt((2g-2a)! (2g-2b)! (2g-2c)! / (2g+1)!) g! / ((g-a)! (g-b)! (g-c)!)
double h3j(int a, int b, int c) {
  if (((a + b + c) & 1) || !triangle(a, b, c)) return 0.0;
  const int g = (a + b + c) / 2;
  const double lg = 0.5 * (lfac(2 * g - 2 * a) + lfac(2 * g - 2 * b) + lfac(2 * g - 2 * c) - lfac(2 * g + 1)) +
                    lfac(g) - lfac(g - a) - lfac(g - b) - lfac(g - c);
  return ((g & 1) ? -1.0 : 1.0) * std::exp(lg);
}

double nlll(int a, int b, int c) { return (double)((2 * a + 1) * (2 * b + 1) * (2 * c + 1)); }

// spherical Bessel function j_l(x), x >= 0: the power series below x = max(l, 1), the upward
// recurrence from j_0 = sin x / x and j_1 = sin x / x^2 - cos x / x above it
double sph_jl(int l, double x) {
  if (x == 0.0) return l == 0 ? 1.0 : 0.0;
  if (x < std::max(l, 1)) {
    // j_l(x) = x^l sum_k (-x^2/2)^k / (k! (2l + 2k + 1)!!)
    double df = 1.0;
    for (int i = 3; i <= 2 * l + 1; i += 2) df *= i;
    double term = std::pow(x, l) / df, s = term;
    const double h = -0.5 * x * x;
    for (int k = 1; k < 200; ++k) {
      term *= h / (k * (2.0 * l + 2.0 * k + 1.0));
      s += term;
      if (std::fabs(term) < 1e-17 * std::fabs(s)) break;
    }
    return s;
  }
  const double sx = std::sin(x), cx = std::cos(x);
  double jm = sx / x;
  if (l == 0) return jm;
  double j = sx / (x * x) - cx / x;
  for (int n = 1; n < l; ++n) {
    const double jn = (2.0 * n + 1.0) / x * j - jm;
    jm = j;
    j = jn;
  }
  return j;
}

// 3j symbol (j1 j2 j3; m1 m2 m3) by Racah's formula
double wigner3j_gen(int j1, int j2, int j3, int m1, int m2, int m3) {
  if (m1 + m2 + m3 != 0 || std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3 || !triangle(j1, j2, j3))
    return 0.0;
  const double pre = log_delta(j1, j2, j3) + 0.5 * (lfac(j1 + m1) + lfac(j1 - m1) + lfac(j2 + m2) + lfac(j2 - m2) +
                                                   lfac(j3 + m3) + lfac(j3 - m3));
  const int t0 = std::max(std::max(0, j2 - j3 - m1), j1 - j3 + m2);
  const int t1 = std::min(std::min(j1 + j2 - j3, j1 - m1), j2 + m2);
  double s = 0.0;
  for (int t = t0; t <= t1; ++t) {
    const double lg = -(lfac(t) + lfac(j3 - j2 + t + m1) + lfac(j3 - j1 + t - m2) + lfac(j1 + j2 - j3 - t) +
                        lfac(j1 - t - m1) + lfac(j2 - t + m2));
    s += ((t & 1) ? -1.0 : 1.0) * std::exp(lg + pre);
  }
  return (((j1 - j2 - m3) & 1) ? -1.0 : 1.0) * s;
}

// y_l^m(u) = sqrt(4 pi / (2l+1)) Y_l^m(u) of a unit vector u, any m, Condon-Shortley phase
void ylm_unit(int l, int m, double x, double y, double z, double* re, double* im) {
  const int am = std::abs(m);
  double pmm = 1.0;  // P_m^m without the (1 - z^2)^{m/2} factor: (-1)^m (2m-1)!!
  for (int k = 1; k <= am; ++k) pmm *= -(2.0 * k - 1.0);
  double p = pmm;
  if (l > am) {
    double p2 = pmm, p1 = (2.0 * am + 1.0) * z * pmm;
    p = p1;
    for (int ll = am + 2; ll <= l; ++ll) {
      p = ((2.0 * ll - 1.0) * z * p1 - (ll + am - 1.0) * p2) / (ll - am);
      p2 = p1;
      p1 = p;
    }
  }
  double er = 1.0, ei = 0.0;  // (x + i y)^m
  for (int k = 0; k < am; ++k) {
    const double t = er * x - ei * y;
    ei = er * y + ei * x;
    er = t;
  }
  const double a = std::exp(0.5 * (lfac(l - am) - lfac(l + am))) * p;
  double r = a * er, i = a * ei;
  if (m < 0) {  // y_l^{-m} = (-1)^m conj(y_l^m)
    const double sg = (am & 1) ? -1.0 : 1.0;
    r *= sg;
    i *= -sg;
  }
  *re = r;
  *im = i;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n from the Chebyshev guesses)
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double pn = n == 1 ? z : p1, pm = n == 1 ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
      const double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

bool valid_ell(const int* e) {
  for (int i = 0; i < 3; ++i)
    if (e[i] < 0 || e[i] > LMAX_MODEL) return false;
  return triangle(e[0], e[1], e[2]);
}

}  // namespace

extern "C" {

bisp_status bisp_wigner9j(const int* j, double* out) {
  if (!j || !out) return bad(BISP_EINVAL, "bisp_wigner9j: NULL argument");
  for (int i = 0; i < 9; ++i)
    if (j[i] < 0 || j[i] > 4 * LMAX_MODEL) return bad(BISP_EINVAL, "bisp_wigner9j: j out of range");
  *out = wigner9j(j);
  return BISP_OK;
}

bisp_status bisp_masked_zeta(const int* ells_t, int n_t, const double* zeta_t, const int* ells_q, int n_q,
                             const double* Q, const int* ells_o, int n_o, const double* r, const double* w, int nr,
                             int ic, double* out, double* zeta_bar) {
  if (!ells_t || !zeta_t || !ells_q || !Q || !ells_o || !out || !r || !w || n_t < 1 || n_q < 1 || n_o < 1 || nr < 1)
    return bad(BISP_EINVAL, "bisp_masked_zeta: NULL argument or empty set");
  for (int i = 0; i < n_t; ++i)
    if (!valid_ell(ells_t + 3 * i)) return bad(BISP_EINVAL, "bisp_masked_zeta: invalid theory multipole");
  for (int i = 0; i < n_q; ++i)
    if (!valid_ell(ells_q + 3 * i)) return bad(BISP_EINVAL, "bisp_masked_zeta: invalid window multipole");
  for (int i = 0; i < n_o; ++i)
    if (!valid_ell(ells_o + 3 * i)) return bad(BISP_EINVAL, "bisp_masked_zeta: invalid output multipole");
  const size_t np2 = (size_t)nr * nr;
  auto find = [](const int* ells, int n, const int* e) {
    for (int i = 0; i < n; ++i)
      if (ells[3 * i] == e[0] && ells[3 * i + 1] == e[1] && ells[3 * i + 2] == e[2]) return i;
    return -1;
  };
  // integral constraint (Eq. IC): multipoles present in both sets over the window monopole
  double zb = 0.0;
  if (ic) {
    const int z0[3] = {0, 0, 0};
    const int q0 = find(ells_q, n_q, z0);
    if (q0 < 0) return bad(BISP_EINVAL, "bisp_masked_zeta: the integral constraint needs the window monopole Q_000");
    std::vector<double> wr(nr);
    for (int i = 0; i < nr; ++i) wr[i] = w[i] * r[i] * r[i];
    auto integral = [&](const double* a, const double* b) {
      double s = 0.0;
      for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nr; ++j) s += wr[i] * wr[j] * a[(size_t)i * nr + j] * (b ? b[(size_t)i * nr + j] : 1.0);
      return s;
    };
    double num = 0.0;
    for (int t = 0; t < n_t; ++t) {
      const int* e = ells_t + 3 * t;
      const int q = find(ells_q, n_q, e);
      if (q < 0) continue;
      const double h = h3j(e[0], e[1], e[2]);
      if (h == 0.0) continue;
      num += integral(Q + q * np2, zeta_t + t * np2) / (h * h * nlll(e[0], e[1], e[2]));
    }
    const double den = integral(Q + q0 * np2, nullptr);
    if (!(den != 0.0)) return bad(BISP_EINVAL, "bisp_masked_zeta: the window monopole integrates to zero");
    zb = num / den;
  }
  // Eq. zetaMask: N_l sum_{l' l''} {l''; l'; l} H_l H_{l1 l1' l1''} H_{l2 l2' l2''} H_{L L' L''}
  //               / (H_{l'} H_{l''}) Q_{l''} zeta_{l'}  -  Q_l zeta_bar
  for (int o = 0; o < n_o; ++o) {
    const int* e = ells_o + 3 * o;
    double* dst = out + o * np2;
    for (size_t i = 0; i < np2; ++i) dst[i] = 0.0;
    const double hl = h3j(e[0], e[1], e[2]);
    for (int t = 0; t < n_t; ++t) {
      const int* a = ells_t + 3 * t;
      for (int q = 0; q < n_q; ++q) {
        const int* b = ells_q + 3 * q;
        const double den = h3j(a[0], a[1], a[2]) * h3j(b[0], b[1], b[2]);
        const double num = hl * h3j(e[0], a[0], b[0]) * h3j(e[1], a[1], b[1]) * h3j(e[2], a[2], b[2]);
        if (den == 0.0 || num == 0.0) continue;
        const int j9[9] = {b[0], b[1], b[2], a[0], a[1], a[2], e[0], e[1], e[2]};
        const double c = nlll(e[0], e[1], e[2]) * wigner9j(j9) * num / den;
        if (c == 0.0) continue;
        const double* zq = Q + q * np2;
        const double* zt = zeta_t + t * np2;
        for (size_t i = 0; i < np2; ++i) dst[i] += c * zq[i] * zt[i];
      }
    }
    const int qo = find(ells_q, n_q, e);
    if (ic && qo >= 0)
      for (size_t i = 0; i < np2; ++i) dst[i] -= Q[qo * np2 + i] * zb;
  }
  if (zeta_bar) *zeta_bar = zb;
  return BISP_OK;
}

bisp_status bisp_zeta_to_bk(int l1, int l2, const double* r, const double* w, int nr, const double* zeta,
                            const double* k1, int nk1, const double* k2, int nk2, double* B) {
  if (!r || !w || !zeta || !k1 || !k2 || !B || nr < 1 || nk1 < 1 || nk2 < 1 || l1 < 0 || l2 < 0 ||
      l1 > LMAX_MODEL || l2 > LMAX_MODEL)
    return bad(BISP_EINVAL, "bisp_zeta_to_bk: NULL argument, empty grid or l out of range");
  if ((l1 + l2) & 1) return bad(BISP_EUNSUPPORTED, "bisp_zeta_to_bk: l1 + l2 odd (an imaginary bispectrum)");
  const double ph = (((l1 + l2) / 2) & 1) ? -1.0 : 1.0, fp = 16.0 * M_PI * M_PI;
  // T[a][j] = sum_i w_i r_i^2 j_l1(k1_a r_i) zeta_ij, then B[a][b] = sum_j w_j r_j^2 j_l2(k2_b r_j) T[a][j]
  std::vector<double> T((size_t)nk1 * nr, 0.0);
  for (int a = 0; a < nk1; ++a)
    for (int i = 0; i < nr; ++i) {
      const double f = w[i] * r[i] * r[i] * sph_jl(l1, k1[a] * r[i]);
      for (int j = 0; j < nr; ++j) T[(size_t)a * nr + j] += f * zeta[(size_t)i * nr + j];
    }
  for (int b = 0; b < nk2; ++b) {
    std::vector<double> g(nr);
    for (int j = 0; j < nr; ++j) g[j] = w[j] * r[j] * r[j] * sph_jl(l2, k2[b] * r[j]);
    for (int a = 0; a < nk1; ++a) {
      double s = 0.0;
      for (int j = 0; j < nr; ++j) s += g[j] * T[(size_t)a * nr + j];
      B[(size_t)a * nk2 + b] = ph * fp * s;
    }
  }
  return BISP_OK;
}

bisp_status bisp_bk_to_zeta(int l1, int l2, const double* k, const double* wk, int nk, const double* B,
                            const double* r1, int nr1, const double* r2, int nr2, double* zeta) {
  if (!k || !wk || !B || !r1 || !r2 || !zeta || nk < 1 || nr1 < 1 || nr2 < 1 || l1 < 0 || l2 < 0 ||
      l1 > LMAX_MODEL || l2 > LMAX_MODEL)
    return bad(BISP_EINVAL, "bisp_bk_to_zeta: NULL argument, empty grid or l out of range");
  if ((l1 + l2) & 1) return bad(BISP_EUNSUPPORTED, "bisp_bk_to_zeta: l1 + l2 odd");
  const double ph = (((l1 + l2) / 2) & 1) ? -1.0 : 1.0, c = 1.0 / (2.0 * M_PI * M_PI);
  std::vector<double> T((size_t)nr1 * nk, 0.0);
  for (int a = 0; a < nr1; ++a)
    for (int i = 0; i < nk; ++i) {
      const double f = wk[i] * k[i] * k[i] * c * sph_jl(l1, r1[a] * k[i]);
      for (int j = 0; j < nk; ++j) T[(size_t)a * nk + j] += f * B[(size_t)i * nk + j];
    }
  for (int b = 0; b < nr2; ++b) {
    std::vector<double> g(nk);
    for (int j = 0; j < nk; ++j) g[j] = wk[j] * k[j] * k[j] * c * sph_jl(l2, r2[b] * k[j]);
    for (int a = 0; a < nr1; ++a) {
      double s = 0.0;
      for (int j = 0; j < nk; ++j) s += g[j] * T[(size_t)a * nk + j];
      zeta[(size_t)a * nr2 + b] = ph * s;
    }
  }
  return BISP_OK;
}

bisp_status bisp_tree_multipoles(const double* k_tab, const double* p_tab, int n_tab, double b1, double b2, double f,
                                 const int* ells, int n_mult, const double* k1, int nk1, const double* k2, int nk2,
                                 int n_mu, double* out) {
  if (!k_tab || !p_tab || !ells || !k1 || !k2 || !out || n_tab < 2 || n_mult < 1 || nk1 < 1 || nk2 < 1 || n_mu < 2)
    return bad(BISP_EINVAL, "bisp_tree_multipoles: NULL argument, fewer than 2 table points or empty grids");
  for (int i = 0; i < n_tab; ++i)
    if (!(k_tab[i] > 0.0) || !(p_tab[i] > 0.0) || (i && !(k_tab[i] > k_tab[i - 1])))
      return bad(BISP_EINVAL, "bisp_tree_multipoles: the P(k) table needs ascending k > 0 and P > 0");
  for (int i = 0; i < n_mult; ++i)
    if (!valid_ell(ells + 3 * i)) return bad(BISP_EINVAL, "bisp_tree_multipoles: invalid multipole");
  for (int i = 0; i < nk1; ++i)
    if (!(k1[i] > 0.0)) return bad(BISP_EINVAL, "bisp_tree_multipoles: k1 must be positive");
  for (int i = 0; i < nk2; ++i)
    if (!(k2[i] > 0.0)) return bad(BISP_EINVAL, "bisp_tree_multipoles: k2 must be positive");
  // P(k): log-log interpolation, the end values outside the table
  std::vector<double> lk(n_tab), lp(n_tab);
  for (int i = 0; i < n_tab; ++i) {
    lk[i] = std::log(k_tab[i]);
    lp[i] = std::log(p_tab[i]);
  }
  auto P = [&](double k) {
    const double x = std::log(k);
    if (x <= lk[0]) return p_tab[0];
    if (x >= lk[n_tab - 1]) return p_tab[n_tab - 1];
    const int j = (int)(std::upper_bound(lk.begin(), lk.end(), x) - lk.begin()) - 1;
    const double t = (x - lk[j]) / (lk[j + 1] - lk[j]);
    return std::exp(lp[j] + t * (lp[j + 1] - lp[j]));
  };
  // second-order kernels (App. F) with the line of sight n = z
  auto Z1 = [&](const double* v) {
    const double k = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]), mu = v[2] / k;
    return b1 + f * mu * mu;
  };
  auto Z2 = [&](const double* a, const double* b) {
    const double ka = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    const double kb = std::sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    const double mab = (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) / (ka * kb);
    const double F2 = 5.0 / 7.0 + 0.5 * mab * (ka / kb + kb / ka) + 2.0 / 7.0 * mab * mab;
    const double G2 = 3.0 / 7.0 + 0.5 * mab * (ka / kb + kb / ka) + 4.0 / 7.0 * mab * mab;
    const double s[3] = {a[0] + b[0], a[1] + b[1], a[2] + b[2]};
    const double k = std::sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    const double muk = s[2];  // mu k = (a + b) . n
    const double mu2 = k > 0.0 ? (s[2] / k) * (s[2] / k) : 0.0;
    return b1 * F2 + 0.5 * b2 + f * mu2 * G2 + 0.5 * f * muk * (a[2] / (ka * ka) * Z1(b) + b[2] / (kb * kb) * Z1(a));
  };
  auto term = [&](const double* a, const double* b) {
    const double ka = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    const double kb = std::sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    return 2.0 * Z2(a, b) * Z1(a) * Z1(b) * P(ka) * P(kb);
  };
  std::vector<double> mu, wmu;
  gauss_legendre(n_mu, mu, wmu);
  const int n_phi = 2 * n_mu;
  // Phi_l(k1_hat, k2_hat) = sum_m1 3j(l1 l2 L; m1, -m1, 0) y_l1^{m1*}(k1_hat) y_l2^{-m1*}(k2_hat), y_L^0(z) = 1:
  // the TripoSH weight with n = z (Eq. reduced_ones with Eq. Slll; rotation invariant)
  for (int q = 0; q < n_mult * nk1 * nk2; ++q) out[q] = 0.0;
  for (int i1 = 0; i1 < n_mu; ++i1)
    for (int i2 = 0; i2 < n_mu; ++i2)
      for (int jp = 0; jp < n_phi; ++jp) {
        const double ph = 2.0 * M_PI * (jp + 0.5) / n_phi;
        const double s1 = std::sqrt(1.0 - mu[i1] * mu[i1]), s2 = std::sqrt(1.0 - mu[i2] * mu[i2]);
        const double u1[3] = {s1 * std::cos(ph), s1 * std::sin(ph), mu[i1]}, u2[3] = {s2, 0.0, mu[i2]};
        const double wq = wmu[i1] * wmu[i2] / (4.0 * n_phi);
        std::vector<double> phi(n_mult, 0.0);
        for (int e = 0; e < n_mult; ++e) {
          const int l1 = ells[3 * e], l2 = ells[3 * e + 1], L = ells[3 * e + 2];
          double acc = 0.0;
          for (int m1 = -std::min(l1, l2); m1 <= std::min(l1, l2); ++m1) {
            const double c = wigner3j_gen(l1, l2, L, m1, -m1, 0);
            if (c == 0.0) continue;
            double r1, i1, r2, i2;
            ylm_unit(l1, m1, u1[0], u1[1], u1[2], &r1, &i1);
            ylm_unit(l2, -m1, u2[0], u2[1], u2[2], &r2, &i2);
            acc += c * (r1 * r2 - i1 * i2);  // Re(conj(y1) conj(y2)) = Re(y1 y2)
          }
          phi[e] = acc;
        }
        for (int a = 0; a < nk1; ++a)
          for (int b = 0; b < nk2; ++b) {
            const double v1[3] = {k1[a] * u1[0], k1[a] * u1[1], k1[a] * u1[2]};
            const double v2[3] = {k2[b] * u2[0], k2[b] * u2[1], k2[b] * u2[2]};
            const double v3[3] = {-v1[0] - v2[0], -v1[1] - v2[1], -v1[2] - v2[2]};
            const double B = term(v1, v2) + term(v2, v3) + term(v3, v1);
            for (int e = 0; e < n_mult; ++e) out[((size_t)e * nk1 + a) * nk2 + b] += wq * phi[e] * B;
          }
      }
  for (int e = 0; e < n_mult; ++e) {
    const int l1 = ells[3 * e], l2 = ells[3 * e + 1], L = ells[3 * e + 2];
    const double pre = nlll(l1, l2, L) * h3j(l1, l2, L);
    for (int q = 0; q < nk1 * nk2; ++q) out[(size_t)e * nk1 * nk2 + q] *= pre;
  }
  return BISP_OK;
}

}  // extern "C"
