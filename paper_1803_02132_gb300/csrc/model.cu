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

}  // extern "C"
