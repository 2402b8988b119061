// Covariance statistics of a batch of measurements (Sec. 5.5, Eq. Covariance; App. E):
// host FP64 code on the small output vectors of many realisations (mocks), fixed summation
// order.  The C ABI is declared in include/bisp.h.
#include <cmath>
#include <string>
#include <vector>

#include "../../include/bisp.h"
#include "internal.h"

namespace {

bisp_status bad(const char* msg) {
  bisp::set_last_error(msg);
  return BISP_EINVAL;
}

}  // namespace

extern "C" {

bisp_status bisp_covariance(const double* X, int n_mock, int n_bin, double* mean, double* cov, double* corr) {
  if (!X || n_mock < 2 || n_bin < 1) return bad("bisp_covariance: need X, n_mock >= 2 and n_bin >= 1");
  std::vector<double> m(n_bin, 0.0);
  for (int n = 0; n < n_mock; ++n)
    for (int i = 0; i < n_bin; ++i) m[i] += X[(size_t)n * n_bin + i];
  for (int i = 0; i < n_bin; ++i) m[i] /= n_mock;
  std::vector<double> c((size_t)n_bin * n_bin, 0.0), d(n_bin);
  for (int n = 0; n < n_mock; ++n) {
    for (int i = 0; i < n_bin; ++i) d[i] = X[(size_t)n * n_bin + i] - m[i];
    for (int i = 0; i < n_bin; ++i)
      for (int j = i; j < n_bin; ++j) c[(size_t)i * n_bin + j] += d[i] * d[j];
  }
  for (int i = 0; i < n_bin; ++i)
    for (int j = i; j < n_bin; ++j) {
      const double v = c[(size_t)i * n_bin + j] / (n_mock - 1);
      c[(size_t)i * n_bin + j] = v;
      c[(size_t)j * n_bin + i] = v;
    }
  if (mean)
    for (int i = 0; i < n_bin; ++i) mean[i] = m[i];
  if (cov)
    for (size_t k = 0; k < c.size(); ++k) cov[k] = c[k];
  if (corr)
    for (int i = 0; i < n_bin; ++i)
      for (int j = 0; j < n_bin; ++j) {
        const double den = std::sqrt(c[(size_t)i * n_bin + i] * c[(size_t)j * n_bin + j]);
        corr[(size_t)i * n_bin + j] = den > 0.0 ? c[(size_t)i * n_bin + j] / den : NAN;
      }
  bisp::set_last_error("");
  return BISP_OK;
}

bisp_status bisp_covariance_factors(int n_mock, int n_bin, int n_par, double* hartlap, double* percival_m) {
  if (n_mock < 2 || n_bin < 1 || n_par < 0) return bad("bisp_covariance_factors: need n_mock >= 2, n_bin >= 1, n_par >= 0");
  if (hartlap) *hartlap = (double)(n_mock - n_bin - 2) / (double)(n_mock - 1);
  if (percival_m) {
    const double q = (double)(n_mock - n_bin - 1) * (double)(n_mock - n_bin - 4);
    if (!(q > 0.0)) return bad("bisp_covariance_factors: the Percival factor needs n_mock > n_bin + 4");
    // A and B without the square roots App. E prints (with them M would not tend to 1 for
    // infinitely many realisations)
    const double A = 2.0 / q, B = (double)(n_mock - n_bin - 2) / q;
    *percival_m = (1.0 + B * (n_bin - n_par)) / (1.0 + A + B * (n_par + 1));
  }
  bisp::set_last_error("");
  return BISP_OK;
}

bisp_status bisp_chi2(const double* cov, int n_bin, int n_mock, const double* x_obs, const double* x_theory,
                      double* chi2) {
  if (!cov || !x_obs || !x_theory || !chi2 || n_bin < 1 || n_mock < 2)
    return bad("bisp_chi2: NULL argument or n_bin < 1 or n_mock < 2");
  // Cholesky factor C = R R^T (lower R), then chi2 = |R^{-1} d|^2 times the Hartlap factor
  std::vector<double> R((size_t)n_bin * n_bin, 0.0);
  for (int j = 0; j < n_bin; ++j) {
    double s = cov[(size_t)j * n_bin + j];
    for (int k = 0; k < j; ++k) s -= R[(size_t)j * n_bin + k] * R[(size_t)j * n_bin + k];
    if (!(s > 0.0)) return bad("bisp_chi2: the covariance is not positive definite");
    const double rjj = std::sqrt(s);
    R[(size_t)j * n_bin + j] = rjj;
    for (int i = j + 1; i < n_bin; ++i) {
      double t = cov[(size_t)i * n_bin + j];
      for (int k = 0; k < j; ++k) t -= R[(size_t)i * n_bin + k] * R[(size_t)j * n_bin + k];
      R[(size_t)i * n_bin + j] = t / rjj;
    }
  }
  std::vector<double> y(n_bin);
  double acc = 0.0;
  for (int i = 0; i < n_bin; ++i) {
    double t = x_obs[i] - x_theory[i];
    for (int k = 0; k < i; ++k) t -= R[(size_t)i * n_bin + k] * y[k];
    y[i] = t / R[(size_t)i * n_bin + i];
    acc += y[i] * y[i];
  }
  *chi2 = acc * (double)(n_mock - n_bin - 2) / (double)(n_mock - 1);
  bisp::set_last_error("");
  return BISP_OK;
}

}  // extern "C"
