// Host side of the library: plan (validation, k-shell thresholds, channels, Wigner 3j
// contraction recipes in FP64), orchestration of bisp_assign / bisp_measure, and the
// C ABI declared in include/bisp.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/bisp.h"
#include "common.cuh"
#include "internal.h"

using namespace bisp;

namespace {

thread_local std::string g_err;

// host threads of bisp_measure_batch (plans measured at the same time)
constexpr int kBatchThreads = 8;

struct Fail {
  int status;
  std::string msg;
};
[[noreturn]] void fail(int st, const std::string& m) { throw Fail{st, m}; }

// ---------------------------------------------------------------------------------
// FP64 helpers: Wigner 3j (Racah's formula), y_l^m normalisation, y_l^{m*}
// ---------------------------------------------------------------------------------
double lfact(int n) { return std::lgamma((double)n + 1.0); }

double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3) {
  if (m1 + m2 + m3 != 0) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
  if (j3 < std::abs(j1 - j2) || j3 > j1 + j2) return 0.0;
  // exact integer factorials up to 20! fit in double mantissa only approximately; use
  // long double products of small integers (arguments here are <= 12)
  auto f = [](int n) {
    long double r = 1.0L;
    for (int i = 2; i <= n; ++i) r *= (long double)i;
    return r;
  };
  const long double tri = f(j1 + j2 - j3) * f(j1 - j2 + j3) * f(-j1 + j2 + j3) / f(j1 + j2 + j3 + 1);
  const long double pref = std::sqrt(tri * f(j1 + m1) * f(j1 - m1) * f(j2 + m2) * f(j2 - m2) * f(j3 + m3) * f(j3 - m3));
  const int tmin = std::max({0, j2 - j3 - m1, j1 - j3 + m2});
  const int tmax = std::min({j1 + j2 - j3, j1 - m1, j2 + m2});
  long double s = 0.0L;
  for (int t = tmin; t <= tmax; ++t) {
    const long double den =
        f(t) * f(j3 - j2 + t + m1) * f(j3 - j1 + t - m2) * f(j1 + j2 - j3 - t) * f(j1 - t - m1) * f(j2 - t + m2);
    s += ((t & 1) ? -1.0L : 1.0L) / den;
  }
  const double sign = ((j1 - j2 - m3) & 1) ? -1.0 : 1.0;
  return sign * (double)(pref * s);
}

// y_l^m (m >= 0) of the direction (x, y, z), FP64, Condon-Shortley phase
void ylm_host(int l, int m, double x, double y, double z, double* re, double* im) {
  const double r = std::sqrt(x * x + y * y + z * z);
  if (r == 0.0) {
    *re = l == 0 ? 1.0 : 0.0;
    *im = 0.0;
    return;
  }
  const double mu = z / r;
  double pmm = 1.0;
  for (int k = 1; k <= m; ++k) pmm *= -(2.0 * k - 1.0);
  double p = pmm;
  if (l > m) {
    double pm2 = pmm, pm1 = (2.0 * m + 1.0) * mu * pmm;
    p = pm1;
    for (int ll = m + 2; ll <= l; ++ll) {
      p = ((2.0 * ll - 1.0) * mu * pm1 - (double)(ll + m - 1) * pm2) / (double)(ll - m);
      pm2 = pm1;
      pm1 = p;
    }
  }
  double er = 1.0, ei = 0.0;
  const double cx = x / r, cy = y / r;
  for (int k = 0; k < m; ++k) {
    const double t = er * cx - ei * cy;
    ei = er * cy + ei * cx;
    er = t;
  }
  static const std::vector<double> ntab = [] {
    std::vector<double> t((BISP_LMAX + 1) * (BISP_LMAX + 1));
    for (int a = 0; a <= BISP_LMAX; ++a)
      for (int b = 0; b <= a; ++b) t[a * (BISP_LMAX + 1) + b] = std::exp(0.5 * (lfact(a - b) - lfact(a + b)));
    return t;
  }();
  const double norm = ntab[l * (BISP_LMAX + 1) + m];
  *re = norm * p * er;
  *im = norm * p * ei;
}

// y_l^{m*} for signed m
void ystar_host(int l, int m, double x, double y, double z, double* re, double* im) {
  const int am = std::abs(m);
  double a, b;
  ylm_host(l, am, x, y, z, &a, &b);
  if (m >= 0) {
    *re = a;
    *im = -b;
  } else {  // y_l^{-m*} = (-1)^m y_l^m
    const double s = (am & 1) ? -1.0 : 1.0;
    *re = s * a;
    *im = s * b;
  }
}

struct cplx {
  double r = 0, i = 0;
};
cplx cm(cplx a, cplx b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }

// ---------------------------------------------------------------------------------
// device buffer cache
// ---------------------------------------------------------------------------------
// Allocation-failure injection for tests: with BISP_FAIL_ALLOC=k in the environment, the k-th
// device allocation within one library call fails as if cudaMalloc had (the count restarts at
// every call of the C ABI).
thread_local int g_alloc_calls = 0;
bool inject_alloc_failure() {
  const char* e = getenv("BISP_FAIL_ALLOC");
  if (!e || !*e) return false;
  return ++g_alloc_calls == atoi(e);
}

struct DBuf {
  void* p = nullptr;
  size_t n = 0;
  void ensure(size_t bytes, size_t* total) {
    if (bytes <= n) return;
    release(total);
    if (inject_alloc_failure()) {
      char buf[200];
      snprintf(buf, sizeof buf, "device allocation of %.3f GB failed (injected by BISP_FAIL_ALLOC)", bytes / 1e9);
      fail(BISP_ENOMEM, buf);
    }
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      char buf[160];
      snprintf(buf, sizeof buf, "device allocation of %.3f GB failed (%s)", bytes / 1e9, cudaGetErrorString(e));
      fail(BISP_ENOMEM, buf);
    }
    n = bytes;
    *total += bytes;
  }
  void release(size_t* total) {
    if (p) {
      cudaFree(p);
      *total -= n;
    }
    p = nullptr;
    n = 0;
  }
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

struct Comp {
  int l, m, part;
};

struct Catalog {
  bool assigned = false;
  int64_t n = 0;
  bool unit_w = true;   // N channels alias the D channels (no weights)
  int nspec = 0;
  DBuf spec;            // [nspec][Nk] float2
  double sumw = 0.0;
  std::vector<double> sbar;  // per D channel: sum w^3 part(y*)
  double sumR3 = 0.0;
  DBuf dbg_mesh;
  int launches = 0;
  double ms = 0.0;
};

}  // namespace

void bisp::set_last_error(const std::string& m) { g_err = m; }

// one injected stall per kernel kind and library call (the first launch), reset by guarded()
thread_local unsigned g_stalls_used = 0;
bool bisp::inject_stall(const char* kernel) {
  const char* e = getenv("BISP_INJECT_STALL");
  if (!e || !strstr(e, kernel)) return false;
  const unsigned bit = strcmp(kernel, "pair") == 0 ? 1u : 2u;
  if (g_stalls_used & bit) return false;
  g_stalls_used |= bit;
  return true;
}

struct bisp_plan {
  // parameters
  int N = 0, NH = 0, nb = 0, nmult = 0, los = 0, mas = 2, interlace = 0, want_window = 0, precision = 0;
  int estimator = 0;  // bisp_estimator
  int los_obj = 3;    // object of the triplet carrying y_L^{M*}(x_hat): 3 (main text), 1 or 2 (App. B)
  // autotuned launch shape: z-pass row groups per CTA (0 until measured), and the timings seen
  int zgroups = 0;
  std::vector<std::pair<int, float>> tune_log;
  int diagonal = 0;   // only k1 = k2 outputs
  double L = 0, H = 0, kF = 0, V = 0, P0 = 0, obs[3] = {0, 0, 0};
  size_t max_bytes = 0;
  int64_t Ng = 0, Nk = 0;
  std::vector<double> edges;
  std::vector<std::array<int, 3>> ells;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool debug_mesh = false;
  // channels
  std::vector<Chan> dch, nch;
  std::vector<int> Ls, ls;
  int d00 = 0, n00 = 0;
  // shells
  std::vector<long long> qlo, qhi;
  std::vector<int> Pb;
  std::vector<double> nmodes;
  std::vector<uint32_t> zlist;
  std::vector<int64_t> zoff;
  // three-point function: separations of r-bin a at roff[roff_off[a] .. roff_off[a+1]), packed
  // (sx+512) | (sy+512) << 10 | (sz+512) << 20
  std::vector<uint32_t> roff;
  std::vector<int64_t> roff_off;
  std::vector<Comp> comps;
  std::map<std::tuple<int, int, int>, int> comp_index;  // (l, m, part) -> index
  std::vector<std::vector<cplx>> Y;                     // [b][lm index (l, m signed)]
  // contraction recipes per multipole (pair-kernel terms with g indices into a G set)
  struct Term {
    std::vector<PairRecipe> x, y;
  };
  std::vector<std::vector<Term>> terms;
  // line of sight on x1 or x2 (App. B): per multipole and per m of the other object, the
  // contraction over m and M of the weighted object's fields is done in k space, giving the real
  // fields K_A, K_B of i^l (K_A + i K_B) = sum_m 3j F_l^m[delta n_L^M] (SRC_SHELL_SUM fields,
  // entries (coef, |m|, part, D channel)); kterms are the data and window passes' terms over the
  // components followed by these fields
  struct KField {
    int l;
    std::vector<std::tuple<float, int, int, int>> ent;
  };
  std::vector<KField> kfields;
  std::vector<std::vector<Term>> kterms;
  int pass_ncomp(bool unit) const {  // field slots per bin in the pool
    return (int)comps.size() + (unit || los_obj == 3 ? 0 : (int)kfields.size());
  }
  // the same expansion as plain FP64 terms per multipole: sum_x coef F_c1(b1) F_c2(b2) G_g
  struct Tri {
    int c1, c2, g;
    double coef;
  };
  std::vector<std::vector<Tri>> tri64;
  // device constants
  DBuf tw, winv, ynorm, cw2, qlo_d, qhi_d, zmodes, zmode_off;
  Catalog cat[2];
  // measurement buffers
  DBuf pass_spec[2], gf[2], qf, pool, invscr, pairscr, pairout, zpart;
  DBuf ws;  // assignment workspace (grow-only)
  DBuf flags;  // device error flags of the measurement kernels
  // plain FP64 form (precision BISP_FP64)
  DBuf ynorm_d, cw2_d, f64work, f64spec, f64g, f64q, f64shell, f64part, f64out;
  // three-point function: separation lists, unit deconvolution table, kernel meshes, gathers
  DBuf roff_d, ones, kmesh, gath;
  F64Fft fft64;
  size_t bytes = 0;
  // bookkeeping
  double alpha = 0.0, normI = 0.0;
  int launches_measure = 0, pair_launches = 0, pair_kernel = -1;
  double ms_measure = 0.0, ms_pair = 0.0, pair_bytes = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  int lm_index(int l, int m) const {  // index of (l, m) in the Y table: l^2 + (m + l)
    return l * l + (m + l);
  }
  int dchan(int L_, int M_, int part) const {
    for (size_t c = 0; c < dch.size(); ++c)
      if (dch[c].L == L_ && dch[c].M == M_ && dch[c].part == part) return (int)c;
    return -1;
  }
  int nchan(int L_, int M_, int part) const {
    for (size_t c = 0; c < nch.size(); ++c)
      if (nch[c].L == L_ && nch[c].M == M_ && nch[c].part == part) return (int)c;
    return -1;
  }
};

namespace {

// ---------------------------------------------------------------------------------
// plan construction
// ---------------------------------------------------------------------------------
void validate(const bisp_params* p) {
  if (!p) fail(BISP_EINVAL, "params is NULL");
  const int N = p->nmesh;
  if (N < 16 || N > BISP_NMAX || (N & (N - 1))) fail(BISP_EINVAL, "nmesh must be a power of two in [16, 1024]");
  if (!(p->box_len > 0.0) || !std::isfinite(p->box_len)) fail(BISP_EINVAL, "box_len must be positive");
  if (p->estimator != BISP_BISPECTRUM && p->estimator != BISP_THREEPT) fail(BISP_EINVAL, "estimator");
  const bool three = p->estimator == BISP_THREEPT;
  if (three && p->precision != BISP_FP32) fail(BISP_EUNSUPPORTED, "the FP64 form covers the bispectrum only");
  if (p->nbins < 1 || !p->k_edges) fail(BISP_EINVAL, "need nbins >= 1 and k_edges");
  for (int b = 0; b <= p->nbins; ++b) {
    const double e = p->k_edges[b];
    if (!std::isfinite(e) || (three ? !(e >= 0.0) : !(e > 0.0)))
      fail(BISP_EINVAL, three ? "r edges must be non-negative and finite" : "k_edges must be positive and finite");
    if (b && !(p->k_edges[b] > p->k_edges[b - 1])) fail(BISP_EINVAL, "k_edges must be ascending");
  }
  if (p->n_mult < 1 || !p->ells) fail(BISP_EINVAL, "need n_mult >= 1 and ells");
  for (int i = 0; i < p->n_mult; ++i) {
    const int l1 = p->ells[3 * i], l2 = p->ells[3 * i + 1], L = p->ells[3 * i + 2];
    const bool ok = l1 >= l2 && l2 >= 0 && L % 2 == 0 && L >= std::abs(l1 - l2) && L <= l1 + l2 &&
                    (l1 + l2 + L) % 2 == 0;
    if (!ok) {
      char buf[128];
      snprintf(buf, sizeof buf, "multipole (%d,%d,%d) violates the selection rules", l1, l2, L);
      fail(BISP_EINVAL, buf);
    }
    if (l1 > BISP_LMAX || L > BISP_LMAX) fail(BISP_EUNSUPPORTED, "l and L above 4 are not built");
  }
  if (p->los != BISP_LOS_GLOBAL_Z && p->los != BISP_LOS_LOCAL) fail(BISP_EINVAL, "los");
  if (p->los_object < 0 || p->los_object > 3) fail(BISP_EINVAL, "los_object must be 0, 1, 2 or 3");
  if ((p->los_object == 1 || p->los_object == 2) && p->los == BISP_LOS_LOCAL &&
      (p->estimator != BISP_BISPECTRUM || p->precision != BISP_FP32))
    fail(BISP_EUNSUPPORTED, "the line of sight on x1 or x2 is built for the FP32 bispectrum only");
  if (p->mas < 1 || p->mas > 3) fail(BISP_EINVAL, "mas must be 1 (NGP), 2 (CIC) or 3 (TSC)");
  if (p->precision != BISP_FP32 && p->precision != BISP_FP64) fail(BISP_EINVAL, "precision must be BISP_FP32 or BISP_FP64");
  if (!std::isfinite(p->fkp_P0) || p->fkp_P0 < 0) fail(BISP_EINVAL, "fkp_P0");
  if (p->los == BISP_LOS_LOCAL)
    for (int k = 0; k < 3; ++k)
      if (!std::isfinite(p->observer[k])) fail(BISP_EINVAL, "observer");
}

void build_channels(bisp_plan* P) {
  std::vector<int> Ls = {0}, ls;
  for (auto& e : P->ells) {
    Ls.push_back(e[2]);
    ls.push_back(e[0]);
    ls.push_back(e[1]);
  }
  std::sort(Ls.begin(), Ls.end());
  Ls.erase(std::unique(Ls.begin(), Ls.end()), Ls.end());
  std::sort(ls.begin(), ls.end());
  ls.erase(std::unique(ls.begin(), ls.end()), ls.end());
  P->Ls = Ls;
  P->ls = ls;
  P->dch.clear();
  P->nch.clear();
  if (P->los == BISP_LOS_GLOBAL_Z) {
    P->dch.push_back({0, 0, 0, 1, 1});
    P->nch.push_back({0, 0, 0, 2, 0});
  } else {
    for (int L : Ls)
      for (int M = 0; M <= L; ++M)
        for (int part = 0; part < (M ? 2 : 1); ++part) {
          P->dch.push_back({L, M, part, 1, 1});
          P->nch.push_back({L, M, part, 2, 0});
        }
  }
  P->d00 = P->dchan(0, 0, 0);
  P->n00 = P->nchan(0, 0, 0);
  P->comps.clear();
  P->comp_index.clear();
  for (int l : ls)
    for (int m = 0; m <= l; ++m)
      for (int part = 0; part < (m ? 2 : 1); ++part) {
        P->comp_index[{l, m, part}] = (int)P->comps.size();
        P->comps.push_back({l, m, part});
      }
  if ((int)P->comps.size() > 32) fail(BISP_EUNSUPPORTED, "too many field components");
}

void build_shells(bisp_plan* P) {
  const int N = P->N, nb = P->nb;
  const long long qmax = 3LL * (N / 2) * (N / 2);
  P->qlo.assign(nb, -1);
  P->qhi.assign(nb, -1);
  // bin of q: e_b <= kF sqrt(q) < e_{b+1}, FP64
  std::vector<int> binq(qmax + 1, -1);
  for (long long q = 1; q <= qmax; ++q) {
    const double k = P->kF * std::sqrt((double)q);
    const auto it = std::upper_bound(P->edges.begin(), P->edges.end(), k);
    const int b = (int)(it - P->edges.begin()) - 1;
    if (b >= 0 && b < nb) binq[q] = b;
  }
  for (int b = 0; b < nb; ++b) {
    for (long long q = 1; q <= qmax; ++q)
      if (binq[q] == b) {
        if (P->qlo[b] < 0) P->qlo[b] = q;
        P->qhi[b] = q + 1;
      }
    if (P->qlo[b] < 0) P->qlo[b] = P->qhi[b] = 1;  // empty bin
  }
  P->Pb.assign(nb, 0);
  for (int b = 0; b < nb; ++b) {
    int pb = (int)std::floor(std::sqrt((double)(P->qhi[b] - 1)));
    while ((long long)(pb + 1) * (pb + 1) <= P->qhi[b] - 1) ++pb;
    while ((long long)pb * pb > P->qhi[b] - 1) --pb;
    P->Pb[b] = std::min(pb, N / 2 - 1);
  }
  // mode counts and shell averages of y_l^{m*} over the full cube (Nyquist planes out)
  const int Pm = *std::max_element(P->Pb.begin(), P->Pb.end());
  const int lmax = P->ls.empty() ? 0 : P->ls.back();
  const int nlm = (lmax + 1) * (lmax + 1);
  std::vector<std::vector<cplx>> S(nb, std::vector<cplx>(nlm));
  std::vector<double> cnt(nb, 0.0);
  for (int x = -Pm; x <= Pm; ++x)
    for (int y = -Pm; y <= Pm; ++y)
      for (int z = -Pm; z <= Pm; ++z) {
        const long long q = (long long)x * x + (long long)y * y + (long long)z * z;
        if (q == 0 || q > qmax) continue;
        const int b = binq[q];
        if (b < 0 || std::abs(x) > P->Pb[b] || std::abs(y) > P->Pb[b] || std::abs(z) > P->Pb[b]) continue;
        cnt[b] += 1.0;
        for (int l : P->ls)
          for (int m = -l; m <= l; ++m) {
            double re, im;
            ystar_host(l, m, x, y, z, &re, &im);
            cplx& s = S[b][P->lm_index(l, m)];
            s.r += re;
            s.i += im;
          }
      }
  P->nmodes = cnt;
  // half-spectrum shell mode lists (nz >= 0; for nz = 0 both k and -k are listed)
  {
    std::vector<std::vector<uint32_t>> lists(nb);
    for (int x = -Pm; x <= Pm; ++x)
      for (int y = -Pm; y <= Pm; ++y)
        for (int z = 0; z <= Pm; ++z) {
          const long long q = (long long)x * x + (long long)y * y + (long long)z * z;
          if (q == 0 || q > qmax) continue;
          const int b = binq[q];
          if (b < 0 || std::abs(x) > P->Pb[b] || std::abs(y) > P->Pb[b] || z > P->Pb[b]) continue;
          lists[b].push_back((uint32_t)(x + 512) | ((uint32_t)(y + 512) << 10) | ((uint32_t)z << 20));
        }
    P->zlist.clear();
    P->zoff.assign(nb + 1, 0);
    for (int b = 0; b < nb; ++b) {
      P->zoff[b] = (int64_t)P->zlist.size();
      P->zlist.insert(P->zlist.end(), lists[b].begin(), lists[b].end());
    }
    P->zoff[nb] = (int64_t)P->zlist.size();
  }
  P->Y.assign(nb, std::vector<cplx>(nlm));
  for (int b = 0; b < nb; ++b)
    for (int i = 0; i < nlm; ++i)
      if (cnt[b] > 0) P->Y[b][i] = {S[b][i].r / cnt[b], S[b][i].i / cnt[b]};
}

// r-bins of the three-point function (Sec. 4.3): separations s, integer with |s_i| <= N/2 - 1,
// in bin a when e_a <= H |s| < e_{a+1} (FP64); N_r(a) separations per bin.  The filtered fields
// use every mode but the Nyquist planes (prune extent N/2 - 1).
void build_rshells(bisp_plan* P) {
  const int N = P->N, nb = P->nb, h = N / 2 - 1;
  const int ext = (int)std::min<double>(h, std::floor(P->edges[nb] / P->H) + 1.0);
  // the separation lists hold at most (2 ext + 1)^3 entries of 4 bytes
  if ((double)(2 * ext + 1) * (2 * ext + 1) * (2 * ext + 1) > 6.4e7)
    fail(BISP_EUNSUPPORTED, "r-bins up to this radius reach beyond 199 cells (more than 6.4e7 separations)");
  const long long qmax = 3LL * ext * ext;
  std::vector<int> binq(qmax + 1, -1);
  for (long long q = 0; q <= qmax; ++q) {
    const double r = P->H * std::sqrt((double)q);
    const auto it = std::upper_bound(P->edges.begin(), P->edges.end(), r);
    const int a = (int)(it - P->edges.begin()) - 1;
    if (a >= 0 && a < nb) binq[q] = a;
  }
  std::vector<std::vector<uint32_t>> lists(nb);
  for (int x = -ext; x <= ext; ++x)
    for (int y = -ext; y <= ext; ++y)
      for (int z = -ext; z <= ext; ++z) {
        const int a = binq[(long long)x * x + (long long)y * y + (long long)z * z];
        if (a >= 0)
          lists[a].push_back((uint32_t)(x + 512) | ((uint32_t)(y + 512) << 10) | ((uint32_t)(z + 512) << 20));
      }
  P->roff.clear();
  P->roff_off.assign(nb + 1, 0);
  P->nmodes.assign(nb, 0.0);
  for (int a = 0; a < nb; ++a) {
    P->roff_off[a] = (int64_t)P->roff.size();
    P->roff.insert(P->roff.end(), lists[a].begin(), lists[a].end());
    P->nmodes[a] = (double)lists[a].size();
  }
  P->roff_off[nb] = (int64_t)P->roff.size();
  P->Pb.assign(nb, N / 2 - 1);
  P->qlo.assign(nb, 1);
  P->qhi.assign(nb, 1);
  P->zlist.clear();
  P->zoff.assign(nb + 1, 0);
  const int lmax = P->ls.empty() ? 0 : P->ls.back();
  P->Y.assign(nb, std::vector<cplx>((lmax + 1) * (lmax + 1)));
}

// Real-component expansion of Re sum_{m1 m2 M} 3j F_{l1}^{m1} F_{l2}^{m2} G_L^M with
//   F_l^m = i^l (A + i B),  F_l^{-m} = (-1)^m i^l (A - i B)   (three-point function: no i^l),
//   G_L^M = R + i I,        G_L^{-M} = (-1)^M (R - i I)   (global LOS: G_L^M = delta_M0 G)
// grouped into pair-kernel terms on the side with fewer components.
// Contraction terms of one multipole from its trilinear expansion, grouped by the side with
// fewer distinct components: each term pairs one bare component field with a built side
// sum_(c, g) coef F_c G_g; a built side spans at most 8 components (a term with more is split
// into terms over groups of 8 components, whose sum is the same).
std::vector<bisp_plan::Term> terms_of(const std::map<int, std::vector<std::tuple<int, int, double>>>& by1,
                                      const std::map<int, std::vector<std::tuple<int, int, double>>>& by2) {
  std::vector<bisp_plan::Term> ts;
  const bool bare_y = by2.size() <= by1.size();
  for (auto& kv : bare_y ? by2 : by1) {
    // the built side's entries in component order, cut into groups of at most 8 components
    std::vector<std::tuple<int, int, double>> ent = kv.second;
    std::stable_sort(ent.begin(), ent.end(), [](const auto& a, const auto& b) { return std::get<0>(a) < std::get<0>(b); });
    std::vector<PairRecipe> built;
    int ncomp = 0, last = -1;
    auto flush = [&] {
      if (built.empty()) return;
      bisp_plan::Term t;
      if (bare_y) {
        t.x = built;
        t.y.push_back({kv.first, -1, 1.0f});
      } else {
        t.x.push_back({kv.first, -1, 1.0f});
        t.y = built;
      }
      ts.push_back(t);
      built.clear();
      ncomp = 0;
      last = -1;
    };
    for (auto& r : ent) {
      if (std::get<0>(r) != last) {
        if (ncomp == 8) flush();
        ++ncomp;
        last = std::get<0>(r);
      }
      built.push_back({std::get<0>(r), std::get<1>(r), (float)std::get<2>(r)});
    }
    flush();
  }
  return ts;
}

void build_recipes(bisp_plan* P) {
  P->terms.clear();
  P->tri64.clear();
  const bool glob = P->los == BISP_LOS_GLOBAL_Z;
  for (auto& e : P->ells) {
    const int l1 = e[0], l2 = e[1], L = e[2];
    std::map<std::tuple<int, int, int>, double> tri;  // (c1, c2, g) -> coef
    // i^{l1+l2}: the bispectrum's fields are F_l^m = i^l (A + i B); the three-point function's
    // separation averages are F_l^m = A + i B (F_l^{-m} = (-1)^m conj F_l^m)
    const double il = P->estimator == BISP_THREEPT ? 1.0 : ((((l1 + l2) / 2) & 1) ? -1.0 : 1.0);
    for (int m1 = -l1; m1 <= l1; ++m1)
      for (int m2 = -l2; m2 <= l2; ++m2) {
        const int M = -m1 - m2;
        if (std::abs(M) > L || (glob && M != 0)) continue;
        const double w = wigner3j(l1, l2, L, m1, m2, M);
        if (w == 0.0) continue;
        const int a1 = std::abs(m1), a2 = std::abs(m2), aM = std::abs(M);
        const double k1 = (m1 < 0 && (a1 & 1)) ? -1.0 : 1.0;
        const double k2 = (m2 < 0 && (a2 & 1)) ? -1.0 : 1.0;
        const double s1 = m1 < 0 ? -1.0 : 1.0, s2 = m2 < 0 ? -1.0 : 1.0;
        const int A1 = P->comp_index.at({l1, a1, 0}), B1 = a1 ? P->comp_index.at({l1, a1, 1}) : -1;
        const int A2 = P->comp_index.at({l2, a2, 0}), B2 = a2 ? P->comp_index.at({l2, a2, 1}) : -1;
        int R, I;
        double kG, sG;
        if (glob) {
          R = P->d00;
          I = -1;
          kG = 1.0;
          sG = 1.0;
        } else {
          R = P->dchan(L, aM, 0);
          I = aM ? P->dchan(L, aM, 1) : -1;
          kG = (M < 0 && (aM & 1)) ? -1.0 : 1.0;
          sG = M < 0 ? -1.0 : 1.0;
        }
        const double kap = w * il * k1 * k2 * kG;
        tri[{A1, A2, R}] += kap;
        if (B1 >= 0 && B2 >= 0) tri[{B1, B2, R}] += -kap * s1 * s2;
        if (B1 >= 0 && I >= 0) tri[{B1, A2, I}] += -kap * s1 * sG;
        if (B2 >= 0 && I >= 0) tri[{A1, B2, I}] += -kap * s2 * sG;
      }
    double mx = 0.0;
    for (auto& kv : tri) mx = std::max(mx, std::fabs(kv.second));
    std::map<int, std::vector<std::tuple<int, int, double>>> by1, by2;
    std::vector<bisp_plan::Tri> t64;
    for (auto& kv : tri) {
      if (std::fabs(kv.second) <= 1e-13 * mx) continue;
      const int c1 = std::get<0>(kv.first), c2 = std::get<1>(kv.first), g = std::get<2>(kv.first);
      t64.push_back({c1, c2, g, kv.second});
      by1[c1].push_back({c2, g, kv.second});
      by2[c2].push_back({c1, g, kv.second});
    }
    P->terms.push_back(terms_of(by1, by2));
    P->tri64.push_back(t64);
  }
  P->kfields.clear();
  P->kterms.clear();
  if (P->los_obj == 3) return;
  // line of sight on object a (App. B): K_{m_o}(x; b_a) = sum_{m_a} 3j F_{l_a}^{m_a}[delta n_L^M](x; b_a),
  // M = -m1 - m2, with delta n_L^M = kX (R + i sX I) in its real channels and, for signed m,
  // Re y^{m*} = sr part0(|m|), Im y^{m*} = si part1(|m|); then
  // Re[K_{m_o} F_{l_o}^{m_o}[delta n_0^0] G_0^0] = il k_o (K_A A_o - s_o K_B B_o) G_0^0.
  const int a = P->los_obj;
  for (auto& e : P->ells) {
    const int l1 = e[0], l2 = e[1], L = e[2];
    const int la = a == 1 ? l1 : l2, lo = a == 1 ? l2 : l1;
    const double il = (((l1 + l2) / 2) & 1) ? -1.0 : 1.0;
    std::map<std::tuple<int, int, int>, double> tri;  // (c1, c2, g) -> coef
    for (int mo = -lo; mo <= lo; ++mo) {
      std::map<std::tuple<int, int, int>, double> KA, KB;  // (|m|, part, channel) -> coef
      for (int ma = -la; ma <= la; ++ma) {
        const int m1 = a == 1 ? ma : mo, m2 = a == 1 ? mo : ma;
        const int M = -m1 - m2;
        if (std::abs(M) > L) continue;
        const double w = wigner3j(l1, l2, L, m1, m2, M);
        if (w == 0.0) continue;
        const int aM = std::abs(M), am = std::abs(ma);
        const int R = P->dchan(L, aM, 0), I = aM ? P->dchan(L, aM, 1) : -1;
        const double kX = (M < 0 && (aM & 1)) ? -1.0 : 1.0, sX = M < 0 ? -1.0 : 1.0;
        const double sr = (ma < 0 && (am & 1)) ? -1.0 : 1.0, si = ma < 0 ? -sr : sr;
        const double c = w * kX;
        KA[{am, 0, R}] += c * sr;
        if (I >= 0 && am) KA[{am, 1, I}] += -c * sX * si;
        if (am) KB[{am, 1, R}] += c * si;
        if (I >= 0) KB[{am, 0, I}] += c * sX * sr;
      }
      auto add_field = [&](const std::map<std::tuple<int, int, int>, double>& ent) {
        bisp_plan::KField f;
        f.l = la;
        double mx = 0.0;
        for (auto& kv : ent) mx = std::max(mx, std::fabs(kv.second));
        for (auto& kv : ent)
          if (std::fabs(kv.second) > 1e-13 * mx)
            f.ent.push_back({(float)kv.second, std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first)});
        if (f.ent.empty()) return -1;
        if ((int)f.ent.size() > INV_MAXE) fail(BISP_EUNSUPPORTED, "line-of-sight field with too many entries");
        P->kfields.push_back(f);
        return (int)(P->comps.size() + P->kfields.size() - 1);
      };
      const int iA = add_field(KA), iB = add_field(KB);
      const int amo = std::abs(mo);
      const double ko = (mo < 0 && (amo & 1)) ? -1.0 : 1.0, so = mo < 0 ? -1.0 : 1.0;
      const int Ao = P->comp_index.at({lo, amo, 0}), Bo = amo ? P->comp_index.at({lo, amo, 1}) : -1;
      auto put = [&](int kf, int comp, double coef) {
        if (kf < 0 || comp < 0) return;
        if (a == 1) tri[{kf, comp, P->d00}] += coef;
        else tri[{comp, kf, P->d00}] += coef;
      };
      put(iA, Ao, il * ko);
      put(iB, Bo, -il * ko * so);
    }
    double mx = 0.0;
    for (auto& kv : tri) mx = std::max(mx, std::fabs(kv.second));
    std::map<int, std::vector<std::tuple<int, int, double>>> by1, by2;
    for (auto& kv : tri) {
      if (std::fabs(kv.second) <= 1e-13 * mx) continue;
      const int c1 = std::get<0>(kv.first), c2 = std::get<1>(kv.first), g = std::get<2>(kv.first);
      by1[c1].push_back({c2, g, kv.second});
      by2[c2].push_back({c1, g, kv.second});
    }
    P->kterms.push_back(terms_of(by1, by2));
  }
}

void upload_tables(bisp_plan* P) {
  const int N = P->N;
  std::vector<float2> tw(BISP_TWN);
  for (int j = 0; j < BISP_TWN; ++j) {
    const double a = -2.0 * M_PI * (double)j / BISP_TWN;
    tw[j] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  // deconvolution 1/W per axis, alias-sum tables C/W^2 (even and alternating images)
  std::vector<float> winv(N), cw2(2 * N);
  std::vector<double> cw2d(2 * N);
  const int p = P->mas;
  for (int j = 0; j < N; ++j) {
    const int n = j < N / 2 ? j : j - N;
    const double x = M_PI * n / N;
    const double sc = n == 0 ? 1.0 : std::sin(x) / x;
    const double w = std::pow(sc, p);
    winv[j] = (float)(1.0 / w);
    const double s2 = std::sin(x) * std::sin(x), c = std::cos(x), c2 = c * c;
    double E, O;  // sum_m sinc^{2p}(x + pi m), sum_m (-1)^m sinc^{2p}(x + pi m)
    if (p == 1) {
      E = 1.0;
      O = c;
    } else if (p == 2) {
      E = 1.0 - 2.0 / 3.0 * s2;
      O = c * (5.0 + c2) / 6.0;
    } else {
      E = 1.0 - s2 + 2.0 / 15.0 * s2 * s2;
      O = c * (61.0 + 58.0 * c2 + c2 * c2) / 120.0;
    }
    cw2d[j] = E / (w * w);
    cw2d[N + j] = O / (w * w);
    cw2[j] = (float)cw2d[j];
    cw2[N + j] = (float)cw2d[N + j];
  }
  std::vector<float> yn((BISP_LMAX + 1) * (BISP_LMAX + 1), 0.f);
  std::vector<double> ynd(yn.size(), 0.0);
  for (int l = 0; l <= BISP_LMAX; ++l)
    for (int m = 0; m <= l; ++m) {
      ynd[l * (BISP_LMAX + 1) + m] = std::exp(0.5 * (lfact(l - m) - lfact(l + m)));
      yn[l * (BISP_LMAX + 1) + m] = (float)ynd[l * (BISP_LMAX + 1) + m];
    }
  P->tw.ensure(tw.size() * sizeof(float2), &P->bytes);
  P->winv.ensure(winv.size() * sizeof(float), &P->bytes);
  P->cw2.ensure(cw2.size() * sizeof(float), &P->bytes);
  P->ynorm.ensure(yn.size() * sizeof(float), &P->bytes);
  P->zmodes.ensure(std::max<size_t>(P->zlist.size(), 1) * 4, &P->bytes);
  P->zmode_off.ensure(P->zoff.size() * 8, &P->bytes);
  if (!P->zlist.empty())
    BISP_CUDA(cudaMemcpy(P->zmodes.p, P->zlist.data(), P->zlist.size() * 4, cudaMemcpyHostToDevice));
  BISP_CUDA(cudaMemcpy(P->zmode_off.p, P->zoff.data(), P->zoff.size() * 8, cudaMemcpyHostToDevice));
  P->qlo_d.ensure(P->nb * sizeof(long long), &P->bytes);
  P->qhi_d.ensure(P->nb * sizeof(long long), &P->bytes);
  BISP_CUDA(cudaMemcpy(P->tw.p, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
  BISP_CUDA(cudaMemcpy(P->winv.p, winv.data(), winv.size() * sizeof(float), cudaMemcpyHostToDevice));
  BISP_CUDA(cudaMemcpy(P->cw2.p, cw2.data(), cw2.size() * sizeof(float), cudaMemcpyHostToDevice));
  BISP_CUDA(cudaMemcpy(P->ynorm.p, yn.data(), yn.size() * sizeof(float), cudaMemcpyHostToDevice));
  BISP_CUDA(cudaMemcpy(P->qlo_d.p, P->qlo.data(), P->nb * sizeof(long long), cudaMemcpyHostToDevice));
  BISP_CUDA(cudaMemcpy(P->qhi_d.p, P->qhi.data(), P->nb * sizeof(long long), cudaMemcpyHostToDevice));
  if (P->estimator == BISP_THREEPT) {
    P->roff_d.ensure(std::max<size_t>(P->roff.size(), 1) * 4, &P->bytes);
    if (!P->roff.empty())
      BISP_CUDA(cudaMemcpy(P->roff_d.p, P->roff.data(), P->roff.size() * 4, cudaMemcpyHostToDevice));
    const std::vector<float> one(N, 1.f);
    P->ones.ensure(N * sizeof(float), &P->bytes);
    BISP_CUDA(cudaMemcpy(P->ones.p, one.data(), N * sizeof(float), cudaMemcpyHostToDevice));
  }
  if (P->precision == BISP_FP64) {
    P->ynorm_d.ensure(ynd.size() * 8, &P->bytes);
    P->cw2_d.ensure(cw2d.size() * 8, &P->bytes);
    BISP_CUDA(cudaMemcpy(P->ynorm_d.p, ynd.data(), ynd.size() * 8, cudaMemcpyHostToDevice));
    BISP_CUDA(cudaMemcpy(P->cw2_d.p, cw2d.data(), cw2d.size() * 8, cudaMemcpyHostToDevice));
    P->fft64 = f64_fft_create(N);
  }
}

void admit(bisp_plan* P, size_t extra) {
  size_t fre = 0, tot = 0;
  BISP_CUDA(cudaMemGetInfo(&fre, &tot));
  const size_t reserve = (size_t)2 << 30;
  size_t cap = fre > reserve ? fre - reserve : 0;
  if (P->max_bytes && P->bytes + extra > P->max_bytes) {
    char buf[200];
    snprintf(buf, sizeof buf, "admission: needs %.3f GB, cap max_device_bytes = %.3f GB", (P->bytes + extra) / 1e9,
             P->max_bytes / 1e9);
    fail(BISP_ENOMEM, buf);
  }
  if (extra > cap) {
    char buf[200];
    snprintf(buf, sizeof buf, "admission: needs %.3f GB more device memory, %.3f GB free", extra / 1e9, fre / 1e9);
    fail(BISP_ENOMEM, buf);
  }
}

// ---------------------------------------------------------------------------------
// assign
// ---------------------------------------------------------------------------------
void do_assign(bisp_plan* P, int which, const float* xyz, const float* w, const float* nbar, int64_t n,
               int ptr_is_device) {
  if (which != BISP_DATA && which != BISP_RANDOMS) fail(BISP_EINVAL, "which must be BISP_DATA or BISP_RANDOMS");
  if (n < 0) fail(BISP_EINVAL, "n < 0");
  if (n > 0 && !xyz) fail(BISP_EINVAL, "xyz is NULL");
  if (n >= (int64_t)0xffffffffLL) fail(BISP_EUNSUPPORTED, "more than 2^32-1 particles");
  NvtxRange nv(which == BISP_DATA ? "bisp_assign data" : "bisp_assign randoms");
  Catalog& C = P->cat[which];
  cudaStream_t s = P->stream;
  int launches = 0;
  C.assigned = false;  // set again only when this assignment completes (its buffers may be replaced)
  BISP_CUDA(cudaEventRecord(P->ev0, s));
  const int N = P->N;
  const int64_t Ng = P->Ng;
  const bool unit_w = !w && !(nbar && P->P0 > 0);
  // channels assigned for this catalogue: D channels, plus N channels unless aliased
  std::vector<Chan> ch = P->dch;
  if (!unit_w)
    for (auto& c : P->nch) ch.push_back(c);
  const int nchan = (int)ch.size();
  if (nchan > 32) fail(BISP_EUNSUPPORTED, "too many channels");
  const int ilv = P->interlace ? 1 : 0;
  // workspace: one grow-only device arena kept by the plan (no allocation once it is large
  // enough).  Region 1 holds what is dead after the particle gather (host input copy, unsorted
  // keys, indices, offsets, channel values, sort scratch) and is then reused for the
  // interlaced mesh; region 2 holds what the deposit still reads.
  const int64_t nn = std::max<int64_t>(n, 1);
  const int nsum = 1 + (int)P->dch.size();
  const int pblk = prep_blocks(n);
  const size_t sortb = radix_sort_scratch_bytes(n);
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t b_din = ptr_is_device ? 0 : al((size_t)n * 4 * (3 + (w ? 1 : 0) + (nbar ? 1 : 0)));
  const size_t b_keys = al(nn * 4), b_frac = al(nn * 16), b_vals = al((size_t)nn * 4 * nchan), b_sort = al(sortb);
  const size_t r1a = b_din + 2 * b_keys + b_frac + b_vals + b_sort;
  const size_t b_mesh1 = ilv ? al((size_t)nchan * Ng * 4) : 0;
  const size_t r1 = std::max(r1a, b_mesh1);
  const size_t b_cells = al((size_t)(Ng + 1) * 4 * 2), b_scan = al(scan_scratch_bytes(Ng + 1));
  const size_t b_part = al(std::max<size_t>((size_t)pblk * nsum * 8, 1024 * 8));
  const size_t r2 = 2 * b_keys + b_cells + b_scan + b_frac + b_vals + b_part + 256;
  // The field pool of the measurement is idle during an assignment (calls on a plan never
  // overlap), so the arena borrows it when it is large enough.
  const size_t spec_need = (size_t)nchan * Ng * 4;
  const bool in_pool = P->pool.n >= r1 + r2;
  admit(P, (!in_pool && r1 + r2 > P->ws.n ? r1 + r2 - P->ws.n : 0) +
               (spec_need > C.spec.n ? spec_need - C.spec.n : 0));
  if (!in_pool) P->ws.ensure(r1 + r2, &P->bytes);
  unsigned char* const arena = in_pool ? P->pool.as<unsigned char>() : P->ws.as<unsigned char>();
  unsigned char* wp = arena;
  unsigned char* const mesh1p = wp;  // overlays region 1 after the gather
  auto take = [&](size_t bytes) {
    unsigned char* q = wp;
    wp += bytes;
    return q;
  };
  float* dinp = reinterpret_cast<float*>(take(b_din));
  uint32_t* keysp = reinterpret_cast<uint32_t*>(take(b_keys));
  uint32_t* idxp = reinterpret_cast<uint32_t*>(take(b_keys));
  float4* fracp = reinterpret_cast<float4*>(take(b_frac));
  float* valsp = reinterpret_cast<float*>(take(b_vals));
  void* sortp = take(b_sort);
  wp = arena + r1;
  uint32_t* skeysp = reinterpret_cast<uint32_t*>(take(b_keys));
  uint32_t* permp = reinterpret_cast<uint32_t*>(take(b_keys));
  uint32_t* cellsp = reinterpret_cast<uint32_t*>(take(b_cells));
  void* scanp = take(b_scan);
  float4* sfracp = reinterpret_cast<float4*>(take(b_frac));
  float* svalsp = reinterpret_cast<float*>(take(b_vals));
  double* partp = reinterpret_cast<double*>(take(b_part));
  int* badp = reinterpret_cast<int*>(take(256));
  const float *dxyz = xyz, *dw = w, *dnb = nbar;
  if (!ptr_is_device && n > 0) {
    float* q = dinp;
    BISP_CUDA(cudaMemcpyAsync(q, xyz, (size_t)n * 12, cudaMemcpyHostToDevice, s));
    dxyz = q;
    q += 3 * n;
    if (w) {
      BISP_CUDA(cudaMemcpyAsync(q, w, (size_t)n * 4, cudaMemcpyHostToDevice, s));
      dw = q;
      q += n;
    }
    if (nbar) {
      BISP_CUDA(cudaMemcpyAsync(q, nbar, (size_t)n * 4, cudaMemcpyHostToDevice, s));
      dnb = q;
    }
  }
  BISP_CUDA(cudaMemsetAsync(badp, 0, sizeof(int), s));
  PrepArgs a{};
  a.xyz = dxyz;
  a.w = dw;
  a.nbar = dnb;
  a.n = n;
  a.N = N;
  a.H = P->H;
  a.box = P->L;
  a.mas = P->mas;
  a.P0 = (float)P->P0;
  a.local = P->los == BISP_LOS_LOCAL;
  for (int k = 0; k < 3; ++k) a.obs[k] = (float)P->obs[k];
  a.nchan = nchan;
  for (int c = 0; c < nchan; ++c) a.chan[c] = ch[c];
  a.ynorm = P->ynorm.as<float>();
  a.keys = keysp;
  a.idx = idxp;
  a.frac = fracp;
  a.vals = valsp;
  a.partials = partp;
  a.nsum = nsum;
  a.bad = badp;
#ifdef BISP_CHECKED
  {
    const char* e = getenv("BISP_CHECK_SELFTEST");
    a.selftest = e && atoi(e) == 1;
  }
#endif
  if (n > 0) {
    launch_prep(a, s);
    ++launches;
  }
  int nbad = 0;
  std::vector<double> hp((size_t)pblk * nsum, 0.0);
  if (n > 0) {
    BISP_CUDA(cudaMemcpyAsync(&nbad, badp, sizeof(int), cudaMemcpyDeviceToHost, s));
    BISP_CUDA(cudaMemcpyAsync(hp.data(), partp, hp.size() * 8, cudaMemcpyDeviceToHost, s));
    BISP_CUDA(cudaStreamSynchronize(s));
  }
  if (nbad) {
    char buf[160];
    snprintf(buf, sizeof buf, "%d particles have non-finite or out-of-box positions", nbad);
    fail(BISP_EINVAL, buf);
  }
  std::vector<double> sums(nsum, 0.0);
  for (int b = 0; b < pblk; ++b)
    for (int q = 0; q < nsum; ++q) sums[q] += hp[(size_t)b * nsum + q];
  if (n > 0 && !(sums[0] > 0.0)) fail(BISP_EINVAL, "total weight must be positive");
  // sort by home cell
  int bits = 0;
  while ((1LL << bits) < Ng) ++bits;
  radix_sort(keysp, idxp, skeysp, permp, n, bits, sortp, s, &launches);
  // cell starts
  uint32_t* counts = cellsp;
  uint32_t* cstart = counts + (Ng + 1);
  BISP_CUDA(cudaMemsetAsync(counts, 0, (size_t)(Ng + 1) * 4, s));
  launch_count_cells(skeysp, n, counts, s);
  ++launches;
  exclusive_scan_u32(counts, cstart, Ng + 1, scanp, s, &launches);
  // particles in sorted order
  launch_gather_particles(permp, n, fracp, valsp, nchan, sfracp, svalsp, s);
  ++launches;
  // deposit onto the meshes; mesh 0 becomes the spectrum storage, mesh 1 overlays region 1
  C.spec.ensure(spec_need, &P->bytes);
  float* mesh1 = ilv ? reinterpret_cast<float*>(mesh1p) : nullptr;
  DepositArgs da{};
  da.cell_start = cstart;
  da.keys = skeysp;
  da.frac = sfracp;
  da.vals = svalsp;
  da.n = n;
  da.N = N;
  da.mas = P->mas;
  da.interlace = ilv;
  da.nchan = nchan;
  da.mesh0 = C.spec.as<float>();
  da.mesh1 = mesh1;
  launch_deposit(da, s, &launches);
  if (P->debug_mesh) {
    C.dbg_mesh.ensure((size_t)nchan * Ng * 4, &P->bytes);
    BISP_CUDA(cudaMemcpyAsync(C.dbg_mesh.p, C.spec.p, (size_t)nchan * Ng * 4, cudaMemcpyDeviceToDevice, s));
  }
  C.sumR3 = 0.0;
  if (which == BISP_RANDOMS) {
    const int nbk = launch_sum_cubes(C.spec.as<float>() + (size_t)P->d00 * Ng, Ng, partp, s);
    ++launches;
    std::vector<double> hr(nbk);
    BISP_CUDA(cudaMemcpyAsync(hr.data(), partp, nbk * 8, cudaMemcpyDeviceToHost, s));
    BISP_CUDA(cudaStreamSynchronize(s));
    for (double v : hr) C.sumR3 += v;
  }
  forward_fft(C.spec.as<float>(), mesh1, nchan, N, P->mas, P->tw.as<float2>(), P->winv.as<float>(), s, &launches);
  BISP_CUDA(cudaEventRecord(P->ev1, s));
  BISP_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  BISP_CUDA(cudaEventElapsedTime(&ms, P->ev0, P->ev1));
  C.ms = ms;
  C.launches = launches;
  C.assigned = true;
  C.n = n;
  C.unit_w = unit_w;
  C.nspec = nchan;
  C.sumw = sums[0];
  C.sbar.assign(sums.begin() + 1, sums.end());
}

// pointer + sign of the N channel c of a catalogue (aliases the D channel when unit weights)
std::pair<const float2*, double> nspec_of(const bisp_plan* P, const Catalog& C, int c) {
  const Chan& n = P->nch[c];
  if (C.unit_w) {
    const int d = P->dchan(n.L, n.M, n.part);
    return {C.spec.as<float2>() + (size_t)d * P->Nk, n.part ? -1.0 : 1.0};
  }
  return {C.spec.as<float2>() + (size_t)(P->dch.size() + c) * P->Nk, 1.0};
}

// ---------------------------------------------------------------------------------
// measure
// ---------------------------------------------------------------------------------
struct PassState {
  std::map<std::pair<int, int>, cplx> sbar;  // (L, M>=0) -> Sbar_L^M
  // Z[(l, m, L, M)] per bin; Zp: the primed sums of the line of sight on x1 or x2
  std::map<std::tuple<int, int, int, int>, std::vector<cplx>> Z, Zp;
};

// pair reduction over the first nbu bins held in the field pool, for the term lists tl (one
// per multipole).  A job whose terms do not fit one contraction launch is split: per G set
// first, then into halves of the multipole list, then a single multipole's terms into halves
// whose results are added in FP64 (a fixed order, so results stay reproducible); the outputs
// keep the layout [gset][mult][b1][b2] of a single launch.
using TermList = std::vector<bisp_plan::Term>;
void run_pair_terms(bisp_plan* P, const std::vector<const TermList*>& tl, int gsets, int gstride, const float* gbase,
                    int nbu, int ncomp, std::vector<double>& out, int* launches) {
  // build a pair job with nout = tl.size() * gsets outputs
  PairJob J{};
  J.fields = P->pool.as<float>();
  J.gfields = gbase;
  J.Ng = P->Ng;
  J.nb = nbu;
  J.ncomp = ncomp;
  J.ng = gsets * gstride;
  J.nout = (int)tl.size() * gsets;
  int t = 0, r = 0;
  bool tables_ok = true;
  for (int gs = 0; gs < gsets && tables_ok; ++gs)
    for (size_t i = 0; i < tl.size() && tables_ok; ++i) {
      const int o = gs * (int)tl.size() + (int)i;
      J.out_term_off[o] = t;
      for (auto& term : *tl[i]) {
        if (t >= 64 || r + (int)(term.x.size() + term.y.size()) > 512) {
          tables_ok = false;
          break;
        }
        J.term[t].xoff = r;
        J.term[t].xcnt = (int)term.x.size();
        for (auto e : term.x) {
          if (e.g >= 0) e.g += gs * gstride;
          J.rec[r++] = e;
        }
        J.term[t].yoff = r;
        J.term[t].ycnt = (int)term.y.size();
        for (auto e : term.y) {
          if (e.g >= 0) e.g += gs * gstride;
          J.rec[r++] = e;
        }
        ++t;
      }
    }
  J.out_term_off[J.nout] = t;
  J.nterm = t;
  J.nrec = r;
  if (!tables_ok || !pair_fits(J)) {
    std::vector<double> part;
    out.clear();
    if (gsets > 1) {
      for (int gs = 0; gs < gsets; ++gs) {
        run_pair_terms(P, tl, 1, gstride, gbase + (size_t)gs * gstride * P->Ng, nbu, ncomp, part, launches);
        out.insert(out.end(), part.begin(), part.end());
      }
      return;
    }
    if (tl.size() > 1) {
      const size_t h = tl.size() / 2;
      run_pair_terms(P, std::vector<const TermList*>(tl.begin(), tl.begin() + h), 1, gstride, gbase, nbu, ncomp,
                     part, launches);
      out.insert(out.end(), part.begin(), part.end());
      run_pair_terms(P, std::vector<const TermList*>(tl.begin() + h, tl.end()), 1, gstride, gbase, nbu, ncomp, part,
                     launches);
      out.insert(out.end(), part.begin(), part.end());
      return;
    }
    if (tl[0]->size() < 2) fail(BISP_EUNSUPPORTED, "a contraction term does not fit one launch");
    const size_t h = tl[0]->size() / 2;
    const TermList lo(tl[0]->begin(), tl[0]->begin() + h), hi(tl[0]->begin() + h, tl[0]->end());
    run_pair_terms(P, {&lo}, 1, gstride, gbase, nbu, ncomp, out, launches);
    run_pair_terms(P, {&hi}, 1, gstride, gbase, nbu, ncomp, part, launches);
    for (size_t i = 0; i < out.size(); ++i) out[i] += part[i];
    return;
  }
  const size_t sb = pair_scratch_bytes(J);
  admit(P, sb > P->pairscr.n ? sb - P->pairscr.n : 0);
  P->pairscr.ensure(sb, &P->bytes);
  const size_t ob = (size_t)J.nout * J.nb * J.nb * 8;
  P->pairout.ensure(ob, &P->bytes);
  NvtxRange nv("contraction (mesh sum of F F G)");
  cudaEvent_t e0, e1;
  BISP_CUDA(cudaEventCreate(&e0));
  BISP_CUDA(cudaEventCreate(&e1));
  pair_reduce(J, P->pairout.as<double>(), P->pairscr.p, P->pairscr.n, P->stream, launches, &P->pair_kernel, e0, e1);
  out.resize((size_t)J.nout * J.nb * J.nb);
  BISP_CUDA(cudaMemcpyAsync(out.data(), P->pairout.p, ob, cudaMemcpyDeviceToHost, P->stream));
  BISP_CUDA(cudaStreamSynchronize(P->stream));
  float ms = 0.f;
  BISP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  P->ms_pair += ms;
  P->pair_launches += 1;
  P->pair_bytes += (double)(J.nb * J.ncomp + J.ng) * (double)P->Ng * 4.0;
}

// inverse-transform a batch of fields (shared prune extent)
void run_inverse(bisp_plan* P, InvBatch& b, int* launches) {
  b.N = P->N;
  b.ynorm = P->ynorm.as<float>();
  b.cw2_1d = P->cw2.as<float>();
  b.interlace = P->interlace;
  b.err = P->flags.as<int>();
  b.stall = inject_stall("zpass") ? 1 : 0;
  b.zgroups = P->zgroups;
  const size_t need = inverse_scratch_bytes(P->N, b.P, b.nf);
  if (need > P->invscr.n) {
    admit(P, need - P->invscr.n);
    P->invscr.ensure(need, &P->bytes);
  }
  inverse_fft(b, P->tw.as<float2>(), P->invscr.p, P->stream, launches);
}

// Autotuner of the inverse transforms' z pass: the number of 16-row groups a CTA takes (more
// groups share one twiddle-table setup and prefetch pipeline; fewer give more CTAs).  Every value
// computes the same fields bit for bit, so the choice only moves time.  The plan times its
// largest shell batch (the costliest prune extent) once with each candidate and keeps the
// fastest; the choice is cached per (N, prune extent, batch width) for every plan of the process.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune_cache;

void tune_zgroups(bisp_plan* P, InvBatch& b, int* launches) {
  const char* e = getenv("BISP_ZGROUPS");  // fixed value (tests, comparisons): no timing
  if (e && atoi(e) > 0) {
    P->zgroups = inverse_zgroups(P->N, atoi(e));
    run_inverse(P, b, launches);
    return;
  }
  const auto key = std::make_tuple(P->N, b.P, b.nf);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      P->zgroups = it->second;
      run_inverse(P, b, launches);
      return;
    }
  }
  cudaEvent_t e0, e1;
  BISP_CUDA(cudaEventCreate(&e0));
  BISP_CUDA(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 0.f;
  std::vector<int> tried;
  P->tune_log.clear();
  for (int cand : {1, 2, 4, 8, 16, 32}) {
    const int g = inverse_zgroups(P->N, cand);
    if (std::find(tried.begin(), tried.end(), g) != tried.end()) continue;
    tried.push_back(g);
    P->zgroups = g;
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {  // the first run warms the caches and the module
      BISP_CUDA(cudaEventRecord(e0, P->stream));
      run_inverse(P, b, launches);
      BISP_CUDA(cudaEventRecord(e1, P->stream));
      BISP_CUDA(cudaEventSynchronize(e1));
      BISP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    }
    P->tune_log.push_back({g, ms});
    if (!best || ms < best_ms) {
      best = g;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  P->zgroups = best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = best;
}

// shell fields of bins [b0, b1) into the pool, bin b at pool bin slot b - b0 + slot; Dp: the
// pass's delta n channel spectra (nullptr for unit shells)
void shell_fields(bisp_plan* P, const float2* Dp, bool unit, int b0, int b1, int slot, int* launches) {
  NvtxRange nv(unit ? "unit-shell fields" : "shell-filtered fields");
  const int nc = (int)P->comps.size();
  const int stride = P->pass_ncomp(unit);
  const float2* D00 = Dp ? Dp + (size_t)P->d00 * P->Nk : nullptr;
  if (P->estimator == BISP_THREEPT) {
    // per r-bin: the separation kernels of its nc components, their forward FFT (no
    // deconvolution), then the full inverse transforms of conj(K) Delta
    const size_t kb = (size_t)nc * P->Ng * 4;
    P->kmesh.ensure(kb, &P->bytes);
    for (int b = b0; b < b1; ++b) {
      BISP_CUDA(cudaMemsetAsync(P->kmesh.p, 0, kb, P->stream));
      RKernelArgs ka{};
      ka.N = P->N;
      ka.nc = nc;
      for (int c = 0; c < nc; ++c) {
        ka.l[c] = P->comps[c].l;
        ka.m[c] = P->comps[c].m;
        ka.part[c] = P->comps[c].part;
      }
      ka.n = P->roff_off[b + 1] - P->roff_off[b];
      ka.inv_nr = ka.n > 0 ? (float)(1.0 / (double)ka.n) : 0.f;
      ka.offs = P->roff_d.as<uint32_t>() + P->roff_off[b];
      ka.ynorm = P->ynorm.as<float>();
      ka.mesh = P->kmesh.as<float>();
      launch_rshell_kernel(ka, P->stream);
      *launches += ka.n > 0 ? 1 : 0;
      forward_fft(P->kmesh.as<float>(), nullptr, nc, P->N, P->mas, P->tw.as<float2>(), P->ones.as<float>(), P->stream,
                  launches);
      InvBatch B{};
      B.P = P->N / 2 - 1;
      B.nf = nc;
      for (int c = 0; c < nc; ++c) {
        InvField& f = B.f[c];
        f.kind = SRC_KERNEL;
        f.A = D00;
        f.K = reinterpret_cast<const float2*>(P->kmesh.as<float>() + (size_t)c * P->Ng);
        f.l = P->comps[c].l;
        f.m = P->comps[c].m;
        f.part = P->comps[c].part;
        f.unit = unit ? 1 : 0;
        f.scale = 1.f;
        f.out = P->pool.as<float>() + ((size_t)(b - b0 + slot) * nc + c) * P->Ng;
      }
      run_inverse(P, B, launches);
    }
    return;
  }
  for (int b = b0; b < b1; ++b) {
    InvBatch B{};
    B.P = P->Pb[b];
    B.nf = nc;
    B.qlo = P->qlo[b];
    B.qhi = P->qhi[b];
    B.inv_nmodes = P->nmodes[b] > 0 ? (float)(1.0 / P->nmodes[b]) : 0.f;
    for (int c = 0; c < nc; ++c) {
      InvField& f = B.f[c];
      f.kind = SRC_SHELL;
      f.A = D00;
      f.l = P->comps[c].l;
      f.m = P->comps[c].m;
      f.part = P->comps[c].part;
      f.unit = unit ? 1 : 0;
      f.scale = 1.f;
      f.out = P->pool.as<float>() + ((size_t)(b - b0 + slot) * stride + c) * P->Ng;
    }
    // the first shell batch of the largest prune extent tunes the z pass (and computes the fields)
    if (!P->zgroups && P->Pb[b] == *std::max_element(P->Pb.begin(), P->Pb.end()))
      tune_zgroups(P, B, launches);
    else
      run_inverse(P, B, launches);
    // line of sight on x1 or x2: the k-space contractions over the weighted object's (m, M)
    const int nk = stride - nc;
    for (int k0 = 0; k0 < nk; k0 += 32) {
      InvBatch K{};
      K.P = P->Pb[b];
      K.nf = std::min(32, nk - k0);
      K.qlo = P->qlo[b];
      K.qhi = P->qhi[b];
      K.inv_nmodes = B.inv_nmodes;
      for (size_t ch = 0; ch < P->dch.size() && ch < 16; ++ch) K.spec[ch] = Dp + ch * P->Nk;
      for (int j = 0; j < K.nf; ++j) {
        const bisp_plan::KField& kf = P->kfields[k0 + j];
        InvField& f = K.f[j];
        f.kind = SRC_SHELL_SUM;
        f.l = kf.l;
        f.ne = (int)kf.ent.size();
        for (int q = 0; q < f.ne && q < INV_MAXE; ++q) {
          f.ecoef[q] = std::get<0>(kf.ent[q]);
          f.em[q] = (signed char)std::get<1>(kf.ent[q]);
          f.epart[q] = (signed char)std::get<2>(kf.ent[q]);
          f.espec[q] = (signed char)std::get<3>(kf.ent[q]);
        }
        f.out = P->pool.as<float>() + ((size_t)(b - b0 + slot) * stride + nc + k0 + j) * P->Ng;
      }
      run_inverse(P, K, launches);
    }
  }
}

// Shell fields of one set (unit shells, data or window) and their pair reductions, out laid
// out [gset][mult][b1][b2].  When the pool holds fewer than n_b bins (nbk < n_b), the bins are
// taken in blocks of nbk: block I sits in the pool's first slots and block J > I after it, and
// one pair launch covers their union; a pair (b1, b2) is kept from exactly one union (cross
// pairs from (I, J), a block's own pairs from (I, I + 1), the last block's from the last union).
void pair_set(bisp_plan* P, const float2* Dp, bool unit, int gsets, const float* gbase, int nbk,
              std::vector<double>& out, int* launches) {
  const float2* D00 = Dp;  // shell_fields takes the pass's channel spectra
  const int nb = P->nb, nmult = P->nmult, nD = (int)P->dch.size();
  std::vector<int> all(nmult);
  for (int i = 0; i < nmult; ++i) all[i] = i;
  std::vector<const TermList*> tl;
  const bool kt = !unit && P->los_obj != 3;
  for (int i : all) tl.push_back(kt ? &P->kterms[i] : &P->terms[i]);
  const int ncomp = P->pass_ncomp(unit);
  auto pairs = [&](int nbu, std::vector<double>& res) {
    if (gsets > 1 && pair_split_gsets()) {
      // one launch per G set: outputs [gset][mult][b1][b2] as with a single launch
      res.clear();
      for (int gs = 0; gs < gsets; ++gs) {
        std::vector<double> part;
        run_pair_terms(P, tl, 1, nD, gbase + (size_t)gs * nD * P->Ng, nbu, ncomp, part, launches);
        res.insert(res.end(), part.begin(), part.end());
      }
    } else {
      run_pair_terms(P, tl, gsets, nD, gbase, nbu, ncomp, res, launches);
    }
  };
  if (nbk >= nb) {
    shell_fields(P, D00, unit, 0, nb, 0, launches);
    pairs(nb, out);
    return;
  }
  const int nout = gsets * nmult, nblocks = (nb + nbk - 1) / nbk;
  out.assign((size_t)nout * nb * nb, 0.0);
  std::vector<double> res;
  if (P->diagonal) {  // every block alone: its own pairs hold the diagonal
    for (int I = 0; I < nblocks; ++I) {
      const int i0 = I * nbk, ni = std::min(nbk, nb - i0);
      shell_fields(P, D00, unit, i0, i0 + ni, 0, launches);
      pairs(ni, res);
      for (int o = 0; o < nout; ++o)
        for (int u = 0; u < ni; ++u)
          out[((size_t)o * nb + i0 + u) * nb + i0 + u] = res[((size_t)o * ni + u) * ni + u];
    }
    return;
  }
  for (int I = 0; I + 1 < nblocks; ++I) {
    const int i0 = I * nbk, ni = std::min(nbk, nb - i0);
    shell_fields(P, D00, unit, i0, i0 + ni, 0, launches);
    for (int J = I + 1; J < nblocks; ++J) {
      const int j0 = J * nbk, nj = std::min(nbk, nb - j0), nbu = ni + nj;
      shell_fields(P, D00, unit, j0, j0 + nj, ni, launches);
      pairs(nbu, res);
      const bool own_i = J == I + 1, own_j = J == nblocks - 1 && I == nblocks - 2;
      for (int o = 0; o < nout; ++o)
        for (int u1 = 0; u1 < nbu; ++u1)
          for (int u2 = 0; u2 < nbu; ++u2) {
            const bool in1 = u1 < ni, in2 = u2 < ni;
            if (in1 == in2 && !(in1 ? own_i : own_j)) continue;
            const int b1 = in1 ? i0 + u1 : j0 + u1 - ni, b2 = in2 ? i0 + u2 : j0 + u2 - ni;
            out[((size_t)o * nb + b1) * nb + b2] = res[((size_t)o * nbu + u1) * nbu + u2];
          }
    }
  }
}

// Bins per resident block of FP32 shell fields: all n_b when they fit and n_b <= 32 (a pair
// launch covers at most 32 bins), else blocks of at most 16 with two resident.  other_need is
// the device memory the measurement still has to allocate besides the pool.
// BISP_BLOCK_BINS=n in the environment caps the block at n bins (tests of the blocking).
int fp32_block_bins(bisp_plan* P, size_t other_need) {
  const size_t per_bin = (size_t)P->pass_ncomp(false) * (size_t)P->Ng * 4;
  size_t fre = 0, tot = 0;
  BISP_CUDA(cudaMemGetInfo(&fre, &tot));
  const size_t reserve = (size_t)2 << 30;
  const size_t movable = P->pool.n + P->ws.n;  // the pool is re-sized, the arena released
  size_t cap = (fre > reserve ? fre - reserve : 0) + movable;
  cap = cap > other_need ? cap - other_need : 0;
  if (P->max_bytes) {
    const size_t held = P->bytes - movable + other_need;
    cap = std::min(cap, P->max_bytes > held ? P->max_bytes - held : 0);
  }
  const char* env = std::getenv("BISP_BLOCK_BINS");
  const int force = env ? std::atoi(env) : 0;
  if (P->nb <= 32 && (size_t)P->nb * per_bin <= cap && (force <= 0 || force >= P->nb)) return P->nb;
  // diagonal outputs only: one block resident, up to the 32 bins of a pair launch
  int nbk = P->diagonal ? (int)std::min<size_t>(32, cap / per_bin) : (int)std::min<size_t>(16, cap / (2 * per_bin));
  if (force > 0) nbk = std::min(nbk, force);
  if (nbk < 1) {
    char buf[200];
    snprintf(buf, sizeof buf, "admission: two bins of shell fields need %.3f GB, %.3f GB available",
             2.0 * per_bin / 1e9, cap / 1e9);
    fail(BISP_ENOMEM, buf);
  }
  return std::min(nbk, P->nb);
}

// ---------------------------------------------------------------------------------
// plain FP64 form (precision BISP_FP64): full cuFFT Z2D transforms of FP64 half
// spectra, one FP64 mesh sum per (bin pair, 3j term), nothing fused
// ---------------------------------------------------------------------------------
constexpr int F64_MAX_PENDING = 4096;  // mesh sums per partials buffer

void f64_field(bisp_plan* P, const F64Spec& sp, double* out, int* launches) {
  const F64Tables t{P->ynorm_d.as<double>(), P->cw2_d.as<double>(), P->interlace};
  f64_spectrum(sp, t, P->N, P->f64spec.as<double2>(), P->stream);
  f64_fft_c2r(P->fft64, P->f64work.p, P->f64spec.as<double2>(), out, P->stream);
  *launches += 2;
}

// shell fields of bins [b0, b1), component c of bin b at dst + ((b - b0) * ncomp + c) * Ng
void f64_shells(bisp_plan* P, const float2* D00, bool unit, int b0, int b1, double* dst, int* launches) {
  const int nc = (int)P->comps.size();
  for (int b = b0; b < b1; ++b)
    for (int c = 0; c < nc; ++c) {
      F64Spec sp{};
      sp.kind = SRC_SHELL;
      sp.A = D00;
      sp.unit = unit ? 1 : 0;
      sp.l = P->comps[c].l;
      sp.m = P->comps[c].m;
      sp.part = P->comps[c].part;
      sp.qlo = P->qlo[b];
      sp.qhi = P->qhi[b];
      sp.inv_nmodes = P->nmodes[b] > 0 ? 1.0 / P->nmodes[b] : 0.0;
      sp.scale = 1.0;
      f64_field(P, sp, dst + ((size_t)(b - b0) * nc + c) * P->Ng, launches);
    }
}

// out[((gs * nmult + mu) * nb + b1) * nb + b2] = sum over the terms of multipole mu of
// coef * sum_x F_c1(x; b1) F_c2(x; b2) G_{gs, g}(x).  Shell fields are held for two blocks
// of nbk bins at a time (one block when every bin fits) and recomputed per block pair.
void f64_pairs(bisp_plan* P, const float2* D00, bool unit, const double* gbase, int gsets, int nbk,
               std::vector<double>& out, int* launches) {
  const int nb = P->nb, nmult = P->nmult, nc = (int)P->comps.size(), nD = (int)P->dch.size();
  const int64_t Ng = P->Ng;
  out.assign((size_t)gsets * nmult * nb * nb, 0.0);
  const size_t fb = (size_t)nc * Ng;
  double* slotA = P->f64shell.as<double>();
  double* slotB = slotA + (size_t)nbk * fb;
  const int nblk = f64_dot_blocks();
  struct Pend {
    size_t o;
    double coef;
  };
  std::vector<Pend> pend;
  cudaEvent_t e0, e1;
  BISP_CUDA(cudaEventCreate(&e0));
  BISP_CUDA(cudaEventCreate(&e1));
  auto flush = [&]() {
    if (pend.empty()) return;
    f64_dot_final(P->f64part.as<double>(), nblk, (int)pend.size(), P->f64out.as<double>(), P->stream);
    ++*launches;
    BISP_CUDA(cudaEventRecord(e1, P->stream));
    std::vector<double> v(pend.size());
    BISP_CUDA(cudaMemcpyAsync(v.data(), P->f64out.p, v.size() * 8, cudaMemcpyDeviceToHost, P->stream));
    BISP_CUDA(cudaStreamSynchronize(P->stream));
    float ms = 0.f;
    BISP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    P->ms_pair += ms;
    for (size_t i = 0; i < pend.size(); ++i) out[pend[i].o] += pend[i].coef * v[i];
    pend.clear();
  };
  auto dot = [&](const double* a, const double* b, const double* g, size_t o, double coef) {
    if (pend.empty()) BISP_CUDA(cudaEventRecord(e0, P->stream));
    f64_dot3(a, b, g, Ng, P->f64part.as<double>() + pend.size() * nblk, nblk, P->stream);
    ++*launches;
    P->pair_launches += 1;
    P->pair_bytes += 3.0 * 8.0 * (double)Ng;
    pend.push_back({o, coef});
    if ((int)pend.size() == F64_MAX_PENDING) flush();
  };
  const int nblocks = (nb + nbk - 1) / nbk;
  for (int I = 0; I < nblocks; ++I) {
    const int i0 = I * nbk, i1 = std::min(nb, i0 + nbk);
    f64_shells(P, D00, unit, i0, i1, slotA, launches);
    for (int J = I; J < nblocks; ++J) {
      const int j0 = J * nbk, j1 = std::min(nb, j0 + nbk);
      if (J != I) f64_shells(P, D00, unit, j0, j1, slotB, launches);
      auto field = [&](int b, int c) -> const double* {
        if (b >= i0 && b < i1) return slotA + (size_t)(b - i0) * fb + (size_t)c * Ng;
        return slotB + (size_t)(b - j0) * fb + (size_t)c * Ng;
      };
      auto pair = [&](int b1, int b2) {
        if (P->diagonal && b1 != b2) return;
        for (int gs = 0; gs < gsets; ++gs)
          for (int mu = 0; mu < nmult; ++mu)
            for (const auto& t : P->tri64[mu])
              dot(field(b1, t.c1), field(b2, t.c2), gbase + ((size_t)gs * nD + t.g) * Ng,
                  (((size_t)gs * nmult + mu) * nb + b1) * nb + b2, t.coef);
      };
      for (int b1 = i0; b1 < i1; ++b1)
        for (int b2 = j0; b2 < j1; ++b2) {
          pair(b1, b2);
          if (J != I) pair(b2, b1);
        }
      flush();
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  P->pair_kernel = 3;
}

// bins per resident block of FP64 shell fields: every bin if they fit, else what two
// blocks fit in the device memory left (free memory minus a reserve, or the plan's cap)
int f64_block_bins(bisp_plan* P) {
  const size_t per_bin = P->comps.size() * (size_t)P->Ng * 8;
  size_t fre = 0, tot = 0;
  BISP_CUDA(cudaMemGetInfo(&fre, &tot));
  const size_t reserve = (size_t)2 << 30;
  size_t cap = (fre > reserve ? fre - reserve : 0) + P->f64shell.n;
  if (P->max_bytes) {
    const size_t held = P->bytes - P->f64shell.n;
    cap = std::min(cap, P->max_bytes > held ? P->max_bytes - held : 0);
  }
  // BISP_FP64_BLOCK_BINS=n in the environment caps the block at n bins (tests of the blocking)
  const char* env = std::getenv("BISP_FP64_BLOCK_BINS");
  const int force = env ? std::atoi(env) : 0;
  if ((size_t)P->nb * per_bin <= cap && (force <= 0 || force >= P->nb)) return P->nb;
  int nbk = (int)std::min<size_t>(P->nb, cap / (2 * per_bin));
  if (force > 0) nbk = std::min(nbk, force);
  if (nbk < 1) {
    char buf[200];
    snprintf(buf, sizeof buf, "admission: FP64 shell fields need %.3f GB, %.3f GB available", 2.0 * per_bin / 1e9,
             cap / 1e9);
    fail(BISP_ENOMEM, buf);
  }
  return nbk;
}

// Three-point function (Sec. 4.3, Eq. reduced_xi_estimator): zeta = (N H / I) raw / (Ng V^2)
// from the mesh sums of unnormalised c2r fields, and on r_a = r_b the i = j != k term
// (N H / I) sum 3j (1/N_r^2) sum_{s in a} y_{l1}^{m1*} y_{l2}^{m2*}(s_hat) (Ng / V^2) q_L^M(-s),
// q the unnormalised c2r of Q_L^M = delta n_L^M N_0^{0*} - Sbar_L^M C/W^2 (FP64 on the host).
void threept_combine(bisp_plan* P, int npass, const std::vector<double>& cD, const std::vector<double>& cW,
                     const std::vector<float>* gq, double* outB, double* outShot, double* outW, double* outWS,
                     double* outNm) {
  const int nb = P->nb, nmult = P->nmult, nD = (int)P->dch.size();
  const bool local = P->los == BISP_LOS_LOCAL;
  const double Ngd = (double)P->Ng, V2 = P->V * P->V;
  const int64_t noff = (int64_t)P->roff.size();
  const int lmax = P->ls.empty() ? 0 : P->ls.back();
  // y_l^{m*}(s_hat) of every separation, m signed, at [l^2 + m + l][offset]
  std::vector<std::vector<cplx>> ys((lmax + 1) * (lmax + 1));
  for (int l : P->ls)
    for (int m = -l; m <= l; ++m) {
      auto& t = ys[P->lm_index(l, m)];
      t.resize(noff);
      for (int64_t i = 0; i < noff; ++i) {
        const uint32_t o = P->roff[i];
        const double sx = (double)((int)(o & 1023u) - 512), sy = (double)((int)((o >> 10) & 1023u) - 512),
                     sz = (double)((int)((o >> 20) & 1023u) - 512);
        ystar_host(l, m, sx, sy, sz, &t[i].r, &t[i].i);
      }
    }
  for (int k = 0; k < npass; ++k) {
    const std::vector<double>& raw = k == 0 ? cD : cW;
    const std::vector<float>& g = gq[k];
    double* oB = k == 0 ? outB : outW;
    double* oS = k == 0 ? outShot : outWS;
    for (int mu = 0; mu < nmult; ++mu) {
      const int l1 = P->ells[mu][0], l2 = P->ells[mu][1], L = P->ells[mu][2];
      const double pref = (double)((2 * l1 + 1) * (2 * l2 + 1) * (2 * L + 1)) * wigner3j(l1, l2, L, 0, 0, 0) / P->normI;
      for (int a = 0; a < nb; ++a) {
        double shot = 0.0;
        if (P->nmodes[a] > 0) {
          double acc = 0.0;
          for (int m1 = -l1; m1 <= l1; ++m1)
            for (int m2 = -l2; m2 <= l2; ++m2) {
              const int M = -m1 - m2;
              if (std::abs(M) > L || (!local && M != 0)) continue;
              const double w = wigner3j(l1, l2, L, m1, m2, M);
              if (w == 0.0) continue;
              const int Lz = local ? L : 0, aM = std::abs(M);
              const int cr = P->dchan(Lz, aM, 0), ci = aM ? P->dchan(Lz, aM, 1) : -1;
              const double sg = (M < 0 && (aM & 1)) ? -1.0 : 1.0;  // q^{-M} = (-1)^M conj(q^M)
              const auto& y1 = ys[P->lm_index(l1, m1)];
              const auto& y2 = ys[P->lm_index(l2, m2)];
              for (int64_t i = P->roff_off[a]; i < P->roff_off[a + 1]; ++i) {
                const double qr = sg * g[(size_t)i * nD + cr];
                const double qi = ci >= 0 ? (M < 0 ? -sg : sg) * g[(size_t)i * nD + ci] : 0.0;
                const cplx yy = cm(y1[i], y2[i]);
                acc += w * (yy.r * qr - yy.i * qi);
              }
            }
          shot = pref * acc * Ngd / V2 / (P->nmodes[a] * P->nmodes[a]);
        }
        for (int b = 0; b < nb; ++b) {
          const size_t o = ((size_t)mu * nb + a) * nb + b;
          const double s_ab = a == b ? shot : 0.0;
          const double z = pref * raw[(size_t)mu * nb * nb + (size_t)a * nb + b] / (Ngd * V2);
          const bool off = P->diagonal && a != b;  // not computed
          if (oB) oB[o] = off ? NAN : z - s_ab;
          if (oS) oS[o] = off ? NAN : s_ab;
        }
      }
    }
  }
  if (outNm)
    for (int a = 0; a < nb; ++a) outNm[a] = P->nmodes[a];
}

void do_measure(bisp_plan* P, double* outB, double* outShot, double* outW, double* outWS, double* outNm) {
  NvtxRange nv("bisp_measure");
  Catalog& G = P->cat[BISP_DATA];
  Catalog& R = P->cat[BISP_RANDOMS];
  if (!G.assigned) fail(BISP_ESTATE, "measure before the data catalogue was assigned");
  const bool local = P->los == BISP_LOS_LOCAL;
  if ((local || P->want_window) && !R.assigned) fail(BISP_ESTATE, "this plan needs the random catalogue");
  if (P->want_window && (outW || outWS) && !R.assigned) fail(BISP_ESTATE, "window needs randoms");
  cudaStream_t s = P->stream;
  int launches = 0;
  P->ms_pair = 0.0;
  P->pair_launches = 0;
  P->pair_bytes = 0.0;
  BISP_CUDA(cudaEventRecord(P->ev0, s));
  P->flags.ensure(256, &P->bytes);
  BISP_CUDA(cudaMemsetAsync(P->flags.p, 0, 256, s));
  const int nD = (int)P->dch.size(), nN = (int)P->nch.size();
  const int64_t Ng = P->Ng, Nk = P->Nk;
  const bool have_r = R.assigned;
  const double alpha = have_r ? G.sumw / R.sumw : 0.0;
  P->alpha = alpha;
  // normalisation I (Eq. normalization): alpha^3 sum R^3 / H^6, or Np^3 / V^2 for a box
  if (have_r) P->normI = alpha * alpha * alpha * R.sumR3 / std::pow(P->H, 6);
  else P->normI = G.sumw * G.sumw * G.sumw / (P->V * P->V);
  const int npass = (P->want_window && have_r) ? 2 : 1;
  const int nb = P->nb, nmult = P->nmult;
  const bool f64 = P->precision == BISP_FP64;
  const bool three = P->estimator == BISP_THREEPT;
  int nbk = nb;  // bins per resident block of FP32 shell fields
  // memory admission for the measurement buffers
  {
    size_t need = 0;
    auto add = [&](DBuf& d, size_t b) { need += b > d.n ? b - d.n : 0; };
    for (int k = 0; k < npass; ++k) {
      add(P->pass_spec[k], (size_t)(nD + nN) * Nk * 8);
      if (!f64) add(P->gf[k], (size_t)nD * Ng * 4);
    }
    if (three) add(P->kmesh, P->comps.size() * (size_t)Ng * 4);
    if (!f64) {
      add(P->qf, (size_t)npass * nD * Ng * 4);
      // inverse-transform scratch still to grow (G and Q batches, the widest shell batch)
      const int pmax = *std::max_element(P->Pb.begin(), P->Pb.end());
      const size_t inv = std::max(inverse_scratch_bytes(P->N, P->N / 2 - 1, nD),
                                  inverse_scratch_bytes(P->N, pmax, (int)P->comps.size()));
      nbk = fp32_block_bins(P, need + (inv > P->invscr.n ? inv - P->invscr.n : 0));
      const size_t pool_need = (size_t)(nbk == nb || P->diagonal ? nbk : 2 * nbk) * P->pass_ncomp(false) * Ng * 4;
      // the assignment arena moves into the pool from now on: free it before admission
      if (pool_need > P->pool.n) P->ws.release(&P->bytes);
      add(P->pool, pool_need);
    } else {
      P->ws.release(&P->bytes);
      add(P->f64spec, (size_t)P->N * P->N * (P->N / 2 + 1) * 16);
      add(P->f64work, P->fft64.work_bytes);
      add(P->f64g, (size_t)npass * nD * Ng * 8);
      add(P->f64q, (size_t)npass * nD * Ng * 8);
      add(P->f64part, (size_t)F64_MAX_PENDING * f64_dot_blocks() * 8);
      add(P->f64out, (size_t)F64_MAX_PENDING * 8);
      add(P->f64shell, 2 * P->comps.size() * (size_t)Ng * 8);
    }
    admit(P, need);
  }
  if (f64) {
    P->f64spec.ensure((size_t)P->N * P->N * (P->N / 2 + 1) * 16, &P->bytes);
    P->f64work.ensure(std::max<size_t>(P->fft64.work_bytes, 256), &P->bytes);
    P->f64g.ensure((size_t)npass * nD * Ng * 8, &P->bytes);
    P->f64q.ensure((size_t)npass * nD * Ng * 8, &P->bytes);
    P->f64part.ensure((size_t)F64_MAX_PENDING * f64_dot_blocks() * 8, &P->bytes);
    P->f64out.ensure((size_t)F64_MAX_PENDING * 8, &P->bytes);
  }
  PassState ps[2];
  for (int k = 0; k < npass; ++k) {
    const bool win = k == 1;
    P->pass_spec[k].ensure((size_t)(nD + nN) * Nk * 8, &P->bytes);
    float2* Dp = P->pass_spec[k].as<float2>();
    float2* Np = Dp + (size_t)nD * Nk;
    const float2* Dg = G.spec.as<float2>();
    const float2* Dr = have_r ? R.spec.as<float2>() : nullptr;
    for (int c = 0; c < nD; ++c) {
      if (!win) {
        if (have_r)
          launch_axpby(Dp + c * Nk, Dg + c * Nk, 1.0, Dr + c * Nk, -alpha, Nk, 1, s);
        else
          launch_axpby(Dp + c * Nk, Dg + c * Nk, 1.0, nullptr, 0.0, Nk, 1, s);
      } else {
        launch_axpby(Dp + c * Nk, Dr + c * Nk, alpha, nullptr, 0.0, Nk, 0, s);
      }
      ++launches;
    }
    for (int c = 0; c < nN; ++c) {
      auto ng = nspec_of(P, G, c);
      if (!win) {
        if (have_r) {
          auto nr = nspec_of(P, R, c);
          launch_axpby(Np + c * Nk, ng.first, ng.second, nr.first, alpha * alpha * nr.second, Nk, 0, s);
        } else {
          launch_axpby(Np + c * Nk, ng.first, ng.second, nullptr, 0.0, Nk, 0, s);
        }
      } else {
        auto nr = nspec_of(P, R, c);
        launch_axpby(Np + c * Nk, nr.first, alpha * alpha * nr.second, nullptr, 0.0, Nk, 0, s);
      }
      ++launches;
    }
    // Sbar_L^M per (L, M >= 0)
    for (int L : P->Ls)
      for (int M = 0; M <= L; ++M) {
        if (!local && (L > 0 || M > 0)) continue;
        const int cr = P->dchan(L, M, 0), ci = M ? P->dchan(L, M, 1) : -1;
        auto sb = [&](const Catalog& C) {
          return cplx{C.sbar[cr], ci >= 0 ? C.sbar[ci] : 0.0};
        };
        cplx v;
        if (!win) {
          v = sb(G);
          if (have_r) {
            const cplx r = sb(R);
            v.r -= alpha * alpha * alpha * r.r;
            v.i -= alpha * alpha * alpha * r.i;
          }
        } else {
          const cplx r = sb(R);
          v = {alpha * alpha * alpha * r.r, alpha * alpha * alpha * r.i};
        }
        ps[k].sbar[{L, M}] = v;
      }
    // G fields: c2r of each delta n channel
    if (f64) {
      for (int c = 0; c < nD; ++c) {
        F64Spec sp{};
        sp.kind = SRC_PLAIN;
        sp.A = Dp + c * Nk;
        sp.scale = 1.0;
        f64_field(P, sp, P->f64g.as<double>() + ((size_t)k * nD + c) * Ng, &launches);
      }
      for (int c = 0; c < nD; ++c) {
        const Chan& ch = P->dch[c];
        const cplx sbv = ps[k].sbar.at({local ? ch.L : 0, local ? ch.M : 0});
        F64Spec sp{};
        sp.kind = SRC_QSHOT;
        sp.A = Dp + c * Nk;
        sp.B = Np + (size_t)P->n00 * Nk;
        sp.sbar = ch.part ? sbv.i : sbv.r;
        sp.scale = 1.0;
        f64_field(P, sp, P->f64q.as<double>() + ((size_t)k * nD + c) * Ng, &launches);
      }
    } else {
      P->gf[k].ensure((size_t)nD * Ng * 4, &P->bytes);
      P->qf.ensure((size_t)npass * nD * Ng * 4, &P->bytes);
      {
        InvBatch B{};
        B.P = P->N / 2 - 1;
        B.nf = nD;
        for (int c = 0; c < nD; ++c) {
          B.f[c].kind = SRC_PLAIN;
          B.f[c].A = Dp + c * Nk;
          B.f[c].scale = 1.f;
          B.f[c].out = P->gf[k].as<float>() + (size_t)c * Ng;
        }
        run_inverse(P, B, &launches);
        // q fields: c2r of D_c conj(N_00) - Sbar_part C/W^2
        InvBatch Q{};
        Q.P = P->N / 2 - 1;
        Q.nf = nD;
        for (int c = 0; c < nD; ++c) {
          const Chan& ch = P->dch[c];
          const cplx sbv = ps[k].sbar.at({local ? ch.L : 0, local ? ch.M : 0});
          Q.f[c].kind = SRC_QSHOT;
          Q.f[c].A = Dp + c * Nk;
          Q.f[c].B = Np + (size_t)P->n00 * Nk;
          Q.f[c].sbar = (float)(ch.part ? sbv.i : sbv.r);
          Q.f[c].scale = 1.f;
          if (local && P->los_obj != 3) {
            // the distinct object is unweighted, the coincident pair carries y_L^M (App. B):
            // Q = delta n_0^0 conj(N_L^M) - Sbar_L^M C/W^2, N_L^M = N_R + i N_I in real channels
            Q.f[c].A = Dp + (size_t)P->d00 * Nk;
            Q.f[c].B = Np + (size_t)P->nchan(ch.L, ch.M, ch.part) * Nk;
            Q.f[c].scale = ch.part ? -1.f : 1.f;
            Q.f[c].sbar = (float)(ch.part ? -sbv.i : sbv.r);
          }
          Q.f[c].out = P->qf.as<float>() + ((size_t)k * nD + c) * Ng;
        }
        run_inverse(P, Q, &launches);
      }
    }
    // shell sums Z(b; l, m, L, M) for M >= 0 (FP64; the bispectrum's i != j = k, i = k != j)
    if (!three) {
      std::vector<std::pair<int, int>> lm;
      for (int l : P->ls)
        for (int m = -l; m <= l; ++m) lm.push_back({l, m});
      const int nblk = 64;
      // primed: the distinct object carries y_L^{M*} and the pair is unweighted (line of sight on
      // x1 or x2, App. B), Z' = avg y_l^{m*} [delta n_L^M conj(N_0^0) - Sbar_L^M C/W^2]
      const int nkind = (local && P->los_obj != 3) ? 2 : 1;
      for (int kind = 0; kind < nkind; ++kind)
      for (int L : P->Ls)
        for (int M = 0; M <= L; ++M) {
          if (!local && (L > 0 || M > 0)) continue;
          const cplx sbv = ps[k].sbar.at({L, M});
          for (size_t g0 = 0; g0 < lm.size(); g0 += 9) {
            const int cnt = (int)std::min<size_t>(9, lm.size() - g0);
            ZsumArgs z{};
            if (kind == 0) {
              z.XR = Dp + (size_t)P->d00 * Nk;
              z.XI = nullptr;
              const int cr = P->nchan(L, M, 0), ci = M ? P->nchan(L, M, 1) : -1;
              z.NR = Np + (size_t)cr * Nk;
              z.NI = ci >= 0 ? Np + (size_t)ci * Nk : nullptr;
            } else {
              const int dr = P->dchan(L, M, 0), di = M ? P->dchan(L, M, 1) : -1;
              z.XR = Dp + (size_t)dr * Nk;
              z.XI = di >= 0 ? Dp + (size_t)di * Nk : nullptr;
              z.NR = Np + (size_t)P->n00 * Nk;
              z.NI = nullptr;
            }
            z.sbar_re = sbv.r;
            z.sbar_im = sbv.i;
            z.N = P->N;
            z.nbins = nb;
            z.modes = P->zmodes.as<uint32_t>();
            z.mode_off = P->zmode_off.as<int64_t>();
            z.cw2_1d = P->cw2.as<float>();
            z.interlace = P->interlace;
            z.nlm = cnt;
            for (int t = 0; t < cnt; ++t) {
              z.lm[t][0] = lm[g0 + t].first;
              z.lm[t][1] = lm[g0 + t].second;
            }
            z.ynorm = P->ynorm.as<float>();
            z.nblk = nblk;
            const size_t zb = (size_t)nb * nblk * cnt * 2 * 8;
            P->zpart.ensure(zb, &P->bytes);
            z.partials = P->zpart.as<double>();
            launch_zsum(z, s);
            ++launches;
            std::vector<double> hz((size_t)nb * nblk * cnt * 2);
            BISP_CUDA(cudaMemcpyAsync(hz.data(), P->zpart.p, zb, cudaMemcpyDeviceToHost, s));
            BISP_CUDA(cudaStreamSynchronize(s));
            for (int t = 0; t < cnt; ++t) {
              std::vector<cplx> zz(nb);
              for (int b = 0; b < nb; ++b) {
                double re = 0, im = 0;
                for (int q = 0; q < nblk; ++q) {
                  re += hz[(((size_t)b * nblk + q) * cnt + t) * 2];
                  im += hz[(((size_t)b * nblk + q) * cnt + t) * 2 + 1];
                }
                if (P->nmodes[b] > 0) zz[b] = {re / P->nmodes[b], im / P->nmodes[b]};
              }
              (kind ? ps[k].Zp : ps[k].Z)[{lm[g0 + t].first, lm[g0 + t].second, L, M}] = zz;
            }
          }
        }
    }
  }
  std::vector<double> cU, cD, cW;
  if (f64) {
    const int nbk = f64_block_bins(P);
    P->f64shell.ensure((size_t)(nbk == nb ? nb : 2 * nbk) * P->comps.size() * Ng * 8, &P->bytes);
    f64_pairs(P, nullptr, true, P->f64q.as<double>(), npass, nbk, cU, &launches);
    f64_pairs(P, P->pass_spec[0].as<float2>() + (size_t)P->d00 * Nk, false, P->f64g.as<double>(), 1, nbk, cD,
              &launches);
    if (npass == 2)
      f64_pairs(P, P->pass_spec[1].as<float2>() + (size_t)P->d00 * Nk, false, P->f64g.as<double>() + (size_t)nD * Ng,
                1, nbk, cW, &launches);
    // the shell blocks take what memory was free: give it back for the next assignment
    BISP_CUDA(cudaStreamSynchronize(s));
    P->f64shell.release(&P->bytes);
  } else {
    // pair reductions
    P->pool.ensure((size_t)(nbk == nb || P->diagonal ? nbk : 2 * nbk) * P->pass_ncomp(false) * Ng * 4, &P->bytes);
    // i = j != k shot term: unit shells, q fields of every pass (the three-point function
    // reads its q fields at the separations of each r-bin instead, below)
    if (!three) pair_set(P, nullptr, true, npass, P->qf.as<float>(), nbk, cU, &launches);
    // data
    pair_set(P, P->pass_spec[0].as<float2>(), false, 1, P->gf[0].as<float>(), nbk, cD,
             &launches);
    if (npass == 2)
      pair_set(P, P->pass_spec[1].as<float2>(), false, 1, P->gf[1].as<float>(), nbk, cW,
               &launches);
  }
  std::vector<float> gq[2];
  if (three) {
    const int64_t noff = (int64_t)P->roff.size();
    P->gath.ensure(std::max<size_t>((size_t)noff * nD * 4, 256), &P->bytes);
    for (int k = 0; k < npass; ++k) {
      launch_gather_neg(P->qf.as<float>() + (size_t)k * nD * Ng, Ng, nD, P->roff_d.as<uint32_t>(), noff, P->N,
                        P->gath.as<float>(), s);
      ++launches;
      gq[k].resize((size_t)noff * nD);
      if (noff)
        BISP_CUDA(cudaMemcpyAsync(gq[k].data(), P->gath.p, gq[k].size() * 4, cudaMemcpyDeviceToHost, s));
      BISP_CUDA(cudaStreamSynchronize(s));
    }
  }
  BISP_CUDA(cudaEventRecord(P->ev1, s));
  int flag = 0;
  BISP_CUDA(cudaMemcpyAsync(&flag, P->flags.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  BISP_CUDA(cudaStreamSynchronize(s));
  if (flag) fail(BISP_ETIMEOUT, "inverse FFT: a staged row group did not arrive within 2 s");
  float ms = 0.f;
  BISP_CUDA(cudaEventElapsedTime(&ms, P->ev0, P->ev1));
  P->ms_measure = ms;
  P->launches_measure = launches;
  if (three) {
    threept_combine(P, npass, cD, cW, gq, outB, outShot, outW, outWS, outNm);
    return;
  }
  // host FP64: normalisation, 3j-contracted shell terms, subtraction
  const double Ngd = (double)Ng;
  for (int k = 0; k < npass; ++k) {
    const std::vector<double>& raw = k == 0 ? cD : cW;
    double* oB = k == 0 ? outB : outW;
    double* oS = k == 0 ? outShot : outWS;
    for (int mu = 0; mu < nmult; ++mu) {
      const int l1 = P->ells[mu][0], l2 = P->ells[mu][1], L = P->ells[mu][2];
      const double pref = (double)((2 * l1 + 1) * (2 * l2 + 1) * (2 * L + 1)) * wigner3j(l1, l2, L, 0, 0, 0) / P->normI;
      for (int b1 = 0; b1 < nb; ++b1)
        for (int b2 = 0; b2 < nb; ++b2) {
          cplx sh;
          for (int m1 = -l1; m1 <= l1; ++m1)
            for (int m2 = -l2; m2 <= l2; ++m2) {
              const int M = -m1 - m2;
              if (std::abs(M) > L || (!local && M != 0)) continue;
              const double w = wigner3j(l1, l2, L, m1, m2, M);
              if (w == 0.0) continue;
              const int Lz = local ? L : 0;
              const cplx Y1 = P->Y[b1][P->lm_index(l1, m1)], Y2 = P->Y[b2][P->lm_index(l2, m2)];
              // Sbar_L^M and Z for signed M via Z(l,m,L,-M) = (-1)^{m+M+l} conj Z(l,-m,L,M)
              auto sbar_at = [&](int MM) {
                const cplx v = ps[k].sbar.at({Lz, std::abs(MM)});
                if (MM >= 0) return v;
                const double sg = (std::abs(MM) & 1) ? -1.0 : 1.0;
                return cplx{sg * v.r, -sg * v.i};
              };
              auto z_at = [&](int l, int m, int MM, int b, bool primed) {
                const auto& Zm = primed ? ps[k].Zp : ps[k].Z;
                if (MM >= 0) return Zm.at({l, m, Lz, MM})[b];
                const cplx v = Zm.at({l, -m, Lz, -MM})[b];
                const double sg = ((m + MM + l) & 1) ? -1.0 : 1.0;
                return cplx{sg * v.r, -sg * v.i};
              };
              const cplx S = sbar_at(M);
              // the slot that carries the line of sight takes the primed sums (App. B)
              const bool p1 = local && P->los_obj == 1, p2 = local && P->los_obj == 2;
              const cplx Z1 = z_at(l1, m1, M, b1, p1), Z2 = z_at(l2, m2, M, b2, p2);
              const cplx iii = cm(S, cm(Y1, Y2));
              const cplx ijj = cm(Z1, Y2);
              const cplx iji = cm(Y1, Z2);
              sh.r += w * (iii.r + ijj.r + iji.r);
            }
          const size_t o = ((size_t)mu * nb + b1) * nb + b2;
          const double iij = cU[(size_t)(k * nmult + mu) * nb * nb + b1 * nb + b2] / Ngd;
          const double shot = pref * (sh.r + iij);
          const double braw = pref * raw[(size_t)mu * nb * nb + b1 * nb + b2] / Ngd;
          const bool off = P->diagonal && b1 != b2;  // not computed
          if (oB) oB[o] = off ? NAN : braw - shot;
          if (oS) oS[o] = off ? NAN : shot;
        }
    }
  }
  if (outNm)
    for (int b = 0; b < nb; ++b) outNm[b] = P->nmodes[b];
}

void destroy(bisp_plan* P) {
  if (!P) return;
  size_t* t = &P->bytes;
  for (auto* d : {&P->tw, &P->winv, &P->ynorm, &P->cw2, &P->qlo_d, &P->qhi_d, &P->zmodes, &P->zmode_off, &P->pool, &P->invscr, &P->pairscr,
                  &P->pairout, &P->zpart, &P->ws, &P->flags, &P->ynorm_d, &P->cw2_d, &P->f64work, &P->f64spec,
                  &P->f64g, &P->f64q, &P->f64shell, &P->f64part, &P->f64out, &P->roff_d, &P->ones,
                  &P->kmesh, &P->gath})
    d->release(t);
  f64_fft_destroy(P->fft64);
  for (int k = 0; k < 2; ++k) {
    P->cat[k].spec.release(t);
    P->cat[k].dbg_mesh.release(t);
    P->pass_spec[k].release(t);
    P->gf[k].release(t);
  }
  P->qf.release(t);
  if (P->ev0) cudaEventDestroy(P->ev0);
  if (P->ev1) cudaEventDestroy(P->ev1);
  if (P->own_stream && P->stream) cudaStreamDestroy(P->stream);
  delete P;
}

template <class F>
bisp_status guarded(F&& f) {
  g_alloc_calls = 0;
  g_stalls_used = 0;
  try {
    f();
    return BISP_OK;
  } catch (const Fail& e) {
    g_err = e.msg;
    return (bisp_status)e.status;
  } catch (const Error& e) {
    g_err = e.msg;
    return (bisp_status)e.status;
  } catch (const std::exception& e) {
    g_err = e.what();
    return BISP_EINVAL;
  }
}

}  // namespace

// =====================================================================================
// C ABI
// =====================================================================================
#ifdef BISP_CHECKED
namespace bisp {
__device__ unsigned long long g_bisp_check = 0;  // first failed device check (checked build)
}
#endif
extern "C" {

bisp_status bisp_plan_create(bisp_plan** out, const bisp_params* p, void* stream) {
  if (!out) {
    g_err = "out is NULL";
    return BISP_EINVAL;
  }
  *out = nullptr;
  bisp_plan* P = new bisp_plan();
  bisp_status st = guarded([&] {
    validate(p);
    P->N = p->nmesh;
    P->NH = P->N / 2;
    P->L = p->box_len;
    P->H = P->L / P->N;
    P->kF = 2.0 * M_PI / P->L;
    P->V = P->L * P->L * P->L;
    P->Ng = (int64_t)P->N * P->N * P->N;
    P->Nk = (int64_t)P->N * P->N * (P->N / 2);
    P->nb = p->nbins;
    P->edges.assign(p->k_edges, p->k_edges + p->nbins + 1);
    P->nmult = p->n_mult;
    for (int i = 0; i < p->n_mult; ++i) P->ells.push_back({p->ells[3 * i], p->ells[3 * i + 1], p->ells[3 * i + 2]});
    P->los = p->los;
    for (int k = 0; k < 3; ++k) P->obs[k] = p->observer[k];
    P->mas = p->mas;
    P->interlace = p->interlace ? 1 : 0;
    P->P0 = p->fkp_P0;
    P->max_bytes = p->max_device_bytes;
    P->want_window = p->want_window ? 1 : 0;
    P->precision = p->precision;
    P->estimator = p->estimator;
    P->diagonal = p->diagonal_only ? 1 : 0;
    P->los_obj = (p->los_object == 0 || p->los == BISP_LOS_GLOBAL_Z) ? 3 : p->los_object;
    const char* dbg = std::getenv("BISP_DEBUG");
    P->debug_mesh = dbg && std::strstr(dbg, "BISP_DEBUG_KEEP_MESH");
    int dev = 0;
    BISP_CUDA(cudaGetDevice(&dev));
    if (stream) {
      P->stream = (cudaStream_t)stream;
    } else {
      BISP_CUDA(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
      P->own_stream = true;
    }
    BISP_CUDA(cudaEventCreate(&P->ev0));
    BISP_CUDA(cudaEventCreate(&P->ev1));
    build_channels(P);
    if (P->estimator == BISP_THREEPT)
      build_rshells(P);
    else
      build_shells(P);
    build_recipes(P);
    upload_tables(P);
  });
  if (st != BISP_OK) {
    destroy(P);
    return st;
  }
  *out = P;
  return BISP_OK;
}

bisp_status bisp_assign(bisp_plan* plan, int which, const float* xyz, const float* w, const float* nbar, int64_t n,
                        int ptr_is_device) {
  if (!plan) {
    g_err = "plan is NULL";
    return BISP_EINVAL;
  }
  return guarded([&] { do_assign(plan, which, xyz, w, nbar, n, ptr_is_device); });
}

bisp_status bisp_measure(bisp_plan* plan, double* B, double* shot, double* window, double* window_shot,
                         double* nmodes) {
  if (!plan) {
    g_err = "plan is NULL";
    return BISP_EINVAL;
  }
  return guarded([&] { do_measure(plan, B, shot, window, window_shot, nmodes); });
}

bisp_status bisp_measure_batch(bisp_plan* const* plans, const bisp_outputs* outs, int nplans) {
  if (nplans < 0 || (nplans > 0 && (!plans || !outs))) {
    g_err = "bisp_measure_batch: nplans < 0 or NULL arrays";
    return BISP_EINVAL;
  }
  for (int i = 0; i < nplans; ++i) {
    if (!plans[i]) {
      g_err = "bisp_measure_batch: plan " + std::to_string(i) + " is NULL";
      return BISP_EINVAL;
    }
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) {
        g_err = "bisp_measure_batch: plan " + std::to_string(i) + " repeats plan " + std::to_string(j);
        return BISP_EINVAL;
      }
  }
  if (nplans == 0) return BISP_OK;
  // Host worker threads measure the plans concurrently, each plan on its own stream, so that the
  // GPU overlaps the small kernels and host round trips of many realisations.  Plans share no
  // device buffers; job tables are launch parameters, or (the contraction's) a constant slot held
  // under a lock until its launches complete.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    g_err = "bisp_measure_batch: cudaGetDevice failed";
    return BISP_ECUDA;
  }
  std::vector<int> st(nplans, BISP_OK);
  std::vector<std::string> msg(nplans);
  std::atomic<int> next{0};
  auto work = [&] {
    cudaSetDevice(dev);
    for (int i = next++; i < nplans; i = next++) {
      const bisp_outputs& o = outs[i];
      st[i] = guarded([&] { do_measure(plans[i], o.B, o.shot, o.window, o.window_shot, o.nmodes); });
      if (st[i] != BISP_OK) msg[i] = g_err;
    }
  };
  const int nthr = std::min(nplans, kBatchThreads);
  std::vector<std::thread> pool;
  try {
    for (int t = 1; t < nthr; ++t) pool.emplace_back(work);
  } catch (const std::exception&) {
    // fewer workers (the calling thread still takes part)
  }
  work();
  for (auto& th : pool) th.join();
  for (int i = 0; i < nplans; ++i)
    if (st[i] != BISP_OK) {
      g_err = "bisp_measure_batch: plan " + std::to_string(i) + ": " + msg[i];
      return (bisp_status)st[i];
    }
  return BISP_OK;
}

bisp_status bisp_plan_destroy(bisp_plan* plan) {
  destroy(plan);
  return BISP_OK;
}

const char* bisp_last_error(void) { return g_err.c_str(); }

bisp_status bisp_plan_query(const bisp_plan* P, bisp_plan_info* info) {
  if (!P || !info) {
    g_err = "NULL argument";
    return BISP_EINVAL;
  }
  std::memset(info, 0, sizeof(*info));
  info->nmesh = P->N;
  info->nbins = P->nb;
  info->n_mult = P->nmult;
  info->n_dchan = (int)P->dch.size();
  info->n_nchan = (int)P->nch.size();
  info->n_fcomp = (int)P->comps.size();
  info->alpha = P->alpha;
  info->norm_I = P->normI;
  info->n_data = P->cat[0].n;
  info->n_randoms = P->cat[1].n;
  info->device_bytes = P->bytes;
  info->kernel_launches = P->cat[0].launches + P->cat[1].launches + P->launches_measure;
  info->ms_assign_data = P->cat[0].ms;
  info->ms_assign_randoms = P->cat[1].ms;
  info->ms_measure = P->ms_measure;
  info->ms_pair = P->ms_pair;
  info->pair_bytes = P->pair_bytes;
  info->pair_launches = P->pair_launches;
  info->pair_kernel = P->pair_kernel;
  info->zpass_groups = P->zgroups;
  return BISP_OK;
}

bisp_status bisp_cell_order(int nmesh, double box_len, int mas, const float* xyz, int64_t n, uint32_t* keys_out,
                            uint32_t* order_out, void* stream) {
  return guarded([&] {
    if (nmesh < 16 || nmesh > BISP_NMAX || (nmesh & (nmesh - 1))) fail(BISP_EINVAL, "nmesh");
    if (!(box_len > 0)) fail(BISP_EINVAL, "box_len");
    if (mas < 1 || mas > 3) fail(BISP_EINVAL, "mas");
    if (n < 0 || (n > 0 && (!xyz || !keys_out || !order_out))) fail(BISP_EINVAL, "bad pointers or size");
    if (n == 0) return;
    cudaStream_t s = (cudaStream_t)stream;
    size_t tb = 0;
    DBuf keys, idx, frac, part, bad, scr;
    keys.ensure(n * 4, &tb);
    idx.ensure(n * 4, &tb);
    frac.ensure(n * 16, &tb);
    part.ensure((size_t)prep_blocks(n) * 8, &tb);
    bad.ensure(64, &tb);
    BISP_CUDA(cudaMemsetAsync(bad.p, 0, 64, s));
    PrepArgs a{};
    a.xyz = xyz;
    a.n = n;
    a.N = nmesh;
    a.H = box_len / nmesh;
    a.box = box_len;
    a.mas = mas;
    a.nchan = 0;
    a.keys = keys.as<uint32_t>();
    a.idx = idx.as<uint32_t>();
    a.frac = frac.as<float4>();
    a.vals = nullptr;
    a.partials = part.as<double>();
    a.nsum = 1;
    a.bad = bad.as<int>();
    std::vector<float> yn((BISP_LMAX + 1) * (BISP_LMAX + 1), 1.f);
    DBuf ynd;
    ynd.ensure(yn.size() * 4, &tb);
    BISP_CUDA(cudaMemcpyAsync(ynd.p, yn.data(), yn.size() * 4, cudaMemcpyHostToDevice, s));
    a.ynorm = ynd.as<float>();
    launch_prep(a, s);
    int nbad = 0;
    BISP_CUDA(cudaMemcpyAsync(&nbad, bad.p, 4, cudaMemcpyDeviceToHost, s));
    BISP_CUDA(cudaStreamSynchronize(s));
    if (nbad) fail(BISP_EINVAL, std::to_string(nbad) + " particles have non-finite or out-of-box positions");
    int bits = 0;
    while ((1LL << bits) < (int64_t)nmesh * nmesh * nmesh) ++bits;
    scr.ensure(radix_sort_scratch_bytes(n), &tb);
    radix_sort(keys.as<uint32_t>(), idx.as<uint32_t>(), keys_out, order_out, n, bits, scr.p, s, nullptr);
    BISP_CUDA(cudaStreamSynchronize(s));
    for (DBuf* d : {&keys, &idx, &frac, &part, &bad, &scr, &ynd}) d->release(&tb);
  });
}

bisp_status bisp_check_word(uint64_t* word, int reset) {
  if (!word) {
    g_err = "NULL argument";
    return BISP_EINVAL;
  }
#ifdef BISP_CHECKED
  return guarded([&] {
    unsigned long long w = 0;
    BISP_CUDA(cudaDeviceSynchronize());
    BISP_CUDA(cudaMemcpyFromSymbol(&w, bisp::g_bisp_check, sizeof(w)));
    if (reset) {
      const unsigned long long z = 0;
      BISP_CUDA(cudaMemcpyToSymbol(bisp::g_bisp_check, &z, sizeof(z)));
    }
    *word = (uint64_t)w;
  });
#else
  (void)reset;
  *word = 0;
  g_err = "device bounds checks are compiled only into the checked build";
  return BISP_EUNSUPPORTED;
#endif
}

bisp_status bisp_debug_fetch(const bisp_plan* P, int what, int which, int index, void* host_out, size_t bytes) {
  return guarded([&] {
    if (!P || !host_out) fail(BISP_EINVAL, "NULL argument");
    if (which != 0 && which != 1) fail(BISP_EINVAL, "which");
    const Catalog& C = P->cat[which];
    if (!C.assigned) fail(BISP_ESTATE, "catalogue not assigned");
    if (index < 0 || index >= C.nspec) fail(BISP_EINVAL, "channel index");
    if (what == BISP_DBG_SPECTRUM) {
      const size_t b = (size_t)P->Nk * 8;
      if (bytes != b) fail(BISP_EINVAL, "bytes");
      BISP_CUDA(cudaMemcpy(host_out, C.spec.as<float2>() + (size_t)index * P->Nk, b, cudaMemcpyDeviceToHost));
    } else if (what == BISP_DBG_MESH) {
      if (!C.dbg_mesh.p) fail(BISP_ESTATE, "mesh not kept (set BISP_DEBUG=BISP_DEBUG_KEEP_MESH)");
      const size_t b = (size_t)P->Ng * 4;
      if (bytes != b) fail(BISP_EINVAL, "bytes");
      BISP_CUDA(cudaMemcpy(host_out, C.dbg_mesh.as<float>() + (size_t)index * P->Ng, b, cudaMemcpyDeviceToHost));
    } else {
      fail(BISP_EINVAL, "what");
    }
  });
}

}  // extern "C"
