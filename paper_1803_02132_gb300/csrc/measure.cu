// Measurement kernels:
//  * k_axpby: the spectra of one estimator pass, delta n = D_gal - alpha D_ran (Eq. dn)
//    and N = N_gal + alpha^2 N_ran (Eq. ShotNoise definitions);
//  * k_zsum: FP64 shell sums (1/N_mode) sum_shell y_l^{m*}(k) [D(k) N_L^{M*}(k) -
//    Sbar_L^M C(k)/W^2(k)] of the i!=j=k and i=k!=j shot-noise terms (Eq. ShotNoise);
//  * k_pair: the mesh sum of Eq. bi_estimator_FFTs, contracted over the (m1, m2, M)
//    terms: out[o][b1][b2] = sum_x sum_t X_t(x; b1) Y_t(x; b2), where each side is a
//    small combination of filtered fields and G fields prepared per x chunk in shared
//    memory.  FP32 products in 4x4 register tiles, FP32 partials over at most 1024
//    cells, FP64 above that; per-CTA partials are reduced in a fixed order.
#include <algorithm>
#include <cstdlib>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace bisp {

// ------------------------------------------------------------------------------------
__global__ void k_axpby(float2* out, const float2* x, double a, const float2* y, double b, size_t n,
                        int zero_k0) {
  const float fa = (float)a, fb = (float)b;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float2 v = x[i];
    v = make_float2(fa * v.x, fa * v.y);
    if (y) {
      const float2 w = y[i];
      v = make_float2(fmaf(fb, w.x, v.x), fmaf(fb, w.y, v.y));
    }
    if (zero_k0 && i == 0) v = make_float2(0.f, 0.f);
    out[i] = v;
  }
}

void launch_axpby(float2* out, const float2* x, double a, const float2* y, double b, size_t n, int zero_k0,
                  cudaStream_t s) {
  size_t blocks = (n + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  k_axpby<<<(unsigned)blocks, 256, 0, s>>>(out, x, a, y, b, n, zero_k0);
  BISP_CHECK_LAUNCH();
}

// ------------------------------------------------------------------------------------
// shell sums
// ------------------------------------------------------------------------------------
__constant__ ZsumArgs c_zs;
constexpr int ZS_THREADS = 256;
constexpr int ZS_MAXLM = 9;

__device__ __forceinline__ float2 ystar(int l, int m, float x, float y, float z, const float* ynorm);

__global__ void __launch_bounds__(ZS_THREADS) k_zsum() {
  const ZsumArgs& A = c_zs;
  const int b = blockIdx.y;
  const int N = A.N, NH = N / 2;
  const int64_t m0 = A.mode_off[b], m1 = A.mode_off[b + 1];
  double acc[ZS_MAXLM][2];
#pragma unroll
  for (int q = 0; q < ZS_MAXLM; ++q) acc[q][0] = acc[q][1] = 0.0;
  for (int64_t i = m0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m1; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t code = A.modes[i];
    const int sx = (int)(code & 1023u) - 512, sy = (int)((code >> 10) & 1023u) - 512, nz = (int)(code >> 20);
    const int jx = sx & (N - 1), jy = sy & (N - 1);
    const size_t gi = ((size_t)jx * N + jy) * NH + nz;
    const float2 d = A.D00[gi];
    const float2 nr = A.NR[gi];
    const float2 ni = A.NI ? A.NI[gi] : make_float2(0.f, 0.f);
    // N(k) = NR + i NI ; N(-k) = conj(NR) + i conj(NI)
    const double nkr = (double)nr.x - (double)ni.y, nki = (double)nr.y + (double)ni.x;
    const double nmr = (double)nr.x + (double)ni.y, nmi = -(double)nr.y + (double)ni.x;
    double cw = (double)A.cw2_1d[jx] * A.cw2_1d[jy] * A.cw2_1d[nz];
    if (A.interlace) cw = 0.5 * (cw + (double)A.cw2_1d[N + jx] * A.cw2_1d[N + jy] * A.cw2_1d[N + nz]);
    // T(k) = D(k) conj(N(k)) - Sbar C/W^2
    const double dr = d.x, di = d.y;
    const double tkr = dr * nkr + di * nki - A.sbar_re * cw;
    const double tki = di * nkr - dr * nki - A.sbar_im * cw;
    // T(-k) = conj(D(k)) conj(N(-k)) - Sbar C/W^2
    const double tmr = dr * nmr - di * nmi - A.sbar_re * cw;
    const double tmi = -di * nmr - dr * nmi - A.sbar_im * cw;
    const bool pair = nz > 0;
#pragma unroll
    for (int t = 0; t < ZS_MAXLM; ++t) {
      if (t < A.nlm) {
        const int l = A.lm[t][0], m = A.lm[t][1];
        const float2 ys = ystar(l, m, (float)sx, (float)sy, (float)nz, A.ynorm);
        double yr = ys.x, yi = ys.y;
        acc[t][0] += yr * tkr - yi * tki;
        acc[t][1] += yr * tki + yi * tkr;
        if (pair) {  // y*(-k) = (-1)^l y*(k)
          const double sg = (l & 1) ? -1.0 : 1.0;
          acc[t][0] += sg * (yr * tmr - yi * tmi);
          acc[t][1] += sg * (yr * tmi + yi * tmr);
        }
      }
    }
  }
  __shared__ double red[ZS_THREADS / 32];
#pragma unroll
  for (int t = 0; t < ZS_MAXLM; ++t) {
    if (t >= A.nlm) break;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      double v = acc[t][c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < ZS_THREADS / 32; ++w) s += red[w];
        A.partials[(((size_t)b * A.nblk + blockIdx.x) * A.nlm + t) * 2 + c] = s;
      }
      __syncthreads();
    }
  }
}

// y_l^{m*}(n) for signed m; y_l^{-m} = (-1)^m conj(y_l^m)
__device__ __forceinline__ float2 ystar(int l, int m, float x, float y, float z, const float* ynorm) {
  const int am = m < 0 ? -m : m;
  const float r2 = x * x + y * y + z * z;
  if (r2 == 0.f) return l == 0 ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
  const float rinv = rsqrtf(r2);
  const float mu = z * rinv;
  float pmm = 1.f;
  for (int k = 1; k <= am; ++k) pmm *= -(2.f * k - 1.f);
  float p = pmm;
  if (l > am) {
    float pm2 = pmm, pm1 = (2.f * am + 1.f) * mu * pmm;
    p = pm1;
    for (int ll = am + 2; ll <= l; ++ll) {
      p = ((2.f * ll - 1.f) * mu * pm1 - (float)(ll + am - 1) * pm2) / (float)(ll - am);
      pm2 = pm1;
      pm1 = p;
    }
  }
  float2 e = make_float2(1.f, 0.f);
  const float2 e1 = make_float2(x * rinv, y * rinv);
  for (int k = 0; k < am; ++k) e = cmul(e, e1);
  const float a = ynorm[l * (BISP_LMAX + 1) + am] * p;
  float2 yv = make_float2(a * e.x, a * e.y);  // y_l^{|m|}
  if (m >= 0) return cconj(yv);
  // y_l^{-|m|*} = (-1)^m y_l^{|m|}
  if (am & 1) yv = make_float2(-yv.x, -yv.y);
  return yv;
}

void launch_zsum(const ZsumArgs& a, cudaStream_t s) {
  if (a.nlm > ZS_MAXLM) throw Error{6, "zsum: too many (l, m) per launch"};
  BISP_CUDA(cudaMemcpyToSymbolAsync(c_zs, &a, sizeof(ZsumArgs), 0, cudaMemcpyHostToDevice, s));
  k_zsum<<<dim3(a.nblk, a.nbins), ZS_THREADS, 0, s>>>();
  BISP_CHECK_LAUNCH();
}

// ------------------------------------------------------------------------------------
// pair reduction
//   out[o][b1][b2] = sum_x sum_{t in o} X_t(x; b1) Y_t(x; b2)
// Each CTA streams chunks of PR_CH cells.  All component fields and G fields of a chunk
// are copied to shared memory with 16-byte cp.async, PR_NSTAGE chunks in flight.  Sides
// that are combinations of fields are built in shared memory; bare component sides are
// read in place.  One warp owns one (term, x slice): its 32 lanes form a 4 x 8 grid and
// each lane holds a TM x TN register tile of (b1, b2), so the warp covers 4TM x 8TN bins.
// FP32 partials over at most PR_FLUSH chunks are added to lane-owned FP64 slots in global
// memory; a second kernel reduces the slots in a fixed order.
// ------------------------------------------------------------------------------------
__constant__ PairJob c_pj;
constexpr int PR_CH = 64;          // cells per chunk
constexpr int PR_LD = PR_CH + 4;   // padded row (bank spread for 16-byte loads)
constexpr int PR_FLUSH = 16;       // chunks per FP32 partial (<= 1024 cells)
constexpr int PR_NSTAGE = 2;       // chunks staged ahead
constexpr int PR_MAXWARP = 16;

struct PairLaunch {
  int TM, TN, nbp, bs, ksplit, warps, nblk, rows;
  size_t smem;
};

static void pick_tile(int nb, int* TM, int* TN) {
  static const int tab[][2] = {{1, 1}, {2, 1}, {3, 2}, {4, 2}, {5, 3}, {6, 3}, {7, 4}, {8, 4}, {10, 5}};
  for (auto& t : tab)
    if (4 * t[0] >= nb && 8 * t[1] >= nb) {
      *TM = t[0];
      *TN = t[1];
      return;
    }
  throw Error{6, "pair reduction: more than 40 bins"};
}

static PairLaunch pair_launch_cfg(const PairJob& j) {
  PairLaunch c;
  pick_tile(j.nb, &c.TM, &c.TN);
  c.nbp = std::max(4 * c.TM, 8 * c.TN);
  if (j.nterm > 2 * PR_MAXWARP || (j.nterm > PR_MAXWARP && c.TM * c.TN > 18))
    throw Error{6, "pair reduction: too many terms for one CTA"};
  c.ksplit = 1;
  while (c.ksplit < 4 && j.nterm * c.ksplit * 2 <= PR_MAXWARP) c.ksplit *= 2;  // slices of >= 16 cells
  c.warps = j.nterm * c.ksplit;
  c.bs = j.ncomp | 1;  // odd rows per bin: consecutive bins fall on different banks
  c.rows = j.nb * c.bs + j.ng;  // padded bins (b >= nb) read a valid row; their outputs are dropped
  c.smem = ((size_t)PR_NSTAGE * c.rows * PR_LD + (size_t)j.nslot * j.nb * PR_LD + (size_t)j.nh * PR_CH +
            (size_t)(j.nb * j.ncomp + j.ng)) *
           sizeof(float);
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  c.nblk = nsm;
  return c;
}

// merge terms equal up to a scalar, then classify the sides of every term: bare component
// field (read in place) or built
static PairJob classify(const PairJob& job) {
  PairJob j = job;
  {
    // normalised term: a single-entry X side (c, g, coef) with a bare Y side is coef times
    // the unit term (c, g, 1 | Y); other terms are kept as they are (multiplier 1)
    struct Key {
      std::vector<std::tuple<int, int, float>> x, y;
      bool operator==(const Key& o) const { return x == o.x && y == o.y; }
    };
    std::vector<Key> keys;
    std::vector<PairTermDesc> nterm;
    std::vector<PairRecipe> nrec;
    int ne = 0;
    for (int o = 0; o < j.nout; ++o) {
      j.out_ent_off[o] = ne;
      for (int t = job.out_term_off[o]; t < job.out_term_off[o + 1]; ++t) {
        const PairTermDesc& T = job.term[t];
        Key k;
        double mult = 1.0;
        for (int e = 0; e < T.xcnt; ++e) {
          const PairRecipe& R = job.rec[T.xoff + e];
          k.x.push_back({R.comp, R.g, R.coef});
        }
        for (int e = 0; e < T.ycnt; ++e) {
          const PairRecipe& R = job.rec[T.yoff + e];
          k.y.push_back({R.comp, R.g, R.coef});
        }
        auto bare_y = [&]() { return k.y.size() == 1 && std::get<1>(k.y[0]) < 0 && std::get<2>(k.y[0]) == 1.0f; };
        if (k.x.size() == 1 && bare_y()) {
          mult = std::get<2>(k.x[0]);
          std::get<2>(k.x[0]) = 1.0f;
        }
        int u = -1;
        for (size_t i = 0; i < keys.size(); ++i)
          if (keys[i] == k) u = (int)i;
        if (u < 0) {
          u = (int)keys.size();
          keys.push_back(k);
          PairTermDesc d{};
          d.xoff = (int)nrec.size();
          d.xcnt = (int)k.x.size();
          for (auto& r : k.x) nrec.push_back({std::get<0>(r), std::get<1>(r), std::get<2>(r)});
          d.yoff = (int)nrec.size();
          d.ycnt = (int)k.y.size();
          for (auto& r : k.y) nrec.push_back({std::get<0>(r), std::get<1>(r), std::get<2>(r)});
          nterm.push_back(d);
        }
        if (ne >= 128) throw Error{6, "pair reduction: too many output entries"};
        j.out_ent_term[ne] = u;
        j.out_ent_mult[ne] = mult;
        ++ne;
      }
    }
    j.out_ent_off[j.nout] = ne;
    if (nterm.size() > 64 || nrec.size() > 512) throw Error{6, "pair reduction: recipe tables overflow"};
    j.nterm = (int)nterm.size();
    for (int t = 0; t < j.nterm; ++t) j.term[t] = nterm[t];
    j.nrec = (int)nrec.size();
    for (int r = 0; r < j.nrec; ++r) j.rec[r] = nrec[r];
  }
  j.nslot = 0;
  for (int t = 0; t < j.nterm; ++t) {
    PairTermDesc& T = j.term[t];
    auto bare = [&](int off, int cnt) {
      return cnt == 1 && j.rec[off].g < 0 && j.rec[off].coef == 1.0f ? j.rec[off].comp : -1;
    };
    T.xdir = bare(T.xoff, T.xcnt);
    T.ydir = bare(T.yoff, T.ycnt);
    T.xslot = T.xdir >= 0 ? -1 : j.nslot++;
    T.yslot = T.ydir >= 0 ? -1 : j.nslot++;
  }
  // factor every built side by component: H rows shared between sides when identical
  std::vector<std::vector<std::pair<int, float>>> rows;
  j.nh = 0;
  int ns = 0, nse = 0;
  for (int t = 0; t < j.nterm; ++t)
    for (int side = 0; side < 2; ++side) {
      const PairTermDesc& T = j.term[t];
      const int slot = side ? T.yslot : T.xslot;
      if (slot < 0) continue;
      if (slot != ns) throw Error{6, "pair reduction: slot order"};
      j.s_off[ns] = nse;
      const int off = side ? T.yoff : T.xoff, cnt = side ? T.ycnt : T.xcnt;
      std::vector<int> comps;
      for (int e = 0; e < cnt; ++e)
        if (std::find(comps.begin(), comps.end(), j.rec[off + e].comp) == comps.end()) comps.push_back(j.rec[off + e].comp);
      for (int c : comps) {
        std::vector<std::pair<int, float>> row;
        for (int e = 0; e < cnt; ++e)
          if (j.rec[off + e].comp == c) row.push_back({j.rec[off + e].g, j.rec[off + e].coef});
        int h = -1;
        for (size_t r = 0; r < rows.size(); ++r)
          if (rows[r] == row) h = (int)r;
        if (h < 0) {
          h = (int)rows.size();
          rows.push_back(row);
        }
        if (nse >= 512) throw Error{6, "pair reduction: too many side entries"};
        j.s_ent[nse][0] = c;
        j.s_ent[nse][1] = h;
        ++nse;
      }
      ++ns;
    }
  j.s_off[ns] = nse;
  for (int q = 0; q < ns; ++q)
    if (j.s_off[q + 1] - j.s_off[q] > 8) throw Error{6, "pair reduction: more than 8 components in a side"};
  for (int t = 0; t < j.nterm; ++t)
    if (j.term[t].xslot >= 0 && j.term[t].yslot >= 0) throw Error{6, "pair reduction: both sides built"};
  if (rows.size() > 128) throw Error{6, "pair reduction: too many H rows"};
  int ne = 0;
  for (size_t r = 0; r < rows.size(); ++r) {
    j.h_off[r] = ne;
    for (auto& e : rows[r]) {
      if (ne >= 512) throw Error{6, "pair reduction: too many H entries"};
      j.h_ent[ne++] = {0, e.first, e.second};
    }
  }
  j.nh = (int)rows.size();
  j.h_off[j.nh] = ne;
  return j;
}

// the tensor-core contraction covers up to 32 bins; BISP_PAIR_FP32=1 forces the FP32 FMA kernel
static bool pair_use_tc(const PairJob& j) {
  const char* e = getenv("BISP_PAIR_FP32");
  return j.nb <= 32 && !(e && e[0] == '1');
}

size_t pair_scratch_bytes(const PairJob& job) {
  const PairJob j = classify(job);
  const PairLaunch c = pair_launch_cfg(j);
  const size_t per = pair_use_tc(j) ? 32 : (size_t)c.TM * c.TN;
  return (size_t)c.nblk * c.warps * 32 * per * sizeof(double);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int NW>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NW)); }

// copy one chunk of every component row [b][comp] and G row into shared memory;
// rowmap[f] = destination row of source row f (f < nb*ncomp: field (b, comp); then G rows)
__device__ __forceinline__ void pair_stage(float* raw, int64_t x0, const int* rowmap) {
  const PairJob& J = c_pj;
  constexpr int Q = PR_CH / 4;  // 16-byte pieces per row (a power of two)
  constexpr int QS = Q == 16 ? 4 : (Q == 8 ? 3 : 2);
  const int nraw = J.nb * J.ncomp;
  const int n = (nraw + J.ng) << QS;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int f = i >> QS, q = i & (Q - 1);
    const float* src = (f < nraw ? J.fields + (size_t)f * J.Ng : J.gfields + (size_t)(f - nraw) * J.Ng) + x0 + 4 * q;
    cp_async16(raw + (size_t)rowmap[f] * PR_LD + 4 * q, src);
  }
}

// built sides, block-wide: first the H rows of the chunk, H_h(x) = sum coef G_g(x) (shared by
// all bins), then one thread per (side, bin, 4-cell quad): X(b, x) = sum_(c,h) P_c(b, x) H_h(x).
// mnb = ceil(2^32 / nb): j / nb = umulhi(j, mnb) for the small j used here.
__device__ __forceinline__ void pair_build_sides(const float* raw, float* mat, float* Hs, int bs, unsigned mnb) {
  const PairJob& J = c_pj;
  constexpr int Q = PR_CH / 4;
  constexpr int QS = Q == 16 ? 4 : (Q == 8 ? 3 : 2);
  const int grow0 = J.nb * bs;
  for (int i = threadIdx.x; i < (J.nh << QS); i += blockDim.x) {
    const int h = i >> QS, q = i & (Q - 1);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = J.h_off[h]; e < J.h_off[h + 1]; ++e) {
      const PairRecipe R = J.h_ent[e];
      if (R.g >= 0) {
        const float4 gv = *reinterpret_cast<const float4*>(raw + (size_t)(grow0 + R.g) * PR_LD + 4 * q);
        v.x = fmaf(R.coef, gv.x, v.x);
        v.y = fmaf(R.coef, gv.y, v.y);
        v.z = fmaf(R.coef, gv.z, v.z);
        v.w = fmaf(R.coef, gv.w, v.w);
      } else {
        v.x += R.coef;
        v.y += R.coef;
        v.z += R.coef;
        v.w += R.coef;
      }
    }
    *reinterpret_cast<float4*>(Hs + (size_t)h * PR_CH + 4 * q) = v;
  }
  __syncthreads();
  const int n = (J.nslot * J.nb) << QS;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const unsigned j = (unsigned)i >> QS;
    const int q = i & (Q - 1);
    const int sl = (int)__umulhi(j, mnb);
    const int b = (int)j - sl * J.nb;
    const float* rb = raw + (size_t)b * bs * PR_LD + 4 * q;
    const float* hq = Hs + 4 * q;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    const int e1 = J.s_off[sl + 1];
    for (int e = J.s_off[sl]; e < e1; ++e) {
      const float4 pv = *reinterpret_cast<const float4*>(rb + J.s_ent[e][0] * PR_LD);
      const float4 hv = *reinterpret_cast<const float4*>(hq + J.s_ent[e][1] * PR_CH);
      v.x = fmaf(pv.x, hv.x, v.x);
      v.y = fmaf(pv.y, hv.y, v.y);
      v.z = fmaf(pv.z, hv.z, v.z);
      v.w = fmaf(pv.w, hv.w, v.w);
    }
    *reinterpret_cast<float4*>(mat + ((size_t)sl * J.nb + b) * PR_LD + 4 * q) = v;
  }
}

template <int TM, int TN, int NTHR>
__global__ void __launch_bounds__(NTHR, 1) k_pair(int nbp, int bs, int rows, int ksplit, double* partials) {
  const PairJob& J = c_pj;
  extern __shared__ __align__(16) float sh[];
  float* mat = sh + (size_t)PR_NSTAGE * rows * PR_LD;  // [nslot][nb][PR_LD]
  float* Hs = mat + (size_t)J.nslot * J.nb * PR_LD;  // [nh][PR_CH]
  int* rowmap = reinterpret_cast<int*>(Hs + (size_t)J.nh * PR_CH);
  const unsigned mnb = (unsigned)((0x100000000ull + J.nb - 1) / J.nb);
  const int64_t nchunk = J.Ng / PR_CH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int t = warp / ksplit, ks = warp % ksplit;
  const int slice = PR_CH / ksplit;
  const int b1 = lane >> 3, b2 = lane & 7;  // rows b1 + 4 i and b2 + 8 j
  const PairTermDesc T = J.term[t];
  for (int f = threadIdx.x; f < J.nb * J.ncomp + J.ng; f += blockDim.x) {
    const int nraw = J.nb * J.ncomp;
    rowmap[f] = f < nraw ? (f / J.ncomp) * bs + f % J.ncomp : J.nb * bs + (f - nraw);
  }
  __syncthreads();
  double* slot = partials + (((size_t)blockIdx.x * nwarp + warp) * 32 + lane) * (TM * TN);
#pragma unroll
  for (int q = 0; q < TM * TN; ++q) slot[q] = 0.0;
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  if (blockIdx.x < nchunk) pair_stage(sh, (int64_t)blockIdx.x * PR_CH, rowmap);
  cp_async_commit();
  int since_flush = 0, stage = 0;
  for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    cp_async_wait<0>();
    __syncthreads();
    {
      const int64_t nx = ch + gridDim.x;
      if (nx < nchunk) pair_stage(sh + (size_t)(stage ^ 1) * rows * PR_LD, nx * PR_CH, rowmap);
      cp_async_commit();
    }
    const float* raw = sh + (size_t)stage * rows * PR_LD;
    if (J.nslot) {
      pair_build_sides(raw, mat, Hs, bs, mnb);
      __syncthreads();
    }
    // row pointers of this lane's bins b1 + 4 i and b2 + 8 j (clamped to a valid row)
    const float* xrow[TM];
    const float* yrow[TN];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int b = min(b1 + 4 * i, J.nb - 1);
      xrow[i] = (T.xdir >= 0 ? raw + (size_t)(b * bs + T.xdir) * PR_LD : mat + ((size_t)T.xslot * J.nb + b) * PR_LD) +
                ks * slice;
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int b = min(b2 + 8 * j, J.nb - 1);
      yrow[j] = (T.ydir >= 0 ? raw + (size_t)(b * bs + T.ydir) * PR_LD : mat + ((size_t)T.yslot * J.nb + b) * PR_LD) +
                ks * slice;
    }
    for (int xb = 0; xb < slice; xb += 16) {
#pragma unroll
      for (int x = xb; x < xb + 16; x += 4) {
        float4 a[TM], c[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = *reinterpret_cast<const float4*>(xrow[i] + x);
#pragma unroll
        for (int j = 0; j < TN; ++j) c[j] = *reinterpret_cast<const float4*>(yrow[j] + x);
        // component-outer order: consecutive FMAs update different accumulators
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i].x, c[j].x, acc[i][j]);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i].y, c[j].y, acc[i][j]);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i].z, c[j].z, acc[i][j]);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i].w, c[j].w, acc[i][j]);
      }
    }
    if (++since_flush == PR_FLUSH || ch + gridDim.x >= nchunk) {
      since_flush = 0;
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          slot[i * TN + j] += (double)acc[i][j];
          acc[i][j] = 0.f;
        }
    }
    stage ^= 1;
  }
  cp_async_wait<0>();
}

// ------------------------------------------------------------------------------------
// Tensor-core variant of the contraction (nb <= 32): per warp and term, C (32 x 32 bins)
// += X (32 bins x cells) Y^T with mma.sync m16n8k8 TF32 in three passes (split FP32 values
// v = hi + lo, hi and lo TF32: X_hi Y_hi + X_hi Y_lo + X_lo Y_hi), which keeps FP32-level
// accuracy.  The MMA accumulators restart from zero every chunk; chunk results are added
// with FP32 round-to-nearest adds and flushed to FP64 as in k_pair.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tf32_hi(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ void split_tf32(float v, uint32_t& hi, uint32_t& lo) {
  hi = tf32_hi(v);
  lo = tf32_hi(v - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int NTHR>
__global__ void __launch_bounds__(NTHR, 1) k_pair_tc(int nbp, int bs, int rows, int ksplit, double* partials) {
  const PairJob& J = c_pj;
  extern __shared__ __align__(16) float sh[];
  float* mat = sh + (size_t)PR_NSTAGE * rows * PR_LD;  // [nslot][nb][PR_LD]
  float* Hs = mat + (size_t)J.nslot * J.nb * PR_LD;  // [nh][PR_CH]
  int* rowmap = reinterpret_cast<int*>(Hs + (size_t)J.nh * PR_CH);
  const unsigned mnb = (unsigned)((0x100000000ull + J.nb - 1) / J.nb);
  const int64_t nchunk = J.Ng / PR_CH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = warp / ksplit, ks = warp % ksplit;
  const int slice = PR_CH / ksplit;
  const int g = lane >> 2, tq = lane & 3;
  const PairTermDesc T = J.term[t];
  for (int f = threadIdx.x; f < J.nb * J.ncomp + J.ng; f += blockDim.x) {
    const int nraw = J.nb * J.ncomp;
    rowmap[f] = f < nraw ? (f / J.ncomp) * bs + f % J.ncomp : J.nb * bs + (f - nraw);
  }
  __syncthreads();
  double* slot = partials + (((size_t)blockIdx.x * (blockDim.x >> 5) + warp) * 32 + lane) * 32;
#pragma unroll
  for (int q = 0; q < 32; ++q) slot[q] = 0.0;
  float run[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) run[q] = 0.f;
  if (blockIdx.x < nchunk) pair_stage(sh, (int64_t)blockIdx.x * PR_CH, rowmap);
  cp_async_commit();
  int since_flush = 0, stage = 0;
  for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    cp_async_wait<0>();
    __syncthreads();
    {
      const int64_t nx = ch + gridDim.x;
      if (nx < nchunk) pair_stage(sh + (size_t)(stage ^ 1) * rows * PR_LD, nx * PR_CH, rowmap);
      cp_async_commit();
    }
    const float* raw = sh + (size_t)stage * rows * PR_LD;
    if (J.nslot) {
      pair_build_sides(raw, mat, Hs, bs, mnb);
      __syncthreads();
    }
    // rows of the fragments: A rows b1 = 16 mi + g (+8), B rows b2 = 8 ni + g (clamped)
    const float* ar[4];
    const float* br[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int b = min(8 * r + g, J.nb - 1);
      ar[r] = (T.xdir >= 0 ? raw + (size_t)(b * bs + T.xdir) * PR_LD : mat + ((size_t)T.xslot * J.nb + b) * PR_LD) +
              ks * slice + tq;
      br[r] = (T.ydir >= 0 ? raw + (size_t)(b * bs + T.ydir) * PR_LD : mat + ((size_t)T.yslot * J.nb + b) * PR_LD) +
              ks * slice + tq;
    }
    float c[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) c[q] = 0.f;
    for (int k0 = 0; k0 < slice; k0 += 8) {
      uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        split_tf32(ar[2 * mi][k0], ah[mi][0], al[mi][0]);
        split_tf32(ar[2 * mi + 1][k0], ah[mi][1], al[mi][1]);
        split_tf32(ar[2 * mi][k0 + 4], ah[mi][2], al[mi][2]);
        split_tf32(ar[2 * mi + 1][k0 + 4], ah[mi][3], al[mi][3]);
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        split_tf32(br[ni][k0], bh[ni][0], bl[ni][0]);
        split_tf32(br[ni][k0 + 4], bh[ni][1], bl[ni][1]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
          float* cc = c + (mi * 4 + ni) * 4;
          mma_tf32(cc, al[mi], bh[ni]);
          mma_tf32(cc, ah[mi], bl[ni]);
          mma_tf32(cc, ah[mi], bh[ni]);
        }
    }
#pragma unroll
    for (int q = 0; q < 32; ++q) run[q] += c[q];
    if (++since_flush == PR_FLUSH || ch + gridDim.x >= nchunk) {
      since_flush = 0;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        slot[q] += (double)run[q];
        run[q] = 0.f;
      }
    }
    stage ^= 1;
  }
  cp_async_wait<0>();
}

// final reduction for k_pair_tc: bin (b1, b2) of term t sits in warp t*ksplit+ks, lane
// (b1%8)*4 + (b2%8)/2, register ((b1/16)*4 + b2/8)*4 + ((b1/8)%2)*2 + b2%2
__global__ void k_pair_tc_final(const double* partials, int nblk, int warps, int ksplit, int nb, int nout,
                                double* out) {
  const PairJob& J = c_pj;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (gw >= nout * nb * nb) return;
  const int o = gw / (nb * nb), b1 = (gw / nb) % nb, b2 = gw % nb;
  const int ln = (b1 % 8) * 4 + (b2 % 8) / 2;
  const int q = ((b1 / 16) * 4 + b2 / 8) * 4 + ((b1 / 8) % 2) * 2 + (b2 % 2);
  double tot = 0.0;
  for (int e = J.out_ent_off[o]; e < J.out_ent_off[o + 1]; ++e) {
    const int t = J.out_ent_term[e];
    double s = 0.0;
    for (int ks = 0; ks < ksplit; ++ks) {
      const int w = t * ksplit + ks;
      for (int c = lane; c < nblk; c += 32) s += partials[(((size_t)c * warps + w) * 32 + ln) * 32 + q];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    tot += J.out_ent_mult[e] * s;
  }
  if (lane == 0) out[gw] = tot;
}

// out[o][b1][b2] = sum over terms of o, then CTAs and x slices in a fixed order; one warp
// per output value, lanes stride over CTAs, fixed shuffle tree.
__global__ void k_pair_final(const double* partials, int nblk, int warps, int ksplit, int TM, int TN, int nb,
                             int nout, double* out) {
  const PairJob& J = c_pj;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (gw >= nout * nb * nb) return;
  const int o = gw / (nb * nb), b1 = (gw / nb) % nb, b2 = gw % nb;
  const int ln = (b1 % 4) * 8 + b2 % 8, q = (b1 / 4) * TN + b2 / 8;
  double tot = 0.0;
  for (int e = J.out_ent_off[o]; e < J.out_ent_off[o + 1]; ++e) {
    const int t = J.out_ent_term[e];
    double s = 0.0;
    for (int ks = 0; ks < ksplit; ++ks) {
      const int w = t * ksplit + ks;
      for (int c = lane; c < nblk; c += 32) s += partials[(((size_t)c * warps + w) * 32 + ln) * (TM * TN) + q];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    tot += J.out_ent_mult[e] * s;
  }
  if (lane == 0) out[gw] = tot;
}

void pair_reduce(const PairJob& job, double* out_dev, void* scratch, size_t scratch_bytes, cudaStream_t s,
                 int* launches) {
  const PairJob j = classify(job);
  const PairLaunch c = pair_launch_cfg(j);
  if (scratch_bytes < pair_scratch_bytes(j)) throw Error{2, "pair reduction scratch too small"};
  if (j.Ng % PR_CH) throw Error{6, "mesh size not a multiple of the chunk"};
  if (c.smem > 227 * 1024) throw Error{6, "pair reduction: shared memory budget exceeded"};
  BISP_CUDA(cudaMemcpyToSymbolAsync(c_pj, &j, sizeof(PairJob), 0, cudaMemcpyHostToDevice, s));
  double* partials = reinterpret_cast<double*>(scratch);
  if (pair_use_tc(j)) {
    const int nthr = c.warps * 32;
    if (nthr <= 512) {
      BISP_CUDA(cudaFuncSetAttribute(k_pair_tc<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem));
      k_pair_tc<512><<<c.nblk, nthr, c.smem, s>>>(c.nbp, c.bs, c.rows, c.ksplit, partials);
    } else {
      BISP_CUDA(cudaFuncSetAttribute(k_pair_tc<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem));
      k_pair_tc<1024><<<c.nblk, nthr, c.smem, s>>>(c.nbp, c.bs, c.rows, c.ksplit, partials);
    }
    BISP_CHECK_LAUNCH();
    const int nout = j.nout * j.nb * j.nb;
    k_pair_tc_final<<<(nout * 32 + 255) / 256, 256, 0, s>>>(partials, c.nblk, c.warps, c.ksplit, j.nb, j.nout,
                                                            out_dev);
    BISP_CHECK_LAUNCH();
    if (launches) *launches += 2;
    return;
  }
#define BISP_PAIR3(A, B, NT)                                                                              \
  if (c.TM == A && c.TN == B && c.warps * 32 <= NT) {                                                   \
    BISP_CUDA(cudaFuncSetAttribute(k_pair<A, B, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem)); \
    k_pair<A, B, NT><<<c.nblk, c.warps * 32, c.smem, s>>>(c.nbp, c.bs, c.rows, c.ksplit, partials);           \
    launched = true;                                                                                     \
  }
#define BISP_PAIR(A, B) \
  if (!launched) BISP_PAIR3(A, B, 512) if (!launched) BISP_PAIR3(A, B, 1024)
#define BISP_PAIR_S(A, B) \
  if (!launched) BISP_PAIR3(A, B, 512)
  bool launched = false;
  BISP_PAIR(1, 1) BISP_PAIR(2, 1) BISP_PAIR(3, 2) BISP_PAIR(4, 2) BISP_PAIR(5, 3) BISP_PAIR(6, 3)
  BISP_PAIR_S(7, 4) BISP_PAIR_S(8, 4) BISP_PAIR_S(10, 5)
#undef BISP_PAIR
#undef BISP_PAIR_S
#undef BISP_PAIR3
  if (!launched) throw Error{6, "pair reduction: no kernel for this shape"};
  BISP_CHECK_LAUNCH();
  const int nout = j.nout * j.nb * j.nb;
  k_pair_final<<<(nout * 32 + 255) / 256, 256, 0, s>>>(partials, c.nblk, c.warps, c.ksplit, c.TM, c.TN, j.nb,
                                                       j.nout, out_dev);
  BISP_CHECK_LAUNCH();
  if (launches) *launches += 2;
}

}  // namespace bisp
