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
constexpr int PR_CH = 32;          // cells per chunk
constexpr int PR_LD = PR_CH + 4;   // padded row (bank spread for 16-byte loads)
constexpr int PR_FLUSH = 32;       // chunks per FP32 partial (<= 1024 cells)
constexpr int PR_NSTAGE = 3;       // chunks staged ahead
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
  while (c.ksplit < 2 && j.nterm * c.ksplit * 2 <= PR_MAXWARP) c.ksplit *= 2;  // slices of >= 16 cells
  c.warps = j.nterm * c.ksplit;
  c.bs = j.ncomp | 1;  // odd rows per bin: consecutive bins fall on different banks
  c.rows = c.nbp * c.bs + j.ng;
  c.smem = ((size_t)PR_NSTAGE * c.rows * PR_LD + (size_t)j.nslot * c.nbp * PR_LD + (size_t)j.nh * PR_CH) *
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

size_t pair_scratch_bytes(const PairJob& job) {
  const PairLaunch c = pair_launch_cfg(classify(job));
  return (size_t)c.nblk * c.warps * 32 * c.TM * c.TN * sizeof(double);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int NW>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NW)); }

// copy one chunk of every component row [b][comp] and G row into shared memory
__device__ __forceinline__ void pair_stage(float* raw, int64_t x0, int nbp, int bs) {
  const PairJob& J = c_pj;
  constexpr int Q = PR_CH / 4;
  const int nraw = J.nb * J.ncomp;
  const int n = (nraw + J.ng) * Q;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int f = i / Q, q = i % Q;
    const float* src;
    int row;
    if (f < nraw) {
      src = J.fields + (size_t)f * J.Ng + x0 + 4 * q;
      const int b = f / J.ncomp;
      row = b * bs + (f - b * J.ncomp);
    } else {
      src = J.gfields + (size_t)(f - nraw) * J.Ng + x0 + 4 * q;
      row = nbp * bs + (f - nraw);
    }
    cp_async16(raw + (size_t)row * PR_LD + 4 * q, src);
  }
}

template <int TM, int TN, int NTHR>
__global__ void __launch_bounds__(NTHR, 1) k_pair(int nbp, int bs, int rows, int ksplit, double* partials) {
  const PairJob& J = c_pj;
  extern __shared__ __align__(16) float sh[];
  float* mat = sh + (size_t)PR_NSTAGE * rows * PR_LD;  // [nslot][nbp][PR_LD], then H rows
  const int grow0 = nbp * bs;
  const int64_t nchunk = J.Ng / PR_CH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int t = warp / ksplit, ks = warp % ksplit;
  const int slice = PR_CH / ksplit;
  const int b1 = lane >> 3, b2 = lane & 7;  // rows b1 + 4 i and b2 + 8 j
  const PairTermDesc T = J.term[t];
  double* slot = partials + (((size_t)blockIdx.x * nwarp + warp) * 32 + lane) * (TM * TN);
#pragma unroll
  for (int q = 0; q < TM * TN; ++q) slot[q] = 0.0;
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  // prologue: the first PR_NSTAGE - 1 chunks
  int64_t chs[PR_NSTAGE];
#pragma unroll
  for (int s = 0; s < PR_NSTAGE - 1; ++s) {
    chs[s] = blockIdx.x + (int64_t)s * gridDim.x;
    if (chs[s] < nchunk) pair_stage(sh + (size_t)s * rows * PR_LD, chs[s] * PR_CH, nbp, bs);
    cp_async_commit();
  }
  int since_flush = 0, stage = 0;
  for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    cp_async_wait<PR_NSTAGE - 2>();
    __syncthreads();  // chunk ch has landed; every warp is done with the previous chunk
    {
      const int64_t nx = ch + (int64_t)(PR_NSTAGE - 1) * gridDim.x;
      const int ns = (stage + PR_NSTAGE - 1) % PR_NSTAGE;
      if (nx < nchunk) pair_stage(sh + (size_t)ns * rows * PR_LD, nx * PR_CH, nbp, bs);
      cp_async_commit();
    }
    const float* raw = sh + (size_t)stage * rows * PR_LD;
    // built sides: H_h(x) = sum coef G_g(x) (shared by all bins), then
    // mat[slot][b][x] = sum_(c,h) P_c(b, x) H_h(x); four cells per thread
    if (J.nslot) {
      float* Hs = mat + (size_t)J.nslot * nbp * PR_LD;  // [nh][PR_CH]
      constexpr int Q = PR_CH / 4;
      for (int i = threadIdx.x; i < J.nh * Q; i += blockDim.x) {
        const int h = i / Q, q = i % Q;
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
      const int per_slot = J.nb * Q;
      for (int i = threadIdx.x; i < J.nslot * per_slot; i += blockDim.x) {
        const int sl = i / per_slot, r = i - sl * per_slot;
        const int b = r / Q, q = r % Q;
        const float* rb = raw + (size_t)b * bs * PR_LD + 4 * q;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int e = J.s_off[sl]; e < J.s_off[sl + 1]; ++e) {
          const int c = J.s_ent[e][0], h = J.s_ent[e][1];
          const float4 pv = *reinterpret_cast<const float4*>(rb + (size_t)c * PR_LD);
          const float4 hv = *reinterpret_cast<const float4*>(Hs + (size_t)h * PR_CH + 4 * q);
          v.x = fmaf(pv.x, hv.x, v.x);
          v.y = fmaf(pv.y, hv.y, v.y);
          v.z = fmaf(pv.z, hv.z, v.z);
          v.w = fmaf(pv.w, hv.w, v.w);
        }
        *reinterpret_cast<float4*>(mat + ((size_t)sl * nbp + b) * PR_LD + 4 * q) = v;
      }
      __syncthreads();
    }
    const float* xr;
    const float* yr;
    int sx, sy;
    if (T.xdir >= 0) {
      xr = raw + (size_t)(b1 * bs + T.xdir) * PR_LD;
      sx = 4 * bs * PR_LD;
    } else {
      xr = mat + ((size_t)T.xslot * nbp + b1) * PR_LD;
      sx = 4 * PR_LD;
    }
    if (T.ydir >= 0) {
      yr = raw + (size_t)(b2 * bs + T.ydir) * PR_LD;
      sy = 8 * bs * PR_LD;
    } else {
      yr = mat + ((size_t)T.yslot * nbp + b2) * PR_LD;
      sy = 8 * PR_LD;
    }
    xr += ks * slice;
    yr += ks * slice;
    for (int xb = 0; xb < slice; xb += 16) {
#pragma unroll
      for (int x = xb; x < xb + 16; x += 4) {
        float4 a[TM], c[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = *reinterpret_cast<const float4*>(xr + i * sx + x);
#pragma unroll
        for (int j = 0; j < TN; ++j) c[j] = *reinterpret_cast<const float4*>(yr + j * sy + x);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            float s = acc[i][j];
            s = fmaf(a[i].x, c[j].x, s);
            s = fmaf(a[i].y, c[j].y, s);
            s = fmaf(a[i].z, c[j].z, s);
            s = fmaf(a[i].w, c[j].w, s);
            acc[i][j] = s;
          }
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
    stage = (stage + 1) % PR_NSTAGE;
  }
  cp_async_wait<0>();
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
