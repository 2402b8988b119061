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
  const long long qlo = A.qlo[b], qhi = A.qhi[b];
  int P = (int)floor(sqrt((double)(qhi - 1)));
  if (P > A.N / 2 - 1) P = A.N / 2 - 1;
  const int N = A.N, NH = N / 2;
  const int ny_ = 2 * P + 1;
  const long long nmode = (long long)ny_ * ny_ * (P + 1);
  double acc[ZS_MAXLM][2];
#pragma unroll
  for (int q = 0; q < ZS_MAXLM; ++q) acc[q][0] = acc[q][1] = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nmode; i += (long long)gridDim.x * blockDim.x) {
    const int nz = (int)(i % (P + 1));
    const int sy = (int)((i / (P + 1)) % ny_) - P;
    const int sx = (int)(i / ((long long)(P + 1) * ny_)) - P;
    const long long q = (long long)sx * sx + (long long)sy * sy + (long long)nz * nz;
    if (q < qlo || q >= qhi) continue;
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
// ------------------------------------------------------------------------------------
__constant__ PairJob c_pj;
constexpr int PR_THREADS = 256;
constexpr int PR_CH = 32;          // cells per chunk
constexpr int PR_LD = PR_CH + 4;   // padded row (bank spread for 16-byte loads)
constexpr int PR_FLUSH = 32;       // chunks per FP32 partial (<= 1024 cells)
constexpr int PR_IPT = 2;          // work items per thread

struct PairLaunch {
  int nbp;      // nb rounded up to 4
  int ntile;    // nbp / 4
  int units;    // nout * ntile^2
  int ksplit;   // x slices per chunk
  int items;    // units * ksplit (<= PR_IPT * PR_THREADS)
  int nblk;
  size_t smem;
};

static PairLaunch pair_launch_cfg(const PairJob& j) {
  PairLaunch c;
  c.nbp = (j.nb + 3) / 4 * 4;
  c.ntile = c.nbp / 4;
  c.units = j.nout * c.ntile * c.ntile;
  c.ksplit = 1;
  while (c.ksplit < 8 && c.units * c.ksplit * 2 <= PR_IPT * PR_THREADS) c.ksplit *= 2;
  c.items = c.units * c.ksplit;
  if (c.items > PR_IPT * PR_THREADS) throw Error{6, "pair reduction: too many outputs for one CTA"};
  c.nblk = 2 * 152;
  c.smem = ((size_t)2 * j.nterm * c.nbp * PR_LD + (size_t)(j.nb * j.ncomp + j.ng) * PR_CH) * sizeof(float);
  return c;
}

size_t pair_scratch_bytes(const PairJob& j) {
  const PairLaunch c = pair_launch_cfg(j);
  return (size_t)c.nblk * c.items * 16 * sizeof(double);
}

__global__ void __launch_bounds__(PR_THREADS) k_pair(int nbp, int ntile, int ksplit, int items, double* partials) {
  const PairJob& J = c_pj;
  extern __shared__ float sh[];
  float* Xs = sh;                                  // [nterm][nbp][PR_LD]
  float* Ys = sh + (size_t)J.nterm * nbp * PR_LD;  // [nterm][nbp][PR_LD]
  float* raw = Ys + (size_t)J.nterm * nbp * PR_LD; // [nb*ncomp + ng][PR_CH]
  const int nraw = J.nb * J.ncomp;
  const int64_t nchunk = J.Ng / PR_CH;
  // zero padded rows once
  for (int i = threadIdx.x; i < 2 * J.nterm * nbp * PR_LD; i += blockDim.x) sh[i] = 0.f;
  __syncthreads();
  // work items of this thread
  int it_o[PR_IPT], it_b1[PR_IPT], it_b2[PR_IPT], it_x0[PR_IPT];
  bool it_ok[PR_IPT];
  const int slice = PR_CH / ksplit;
#pragma unroll
  for (int k = 0; k < PR_IPT; ++k) {
    const int w = threadIdx.x + k * PR_THREADS;
    it_ok[k] = w < items;
    const int u = w / ksplit, ks = w % ksplit;
    const int o = u / (ntile * ntile), r = u % (ntile * ntile);
    it_o[k] = it_ok[k] ? o : 0;
    it_b1[k] = 4 * (r / ntile);
    it_b2[k] = 4 * (r % ntile);
    it_x0[k] = ks * slice;
  }
  float acc[PR_IPT][16];
  double acc64[PR_IPT][16];
#pragma unroll
  for (int k = 0; k < PR_IPT; ++k)
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[k][q] = 0.f, acc64[k][q] = 0.0;
  int since_flush = 0;
  for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    const int64_t x0 = ch * PR_CH;
    __syncthreads();
    // stage the chunk of every field component and G field (one coalesced read each)
    for (int i = threadIdx.x; i < (nraw + J.ng) * PR_CH; i += blockDim.x) {
      const int f = i / PR_CH, x = i % PR_CH;
      raw[i] = f < nraw ? __ldg(J.fields + (size_t)f * J.Ng + x0 + x)
                        : __ldg(J.gfields + (size_t)(f - nraw) * J.Ng + x0 + x);
    }
    __syncthreads();
    // build the two sides of every term for this chunk
    const int per_side = J.nb * PR_CH;
    for (int i = threadIdx.x; i < 2 * J.nterm * per_side; i += blockDim.x) {
      const int x = i % PR_CH;
      const int b = (i / PR_CH) % J.nb;
      const int ts = i / per_side;  // term * 2 + side
      const int t = ts >> 1, side = ts & 1;
      const PairTermDesc& T = J.term[t];
      const int off = side ? T.yoff : T.xoff, cnt = side ? T.ycnt : T.xcnt;
      float v = 0.f;
      for (int e = 0; e < cnt; ++e) {
        const PairRecipe R = J.rec[off + e];
        float f = raw[(b * J.ncomp + R.comp) * PR_CH + x];
        if (R.g >= 0) f *= raw[(nraw + R.g) * PR_CH + x];
        v = fmaf(R.coef, f, v);
      }
      (side ? Ys : Xs)[((size_t)t * nbp + b) * PR_LD + x] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PR_IPT; ++k) {
      if (!it_ok[k]) continue;
      const int o = it_o[k];
      for (int t = J.out_term_off[o]; t < J.out_term_off[o + 1]; ++t) {
        const float* xr = Xs + ((size_t)t * nbp + it_b1[k]) * PR_LD + it_x0[k];
        const float* yr = Ys + ((size_t)t * nbp + it_b2[k]) * PR_LD + it_x0[k];
        for (int x = 0; x < slice; x += 4) {
          float4 a[4], c[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            a[i] = *reinterpret_cast<const float4*>(xr + i * PR_LD + x);
            c[i] = *reinterpret_cast<const float4*>(yr + i * PR_LD + x);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              float s = acc[k][i * 4 + j];
              s = fmaf(a[i].x, c[j].x, s);
              s = fmaf(a[i].y, c[j].y, s);
              s = fmaf(a[i].z, c[j].z, s);
              s = fmaf(a[i].w, c[j].w, s);
              acc[k][i * 4 + j] = s;
            }
        }
      }
    }
    if (++since_flush == PR_FLUSH) {
      since_flush = 0;
#pragma unroll
      for (int k = 0; k < PR_IPT; ++k)
#pragma unroll
        for (int q = 0; q < 16; ++q) acc64[k][q] += (double)acc[k][q], acc[k][q] = 0.f;
    }
  }
#pragma unroll
  for (int k = 0; k < PR_IPT; ++k) {
    const int w = threadIdx.x + k * PR_THREADS;
    if (w >= items) continue;
#pragma unroll
    for (int q = 0; q < 16; ++q)
      partials[((size_t)blockIdx.x * items + w) * 16 + q] = acc64[k][q] + (double)acc[k][q];
  }
}

// out[o][b1][b2] = sum over CTAs (in order) and k slices (in order)
__global__ void k_pair_final(const double* partials, int nblk, int items, int ksplit, int ntile, int nb, int nout,
                             double* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nout * nb * nb) return;
  const int o = idx / (nb * nb), b1 = (idx / nb) % nb, b2 = idx % nb;
  const int u = (o * ntile + b1 / 4) * ntile + b2 / 4;
  const int q = (b1 % 4) * 4 + (b2 % 4);
  double s = 0.0;
  for (int c = 0; c < nblk; ++c)
    for (int ks = 0; ks < ksplit; ++ks) s += partials[((size_t)c * items + u * ksplit + ks) * 16 + q];
  out[idx] = s;
}

void pair_reduce(const PairJob& job, double* out_dev, void* scratch, size_t scratch_bytes, cudaStream_t s,
                 int* launches) {
  const PairLaunch c = pair_launch_cfg(job);
  if (scratch_bytes < pair_scratch_bytes(job)) throw Error{2, "pair reduction scratch too small"};
  if (job.Ng % PR_CH) throw Error{6, "mesh size not a multiple of the chunk"};
  BISP_CUDA(cudaMemcpyToSymbolAsync(c_pj, &job, sizeof(PairJob), 0, cudaMemcpyHostToDevice, s));
  if (c.smem > 48 * 1024)
    BISP_CUDA(cudaFuncSetAttribute(k_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem));
  double* partials = reinterpret_cast<double*>(scratch);
  k_pair<<<c.nblk, PR_THREADS, c.smem, s>>>(c.nbp, c.ntile, c.ksplit, c.items, partials);
  BISP_CHECK_LAUNCH();
  const int nout = job.nout * job.nb * job.nb;
  k_pair_final<<<(nout + 255) / 256, 256, 0, s>>>(partials, c.nblk, c.items, c.ksplit, c.ntile, job.nb, job.nout,
                                                  out_dev);
  BISP_CHECK_LAUNCH();
  if (launches) *launches += 2;
}

}  // namespace bisp
