// Measurement kernels:
//  * k_axpby: the spectra of one estimator pass, delta n = D_gal - alpha D_ran (Eq. dn)
//    and N = N_gal + alpha^2 N_ran (Eq. ShotNoise definitions);
//  * k_zsum: shell sums (1/N_mode) sum_shell y_l^{m*}(k) [D(k) N_L^{M*}(k) -
//    Sbar_L^M C(k)/W^2(k)] of the i!=j=k and i=k!=j shot-noise terms (Eq. ShotNoise);
//  (the mesh sum of Eq. bi_estimator_FFTs is in pair.cu).
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
constexpr int ZS_THREADS = 256;
constexpr int ZS_MAXLM = 9;

__device__ __forceinline__ float2 ystar(int l, int m, float x, float y, float z, const float* ynorm);

// FP32 per-mode arithmetic (FMA-contracted, relative error ~1e-7 of |D N*| per mode) with
// Kahan-compensated FP32 sums per thread; FP64 above the thread level.  GB300's FP64 rate
// is a small fraction of its FP32 rate, so FP64 per-mode arithmetic bound this kernel.
__device__ __forceinline__ void zs_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// the job is a __grid_constant__ parameter (each launch carries its own copy)
__global__ void __launch_bounds__(ZS_THREADS) k_zsum(const __grid_constant__ ZsumArgs A) {
  const int b = blockIdx.y;
  const int N = A.N, NH = N / 2;
  const int64_t m0 = A.mode_off[b], m1 = A.mode_off[b + 1];
  float acc[ZS_MAXLM][2], cmp[ZS_MAXLM][2];
#pragma unroll
  for (int q = 0; q < ZS_MAXLM; ++q) acc[q][0] = acc[q][1] = cmp[q][0] = cmp[q][1] = 0.f;
  const float sr = (float)A.sbar_re, si = (float)A.sbar_im;
  for (int64_t i = m0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m1; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t code = A.modes[i];
    const int sx = (int)(code & 1023u) - 512, sy = (int)((code >> 10) & 1023u) - 512, nz = (int)(code >> 20);
    const int jx = sx & (N - 1), jy = sy & (N - 1);
    const size_t gi = ((size_t)jx * N + jy) * NH + nz;
    if (!BISP_DCHECK(nz < NH && i >= 0, 10, gi)) continue;
    const float2 xr = A.XR[gi];
    const float2 xi = A.XI ? A.XI[gi] : make_float2(0.f, 0.f);
    const float2 nr = A.NR[gi];
    const float2 ni = A.NI ? A.NI[gi] : make_float2(0.f, 0.f);
    // X(k) = XR + i XI, X(-k) = conj(XR) + i conj(XI); the same for N (spectra of real meshes)
    const float xkr = xr.x - xi.y, xki = xr.y + xi.x;
    const float xmr = xr.x + xi.y, xmi = xi.x - xr.y;
    const float nkr = nr.x - ni.y, nki = nr.y + ni.x;
    const float nmr = nr.x + ni.y, nmi = ni.x - nr.y;
    float cw = A.cw2_1d[jx] * A.cw2_1d[jy] * A.cw2_1d[nz];
    if (A.interlace) cw = 0.5f * (cw + A.cw2_1d[N + jx] * A.cw2_1d[N + jy] * A.cw2_1d[N + nz]);
    // T(k) = X(k) conj(N(k)) - Sbar C/W^2
    const float tkr = fmaf(xkr, nkr, fmaf(xki, nki, -sr * cw));
    const float tki = fmaf(xki, nkr, fmaf(-xkr, nki, -si * cw));
    // T(-k) = X(-k) conj(N(-k)) - Sbar C/W^2
    const float tmr = fmaf(xmr, nmr, fmaf(xmi, nmi, -sr * cw));
    const float tmi = fmaf(xmi, nmr, fmaf(-xmr, nmi, -si * cw));
    const bool pair = nz > 0;
#pragma unroll
    for (int t = 0; t < ZS_MAXLM; ++t) {
      if (t < A.nlm) {
        const int l = A.lm[t][0], m = A.lm[t][1];
        const float2 ys = ystar(l, m, (float)sx, (float)sy, (float)nz, A.ynorm);
        const float yr = ys.x, yi = ys.y;
        float cr = fmaf(yr, tkr, -yi * tki), ci = fmaf(yr, tki, yi * tkr);
        if (pair) {  // y*(-k) = (-1)^l y*(k)
          const float sg = (l & 1) ? -1.f : 1.f;
          cr = fmaf(sg, fmaf(yr, tmr, -yi * tmi), cr);
          ci = fmaf(sg, fmaf(yr, tmi, yi * tmr), ci);
        }
        zs_add(acc[t][0], cmp[t][0], cr);
        zs_add(acc[t][1], cmp[t][1], ci);
      }
    }
  }
  __shared__ double red[ZS_THREADS / 32];
#pragma unroll
  for (int t = 0; t < ZS_MAXLM; ++t) {
    if (t >= A.nlm) break;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      double v = (double)acc[t][c] - (double)cmp[t][c];
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
  k_zsum<<<dim3(a.nblk, a.nbins), ZS_THREADS, 0, s>>>(a);
  BISP_CHECK_LAUNCH();
}


// real fields at the negated separations of the r-bins (three-point shot noise, Sec. 4.3)
__global__ void __launch_bounds__(256) k_gather_neg(const float* __restrict__ fields, int64_t Ng, int nf,
                                                     const uint32_t* __restrict__ offs, int64_t n, int N,
                                                     float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t o = offs[i];
    const int sx = 512 - (int)(o & 1023u), sy = 512 - (int)((o >> 10) & 1023u), sz = 512 - (int)((o >> 20) & 1023u);
    const size_t cell = ((size_t)(sx & (N - 1)) * N + (size_t)(sy & (N - 1))) * N + (size_t)(sz & (N - 1));
    if (!BISP_DCHECK(cell < (size_t)Ng, 11, cell)) continue;
    for (int c = 0; c < nf; ++c) out[i * nf + c] = fields[c * Ng + cell];
  }
}

void launch_gather_neg(const float* fields, int64_t Ng, int nf, const uint32_t* offs, int64_t n, int N, float* out,
                       cudaStream_t s) {
  if (n <= 0) return;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  k_gather_neg<<<blocks, 256, 0, s>>>(fields, Ng, nf, offs, n, N, out);
  BISP_CHECK_LAUNCH();
}

}  // namespace bisp
