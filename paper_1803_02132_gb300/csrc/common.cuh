// Shared device helpers of the bispectrum kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define BISP_NMAX 1024          // largest mesh side
#define BISP_TWN 2048           // twiddle table resolution (2 BISP_NMAX: half-cell phases)
#define BISP_LMAX 4             // largest l, L handled by the kernels

namespace bisp {

// Checked build (compiled with -DBISP_CHECKED, relocatable device code): BISP_DCHECK(cond, site)
// is the condition itself, and a false condition records (site << 32) | (low 32 bits of the
// value passed as `what`) in the device word g_bisp_check unless an earlier failure is recorded;
// the caller skips the guarded access.  The release build compiles every check to `true`.  The
// host reads and clears the word with bisp_check_word().
#ifdef BISP_CHECKED
extern __device__ unsigned long long g_bisp_check;
__device__ __forceinline__ bool bisp_dcheck(bool ok, unsigned site, unsigned long long what) {
  if (!ok) atomicCAS(&g_bisp_check, 0ull, ((unsigned long long)site << 32) | (what & 0xffffffffull) | 1ull << 31);
  return ok;
}
#define BISP_DCHECK(cond, site, what) ::bisp::bisp_dcheck((cond), (site), (unsigned long long)(what))
#else
#define BISP_DCHECK(cond, site, what) true
#endif

// Twiddles: kernels take `tw`, a device table of e^{-2 pi i j / BISP_TWN}, j < BISP_TWN,
// rounded to FP32 from FP64 values computed on the host.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by s*i (s = +1 or -1)
template <int S>
__device__ __forceinline__ float2 cmul_si(float2 a) { return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x); }

// ---------------------------------------------------------------------------------
// Normalised spherical harmonics y_l^m (App. A, Eq. YL), m >= 0, Condon-Shortley phase:
// y_l^m = sqrt((l-m)!/(l+m)!) Pt_l^m(mu) ((x + i y)/r)^m, where Pt_l^m is the associated
// Legendre function with the (1-mu^2)^{m/2} factor removed:
//   Pt_m^m = (-1)^m (2m-1)!!,  Pt_{m+1}^m = (2m+1) mu Pt_m^m,
//   (l-m) Pt_l^m = (2l-1) mu Pt_{l-1}^m - (l+m-1) Pt_{l-2}^m.
// ynorm[l][m] = sqrt((l-m)!/(l+m)!) is passed in (computed in FP64 on the host).
// Returns y for all (l, m) with l <= lmax, m <= l into out[l*(l+1)/2 + m].
// ---------------------------------------------------------------------------------
template <int LMAX>
__device__ __forceinline__ void ylm_all(float x, float y, float z, const float* __restrict__ ynorm,
                                        float2* out) {
  const float r2 = x * x + y * y + z * z;
  const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
  const float mu = z * rinv;
  const float2 e1 = make_float2(x * rinv, y * rinv);
  float2 ep = make_float2(1.f, 0.f);  // ((x+iy)/r)^m
#pragma unroll
  for (int m = 0; m <= LMAX; ++m) {
    float pmm = 1.f;  // (-1)^m (2m-1)!!
#pragma unroll
    for (int k = 1; k <= m; ++k) pmm *= -(2.f * k - 1.f);
    float p_lm2 = 0.f, p_lm1 = pmm;
#pragma unroll
    for (int l = m; l <= LMAX; ++l) {
      float p;
      if (l == m) p = pmm;
      else if (l == m + 1) p = (2.f * m + 1.f) * mu * pmm;
      else p = ((2.f * l - 1.f) * mu * p_lm1 - (float)(l + m - 1) * p_lm2) / (float)(l - m);
      if (l > m) { p_lm2 = p_lm1; p_lm1 = p; }
      const float a = ynorm[l * (BISP_LMAX + 1) + m] * p;
      out[l * (l + 1) / 2 + m] = make_float2(a * ep.x, a * ep.y);
    }
    ep = cmul(ep, e1);
  }
  if (r2 == 0.f) {
#pragma unroll
    for (int i = 1; i < (LMAX + 1) * (LMAX + 2) / 2; ++i) out[i] = make_float2(0.f, 0.f);
    out[0] = make_float2(1.f, 0.f);
  }
}

// ---------------------------------------------------------------------------------
// In-place complex FFT of LB interleaved lines of length NF held in shared memory,
// s[e * LB + l] = element e of line l.  Stockham autosort, radix 8 (then 4 or 2), each
// thread holding 8 values per stage; blockDim.x == LB * NF / 8.  SIGN = -1 forward
// (e^{-2 pi i n k / NF}), +1 inverse; both unnormalised.
// ---------------------------------------------------------------------------------
template <int R, int SIGN>
__device__ __forceinline__ void dft_r(float2* a) {
  if (R == 2) {
    float2 t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  } else if (R == 4) {
    float2 s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
    float2 s13 = cadd(a[1], a[3]), d13 = cmul_si<SIGN>(csub(a[1], a[3]));
    a[0] = cadd(s02, s13);
    a[2] = csub(s02, s13);
    a[1] = cadd(d02, d13);
    a[3] = csub(d02, d13);
  } else if (R == 8) {
    float2 e[4] = {a[0], a[2], a[4], a[6]};
    float2 o[4] = {a[1], a[3], a[5], a[7]};
    dft_r<4, SIGN>(e);
    dft_r<4, SIGN>(o);
    const float h = 0.70710678118654752440f;
    // W8^k = e^{SIGN 2 pi i k / 8}
    float2 o1 = cmul(o[1], make_float2(h, SIGN * h));
    float2 o2 = cmul_si<SIGN>(o[2]);
    float2 o3 = cmul(o[3], make_float2(-h, SIGN * h));
    a[0] = cadd(e[0], o[0]);
    a[4] = csub(e[0], o[0]);
    a[1] = cadd(e[1], o1);
    a[5] = csub(e[1], o1);
    a[2] = cadd(e[2], o2);
    a[6] = csub(e[2], o2);
    a[3] = cadd(e[3], o3);
    a[7] = csub(e[3], o3);
  }
}

// One Stockham stage (radix R, current sub-transform length NS), then the rest.
template <int NF, int LB, int SIGN, int NS, int REM>
struct FftStage {
  static __device__ __forceinline__ void run(float2* s, const float2* __restrict__ tw, int ldl, int l, int t) {
    constexpr int R = REM >= 8 ? 8 : REM;
    constexpr int T = NF / 8;   // threads per line
    constexpr int NQ = 8 / R;   // butterflies per thread
    float2 v[8];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int r = 0; r < R; ++r) v[q * R + r] = s[(t + q * T + r * (NF / R)) * ldl + l];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int j = t + q * T;
      const int k = j & (NS - 1);
      constexpr int tstep = (NF / (NS * R)) * (BISP_TWN / NF);
      if (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[(r * k * tstep) & (BISP_TWN - 1)];
          if (SIGN > 0) w.y = -w.y;
          v[q * R + r] = cmul(v[q * R + r], w);
        }
      }
      dft_r<R, SIGN>(v + q * R);
      const int idxD = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) s[(idxD + r * NS) * ldl + l] = v[q * R + r];
    }
    __syncthreads();
    FftStage<NF, LB, SIGN, NS * R, REM / R>::run(s, tw, ldl, l, t);
  }
};
template <int NF, int LB, int SIGN, int NS>
struct FftStage<NF, LB, SIGN, NS, 1> {
  static __device__ __forceinline__ void run(float2*, const float2* __restrict__, int, int, int) {}
};

template <int NF, int LB, int SIGN>
__device__ __forceinline__ void fft_smem(float2* s, const float2* __restrict__ tw, int ldl = LB) {
  static_assert(NF >= 8 && (NF & (NF - 1)) == 0, "NF");
  FftStage<NF, LB, SIGN, 1, NF>::run(s, tw, ldl, threadIdx.x % LB, threadIdx.x / LB);
}

// ---------------------------------------------------------------------------------
// In-register DFT of R = 2..32 points (R a power of two), radix-2 decimation in time,
// unnormalised, sign SIGN: X[k] = sum_n v[n] e^{SIGN 2 pi i n k / R}; tw is the twiddle
// table e^{-2 pi i j / BISP_TWN}.
// ---------------------------------------------------------------------------------

// o * w^j, w = e^{SIGN 2 pi i / 32}, j < 16 a compile-time constant after unrolling: the
// trivial twiddles (1 and +-i) cost no multiplies; the others are literal constants,
// cos(2 pi j / 32) and sin(2 pi j / 32) rounded to FP32.
__host__ __device__ constexpr float root32_cos(int j) {
  return j == 0 ? 1.0f : j == 1 ? 0.98078525f : j == 2 ? 0.92387953f : j == 3 ? 0.83146961f :
         j == 4 ? 0.70710677f : j == 5 ? 0.55557024f : j == 6 ? 0.38268343f : j == 7 ? 0.19509032f :
         j == 8 ? 0.0f : j == 9 ? -0.19509032f : j == 10 ? -0.38268343f : j == 11 ? -0.55557024f :
         j == 12 ? -0.70710677f : j == 13 ? -0.83146961f : j == 14 ? -0.92387953f : -0.98078525f;
}
__host__ __device__ constexpr float root32_sin(int j) { return j <= 8 ? root32_cos(8 - j) : root32_cos(j - 8); }
template <int SIGN>
__device__ __forceinline__ float2 twiddle32(int j, float2 o) {
  if (j == 0) return o;
  if (j == 8) return SIGN > 0 ? make_float2(-o.y, o.x) : make_float2(o.y, -o.x);
  const float c = root32_cos(j), sn = SIGN > 0 ? root32_sin(j) : -root32_sin(j);
  return make_float2(fmaf(c, o.x, -sn * o.y), fmaf(c, o.y, sn * o.x));
}

template <int R, int SIGN>
struct DftReg {
  static __device__ __forceinline__ void run(float2* v, const float2* __restrict__ tw) {
    float2 e[R / 2], o[R / 2];
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      e[k] = v[2 * k];
      o[k] = v[2 * k + 1];
    }
    DftReg<R / 2, SIGN>::run(e, tw);
    DftReg<R / 2, SIGN>::run(o, tw);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      const float2 t = twiddle32<SIGN>(k * (32 / R), o[k]);
      v[k] = cadd(e[k], t);
      v[k + R / 2] = csub(e[k], t);
    }
  }
};
template <int SIGN>
struct DftReg<1, SIGN> {
  static __device__ __forceinline__ void run(float2*, const float2* __restrict__) {}
};

}  // namespace bisp
