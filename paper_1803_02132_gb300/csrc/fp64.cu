// Plain FP64 form of the estimator (Eq. bi_estimator_FFTs), a speed and accuracy baseline
// for the fused FP32 path: FP64 half spectra (shell filter, y_l^{m*} weight, shot-noise
// source), full cuFFT Z2D transforms, and one FP64 mesh sum per (bin pair, 3j term) that
// reads its three fields from HBM.  Nothing here is blocked, pruned or fused.
#include <cufft.h>

#include "common.cuh"
#include "internal.h"

namespace bisp {

namespace {

// y_l^m(n), m >= 0, FP64: the associated-Legendre recurrence of App. A (Eq. YL) with the
// (1 - mu^2)^{m/2} factor carried by ((x + i y)/r)^m; ynorm[l][m] = sqrt((l-m)!/(l+m)!).
__device__ double2 ylm_d(int l, int m, double x, double y, double z, const double* __restrict__ ynorm) {
  const double r2 = x * x + y * y + z * z;
  if (r2 == 0.0) return l == 0 ? make_double2(1.0, 0.0) : make_double2(0.0, 0.0);
  const double rinv = 1.0 / sqrt(r2);
  const double mu = z * rinv;
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
  const double cx = x * rinv, cy = y * rinv;
  for (int k = 0; k < m; ++k) {
    const double t = er * cx - ei * cy;
    ei = er * cy + ei * cx;
    er = t;
  }
  const double a = ynorm[l * (BISP_LMAX + 1) + m] * p;
  return make_double2(a * er, a * ei);
}

// One FP64 half spectrum [N][N][N/2+1] (cuFFT's c2r input) from the FP32 half spectra
// [N][N][N/2]; modes with a component on a Nyquist plane are zero.
__global__ void k_f64_spec(F64Spec S, F64Tables T, int N, double2* __restrict__ out) {
  const int NH = N / 2, NZ = NH + 1;
  const int64_t total = (int64_t)N * N * NZ;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int iz = (int)(i % NZ);
    const int64_t r = i / NZ;
    const int iy = (int)(r % N), ix = (int)(r / N);
    const int sx = ix < NH ? ix : ix - N, sy = iy < NH ? iy : iy - N;
    double2 v = make_double2(0.0, 0.0);
    if (iz < NH && sx != -NH && sy != -NH) {
      const size_t gi = ((size_t)ix * N + iy) * NH + iz;
      if (S.kind == SRC_PLAIN) {
        const float2 a = S.A[gi];
        v = make_double2(S.scale * a.x, S.scale * a.y);
      } else if (S.kind == SRC_QSHOT) {
        // A conj(B) - Sbar C(k)/W^2(k), the alias sum of the shot-noise power (Eq. shotnoise)
        const float2 a = S.A[gi], b = S.B[gi];
        const double re = (double)a.x * b.x + (double)a.y * b.y;
        const double im = (double)a.y * b.x - (double)a.x * b.y;
        double c = T.cw2[ix] * T.cw2[iy] * T.cw2[iz];
        if (T.interlace) c = 0.5 * (c + T.cw2[N + ix] * T.cw2[N + iy] * T.cw2[N + iz]);
        v = make_double2((re - S.sbar * c) * S.scale, im * S.scale);
      } else {
        // shell b: (1/N_mode) (-i)^l part(y_l^{m*}(k)) (Delta(k) or 1)  (Eq. bi_estimator_FFTs)
        const long long q = (long long)sx * sx + (long long)sy * sy + (long long)iz * iz;
        if (q >= S.qlo && q < S.qhi) {
          double2 a = make_double2(1.0, 0.0);
          if (!S.unit) {
            const float2 af = S.A[gi];
            a = make_double2(af.x, af.y);
          }
          const double2 y = ylm_d(S.l, S.m, sx, sy, iz, T.ynorm);
          const double c = (S.part ? -y.y : y.x) * S.inv_nmodes;
          const double tr = a.x * c, ti = a.y * c;
          switch (S.l & 3) {
            case 0: v = make_double2(tr, ti); break;
            case 1: v = make_double2(ti, -tr); break;
            case 2: v = make_double2(-tr, -ti); break;
            default: v = make_double2(-ti, tr); break;
          }
        }
      }
    }
    out[i] = v;
  }
}

constexpr int DOT_THREADS = 256;

// partial[blockIdx.x] = sum over this block's cells of a b c (FP64, fixed order)
__global__ void __launch_bounds__(DOT_THREADS) k_f64_dot3(const double2* __restrict__ a,
                                                          const double2* __restrict__ b,
                                                          const double2* __restrict__ c, int64_t n2,
                                                          double* __restrict__ partial) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)DOT_THREADS + threadIdx.x; i < n2; i += (int64_t)gridDim.x * DOT_THREADS) {
    const double2 x = a[i], y = b[i], z = c[i];
    s = fma(x.x * y.x, z.x, s);
    s = fma(x.y * y.y, z.y, s);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double ws[DOT_THREADS / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < DOT_THREADS / 32; ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

// out[d] = sum over blocks of partial[d][blk], in block order
__global__ void k_f64_final(const double* __restrict__ partial, int nblk, int nd, double* __restrict__ out) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= nd) return;
  double t = 0.0;
  for (int k = 0; k < nblk; ++k) t += partial[(size_t)d * nblk + k];
  out[d] = t;
}

void cufft_check(cufftResult r, const char* what) {
  if (r != CUFFT_SUCCESS) throw Error{3, std::string(what) + ": cuFFT error " + std::to_string((int)r)};
}

}  // namespace

void f64_spectrum(const F64Spec& s, const F64Tables& t, int N, double2* out, cudaStream_t st) {
  int sms = 0, dev = 0;
  BISP_CUDA(cudaGetDevice(&dev));
  BISP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  k_f64_spec<<<sms * 8, 256, 0, st>>>(s, t, N, out);
  BISP_CHECK_LAUNCH();
}

F64Fft f64_fft_create(int N) {
  F64Fft f;
  cufftHandle h;
  cufft_check(cufftCreate(&h), "cufftCreate");
  f.handle = (long long)h;
  cufft_check(cufftSetAutoAllocation(h, 0), "cufftSetAutoAllocation");
  size_t ws = 0;
  cufft_check(cufftMakePlan3d(h, N, N, N, CUFFT_Z2D, &ws), "cufftMakePlan3d");
  f.work_bytes = ws;
  return f;
}

void f64_fft_c2r(const F64Fft& f, void* work, double2* in, double* out, cudaStream_t s) {
  const cufftHandle h = (cufftHandle)f.handle;
  cufft_check(cufftSetWorkArea(h, work), "cufftSetWorkArea");
  cufft_check(cufftSetStream(h, s), "cufftSetStream");
  cufft_check(cufftExecZ2D(h, reinterpret_cast<cufftDoubleComplex*>(in), out), "cufftExecZ2D");
}

void f64_fft_destroy(F64Fft& f) {
  if (f.handle >= 0) cufftDestroy((cufftHandle)f.handle);
  f.handle = -1;
}

int f64_dot_blocks() {
  int sms = 0, dev = 0;
  BISP_CUDA(cudaGetDevice(&dev));
  BISP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  return sms * 8;
}

void f64_dot3(const double* a, const double* b, const double* c, int64_t n, double* partial, int nblk,
              cudaStream_t s) {
  if (n % 2) throw Error{1, "f64_dot3: odd length"};
  k_f64_dot3<<<nblk, DOT_THREADS, 0, s>>>(reinterpret_cast<const double2*>(a), reinterpret_cast<const double2*>(b),
                                          reinterpret_cast<const double2*>(c), n / 2, partial);
  BISP_CHECK_LAUNCH();
}

void f64_dot_final(const double* partial, int nblk, int nd, double* out, cudaStream_t s) {
  if (nd <= 0) return;
  k_f64_final<<<(nd + 255) / 256, 256, 0, s>>>(partial, nblk, nd, out);
  BISP_CHECK_LAUNCH();
}

}  // namespace bisp
