// Hand-written batched 3D FFTs of the estimator (Sec. 4.2, Eq. nlm_bi):
//  * forward: real meshes -> deconvolved half spectra, three shared-memory passes
//    (z: real-to-complex, y, x).  The x pass also combines the interlaced pair and
//    divides by W_mass(k);
//  * inverse: half spectra -> real fields, pruned to the box |n_i| <= P that holds the
//    non-zero modes.  The first pass (x) builds the spectrum on the fly: a plain channel,
//    the shot-noise product Q = A conj(B) - Sbar C/W^2, or a k shell times
//    (-i)^l Re/Im y_l^{m*}(k) / N_mode (times the density or 1).
// Layout: real mesh [x][y][z] (z fastest); half spectrum [nx][ny][nz], nz < N/2 (the
// nz = N/2 plane is dropped: every spectrum is zero on the Nyquist planes).
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace bisp {

template <int N>
struct Geo {
  static constexpr int NH = N / 2;
  static constexpr int LB = (N >= 1024 || N < 32) ? 8 : 16;   // lines per CTA, strided passes
  static constexpr int LBZ = (N >= 1024 || N < 32) ? 8 : 16;  // rows per CTA, z passes
  static constexpr int TS = LB * N / 8;                       // threads, strided passes
  static constexpr int TZ = LBZ * NH / 8;                     // threads, z passes
};

__device__ __forceinline__ int sgn_idx(int j, int N) { return j < N / 2 ? j : j - N; }

// ------------------------------------------------------------------------------------
// forward z pass: rows of N reals -> N/2 complex (X[0] real, Nyquist dropped), in place
// ------------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Geo<N>::TZ) k_fwd_z(float* data, const float2* __restrict__ tw) {
  constexpr int NH = N / 2, LBZ = Geo<N>::LBZ, LD = LBZ + 1;
  __shared__ float2 s[NH * LD];
  float2* rows = reinterpret_cast<float2*>(data) + (size_t)blockIdx.x * LBZ * NH;
  for (int i = threadIdx.x; i < LBZ * NH; i += blockDim.x) {
    const int l = i / NH, e = i % NH;
    s[e * LD + l] = rows[(size_t)l * NH + e];
  }
  __syncthreads();
  fft_smem<NH, LBZ, -1>(s, tw, LD);
  // X[k] = (Z[k] + Z*[NH-k])/2 - i w^k (Z[k] - Z*[NH-k])/2,  w = e^{-2 pi i / N}
  for (int i = threadIdx.x; i < LBZ * (NH / 2 + 1); i += blockDim.x) {
    const int l = i % LBZ, k = i / LBZ;
    if (k == 0) {
      const float2 z0 = s[l];
      s[l] = make_float2(z0.x + z0.y, 0.f);
    } else {
      const int kp = NH - k;
      const float2 a = s[k * LD + l], b = s[kp * LD + l];
      const float2 wk = tw[k * (BISP_TWN / N)];
      const float2 wkp = tw[kp * (BISP_TWN / N)];
      // X[k]
      float2 sp = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));      // (a + b*)/2
      float2 dm = make_float2(0.5f * (a.x - b.x), 0.5f * (a.y + b.y));      // (a - b*)/2
      float2 t = cmul(wk, dm);
      const float2 xk = make_float2(sp.x + t.y, sp.y - t.x);                // sp - i t
      // X[kp]
      float2 sp2 = make_float2(0.5f * (b.x + a.x), 0.5f * (b.y - a.y));
      float2 dm2 = make_float2(0.5f * (b.x - a.x), 0.5f * (b.y + a.y));
      float2 t2 = cmul(wkp, dm2);
      const float2 xkp = make_float2(sp2.x + t2.y, sp2.y - t2.x);
      s[k * LD + l] = xk;
      if (kp != k) s[kp * LD + l] = xkp;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < LBZ * NH; i += blockDim.x) {
    const int l = i / NH, e = i % NH;
    rows[(size_t)l * NH + e] = s[e * LD + l];
  }
}

// ------------------------------------------------------------------------------------
// forward y pass: complex lines along y, in place.  data: [cnt][N][N][NH]
// ------------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Geo<N>::TS) k_fwd_y(float2* data, const float2* __restrict__ tw) {
  constexpr int NH = N / 2, LB = Geo<N>::LB;
  extern __shared__ float2 s[];
  const int nz0 = blockIdx.x * LB, x = blockIdx.y, mesh = blockIdx.z;
  float2* base = data + (((size_t)mesh * N + x) * N) * NH + nz0;
  for (int i = threadIdx.x; i < N * LB; i += blockDim.x) {
    const int l = i % LB, e = i / LB;
    s[i] = base[(size_t)e * NH + l];
  }
  __syncthreads();
  fft_smem<N, LB, -1>(s, tw);
  for (int i = threadIdx.x; i < N * LB; i += blockDim.x) {
    const int l = i % LB, e = i / LB;
    base[(size_t)e * NH + l] = s[i];
  }
}

// ------------------------------------------------------------------------------------
// forward x pass + interlacing + deconvolution, written over mesh0.
//   D = [ (D0 + e^{-i pi (nx+ny+nz)/N} D1) / 2 ] / W(k)   (ILV)   or   D0 / W(k)
// winv[j] = 1 / sinc(pi n_j / N)^p for the signed frequency of index j.  LB lines per CTA: with
// interlacing two meshes' lines sit in shared memory, so the pass takes half the strided passes'
// lines per CTA (more CTAs per SM).
// ------------------------------------------------------------------------------------
template <int N, int ILV>
struct FwdX {
  static constexpr int LB = ILV && Geo<N>::LB > 8 ? Geo<N>::LB / 2 : Geo<N>::LB;
  static constexpr int TS = LB * N / 8;
};
template <int N, int ILV>
__global__ void __launch_bounds__(FwdX<N, ILV>::TS) k_fwd_x(float2* m0, const float2* m1, const float2* __restrict__ tw,
                                                           const float* __restrict__ winv) {
  constexpr int NH = N / 2, LB = FwdX<N, ILV>::LB;
  extern __shared__ float2 sm[];  // dynamic: (1 + ILV) * N * LB
  float2* s0 = sm;
  float2* s1 = sm + N * LB;
  const int nz0 = blockIdx.x * LB, ny = blockIdx.y, mesh = blockIdx.z;
  const size_t moff = (size_t)mesh * N * N * NH;
  float2* b0 = m0 + moff + (size_t)ny * NH + nz0;
  const float2* b1 = ILV ? m1 + moff + (size_t)ny * NH + nz0 : nullptr;
  for (int i = threadIdx.x; i < N * LB; i += blockDim.x) {
    const int l = i % LB, e = i / LB;
    s0[i] = b0[(size_t)e * N * NH + l];
    if (ILV) s1[i] = b1[(size_t)e * N * NH + l];
  }
  __syncthreads();
  fft_smem<N, LB, -1>(s0, tw);
  if (ILV) fft_smem<N, LB, -1>(s1, tw);
  const int sy = sgn_idx(ny, N);
  const float wy = winv[ny];
  for (int i = threadIdx.x; i < N * LB; i += blockDim.x) {
    const int l = i % LB, e = i / LB;
    const int nz = nz0 + l;
    float2 v = s0[i];
    if (ILV) {
      const int ph = (sgn_idx(e, N) + sy + nz) * (BISP_TWN / (2 * N));
      const float2 p = tw[ph & (BISP_TWN - 1)];
      const float2 d1 = cmul(p, s1[i]);
      v = make_float2(0.5f * (v.x + d1.x), 0.5f * (v.y + d1.y));
    }
    const float wi = winv[e] * wy * winv[nz];
    v = make_float2(v.x * wi, v.y * wi);
    if (e == NH || ny == NH) v = make_float2(0.f, 0.f);
    b0[(size_t)e * N * NH + l] = v;
  }
}

template <typename K>
static void smem_attr(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    BISP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

template <int N>
static void fwd_impl(float* mesh0, float* mesh1, int count, int mas, const float2* tw, const float* winv,
                     cudaStream_t s, int* launches) {
  using G = Geo<N>;
  const int rows = count * N * N;
  k_fwd_z<N><<<rows / G::LBZ, G::TZ, 0, s>>>(mesh0, tw);
  BISP_CHECK_LAUNCH();
  if (mesh1) {
    k_fwd_z<N><<<rows / G::LBZ, G::TZ, 0, s>>>(mesh1, tw);
    BISP_CHECK_LAUNCH();
  }
  dim3 gy(G::NH / G::LB, N, count);
  const size_t s1 = (size_t)N * G::LB * sizeof(float2);
  smem_attr(k_fwd_y<N>, s1);
  k_fwd_y<N><<<gy, G::TS, s1, s>>>(reinterpret_cast<float2*>(mesh0), tw);
  BISP_CHECK_LAUNCH();
  if (mesh1) {
    k_fwd_y<N><<<gy, G::TS, s1, s>>>(reinterpret_cast<float2*>(mesh1), tw);
    BISP_CHECK_LAUNCH();
  }
  if (mesh1) {
    using X = FwdX<N, 1>;
    const size_t sh = 2 * (size_t)N * X::LB * sizeof(float2);
    smem_attr(k_fwd_x<N, 1>, sh);
    k_fwd_x<N, 1><<<dim3(G::NH / X::LB, N, count), X::TS, sh, s>>>(
        reinterpret_cast<float2*>(mesh0), reinterpret_cast<const float2*>(mesh1), tw, winv);
  } else {
    using X = FwdX<N, 0>;
    const size_t sh = (size_t)N * X::LB * sizeof(float2);
    smem_attr(k_fwd_x<N, 0>, sh);
    k_fwd_x<N, 0><<<dim3(G::NH / X::LB, N, count), X::TS, sh, s>>>(reinterpret_cast<float2*>(mesh0), nullptr, tw,
                                                                   winv);
  }
  BISP_CHECK_LAUNCH();
  if (launches) *launches += mesh1 ? 5 : 3;
  (void)mas;
}

void forward_fft(float* mesh0, float* mesh1, int count, int N, int mas, const float2* tw, const float* winv,
                 cudaStream_t s, int* launches) {
  switch (N) {
    case 16: fwd_impl<16>(mesh0, mesh1, count, mas, tw, winv, s, launches); break;
    case 32: fwd_impl<32>(mesh0, mesh1, count, mas, tw, winv, s, launches); break;
    case 64: fwd_impl<64>(mesh0, mesh1, count, mas, tw, winv, s, launches); break;
    case 128: fwd_impl<128>(mesh0, mesh1, count, mas, tw, winv, s, launches); break;
    case 256: fwd_impl<256>(mesh0, mesh1, count, mas, tw, winv, s, launches); break;
    case 512: fwd_impl<512>(mesh0, mesh1, count, mas, tw, winv, s, launches); break;
    case 1024: fwd_impl<1024>(mesh0, mesh1, count, mas, tw, winv, s, launches); break;
    default: throw Error{1, "unsupported mesh size"};
  }
}

// ====================================================================================
// inverse, pruned
// ====================================================================================

// y_l^m(n) for one (l, m >= 0) by the associated-Legendre recurrence (see common.cuh)
__device__ __forceinline__ float2 ylm_one(int l, int m, float x, float y, float z, const float* ynorm) {
  const float r2 = x * x + y * y + z * z;
  if (r2 == 0.f) return l == 0 ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
  const float rinv = rsqrtf(r2);
  const float mu = z * rinv;
  float pmm = 1.f;
  for (int k = 1; k <= m; ++k) pmm *= -(2.f * k - 1.f);
  float p = pmm;
  if (l > m) {
    float pm2 = pmm, pm1 = (2.f * m + 1.f) * mu * pmm;
    p = pm1;
    for (int ll = m + 2; ll <= l; ++ll) {
      p = ((2.f * ll - 1.f) * mu * pm1 - (float)(ll + m - 1) * pm2) / (float)(ll - m);
      pm2 = pm1;
      pm1 = p;
    }
  }
  float2 e = make_float2(1.f, 0.f);
  const float2 e1 = make_float2(x * rinv, y * rinv);
  for (int k = 0; k < m; ++k) e = cmul(e, e1);
  const float a = ynorm[l * (BISP_LMAX + 1) + m] * p;
  return make_float2(a * e.x, a * e.y);
}

__device__ __forceinline__ float cw2_val(const float* t, int N, int ix, int iy, int iz, int interlace) {
  // t = [e1 (N), o1 (N)] with e1 = E/W^2, o1 = O/W^2 per axis
  float v = t[ix] * t[iy] * t[iz];
  if (interlace) v = 0.5f * (v + t[N + ix] * t[N + iy] * t[N + iz]);
  return v;
}

// separation kernels of one r-bin (three-point function), see RKernelArgs
__global__ void __launch_bounds__(256) k_rshell_kernel(const RKernelArgs a) {
  const int N = a.N;
  const size_t Ng = (size_t)N * N * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t o = a.offs[i];
    const int sx = (int)(o & 1023u) - 512, sy = (int)((o >> 10) & 1023u) - 512, sz = (int)((o >> 20) & 1023u) - 512;
    const size_t cell = ((size_t)(sx & (N - 1)) * N + (size_t)(sy & (N - 1))) * N + (size_t)(sz & (N - 1));
    for (int c = 0; c < a.nc; ++c) {
      // part of y_l^{m*}(s_hat): F_l^m = A + i B with A, B the separation averages of its real
      // and imaginary parts
      const float2 y = ylm_one(a.l[c], a.m[c], (float)sx, (float)sy, (float)sz, a.ynorm);
      a.mesh[c * Ng + cell] = (a.part[c] ? -y.y : y.x) * a.inv_nr;
    }
  }
}

void launch_rshell_kernel(const RKernelArgs& a, cudaStream_t s) {
  if (a.n <= 0) return;
  if (a.nc < 1 || a.nc > 32) throw Error{1, "launch_rshell_kernel: nc out of range"};
  const int blocks = (int)std::min<int64_t>((a.n + 255) / 256, 4096);
  k_rshell_kernel<<<blocks, 256, 0, s>>>(a);
  BISP_CHECK_LAUNCH();
}

// scratch layout per field: T1 [N][2P+1][Pz], T2 [N][N][Pz]
struct InvGeo {
  int N, P, Pz, ny;
  size_t t1, t2;
};
__host__ __device__ __forceinline__ InvGeo inv_geo(int N, int P, int LB) {
  InvGeo g;
  g.N = N;
  g.P = P;
  g.Pz = ((P + 1 + LB - 1) / LB) * LB;
  g.ny = 2 * P + 1;
  g.t1 = (size_t)N * g.ny * g.Pz;
  g.t2 = (size_t)N * N * g.Pz;
  return g;
}

// lines per CTA of the first inverse pass: half the strided passes' (the prune extent stays a
// multiple of Geo<N>::LB, so of LX)
template <int N>
struct InvX {
  static constexpr int LX = Geo<N>::LB > 8 ? Geo<N>::LB / 2 : Geo<N>::LB;
  static constexpr int TS = LX * N / 8;
};
template <int N>
__global__ void __launch_bounds__(InvX<N>::TS, InvX<N>::TS <= 512 ? 2 : 1) k_inv_x(const __grid_constant__ InvBatch B, float2* t1all,
                                                       const float2* __restrict__ tw) {
  constexpr int NH = N / 2, LB = InvX<N>::LX, TS = InvX<N>::TS;
  constexpr int EPT = N * LB / TS;  // elements per thread
  extern __shared__ float2 s[];
  const InvGeo g = inv_geo(N, B.P, Geo<N>::LB);
  const int nz0 = blockIdx.x * LB, iy = blockIdx.y;
  const int sy = iy - g.P;
  const int jy = sy & (N - 1);
  // shell batches: every field filters the same spectrum over the same shell, so the spectrum
  // values and the shell mask are loaded once, before the field loop
  const bool shell = B.f[0].kind == SRC_SHELL || B.f[0].kind == SRC_SHELL_SUM;
  float2 av[EPT];
  unsigned inmask = 0;
  if (shell) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int i = threadIdx.x + k * TS;
      const int l = i % LB, e = i / LB;
      const int nz = nz0 + l;
      const int sx = sgn_idx(e, N);
      av[k] = make_float2(0.f, 0.f);
      if (sx <= g.P && sx >= -g.P && nz <= g.P) {
        const long long q = (long long)sx * sx + (long long)sy * sy + (long long)nz * nz;
        if (q >= B.qlo && q < B.qhi) {
          inmask |= 1u << k;
          if (B.f[0].kind == SRC_SHELL)
            av[k] = B.f[0].unit ? make_float2(1.f, 0.f) : B.f[0].A[((size_t)e * N + jy) * NH + nz];
        }
      }
    }
  }
  for (int f = 0; f < B.nf; ++f) {
    const InvField& F = B.f[f];
    if (shell) {
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int i = threadIdx.x + k * TS;
        float2 v = make_float2(0.f, 0.f);
        if (inmask & (1u << k)) {
          const int l = i % LB, e = i / LB;
          const int nz = nz0 + l;
          const int sx = sgn_idx(e, N);
          float2 t;
          if (F.kind == SRC_SHELL_SUM) {
            // sum over (m, part, channel) entries of part(y_l^{m*}) S(k), then / N_mode
            const size_t gi = ((size_t)e * N + jy) * NH + nz;
            float2 acc = make_float2(0.f, 0.f);
            for (int q = 0; q < F.ne; ++q) {
              const float2 y = ylm_one(F.l, F.em[q], (float)sx, (float)sy, (float)nz, B.ynorm);
              const float c = F.ecoef[q] * (F.epart[q] ? -y.y : y.x);
              const float2 a = B.spec[F.espec[q]][gi];
              acc.x = fmaf(c, a.x, acc.x);
              acc.y = fmaf(c, a.y, acc.y);
            }
            t = make_float2(acc.x * B.inv_nmodes, acc.y * B.inv_nmodes);
          } else {
            const float2 y = ylm_one(F.l, F.m, (float)sx, (float)sy, (float)nz, B.ynorm);
            // part of y_l^{m*}: Re y or -Im y, times (-i)^l
            const float c = (F.part ? -y.y : y.x) * B.inv_nmodes;
            t = make_float2(av[k].x * c, av[k].y * c);
          }
          switch (F.l & 3) {
            case 0: v = t; break;
            case 1: v = make_float2(t.y, -t.x); break;
            case 2: v = make_float2(-t.x, -t.y); break;
            default: v = make_float2(-t.y, t.x); break;
          }
        }
        s[i] = v;
      }
    } else {
      for (int i = threadIdx.x; i < N * LB; i += blockDim.x) {
        const int l = i % LB, e = i / LB;
        const int nz = nz0 + l;
        const int sx = sgn_idx(e, N);
        float2 v = make_float2(0.f, 0.f);
        if (sx <= g.P && sx >= -g.P && nz <= g.P) {
          const size_t gi = ((size_t)e * N + jy) * NH + nz;
          if (F.kind == SRC_PLAIN) {
            v = cscale(F.A[gi], F.scale);
          } else if (F.kind == SRC_KERNEL) {
            // conj(K) A: the k-space filter of the separation average (Sec. 4.3); the kernel
            // is real, so the product is Hermitian for every l
            v = cmul(cconj(F.K[gi]), F.unit ? make_float2(1.f, 0.f) : F.A[gi]);
          } else {  // SRC_QSHOT
            const float2 a = F.A[gi], b = F.B[gi];
            v = cmul(a, cconj(b));
            const float c = F.sbar * cw2_val(B.cw2_1d, N, e, jy, nz, B.interlace);
            v = make_float2((v.x - c) * F.scale, v.y * F.scale);
          }
        }
        s[i] = v;
      }
    }
    __syncthreads();
    fft_smem<N, LB, +1>(s, tw);
    float2* t1 = t1all + (size_t)f * g.t1;
    for (int i = threadIdx.x; i < N * LB; i += blockDim.x) {
      const int l = i % LB, e = i / LB;
      const size_t o = ((size_t)e * g.ny + iy) * g.Pz + nz0 + l;
      if (BISP_DCHECK(o < g.t1 && iy < g.ny, 20, o)) t1[o] = s[i];
    }
    __syncthreads();
  }
}

// c2r along z: X[k], k <= P (Pz stored, zero above P), Nyquist zero.
//   Z[k] = (X[k] + X*[NH-k]) + i (X[k] - X*[NH-k]) e^{2 pi i k / N};  z = IDFT_NH(Z)
//   x[2j] = Re z[j], x[2j+1] = Im z[j]
// c2r along z with the FFT held in registers: NH = A x B, A threads per row, each holding
// B values.  Step 1: Z[n] for n = a + A b (c2r pre-processing from the T2 row, read from
// global memory); step 2: B-point DFTs over b; step 3: twiddle e^{2 pi i a kb / NH};
// step 4: transpose through shared memory; step 5: A-point DFTs over a; outputs
// z[kb + B ka] -> cells 2m, 2m+1 with m = kb + B ka.
__host__ __device__ constexpr int regz_a(int nh) {
  return nh >= 256 ? 16 : (nh >= 64 ? 8 : (nh >= 32 ? 4 : 2));
}
template <int N>
struct RegZ {
  static constexpr int NH = N / 2;
  static constexpr int A = regz_a(NH);  // threads per row
  static constexpr int B = NH / A;      // values per thread (a multiple of A)
  static constexpr int ROWS = 256 / A;  // rows per group (256 threads)
  // input tiles of the row groups, double-buffered (bulk copies): 2 ROWS rows of Pz complex
  // row groups per CTA (the twiddle tables are built once per CTA); N^2 / ROWS is a power of two
  static constexpr int GROUPS = (N * N / ROWS) >= 8 ? 8 : (N * N / ROWS);
  // transpose buffer, e^{2 pi i j / NH} (NH entries), e^{2 pi i j / N} (NH entries), then the
  // two input tiles (sized per launch) and two mbarriers
  static constexpr size_t SMEM_FIXED = ((size_t)ROWS * B * (A + 1) + 2 * NH) * sizeof(float2);
  static size_t smem(int Pz) { return SMEM_FIXED + (size_t)2 * ROWS * Pz * sizeof(float2) + 16; }
};

__device__ __forceinline__ unsigned fft_su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool fft_wait(unsigned bar, unsigned parity) {
  unsigned ok = 0;
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  do {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (ok) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  } while (t - t0 < 2000000000ull);
  return false;
}
// one contiguous global range into shared memory (16-byte aligned, multiple of 16 bytes)
__device__ __forceinline__ void fft_bulk_load(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

template <int N>
__global__ void __launch_bounds__(256) k_inv_z_reg(const __grid_constant__ InvBatch Bt, const float2* t2all,
                                                   const float2* __restrict__ tw, int* err) {
  constexpr int NH = N / 2, A = RegZ<N>::A, B = RegZ<N>::B, ROWS = RegZ<N>::ROWS;
  constexpr int LDT = A + 1;  // padded transpose row
  static_assert(B % A == 0, "B must be a multiple of A");
  extern __shared__ float2 sbuf[];
  float2* wNH = sbuf + ROWS * B * LDT;  // e^{+2 pi i j / NH}
  float2* wN = wNH + NH;                // e^{+2 pi i j / N}, j < NH
  float2* tin = wN + NH;                // two input tiles [ROWS][Pz]
  const InvGeo g = inv_geo(N, Bt.P, Geo<N>::LB);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(tin + 2 * ROWS * g.Pz);
  const int f = blockIdx.y;
  const int GROUPS = Bt.zgroups;  // row groups per CTA (a power of two; tuned by the plan)
  const unsigned tile_bytes = (unsigned)(ROWS * g.Pz * sizeof(float2));
  const float2* src0 = t2all + (size_t)f * g.t2 + (size_t)blockIdx.x * GROUPS * ROWS * g.Pz;
  // every row group of this CTA lies inside field f's T2 block
  const bool src_ok = BISP_DCHECK(((size_t)blockIdx.x + 1) * GROUPS * ROWS * g.Pz <= g.t2, 24, blockIdx.x);
  if (!src_ok) return;
  const unsigned bar0 = fft_su32(bars);
  __shared__ int s_abort;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
    // the first group's rows (contiguous: ROWS consecutive T2 rows)
    if (!Bt.stall) fft_bulk_load(fft_su32(tin), src0, tile_bytes, bar0);
  }
  for (int j = threadIdx.x; j < NH; j += blockDim.x) {
    wNH[j] = cconj(tw[(j * (BISP_TWN / NH)) & (BISP_TWN - 1)]);
    wN[j] = cconj(tw[(j * (BISP_TWN / N)) & (BISP_TWN - 1)]);
  }
  __syncthreads();
  const int l = threadIdx.x / A, a = threadIdx.x % A;
  int grp = 0;
  for (; grp < GROUPS; ++grp) {
    const int cur = grp & 1;
    // prefetch the next group's rows into the other tile (its previous reader, group grp-1,
    // finished before the barrier that ended it)
    if (threadIdx.x == 0 && grp + 1 < GROUPS && !Bt.stall) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      fft_bulk_load(fft_su32(tin + (cur ^ 1) * ROWS * g.Pz), src0 + (size_t)(grp + 1) * ROWS * g.Pz, tile_bytes,
                    bar0 + 8u * (cur ^ 1));
    }
    if (!fft_wait(bar0 + 8u * cur, (unsigned)(grp >> 1) & 1u)) {
      s_abort = 1;
      atomicExch(err, 1);
    }
    const size_t row = ((size_t)blockIdx.x * GROUPS + grp) * ROWS + l;
    const float2* x = tin + cur * ROWS * g.Pz + l * g.Pz;
    const int P = Bt.P;
    float2 v[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int n = a + A * b;
      // X[k], k <= P (and X[0] real); X[NH] = 0 (Nyquist dropped)
      float2 xa = n <= P ? x[n] : make_float2(0.f, 0.f);
      const int nm = NH - n;
      float2 xb = (n > 0 && nm <= P) ? x[nm] : make_float2(0.f, 0.f);
      if (n == 0) xa.y = 0.f;
      // Z[n] = (X[n] + X*[NH-n]) + i (X[n] - X*[NH-n]) e^{2 pi i n / N}
      const float2 sp = make_float2(xa.x + xb.x, xa.y - xb.y);
      const float2 dm = make_float2(xa.x - xb.x, xa.y + xb.y);
      const float2 t = cmul(dm, wN[n]);
      v[b] = make_float2(sp.x - t.y, sp.y + t.x);
    }
    DftReg<B, +1>::run(v, tw);
    if (grp > 0) __syncthreads();  // the previous group's stage 2 has read the transpose buffer
    // twiddle e^{+2 pi i a kb / NH} and transpose: element (a, kb) -> sbuf[l][kb][a]
#pragma unroll
    for (int kb = 0; kb < B; ++kb) {
      sbuf[(l * B + kb) * LDT + a] = cmul(v[kb], wNH[(a * kb) & (NH - 1)]);
    }
    __syncthreads();  // also: every thread has read input tile cur
    if (s_abort) break;  // uniform: set before the barrier; nothing is stored after a timeout
    // stage 2: thread a handles kb = a + A r, r < B / A, an A-point DFT over a' each
    float* out = Bt.f[f].out + row * N;
    const bool row_ok = BISP_DCHECK((size_t)row < (size_t)N * N, 23, row);
#pragma unroll
    for (int r = 0; r < B / A; ++r) {
      const int kb = a + A * r;
      float2 u[A];
#pragma unroll
      for (int aa = 0; aa < A; ++aa) u[aa] = sbuf[(l * B + kb) * LDT + aa];
      DftReg<A, +1>::run(u, tw);
#pragma unroll
      for (int ka = 0; ka < A; ++ka) {
        const int m = kb + B * ka;
        if (row_ok) reinterpret_cast<float2*>(out)[m] = u[ka];
      }
    }
  }
  // after a timeout, the copies of this group and of the prefetched next one may still be in
  // flight: wait for them (bounded) before the CTA's shared memory is released
  if (s_abort && threadIdx.x == 0 && !Bt.stall) {
    fft_wait(bar0 + 8u * (grp & 1), (unsigned)(grp >> 1) & 1u);
    if (grp + 1 < GROUPS) fft_wait(bar0 + 8u * ((grp + 1) & 1), (unsigned)((grp + 1) >> 1) & 1u);
  }
}

// ------------------------------------------------------------------------------------
// Register four-step FFT of LB interleaved complex lines of NF points (strided passes):
// thread (line l = tid % LB, a = tid / LB) holds x[a + A b], b < B; B-point DFTs in
// registers, twiddle e^{SIGN 2 pi i a kb / NF}, transpose through shared memory laid out
// [kb][a][l], A-point DFTs; output m = kb + B ka.
// ------------------------------------------------------------------------------------
__host__ __device__ constexpr int regl_a(int nf) {
  return nf >= 1024 ? 32 : (nf >= 256 ? 16 : (nf >= 64 ? 8 : (nf >= 32 ? 4 : 2)));
}
template <int N>
struct RegL {
  static constexpr int LB = Geo<N>::LB;
  static constexpr int A = regl_a(N);
  static constexpr int B = N / A;
  static constexpr int THREADS = LB * A;
  static constexpr size_t SMEM = ((size_t)B * A * LB + N) * sizeof(float2);
};

// stage 2 + output: the caller has written v (after stage 1 and the twiddle) into s
template <int N, int SIGN, class Store>
__device__ __forceinline__ void regl_finish(const float2* s, int l, int a, const Store& store) {
  constexpr int A = RegL<N>::A, B = RegL<N>::B, LB = RegL<N>::LB;
#pragma unroll
  for (int r = 0; r < B / A; ++r) {
    const int kb = a + A * r;
    float2 u[A];
#pragma unroll
    for (int aa = 0; aa < A; ++aa) u[aa] = s[(kb * A + aa) * LB + l];
    DftReg<A, SIGN>::run(u, nullptr);
#pragma unroll
    for (int ka = 0; ka < A; ++ka) store(kb + B * ka, u[ka]);
  }
}

template <int N, int SIGN>
__device__ __forceinline__ void regl_stage1(float2* v, float2* s, const float2* wtab, int l, int a) {
  constexpr int A = RegL<N>::A, B = RegL<N>::B, LB = RegL<N>::LB;
  DftReg<B, SIGN>::run(v, nullptr);
#pragma unroll
  for (int kb = 0; kb < B; ++kb) s[(kb * A + a) * LB + l] = cmul(v[kb], wtab[(a * kb) & (N - 1)]);
}

// twiddle table e^{SIGN 2 pi i j / N} in shared memory
template <int N, int SIGN>
__device__ __forceinline__ void regl_twiddles(float2* wtab, const float2* __restrict__ tw) {
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    float2 w = tw[(j * (BISP_TWN / N)) & (BISP_TWN - 1)];
    if (SIGN > 0) w.y = -w.y;
    wtab[j] = w;
  }
}

template <int N>
__global__ void __launch_bounds__(RegL<N>::THREADS) k_inv_y_reg(const __grid_constant__ InvBatch Bt,
                                                                  const float2* t1all, float2* t2all,
                                                                  const float2* __restrict__ tw) {
  constexpr int A = RegL<N>::A, B = RegL<N>::B, LB = RegL<N>::LB;
  extern __shared__ float2 sm[];
  float2* s = sm;
  float2* wtab = sm + (size_t)B * A * LB;
  regl_twiddles<N, +1>(wtab, tw);
  const InvGeo g = inv_geo(N, Bt.P, LB);
  const int nz0 = blockIdx.x * LB, x = blockIdx.y, f = blockIdx.z;
  const int l = threadIdx.x % LB, a = threadIdx.x / LB;
  const float2* t1 = t1all + (size_t)f * g.t1 + (size_t)x * g.ny * g.Pz + nz0 + l;
  float2 v[B];
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int n = a + A * b;
    const int sy = sgn_idx(n, N);
    const bool in = sy >= -g.P && sy <= g.P &&
                    BISP_DCHECK((size_t)x * g.ny * g.Pz + (size_t)(sy + g.P) * g.Pz + nz0 + l < g.t1, 21, x);
    v[b] = in ? t1[(size_t)(sy + g.P) * g.Pz] : make_float2(0.f, 0.f);
  }
  __syncthreads();  // twiddle table ready
  regl_stage1<N, +1>(v, s, wtab, l, a);
  __syncthreads();
  float2* t2 = t2all + (size_t)f * g.t2 + (size_t)x * N * g.Pz + nz0 + l;
  regl_finish<N, +1>(s, l, a, [&](int m, float2 u) {
    if (BISP_DCHECK((size_t)x * N * g.Pz + (size_t)m * g.Pz + nz0 + l < g.t2, 22, m)) t2[(size_t)m * g.Pz] = u;
  });
}

int inverse_zgroups(int N, int requested) {
  int rows = 0, def = 8;
  switch (N) {
    case 16: rows = RegZ<16>::ROWS; def = RegZ<16>::GROUPS; break;
    case 32: rows = RegZ<32>::ROWS; def = RegZ<32>::GROUPS; break;
    case 64: rows = RegZ<64>::ROWS; def = RegZ<64>::GROUPS; break;
    case 128: rows = RegZ<128>::ROWS; def = RegZ<128>::GROUPS; break;
    case 256: rows = RegZ<256>::ROWS; def = RegZ<256>::GROUPS; break;
    case 512: rows = RegZ<512>::ROWS; def = RegZ<512>::GROUPS; break;
    default: rows = RegZ<1024>::ROWS; def = RegZ<1024>::GROUPS; break;
  }
  int groups = requested > 0 ? requested : def;
  while (groups > 1 && (groups & (groups - 1))) groups &= groups - 1;
  if (groups > N * N / rows) groups = N * N / rows;
  return groups;
}

template <int N>
static void inv_impl(const InvBatch& b, const float2* tw, void* scratch, cudaStream_t s, int* launches) {
  using G = Geo<N>;
  const InvGeo g = inv_geo(N, b.P, G::LB);
  float2* t1 = reinterpret_cast<float2*>(scratch);
  float2* t2 = t1 + (size_t)b.nf * g.t1;
  using RL = RegL<N>;
  const size_t s1 = (size_t)N * InvX<N>::LX * sizeof(float2);
  smem_attr(k_inv_x<N>, s1);
  smem_attr(k_inv_y_reg<N>, RL::SMEM);
  k_inv_x<N><<<dim3(g.Pz / InvX<N>::LX, g.ny), InvX<N>::TS, s1, s>>>(b, t1, tw);
  BISP_CHECK_LAUNCH();
  k_inv_y_reg<N><<<dim3(g.Pz / G::LB, N, b.nf), RL::THREADS, RL::SMEM, s>>>(b, t1, t2, tw);
  BISP_CHECK_LAUNCH();
  using RZ = RegZ<N>;
  const size_t zs = RZ::smem(g.Pz);
  smem_attr(k_inv_z_reg<N>, RZ::smem(N / 2));
  // row groups per CTA: the plan's tuned value, else the default; a power of two that divides
  // the N^2 / ROWS row groups
  const int groups = inverse_zgroups(N, b.zgroups);
  InvBatch bz = b;
  bz.zgroups = groups;
  k_inv_z_reg<N><<<dim3(N * N / (RZ::ROWS * groups), b.nf), 256, zs, s>>>(bz, t2, tw, b.err);
  BISP_CHECK_LAUNCH();
  if (launches) *launches += 3;
}

size_t inverse_scratch_bytes(int N, int P, int nf) {
  const int LB = (N >= 1024 || N < 32) ? 8 : 16;
  const InvGeo g = inv_geo(N, P, LB);
  return (size_t)nf * (g.t1 + g.t2) * sizeof(float2);
}

void inverse_fft(const InvBatch& b, const float2* tw, void* scratch, cudaStream_t s, int* launches) {
  if (b.nf <= 0) return;
  if (b.P < 0 || b.P > b.N / 2 - 1) throw Error{1, "inverse_fft: bad prune extent"};
  switch (b.N) {
    case 16: inv_impl<16>(b, tw, scratch, s, launches); break;
    case 32: inv_impl<32>(b, tw, scratch, s, launches); break;
    case 64: inv_impl<64>(b, tw, scratch, s, launches); break;
    case 128: inv_impl<128>(b, tw, scratch, s, launches); break;
    case 256: inv_impl<256>(b, tw, scratch, s, launches); break;
    case 512: inv_impl<512>(b, tw, scratch, s, launches); break;
    case 1024: inv_impl<1024>(b, tw, scratch, s, launches); break;
    default: throw Error{1, "unsupported mesh size"};
  }
}

}  // namespace bisp
