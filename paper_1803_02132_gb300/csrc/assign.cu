// Mass assignment (Sec. 4.1 Eq. mean_n, Eq. dn, Eq. nlm; Sec. 4.2; App. C):
// per-particle weights and line-of-sight channels, a stable LSD radix sort of the
// particles by home mesh node, cell starts, and a gather deposit in which every mesh
// node sums the particles around it in a fixed order (no float atomics, so the meshes
// are bit-reproducible run to run).
#include "common.cuh"
#include "internal.h"

namespace bisp {

// =====================================================================================
// prep: FP64 cell keys, FP32 offsets, weights, channel values, FP64 partial sums
// =====================================================================================
constexpr int PREP_THREADS = 256;
constexpr int PREP_MAXBLK = 4096;

int prep_blocks(int64_t n) {
  int64_t b = (n + PREP_THREADS - 1) / PREP_THREADS;
  if (b < 1) b = 1;
  if (b > PREP_MAXBLK) b = PREP_MAXBLK;
  return (int)b;
}

// The job arrives as a __grid_constant__ kernel parameter: every launch carries its own copy,
// so launches from different plans, streams or host threads never share it.
__global__ void __launch_bounds__(PREP_THREADS) k_prep(const __grid_constant__ PrepArgs a) {
  constexpr int NSMAX = 34;
#ifdef BISP_CHECKED
  // test of the check mechanism: the check fails without touching memory
  if (a.selftest && blockIdx.x == 0 && threadIdx.x == 0) BISP_DCHECK(false, 99, 0);
#endif
  double acc[NSMAX];
#pragma unroll
  for (int q = 0; q < NSMAX; ++q) acc[q] = 0.0;
  const int N = a.N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const float x = a.xyz[3 * i], y = a.xyz[3 * i + 1], z = a.xyz[3 * i + 2];
    const bool ok = isfinite(x) && isfinite(y) && isfinite(z) && x >= 0.f && y >= 0.f && z >= 0.f &&
                    (double)x < a.box && (double)y < a.box && (double)z < a.box;
    if (!ok) {
      atomicAdd(a.bad, 1);
      a.keys[i] = 0;
      a.idx[i] = (uint32_t)i;
      a.frac[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int c = 0; c < a.nchan; ++c) a.vals[(size_t)c * a.n + i] = 0.f;
      continue;
    }
    // u = x / H in FP64; home node floor(u) (CIC) or floor(u + 1/2) (NGP, TSC)
    const double ux = (double)x / a.H, uy = (double)y / a.H, uz = (double)z / a.H;
    double hx, hy, hz;
    if (a.mas == 2) {
      hx = floor(ux); hy = floor(uy); hz = floor(uz);
    } else {
      hx = floor(ux + 0.5); hy = floor(uy + 0.5); hz = floor(uz + 0.5);
    }
    const int ix = ((int)hx) & (N - 1), iy = ((int)hy) & (N - 1), iz = ((int)hz) & (N - 1);
    a.keys[i] = ((uint32_t)ix * (uint32_t)N + (uint32_t)iy) * (uint32_t)N + (uint32_t)iz;
    a.idx[i] = (uint32_t)i;
    a.frac[i] = make_float4((float)(ux - hx), (float)(uy - hy), (float)(uz - hz), 0.f);
    // weight: w / (1 + nbar P0)
    double wd = a.w ? (double)a.w[i] : 1.0;
    if (a.nbar && a.P0 > 0.f) wd = wd / (1.0 + (double)a.nbar[i] * (double)a.P0);
    const float wf = (float)wd;
    // line-of-sight harmonics
    float2 yl[(BISP_LMAX + 1) * (BISP_LMAX + 2) / 2];
    if (a.local) {
      ylm_all<BISP_LMAX>(x - a.obs[0], y - a.obs[1], z - a.obs[2], a.ynorm, yl);
    } else {
      ylm_all<BISP_LMAX>(0.f, 0.f, 1.f, a.ynorm, yl);
    }
    acc[0] += wd;
    const double w3 = wd * wd * wd;
    int q = 1;
    for (int c = 0; c < a.nchan; ++c) {
      const Chan ch = a.chan[c];
      const int am = ch.M < 0 ? -ch.M : ch.M;
      float2 yv = yl[ch.L * (ch.L + 1) / 2 + am];
      if (ch.M < 0) {  // y_l^{-m} = (-1)^m conj(y_l^m)
        yv = cconj(yv);
        if (am & 1) yv = make_float2(-yv.x, -yv.y);
      }
      if (ch.conj) yv = cconj(yv);
      const float pv = ch.part ? yv.y : yv.x;
      const float wp = ch.power == 2 ? wf * wf : wf;
      a.vals[(size_t)c * a.n + i] = wp * pv;
      if (ch.power == 1 && q < a.nsum && q < NSMAX) {
        acc[q] += w3 * (double)pv;
        ++q;
      }
    }
  }
  // deterministic block reduction of the FP64 sums
  __shared__ double red[PREP_THREADS / 32];
  for (int q = 0; q < a.nsum && q < NSMAX; ++q) {
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int wv = 0; wv < PREP_THREADS / 32; ++wv) s += red[wv];
      a.partials[(size_t)blockIdx.x * a.nsum + q] = s;
    }
    __syncthreads();
  }
}

void launch_prep(const PrepArgs& a, cudaStream_t s) {
  k_prep<<<prep_blocks(a.n), PREP_THREADS, 0, s>>>(a);
  BISP_CHECK_LAUNCH();
}

// =====================================================================================
// exclusive scan of uint32 (three phases, recursive on the block sums)
// =====================================================================================
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t ws[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t t = lane < SCAN_THREADS / 32 ? ws[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < SCAN_THREADS / 32) ws[lane] = t;
  }
  __syncthreads();
  const uint32_t wpre = wid ? ws[wid - 1] : 0u;
  if (total) *total = ws[SCAN_THREADS / 32 - 1];
  __syncthreads();
  return wpre + x - v;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const uint32_t* in, uint32_t* out, int64_t n,
                                                              uint32_t* sums) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS];
  uint32_t tsum = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    tsum += v[k];
  }
  uint32_t total;
  uint32_t pre = block_exclusive_scan(tsum, &total);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < n) out[base + k] = pre;
    pre += v[k];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_add(uint32_t* out, int64_t n, const uint32_t* offs) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  const uint32_t o = offs[blockIdx.x];
  for (int k = threadIdx.x; k < SCAN_TILE; k += blockDim.x)
    if (base + k < n) out[base + k] += o;
}

static int64_t ntiles(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

size_t scan_scratch_bytes(int64_t n) {
  size_t b = 0;
  int64_t m = n;
  while (m > 1) {
    m = ntiles(m);
    b += 2 * (size_t)(m + 1) * sizeof(uint32_t);
  }
  return b + 64;
}

void exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, void* scratch, cudaStream_t s,
                        int* launches) {
  if (n <= 0) return;
  const int64_t nt = ntiles(n);
  uint32_t* sums = (uint32_t*)scratch;
  uint32_t* offs = sums + nt + 1;
  k_scan_tiles<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, out, n, sums);
  BISP_CHECK_LAUNCH();
  if (launches) ++*launches;
  if (nt > 1) {
    exclusive_scan_u32(sums, offs, nt, offs + nt + 1, s, launches);
    k_scan_add<<<(unsigned)nt, 256, 0, s>>>(out, n, offs);
    BISP_CHECK_LAUNCH();
    if (launches) ++*launches;
  }
}

// =====================================================================================
// stable LSD radix sort, 8-bit digits
// =====================================================================================
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int RS_BINS = 256;

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint32_t* keys, int64_t n, int shift,
                                                        uint32_t* hist, int64_t nt) {
  __shared__ uint32_t h[RS_BINS];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int64_t i = base + r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & (RS_BINS - 1)], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nt + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint32_t* kin, const uint32_t* vin, int64_t n,
                                                           int shift, const uint32_t* offs, int64_t nt,
                                                           uint32_t* kout, uint32_t* vout) {
  constexpr int NW = RS_THREADS / 32;
  __shared__ uint32_t wc[NW][RS_BINS];
  __shared__ uint32_t base[RS_BINS];
  __shared__ uint32_t tot[RS_BINS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  base[threadIdx.x] = offs[(int64_t)threadIdx.x * nt + blockIdx.x];
  const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
  const uint32_t lt = (1u << lane) - 1u;
  for (int r = 0; r < RS_ROUNDS; ++r) {
#pragma unroll
    for (int w = 0; w < NW; ++w) wc[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = t0 + r * RS_THREADS + threadIdx.x;
    const bool valid = i < n;
    uint32_t k = 0, v = 0, d = RS_BINS;  // invalid items take a digit no one uses
    if (valid) {
      k = kin[i];
      v = vin[i];
      d = (k >> shift) & (RS_BINS - 1);
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & lt);
    if (valid && rank == 0) wc[wid][d] = __popc(peers);
    __syncthreads();
    {  // per-digit prefix over warps (thread = digit)
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint32_t c = wc[w][threadIdx.x];
        wc[w][threadIdx.x] = run;
        run += c;
      }
      tot[threadIdx.x] = run;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = base[d] + wc[wid][d] + rank;
      kout[pos] = k;
      vout[pos] = v;
    }
    __syncthreads();
    base[threadIdx.x] += tot[threadIdx.x];
    __syncthreads();
  }
}

size_t radix_sort_scratch_bytes(int64_t n) {
  const int64_t nt = (n + RS_TILE - 1) / RS_TILE;
  const int64_t nh = nt * RS_BINS;
  return 2 * (size_t)n * sizeof(uint32_t) + 2 * (size_t)nh * sizeof(uint32_t) + scan_scratch_bytes(nh) + 256;
}

void radix_sort(uint32_t* keys, uint32_t* vals, uint32_t* keys_out, uint32_t* vals_out, int64_t n, int bits,
                void* scratch, cudaStream_t s, int* launches) {
  if (n <= 0) return;
  const int64_t nt = (n + RS_TILE - 1) / RS_TILE;
  const int64_t nh = nt * RS_BINS;
  uint32_t* tk = (uint32_t*)scratch;
  uint32_t* tv = tk + n;
  uint32_t* hist = tv + n;
  uint32_t* offs = hist + nh;
  void* sscr = offs + nh;
  int npass = (bits + 7) / 8;
  if (npass < 1) npass = 1;
  // ping-pong so that the last pass writes keys_out/vals_out
  const uint32_t* kin = keys;
  const uint32_t* vin = vals;
  for (int p = 0; p < npass; ++p) {
    const bool last = p == npass - 1;
    // even distance from the end -> out, odd -> temp
    const bool to_out = ((npass - 1 - p) % 2) == 0;
    uint32_t* ko = to_out ? keys_out : tk;
    uint32_t* vo = to_out ? vals_out : tv;
    (void)last;
    k_rs_hist<<<(unsigned)nt, RS_THREADS, 0, s>>>(kin, n, 8 * p, hist, nt);
    BISP_CHECK_LAUNCH();
    exclusive_scan_u32(hist, offs, nh, sscr, s, launches);
    k_rs_scatter<<<(unsigned)nt, RS_THREADS, 0, s>>>(kin, vin, n, 8 * p, offs, nt, ko, vo);
    BISP_CHECK_LAUNCH();
    if (launches) *launches += 2;
    kin = ko;
    vin = vo;
  }
}

// =====================================================================================
// cell counts, particle gather, deposit
// =====================================================================================
__global__ void k_count_cells(const uint32_t* keys, int64_t n, uint32_t* counts) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&counts[keys[i]], 1u);
}

void launch_count_cells(const uint32_t* keys, int64_t n, uint32_t* counts, cudaStream_t s) {
  if (n <= 0) return;
  int64_t b = (n + 255) / 256;
  if (b > 65536) b = 65536;
  k_count_cells<<<(unsigned)b, 256, 0, s>>>(keys, n, counts);
  BISP_CHECK_LAUNCH();
}

__global__ void k_gather_particles(const uint32_t* perm, int64_t n, const float4* frac_in, const float* vals_in,
                                   int nchan, float4* frac_out, float* vals_out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t p = perm[i];
    if (!BISP_DCHECK(p < (uint64_t)n, 1, p)) continue;
    frac_out[i] = frac_in[p];
    for (int c = 0; c < nchan; ++c) vals_out[(size_t)c * n + i] = vals_in[(size_t)c * n + p];
  }
}

void launch_gather_particles(const uint32_t* perm, int64_t n, const float4* frac_in, const float* vals_in,
                             int nchan, float4* frac_out, float* vals_out, cudaStream_t s) {
  if (n <= 0) return;
  int64_t b = (n + 255) / 256;
  if (b > 65536) b = 65536;
  k_gather_particles<<<(unsigned)b, 256, 0, s>>>(perm, n, frac_in, vals_in, nchan, frac_out, vals_out);
  BISP_CHECK_LAUNCH();
}

// 1D assignment kernel as a function of the distance t between particle and node
template <int P>
__device__ __forceinline__ float wker(float t) {
  if (P == 1) return (t >= -0.5f && t < 0.5f) ? 1.f : 0.f;
  const float a = fabsf(t);
  if (P == 2) return a < 1.f ? 1.f - a : 0.f;
  if (a < 0.5f) return 0.75f - t * t;
  if (a < 1.5f) {
    const float b = 1.5f - a;
    return 0.5f * b * b;
  }
  return 0.f;
}

// Gather deposit over CTA-owned node tiles.  A CTA owns DT_X x DT_Y x DZ mesh nodes (z
// fastest), one node per thread; DZ = 32 (16 for a 16^3 mesh), so that a warp is one line of
// nodes along z: its lanes need the same halo rows, and a staged batch keeps a warp's lanes
// either all busy or all idle.  The home cells its nodes draw from, h = c + o with o in
// [OLO, OHI]^3, form a halo box of RX x RY x RZ cells; their particles, which sit in the sorted
// arrays as one contiguous range per cell, are listed in (rx, ry, rz) order and staged through
// shared memory in batches of MAXP, read coalesced.  Every node then visits its (ox, oy, oz)
// cells in increasing order and each cell's particles in sorted (stable) order: the same order
// and the same FP32 operations as a node-by-node gather, so the meshes are bit-reproducible.
// A tile whose halo holds no particle (most of a survey's volume) writes its zeros and returns
// after one count per halo row.  Node positions: mesh 0 at c H, mesh 1 (interlaced) at
// (c + 1/2) H.  All channels are accumulated in one pass (NC >= nchan registers per mesh).
constexpr int DT_X = 4, DT_Y = 4;

template <int P, int ILV, int DZ>
struct DepTile {
  static constexpr int THREADS = DT_X * DT_Y * DZ;
  static constexpr int OLO = (P == 1) ? 0 : -1;
  static constexpr int OHI = ILV ? (P == 3 ? 2 : 1) : (P == 3 ? 1 : 0);
  static constexpr int W = OHI - OLO + 1;
  static constexpr int RX = DT_X + W - 1, RY = DT_Y + W - 1, RZ = DZ + W - 1;
  static constexpr int NCELL = RX * RY * RZ;
};

// Batch of staged particles: two CTAs of DT_X DT_Y DZ threads per SM share the SM's shared memory
// (112 KB each with the static halo tables): 736 particles for 12 channels with TSC and
// interlacing.  Measured at 512^3 (random catalogue's assignment): 256 particles 86.0 ms, 512
// 66.6 ms, 672 65.6 ms, 1440 with one CTA per SM 70.3 ms; mesh 0 keeps only the offsets where
// its weights can be non-zero (3 of 4 per axis for TSC with interlacing): 736 particles, 64.7 ms.
template <int P, int ILV, int NC, int DZ>
struct DepBatch {
  using T = DepTile<P, ILV, DZ>;
  static constexpr int W0 = (P == 3 ? 1 : 0) - T::OLO + 1;  // mesh 0's non-zero offsets per axis
  static constexpr int PER = 4 * (3 * W0 + (ILV ? 3 * T::W : 0) + NC) + 1;  // bytes per staged particle
  static constexpr int FIT = (112 * 1024 - 8 * T::NCELL - 512) / PER;
  static constexpr int MAXP = (FIT / 32) * 32;
  static constexpr size_t BYTES = (size_t)PER * MAXP;
};

template <int P, int ILV, int NC, int DZ>
__global__ void __launch_bounds__(DT_X * DT_Y * DZ) k_deposit(const uint32_t* __restrict__ cell_start,
                                                        const float4* __restrict__ frac,
                                                        const float* __restrict__ vals, int64_t n, int N,
                                                        int nchan, float* mesh0, float* mesh1) {
  using T = DepTile<P, ILV, DZ>;
  constexpr int DT_THREADS = T::THREADS, DT_Z = DZ;
  constexpr int OLO = T::OLO, OHI = T::OHI, W = T::W, RY = T::RY, RZ = T::RZ, NCELL = T::NCELL;
  // mesh 0's weight vanishes for every offset in the particle's cell once an offset exceeds O0HI
  constexpr int O0HI = (P == 3) ? 1 : 0;
  constexpr int W0 = DepBatch<P, ILV, NC, DZ>::W0;       // mesh 0's offsets OLO..O0HI
  constexpr int W1 = ILV ? W : 1;
  constexpr int MAXP = DepBatch<P, ILV, NC, DZ>::MAXP;  // particles per staged batch
  __shared__ uint32_t s_gs[NCELL];             // first sorted index of each halo cell
  __shared__ uint32_t s_ts[NCELL + 1];         // position of each halo cell in the tile list
  // staged batch (dynamic shared memory): per axis the 1D weights W_p(o + d) of mesh 0 (offsets
  // OLO..O0HI, where they can be non-zero) and W_p(o + d - 1/2) of mesh 1, channel values, halo z
  // index of each particle's cell
  constexpr size_t SW1 = ILV ? 3 * W : 0;
  extern __shared__ __align__(16) unsigned char dep_dyn[];
  auto& s_w0 = *reinterpret_cast<float (*)[3][W0][MAXP]>(dep_dyn);
  auto& s_w1 = *reinterpret_cast<float (*)[3][W1][MAXP]>(dep_dyn + sizeof(float) * 3 * W0 * MAXP);
  auto& s_val = *reinterpret_cast<float (*)[NC][MAXP]>(dep_dyn + sizeof(float) * (3 * W0 + SW1) * MAXP);
  auto& s_rz =
      *reinterpret_cast<unsigned char (*)[MAXP]>(dep_dyn + sizeof(float) * (3 * W0 + SW1 + NC) * MAXP);
  __shared__ uint32_t s_wsum[DT_THREADS / 32];
  __shared__ int s_any;
  const int ntz = N / DT_Z, nty = N / DT_Y;
  const int tz = (int)(blockIdx.x % ntz), ty = (int)((blockIdx.x / ntz) % nty), tx = (int)(blockIdx.x / (ntz * nty));
  const int x0 = tx * DT_X, y0 = ty * DT_Y, z0 = tz * DT_Z;
  const int lz = threadIdx.x % DT_Z, ly = (threadIdx.x / DT_Z) % DT_Y, lx = threadIdx.x / (DT_Z * DT_Y);
  const int64_t Ng = (int64_t)N * N * N;
  const int64_t cell = ((int64_t)(x0 + lx) * N + (y0 + ly)) * N + (z0 + lz);
  const uint32_t msk = (uint32_t)(N - 1);
  const bool zwrap = z0 + OLO < 0 || z0 + DT_Z - 1 + OHI > N - 1;
  // (1) any particle in the halo?  one range per halo row unless the z run wraps around
  if (threadIdx.x == 0) s_any = 0;
  __syncthreads();
  for (int r = threadIdx.x; r < T::RX * RY; r += blockDim.x) {
    const uint32_t hx = (uint32_t)(x0 + OLO + r / RY) & msk, hy = (uint32_t)(y0 + OLO + r % RY) & msk;
    const uint32_t rowkey = (hx * (uint32_t)N + hy) * (uint32_t)N;
    uint32_t cnt = 0;
    if (!zwrap) {
      if (BISP_DCHECK(rowkey + (uint64_t)(z0 + DT_Z - 1 + OHI) + 1 <= (uint64_t)Ng && z0 + OLO >= 0, 2, rowkey))
        cnt = cell_start[rowkey + (uint32_t)(z0 + DT_Z - 1 + OHI) + 1] - cell_start[rowkey + (uint32_t)(z0 + OLO)];
    } else {
      for (int rz = 0; rz < RZ; ++rz) {
        const uint32_t k = rowkey + ((uint32_t)(z0 + OLO + rz) & msk);
        cnt += cell_start[k + 1] - cell_start[k];
      }
    }
    if (cnt) s_any = 1;
  }
  __syncthreads();
  float a0[NC], a1[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) a0[k] = a1[k] = 0.f;
  if (s_any) {
    // (2) per halo cell: first sorted index and count, then the exclusive scan of the counts
    constexpr int PER = (NCELL + DT_THREADS - 1) / DT_THREADS;
    uint32_t cnt[PER];
    uint32_t tsum = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int c = threadIdx.x * PER + j;
      cnt[j] = 0;
      if (c < NCELL) {
        const int rz = c % RZ, ry = (c / RZ) % RY, rx = c / (RZ * RY);
        const uint32_t hx = (uint32_t)(x0 + OLO + rx) & msk, hy = (uint32_t)(y0 + OLO + ry) & msk;
        const uint32_t hz = (uint32_t)(z0 + OLO + rz) & msk;
        const uint32_t k = (hx * (uint32_t)N + hy) * (uint32_t)N + hz;
        if (!BISP_DCHECK(k < (uint64_t)Ng, 3, k)) continue;
        const uint32_t g0 = cell_start[k];
        s_gs[c] = g0;
        cnt[j] = cell_start[k + 1] - g0;
      }
      tsum += cnt[j];
    }
    // block exclusive scan of the per-thread sums (warp shuffles, then the warp totals)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_wsum[wid] = incl;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < wid; ++w) wpre += s_wsum[w];
    uint32_t pos = wpre + incl - tsum;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int c = threadIdx.x * PER + j;
      if (c < NCELL) s_ts[c] = pos;
      pos += cnt[j];
    }
    if (threadIdx.x == DT_THREADS - 1) s_ts[NCELL] = pos;
    __syncthreads();
    const uint32_t total = s_ts[NCELL];
    // (3) batches of the tile list
    for (uint32_t b0 = 0; b0 < total; b0 += MAXP) {
      const uint32_t b1 = min(total, b0 + (uint32_t)MAXP);
      __syncthreads();  // the previous batch is consumed
      for (uint32_t q = b0 + threadIdx.x; q < b1; q += DT_THREADS) {
        // halo cell of list position q: the last c with s_ts[c] <= q
        int lo = 0, hi = NCELL - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_ts[mid] <= q) lo = mid;
          else hi = mid - 1;
        }
        const uint32_t g = s_gs[lo] + (q - s_ts[lo]);
        if (!BISP_DCHECK(g < (uint64_t)n && q - b0 < (uint32_t)MAXP, 4, g)) continue;
        const float4 d = frac[g];
        s_rz[q - b0] = (unsigned char)(lo % RZ);
        // 1D weights of this particle for every offset o (distance particle - node = o + d)
#pragma unroll
        for (int o = OLO; o <= OHI; ++o) {
          const float tx_ = (float)o + d.x, ty_ = (float)o + d.y, tz_ = (float)o + d.z;
          if (o <= O0HI) {
            s_w0[0][o - OLO][q - b0] = wker<P>(tx_);
            s_w0[1][o - OLO][q - b0] = wker<P>(ty_);
            s_w0[2][o - OLO][q - b0] = wker<P>(tz_);
          }
          if (ILV) {
            s_w1[0][o - OLO][q - b0] = wker<P>(tx_ - 0.5f);
            s_w1[1][o - OLO][q - b0] = wker<P>(ty_ - 0.5f);
            s_w1[2][o - OLO][q - b0] = wker<P>(tz_ - 0.5f);
          }
        }
#pragma unroll
        for (int k = 0; k < NC; ++k)
          if (k < nchan) s_val[k][q - b0] = vals[(size_t)k * n + g];
      }
      __syncthreads();
      // every (ox, oy) in increasing order; the node's W cells of that halo row are consecutive in
      // the tile list, so one range holds them, oz ascending and each cell's particles in sorted
      // order (the order of a cell-by-cell visit)
#pragma unroll
      for (int ox = OLO; ox <= OHI; ++ox) {
#pragma unroll
        for (int oy = OLO; oy <= OHI; ++oy) {
          const int c = ((lx + ox - OLO) * RY + (ly + oy - OLO)) * RZ + lz;  // cell of oz = OLO
          const uint32_t p0 = max(s_ts[c], b0), p1 = min(s_ts[c + W], b1);
          const bool mxy = ox <= O0HI && oy <= O0HI;  // else mesh 0's weight is 0
          for (uint32_t q = p0; q < p1; ++q) {
            const uint32_t i = q - b0;
            const int zo = (int)s_rz[i] - lz;  // oz - OLO
            const bool m0 = mxy && zo + OLO <= O0HI;
            float w0 = 0.f, w1 = 0.f;
            if (m0) w0 = s_w0[0][ox - OLO][i] * s_w0[1][oy - OLO][i] * s_w0[2][zo][i];
            if (ILV) w1 = s_w1[0][ox - OLO][i] * s_w1[1][oy - OLO][i] * s_w1[2][zo][i];
#pragma unroll
            for (int k = 0; k < NC; ++k) {
              if (k < nchan) {
                const float v = s_val[k][i];
                if (m0) a0[k] = fmaf(w0, v, a0[k]);
                if (ILV) a1[k] = fmaf(w1, v, a1[k]);
              }
            }
          }
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    if (k < nchan) {
      mesh0[(size_t)k * Ng + cell] = a0[k];
      if (ILV) mesh1[(size_t)k * Ng + cell] = a1[k];
    }
  }
}

template <int P, int ILV, int DZ>
static void deposit_pz(const DepositArgs& a, cudaStream_t s) {
  const int64_t Ng = (int64_t)a.N * a.N * a.N;
  constexpr int TH = DepTile<P, ILV, DZ>::THREADS;
  const unsigned grid = (unsigned)(Ng / TH);
#define BISP_DEP(NC_)                                                                                    \
  do {                                                                                                   \
    constexpr size_t sh = DepBatch<P, ILV, NC_, DZ>::BYTES;                                              \
    BISP_CUDA(cudaFuncSetAttribute(k_deposit<P, ILV, NC_, DZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                   (int)sh));                                                            \
    k_deposit<P, ILV, NC_, DZ><<<grid, TH, sh, s>>>(a.cell_start, a.frac, a.vals, a.n, a.N, a.nchan, a.mesh0, \
                                                  a.mesh1);                                              \
  } while (0)
  if (a.nchan <= 1) BISP_DEP(1);
  else if (a.nchan <= 2) BISP_DEP(2);
  else if (a.nchan <= 6) BISP_DEP(6);
  else if (a.nchan <= 12) BISP_DEP(12);
  else if (a.nchan <= 16) BISP_DEP(16);
  else throw Error{6, "deposit: more than 16 channels"};
#undef BISP_DEP
}

template <int P, int ILV>
static void deposit_p(const DepositArgs& a, cudaStream_t s) {
  if (a.N >= 32) deposit_pz<P, ILV, 32>(a, s);
  else deposit_pz<P, ILV, 16>(a, s);
}

void launch_deposit(const DepositArgs& a0, cudaStream_t s, int* launches) {
  // at most 16 channels per launch (register accumulators); more channels go in groups
  const int64_t Ng = (int64_t)a0.N * a0.N * a0.N;
  for (int c0 = 0; c0 < a0.nchan; c0 += 16) {
    DepositArgs a = a0;
    a.nchan = a0.nchan - c0 < 16 ? a0.nchan - c0 : 16;
    a.vals = a0.vals + (size_t)c0 * a0.n;
    a.mesh0 = a0.mesh0 + (size_t)c0 * Ng;
    a.mesh1 = a0.mesh1 ? a0.mesh1 + (size_t)c0 * Ng : nullptr;
    if (a.interlace) {
      if (a.mas == 1) deposit_p<1, 1>(a, s);
      else if (a.mas == 2) deposit_p<2, 1>(a, s);
      else deposit_p<3, 1>(a, s);
    } else {
      if (a.mas == 1) deposit_p<1, 0>(a, s);
      else if (a.mas == 2) deposit_p<2, 0>(a, s);
      else deposit_p<3, 0>(a, s);
    }
    BISP_CHECK_LAUNCH();
    if (launches) ++*launches;
  }
}

// =====================================================================================
// sum of cubes of a mesh (normalisation I from the random catalogue), FP64 partials
// =====================================================================================
__global__ void __launch_bounds__(256) k_sum_cubes(const float* m, int64_t ncell, double* partials) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)m[i];
    acc += v * v * v;
  }
  __shared__ double red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    partials[blockIdx.x] = s;
  }
}

int launch_sum_cubes(const float* mesh, int64_t ncell, double* partials, cudaStream_t s) {
  const int nb = 1024;
  k_sum_cubes<<<nb, 256, 0, s>>>(mesh, ncell, partials);
  BISP_CHECK_LAUNCH();
  return nb;
}

}  // namespace bisp
