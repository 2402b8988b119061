// The mesh sum of Eq. bi_estimator_FFTs (Sec. 4.2), contracted over the (m1, m2, M) terms
// of the real expansion:  out[o][b1][b2] = sum_x sum_{t in o} X_t(x; b1) Y_t(x; b2), where
// each side is either one filtered component field F_c(x; b) ("bare") or a small
// combination sum_(c,h) F_c(x; b) H_h(x) with H_h = sum_g coef G_g ("built").
//  * k_pair_tma (default): bins <= 32.  TMA tensor-map loads (128-byte swizzle, mbarrier
//    completion) stage 64-cell chunks of every field in shared memory, one barrier per chunk;
//    the H rows are formed once per chunk, built sides directly in MMA fragment registers; each
//    warp multiplies its term's X and Y tiles with mma.sync m16n8k8 TF32 in three passes
//    (v = hi + lo split, X_hi Y_hi + X_hi Y_lo + X_lo Y_hi: FP32-class products).  Warp tables
//    from the host balance the terms (cell halves split for the heaviest, two-term warps for
//    terms that differ only in their H rows); at 25 bins the 25th column is formed by FMA.
//  * k_pair_umma (opt-in): the same contraction on tcgen05 with TMEM accumulators.
//  * k_pair: any bin count up to 40, FP32 FMA register tiles (fallback).
// Chunk sums go to FP32 running sums over at most 1024 cells, then to compensated FP32 (TMA,
// tcgen05) or FP64 (FMA) slots; the slots are reduced in FP64 in a fixed order, so results are
// bit-reproducible.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace bisp {

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
// The FMA and tcgen05 kernels take their PairJob as a __grid_constant__ parameter (about 22 KB,
// inside the 32 KB parameter space): each launch carries its own copy.  The TMA kernel reads it from
// a constant-memory slot held under a lock until its launches complete (see c_pj below).
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
static PairJob classify_impl(const PairJob& job);

// classify() of the last job seen by this thread, kept so that the fit check, the scratch size
// and the launch of one job classify it once (the tables are a few tens of KB of host work)
static const PairJob& classify(const PairJob& job) {
  thread_local PairJob last_in, last_out;
  thread_local bool valid = false;
  if (valid && std::memcmp(&last_in, &job, sizeof(PairJob)) == 0) return last_out;
  valid = false;
  last_out = classify_impl(job);
  last_in = job;
  valid = true;
  return last_out;
}

static PairJob classify_impl(const PairJob& job) {
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

struct TmaLayout;
static bool tma_layout(const PairJob& j, TmaLayout* L, int* warps);
static bool pairable(const PairJob& j, int a, int b);
static int pair_blocks();

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int NW>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NW)); }

// copy one chunk of every component row [b][comp] and G row into shared memory;
// rowmap[f] = destination row of source row f (f < nb*ncomp: field (b, comp); then G rows)
__device__ __forceinline__ void pair_stage(const PairJob& J, float* raw, int64_t x0, const int* rowmap) {
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
__device__ __forceinline__ void pair_build_sides(const PairJob& J, const float* raw, float* mat, float* Hs, int bs,
                                                 unsigned mnb) {
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
__global__ void __launch_bounds__(NTHR, 1) k_pair(const __grid_constant__ PairJob J, int nbp, int bs, int rows,
                                                  int ksplit, double* partials) {
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
  if (blockIdx.x < nchunk) pair_stage(J, sh, (int64_t)blockIdx.x * PR_CH, rowmap);
  cp_async_commit();
  int since_flush = 0, stage = 0;
  for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    cp_async_wait<0>();
    __syncthreads();
    {
      const int64_t nx = ch + gridDim.x;
      if (nx < nchunk) pair_stage(J, sh + (size_t)(stage ^ 1) * rows * PR_LD, nx * PR_CH, rowmap);
      cp_async_commit();
    }
    const float* raw = sh + (size_t)stage * rows * PR_LD;
    if (J.nslot) {
      pair_build_sides(J, raw, mat, Hs, bs, mnb);
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
// Tensor-core variant (nb <= 32).  Per chunk of 64 cells, for every term t:
//   C_t (32 x 32 bins) += X_t (32 bins x 64 cells) Y_t^T
// with mma.sync m16n8k8 TF32 in three passes over a split v = hi + lo of each FP32 value
// (hi, lo both TF32: X_hi Y_hi + X_hi Y_lo + X_lo Y_hi), i.e. FP32-class products.
//
// Staging: a 3D TMA tensor map views the component fields as [nb][ncomp][Ng] and loads, per
// 32-cell half and component c, the box of all bins as a [32 bins][32 cells] block (bins
// >= nb read as zeros); a 2D map loads the G fields as [ng][32 cells].  Blocks use the
// 128-byte swizzle (16-byte piece p of row r stored at piece p ^ (r & 7)), so the 8-row
// ldmatrix reads below hit 8 different bank groups.  Two stages: the TMA of chunk i+1 runs
// while chunk i is used; an mbarrier per stage carries the transaction bytes.  Every wait
// is bounded in time and reports a timeout through err instead of hanging.
//
// Per chunk: (1) H rows H_h(x) = sum coef G_g(x) (shared by all bins), stored in the order
// the MMA fragments read them; (2) two warps per (term, cell half), one per 16-row half of
// the 32 x 32 tile: a built side X(b, x) = sum_(c,h) F_c(b, x) H_h(x) is accumulated directly
// in fragment registers from ldmatrix loads of the F_c blocks, a bare side is loaded as it
// is; then the three MMA passes.  Terms are normalised so that only X is ever built (a term
// with a built Y is computed as Y X^T and read back transposed).
// The MMA accumulators restart every chunk; chunk results go to FP32 running sums, and every
// chunk one of the 16 (round robin, so each covers at most 1024 cells) is added with Kahan
// compensation to a lane-owned FP32 (sum, compensation) slot in global memory, whose load is
// issued at the start of the chunk.
// ------------------------------------------------------------------------------------
constexpr int TMA_MAXWARP = 20;  // warps of a CTA
struct TmaLayout {
  unsigned fsz, gsz;  // bytes of the F blocks (ncomp x 4096) and of the G block of one half
  unsigned half;      // fsz + gsz
  unsigned stage;     // 2 * half
  unsigned hs;        // offset of the H rows, two buffers [2][nh][64 floats], fragment order
  unsigned bar;       // offset of the two mbarriers
  unsigned bytes;     // dynamic shared memory to request (includes 1024 B alignment slack)
  unsigned tx;        // transaction bytes per stage
  int ncomp, gbox;    // F blocks per half, G rows
  int stall;          // test knob: start no stage copy, so that every bounded wait runs out
  int nst;            // stages (chunks staged ahead + 1): 3 when shared memory allows, else 2
  int nblk;           // CTAs of the launch
  int mh, nt;         // 16-row tiles and 8-column tiles per term (bins covered: 16 mh, 8 nt)
  unsigned cblk;      // bytes of one component block (bh bins x 128 bytes, bh = max(16 mh, 8 nt))
  // warps: one per (term, 16-row tile) over both cell halves of a chunk, or, for a term whose
  // built side makes it the heaviest, one per (term, cell half, row tile)
  unsigned char wterm[TMA_MAXWARP];  // warp -> term
  unsigned char whalf[TMA_MAXWARP];  // warp -> cell half 0 or 1, or 2 for both
  unsigned char wrow[TMA_MAXWARP];   // warp -> 16-row tile
  unsigned char tfirst[64];          // term -> its first warp (then half-major, row tile minor)
  unsigned char tsplit[64];          // term -> 1 (warps over both halves) or 2 (one per half)
  unsigned char tsub[64];            // term -> its slot group in the warp (two-term warps: 0 or 1)
  int ntm;                           // terms per warp: 2 when every term has a partner (see dual_order)
};
constexpr unsigned long long TMA_WAIT_NS = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the phase with the given parity; false after TMA_WAIT_NS without completion
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > TMA_WAIT_NS) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, int x, int y, unsigned bar,
                                            unsigned long long policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar), "l"(policy)
      : "memory");
}

__device__ __forceinline__ void ldsm_x2(unsigned addr, uint32_t* r) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4(unsigned addr, uint32_t* r) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

// v = hi + lo: hi keeps the sign, exponent and top 10 mantissa bits of v (a valid TF32
// value), lo = v - hi is exact in FP32 and the tensor core reads its top 19 bits.  The three
// passes then miss below 3 * 2^-20 of each product, always toward zero by a fraction that does
// not depend on the product's sign or size: a sum is scaled by about 1 - 1.5e-6 plus noise of
// order 1e-6 of its root-sum-square.
__device__ __forceinline__ void split_tf32(uint32_t bits, uint32_t& hi, uint32_t& lo) {
  hi = bits & 0xffffe000u;
  lo = __float_as_uint(__uint_as_float(bits) - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float* c, const uint32_t* a, const uint32_t* b) {
  asm(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// byte offset of 16-byte piece p of row r in a 128-byte-swizzled [rows][32 floats] block
__device__ __forceinline__ unsigned swz(int r, int p) { return (unsigned)r * 128u + ((unsigned)(p ^ (r & 7)) << 4); }

__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, int x, int y, int z, unsigned bar,
                                            unsigned long long policy) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar), "l"(policy)
      : "memory");
}

// compensated (Kahan) FP32 accumulation into a slot (s, e) whose true sum is s - e
__device__ __forceinline__ void kahan_add(float2& v, float x) {
  const float y = x - v.y;
  const float t = v.x + y;
  v.y = (t - v.x) - y;
  v.x = t;
}
// The TMA kernel and its final reduction read their job from module constant memory: its warp-
// uniform table reads in the inner loops are constant-cache hits, measurably faster (4 % of the
// kernel) than the same reads from a kernel parameter or shared memory.  The one slot is guarded
// by g_pj_mu from the copy into it until the launches that read it have completed, so that plans
// driven from several host threads never overwrite a job in use (their contractions serialise;
// one contraction fills the GPU).
__constant__ PairJob c_pj;
static std::mutex g_pj_mu;

// The last 8-column tile when it holds a single bin (n_b = 8 (NT - 1) + 1, the 25-bin workload):
// that column is formed with FP32 FMAs instead of three MMAs on a tile 7/8 padding.  Lanes
// g = lane/4 = 0 hold column 0 of the tile in the B fragment (k = tq and tq + 4); every lane takes
// them by shuffle and adds its A fragment's rows g, g + 8 over its k pair; the four lanes tq of
// a row are summed per chunk (tail_close), so the lane tq = 0 holds the column, in the slots of
// the tile's column 0.
__device__ __forceinline__ void tail_col(float (&t)[2], const uint32_t (&a)[4], uint32_t b0, uint32_t b1, int tq) {
  const float y0 = __uint_as_float(__shfl_sync(0xffffffffu, b0, tq));
  const float y1 = __uint_as_float(__shfl_sync(0xffffffffu, b1, tq));
  t[0] = fmaf(__uint_as_float(a[0]), y0, fmaf(__uint_as_float(a[2]), y1, t[0]));
  t[1] = fmaf(__uint_as_float(a[1]), y0, fmaf(__uint_as_float(a[3]), y1, t[1]));
}
__device__ __forceinline__ void tail_close(float* c, float (&t)[2]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float v = t[h];
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    c[2 * h] = (threadIdx.x & 3) == 0 ? v : 0.f;  // (row g, col 0) and (row g + 8, col 0)
    c[2 * h + 1] = 0.f;
  }
}

// A warp's fragment addressing: ldmatrix row offsets and swizzled pieces, its term's sides
struct PairFrag {
  unsigned loffA, loffB[2], poffA[4], poffB[4];
  unsigned xoff, yoff;  // bare X (when not built) and Y component blocks
  int e0, e1;           // entries of the built X side
  int tq;
  bool xb;
};

// The products of NH consecutive 32-cell halves (from h0) of one staged chunk, accumulated into
// c.  The built sides of all NH halves and four k steps are formed in one pass over the side's
// entries (one table read and address per entry; the shared-memory loads are independent), then
// every k step loads and splits the bare side and issues its 3 NT MMAs.
template <int NT, int NH, bool TAIL1 = false>
__device__ __forceinline__ void pair_halves(float (&c)[16], const PairJob& J, const TmaLayout& L, unsigned sb,
                                            int h0, const float* Hs, const PairFrag& F) {
  constexpr int NM = TAIL1 ? NT - 1 : NT;  // column tiles on the tensor cores
  float tl[2] = {0.f, 0.f};
  uint32_t av[NH][4][4];
  if (F.xb) {
    // built side sum_(c,h) F_c(b, x) H_h(x) for this lane's fragment cells
    float s4[NH][4][4];
#pragma unroll
    for (int hh = 0; hh < NH; ++hh)
#pragma unroll
      for (int u = 0; u < 4; ++u) s4[hh][u][0] = s4[hh][u][1] = s4[hh][u][2] = s4[hh][u][3] = 0.f;
    for (int e = F.e0; e < F.e1; ++e) {
      const unsigned ao = sb + (unsigned)J.s_ent[e][0] * L.cblk + F.loffA;
      const float* hp = Hs + J.s_ent[e][1] * PR_CH + 2 * F.tq;
#pragma unroll
      for (int hh = 0; hh < NH; ++hh) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          uint32_t v[4];
          ldsm_x4(ao + (unsigned)(h0 + hh) * L.half + F.poffA[u], v);
          const float2 hv = *reinterpret_cast<const float2*>(hp + (h0 + hh) * 32 + 8 * u);
          s4[hh][u][0] = fmaf(__uint_as_float(v[0]), hv.x, s4[hh][u][0]);
          s4[hh][u][1] = fmaf(__uint_as_float(v[1]), hv.x, s4[hh][u][1]);
          s4[hh][u][2] = fmaf(__uint_as_float(v[2]), hv.y, s4[hh][u][2]);
          s4[hh][u][3] = fmaf(__uint_as_float(v[3]), hv.y, s4[hh][u][3]);
        }
      }
    }
#pragma unroll
    for (int hh = 0; hh < NH; ++hh)
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int e = 0; e < 4; ++e) av[hh][u][e] = __float_as_uint(s4[hh][u][e]);
  } else {
#pragma unroll
    for (int hh = 0; hh < NH; ++hh)
#pragma unroll
      for (int u = 0; u < 4; ++u) ldsm_x4(sb + (unsigned)(h0 + hh) * L.half + F.xoff + F.loffA + F.poffA[u], av[hh][u]);
  }
#pragma unroll
  for (int hh = 0; hh < NH; ++hh) {
    const unsigned fh = sb + (unsigned)(h0 + hh) * L.half + F.yoff;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      uint32_t bv[2][4];
      if (NT >= 2) {
#pragma unroll
        for (int i = 0; i < NT / 2; ++i) ldsm_x4(fh + F.loffB[i] + F.poffB[kk], bv[i]);
      } else {  // one n tile: matrices (k 0-3, k 4-7) of rows 0-7, addresses from lanes 0-15
        ldsm_x2(fh + F.loffB[0] + F.poffB[kk], bv[0]);
      }
      uint32_t ah[4], al[4], bh[4][2], bl[4][2];
#pragma unroll
      for (int e = 0; e < 4; ++e) split_tf32(av[hh][kk][e], ah[e], al[e]);
      if (NT >= 2) {
#pragma unroll
        for (int i = 0; i < NT / 2; ++i)
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (2 * i + (e >> 1) < NM) split_tf32(bv[i][e], bh[2 * i + (e >> 1)][e & 1], bl[2 * i + (e >> 1)][e & 1]);
      } else {
        split_tf32(bv[0][0], bh[0][0], bl[0][0]);
        split_tf32(bv[0][1], bh[0][1], bl[0][1]);
      }
      if constexpr (TAIL1) tail_col(tl, av[hh][kk], bv[NT / 2 - 1][2], bv[NT / 2 - 1][3], F.tq);
      // small products first, pass-major so that consecutive MMAs are independent
#pragma unroll
      for (int ni = 0; ni < NM; ++ni) mma_tf32(c + ni * 4, al, bh[ni]);
#pragma unroll
      for (int ni = 0; ni < NM; ++ni) mma_tf32(c + ni * 4, ah, bl[ni]);
#pragma unroll
      for (int ni = 0; ni < NM; ++ni) mma_tf32(c + ni * 4, ah, bh[ni]);
    }
  }
  if constexpr (TAIL1) tail_close(c + 4 * (NT - 1), tl);
}

// Two terms in one warp: terms t and t + 1 with the same bare Y side and the same components
// on their built X sides, which differ only in the H rows (the two G sets of a launch).  Per
// cell half the two built sides share every ldmatrix load; per k step the bare side's fragments
// are loaded and split once for both terms' 24 MMAs.
template <int NT, bool TAIL1 = false>
__device__ __forceinline__ void pair_dual(float (&ca)[16], float (&cb)[16], const PairJob& J, const TmaLayout& L,
                                          unsigned sb, const float* Hs, const PairFrag& F, int f0) {
  constexpr int NM = TAIL1 ? NT - 1 : NT;  // column tiles on the tensor cores
  float tl[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    uint32_t av[2][4][4];
    {
      float s4[2][4][4];
#pragma unroll
      for (int z = 0; z < 2; ++z)
#pragma unroll
        for (int u = 0; u < 4; ++u) s4[z][u][0] = s4[z][u][1] = s4[z][u][2] = s4[z][u][3] = 0.f;
      for (int e = F.e0, e2 = f0; e < F.e1; ++e, ++e2) {
        const unsigned ao = sb + (unsigned)hh * L.half + (unsigned)J.s_ent[e][0] * L.cblk + F.loffA;
        const float* hpa = Hs + J.s_ent[e][1] * PR_CH + hh * 32 + 2 * F.tq;
        const float* hpb = Hs + J.s_ent[e2][1] * PR_CH + hh * 32 + 2 * F.tq;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          uint32_t v[4];
          ldsm_x4(ao + F.poffA[u], v);
          const float2 ha = *reinterpret_cast<const float2*>(hpa + 8 * u);
          const float2 hb = *reinterpret_cast<const float2*>(hpb + 8 * u);
          s4[0][u][0] = fmaf(__uint_as_float(v[0]), ha.x, s4[0][u][0]);
          s4[0][u][1] = fmaf(__uint_as_float(v[1]), ha.x, s4[0][u][1]);
          s4[0][u][2] = fmaf(__uint_as_float(v[2]), ha.y, s4[0][u][2]);
          s4[0][u][3] = fmaf(__uint_as_float(v[3]), ha.y, s4[0][u][3]);
          s4[1][u][0] = fmaf(__uint_as_float(v[0]), hb.x, s4[1][u][0]);
          s4[1][u][1] = fmaf(__uint_as_float(v[1]), hb.x, s4[1][u][1]);
          s4[1][u][2] = fmaf(__uint_as_float(v[2]), hb.y, s4[1][u][2]);
          s4[1][u][3] = fmaf(__uint_as_float(v[3]), hb.y, s4[1][u][3]);
        }
      }
#pragma unroll
      for (int z = 0; z < 2; ++z)
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int e = 0; e < 4; ++e) av[z][u][e] = __float_as_uint(s4[z][u][e]);
    }
    const unsigned fh = sb + (unsigned)hh * L.half + F.yoff;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      uint32_t bv[2][4];
#pragma unroll
      for (int i = 0; i < NT / 2; ++i) ldsm_x4(fh + F.loffB[i] + F.poffB[kk], bv[i]);
      uint32_t bh[4][2], bl[4][2];
#pragma unroll
      for (int i = 0; i < NT / 2; ++i)
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (2 * i + (e >> 1) < NM) split_tf32(bv[i][e], bh[2 * i + (e >> 1)][e & 1], bl[2 * i + (e >> 1)][e & 1]);
#pragma unroll
      for (int z = 0; z < 2; ++z) {
        float* c = z ? cb : ca;
        uint32_t ah[4], al[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split_tf32(av[z][kk][e], ah[e], al[e]);
        if constexpr (TAIL1) tail_col(tl[z], av[z][kk], bv[NT / 2 - 1][2], bv[NT / 2 - 1][3], F.tq);
#pragma unroll
        for (int ni = 0; ni < NM; ++ni) mma_tf32(c + ni * 4, al, bh[ni]);
#pragma unroll
        for (int ni = 0; ni < NM; ++ni) mma_tf32(c + ni * 4, ah, bl[ni]);
#pragma unroll
        for (int ni = 0; ni < NM; ++ni) mma_tf32(c + ni * 4, ah, bh[ni]);
      }
    }
  }
  if constexpr (TAIL1) {
    tail_close(ca + 4 * (NT - 1), tl[0]);
    tail_close(cb + 4 * (NT - 1), tl[1]);
  }
}

// MH 16-row tiles (b1) and NT 8-column tiles (b2) per term: (2, 4) covers 32 bins; launches over
// few bins (blocked unions, small bin sets) take (1, 2) for 16 bins or (1, 1) for 8, so that
// their MMAs and staged bytes shrink with the bins.
template <int NTHR, int MH, int NT, int NST, bool DUAL = false, bool TAIL1 = false>
__global__ void __launch_bounds__(NTHR, 1)
    k_pair_tma(const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmG, const TmaLayout L,
               double* partials, int* err) {
  const PairJob& J = c_pj;
  extern __shared__ unsigned char dsm[];
  __shared__ int s_abort[2];  // per chunk parity (see the barrier below)
  const unsigned raw0 = smem_u32(dsm);
  const unsigned base = (raw0 + 1023u) & ~1023u;
  unsigned char* const gb = dsm + (base - raw0);  // generic pointer to the aligned base
  float* const Hs0 = reinterpret_cast<float*>(gb + L.hs);
  const unsigned bar0 = base + L.bar;
  constexpr int chc = PR_CH;  // cells per chunk: two 32-cell halves
  const int64_t nchunk = J.Ng / chc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the warp's term, cell half (2: both) and 16-row tile: rows 16 mi .. 16 mi + 15 of the term tile
  const int t = L.wterm[warp], hc = L.whalf[warp], mi = L.wrow[warp];
  const PairTermDesc T = J.term[t];
  unsigned long long pol = 0;
  if (tid == 0) {
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    for (int k = 0; k < NST; ++k) mbar_init(bar0 + 8u * k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort[0] = s_abort[1] = 0;
  }
  __syncthreads();
  int issued = 0;                         // thread 0: chunks whose copies were started
  auto issue = [&](int64_t ch, int st) {  // thread 0 only
    if (L.stall) return;
    ++issued;
    const unsigned bar = bar0 + 8u * st;
    mbar_expect_tx(bar, L.tx);
    for (int h = 0; h < 2; ++h) {
      const unsigned hb = base + st * L.stage + h * L.half;
      const int x = (int)(ch * chc + 32 * h);
      for (int c = 0; c < L.ncomp; ++c) tma_load_3d(hb + (unsigned)c * L.cblk, &tmF, x, c, 0, bar, pol);
      tma_load_2d(hb + L.fsz, &tmG, x, 0, bar, pol);
    }
  };

  constexpr int NTM = DUAL ? 2 : 1;  // terms per warp
  float2* slot =
      reinterpret_cast<float2*>(partials) + (((size_t)blockIdx.x * (blockDim.x >> 5) + warp) * 32 + lane) * (16 * NTM);
#pragma unroll
  for (int q = 0; q < 16 * NTM; ++q) slot[q] = make_float2(0.f, 0.f);
  // per chunk the MMA accumulators start from zero (the tensor core's accumulation stays at the
  // size of one chunk's products); chunk sums go to FP32 running sums over at most PR_FLUSH
  // chunks (1024 cells), which are added round robin with Kahan compensation to the lane's
  // (sum, compensation) slots
  float run[NTM][16];
#pragma unroll
  for (int z = 0; z < NTM; ++z)
#pragma unroll
    for (int q = 0; q < 16; ++q) run[z][q] = 0.f;

  // ldmatrix rows of this lane: matrix j = lane/8, row r = lane%8 of that matrix; every
  // fragment row is congruent to r mod 8, so its swizzled piece is (piece ^ r).
  // A: matrices (rows 0-7 | 8-15) x (k 0-3 | 4-7) of row block mi: row 16 mi + 8 (j&1) + r,
  //    piece 2 kk + (j>>1); registers hold cells (tq, tq, tq+4, tq+4)
  // B: matrices (ni k 0-3, ni k 4-7, ni+1 k 0-3, ni+1 k 4-7), ni = 2 i: row 8 (2i + (j>>1)) + r,
  //    piece 2 kk + (j&1)
  const int jm = lane >> 3, r = lane & 7, tq = lane & 3;
  const unsigned loffA = (unsigned)(16 * mi + 8 * (jm & 1) + r) * 128u;
  unsigned loffB[2], poffA[4], poffB[4];
#pragma unroll
  for (int i = 0; i < 2; ++i) loffB[i] = (unsigned)(8 * (2 * i + (jm >> 1)) + r) * 128u;
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    poffA[kk] = (unsigned)((2 * kk + (jm >> 1)) ^ r) << 4;
    poffB[kk] = (unsigned)((2 * kk + (jm & 1)) ^ r) << 4;
  }
  // terms are normalised so that only the X (A operand) side can be built
  const bool xb = T.xslot >= 0;
  const int e0 = xb ? J.s_off[T.xslot] : 0, e1 = xb ? J.s_off[T.xslot + 1] : 0;
  const unsigned xoff = xb ? 0u : (unsigned)T.xdir * L.cblk, yoff = (unsigned)T.ydir * L.cblk;
#ifdef BISP_CHECKED
  // every shared-memory row this warp's term addresses lies in the staged blocks and H buffers
  if (lane == 0) {
    BISP_DCHECK(T.ydir >= 0 && T.ydir < L.ncomp && (xb || (T.xdir >= 0 && T.xdir < L.ncomp)), 30, t);
    const int tl = DUAL ? t + 1 : t;
    for (int u = t; u <= tl; ++u) {
      const PairTermDesc& U = J.term[u];
      if (U.xslot < 0) continue;
      for (int e = J.s_off[U.xslot]; e < J.s_off[U.xslot + 1]; ++e)
        BISP_DCHECK(J.s_ent[e][0] >= 0 && J.s_ent[e][0] < L.ncomp && J.s_ent[e][1] >= 0 && J.s_ent[e][1] < J.nh, 31,
                    e);
    }
    if (warp == 0)
      for (int e = 0; e < J.h_off[J.nh]; ++e) BISP_DCHECK(J.h_ent[e].g < L.gbox, 32, e);
  }
#endif

  // NST - 1 chunks staged ahead; chunk index it uses stage it % NST, phase (it / NST) & 1.
  // One barrier per chunk: once every thread has passed the barrier of chunk it, every warp
  // has finished chunk it - 1, so its stage takes chunk it + NST - 1 and its H buffer (it + 1) & 1
  // is free.  The abort flag of chunk it is s_abort[it & 1]: a thread that sets the flag of
  // chunk it + 1 has passed the barrier of chunk it, so every thread has read the same slot for
  // chunk it - 1 before.
  if (tid == 0)
    for (int k = 0; k < NST - 1; ++k)
      if (blockIdx.x + (int64_t)k * gridDim.x < nchunk) issue(blockIdx.x + (int64_t)k * gridDim.x, k);
  const int nhi = J.nh << 4;
  int it = 0;
  for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x, ++it) {
    const int st = NST == 2 ? (it & 1) : it % NST;
    // slot it % 16 is flushed at the end of this chunk; load it now so that the L2 round
    // trip overlaps the chunk's work
    const int fg = it & 15;
    float2 pre[NTM];
#pragma unroll
    for (int z = 0; z < NTM; ++z) pre[z] = slot[16 * z + fg];
    if (!mbar_wait_bounded(bar0 + 8u * st, NST == 2 ? ((unsigned)it >> 1) & 1u : (unsigned)(it / NST) & 1u)) {
      s_abort[it & 1] = 1;
      atomicExch(err, 1);
    }
    const unsigned sbo = st * L.stage;  // offset of this stage
    float* const Hs = Hs0 + (it & 1) * (J.nh * chc);
    // (1) H rows, stored per half as [kk][tq][cell tq | cell tq+4]; the items go to the last
    // threads first (the host orders terms heaviest first, so these are the lightest warps)
    for (int i = (int)blockDim.x - 1 - tid; i < nhi; i += blockDim.x) {
      const int h = i >> 4, q = i & 15, hh = q >> 3, p = q & 7;
      const unsigned char* g0 = gb + sbo + hh * L.half + L.fsz;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int e = J.h_off[h]; e < J.h_off[h + 1]; ++e) {
        const PairRecipe R = J.h_ent[e];
        const float coef = R.coef;
        if (R.g >= 0) {
          const float4 gv = *reinterpret_cast<const float4*>(g0 + swz(R.g, p));
          v.x = fmaf(coef, gv.x, v.x);
          v.y = fmaf(coef, gv.y, v.y);
          v.z = fmaf(coef, gv.z, v.z);
          v.w = fmaf(coef, gv.w, v.w);
        } else {
          v.x += coef;
          v.y += coef;
          v.z += coef;
          v.w += coef;
        }
      }
      // cells 4p..4p+3 of half hh: step kk = p/2, slot s = p%2 of the pairs of lanes tq = 0..3
      float* d = Hs + h * chc + hh * 32 + (p >> 1) * 8 + (p & 1);
      d[0] = v.x;
      d[2] = v.y;
      d[4] = v.z;
      d[6] = v.w;
    }
    __syncthreads();
    if (s_abort[it & 1]) break;
    const int64_t nx = ch + (int64_t)(NST - 1) * gridDim.x;
    if (tid == 0 && nx < nchunk) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(nx, NST == 2 ? (st ^ 1) : (it + NST - 1) % NST);
    }
    // (2) this warp's 16 x 32 block of its term over its cell half (or both halves)
    float c[NTM][16];
#pragma unroll
    for (int z = 0; z < NTM; ++z)
#pragma unroll
      for (int q = 0; q < 16; ++q) c[z][q] = 0.f;
    const PairFrag F{loffA, {loffB[0], loffB[1]}, {poffA[0], poffA[1], poffA[2], poffA[3]},
                     {poffB[0], poffB[1], poffB[2], poffB[3]}, xoff, yoff, e0, e1, tq, xb};
    if constexpr (DUAL)
      pair_dual<NT, TAIL1>(c[0], c[NTM - 1], J, L, base + sbo, Hs, F, J.s_off[J.term[t + 1].xslot]);
    else if (hc == 2)
      pair_halves<NT, 2, TAIL1>(c[0], J, L, base + sbo, 0, Hs, F);
    else
      pair_halves<NT, 1, TAIL1>(c[0], J, L, base + sbo, hc, Hs, F);
#pragma unroll
    for (int z = 0; z < NTM; ++z)
#pragma unroll
      for (int q = 0; q < 16; ++q) run[z][q] += c[z][q];
    // round-robin flush: each FP32 running sum covers at most 16 chunks (1024 cells); fg is
    // warp-uniform, so the switch is one indexed branch
#pragma unroll
    for (int z = 0; z < NTM; ++z) {
      float x = 0.f;
      switch (fg) {
#define BISP_TAKE(q)  \
  case q:             \
    x = run[z][q];    \
    run[z][q] = 0.f;  \
    break;
        BISP_TAKE(0) BISP_TAKE(1) BISP_TAKE(2) BISP_TAKE(3) BISP_TAKE(4) BISP_TAKE(5) BISP_TAKE(6) BISP_TAKE(7)
        BISP_TAKE(8) BISP_TAKE(9) BISP_TAKE(10) BISP_TAKE(11) BISP_TAKE(12) BISP_TAKE(13) BISP_TAKE(14) BISP_TAKE(15)
#undef BISP_TAKE
      }
      kahan_add(pre[z], x);
      slot[16 * z + fg] = pre[z];
    }
  }
  const bool aborted = it < (nchunk - (int64_t)blockIdx.x + gridDim.x - 1) / gridDim.x;  // left at a break
  // the running sums not flushed since their last turn
  if (!aborted) {
#pragma unroll
    for (int z = 0; z < NTM; ++z)
#pragma unroll
      for (int q = 0; q < 16; ++q) kahan_add(slot[16 * z + q], run[z][q]);
  }
  // after an abort the copies of the failed chunk and of the chunks staged ahead may still be in
  // flight: wait for them (bounded) before the CTA's shared memory is released
  if (tid == 0 && aborted)
    for (int k = it; k < issued; ++k) mbar_wait_bounded(bar0 + 8u * (k % NST), (unsigned)(k / NST) & 1u);
}

// ------------------------------------------------------------------------------------
// 5th-generation tensor-core variant (tcgen05; nb <= 32, at most 4 bare components and 8
// terms per launch).  Chunks of 32 cells are staged by the same TMA tensor maps as
// k_pair_tma.  Terms are normalised so that the built side is X and the bare side Y.  One
// tcgen05.mma per k step and pass covers the whole launch: A (M = 128) stacks the bare
// components (32 bins each), B (N = 32 x terms) stacks the built sides, and the useful
// 32 x 32 blocks of D (TMEM: lane = A row, column = B row) are those pairing a term's built
// side with its own bare component.  Per chunk every warp (1) forms the H rows, (2) builds
// X = sum_(c,h) F_c H_h and splits it, and the bare sides, into TF32 hi/lo tiles in the
// K-major 128-byte-swizzled layout the MMA reads; then one thread issues 4 k steps x 3
// passes (lo.hi, hi.lo, hi.hi) into a TMEM accumulator double-buffered over chunks.  While
// the tensor cores work on chunk i the warps read chunk i-1 back with tcgen05.ld (the warp
// of a term sits in the TMEM lane quarter of its bare component) into FP32 running sums
// over at most UM_FLUSH chunks, which go round robin into lane-owned Kahan (sum,
// compensation) slots.  The accumulator restarts every chunk.  Measured on GB300: an
// M = 128 kind::tf32 MMA costs ~48 cycles up to N = 64 and reaches ~2000 MAC/cycle from
// N = 128, so few wide MMAs beat many narrow ones.  Every wait is bounded in time; TMEM is
// freed on every path.  On the 512^3 survey jobs this kernel is bound by shared-memory
// bandwidth (the three TF32 passes need materialised hi/lo tiles: ~230 KB of shared-memory
// traffic per 32-cell chunk between the side builds and the MMA operand reads) and runs
// slower than k_pair_tma, which keeps the split in registers; it is therefore opt-in.
// ------------------------------------------------------------------------------------
constexpr int UM_WARPS = 16;
constexpr int UM_CH = 32;     // cells per chunk
constexpr int UM_FLUSH = 32;  // chunks per FP32 running sum (1024 cells)
constexpr int UM_MAXB = 4;    // bare components (A = 4 x 32 rows)
constexpr int UM_MAXS = 8;    // terms (B = 8 x 32 rows at most)

struct UmmaPlan {
  int nslots, nbare;
  int bare_comp[UM_MAXB];  // component of each 32-row A block
  int slot_side[UM_MAXS];  // side (s_off index) built into B block k
  int warp_slot[UM_WARPS];  // term slot read back by each warp, or -1
};

struct UmmaLayout {
  unsigned fsz, stage;               // F blocks (ncomp x 4096), raw stage (F + G block)
  unsigned ob, obsz;                 // operand buffers: offset, bytes each
  unsigned a_hi, a_lo, b_hi, b_lo;   // tiles within an operand buffer
  unsigned hs, bar, tptr, bytes, tx, tcols;
  unsigned idesc, dcols;             // instruction descriptor (N = 32 x terms), columns per D
  int ncomp, nob;
};

__device__ __forceinline__ uint64_t umma_sdesc(unsigned addr) {
  // K-major, 128-byte swizzle: start >> 4, stride between 8-row groups 1024 B, version 1
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// kind::tf32, FP32 accumulate, K-major A and B, M = 128, N = n
__host__ __device__ constexpr uint32_t umma_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(unsigned dcol, uint64_t da, uint64_t db, unsigned idesc, unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld32(unsigned ta, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ float4 split_hi4(float4 v) {
  return make_float4(__uint_as_float(__float_as_uint(v.x) & 0xffffe000u), __uint_as_float(__float_as_uint(v.y) & 0xffffe000u),
                     __uint_as_float(__float_as_uint(v.z) & 0xffffe000u), __uint_as_float(__float_as_uint(v.w) & 0xffffe000u));
}

__global__ void __launch_bounds__(UM_WARPS * 32, 1)
    k_pair_umma(const __grid_constant__ PairJob J, const __grid_constant__ UmmaPlan U,
                const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmG, const UmmaLayout L,
                float2* slots, int* err) {
  extern __shared__ unsigned char dsm[];
  __shared__ int s_abort;
  const unsigned raw0 = smem_u32(dsm);
  const unsigned base = (raw0 + 1023u) & ~1023u;
  unsigned char* const gb = dsm + (base - raw0);
  float* const Hs = reinterpret_cast<float*>(gb + L.hs);
  const unsigned barF = base + L.bar, barM = barF + 16;  // TMA stages full[2], MMA done[2]
  const int64_t nchunk = J.Ng / UM_CH;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(base + L.tptr), "r"(L.tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  unsigned long long pol = 0;
  if (tid == 0) {
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    for (int k = 0; k < 4; ++k) mbar_init(barF + 8u * k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  tc_before();
  __syncthreads();
  tc_after();
  const unsigned tmem = *reinterpret_cast<const unsigned*>(gb + L.tptr);
  auto issue = [&](int64_t ch, int st) {  // thread 0 only
    const unsigned bar = barF + 8u * st;
    mbar_expect_tx(bar, L.tx);
    const unsigned rb = base + st * L.stage;
    const int x = (int)(ch * UM_CH);
    for (int c = 0; c < L.ncomp; ++c) tma_load_3d(rb + (unsigned)c * 4096u, &tmF, x, c, 0, bar, pol);
    tma_load_2d(rb + L.fsz, &tmG, x, 0, bar, pol);
  };
  // readout role: the warp of term slot k sits in the lane quarter of its bare component
  // (lane = bin of the bare side, run[] = bins of the built side)
  const int rslot = U.warp_slot[warp];
  const bool reader = rslot >= 0;
  float2* slot = slots + (((size_t)blockIdx.x * UM_WARPS + warp) * 32 + lane) * 32;
#pragma unroll
  for (int q = 0; q < 32; ++q) slot[q] = make_float2(0.f, 0.f);
  float run[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) run[q] = 0.f;
  auto readout = [&](int itr) {  // chunk with iteration index itr, all reader lanes
    uint32_t r[32];
    tmem_ld32(tmem + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)(itr & 1) * L.dcols + (unsigned)rslot * 32u, r);
#pragma unroll
    for (int q = 0; q < 32; ++q) run[q] += __uint_as_float(r[q]);
  };
  const unsigned mnb = (unsigned)((0x100000000ull + 8 * J.nb - 1) / (8 * J.nb));  // j / (8 nb) = umulhi(j, mnb)
  int it = 0, tma_issued = 0;
  if (tid == 0) {
    if (blockIdx.x < nchunk) issue(blockIdx.x, 0), ++tma_issued;
    if (blockIdx.x + gridDim.x < nchunk) issue(blockIdx.x + gridDim.x, 1), ++tma_issued;
  }
  for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x, ++it) {
    const int st = it & 1;
    const unsigned obase = base + L.ob + (unsigned)(L.nob == 2 ? st : 0) * L.obsz;
    unsigned char* const og = gb + (obase - base);
    if (!mbar_wait_bounded(barF + 8u * st, (unsigned)(it >> 1) & 1u)) {
      s_abort = 1;
      atomicExch(err, 1);
    }
    const unsigned char* const rs = gb + st * L.stage;  // raw stage (generic pointer)
    const int fq = it & (UM_FLUSH - 1);
    float2 pre = reader ? slot[fq] : make_float2(0.f, 0.f);
    // (1) H rows of this chunk: [h][32 cells]
    for (int i = tid; i < (J.nh << 3); i += blockDim.x) {
      const int h = i >> 3, p = i & 7;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int e = J.h_off[h]; e < J.h_off[h + 1]; ++e) {
        const PairRecipe R = J.h_ent[e];
        if (R.g >= 0) {
          const float4 gv = *reinterpret_cast<const float4*>(rs + L.fsz + swz(R.g, p));
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
      *reinterpret_cast<float4*>(Hs + h * UM_CH + 4 * p) = v;
    }
    __syncthreads();
    if (s_abort) break;
    // (2) with a single operand buffer, the previous chunk's MMAs must have read it
    if (L.nob == 1 && it > 0 && !mbar_wait_bounded(barM + 8u * ((it - 1) & 1), (unsigned)((it - 1) >> 1) & 1u)) {
      s_abort = 1;
      atomicExch(err, 2);
    }
    // built sides, split into TF32 hi / lo tiles: one thread per (slot, bin, 4-cell piece)
    for (int i = tid; i < U.nslots * J.nb * 8; i += blockDim.x) {
      const int k = (int)__umulhi((unsigned)i, mnb);
      const int rem = i - k * J.nb * 8, b = rem >> 3, p = rem & 7;
      const int sd = U.slot_side[k];
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int e = J.s_off[sd]; e < J.s_off[sd + 1]; ++e) {
        const float4 f = *reinterpret_cast<const float4*>(rs + J.s_ent[e][0] * 4096 + swz(b, p));
        const float4 h = *reinterpret_cast<const float4*>(Hs + J.s_ent[e][1] * UM_CH + 4 * p);
        v.x = fmaf(f.x, h.x, v.x);
        v.y = fmaf(f.y, h.y, v.y);
        v.z = fmaf(f.z, h.z, v.z);
        v.w = fmaf(f.w, h.w, v.w);
      }
      const float4 hi = split_hi4(v);
      const unsigned o = (unsigned)k * 4096u + swz(b, p);
      *reinterpret_cast<float4*>(og + L.b_hi + o) = hi;
      *reinterpret_cast<float4*>(og + L.b_lo + o) = make_float4(v.x - hi.x, v.y - hi.y, v.z - hi.z, v.w - hi.w);
    }
    // bare sides
    for (int i = tid; i < U.nbare * J.nb * 8; i += blockDim.x) {
      const int u = (int)__umulhi((unsigned)i, mnb);
      const int rem = i - u * J.nb * 8, b = rem >> 3, p = rem & 7;
      const float4 v = *reinterpret_cast<const float4*>(rs + U.bare_comp[u] * 4096 + swz(b, p));
      const float4 hi = split_hi4(v);
      const unsigned o = (unsigned)u * 4096u + swz(b, p);
      *reinterpret_cast<float4*>(og + L.a_hi + o) = hi;
      *reinterpret_cast<float4*>(og + L.a_lo + o) = make_float4(v.x - hi.x, v.y - hi.y, v.z - hi.z, v.w - hi.w);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_before();
    __syncthreads();
    tc_after();
    if (s_abort) break;
    // (3) this chunk's MMAs, then the TMA of chunk it+2 into the stage the build has consumed
    if (tid == 0) {
      const unsigned dc = tmem + (unsigned)st * L.dcols;
      const unsigned ah = obase + L.a_hi, al = obase + L.a_lo, bh = obase + L.b_hi, bl = obase + L.b_lo;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        umma_tf32(dc, umma_sdesc(al + 32 * kk), umma_sdesc(bh + 32 * kk), L.idesc, kk > 0);
        umma_tf32(dc, umma_sdesc(ah + 32 * kk), umma_sdesc(bl + 32 * kk), L.idesc, 1u);
        umma_tf32(dc, umma_sdesc(ah + 32 * kk), umma_sdesc(bh + 32 * kk), L.idesc, 1u);
      }
      umma_commit(barM + 8u * st);
      if (ch + 2 * (int64_t)gridDim.x < nchunk) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(ch + 2 * (int64_t)gridDim.x, st);
        ++tma_issued;
      }
    }
    // (4) read back the previous chunk while the tensor cores work on this one
    if (it > 0 && reader) {
      if (__all_sync(0xffffffffu, mbar_wait_bounded(barM + 8u * ((it - 1) & 1), (unsigned)((it - 1) >> 1) & 1u))) {
        tc_after();
        readout(it - 1);
      } else {
        s_abort = 1;
        atomicExch(err, 3);
      }
    }
    // round-robin compensated flush of one running sum
    if (reader) {
      float x = 0.f;
#pragma unroll
      for (int q = 0; q < 32; ++q)
        if (q == fq) {
          x = run[q];
          run[q] = 0.f;
        }
      kahan_add(pre, x);
      slot[fq] = pre;
    }
    tc_before();
  }
  // last chunk's read-back and the remaining running sums
  if (!s_abort && it > 0 && reader) {
    if (__all_sync(0xffffffffu, mbar_wait_bounded(barM + 8u * ((it - 1) & 1), (unsigned)((it - 1) >> 1) & 1u))) {
      tc_after();
      readout(it - 1);
#pragma unroll
      for (int q = 0; q < 32; ++q) kahan_add(slot[q], run[q]);
    } else {
      atomicExch(err, 4);
    }
  }
  // after an abort: let in-flight TMA copies and MMAs finish (bounded) before freeing TMEM
  if (tid == 0 && s_abort) {
    // the loop leaves before issuing chunk it's MMAs: chunk it-1's are the last ones
    if (it > 0) mbar_wait_bounded(barM + 8u * ((it - 1) & 1), (unsigned)((it - 1) >> 1) & 1u);
    for (int k = it; k < tma_issued; ++k) mbar_wait_bounded(barF + 8u * (k & 1), (unsigned)(k >> 1) & 1u);
  }
  tc_before();
  __syncthreads();
  tc_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L.tcols));
}

// out[o][b1][b2] from the compensated slots of k_pair_umma: term t lives in warp
// 4 grp + quad, lane = bin of its bare side, slot = bin of its built side (T.tr says which of
// the output's two bins is the lane); fixed-order sums over CTAs.
__global__ void k_pair_umma_final(const __grid_constant__ PairJob J, const float2* slots, int nblk, int nb, int nout,
                                  double* out) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (gw >= nout * nb * nb) return;
  const int o = gw / (nb * nb), c1 = (gw / nb) % nb, c2 = gw % nb;
  double tot = 0.0;
  for (int e = J.out_ent_off[o]; e < J.out_ent_off[o + 1]; ++e) {
    const PairTermDesc& T = J.term[J.out_ent_term[e]];
    const int b1 = T.tr ? c2 : c1, b2 = T.tr ? c1 : c2;
    const int w = 4 * T.grp + T.quad;
    double s = 0.0;
    for (int c = lane; c < nblk; c += 32) {
      const float2 v = slots[(((size_t)c * UM_WARPS + w) * 32 + b1) * 32 + b2];
      s += (double)v.x - (double)v.y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    tot += J.out_ent_mult[e] * s;
  }
  if (lane == 0) out[gw] = tot;
}

static bool tma_layout(const PairJob& j, TmaLayout* L, int* warps) {
  if (j.nb > 32 || (j.nb <= 16 ? 1 : 2) * j.nterm > TMA_MAXWARP || j.ng < 1 || j.ng > 256 || j.ncomp < 1)
    return false;
  auto r1024 = [](size_t b) { return (b + 1023) / 1024 * 1024; };
  const int mh = j.nb <= 16 ? 1 : 2, nt = j.nb <= 8 ? 1 : (j.nb <= 16 ? 2 : 4);
  const int bh = std::max(16 * mh, 8 * nt);  // bins staged per component block
  const size_t fsz = (size_t)j.ncomp * bh * 128, gsz = r1024((size_t)j.ng * 128);
  const size_t half = fsz + gsz, stage = 2 * half;
  const char* env = getenv("BISP_PAIR_STAGES");
  int nst = env && atoi(env) == 2 ? 2 : 3;
  size_t hs = 0, bar = 0, bytes = 0;
  for (; nst >= 2; --nst) {
    hs = (size_t)nst * stage;
    bar = (hs + 2 * (size_t)j.nh * PR_CH * 4 + 15) / 16 * 16;
    bytes = bar + ((size_t)8 * nst + 15) / 16 * 16 + 1024;
    if (bytes <= 227 * 1024 - 256) break;
  }
  if (nst < 2) return false;
  L->nst = nst;
  L->nblk = pair_blocks();
  L->fsz = (unsigned)fsz;
  L->gsz = (unsigned)gsz;
  L->half = (unsigned)half;
  L->stage = (unsigned)stage;
  L->hs = (unsigned)hs;
  L->bar = (unsigned)bar;
  L->bytes = (unsigned)bytes;
  L->ncomp = j.ncomp;
  L->gbox = j.ng;
  L->tx = (unsigned)(2 * (fsz + (size_t)j.ng * 128));
  L->stall = 0;
  L->mh = mh;
  L->nt = nt;
  L->cblk = (unsigned)(bh * 128);
  // Warps.  Work per warp and chunk ~ (entries of the built side + 6.5) per cell half (6.5:
  // the bare side's loads and splits and the MMAs, in units of one entry).  Every term starts
  // with one warp per row tile over both halves; while warps are few (at most 8 after doubling)
  // every term splits its halves over two warps; otherwise the term with the most work per warp
  // splits while that work is more than 15 % above the mean and the warps stay within 12 (the
  // 384-thread instance).  BISP_PAIR_KSPLIT=1 or 2 forces one warp over both halves or one per
  // half for every term (2 while the warps fit the launch).
  // two-term warps (pair_dual) when every term sits next to a partner and pairing brings a
  // launch that would exceed the 384-thread instance back into it (the unit-shell launch's two G
  // sets: 20 warps -> 10); BISP_PAIR_DUAL=0 never, 1 whenever the terms pair
  {
    const char* ed = getenv("BISP_PAIR_DUAL");
    const int fd = ed ? atoi(ed) : -1;
    bool adj = mh == 2 && j.nterm % 2 == 0 && fd != 0;
    for (int u = 0; adj && 2 * u < j.nterm; ++u) adj = pairable(j, 2 * u, 2 * u + 1);
    if (adj && (j.nterm / 2) * mh <= 12 && (fd == 1 || j.nterm * mh > 12)) {
      const int w = (j.nterm / 2) * mh;
      for (int u = 0; 2 * u < j.nterm; ++u) {
        for (int z = 0; z < 2; ++z) {
          L->tfirst[2 * u + z] = (unsigned char)(u * mh);
          L->tsplit[2 * u + z] = 1;
          L->tsub[2 * u + z] = (unsigned char)z;
        }
        for (int mi = 0; mi < mh; ++mi) {
          L->wterm[u * mh + mi] = (unsigned char)(2 * u);
          L->whalf[u * mh + mi] = 2;
          L->wrow[u * mh + mi] = (unsigned char)mi;
        }
      }
      L->ntm = 2;
      *warps = w;
      return true;
    }
  }
  L->ntm = 1;
  const char* eks = getenv("BISP_PAIR_KSPLIT");
  const int force = eks ? atoi(eks) : 0;
  int split[64];
  double cost[64], tot = 0.0;
  for (int t = 0; t < j.nterm; ++t) {
    const PairTermDesc& T = j.term[t];
    const int sl = T.xslot >= 0 ? T.xslot : T.yslot;
    cost[t] = (sl >= 0 ? j.s_off[sl + 1] - j.s_off[sl] : 0) + 6.5;
    tot += cost[t];
    split[t] = 1;
  }
  int w = mh * j.nterm;
  if (force == 2 ? 2 * w <= TMA_MAXWARP : (force != 1 && 2 * w <= 8)) {
    for (int t = 0; t < j.nterm; ++t) split[t] = 2;
    w *= 2;
  } else if (force != 1) {
    for (;;) {
      int tm = 0, nsp = 0;
      for (int t = 0; t < j.nterm; ++t) {
        nsp += split[t];
        if (cost[t] / split[t] > cost[tm] / split[tm]) tm = t;
      }
      if (split[tm] == 1 && cost[tm] > 1.15 * tot / nsp && w + mh <= 12) {
        split[tm] = 2;
        w += mh;
      } else {
        break;
      }
    }
  }
  if (w > TMA_MAXWARP) return false;
  int k = 0;
  for (int t = 0; t < j.nterm; ++t) {
    L->tfirst[t] = (unsigned char)k;
    L->tsplit[t] = (unsigned char)split[t];
    L->tsub[t] = 0;
    for (int h = 0; h < split[t]; ++h)
      for (int mi = 0; mi < mh; ++mi, ++k) {
        L->wterm[k] = (unsigned char)t;
        L->whalf[k] = (unsigned char)(split[t] == 2 ? h : 2);
        L->wrow[k] = (unsigned char)mi;
      }
  }
  *warps = w;
  return true;
}

// Layout of k_pair_umma for a job whose built sides are all X: the bare Y components become
// the 32-row blocks of A, the built sides the 32-row blocks of B; a term whose X is bare gets
// a built side with the single entry (component, H row of ones).  Fills T.grp / T.quad (the
// reading warp is 4 grp + quad, quad = the term's bare block) and flips T.tr (the lane holds
// the bin of the bare side).
static bool umma_plan(PairJob& j, UmmaPlan* U, UmmaLayout* L) {
  if (j.nb > 32 || j.ng < 1 || j.ng > 256 || j.ncomp < 1 || j.nterm > UM_MAXS) return false;
  std::memset(U, 0, sizeof(*U));
  int hone = -1;
  for (int t = 0; t < j.nterm; ++t) {
    PairTermDesc& T = j.term[t];
    if (T.ydir < 0 || (T.xdir < 0 && T.xslot < 0)) return false;
    if (T.xslot < 0) {  // bare X: built side c * 1
      if (hone < 0) {
        if (j.nh >= 128 || j.h_off[j.nh] >= 512) return false;
        hone = j.nh;
        j.h_ent[j.h_off[j.nh]] = {0, -1, 1.0f};
        j.h_off[j.nh + 1] = j.h_off[j.nh] + 1;
        ++j.nh;
      }
      if (j.nslot >= 64 || j.s_off[j.nslot] >= 512) return false;
      j.s_ent[j.s_off[j.nslot]][0] = T.xdir;
      j.s_ent[j.s_off[j.nslot]][1] = hone;
      j.s_off[j.nslot + 1] = j.s_off[j.nslot] + 1;
      T.xslot = j.nslot++;
      T.xdir = -1;
    }
  }
  int per_bare[UM_MAXB] = {0, 0, 0, 0};
  for (int w = 0; w < UM_WARPS; ++w) U->warp_slot[w] = -1;
  for (int t = 0; t < j.nterm; ++t) {
    PairTermDesc& T = j.term[t];
    int u = -1;
    for (int v = 0; v < U->nbare; ++v)
      if (U->bare_comp[v] == T.ydir) u = v;
    if (u < 0) {
      if (U->nbare == UM_MAXB) return false;
      u = U->nbare++;
      U->bare_comp[u] = T.ydir;
    }
    if (per_bare[u] == UM_WARPS / 4) return false;
    U->slot_side[t] = T.xslot;
    T.grp = per_bare[u]++;
    T.quad = u;
    T.tr = !T.tr;
    U->warp_slot[4 * T.grp + u] = t;
  }
  U->nslots = j.nterm;
  auto r1024 = [](size_t b) { return (b + 1023) / 1024 * 1024; };
  const size_t fsz = (size_t)j.ncomp * 4096, gsz = r1024((size_t)j.ng * 128), stage = fsz + gsz;
  // A: always 128 rows (blocks beyond nbare are never written: they only feed unread lanes)
  const size_t a_lo = 4 * 4096, b_hi = 2 * a_lo, b_lo = b_hi + (size_t)U->nslots * 4096;
  const size_t obsz = b_lo + (size_t)U->nslots * 4096;
  for (int nob = 2; nob >= 1; --nob) {
    const size_t ob = 2 * stage, hs = ob + nob * obsz;
    const size_t bar = (hs + (size_t)j.nh * UM_CH * 4 + 15) / 16 * 16;
    const size_t tptr = bar + 32, bytes = tptr + 16 + 1024;
    if (bytes > 227 * 1024 - 256) continue;
    L->fsz = (unsigned)fsz;
    L->stage = (unsigned)stage;
    L->ob = (unsigned)ob;
    L->obsz = (unsigned)obsz;
    L->a_hi = 0;
    L->a_lo = (unsigned)a_lo;
    L->b_hi = (unsigned)b_hi;
    L->b_lo = (unsigned)b_lo;
    L->hs = (unsigned)hs;
    L->bar = (unsigned)bar;
    L->tptr = (unsigned)tptr;
    L->bytes = (unsigned)bytes;
    L->tx = (unsigned)(fsz + (size_t)j.ng * 128);
    L->dcols = 32u * (unsigned)U->nslots;
    L->idesc = umma_idesc(32 * U->nslots);
    unsigned tc = 32;
    while (tc < 2 * L->dcols) tc *= 2;
    L->tcols = tc;
    L->ncomp = j.ncomp;
    L->nob = nob;
    return true;
  }
  return false;
}

// the tensor-core path runs k_pair_tma (mma.sync) unless BISP_PAIR_KERNEL=tcgen05 selects
// k_pair_umma, which is correct but slower on these jobs (see its header comment)
static bool pair_use_umma() {
  const char* e = getenv("BISP_PAIR_KERNEL");
  return e && std::string(e) == "tcgen05";
}

bool pair_split_gsets() { return pair_use_umma(); }

// a job with its terms normalised for the tensor-core kernels: the built side is X (a term
// with a built Y is computed as Y X^T and read back transposed)
// Terms reordered by the entries of their built side, heaviest first (stable), with the output
// table remapped: the TMA kernel hands the per-chunk H rows to the last warps, i.e. the lightest
// terms, which keeps the warps' work per chunk level.
static void heavy_first(PairJob& j) {
  int perm[64], inv[64];
  auto weight = [&](int t) {
    const int x = j.term[t].xslot;
    return x >= 0 ? j.s_off[x + 1] - j.s_off[x] : 0;
  };
  for (int t = 0; t < j.nterm; ++t) perm[t] = t;
  std::stable_sort(perm, perm + j.nterm, [&](int a, int b) { return weight(a) > weight(b); });
  const PairJob src = j;
  for (int n = 0; n < j.nterm; ++n) {
    j.term[n] = src.term[perm[n]];
    j.term_out[n] = src.term_out[perm[n]];
    inv[perm[n]] = n;
  }
  for (int e = 0; e < j.out_ent_off[j.nout]; ++e) j.out_ent_term[e] = inv[src.out_ent_term[e]];
}

// Terms a and b can share a warp (pair_dual): both built on X only, the same bare Y, the same
// orientation and the same components on their built sides (in order); only the H rows differ.
static bool pairable(const PairJob& j, int a, int b) {
  const PairTermDesc &A = j.term[a], &B = j.term[b];
  if (A.xslot < 0 || B.xslot < 0 || A.yslot >= 0 || B.yslot >= 0 || A.ydir != B.ydir || A.tr != B.tr) return false;
  const int na = j.s_off[A.xslot + 1] - j.s_off[A.xslot], nb = j.s_off[B.xslot + 1] - j.s_off[B.xslot];
  if (na != nb) return false;
  for (int e = 0; e < na; ++e)
    if (j.s_ent[j.s_off[A.xslot] + e][0] != j.s_ent[j.s_off[B.xslot] + e][0]) return false;
  return true;
}

// Reorders the terms so that every term sits next to a partner (terms 2u, 2u + 1 pairable),
// keeping the order of the first of each pair; false (job unchanged) unless every term has one.
static bool dual_order(PairJob& j) {
  if (j.nterm % 2) return false;
  int partner[64];
  for (int t = 0; t < j.nterm; ++t) partner[t] = -1;
  for (int a = 0; a < j.nterm; ++a) {
    if (partner[a] >= 0) continue;
    for (int b = a + 1; b < j.nterm; ++b)
      if (partner[b] < 0 && pairable(j, a, b)) {
        partner[a] = b;
        partner[b] = a;
        break;
      }
    if (partner[a] < 0) return false;
  }
  int perm[64], inv[64], n = 0;
  for (int a = 0; a < j.nterm; ++a)
    if (a < partner[a]) {
      perm[n++] = a;
      perm[n++] = partner[a];
    }
  const PairJob src = j;
  for (int k = 0; k < j.nterm; ++k) {
    j.term[k] = src.term[perm[k]];
    j.term_out[k] = src.term_out[perm[k]];
    inv[perm[k]] = k;
  }
  for (int e = 0; e < j.out_ent_off[j.nout]; ++e) j.out_ent_term[e] = inv[src.out_ent_term[e]];
  return true;
}

static PairJob normalised(const PairJob& j) {
  PairJob jt = j;
  for (int t = 0; t < jt.nterm; ++t) {
    PairTermDesc& T = jt.term[t];
    T.tr = 0;
    if (T.yslot >= 0) {
      std::swap(T.xoff, T.yoff);
      std::swap(T.xcnt, T.ycnt);
      std::swap(T.xdir, T.ydir);
      std::swap(T.xslot, T.yslot);
      T.tr = 1;
    }
  }
  return jt;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  if (!fn) throw Error{3, "cuTensorMapEncodeTiled is not available from the driver"};
  return fn;
}

// G fields: rows x Ng FP32 (row stride Ng), boxes of 32 cells x rows, 128-byte swizzle
static CUtensorMap g_map(const float* base, int64_t Ng, int rows) {
  CUtensorMap m;
  const cuuint64_t dim[2] = {(cuuint64_t)Ng, (cuuint64_t)rows};
  const cuuint64_t stride[1] = {(cuuint64_t)Ng * sizeof(float)};
  const cuuint32_t box[2] = {32, (cuuint32_t)rows};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = encode_tiled()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dim, stride, box,
                                    es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error{3, "cuTensorMapEncodeTiled (G fields) failed (" + std::to_string((int)r) + ")"};
  return m;
}

// component fields [nb][ncomp][Ng]: boxes of 32 cells x 1 component x 32 bins (bins >= nb
// are filled with zeros), 128-byte swizzle
static CUtensorMap f_map(const float* base, int64_t Ng, int ncomp, int nb, int bh = 32) {
  CUtensorMap m;
  const cuuint64_t dim[3] = {(cuuint64_t)Ng, (cuuint64_t)ncomp, (cuuint64_t)nb};
  const cuuint64_t stride[2] = {(cuuint64_t)Ng * sizeof(float), (cuuint64_t)Ng * ncomp * sizeof(float)};
  const cuuint32_t box[3] = {32, 1, (cuuint32_t)bh};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = encode_tiled()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dim, stride, box,
                                    es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error{3, "cuTensorMapEncodeTiled (component fields) failed (" + std::to_string((int)r) + ")"};
  return m;
}

static int pair_blocks() {
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm;
}

bool pair_fits(const PairJob& job) {
  try {
    const PairJob& j = classify(job);
    TmaLayout L;
    int warps = 1;
    if (pair_use_tc(j) && tma_layout(j, &L, &warps)) return true;
    const PairLaunch c = pair_launch_cfg(j);
    if (c.smem > 227 * 1024) return false;
    // instantiated kernels: up to 1024 threads for TM x TN <= 18, 512 above
    return c.warps * 32 <= (c.TM * c.TN > 18 ? 512 : 1024);
  } catch (const Error&) {
    return false;
  }
}

size_t pair_scratch_bytes(const PairJob& job) {
  const PairJob j = classify(job);  // a copy: the memo may be refilled below
  if (pair_use_tc(j) && pair_use_umma()) {
    PairJob jt = normalised(j);
    UmmaPlan U;
    UmmaLayout UL;
    if (umma_plan(jt, &U, &UL)) return (size_t)pair_blocks() * UM_WARPS * 32 * 32 * sizeof(float2) + 256;
  }
  TmaLayout L;
  int warps = 1;
  if (pair_use_tc(j) && tma_layout(j, &L, &warps)) return (size_t)L.nblk * warps * 32 * 16 * sizeof(float2) + 256;
  const PairLaunch c = pair_launch_cfg(j);
  return (size_t)c.nblk * c.warps * 32 * c.TM * c.TN * sizeof(double);
}


// final reduction for k_pair_tma (slots are compensated FP32 pairs (s, e), sum s - e): bin
// (b1, b2) of term t (after the transpose (b1, b2) -> (b2, b1) of terms with T.tr) sits in warps
// tfirst[t] + ks*mh + b1/16 for ks < tsplit[t], lane (b1%8)*4 + (b2%8)/2, slot
// 16 tsub[t] + (b2/8)*4 + ((b1/8)%2)*2 + b2%2 of the lane's 16 ntm slots
__global__ void k_pair_tc_final(const double* partials, int nblk, int warps, const TmaLayout L, int nb, int nout,
                                double* out) {
  const PairJob& J = c_pj;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (gw >= nout * nb * nb) return;
  const int o = gw / (nb * nb), c1 = (gw / nb) % nb, c2 = gw % nb;
  double tot = 0.0;
  for (int e = J.out_ent_off[o]; e < J.out_ent_off[o + 1]; ++e) {
    const int t = J.out_ent_term[e];
    const int b1 = J.term[t].tr ? c2 : c1, b2 = J.term[t].tr ? c1 : c2;
    const int ln = (b1 % 8) * 4 + (b2 % 8) / 2;
    const int q = (b2 / 8) * 4 + ((b1 / 8) % 2) * 2 + (b2 % 2);
    double s = 0.0;
    for (int ks = 0; ks < L.tsplit[t]; ++ks) {
      const int w = L.tfirst[t] + ks * L.mh + b1 / 16;
      for (int c = lane; c < nblk; c += 32) {
        const float2 v = reinterpret_cast<const float2*>(
            partials)[(((size_t)c * warps + w) * 32 + ln) * (16 * L.ntm) + 16 * L.tsub[t] + q];
        s += (double)v.x - (double)v.y;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    tot += J.out_ent_mult[e] * s;
  }
  if (lane == 0) out[gw] = tot;
}

// out[o][b1][b2] = sum over terms of o, then CTAs and x slices in a fixed order; one warp
// per output value, lanes stride over CTAs, fixed shuffle tree.
__global__ void k_pair_final(const __grid_constant__ PairJob J, const double* partials, int nblk, int warps,
                             int ksplit, int TM, int TN, int nb, int nout, double* out) {
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
                 int* launches, int* kernel, cudaEvent_t ev0, cudaEvent_t ev1) {
  const PairJob j = classify(job);
  auto mark = [&](cudaEvent_t e) {
    if (e) BISP_CUDA(cudaEventRecord(e, s));
  };
  if (scratch_bytes < pair_scratch_bytes(job)) throw Error{2, "pair reduction scratch too small"};
  if (j.Ng % PR_CH) throw Error{6, "mesh size not a multiple of the chunk"};
  double* partials = reinterpret_cast<double*>(scratch);
  if (pair_use_tc(j) && pair_use_umma()) {
    PairJob jt = normalised(j);
    UmmaPlan U;
    UmmaLayout UL;
    if (umma_plan(jt, &U, &UL)) {
      const int nblk = pair_blocks();
      float2* slots = reinterpret_cast<float2*>(scratch);
      int* err = reinterpret_cast<int*>(static_cast<unsigned char*>(scratch) +
                                        (size_t)nblk * UM_WARPS * 32 * 32 * sizeof(float2));
      BISP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
      const CUtensorMap mf = f_map(j.fields, j.Ng, j.ncomp, j.nb);
      const CUtensorMap mg = g_map(j.gfields, j.Ng, j.ng);
      BISP_CUDA(cudaFuncSetAttribute(k_pair_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)UL.bytes));
      mark(ev0);
      k_pair_umma<<<nblk, UM_WARPS * 32, UL.bytes, s>>>(jt, U, mf, mg, UL, slots, err);
      BISP_CHECK_LAUNCH();
      const int nout = j.nout * j.nb * j.nb;
      k_pair_umma_final<<<(nout * 32 + 255) / 256, 256, 0, s>>>(jt, slots, nblk, j.nb, j.nout, out_dev);
      BISP_CHECK_LAUNCH();
      mark(ev1);
      int herr = 0;
      BISP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
      BISP_CUDA(cudaStreamSynchronize(s));
      if (herr) throw Error{5, "pair reduction: a TMA stage or an MMA batch did not complete within 2 s"};
      if (launches) *launches += 2;
      if (kernel) *kernel = 2;
      return;
    }
  }
  TmaLayout L;
  int warps = 1;
  PairJob jt;
  if (pair_use_tc(j)) {
    // the mma.sync kernel builds only A operands (see normalised); its warp tables follow the
    // order of heavy_first
    jt = normalised(j);
    heavy_first(jt);
    if (j.nb > 16) dual_order(jt);
  }
  if (pair_use_tc(j) && tma_layout(jt, &L, &warps)) {
    const int nblk = L.nblk;
    const size_t need = (size_t)nblk * warps * 32 * 16 * L.ntm * sizeof(float2);
    if (need + sizeof(int) > scratch_bytes) throw Error{2, "pair reduction scratch too small"};
    int* err = reinterpret_cast<int*>(static_cast<unsigned char*>(scratch) + need);
    BISP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    const CUtensorMap mf = f_map(j.fields, j.Ng, j.ncomp, j.nb, (int)(L.cblk / 128));
    const CUtensorMap mg = g_map(j.gfields, j.Ng, j.ng);
    L.stall = inject_stall("pair") ? 1 : 0;
    // the constant slot is ours from the copy until the synchronisation at the end of this call
    std::lock_guard<std::mutex> lk(g_pj_mu);
    BISP_CUDA(cudaMemcpyToSymbolAsync(c_pj, &jt, sizeof(PairJob), 0, cudaMemcpyHostToDevice, s));
    auto launch = [&](auto kern) {
      BISP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes));
      mark(ev0);
      kern<<<nblk, warps * 32, L.bytes, s>>>(mf, mg, L, partials, err);
    };
    // launches of at most 12 warps take the instance bounded at 384 threads (more registers per
    // thread for the unrolled k steps)
    const bool small = warps <= 12;
    // 25 bins: the last column tile holds one bin (FP32 FMAs for it); BISP_PAIR_TAIL=0 keeps it
    // on the tensor cores
    const char* etl = getenv("BISP_PAIR_TAIL");
    const bool tail = L.mh == 2 && L.nt == 4 && j.nb == 25 && small && !(etl && atoi(etl) == 0);
    if (L.ntm == 2) {
      if (tail) L.nst == 3 ? launch(k_pair_tma<384, 2, 4, 3, true, true>) : launch(k_pair_tma<384, 2, 4, 2, true, true>);
      else L.nst == 3 ? launch(k_pair_tma<384, 2, 4, 3, true>) : launch(k_pair_tma<384, 2, 4, 2, true>);
    } else if (tail) {
      L.nst == 3 ? launch(k_pair_tma<384, 2, 4, 3, false, true>) : launch(k_pair_tma<384, 2, 4, 2, false, true>);
    } else if (L.nst == 3) {
      if (L.mh == 2) small ? launch(k_pair_tma<384, 2, 4, 3>) : launch(k_pair_tma<32 * TMA_MAXWARP, 2, 4, 3>);
      else if (L.nt == 2) small ? launch(k_pair_tma<384, 1, 2, 3>) : launch(k_pair_tma<32 * TMA_MAXWARP, 1, 2, 3>);
      else small ? launch(k_pair_tma<384, 1, 1, 3>) : launch(k_pair_tma<32 * TMA_MAXWARP, 1, 1, 3>);
    } else {
      if (L.mh == 2) small ? launch(k_pair_tma<384, 2, 4, 2>) : launch(k_pair_tma<32 * TMA_MAXWARP, 2, 4, 2>);
      else if (L.nt == 2) small ? launch(k_pair_tma<384, 1, 2, 2>) : launch(k_pair_tma<32 * TMA_MAXWARP, 1, 2, 2>);
      else small ? launch(k_pair_tma<384, 1, 1, 2>) : launch(k_pair_tma<32 * TMA_MAXWARP, 1, 1, 2>);
    }
    BISP_CHECK_LAUNCH();
    const int nout = j.nout * j.nb * j.nb;
    k_pair_tc_final<<<(nout * 32 + 255) / 256, 256, 0, s>>>(partials, nblk, warps, L, j.nb, j.nout, out_dev);
    BISP_CHECK_LAUNCH();
    mark(ev1);
    int herr = 0;
    BISP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BISP_CUDA(cudaStreamSynchronize(s));
    if (herr) throw Error{5, "pair reduction: a TMA stage did not arrive within 2 s"};
    if (launches) *launches += 2;
    if (kernel) *kernel = 1;
    return;
  }
  const PairLaunch c = pair_launch_cfg(j);
  if (c.smem > 227 * 1024) throw Error{6, "pair reduction: shared memory budget exceeded"};
#define BISP_PAIR3(A, B, NT)                                                                              \
  if (c.TM == A && c.TN == B && c.warps * 32 <= NT) {                                                   \
    BISP_CUDA(cudaFuncSetAttribute(k_pair<A, B, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem)); \
    k_pair<A, B, NT><<<c.nblk, c.warps * 32, c.smem, s>>>(j, c.nbp, c.bs, c.rows, c.ksplit, partials);           \
    launched = true;                                                                                     \
  }
#define BISP_PAIR(A, B) \
  if (!launched) BISP_PAIR3(A, B, 512) if (!launched) BISP_PAIR3(A, B, 1024)
#define BISP_PAIR_S(A, B) \
  if (!launched) BISP_PAIR3(A, B, 512)
  bool launched = false;
  mark(ev0);
  BISP_PAIR(1, 1) BISP_PAIR(2, 1) BISP_PAIR(3, 2) BISP_PAIR(4, 2) BISP_PAIR(5, 3) BISP_PAIR(6, 3)
  BISP_PAIR_S(7, 4) BISP_PAIR_S(8, 4) BISP_PAIR_S(10, 5)
#undef BISP_PAIR
#undef BISP_PAIR_S
#undef BISP_PAIR3
  if (!launched) throw Error{6, "pair reduction: no kernel for this shape"};
  BISP_CHECK_LAUNCH();
  const int nout = j.nout * j.nb * j.nb;
  k_pair_final<<<(nout * 32 + 255) / 256, 256, 0, s>>>(j, partials, c.nblk, c.warps, c.ksplit, c.TM, c.TN,
                                                       j.nb, j.nout, out_dev);
  BISP_CHECK_LAUNCH();
  mark(ev1);
  if (launches) *launches += 2;
  if (kernel) *kernel = 0;
}

}  // namespace bisp

