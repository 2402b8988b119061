// Host-side declarations shared by the .cu files of the library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

namespace bisp {

// NVTX range for the duration of a scope (stages of bisp_assign / bisp_measure show up by name
// in Nsight timelines; without a tool attached the calls do nothing)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---- error handling -------------------------------------------------------------
struct Error {
  int status;
  std::string msg;
};
#define BISP_CUDA(call)                                                                   \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw ::bisp::Error{3, std::string(#call) + ": " + cudaGetErrorString(e_)};         \
  } while (0)
#define BISP_CHECK_LAUNCH() BISP_CUDA(cudaGetLastError())
// Test knob: BISP_INJECT_STALL names kernels ("pair", "zpass") whose first launch in a library call
// starts none of its staged copies, so that its bounded waits run out and the call reports
// BISP_ETIMEOUT (no copy is left in flight).
bool inject_stall(const char* kernel);
// message returned by bisp_last_error() on the calling thread
void set_last_error(const std::string& m);

// ---- channel descriptors --------------------------------------------------------
// A channel is one real mesh: weight^power * (Re or Im)(y_L^M(x_hat) or its conjugate).
struct Chan {
  int L, M, part;  // part 0: real part, 1: imaginary part
  int power;       // 1: delta n channels (w y*), 2: N channels (w^2 y)
  int conj;        // 1: y_L^{M*}, 0: y_L^M
};

// device-side prep parameters
struct PrepArgs {
  const float* xyz;
  const float* w;      // or nullptr
  const float* nbar;   // or nullptr
  int64_t n;
  int N;
  double H, box;
  int mas;
  float P0;            // FKP P0 (0: off)
  int local;
  float obs[3];
  int nchan;
  Chan chan[32];
  const float* ynorm;  // (BISP_LMAX+1)^2 table
  // outputs
  uint32_t* keys;
  uint32_t* idx;
  float4* frac;        // dx, dy, dz, unused
  float* vals;         // [nchan][n]
  double* partials;    // [blocks][nsum]  sums: w, then w^3 * Re/Im y* for each D channel
  int nsum;
  int* bad;            // count of non-finite / out-of-box positions
  int selftest;        // checked build: record one failed check (site 99) with no other effect
};

// launches (defined in assign.cu)
int prep_blocks(int64_t n);
void launch_prep(const PrepArgs& a, cudaStream_t s);
size_t radix_sort_scratch_bytes(int64_t n);
// Stable sort of (keys, vals) by the low `bits` bits of keys.  Results in keys_out/vals_out.
void radix_sort(uint32_t* keys, uint32_t* vals, uint32_t* keys_out, uint32_t* vals_out, int64_t n,
                int bits, void* scratch, cudaStream_t s, int* launches);
size_t scan_scratch_bytes(int64_t n);
void exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, void* scratch, cudaStream_t s,
                        int* launches);
void launch_count_cells(const uint32_t* keys, int64_t n, uint32_t* counts, cudaStream_t s);
void launch_gather_particles(const uint32_t* perm, int64_t n, const float4* frac_in, const float* vals_in,
                             int nchan, float4* frac_out, float* vals_out, cudaStream_t s);
struct DepositArgs {
  const uint32_t* cell_start;  // N^3 + 1
  const uint32_t* keys;        // sorted home-node keys
  const float4* frac;          // sorted
  const float* vals;           // sorted [nchan][n]
  int64_t n;
  int N, mas, interlace, nchan;
  float* mesh0;                // [nchan][N^3]
  float* mesh1;                // [nchan][N^3] (interlaced) or nullptr
};
void launch_deposit(const DepositArgs& a, cudaStream_t s, int* launches);
// sum_c m(c)^3 over a real mesh, FP64 partials per block (deterministic), returns #blocks
int launch_sum_cubes(const float* mesh, int64_t ncell, double* partials, cudaStream_t s);

// ---- FFT (fft.cu) ---------------------------------------------------------------
// Forward r2c 3D FFT of `count` channel meshes held as [count][N][N][N] floats; if
// mesh1 != nullptr the interlaced pair is combined.  Output: deconvolved half spectra,
// complex [N][N][N/2] (nz < N/2, Nyquist planes zero), written over mesh0.
void forward_fft(float* mesh0, float* mesh1, int count, int N, int mas, const float2* tw,
                 const float* winv1d, cudaStream_t s, int* launches);

// 32nd roots of unity for the in-register DFTs (once per process)

// Inverse transforms from half spectra to real fields, pruned to |n_i| <= P.
enum SrcKind { SRC_PLAIN = 0, SRC_QSHOT = 1, SRC_SHELL = 2, SRC_KERNEL = 3, SRC_SHELL_SUM = 4 };
constexpr int INV_MAXE = 20;  // entries of one SRC_SHELL_SUM field
struct InvField {
  // SRC_PLAIN:  spec(k) = scale * A(k)
  // SRC_QSHOT:  spec(k) = scale * (A(k) conj(B(k)) - sbar * cw2(k))
  // SRC_SHELL:  spec(k) = mask_b(k)/Nm * (-i)^l * part(y_l^{m*}(k)) * (A(k) or 1)
  // SRC_KERNEL: spec(k) = conj(K(k)) * (A(k) or 1), K the forward FFT of a real separation
  //             kernel (three-point function); every mode but the Nyquist planes
  // SRC_SHELL_SUM: spec(k) = mask_b(k)/Nm * (-i)^l * sum_e ecoef[e] part_e(y_l^{m_e*}(k)) S_e(k),
  //             S_e = InvBatch::spec[espec[e]], m_e = em[e] >= 0, part_e = epart[e]: one real field
  //             of a contraction over (m, channel) done in k space
  int kind;
  const float2* A;
  const float2* B;
  const float2* K;
  float sbar;
  float scale;
  int l, m, part, unit;   // SRC_SHELL (l also SRC_SHELL_SUM)
  int ne;                 // SRC_SHELL_SUM entries
  float ecoef[INV_MAXE];
  signed char em[INV_MAXE], epart[INV_MAXE], espec[INV_MAXE];
  float* out;             // real field [N][N][N]
};
struct InvBatch {
  int N, P;               // prune extent: modes with |nx|,|ny|,nz <= P
  int nf;                 // number of fields (<= 32)
  InvField f[32];
  const float2* spec[16]; // spectra of the SRC_SHELL_SUM entries
  // shell geometry (SRC_SHELL)
  long long qlo, qhi;     // |n|^2 in [qlo, qhi)
  float inv_nmodes;
  const float* ynorm;
  const float* cw2_1d;    // QSHOT: per-axis tables (E, O, W) packed, see fft.cu
  int interlace;
  int* err;               // set (never cleared) when a bounded wait gives up
  int stall;              // test knob: the z pass starts no row-group copy (its waits run out)
  int zgroups;            // z pass: row groups per CTA (0: the default); any value gives the same fields
};
// row groups per CTA that inverse_fft's z pass would use for a requested value at mesh N
int inverse_zgroups(int N, int requested);
size_t inverse_scratch_bytes(int N, int P, int nf);

// Separation kernels of one r-bin (three-point function, Sec. 4.3): mesh c of `mesh`
// ([nc][N][N][N] floats, zeroed by the caller) gets part_c(y_{l_c}^{m_c *}(s_hat)) * inv_nr at
// the cell s mod N of every separation s of the list (packed (sx+512) | (sy+512) << 10 |
// (sz+512) << 20); y(0) = delta_{l0}.
struct RKernelArgs {
  int N, nc;
  int l[32], m[32], part[32];
  float inv_nr;
  const uint32_t* offs;
  int64_t n;
  const float* ynorm;
  float* mesh;
};
void launch_rshell_kernel(const RKernelArgs& a, cudaStream_t s);
void inverse_fft(const InvBatch& b, const float2* tw, void* scratch, cudaStream_t s, int* launches);

// ---- shell sums and pair reduction (measure.cu) -----------------------------------
void launch_axpby(float2* out, const float2* x, double a, const float2* y, double b, size_t n,
                  int zero_k0, cudaStream_t s);

// Z = (1/N_mode) sum_shell y_l^{m*}(k) [X(k) conj(N(k)) - Sbar C(k)/W^2(k)], with X = XR + i XI
// and N = NR + i NI combinations of the spectra of real channel meshes
struct ZsumArgs {
  const float2* XR;       // delta n spectrum of the distinct object (real-part channel)
  const float2* XI;       // imaginary-part channel or nullptr
  const float2* NR;       // N spectrum of the coincident pair (real-part channel)
  const float2* NI;       // imaginary-part channel or nullptr (M = 0)
  double sbar_re, sbar_im;
  int N, P;
  int nbins;
  const uint32_t* modes;  // half-spectrum shell modes, (sx+512) | (sy+512) << 10 | nz << 20
  const int64_t* mode_off;  // modes of bin b: [mode_off[b], mode_off[b+1])
  const float* cw2_1d;
  int interlace;
  int nlm;                // number of (l, m) pairs, m >= 0
  int lm[16][2];
  const float* ynorm;
  double* partials;       // [nbins][nblk][nlm][2]
  int nblk;
};
void launch_zsum(const ZsumArgs& a, cudaStream_t s);

// out[i * nf + c] = fields[c * Ng + cell of -s_i] for the packed separations s_i (as in
// RKernelArgs): real fields at the negated separations of the r-bins
void launch_gather_neg(const float* fields, int64_t Ng, int nf, const uint32_t* offs, int64_t n, int N, float* out,
                       cudaStream_t s);

struct PairRecipe { int comp, g; float coef; };
struct PairTermDesc {
  int xoff, xcnt, yoff, ycnt;  // recipe entries of the two sides
  int xdir, ydir;              // side is a bare component field (index), or -1
  int xslot, yslot;            // shared-memory slot of a side built per chunk, or -1
  int tr;                      // 1: computed as Y X^T (tensor-core kernels), read back transposed
  int grp, quad;               // tcgen05 kernel: M = 128 tile and its 32-row quarter
};
struct PairJob {
  const float* fields;    // component field (b, c) at fields + (b*ncomp + c) * Ng
  const float* gfields;   // g field i at gfields + i * Ng
  int64_t Ng;
  int nb, ncomp, ng;
  int nout;               // outputs (multipole x G-set)
  int out_term_off[33];   // terms of output o: [off[o], off[o+1])
  int nterm;
  int nslot;              // sides built per chunk
  int term_out[64];       // output of each term (before merging)
  PairTermDesc term[64];
  // after merging terms that differ only by a scalar: output o = sum over its entries
  // (term u, FP64 multiplier) of the sum over cells of term u
  int out_ent_off[33];
  int out_ent_term[128];
  double out_ent_mult[128];
  // built sides: side s = sum over its entries (c, h) of P_c(b, x) H_h(x), where
  // H_h(x) = sum over its entries (g, coef) of coef G_g(x) (g < 0: the constant coef)
  int nh;
  int h_off[129];         // entries of H row h: [h_off[h], h_off[h+1]) in h_ent
  PairRecipe h_ent[512];  // (comp unused, g, coef)
  int s_off[65];          // entries of side s: [s_off[s], s_off[s+1]) in s_ent
  int s_ent[512][2];      // (c, h)
  int nrec;
  PairRecipe rec[512];
};
// Result: out[o][b1][b2] = sum_x sum_{t in o} X_t(x;b1) Y_t(x;b2)   (FP64)
// ev0 / ev1 (optional) are recorded right before the contraction kernel and after the final
// reduction kernel: their interval is the device time of the two kernels alone
void pair_reduce(const PairJob& job, double* out_dev, void* scratch, size_t scratch_bytes,
                 cudaStream_t s, int* launches, int* kernel = nullptr, cudaEvent_t ev0 = nullptr,
                 cudaEvent_t ev1 = nullptr);
size_t pair_scratch_bytes(const PairJob& job);
// true when one launch of some contraction kernel covers the job (terms, tables, shared memory)
bool pair_fits(const PairJob& job);
// true when the pair kernel in use prefers one launch per G set (at most 8 terms a launch)
bool pair_split_gsets();

// ---- plain FP64 form (fp64.cu) -----------------------------------------------------
// One FP64 half spectrum [N][N][N/2+1] built from the FP32 half spectra [N][N][N/2]:
//   SRC_PLAIN  scale * A;   SRC_QSHOT  scale * (A conj(B) - sbar C/W^2);
//   SRC_SHELL  mask_b(k) inv_nmodes (-i)^l part(y_l^{m*}(k)) (A(k), or 1 if unit)
struct F64Spec {
  int kind;
  const float2* A;
  const float2* B;
  double scale, sbar;
  int l, m, part, unit;
  long long qlo, qhi;
  double inv_nmodes;
};
struct F64Tables {
  const double* ynorm;    // sqrt((l-m)!/(l+m)!) at [l * (BISP_LMAX + 1) + m]
  const double* cw2;      // per-axis E/W^2 (N values) then O/W^2 (N values)
  int interlace;
};
void f64_spectrum(const F64Spec& s, const F64Tables& t, int N, double2* out, cudaStream_t st);
struct F64Fft {
  long long handle = -1;  // cufftHandle of an N^3 Z2D plan (work area supplied by the caller)
  size_t work_bytes = 0;
};
F64Fft f64_fft_create(int N);
void f64_fft_c2r(const F64Fft& f, void* work, double2* in, double* out, cudaStream_t s);
void f64_fft_destroy(F64Fft& f);
// mesh sum of a b c over n doubles: nblk block partials, then out[d] = sum of row d of
// partial [nd][nblk] (both in a fixed order)
int f64_dot_blocks();
void f64_dot3(const double* a, const double* b, const double* c, int64_t n, double* partial, int nblk,
              cudaStream_t s);
void f64_dot_final(const double* partial, int nblk, int nd, double* out, cudaStream_t s);

}  // namespace bisp
