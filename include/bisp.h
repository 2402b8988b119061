/*
 * bisp.h - C ABI of the GB300 (sm_103a) estimator of the redshift-space bispectrum
 * multipoles B_{l1 l2 L}(k1, k2) in the tri-polar spherical-harmonic (TripoSH)
 * decomposition of Sugiyama, Saito, Beutler & Seo (arXiv:1803.02132).
 *
 * The library computes, on one GPU and with hand-written CUDA kernels only:
 *   - the mass assignment of weighted galaxies and randoms onto a mesh (Sec. 4.1,
 *     Eq. mean_n, Eq. dn, Eq. nlm; NGP/CIC/TSC, App. C) with optional interlacing;
 *   - the forward 3D FFT and the W_mass deconvolution (Sec. 4.2);
 *   - the y_l^{m*}(k)-filtered inverse FFTs per k shell and the y_L^{M*}(x)-weighted
 *     density field G_L^M (Eq. nlm_bi);
 *   - the mesh sum of F F G contracted with Wigner 3j symbols (Eq. bi_estimator_FFTs;
 *     global line of sight: Eq. simulation_estimator);
 *   - the four shot-noise terms (Eq. shotnoise, Eq. ShotNoise), the normalisation I
 *     (Eq. normalization; periodic box I = Np^3/V^2, Sec. 4.4);
 *   - the window bispectrum: the same estimator on the random catalogue alone (the
 *     bispectrum-space counterpart of Eq. Q);
 *   - the three-point-function multipoles and the three-point window multipoles Q
 *     (Sec. 4.3, Eq. reduced_xi_estimator; Sec. 6.1, Eq. Q), and a diagonal-only mode;
 *   - the plain FP64 form of the bispectrum estimator, as a speed and accuracy baseline.
 * On the host, for batches of measurements and the window-convolved model: the covariance
 * statistics of Sec. 5.5 and App. E, and the 9j coupling, integral constraint, Hankel
 * transforms and tree-level multipoles of Sec. 6.2 and App. F.
 *
 * Conventions shared by every call:
 *   - Every call returns a bisp_status.  Nothing throws across the ABI.  On failure
 *     bisp_last_error() returns a message for the calling thread (valid until the next
 *     failing call on that thread).
 *   - Positions are in box coordinates [0, box_len)^3, float32, interleaved x,y,z.
 *   - A plan owns all its device memory (meshes, spectra, fields) and a CUDA stream;
 *     the caller owns every pointer it passes, and the library only borrows it for the
 *     duration of the call.  Calls on one plan must not overlap (one thread at a time);
 *     different plans may be driven from different host threads at the same time.
 *   - Device pointers passed in are read on the plan's stream; the call returns after
 *     the work has completed (host outputs are written).
 *   - Output arrays are caller-owned host FP64 arrays.
 */
#ifndef BISP_H
#define BISP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bisp_plan bisp_plan; /* opaque; owns device memory and a stream */

typedef enum {
  BISP_OK = 0,
  BISP_EINVAL = 1,      /* invalid argument (message names it) */
  BISP_ENOMEM = 2,      /* device memory admission failed (message gives bytes needed) */
  BISP_ECUDA = 3,       /* a CUDA runtime call failed */
  BISP_ESTATE = 4,      /* call out of order (e.g. measure before the data catalogue) */
  BISP_ETIMEOUT = 5,    /* a bounded device wait expired */
  BISP_EUNSUPPORTED = 6 /* valid request outside what the library implements */
} bisp_status;

/* Line of sight: global (the z axis of the box, Sec. 4.4) or local (the direction from
 * the observer to each object, Sec. 2 and Sec. 4.1). */
typedef enum { BISP_LOS_GLOBAL_Z = 0, BISP_LOS_LOCAL = 1 } bisp_los;

/* Mass assignment scheme; the value is the exponent p of W_mass (Sec. 4.2). */
typedef enum { BISP_NGP = 1, BISP_CIC = 2, BISP_TSC = 3 } bisp_mas;

typedef enum { BISP_DATA = 0, BISP_RANDOMS = 1 } bisp_catalog;

/* Arithmetic of bisp_measure after the forward transform.  BISP_FP32: the fused path
 * (FP32 filtered fields, pruned FFTs, tensor-core mesh sums with FP64 accumulation).
 * BISP_FP64: the plain FP64 form of the same estimator (Eq. bi_estimator_FFTs), kept as a
 * speed and accuracy baseline: every filtered field is a full cuFFT Z2D transform of an
 * FP64 half spectrum, and every 3j term of every bin pair is its own FP64 mesh sum that
 * re-reads its three fields.  Both share mass assignment, the forward transform (FP32
 * spectra, upcast) and the shell averages of the shot-noise terms. */
typedef enum { BISP_FP32 = 0, BISP_FP64 = 1 } bisp_precision;

/* What bisp_measure estimates.  BISP_BISPECTRUM: B_{l1 l2 L}(k1, k2) (Eq. bi_estimator_FFTs).
 * BISP_THREEPT: the three-point-function multipoles zeta_{l1 l2 L}(r1, r2) (Sec. 4.3,
 * Eq. reduced_xi_estimator) and, as the window output, the three-point window multipoles
 * Q_{l1 l2 L}(r1, r2) (Sec. 6.1, Eq. Q).  For BISP_THREEPT the bins are sets of mesh
 * separations s (integer, |s_i| <= N/2 - 1) with k_edges[a] <= H |s| < k_edges[a+1] (H the
 * cell size, edges in Mpc/h, the first may be 0: a bin [0, e_1) with e_1 < H holds s = 0
 * only); F_l^m(x; r_a) averages y_l^{m*}(s_hat) delta n(x + s) over the bin, applied as a
 * k-space filter (the FFT of the separation kernel); the only shot-noise term is i = j != k,
 * on r_a = r_b; nmodes returns the number of separations per bin.  BISP_FP32 only. */
typedef enum { BISP_BISPECTRUM = 0, BISP_THREEPT = 1 } bisp_estimator;

typedef struct {
  int nmesh;               /* N, a power of two, 16..1024 */
  double box_len;          /* L [Mpc/h]; the mesh covers [0, L)^3 */
  const double* k_edges;   /* nbins+1 ascending edges [h/Mpc]; bin b = [e_b, e_{b+1}).
                              Modes on a Nyquist plane are in no bin. Copied. */
  int nbins;
  const int* ells;         /* 3*n_mult ints (l1, l2, L), each satisfying the selection
                              rules of Table 1 (l1 >= l2, L even, triangle rule,
                              l1+l2+L even), l1, l2, L <= 4. Copied. */
  int n_mult;
  int los;                 /* bisp_los */
  double observer[3];      /* BISP_LOS_LOCAL only: origin of the lines of sight */
  int mas;                 /* bisp_mas */
  int interlace;           /* 0/1: second mesh shifted by half a cell (reading of Sec. 4.2) */
  double fkp_P0;           /* > 0: FKP weight w/(1 + nbar P0) when nbar is given (Sec. 5.2) */
  size_t max_device_bytes; /* 0: free device memory minus a reserve; else the admission cap */
  int want_window;         /* 1: also the randoms-only window bispectrum (needs randoms) */
  int precision;           /* bisp_precision (0: BISP_FP32) */
  int estimator;           /* bisp_estimator (0: BISP_BISPECTRUM) */
  int diagonal_only;       /* 1: only the k1 = k2 (r1 = r2) outputs, the diagonal the paper's
                              signal-to-noise study rests on (Sec. 4.4, Sec. 5.6); every other
                              output is NaN.  When the shell fields of all bins do not fit,
                              each block of bins is then measured alone, with no block pairs. */
  int los_object;          /* object of the triplet whose line of sight x_hat carries the
                              y_L^{M*} weight (App. B): 0 or 3 = x3 (the main text's choice),
                              1 = x1 (the k1 object), 2 = x2 (the k2 object); the shot-noise terms
                              follow the object that carries the weight.  Local line of sight,
                              BISP_BISPECTRUM and BISP_FP32 only (otherwise BISP_EUNSUPPORTED); with
                              the global line of sight every choice gives the same result. */
} bisp_params;

/* Create a plan.  Validates params (BISP_EINVAL names the offending field), computes the
 * bin thresholds, the 3j tables and the per-multipole contraction recipes in FP64, and
 * reserves device memory for the meshes and fields (BISP_ENOMEM with the bytes needed).
 * stream: a cudaStream_t to run on, or NULL for a stream the plan creates and owns. */
bisp_status bisp_plan_create(bisp_plan** out, const bisp_params* p, void* stream);

/* Assign a catalogue (Sec. 4.1): weights w_i (NULL: 1) times the FKP weight when nbar
 * (expected number density at each object, NULL: none) is given and fkp_P0 > 0; the
 * local-LOS channels y_L^{M*}(x_hat) w and y_L^M(x_hat) w^2; deterministic sort-by-cell
 * scatter onto the mesh (no float atomics); forward FFT; interlacing; deconvolution.
 * xyz: 3*n floats; w, nbar: n floats or NULL; ptr_is_device: 1 if the three pointers
 * are device pointers, 0 if host pointers (copied in by the call).
 * Errors: BISP_EINVAL for n < 0, NULL xyz with n > 0, non-finite or out-of-box
 * positions (the message gives the count), non-positive total weight. Re-assigning a
 * catalogue replaces it. */
bisp_status bisp_assign(bisp_plan* plan, int which, const float* xyz, const float* w,
                        const float* nbar, int64_t n, int ptr_is_device);

/* Measure every multipole of the plan.  All outputs are host FP64 arrays of n_mult *
 * nbins * nbins values laid out [mult][b1][b2] (or NULL to skip):
 *   B            shot-noise-subtracted bispectrum multipoles B_{l1 l2 L}(k_b1, k_b2)
 *   shot         the subtracted shot noise (sum of the four terms of Eq. shotnoise)
 *   window       window bispectrum (randoms only), shot noise subtracted; needs
 *                want_window
 *   window_shot  the window's shot noise
 *   nmodes       nbins values: the number of Fourier modes in each shell
 * Needs the data catalogue (BISP_ESTATE otherwise) and, for the local line of sight or
 * the window, the random catalogue. */
bisp_status bisp_measure(bisp_plan* plan, double* B, double* shot, double* window,
                         double* window_shot, double* nmodes);

/* Output arrays of one plan for bisp_measure_batch: the same arrays, shapes and NULL rules as the
 * arguments of bisp_measure. */
typedef struct {
  double* B;
  double* shot;
  double* window;
  double* window_shot;
  double* nmodes;
} bisp_outputs;

/* Measure a batch of plans, e.g. many independent realisations on meshes of different sizes,
 * in one call: the result for plan i is what bisp_measure(plans[i], outs[i].B, ...) returns, bit
 * for bit.  Each plan must have its catalogues assigned, and a plan may appear once.  Up to 8 host
 * worker threads measure the plans concurrently, each plan on its own stream (plans share no
 * device buffers; the kernels' job tables are launch parameters, except the contraction's, which
 * is held under a process-wide lock until its launches complete), so the GPU overlaps the work of
 * several realisations; the call returns when all are done.  Plans created on one shared stream
 * are serialised by that stream.  Errors: BISP_EINVAL for nplans < 0, NULL arrays or a repeated
 * plan; otherwise the status of the failing plan with the lowest index, with that index in the
 * message (the other plans are still measured).  No counterpart in the paper beyond its use of
 * many mocks (Sec. 5.5). */
bisp_status bisp_measure_batch(bisp_plan* const* plans, const bisp_outputs* outs, int nplans);

/* Covariance of a batch of measurements (Sec. 5.5, Eq. Covariance): X holds n_mock data
 * vectors of n_bin values, [n_mock][n_bin] host FP64 (for example flattened bisp_measure
 * outputs of independent realisations).  Outputs (host, caller-owned, NULL to skip): mean
 * [n_bin]; cov [n_bin][n_bin] = 1/(n_mock - 1) sum_n (X_n - mean)^T (X_n - mean); corr
 * [n_bin][n_bin] = cov_ij / sqrt(cov_ii cov_jj) (NaN where a variance is 0).  Host only: no
 * device work.  Errors: BISP_EINVAL for NULL X, n_mock < 2 or n_bin < 1. */
bisp_status bisp_covariance(const double* X, int n_mock, int n_bin, double* mean, double* cov, double* corr);

/* The factors of App. E: hartlap = (n_mock - n_bin - 2)/(n_mock - 1), the factor on the inverse
 * covariance; percival_m = (1 + B (n_bin - n_par)) / (1 + A + B (n_par + 1)), the factor on
 * parameter variances for n_par parameters, with A = 2 / ((n_mock - n_bin - 1)(n_mock - n_bin -
 * 4)) and B = (n_mock - n_bin - 2) / ((n_mock - n_bin - 1)(n_mock - n_bin - 4)) (App. E prints
 * square roots in these denominators; without them M tends to 1 for infinitely many
 * realisations, as a factor for the noise of an estimated covariance must).  Either output may be
 * NULL.  Errors: BISP_EINVAL for n_mock < 2, n_bin < 1, n_par < 0, or a requested percival_m
 * with n_mock <= n_bin + 4. */
bisp_status bisp_covariance_factors(int n_mock, int n_bin, int n_par, double* hartlap, double* percival_m);

/* chi^2 = (x_obs - x_theory)^T C_Hartlap^{-1} (x_obs - x_theory) (App. E) for a covariance cov
 * [n_bin][n_bin] estimated from n_mock realisations (Cholesky solve in FP64, host only).
 * Errors: BISP_EINVAL for NULL pointers, n_bin < 1, n_mock < 2, or a covariance that is not
 * positive definite. */
bisp_status bisp_chi2(const double* cov, int n_bin, int n_mock, const double* x_obs, const double* x_theory,
                      double* chi2);

/* ---- window-convolved model (Sec. 6.2), host FP64, no device work ------------------- */

/* Wigner 9j symbol {j[0] j[1] j[2]; j[3] j[4] j[5]; j[6] j[7] j[8]} of integer arguments
 * (App. A, Eq. Wigner9j), as a sum over three 6j symbols (Racah's formula).  Errors:
 * BISP_EINVAL for NULL pointers or j outside [0, 32]. */
bisp_status bisp_wigner9j(const int* j, double* out);

/* Masked three-point multipoles <zeta_l>_model (Eq. zetaMask) with the integral constraint
 * zeta_bar (Eq. IC), on an (r1, r2) grid of nr radii r[i] with quadrature weights w[i]
 * (int dr r^2 f(r) ~ sum_i w_i r_i^2 f(r_i)).  Theory multipoles: n_t triples ells_t (l1, l2, L)
 * and zeta_t [n_t][nr][nr]; window multipoles: n_q triples ells_q and Q [n_q][nr][nr] (the
 * measured BISP_THREEPT window output); outputs: n_o triples ells_o and out [n_o][nr][nr],
 *   out_l = N_l sum_{l' in theory, l'' in window} {l''; l'; l} H_l H_{l1 l1' l1''} H_{l2 l2' l2''}
 *           H_{L L' L''} / (H_{l'} H_{l''}) Q_{l''} zeta_{l'}  -  Q_l zeta_bar,
 * H the 3j symbols with zero projections, N_l = (2 l1 + 1)(2 l2 + 1)(2L + 1).  ic = 1 computes
 * zeta_bar over the multipoles present in both sets (needs Q_000); ic = 0 takes zeta_bar = 0.
 * zeta_bar may be NULL.  Every l <= 8 and a triangle.  All arrays host, caller-owned.  Errors:
 * BISP_EINVAL for NULL pointers, empty sets, invalid multipoles, or ic without Q_000. */
bisp_status bisp_masked_zeta(const int* ells_t, int n_t, const double* zeta_t, const int* ells_q, int n_q,
                             const double* Q, const int* ells_o, int n_o, const double* r, const double* w, int nr,
                             int ic, double* out, double* zeta_bar);

/* Hankel transform to the bispectrum (Eq. masked_bispectrum, Eq. HankelTransform):
 *   B[a][b] = (-i)^{l1+l2} (4 pi)^2 sum_ij w_i r_i^2 w_j r_j^2 j_l1(k1_a r_i) j_l2(k2_b r_j) zeta[i][j]
 * on host arrays zeta [nr][nr] and B [nk1][nk2]; l1 + l2 even (otherwise the bispectrum is
 * imaginary: BISP_EUNSUPPORTED), l1, l2 <= 8.  Errors: BISP_EINVAL for NULL pointers or empty grids. */
bisp_status bisp_zeta_to_bk(int l1, int l2, const double* r, const double* w, int nr, const double* zeta,
                            const double* k1, int nk1, const double* k2, int nk2, double* B);

/* The inverse transform (Eq. HankelTransform):
 *   zeta[a][b] = i^{l1+l2} sum_ij wk_i k_i^2 wk_j k_j^2 / (2 pi^2)^2 j_l1(r1_a k_i) j_l2(r2_b k_j) B[i][j]
 * with B [nk][nk] on one k grid with weights wk (int dk g(k) ~ sum_i wk_i g(k_i)), zeta [nr1][nr2].
 * Same conditions and errors as bisp_zeta_to_bk. */
bisp_status bisp_bk_to_zeta(int l1, int l2, const double* k, const double* wk, int nk, const double* B,
                            const double* r1, int nr1, const double* r2, int nr2, double* zeta);

/* Tree-level bispectrum multipoles B_{l1 l2 L}(k1, k2) (App. F: the second-order kernels
 * Z1 = b1 + f mu^2 and Z2 = b1 F2 + b2/2 + f mu^2 G2 + (f mu k / 2)(mu1/k1 Z1(k2) + mu2/k2 Z1(k1)),
 * B = 2 Z2(k1, k2) Z1(k1) Z1(k2) P(k1) P(k2) + cyc.), projected on the TripoSH basis
 * (Eq. reduced_ones, Eq. TripoSH_J0) by Gauss-Legendre quadrature in mu1 and mu2 (n_mu nodes)
 * and 2 n_mu azimuths.  P(k) is a host table (n_tab >= 2 ascending k > 0, P > 0), interpolated in
 * log-log (a power law exactly) and held at its end values outside the table.  out
 * [n_mult][nk1][nk2] host FP64.  The paper's linear spectrum comes from CLASS, which is not here;
 * any table (a power law, for instance) serves.  Errors: BISP_EINVAL for NULL pointers, a bad
 * table, k <= 0, n_mu < 2 or multipoles outside l <= 8 / the triangle rule. */
bisp_status bisp_tree_multipoles(const double* k_tab, const double* p_tab, int n_tab, double b1, double b2, double f,
                                 const int* ells, int n_mult, const double* k1, int nk1, const double* k2, int nk2,
                                 int n_mu, double* out);

/* Free every resource of the plan (NULL is accepted). */
bisp_status bisp_plan_destroy(bisp_plan* plan);

/* Message of the calling thread's last failure ("" if none). */
const char* bisp_last_error(void);

/* Sizes and bookkeeping of a plan, for callers and tests. */
typedef struct {
  int nmesh, nbins, n_mult, n_dchan, n_nchan, n_fcomp;
  double alpha;            /* sum w_gal / sum w_ran, 0 before both are assigned */
  double norm_I;           /* normalisation I of Eq. normalization */
  int64_t n_data, n_randoms;
  size_t device_bytes;     /* device memory held by the plan */
  int kernel_launches;     /* kernels launched by the last bisp_assign + bisp_measure */
  double ms_assign_data, ms_assign_randoms, ms_measure; /* device time of the last calls */
  double ms_pair;          /* device time of the pair-reduction kernels in the last measure */
  double pair_bytes;       /* algorithmic bytes read by those pair reductions */
  int pair_launches;
  int pair_kernel;         /* kernel of the last pair reduction: 0 FP32 FMA (jobs outside the tensor-core layout),
                              1 mma.sync TF32 (default), 2 tcgen05 TF32 (BISP_PAIR_KERNEL=tcgen05
                              in the environment, for jobs it covers), 3 FP64 unfused mesh sums
                              (BISP_FP64 plans) */
  int zpass_groups;        /* row groups per CTA of the inverse transforms' z pass, chosen by timing
                              the candidates on the plan's largest shell batch at its first
                              measurement (every value gives the same fields); 0 before that.
                              BISP_ZGROUPS=n in the environment fixes it without timing. */
} bisp_plan_info;

bisp_status bisp_plan_query(const bisp_plan* plan, bisp_plan_info* info);

/* Stable ordering of particles by their home mesh node (Sec. 4.2 mass assignment; the
 * node is floor(x/H) for CIC and floor(x/H + 1/2) for NGP/TSC, with H = box_len/nmesh,
 * computed in FP64).  keys_out[i] = (hx*N + hy)*N + hz of particle order_out[i]; ties
 * keep input order.  xyz (3*n floats), keys_out and order_out (n uint32 each) are device
 * pointers; stream is a cudaStream_t or NULL.  Scratch is allocated by the call.
 * Errors: BISP_EINVAL for bad sizes, non-finite or out-of-box positions. */
bisp_status bisp_cell_order(int nmesh, double box_len, int mas, const float* xyz, int64_t n,
                            uint32_t* keys_out, uint32_t* order_out, void* stream);

/* Largest catalogue accepted by bisp_cell_order_noalloc. */
#define BISP_NOALLOC_MAX_PARTICLES (1 << 20)

/* bisp_cell_order without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory during the call -
 * code running under a framework or memory pool that forbids cudaMalloc/cudaFree inside a
 * step, allocators that must not be re-entered, or processes without spare device memory.
 * Same arguments, outputs and errors as bisp_cell_order.
 *   - Scratch lives in one statically sized device array in the library (about
 *     32 bytes per particle of BISP_NOALLOC_MAX_PARTICLES plus 4 MiB, i.e. 36 MiB); every
 *     GPU that loads the library holds it until the process exits.
 *   - n > BISP_NOALLOC_MAX_PARTICLES returns BISP_EINVAL and names the limit.
 *   - The first call on a device resolves the array's device address with that device
 *     current and keeps it for the life of the process.  After cudaDeviceReset the kept
 *     address is stale: do not call this entry point again in that process.
 *   - The call copies a small table from host memory, reads back an error counter and
 *     synchronises `stream` before it returns, so it cannot be recorded into a CUDA graph:
 *     do not call it while `stream` (or any stream of the device) is being captured.
 *   - All calls share the one array: calls whose GPU work overlaps (on different streams or
 *     host threads) race and corrupt each other's results.  Serialise them.
 *   - The call allocates nothing (no cudaMalloc, cudaFree or allocating library routine). */
bisp_status bisp_cell_order_noalloc(int nmesh, double box_len, int mas, const float* xyz, int64_t n,
                                    uint32_t* keys_out, uint32_t* order_out, void* stream);

/* Copy an internal array of the plan to host memory (tests):
 *   what = BISP_DBG_SPECTRUM: the deconvolved half spectrum of channel `index` of
 *          catalogue `which`, complex64 [N][N][N/2] (nz < N/2), 8*N*N*N/2 bytes;
 *   what = BISP_DBG_MESH: the real mesh of channel `index` (non-shifted) of catalogue
 *          `which` as assigned, float32 [N][N][N]; kept only if the plan was created
 *          with BISP_DEBUG_KEEP_MESH in the environment variable BISP_DEBUG.
 * bytes must equal the array size. */
enum { BISP_DBG_SPECTRUM = 0, BISP_DBG_MESH = 1 };
bisp_status bisp_debug_fetch(const bisp_plan* plan, int what, int which, int index,
                             void* host_out, size_t bytes);

/* Device bounds checks (no paper passage: a debugging aid).  The library built with
 * -DBISP_CHECKED (paper_1803_02132_gb300/build.py, checked=True: libbisp_checked.so) tests the
 * indexes of its main kernels' global and shared-memory accesses (deposit, particle gather,
 * shell sums, the three inverse passes, the contraction's tables) against the buffers they
 * address; a failed check skips the access and, if no failure is recorded yet, records
 * (site << 32) | (1 << 31) | (low 31 bits of the offending index) in a device word.  Nothing traps.
 * word (host, non-NULL) receives that word, 0 when every check passed since it was last
 * cleared; reset != 0 clears it afterwards.  The call synchronises the device.
 * Errors: BISP_EINVAL for NULL word; BISP_EUNSUPPORTED from the release build (word set to 0);
 * BISP_ECUDA if the copy fails. */
bisp_status bisp_check_word(uint64_t* word, int reset);

#ifdef __cplusplus
}
#endif
#endif /* BISP_H */
