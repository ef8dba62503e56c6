/*
 * librpa_gpu -- C ABI of a GB300 (sm_103a) implementation of the low-scaling
 * localized-RI (LRI) space-time RPA correlation energy path of
 * "LibRPA: A Software Package for Low-scaling First-principles Calculations of
 * Random Phase Approximation Electron Correlation Energy Based on Numerical Atomic
 * Orbitals" (arXiv:2407.19930).
 *
 * The calls follow the paper's API groups (Appendix B, "API functions of LibRPA":
 * environment setup, input parsing, computation), adapted to one GPU and no MPI:
 *
 *   paper                                              here
 *   initialize_librpa_environment                      librpa_gpu_create
 *   set_dimension + set_latvec_and_G + set_kgrids_*    librpa_gpu_set_structure
 *   set_ao_basis_aux                                   librpa_gpu_set_lri_coeffs
 *   set_wg_ekb_efermi + set_ao_basis_wfc               librpa_gpu_set_green
 *   set_aux_bare_coulomb_k_*                           librpa_gpu_set_coulomb
 *   (GreenX grids)                                     librpa_gpu_set_grid / librpa_gpu_build_grid
 *   get_rpa_correlation_energy                         librpa_gpu_chi0 + librpa_gpu_ec
 *   finalize_librpa_environment                        librpa_gpu_destroy
 *
 * Conventions used by every call:
 *  - Energies in Hartree, lengths in bohr.  All floating-point arguments are FP64.
 *  - Matrices are dense, row-major, C order; complex data is passed as separate
 *    real and imaginary arrays of the same shape.
 *  - The k-mesh is Gamma-centred: point (i1,i2,i3) has fractional coordinates
 *    (i1/nk1, i2/nk2, i3/nk3) and flat index (i1*nk2 + i2)*nk3 + i3.  The same flat
 *    order enumerates the Born-von Karman (BvK) cells R and the q-mesh.
 *  - Bloch sums carry exp(+i k.R): H(k) = sum_R e^{ik.R} H(R), so the real-space
 *    Green's function carries exp(-i k.R) (Sec. 2, Eq. green_mat) and
 *    chi0(q) = sum_R e^{iq.R} chi0(R) (Sec. 2, R -> q transform).
 *  - NAOs are ordered atom by atom (all NAOs of atom 0, then atom 1, ...); ABFs
 *    likewise.  The NAO basis is orthonormal (S = I) and nbands = total NAOs.
 *  - Host buffers are owned by the caller.  Every call that takes host input copies
 *    it (to host staging or to the device) before returning; the caller may reuse
 *    or free its buffers afterwards.  Output buffers are caller-allocated.
 *  - Every call returns LIBRPA_OK (0) or a negative LIBRPA_E_* code and never exits
 *    or throws; librpa_gpu_last_error() gives a one-line description.
 *  - A handle is not thread-safe; use one handle per host thread.  All device work
 *    of a handle is ordered on the handle's stream.
 */
#ifndef LIBRPA_GPU_H
#define LIBRPA_GPU_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define LIBRPA_OK 0
#define LIBRPA_E_ARG (-1)     /* an argument is out of range, NULL or inconsistent */
#define LIBRPA_E_STATE (-2)   /* call order violated or a required input is missing */
#define LIBRPA_E_NOMEM (-3)   /* device memory beyond the handle's HBM budget, or allocation failed */
#define LIBRPA_E_CUDA (-4)    /* a CUDA runtime error (message in last_error) */
#define LIBRPA_E_NOT_PD (-5)  /* a Cholesky pivot <= 0: V(q) or 1 - V^1/2 chi0 V^1/2 not positive definite */
#define LIBRPA_E_TIMEOUT (-6) /* a bounded device wait ran out */
#define LIBRPA_E_NUMERIC (-7) /* a non-finite or inconsistent intermediate (e.g. complex G for real input) */

/* ---------------------------------------------------------------- precision modes
 * The dense GEMMs of the chi0 contraction (Algorithm 1) and of the ln det stage can run on the
 * BF16 tensor cores with every FP64 operand row split into S exact BF16 digit planes
 * (row value = 2^E sum_s d_s 2^{-7-8(s-1)}, |d_s| <= 128), digit products accumulated exactly
 * and summed in FP64: S = 5 keeps 39 bits per operand (FP64-accurate to ~1e-12 relative),
 * S = 3 about 23 bits.  The plain forms round every element once, to BF16 (8 significant
 * bits) or to TF32 (11 bits, on the TF32 tensor cores), and accumulate in FP32; the 3xTF32
 * split writes x = hi + lo with hi = tf32(x), lo = tf32(x - hi) and sums hi hi + hi lo + lo hi
 * in FP32 (about 21 bits).  In every mode other than LIBRPA_FP64 the O assembly of the chi0
 * contraction also runs on digit planes (5 for LIBRPA_FP64_TC, 3 otherwise), the ln det GEMMs
 * (including the Cholesky panel products and trailing updates) and the G(tau) products
 * C diag(w) C^H on 5 planes.  LIBRPA_SPLIT_FAST alone leaves that rule: its ln det GEMMs use 4
 * planes (~31 bits) and its tau -> omega and R -> q transforms compute in FP32 (the transform
 * weights and phases rounded to FP32), for an E_c still within 0.1 meV/atom.  So LIBRPA_FP64_TC is a ~39-bit mode, not FP64: its results match
 * the FP64 path to chi0(R, tau) 1e-10 normwise and E_c 1e-8 Ha, not bit for bit.  The
 * exponentials of G(tau), the transform weights, the Cholesky factorisations' diagonal blocks
 * and the E_c sum always stay FP64. */
#define LIBRPA_FP64 0     /* every step in FP64 on the FP64 pipes (DMMA / DFMA) */
#define LIBRPA_FP64_TC 1  /* chi0, G and ln det GEMMs with 5 digit planes (~39 bits) on the tensor cores */
#define LIBRPA_SPLIT 2    /* chi0 GEMMs with 3 digit planes (mixed), ln det GEMMs with 5 */
#define LIBRPA_BF16 3     /* chi0 GEMMs in plain BF16 (FP32 accumulation), ln det GEMMs with 5 */
#define LIBRPA_TF32 4     /* chi0 GEMMs in plain TF32 (FP32 accumulation), ln det GEMMs with 5 */
#define LIBRPA_TF32X3 5   /* chi0 GEMMs as 3xTF32 split products (FP32 accumulation), ln det with 5 */
#define LIBRPA_SPLIT_FAST 6 /* as LIBRPA_SPLIT, ln det GEMMs with 4 planes, transforms in FP32 */

/* Grids the library builds (opts.grid_kind) */
#define LIBRPA_GRID_MINIMAX 0         /* minimax tau / omega grids (librpa_gpu_build_grid_minimax) */
#define LIBRPA_GRID_GAUSS_LEGENDRE 1  /* mapped Gauss-Legendre rule (librpa_gpu_build_grid) */

typedef struct librpa_gpu *librpa_gpu_t;

/* Device allocator hooks.  alloc returns a device pointer aligned to >= 256 bytes,
 * or NULL on failure; free releases it.  Both are called on the host thread that
 * drives the handle.  NULL hooks select cudaMalloc / cudaFree. */
typedef void *(*librpa_gpu_alloc_fn)(size_t bytes, void *ctx);
typedef void (*librpa_gpu_free_fn)(void *ptr, void *ctx);

typedef struct {
  int device;                    /* CUDA device ordinal */
  void *stream;                  /* cudaStream_t to run on; NULL = a stream owned by the handle */
  librpa_gpu_alloc_fn dev_alloc; /* NULL = cudaMalloc */
  librpa_gpu_free_fn dev_free;   /* NULL = cudaFree */
  void *alloc_ctx;               /* passed to dev_alloc / dev_free */
  int n_tau;                     /* grid size (tau = omega points) when the library builds the grid */
  int precision;                 /* LIBRPA_FP64, _FP64_TC, _SPLIT, _BF16, _TF32, _TF32X3 or _SPLIT_FAST */
  size_t hbm_budget;             /* bytes the handle may allocate; 0 = no limit */
  int check_level;               /* 0 = none; 1 = check G is real and the pivots finite */
  int chi0_slices;               /* 0 = from precision; 1..5 = digit planes of the chi0 GEMMs */
  int ec_slices;                 /* 0 = from precision; 1..5 = digit planes of the ln det GEMMs */
  int test_stall_gemms;          /* testing only (0 = off): in the handle's first test_stall_gemms
                                    tensor-core GEMM launches the MMA issuer of every CTA waits
                                    (100 us) on a barrier that nothing arrives at, so the bounded-wait
                                    failure path runs: the call returns LIBRPA_E_TIMEOUT, later
                                    calls of the handle run normally */
  int grid_kind;                 /* LIBRPA_GRID_MINIMAX (default) or LIBRPA_GRID_GAUSS_LEGENDRE: the grid
                                    librpa_gpu_chi0 builds when none was set */
} librpa_gpu_opts;

/* Per-stage device times (ms, CUDA events on the handle's stream) and work counts of
 * the most recent librpa_gpu_chi0 / librpa_gpu_ec call. */
typedef struct {
  double ms_green;         /* K1: G^occ / G^vir (R, tau) */
  double ms_chi0;          /* K2: chi0(R, tau) contraction (Algorithm 1) */
  double ms_freq;          /* K3 + K4: tau -> i omega and R -> q */
  double ms_ec;            /* K5 + K6: Cholesky, ln det, E_c */
  double flop_chi0;        /* algorithmic FP64 flops of K2 (no padding), see the design notes */
  double flop_ec;          /* algorithmic FP64 flops of K5 */
  double ms_gemm_chi0;     /* device time of the FP64 MMA GEMM launches of K2 (sum of per-launch events) */
  double flop_gemm_chi0;   /* algorithmic flops of those launches (2 M N K, no padding) */
  long long n_gemm_chi0;   /* number of those launches */
  double ms_gemm_ec;       /* device time of the complex GEMM launches of K5 */
  double flop_gemm_ec;     /* algorithmic flops of those launches (8 per complex MAC on the triangle) */
  long long n_gemm_ec;     /* number of those launches */
  long long launches;      /* kernels launched by the call */
  size_t bytes_device;     /* device bytes held by the handle */
  double flop_exec_gemm_chi0; /* tensor-core MMA flops issued by the timed chi0 GEMMs (digit-plane
                                 products, tile padding and all); 0 in the FP64 mode */
  double flop_exec_gemm_ec;   /* the same for the timed ln det GEMMs */
  size_t bytes_device_peak;   /* largest device footprint of the handle so far */
  long long n_points_chi0;    /* (R, tau) points contracted, summed over spin channels */
  long long n_points_skipped; /* points left out because screening made their chi0 exactly zero */
  long long n_blocks_kept;    /* atom-pair blocks of G kept by screening (all of them when off) */
  long long n_blocks_total;   /* atom-pair blocks of G: nspins * 2 * ntau * nR * natoms^2 */
} librpa_gpu_stats;

/* Fill *o with defaults: device 0, own stream, cudaMalloc, n_tau = 16, FP64,
 * no budget, check_level 1, no test stalls, minimax grids. */
void librpa_gpu_default_opts(librpa_gpu_opts *o);

/* Environment setup (paper: initialize_librpa_environment).  Creates a handle
 * bound to o->device.  *h is set to NULL on failure.
 * Errors: E_ARG (h or o NULL, bad device or n_tau < 1 or > 64 (> 20 with minimax grids),
 *         unknown precision or grid kind, test_stall_gemms < 0), E_CUDA. */
int librpa_gpu_create(librpa_gpu_t *h, const librpa_gpu_opts *o);

/* Structure and k-mesh (paper: set_dimension, set_latvec_and_G, set_kgrids_kvec_tot).
 *   lat[9]   lattice vectors as rows a1, a2, a3 (bohr);
 *   pos      [natoms][3] Cartesian positions (bohr);
 *   n_ao     [natoms] NAOs per atom (1..64); n_aux [natoms] ABFs per atom (1..256);
 *   nk1..nk3 Gamma-centred k-mesh (each >= 1); nspins = 1 (one channel standing for both
 *   spins, spin factor s = 2) or 2 (two channels, s = 1 each, chi0 = sum over channels);
 *   r_cut    LRI cutoff (bohr): set_lri_coeffs rejects blocks whose atoms are farther apart.
 * Resets every other input of the handle.
 * Errors: E_ARG. */
int librpa_gpu_set_structure(librpa_gpu_t h, int natoms, const double lat[9], const double *pos,
                             const int *n_ao, const int *n_aux, int nk1, int nk2, int nk3,
                             int nspins, double r_cut);

/* LRI expansion coefficients (paper: set_ao_basis_aux; Sec. 2, Eq. LRI).
 *   C [n_aux(I)][n_ao(I)][n_ao(K)] row-major = C^{mu(0)}_{i(0), k(R)}: mu and i on atom I
 *   in the home cell, k on atom K in cell R.  R is a true lattice vector (not folded
 *   into the BvK cell).  The neighbour set N[I] of Algorithm 1 is the set of (K, R)
 *   given here.  Setting the same (I, K, R) again replaces the block.
 * Errors: E_STATE (no structure), E_ARG (indices, |tau_K + R - tau_I| > r_cut, C NULL). */
int librpa_gpu_set_lri_coeffs(librpa_gpu_t h, int I, int K, const int R[3], const double *C);

/* KS eigen-data of one k point of spin channel ispin (0 .. nspins-1) (paper:
 * set_wg_ekb_efermi + set_ao_basis_wfc; Sec. 2, Eq. green_mat).
 *   eig [nbands] (Ha), occ [nbands] occupation per spin-orbital in [0, 1];
 *   wfc_re, wfc_im [nbands][n_ao_total]: wfc[n][i] = c_{i,n}(k);
 *   efermi: the chemical potential mu (Ha), the same for every k point and channel.
 * nbands must equal the total number of NAOs.  The path assumes time-reversal
 * symmetry (real H(R)), which makes G(R, tau) real; with check_level >= 1 librpa_gpu_chi0
 * returns E_NUMERIC if G has an imaginary part above 1e-10 relative.
 * Errors: E_STATE (no structure), E_ARG. */
int librpa_gpu_set_green(librpa_gpu_t h, int ispin, int ik, int nbands, const double *eig,
                         const double *occ, const double *wfc_re, const double *wfc_im,
                         double efermi);

/* Coulomb matrix of one q point in the ABF basis (paper: set_aux_bare_coulomb_k_*;
 * Sec. 2, Eq. Coulomb_matr_kspace): V_re, V_im [N_aux][N_aux], Hermitian positive
 * definite.  Copied to the device during the call.
 * Errors: E_STATE (no structure), E_ARG, E_NOMEM, E_CUDA. */
int librpa_gpu_set_coulomb(librpa_gpu_t h, int iq, const double *V_re, const double *V_im);

/* Optional grid override (Sec. 2, cosine transform):
 *   tau [ntau] (1/Ha), omega [nomega] (Ha), w_omega [nomega] quadrature weights of
 *   int_0^inf d omega, gamma [nomega][ntau] = the real transform matrix Gamma_kj with
 *   chi0(R, i omega_k) = sum_j Gamma_kj chi0(R, tau_j)  (the paper's
 *   -i gamma_jk cos(omega_k tau_j) with the -i factors of G taken out).
 * ntau == nomega required (1..64).  Without this call librpa_gpu_chi0 builds the grid
 * from the KS spectrum's transition range [Delta_min, Delta_max] with opts.n_tau points:
 * librpa_gpu_build_grid_minimax (opts.grid_kind = LIBRPA_GRID_MINIMAX, the default) or
 * librpa_gpu_build_grid (LIBRPA_GRID_GAUSS_LEGENDRE).
 * Errors: E_STATE (no structure), E_ARG. */
int librpa_gpu_set_grid(librpa_gpu_t h, int ntau, const double *tau, int nomega,
                        const double *omega, const double *w_omega, const double *gamma);

/* Weights w_q of the q sum of E_c (Sec. 2, E_c equation, whose 1/N_q is the uniform case;
 * Appendix B passes irreducible k points with weights, set_ibz2bz_index_and_weight).
 *   w [nq], one weight per q of the full Gamma-centred mesh (flat order), finite and >= 0,
 *   at least one > 0; w = NULL restores 1/N_q.  The caller maps its irreducible set onto the
 *   mesh: a representative carries its star's weight, the other members 0.  librpa_gpu_ec then
 *   returns E_c = (1/2 pi) sum_q w_q sum_k W_k [...] and ec_q[q] = w_q's term; q of zero weight
 *   are not computed (when V(-q) = conj V(q), a q and -q share one computation).  The weights
 *   are not normalised.  set_structure resets them.
 * Errors: E_STATE (no structure), E_ARG. */
int librpa_gpu_set_q_weights(librpa_gpu_t h, const double *w);

/* Green's-function block screening (Sec. 5: production runs screen G with a threshold of
 * 1e-3; Sec. 2: the decay of G limits the range of R).  The paper gives no formula; the rule
 * here: each atom-pair NAO block G^occ_{IJ}(R, tau_j) and G^vir_{IJ}(R, tau_j) is set to zero
 * when its largest |element| is below `threshold` (absolute, FP64 comparison on the device),
 * and kept unchanged otherwise.  Algorithm 1 then runs on the screened G.  Every term of chi0
 * is a product of a G^occ and a G^vir factor, so chi0(R, tau) is exactly zero at points where
 * every block one of the two Green's functions contributes was dropped; those points are not
 * contracted (stats.n_points_skipped), and N- or X-step operands without a kept block are not
 * multiplied on the FP64 route.  The result is that of the full contraction on the screened
 * G.  threshold = 0 (the default) turns screening off.  The setting belongs to the handle
 * (set_structure keeps it) and takes effect at the next
 * librpa_gpu_chi0; librpa_gpu_get_green then returns the screened G.
 * Errors: E_ARG (h NULL, threshold negative or not finite). */
int librpa_gpu_set_screening(librpa_gpu_t h, double threshold);

/* Stateless grid construction (host; Sec. 2: non-uniform tau/omega grids and gamma
 * from an L2 minimisation).  For n points and transition energies in [dmin, dmax]:
 *   omega_k, w_omega: n-point Gauss-Legendre rule mapped to (0, inf) by
 *     omega = w0 (1 + t) / (1 - t), w0 = sqrt(dmin dmax);
 *   tau_j: the same rule mapped with 1 / w0;
 *   gamma[k][j]: least-squares fit, in relative error over 1000 log-spaced D in
 *     [dmin, dmax], of 2D / (D^2 + omega_k^2) by sum_j gamma[k][j] exp(-D tau_j),
 *     by SVD with singular values below 1e-12 s_max dropped.
 * Outputs are caller-allocated: tau[n], omega[n], w_omega[n], gamma[n][n].
 * Errors: E_ARG (n < 1 or > 64, dmin <= 0, dmax < dmin, NULL outputs). */
int librpa_gpu_build_grid(int n, double dmin, double dmax, double *tau, double *omega,
                          double *w_omega, double *gamma);

/* Minimax grids (host; Sec. 2: the paper's non-uniform tau/omega grids, which it takes from
 * GreenX; built here from their defining property).  In units x = D / dmin on [1, R_b]:
 *   tau_j dmin, a_j: the n-term exponential sum closest to 1/x in the maximum norm,
 *     min max |1/x - sum_j a_j exp(-tau_j dmin x)|;
 *   omega_k / dmin, w_omega_k / dmin: the n-term sum closest to 1/x in the maximum norm among
 *     (1/pi) sum_k w_omega_k 4x^2 / (x^2 + omega_k^2)^2 (squared Lorentzians; w_omega are
 *     weights of int_0^inf d omega);
 * each found by the Remez exchange in double-double arithmetic until its error curve
 * equioscillates (2n + 1 extrema level to 1e-13).  R_b = 2^{ceil(8 log2 R_eff) / 8},
 * R_eff = max(dmax / dmin, exp(n pi^2 / ln 1e9) / 8): narrower ranges, where n terms would fit
 * below ~1e-9, are degenerate, and the 1/8-octave steps let grids be cached per (n, R_b).  The
 * grid covers [dmin, R_b dmin], which contains [dmin, dmax].  gamma[k][j]: the least-squares fit
 * of librpa_gpu_build_grid on [dmin, R_b dmin].  The first call for an (n, R_b) takes a few
 * tenths of a second of host time; later ones are served from a cache (thread-safe).
 * Outputs as in librpa_gpu_build_grid, ascending tau and omega; info (NULL allowed) [3]:
 * R_b, and the largest errors of the two fits in units of 1/dmin.
 * Errors: E_ARG (n < 1 or > 20, dmin <= 0, dmax < dmin or not finite, NULL outputs),
 *         E_NUMERIC (the exchange did not level the error curve). */
int librpa_gpu_build_grid_minimax(int n, double dmin, double dmax, double *tau, double *omega,
                                  double *w_omega, double *gamma, double *info);

/* Grid in use by the handle (after set_grid or after librpa_gpu_chi0 built it).
 * Outputs as in librpa_gpu_build_grid; *n receives the grid size.
 * Errors: E_STATE (no grid yet), E_ARG. */
int librpa_gpu_get_grid(librpa_gpu_t h, int *n, double *tau, double *omega, double *w_omega,
                        double *gamma);

/* Response function (Sec. 2: Eq. green_mat, Algorithm 1, cosine and Fourier transforms):
 *   G^occ, G^vir(R, tau_j)  ->  chi0_{mu nu}(R, tau_j)  ->  chi0(R, i omega_k)  ->  chi0(q, i omega_k).
 * Requires set_structure, set_green for every k and set_lri_coeffs for at least one
 * block per atom.  out_re / out_im may be NULL; otherwise each receives
 * [nq][nomega][N_aux][N_aux] (N_aux^2 * nq * nomega doubles).  The device copies of
 * G, chi0(R, tau) and chi0(q, i omega) stay on the device for librpa_gpu_ec and the
 * librpa_gpu_get_* calls until the next librpa_gpu_chi0 or set_structure.
 * Errors: E_STATE, E_NOMEM, E_CUDA, E_NUMERIC. */
int librpa_gpu_chi0(librpa_gpu_t h, double *out_re, double *out_im);

/* RPA correlation energy (Sec. 2, Eq. for E_c with Pi = chi0 V and Tr ln = ln det):
 *   E_c = (1/2 pi) sum_q w_q sum_k W_k [ln det(1 - Pi(q, i omega_k)) + Tr Pi(q, i omega_k)]
 * with w_q = 1/N_q (or librpa_gpu_set_q_weights).  ln det(1 - chi0 V) is computed as ln det(I - L^H chi0 L) with the
 * Cholesky factor V = L L^H and a blocked Cholesky of I - L^H chi0 L (FP64).
 *   ec    -> E_c in Ha per cell;
 *   ec_q  -> [nq] per-q contributions (nullable);  ec_w -> [nomega] per-frequency (nullable).
 * Requires librpa_gpu_chi0 and set_coulomb for every q.
 * Errors: E_STATE, E_NOT_PD, E_NOMEM, E_CUDA. */
int librpa_gpu_ec(librpa_gpu_t h, double *ec, double *ec_q, double *ec_w);

/* No-allocation variant of the ln det stage, for callers that cannot call cudaMalloc:
 * host codes that give all of the GPU's memory to their own pool at start-up (a further
 * cudaMalloc fails or fragments that pool), and callers whose loop must not stall other
 * streams (cudaMalloc and cudaFree may synchronise the device).  The paper has no
 * counterpart; it computes the same integrand as librpa_gpu_ec, without a handle.
 *
 *   out[k] = ln det(1 - chi_k V) + Re Tr(chi_k V),  k = 0 .. nomega-1,
 * via V = L L^H and the Cholesky factorisation of I - L^H chi_k L, in FP64.
 *   naux    matrix order, 1 .. LIBRPA_NOALLOC_MAX_NAUX (larger: E_ARG, nothing launched);
 *   V       device, [naux][naux] complex interleaved (re, im), row-major, Hermitian positive
 *           definite (lower triangle read), 16-byte aligned;
 *   chi     device, [nomega][naux][naux] complex interleaved, 16-byte aligned;
 *   out     device, [nomega] doubles; NaN where V or I - L^H chi_k L is not positive definite;
 *   stream  cudaStream_t (NULL: the legacy default stream) of the current device, which
 *           must hold V, chi and out;
 *   msg     optional buffer of msg_len bytes for a one-line error description.
 * The caller owns every buffer; the library calls no cudaMalloc, cudaFree or allocating
 * routine.  The work is enqueued on `stream` and the call returns without waiting: out is
 * valid once the stream is synchronised.  Scratch is one static device array of
 * LIBRPA_NOALLOC_SCRATCH_BYTES, shared by all calls and keeping the last call's contents
 * (each call writes every scratch value before reading it): calls that overlap on the GPU
 * race, so order them on one stream or with events.
 * Set-up: the first call made with a given device current looks up the array's device
 * address, once per device.  With lazy module loading (the CUDA default) the device also
 * creates the array at that moment, taking its 16 MiB of device memory, which it holds until
 * the process exits (with CUDA_MODULE_LOADING=EAGER every GPU that loads the library holds it
 * from the start).  So make the first call at start-up, before the caller's own memory pool
 * claims the device and before any stream capture: a call with nomega = 0 does only this
 * set-up (V, chi and out are then not used and may be NULL).
 * Errors: E_ARG (sizes, NULL or misaligned pointers), E_NOMEM (the device had no memory left
 * to create the array at set-up), E_CUDA. */
#define LIBRPA_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
#define LIBRPA_NOALLOC_MAX_NAUX 591
int librpa_gpu_ec_noalloc(int naux, int nomega, const double *V, const double *chi, double *out,
                          void *stream, char *msg, size_t msg_len);

/* Inspection of intermediates kept on the device (host copies of one slice):
 *   get_green:      go, gv  [n_ao_total][n_ao_total] at (itau, iR), spin channel 0;
 *   get_chi0_tau:   out     [N_aux][N_aux] = chi0(R, tau) at (itau, iR);
 *   get_chi0_freq:  re, im  [N_aux][N_aux] = chi0(q, i omega) at (iq, iomega).
 * Errors: E_STATE (not computed yet), E_ARG, E_CUDA. */
int librpa_gpu_get_green(librpa_gpu_t h, int itau, int iR, double *go, double *gv);
int librpa_gpu_get_chi0_tau(librpa_gpu_t h, int itau, int iR, double *out);
int librpa_gpu_get_chi0_freq(librpa_gpu_t h, int iq, int iomega, double *re, double *im);

/* Device-pointer variants (for data already on the GPU, e.g. torch tensors): the same as
 * set_green / set_coulomb / get_chi0_freq, with the complex matrices as device arrays of
 * interleaved (re, im) pairs, 16-byte aligned, on the handle's device:
 *   set_green_dev:     wfc [nbands][n_ao_total] complex (eig and occ stay host arrays: they set
 *                      the grid range);
 *   set_coulomb_dev:   V [N_aux][N_aux] complex;
 *   get_chi0_freq_dev: out [N_aux][N_aux] complex = chi0(q, i omega) at (iq, iomega).
 * The copies are enqueued on the handle's stream and the calls return without waiting: a
 * device input must stay valid, and a device output must not be read, until that stream has
 * reached the copy (work the caller enqueues on the same stream is ordered after it).  Not
 * accepted on request handles of the serving loop (E_STATE).  Errors: as the host versions. */
int librpa_gpu_set_green_dev(librpa_gpu_t h, int ispin, int ik, int nbands, const double *eig, const double *occ,
                             const double *wfc, double efermi);
int librpa_gpu_set_coulomb_dev(librpa_gpu_t h, int iq, const double *V);
int librpa_gpu_get_chi0_freq_dev(librpa_gpu_t h, int iq, int iomega, double *out);

/* Stage timings and counters of the last chi0 / ec calls. Errors: E_ARG. */
int librpa_gpu_get_stats(librpa_gpu_t h, librpa_gpu_stats *s);

/* ---------------------------------------------------------------- batched energies
 * Many independent structures in one pass (not in the paper, which computes one system
 * per call).  Every handle must be filled (set_* calls) before librpa_gpu_batch_run.
 * The FP64-mode, single-channel handles run on the first such handle's stream, and their
 * chi0 contraction runs in rounds: round r takes the r-th batch of (R, tau) points of every
 * one of them, and runs its GEMMs as single grouped launches over all those tiles, which
 * have uneven shapes.  The GEMM tile shape is picked by timing the variants on the first
 * run; from the second run on, that launch sequence is replayed from a CUDA graph.  The
 * single-channel tensor-core handles without screening are grouped by digit-plane count; a
 * group's chi0 contraction runs in rounds whose N-step, X-step and final GEMMs are each one
 * launch over all the group's tiles.  Those groups and the other handles (nspins = 2,
 * screening) run at the same time on up to four library-owned streams (one host thread each).  While a batch exists, run its
 * handles only through the batch.  After changing a handle's LRI blocks or structure, the
 * next run re-plans and captures again.  Destroy the batch before its handles. */
typedef struct librpa_gpu_batch *librpa_gpu_batch_t;

typedef struct {
  int n, n_merged;         /* handles; handles whose chi0 ran in the merged launches */
  int graph;               /* 1 if the last run replayed the captured graph */
  int var_nx, var_fin;     /* FP64 GEMM tile variants chosen: 0 = 64x64, 1 = 32x64, 2 = 64x32,
                              3 = 32x32, 4 = 128x64 (M x N); -1 = none */
  int failed_index;        /* handle of the last error (its last_error has the message), or -1 */
  double ms_green, ms_chi0, ms_freq, ms_ec;   /* device time of the merged handles' stages */
  double ms_total;         /* wall time of the whole last run */
  long long launches;      /* kernel launches of the last run (graph nodes included) */
  int n_merged_tc;         /* tensor-core handles whose chi0 GEMMs ran merged with others of their
                              digit-plane count */
} librpa_gpu_batch_stats;

/* Group n distinct handles of one device.  Errors: E_ARG, E_NOMEM. */
int librpa_gpu_batch_create(librpa_gpu_batch_t *b, librpa_gpu_t *hs, int n);

/* E_c of every handle into ec[n] (Ha per cell).  Errors: those of librpa_gpu_chi0 and
 * librpa_gpu_ec, for the handle in stats.failed_index. */
int librpa_gpu_batch_run(librpa_gpu_batch_t b, double *ec);

int librpa_gpu_batch_get_stats(librpa_gpu_batch_t b, librpa_gpu_batch_stats *st);

/* Free the batch's graph and descriptor buffers (not its handles).  NULL is ignored. */
void librpa_gpu_batch_destroy(librpa_gpu_batch_t b);

/* ---------------------------------------------------------------- serving loop
 * Continuous batching of RPA energy requests on one GPU (not in the paper, whose
 * library computes one system per call; each request runs the same path as
 * librpa_gpu_chi0 + librpa_gpu_ec).  A request is a handle made by
 * librpa_gpu_server_request and filled with the usual set_* calls; its inputs stay on
 * the host until the server admits it.  The server admits queued requests in arrival
 * order, letting a later request go first when the earlier one does not fit yet (not
 * after the earlier one has waited 2 s).  A request is admitted when one of `slots`
 * workers is free and its device-memory estimate (librpa_gpu_estimate_bytes) fits in
 * what is left of the server's HBM budget.  Each worker runs its request on its own
 * stream, from a stream-ordered memory pool, so admitted requests overlap on the device.
 * Once the request is complete, the worker releases its device memory.  A request that
 * fails with E_NOMEM (the device ran out although the estimates fit the budget: memory
 * held outside the server, or pool fragmentation) is queued again at the head and runs
 * once more, alone. */
typedef struct librpa_gpu_server *librpa_gpu_server_t;

typedef struct {
  int device;         /* CUDA device */
  int slots;          /* requests on the GPU at once (1 .. 64) */
  size_t hbm_budget;  /* bytes for all admitted requests together; 0 = 90% of the free memory */
} librpa_gpu_server_opts;

typedef struct {
  int status;             /* LIBRPA_OK or the request's error code */
  double ec;              /* E_c in Ha per cell */
  double ms_queue;        /* submit -> admission */
  double ms_run;          /* admission -> result */
  double ms_total;        /* submit -> result (the latency) */
  size_t bytes_reserved;  /* the estimate the request was admitted with */
  size_t bytes_peak;      /* its largest device footprint */
  int slot;               /* worker that ran it */
} librpa_gpu_result;

typedef struct {
  long long submitted, completed, failed;
  double p50_ms, p99_ms;     /* latency percentiles over the completed requests */
  double mean_queue_ms;
  double energies_per_s;     /* completed / (last completion - first submission) */
  int peak_running;          /* largest number of requests on the GPU at once */
  size_t peak_reserved;      /* largest sum of admitted estimates */
  size_t hbm_budget;         /* the budget in use */
} librpa_gpu_server_stats;

/* Upper bound of the device bytes h will hold during chi0 + ec, from its structure, LRI
 * blocks, precision and grid size (the user grid, else opts.n_tau).  Needs no GPU.
 * Errors: E_STATE (no structure), E_ARG. */
int librpa_gpu_estimate_bytes(librpa_gpu_t h, size_t *bytes);

/* Start the workers.  Errors: E_ARG, E_CUDA. */
int librpa_gpu_server_create(librpa_gpu_server_t *s, const librpa_gpu_server_opts *o);

/* New request handle (deferred inputs) with precision and grid options from *o (its
 * device, stream and allocator fields are ignored: the server supplies them).  Fill it
 * with set_structure, set_lri_coeffs, set_green, set_coulomb and optionally set_grid,
 * then submit it.  Free it with librpa_gpu_destroy after its result was taken.
 * Errors: E_ARG, E_NOMEM. */
int librpa_gpu_server_request(librpa_gpu_server_t s, const librpa_gpu_opts *o, librpa_gpu_t *req);

/* Queue a filled request; *ticket identifies it.  The caller must not use req until
 * librpa_gpu_server_wait has returned its result.  Errors: E_STATE (inputs missing),
 * E_NOMEM (its estimate exceeds the whole budget), E_ARG. */
int librpa_gpu_server_submit(librpa_gpu_server_t s, librpa_gpu_t req, long long *ticket);

/* Wait up to timeout_s seconds (< 0: no limit) for a request's result.  Returns
 * LIBRPA_OK with *r filled (r->status is the request's own code), or E_TIMEOUT if it is
 * not finished yet, E_ARG for an unknown ticket. */
int librpa_gpu_server_wait(librpa_gpu_server_t s, long long ticket, double timeout_s, librpa_gpu_result *r);

/* Counters and latency percentiles so far.  Errors: E_ARG. */
int librpa_gpu_server_get_stats(librpa_gpu_server_t s, librpa_gpu_server_stats *st);

/* Finish the running requests, cancel the queued ones (their status becomes
 * E_STATE), stop the workers and free the pool.  NULL is ignored. */
void librpa_gpu_server_destroy(librpa_gpu_server_t s);

/* One-line description of the last error on h (never NULL; "" after success). */
const char *librpa_gpu_last_error(librpa_gpu_t h);

/* Environment teardown (paper: finalize_librpa_environment): frees every device and
 * host resource of h.  NULL is ignored. */
void librpa_gpu_destroy(librpa_gpu_t h);

#ifdef __cplusplus
}
#endif

#endif /* LIBRPA_GPU_H */
