// Internal declarations of librpa_gpu (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/librpa_gpu.h"

namespace librpa {

// ----------------------------------------------------------------- error plumbing
struct Error {
  int code;
  std::string msg;
};

#define LR_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      throw ::librpa::Error{LIBRPA_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

// ----------------------------------------------------------------- BvK helpers
struct Mesh {
  int n1 = 1, n2 = 1, n3 = 1;
  int size() const { return n1 * n2 * n3; }
  static int fold(int x, int n) { int r = x % n; return r < 0 ? r + n : r; }
  int index(int a, int b, int c) const { return (fold(a, n1) * n2 + fold(b, n2)) * n3 + fold(c, n3); }
  void split(int i, int &a, int &b, int &c) const { a = i / (n2 * n3); b = (i / n3) % n2; c = i % n3; }
  int neg(int i) const { int a, b, c; split(i, a, b, c); return index(-a, -b, -c); }   // index of -R (or -q)
};

// ----------------------------------------------------------------- device buffers
struct Handle;
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

// ----------------------------------------------------------------- chi0 plan (Algorithm 1 data layout)
// Neighbour entry of atom U: block C[U, K, R1] (K an atom, R1 a lattice vector).
struct NbEntry {
  int K;
  int R[3];
  int col;        // first column of this block inside the packed matrix of U (0 .. m_U)
  int ucol;       // first column of (K, R1) inside the union list (0 .. M_all)
};

struct Chi0Plan {
  int natoms = 0, nao = 0, naux = 0;
  std::vector<int> n_ao, n_aux, ao_off, aux_off;
  std::vector<std::vector<NbEntry>> nb;   // per atom U: N[U] sorted by (K, R)
  std::vector<int> m;                     // m_U = sum over N[U] of n_ao(K)
  std::vector<long long> cp_off;          // offset of packed C_U [n_aux_U][n_U][m_U] in the C arena
  long long cp_total = 0;
  // union of all (K, R1) over N[U], U in the home cell
  std::vector<std::tuple<int, int, int, int>> uni;  // (K, R0, R1, R2)
  std::vector<int> uni_col;               // first column of each union block
  int m_all = 0;
  // device index tables (int arrays; see k_chi0.cu for their meaning)
  DevBuf d_lam;      // per-V columns of the packed C: {L, R0, R1, R2, l, ao(L)+l} x sum m_V
  DevBuf d_uni;      // union columns: {K, R0, R1, R2, k, ao(K)+k} x M_all
  DevBuf d_kap;      // per-U columns: {K, R0, R1, R2, ao(K)+k, ucol} x sum m_U
  std::vector<long long> lam_off, kap_off;   // element offsets of each atom's part
  // workspace element offsets (per (R, tau) point)
  std::vector<long long> bg_off, ag_off, n_off, x_off, o_off;
  long long bg_sz = 0, ag_sz = 0, n_sz = 0, x_sz = 0, o_sz = 0;
  double flop_per_point = 0;  // algorithmic FP64 flops per (R, tau) point
  double flop_nx_per_point = 0;  // the part of it in the N and X steps
  double flop_fin_per_point = 0; // the part of it in the final contraction
  // device copies of the per-atom tables, point list, workspace and GEMM descriptors
  DevBuf t_n_ao, t_n_aux, t_ao_off, t_aux_off, t_m, t_lam_off, t_kap_off, t_bg_off, t_ag_off, t_n_off, t_x_off,
      t_o_off, t_pts, ws, gargs1, gargs2;
  // tensor-core route: digit planes of the packed coefficients in the two row groupings
  // (rows (nu, j) per atom with K = m_V for the N and X steps; rows mu with K = n_U m_U for
  // the final contraction), the planes' shape, and the ragged-entry tables of the O operand
  int tc_S = 0, max_m = 0, max_nm = 0, cpnx_rows = 0;
  // FP64 route: tile variants of the N/X and final GEMM launches (-1 = tune on first use), and a
  // generation number bumped by every re-plan (batched runs key their captured graphs on it)
  int var_nx = -1, var_fin = -1;
  long long gen = 0;
  std::vector<int> cpnx_off;
  DevBuf cp_nx, cp_f, t_oe_off, t_oe_k, gargs3;
  DevBuf t_ozero;   // screening: O-assembly blocks that are exactly zero, per point batch
  DevBuf t_ugroups; // atoms grouped by the O assembly's row-block size; group g at [ugroup_off[g], ugroup_off[g+1])
  std::vector<int> ugroup_off;
  std::vector<DevBuf *> all() {
    return {&d_lam, &d_uni, &d_kap, &t_n_ao, &t_n_aux, &t_ao_off, &t_aux_off, &t_m, &t_lam_off, &t_kap_off,
            &t_bg_off, &t_ag_off, &t_n_off, &t_x_off, &t_o_off, &t_pts, &ws, &gargs1, &gargs2,
            &cp_nx, &cp_f, &t_oe_off, &t_oe_k, &gargs3, &t_ozero, &t_ugroups};
  }
};

// ----------------------------------------------------------------- handle
struct Handle {
  librpa_gpu_opts opts{};
  int chi0_S = -1;  // chi0 GEMMs: -1 = FP64 pipes, 0 = plain BF16, 1..5 = BF16 digit planes, 6 = plain TF32,
                    // 7 = 3xTF32
  int ec_S = -1;    // ln det GEMMs: same encoding
  bool freq_f32 = false;   // tau -> omega and R -> q transforms in FP32 (LIBRPA_SPLIT_FAST)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string last_error;
  size_t bytes_held = 0, bytes_peak = 0;
  std::map<void *, size_t> allocs;
  // deferred inputs (requests of the serving loop): set_green and set_coulomb keep the KS
  // coefficients and V(q) on the host until materialize() uploads them
  bool deferred = false;
  std::vector<double> stage_wfc;   // [nk][nb][nao] complex interleaved
  std::vector<double> stage_vq;    // [nq][naux][naux] complex interleaved

  // structure
  bool have_structure = false;
  int natoms = 0, nao = 0, naux = 0, nspins = 1;
  int cur_spin = 0;   // spin channel the chi0 contraction is working on
  double lat[9]{};
  std::vector<double> pos;
  std::vector<int> n_ao, n_aux, ao_off, aux_off;
  Mesh mesh;
  double r_cut = 0;

  // inputs (host staging)
  std::map<std::tuple<int, int, int, int, int>, std::vector<double>> lri;  // (I,K,R0,R1,R2) -> C
  std::vector<double> eig, occ;            // [nk][nb] host copies (grid range, band ranges)
  std::vector<char> have_k;
  std::vector<double> efermi_k;
  std::vector<char> have_q;
  int vq_sym = -1;   // V(-q) = conj V(q) for every q: -1 not checked yet, 0 no, 1 yes
  int vq_real = -1;  // V(q) real at every q = -q (same check): -1 not checked yet, 0 no, 1 yes
  std::vector<double> wq;   // per-q weights of the E_c sum (set_q_weights); empty = 1 / N_q

  // Green's-function block screening: threshold (0 = off), the kept-block mask of the current
  // G [spin][g][tau][R][I][J] (host copy) and its device buffers
  double g_screen = 0;
  std::vector<unsigned char> gmask;
  DevBuf d_gmask, d_screen_tab;

  // grid
  bool have_grid = false, grid_user = false;
  int ntau = 0;
  std::vector<double> tau, omega, w_omega, gamma;

  // device state
  DevBuf d_vq;        // [nq][naux][naux] complex interleaved
  DevBuf d_wfc;       // [nk][nb][nao] complex interleaved: wfc[k][n][i] = c_in(k)
  DevBuf d_eig, d_occ;  // [nk][nb]
  DevBuf d_g;         // G: [2][ntau][nR][nao][nao]  (0 = occ, 1 = vir)
  DevBuf d_chi_tau;   // [ntau][nR][naux][naux]
  DevBuf d_chi_qw;    // [nq][nomega][naux][naux] complex interleaved
  DevBuf d_cpack;     // packed LRI coefficients
  DevBuf zgemm_args;  // descriptors and tile lists of batched GEMM launches
  DevBuf rgemm_args;  // the same for the real GEMMs of the ln det stage
  DevBuf gemm_args;
  DevBuf oz_args;     // descriptors of the tensor-core GEMM launches
  DevBuf work;        // per-call workspace
  double oz_exec_flops = 0;  // MMA flops issued by the last digit-plane GEMM launch
  double oz_alg_flops = 0;   // algorithmic flops (2 M N K over the summed K) of that launch
  int stalls_left = 0;       // testing only: tensor-core GEMM launches still to take the failure path
  double flop_chi0_run = 0;  // algorithmic flops of the last contraction (screened work left out)
  bool chi0_done = false, lri_dirty = true;
  Chi0Plan plan;

  librpa_gpu_stats stats{};

  // event-timed launches of the dense GEMM kernels, resolved after a stream synchronisation
  struct Timed {
    cudaEvent_t a, b;
    double flops;
    int kind;  // 0 = GEMM of the chi0 contraction, 1 = GEMM of the energy stage
    double exec_flops = 0;  // tensor-core MMA flops issued (digit-plane GEMMs only)
  };
  std::vector<Timed> timed;
  void resolve_timers();

  void *dalloc(size_t bytes);
  void dfree(void *p);
  void ensure(DevBuf &b, size_t bytes);
  void release(DevBuf &b);
  // Host -> device upload of small tables (launch descriptors, tile and point lists) through a
  // pinned staging ring, so the copy is asynchronous: a copy from pageable memory would first
  // synchronise the stream and leave the GPU idle between launches.  The ring is reused after the
  // last copy from it has completed (an event), at a wrap or a change of stream.
  void upload_async(DevBuf &dst, const void *src, size_t bytes);
  void free_pinned();
  char *pin = nullptr;
  size_t pin_bytes = 0, pin_head = 0;
  cudaEvent_t pin_done = nullptr;
  cudaStream_t pin_stream = nullptr;
};

// ----------------------------------------------------------------- grid (host, grid.cpp)
int build_grid(int n, double dmin, double dmax, double *tau, double *omega, double *w_omega,
               double *gamma);
// Gamma_kj: relative least-squares fit of 2D / (D^2 + omega_k^2) by sum_j Gamma_kj exp(-D tau_j) on
// 1000 log-spaced D in [dmin, dmax] (SVD, singular values below 1e-12 s_max dropped)
void fit_gamma(int n, const double *tau, const double *omega, double dmin, double dmax, double *gamma);
// minimax grids (minimax.cpp): the range ratio R_b a grid of n points is built for, and the grid
int build_grid_minimax(int n, double dmin, double dmax, double *tau, double *omega, double *w_omega, double *gamma,
                       double *info);
double minimax_range(int n, double dmin, double dmax);
constexpr int kMinimaxMaxN = 20;   // largest minimax grid (the Gauss-Legendre grids go to 64)

// ----------------------------------------------------------------- kernels
// K1 (k_green.cu): G^occ and G^vir for all (tau, R).  Returns max |Im G| / max |G|.
double green_build(Handle &h);
size_t green_work_bytes(const Handle &h);
// K2 (k_chi0.cu)
void chi0_plan(Handle &h);
void chi0_run(Handle &h, double *ms_gemm);
// host part of chi0_plan: neighbour lists, packed-column sizes, workspace offsets, flops
void chi0_shape(const Handle &h, Chi0Plan &P);
// device bytes the chi0 stage holds for this shape (packed C and its digit planes, chi0(R, tau),
// batch workspace, tables)
size_t chi0_device_bytes(const Handle &h, const Chi0Plan &P);
// Batched chi0 of several handles (FP64 route) on hs[0]'s stream, in rounds: round r takes the
// r-th point batch of every handle, and the N/X and final GEMMs of a round are single grouped
// launches over all those handles' tiles.  The launch sequence is captured in a CUDA graph on
// the first call and replayed while no plan changes.
struct MergedChi0 {
  std::vector<Handle *> hs;
  std::vector<long long> gens;
  std::vector<DevBuf> nx_args, fin_args;   // descriptors of every round, allocated through hs[0]
  int var_nx = -1, var_fin = -1;
  cudaGraphExec_t exec = nullptr;
  long long nodes = 0;
  bool graph_failed = false;
  void reset();
};
// returns true when the launches were replayed from the captured graph
bool chi0_run_merged(std::vector<Handle *> &hs, MergedChi0 &m);
// whether h takes part in chi0_run_merged (FP64 route, one spin channel)
bool chi0_fits_one_batch(const Handle &h);
// Batched chi0 of several tensor-core handles (same digit-plane count, one spin channel, no
// screening, all on one stream): in rounds of point batches, each round's N-step, X-step and final
// GEMMs of all handles as one launch over their tiles (operand pairs per handle); gathers, splits
// and O assembly per handle.
bool chi0_fits_tc_batch(const Handle &h);
void chi0_run_tc_merged(std::vector<Handle *> &hs);

// lattice vectors R whose chi0(R, tau) is computed (R <= -R in the flat BvK order); the others
// are filled as chi0(-R, tau)^T
std::vector<int> chi0_r_list(const Mesh &m);
// K3 + K4 (k_freq.cu)
void freq_transform(Handle &h);
size_t freq_work_bytes(const Handle &h);
// K5 + K6 (k_ec.cu); returns LIBRPA_OK or LIBRPA_E_NOT_PD
int ec_run(Handle &h, double *ec, double *ec_q, double *ec_w);
size_t ec_work_bytes(const Handle &h);

// api.cu: upload the deferred inputs of h; release every device buffer of h; an upper bound of
// the device bytes h holds during chi0 + ec (grid size from the user grid or opts.n_tau)
// checks before the chi0 stage (inputs complete, one Fermi level) and the grid from the KS
// spectrum when none was set; returns LIBRPA_OK or an error code with h.last_error set
int chi0_prepare(Handle &h);
void materialize(Handle &h);
void release_device(Handle &h);
size_t estimate_device_bytes(Handle &h);

// generic batched complex FP64 GEMM (k_zgemm.cu), used by K1 and K5
struct ZGemm {
  const double2 *A;   // row-major, lda
  const double2 *B;   // row-major, ldb
  double2 *C;         // row-major, ldc
  const double *kscale;  // optional per-k real scale of the product (length K), or nullptr
  int M, N, K, lda, ldb, ldc;
  double2 alpha, beta;
};
// op(A): transA (A stored [K][M]) / conjA; op(B): transB (B stored [N][K]) / conjB.
// kfrom: 0 = full K range, 1 = start at the tile's first row (A upper-zero rows),
// 2 = start at the tile's first column (B lower-triangular, zero above the diagonal).
// lower_only: skip output tiles strictly above the diagonal.
struct ZGemmFlags {
  bool transA = false, conjA = false, transB = false, conjB = false;
  int kfrom = 0;
  bool lower_only = false;
};
// timed_kind >= 0 records the launch with CUDA events as Handle::Timed{kind, algorithmic flops}.
void zgemm_batched(const std::vector<ZGemm> &batch, const ZGemmFlags &f, cudaStream_t s,
                   Handle &h, int timed_kind = -1, double flops = 0.0);

long long &launch_counter();

}  // namespace librpa

// the opaque handle type of the C ABI
struct librpa_gpu : public librpa::Handle {};
