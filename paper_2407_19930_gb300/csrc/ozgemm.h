// FP64-accurate GEMM on the BF16 tensor cores (tcgen05) by exact digit slicing.
//
// Each FP64 operand row r is written as 2^{E_r} sum_{s=1..S} d_s 2^{-7-8(s-1)} with integer
// digits |d_s| <= 128 (exact in BF16).  A product sums digit products d^A_s d^B_t over the pairs
// s + t <= S + 1; products of one "diagonal" d = s + t share the scale 2^{-14-8(d-2)}, so each
// diagonal accumulates in its own FP32 TMEM accumulator, which is exact while |sum| < 2^24
// (<= 1024 / (pairs of the diagonal) products of K).  Accumulators are flushed into exact int64
// register sums and scaled to FP64 once at the end.  S = 5 keeps 39 bits per operand (relative
// product error ~1e-12); S = 1..3 give the BF16 / split-precision ladder.  Two plain forms
// take one plane of values rounded per element and accumulate in FP32 over all K: S = 0 (BF16,
// kind::f16) and S = S_TF32 (TF32 in FP32 containers, kind::tf32).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <functional>
#include <utility>
#include <vector>

namespace librpa {
struct Handle;
struct DevBuf;
namespace oz {

// S_TF32: one plane of TF32 values; S_TF32X3: two planes hi = tf32(x), lo = tf32(x - hi) and the
// three products hi hi + hi lo + lo hi summed in one FP32 accumulator (the "3xTF32" split)
constexpr int BM = 128, BN = 64, BK = 64, SMAX = 5, S_TF32 = 6, S_TF32X3 = 7;
inline int planes(int S) { return S >= 1 && S <= SMAX ? S : S == S_TF32X3 ? 2 : 1; }
inline int elem_bytes(int S) { return S == S_TF32 || S == S_TF32X3 ? 4 : 2; }

// K-major sliced operand: digit planes [S][rows][kpad] (BF16; FP32 for S_TF32) and row exponents
// [rows].
struct Sliced {
  void *digits = nullptr;
  int *expo = nullptr;
  int rows = 0;     // total rows
  int K = 0;        // logical K (columns beyond K and up to kpad hold zero digits)
  int kpad = 0;     // row pitch in elements (K rounded up to a multiple of 8)
  int S = 0;        // digit planes 1..SMAX; 0 = one plane of plain BF16 values, S_TF32 = one plane
                    // of plain TF32 values (own exponent per element, rounded to nearest)
};
size_t sliced_bytes(int rows, int K, int S);   // bytes for digits + exponents (256-byte aligned parts)
void sliced_bind(Sliced &o, void *mem, int rows, int K, int S);

// Row r of a split source is produced by `Src::get(r, k)` for k < K; rows [row0, row0 + rows)
// of the destination are written (digits for k in [K, kpad) are zero).
enum Op { OP_N = 0, OP_T = 1, OP_H = 2, OP_C = 3 };   // OP_C: complex conjugate, not transposed
//  real:    X[r][k] = src[r * ld + k] (trans = false) or src[k * ld + r] (trans = true); entries of
//           `rows` rows each are `batch_stride` doubles apart.
void split_real(const double *src, long long ld, bool trans, int rows, int K, int batch, long long batch_stride,
                Sliced &out, cudaStream_t s, int row0 = 0);
//  complex: op(Z)[i][k] with op in {N, T, H, C}; Z row-major interleaved (re, im), leading dim ld.
//   as_a = true  -> stacked real matrix A'[2i + c][2k + c'] = [[Re, -Im], [Im, Re]] of op(Z)[i][k]
//   as_a = false -> B'^T[j][2k + c'] = component c' of op(Z)[k][j]
void split_complex(const double2 *src, long long ld, Op op, bool as_a, int n_out, int n_k, int batch,
                   long long batch_stride, Sliced &out, cudaStream_t s);
//  gathered Green's-function blocks of the chi0 contraction (see k_chi0.cu for the tables):
//   kind 0 (Bg): row (p, g, V, kappa), k = lambda of V:  G^g(tau_p)[bvk(R1_kappa - R_p - R2'_lambda)][ao_lambda][ao_kappa]
//   kind 1 (Ag): row (p, g, V, i),     k = lambda of V:  G^g(tau_p)[bvk(R_p + R2'_lambda)][i][ao_lambda]
struct GatherSrc {
  int kind;
  const double *G;
  long long g_gstride;
  int nR, nao, n1, n2, n3, natoms, rows_per_entry;
  const int *pts;        // per point: {iR, itau, R0, R1, R2}
  const int *uni;        // union column table (6 ints per column)
  const int *lam;        // per-atom column tables (6 ints per column)
  const long long *lam_off;
  const int *m;          // m_V
};
void split_gather(const GatherSrc &src, int rows, int K, Sliced &out, cudaStream_t s);
//  ragged entries: row r belongs to entry e = r / rows_per_entry; its K_e columns are
//  base[off[e] + (r % rows_per_entry) * K_e + k] (zero for k >= K_e); off, K on the device.
//  expo_given: out.expo already holds each row's exponent (its largest biased FP64 exponent
//  minus 1022, as the exponent pass would write it), which is then not recomputed.
void split_ragged(const double *base, const long long *off, const int *Ke, int rows_per_entry, int n_entries,
                  int Kmax, Sliced &out, cudaStream_t s, bool expo_given = false);
//  out.expo[r] = -1022 (an all-zero row) for r < rows: the start of an exponent built by atomicMax
void expo_init(Sliced &out, int rows, cudaStream_t s);

// Output of a GEMM entry.
//  mode 0: real C[m][n] (ldc);
//  mode 3: real C[m][n] stored as a pair of FP32 numbers (hi, lo) in the 8 bytes of the double
//          (beta must be 0);
//  mode 1: complex C[i][j] (interleaved) from rows m = 2i + c: component c of C[i][j];
//  mode 2: complex transposed: component c of C[j][i];
//  mode 4: real transposed: C[n][m] (ldc).
struct Out {
  double *C = nullptr;
  long long ldc = 0;
  long long batch_stride = 0;   // doubles (modes 0, 4) or complex numbers (modes 1, 2)
  int mode = 0;
  double alpha = 1.0, beta = 0.0;
};

// One GEMM of a grouped launch: C = alpha A[a_row0 .. + M) B[b_row0 .. + N)^T + beta C over
// K columns.  K range per output tile starts at (m0 * km + n0 * kn) rounded down to BK
// (triangular operands); lower_div > 0 skips the tiles strictly above the diagonal, those with
// n0 * lower_div >= m0 + BM (lower_div stacked rows per output row: 2 for complex outputs).
constexpr int kNoShift = 1 << 30;
struct Entry {
  int a_row0, b_row0, M, N, K;
  int km, kn, lower_div;
  double *C;
  long long ldc;
  int mode;
  double alpha, beta;
  int alpha_shift;   // set by the launch: k when alpha = +-2^k, else kNoShift
  int pair;          // gemm_multi: index of the entry's operand pair (gemm_grouped sets 0)
};

// K stages a tile of entry e must sum (block-sparse operands): stage_fn(e, m0, rows, n0, cols, stage K,
// K, out) appends the needed stage indices (ascending) and returns true, or returns false for all.
using StageFn = std::function<bool(int, int, int, int, int, int, int, std::vector<int> &)>;

// Grouped launch over all tiles of all entries; operand digit planes of the A role in `a`, of
// the B role in `b` (same S).  `err` (device int) is set to 1 if a bounded wait runs out.
// `args` is scratch for the descriptor upload.  Returns the number of tiles.  Sets
// h.oz_exec_flops (MMA flops issued) and h.oz_alg_flops (2 M N K over the summed K).
long long gemm_grouped(const Sliced &a, const Sliced &b, const std::vector<Entry> &entries, int *err,
                       cudaStream_t s, Handle &h, DevBuf &args, const StageFn *stage_fn = nullptr);

// The same over several operand pairs (same S): entry e multiplies ops[e.pair].first (A role) by
// ops[e.pair].second (B role).  All tiles of all entries run in one persistent launch.
long long gemm_multi(const std::vector<std::pair<const Sliced *, const Sliced *>> &ops, const std::vector<Entry> &entries,
                     int *err, cudaStream_t s, Handle &h, DevBuf &args, const StageFn *stage_fn = nullptr);

// Uniform batch: A rows m in [0, M) of entry b are rows b * M .. of `a`, B rows likewise with N;
// an operand with exactly M (N) rows is shared by all entries.
long long gemm(const Sliced &a, const Sliced &b, int M, int N, int batch, const Out &out, int km, int kn,
               int lower_div, int *err, cudaStream_t s, Handle &h);

// One-time host setup (driver entry point for tensor-map encoding).  Throws on failure.
void init();

}  // namespace oz
}  // namespace librpa
