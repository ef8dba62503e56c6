// FP64-accurate GEMM on the BF16 tensor cores (tcgen05) by exact digit slicing.
//
// Each FP64 operand row r is written as 2^{E_r} sum_{s=1..S} d_s 2^{-7-8(s-1)} with integer
// digits |d_s| <= 128 (exact in BF16).  A product sums digit products d^A_s d^B_t over the pairs
// s + t <= S + 1; products of one "diagonal" d = s + t share the scale 2^{-14-8(d-2)}, so each
// diagonal accumulates in its own FP32 TMEM accumulator, which is exact while |sum| < 2^24
// (<= 1024 / (pairs of the diagonal) products of K).  Accumulators are flushed into exact int64
// register sums and scaled to FP64 once at the end.  S = 5 keeps 39 bits per operand (relative
// product error ~1e-12); S = 1..3 give the BF16 / split-precision ladder.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace librpa {
namespace oz {

constexpr int BM = 128, BN = 64, BK = 64, SMAX = 5;

// A K-major sliced operand: digits [S][rows][kpad] (BF16) and row exponents [rows].
struct Sliced {
  __nv_bfloat16 *digits = nullptr;
  int *expo = nullptr;
  int rows = 0;     // total rows (all batch entries stacked)
  int K = 0;        // logical K
  int kpad = 0;     // row pitch in elements (K rounded up to a multiple of 8)
  int S = 0;
};
size_t sliced_bytes(int rows, int K, int S);   // bytes for digits + exponents (256-byte aligned parts)
void sliced_bind(Sliced &o, void *mem, int rows, int K, int S);

// Sources of the splits.
//  real:    X[r][k] = src[r * ld + k]            (trans = false)   or src[k * ld + r] (trans = true)
//  complex: op(Z)[i][k] with op in {N, T, H}; Z row-major interleaved (re, im), leading dim ld.
//   as_a = true  -> stacked real matrix A'[2i + c][2k + c'] = [[Re, -Im], [Im, Re]] of op(Z)[i][k]
//   as_a = false -> B'^T[j][2k + c'] = component c' of op(Z)[k][j]
// batch entries are separated by `batch_stride` elements (doubles or complex numbers).
enum Op { OP_N = 0, OP_T = 1, OP_H = 2 };
void split_real(const double *src, long long ld, bool trans, int rows, int K, int batch, long long batch_stride,
                Sliced &out, cudaStream_t s);
void split_complex(const double2 *src, long long ld, Op op, bool as_a, int n_out, int n_k, int batch,
                   long long batch_stride, Sliced &out, cudaStream_t s);

// Output of a GEMM.
//  mode 0: real C[m][n] (ldc);
//  mode 1: complex C[i][j] (interleaved) from rows m = 2i + c: component c of C[i][j];
//  mode 2: complex transposed: component c of C[j][i].
struct Out {
  double *C = nullptr;
  long long ldc = 0;
  long long batch_stride = 0;   // doubles (mode 0) or complex numbers (modes 1, 2)
  int mode = 0;
  double alpha = 1.0, beta = 0.0;
};

// C = alpha * A B^T + beta * C for `batch` entries: A rows m in [0, M) of entry b are rows
// b * M .. of `a`, B rows likewise with N; an operand with exactly M (N) rows is shared by all
// entries.  K range per output tile starts at
// (m0 * km + n0 * kn) rounded down to BK (for triangular operands); lower_div > 0 skips tiles
// with n0 > m0 / lower_div.  `err` (device int) is set to 1 if a bounded wait runs out.
// Returns the number of tiles launched.
long long gemm(const Sliced &a, const Sliced &b, int M, int N, int batch, const Out &out, int km, int kn,
               int lower_div, int *err, cudaStream_t s);

// One-time host setup (driver entry point for tensor-map encoding).  Throws on failure.
void init();

}  // namespace oz
}  // namespace librpa
