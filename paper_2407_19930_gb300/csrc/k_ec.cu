// K5 + K6: RPA correlation energy (Sec. 2):
//
//   E_c = (1/2 pi) sum_q w_q sum_k W_k { ln det[1 - Pi(q, i omega_k)] + Tr Pi(q, i omega_k) },  Pi = chi0 V.
//
// With the Cholesky factor V(q) = L L^H, det(1 - chi0 V) = det(I - L^H chi0 L) (Sylvester) and
// A = I - L^H chi0 L is Hermitian positive definite (chi0 <= 0), so ln det A = 2 sum_i ln (L_A)_ii
// from a Cholesky factorisation A = L_A L_A^H, and Tr Pi = Tr(L^H chi0 L).  Per q: factor V;
// per (q, omega): W = chi0 L, A = I - L^H W (lower triangle), factor A.  The factorisations are
// right-looking and blocked (panel width NB): the diagonal block is factored in shared memory by
// one CTA per matrix, the panel below it by a triangular solve, and the trailing matrix is
// updated by a batched GEMM; every matrix of a batch advances panel by panel in step, so each
// launch has work from all of them.
//
// Two arithmetic routes for the dense GEMMs (W, L^H W and the trailing updates):
//   * native FP64 (complex GEMM on the FP64 pipe, k_zgemm.cu);
//   * digit-sliced on the BF16 tensor cores (k_ozgemm.cu, S digit planes): complex products as
//     2 x 2 real blocks [[Re, -Im], [Im, Re]], W produced transposed so that the second GEMM reads
//     it row by row.
// The diagonal blocks, the panel solves, the logarithms and the energy sum are FP64 in both.
// On the FP64 route the q with q = -q (chi0 and, when checked, V real there) run every step in
// real arithmetic (A = I - L^T chi0 L, real GEMMs and a real Cholesky): a quarter of the flops.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "ozgemm.h"

namespace librpa {
namespace {

constexpr int NB = 64;

// Factor the NB x NB diagonal block at p0 of every matrix in place (lower triangle).  One CTA per
// matrix.  Adds 2 sum ln d_jj to lndet[b]; sets info[b] = 1 on a non-positive pivot.
// inv (optional, [matrix][NB][NB]): receives L_pp^{-1} of the factored block (lower triangular,
// zero elsewhere), computed in shared memory by forward substitution, one column per thread.
__global__ void __launch_bounds__(256) k_potrf_diag(double2 *const *mats, int n, int ld, int p0, double *lndet,
                                                    int *info, double2 *inv) {
  extern __shared__ double2 a[];   // [NB][NB + 1] (and, with inv, a second such array)
  const int b = blockIdx.x;
  double2 *M = mats[b];
  const int nb = min(NB, n - p0);
  const int lda = NB + 1;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    a[i * lda + j] = j <= i ? M[(size_t)(p0 + i) * ld + p0 + j] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  __shared__ double dsh;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  double lsum = 0.0;
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      double d = a[j * lda + j].x;
      if (!(d > 0.0) || !isfinite(d)) {
        bad = 1;
        d = 1.0;
      }
      d = sqrt(d);
      a[j * lda + j] = make_double2(d, 0.0);
      lsum += 2.0 * log(d);
      dsh = d;
    }
    __syncthreads();
    const double inv = 1.0 / dsh;
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) {
      a[i * lda + j].x *= inv;
      a[i * lda + j].y *= inv;
    }
    __syncthreads();
    // trailing update of the block: a_ik -= a_ij conj(a_kj), j < k <= i
    const int m = nb - j - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e / m, k = j + 1 + e % m;
      if (k > i) continue;
      const double2 x = a[i * lda + j], y = a[k * lda + j];
      a[i * lda + k].x -= x.x * y.x + x.y * y.y;
      a[i * lda + k].y -= x.y * y.x - x.x * y.y;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    if (j <= i) M[(size_t)(p0 + i) * ld + p0 + j] = a[i * lda + j];
  }
  if (threadIdx.x == 0) {
    lndet[b] += lsum;
    if (bad) info[b] = 1;
  }
  if (inv) {
    // y = L^{-1}: column j solves L y_j = e_j (y_ij = 0 for i < j); L's diagonal is real.  Four
    // consecutive lanes per column (blockDim.x == 4 NB), each summing every fourth k of a row.
    double2 *y = a + NB * lda;
    const int j = threadIdx.x >> 2, part = threadIdx.x & 3;
    for (int i = 0; i < NB; ++i) {
      double sr = 0.0, si = 0.0;
      if (j < nb && i < nb && i > j)
        for (int k = j + part; k < i; k += 4) {
          const double2 l = a[i * lda + k], z = y[k * lda + j];
          sr += l.x * z.x - l.y * z.y;
          si += l.x * z.y + l.y * z.x;
        }
      sr += __shfl_xor_sync(0xffffffffu, sr, 1);
      si += __shfl_xor_sync(0xffffffffu, si, 1);
      sr += __shfl_xor_sync(0xffffffffu, sr, 2);
      si += __shfl_xor_sync(0xffffffffu, si, 2);
      if (part == 0) {
        double2 v = make_double2(0.0, 0.0);
        if (j < nb && i < nb && i >= j) {
          const double d = a[i * lda + i].x;
          v = make_double2(((i == j ? 1.0 : 0.0) - sr) / d, -si / d);
        }
        y[i * lda + j] = v;
      }
      __syncwarp();
    }
    __syncthreads();
    double2 *Y = inv + (size_t)b * NB * NB;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) Y[e] = y[(e / NB) * lda + e % NB];
  }
}

// Panel solve: rows i >= p0 + NB, X L_pp^H = B  =>  x_j = (b_j - sum_{k<j} x_k conj(L_jk)) / L_jj.
// One CTA per (matrix, 64-row chunk); one thread per row.
__global__ void __launch_bounds__(64) k_trsm_panel(double2 *const *mats, int n, int ld, int p0) {
  extern __shared__ double2 tsm[];
  double2(*L)[NB + 1] = reinterpret_cast<double2(*)[NB + 1]>(tsm);
  double2(*X)[NB + 1] = reinterpret_cast<double2(*)[NB + 1]>(tsm + NB * (NB + 1));
  const int b = blockIdx.y;
  double2 *M = mats[b];
  const int nb = min(NB, n - p0);
  const int r0 = p0 + nb + blockIdx.x * 64;
  if (r0 >= n) return;
  for (int e = threadIdx.x; e < nb * nb; e += 64) {
    const int i = e / nb, j = e % nb;
    L[i][j] = M[(size_t)(p0 + i) * ld + p0 + j];
  }
  const int rows = min(64, n - r0);
  for (int e = threadIdx.x; e < rows * nb; e += 64) {
    const int i = e / nb, j = e % nb;
    X[i][j] = M[(size_t)(r0 + i) * ld + p0 + j];
  }
  __syncthreads();
  const int i = threadIdx.x;
  if (i < rows) {
    for (int j = 0; j < nb; ++j) {
      double2 s = X[i][j];
      for (int k = 0; k < j; ++k) {
        const double2 x = X[i][k], l = L[j][k];
        // s -= x * conj(l)
        s.x -= x.x * l.x + x.y * l.y;
        s.y -= x.y * l.x - x.x * l.y;
      }
      const double inv = 1.0 / L[j][j].x;
      X[i][j] = make_double2(s.x * inv, s.y * inv);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rows * nb; e += 64) {
    const int r = e / nb, j = e % nb;
    M[(size_t)(r0 + r) * ld + p0 + j] = X[r][j];
  }
}

// Zero the strict upper triangle (so a Cholesky factor can be used as a triangular operand).
__global__ void k_zero_upper(double2 *const *mats, int n, int ld) {
  double2 *M = mats[blockIdx.y];
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (size_t)n * n) return;
  const int i = (int)(x / n), j = (int)(x % n);
  if (j > i) M[(size_t)i * ld + j] = make_double2(0.0, 0.0);
}

// Largest |V(-q) - conj V(q)| over the pairs q < -q (res[0]), largest |V(q)| (res[1]) and largest
// |Im V(q)| over the q = -q (res[2]), as the bit patterns of non-negative doubles (ordered like the
// values) for atomicMax.
__global__ void k_conj_check(const double2 *V, int n, int n1, int n2, int n3, unsigned long long *res) {
  const int q = blockIdx.y;
  const int a = q / (n2 * n3), b = (q / n3) % n2, c = q % n3;
  const int p = (((n1 - a) % n1) * n2 + (n2 - b) % n2) * n3 + (n3 - c) % n3;
  if (p < q) return;
  const bool self = p == q;
  const size_t nn = (size_t)n * n;
  const double2 *Vq = V + nn * q, *Vp = V + nn * p;
  double d = 0.0, m = 0.0;
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < nn; x += (size_t)gridDim.x * blockDim.x) {
    const double2 u = Vq[x], v = Vp[x];
    d = self ? fmax(d, fabs(u.y)) : fmax(d, fmax(fabs(v.x - u.x), fabs(v.y + u.y)));
    m = fmax(m, fmax(fabs(u.x), fabs(u.y)));
    if (isnan(u.x + u.y + v.x + v.y)) d = INFINITY;
  }
  for (int o = 16; o > 0; o >>= 1) {
    d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(res + (self ? 2 : 0), (unsigned long long)__double_as_longlong(d));
    atomicMax(res + 1, (unsigned long long)__double_as_longlong(m));
  }
}

// ---------------------------------------------------------------------------------------
// Real route for the q with q = -q (time-reversal-invariant q: q.R is a multiple of pi for every
// lattice vector, so chi0(q, i omega) = sum_R (+-1) chi0(R, i omega) is real symmetric, and V(q)
// is real when V(-q) = conj V(q)).  There A = I - L^T chi0 L is real and every product runs in
// real arithmetic: a quarter of the complex flops.

// Lt = (Re L)^T, n x n, through 32 x 32 shared-memory tiles
__global__ void k_real_transpose(const double2 *L, int n, double *Lt) {
  __shared__ double t[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int gr = r0 + r, gc = c0 + threadIdx.x;
    if (gr < n && gc < n) t[r][threadIdx.x] = L[(size_t)gr * n + gc].x;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int gr = c0 + r, gc = r0 + threadIdx.x;   // Lt[gr][gc] = L[gc][gr]
    if (gr < n && gc < n) Lt[(size_t)gr * n + gc] = t[threadIdx.x][r];
  }
}

__global__ void k_real_part(const double2 *src, size_t count, double *dst) {
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < count) dst[x] = src[x].x;
}

struct RGemm {
  const double *A, *B;   // A [M][K] (lda), B [N][K] (ldb), row-major
  double *C;             // C [M][N] (ldc)
  int M, N, K, lda, ldb, ldc;
  double alpha, beta;
};
struct RTile {
  int e, m0, n0, k0;     // descriptor, output tile origin, first k (rows of A zero before it)
};

// C = alpha A B^T + beta C on the FP64 tensor cores (mma.sync m8n8k4 f64): one 64 x 64 tile per
// CTA, four warps with 32 x 32 warp tiles, K staged 16 at a time through shared memory from the
// tile's k0 (A is upper triangular in the ln det products, zero left of the tile's first row).
__global__ void __launch_bounds__(128) k_dgemm_tri(const RGemm *__restrict__ gs, const RTile *__restrict__ tiles) {
  constexpr int BM = 64, BN = 64, KS = 16, NT = 128;
  const RTile t = tiles[blockIdx.x];
  const RGemm g = gs[t.e];
  __shared__ double As[BM][KS + 1];
  __shared__ double Bs[BN][KS + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1, gid = lane >> 2, tig = lane & 3;
  double acc[4][4][2];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c][0] = acc[r][c][1] = 0.0;
  for (int k0 = t.k0; k0 < g.K; k0 += KS) {
    for (int e = tid; e < BM * KS; e += NT) {
      const int row = e / KS, k = e % KS, gm = t.m0 + row, gk = k0 + k;
      As[row][k] = (gm < g.M && gk < g.K) ? g.A[(size_t)gm * g.lda + gk] : 0.0;
    }
    for (int e = tid; e < BN * KS; e += NT) {
      const int row = e / KS, k = e % KS, gn = t.n0 + row, gk = k0 + k;
      Bs[row][k] = (gn < g.N && gk < g.K) ? g.B[(size_t)gn * g.ldb + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KS; kk += 4) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[wm * 32 + r * 8 + gid][kk + tig];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[wn * 32 + c * 8 + gid][kk + tig];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                       : "+d"(acc[r][c][0]), "+d"(acc[r][c][1])
                       : "d"(a[r]), "d"(b[c]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gm = t.m0 + wm * 32 + r * 8 + gid;
    if (gm >= g.M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int gn = t.n0 + wn * 32 + c * 8 + tig * 2 + hh;
        if (gn >= g.N) continue;
        double *p = g.C + (size_t)gm * g.ldc + gn;
        const double v = g.alpha * acc[r][c][hh];
        *p = g.beta == 0.0 ? v : v + g.beta * *p;
      }
  }
}

// Real diagonal-block Cholesky (as k_potrf_diag, real arithmetic).
__global__ void __launch_bounds__(256) k_potrf_diag_r(double *const *mats, int n, int ld, int p0, double *lndet,
                                                      int *info) {
  extern __shared__ double ar[];   // [NB][NB + 1]
  const int b = blockIdx.x;
  double *M = mats[b];
  const int nb = min(NB, n - p0);
  const int lda = NB + 1;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    ar[i * lda + j] = j <= i ? M[(size_t)(p0 + i) * ld + p0 + j] : 0.0;
  }
  __syncthreads();
  __shared__ double dsh;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  double lsum = 0.0;
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      double d = ar[j * lda + j];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = 1;
        d = 1.0;
      }
      d = sqrt(d);
      ar[j * lda + j] = d;
      lsum += 2.0 * log(d);
      dsh = d;
    }
    __syncthreads();
    const double inv = 1.0 / dsh;
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) ar[i * lda + j] *= inv;
    __syncthreads();
    const int m = nb - j - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e / m, k = j + 1 + e % m;
      if (k > i) continue;
      ar[i * lda + k] -= ar[i * lda + j] * ar[k * lda + j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    if (j <= i) M[(size_t)(p0 + i) * ld + p0 + j] = ar[i * lda + j];
  }
  if (threadIdx.x == 0) {
    lndet[b] += lsum;
    if (bad) info[b] = 1;
  }
}

// Real panel solve X L_pp^T = B (as k_trsm_panel, real arithmetic).
__global__ void __launch_bounds__(64) k_trsm_panel_r(double *const *mats, int n, int ld, int p0) {
  extern __shared__ double tr[];
  double(*L)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(tr);
  double(*X)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(tr + NB * (NB + 1));
  const int b = blockIdx.y;
  double *M = mats[b];
  const int nb = min(NB, n - p0);
  const int r0 = p0 + nb + blockIdx.x * 64;
  if (r0 >= n) return;
  for (int e = threadIdx.x; e < nb * nb; e += 64) {
    const int i = e / nb, j = e % nb;
    L[i][j] = M[(size_t)(p0 + i) * ld + p0 + j];
  }
  const int rows = min(64, n - r0);
  for (int e = threadIdx.x; e < rows * nb; e += 64) {
    const int i = e / nb, j = e % nb;
    X[i][j] = M[(size_t)(r0 + i) * ld + p0 + j];
  }
  __syncthreads();
  const int i = threadIdx.x;
  if (i < rows) {
    for (int j = 0; j < nb; ++j) {
      double sv = X[i][j];
      for (int k = 0; k < j; ++k) sv -= X[i][k] * L[j][k];
      X[i][j] = sv / L[j][j];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rows * nb; e += 64) {
    const int r = e / nb, j = e % nb;
    M[(size_t)(r0 + r) * ld + p0 + j] = X[r][j];
  }
}

// A = -L^T chi0 L on entry: trace[b] = -sum A_ii, then A_ii += 1 (real route).
__global__ void k_diag_shift_r(double *const *mats, int n, int ld, double *trace) {
  double *M = mats[blockIdx.x];
  double sv = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double *p = M + (size_t)i * ld + i;
    sv -= *p;
    *p += 1.0;
  }
  __shared__ double red[256];
  red[threadIdx.x] = sv;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) trace[blockIdx.x] = red[0];
}

// A = -L^H chi0 L on entry (lower triangle).  trace[b] = Re Tr(L^H chi0 L) = -sum Re A_ii;
// then A_ii += 1 (A = I - L^H chi0 L).  One CTA per matrix.
__global__ void k_diag_shift(double2 *const *mats, int n, int ld, double *trace) {
  double2 *M = mats[blockIdx.x];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double2 *p = M + (size_t)i * ld + i;
    s -= p->x;
    p->x += 1.0;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) trace[blockIdx.x] = red[0];
}

// K6: E_c, per-q and per-omega parts from the per-(q, omega) ln det and trace.  w_q: per-q weights
// of the q sum, or nullptr for 1 / N_q.
__global__ void k_energy(const double *lndet, const double *trace, const double *w_omega, const double *w_q, int nq,
                         int nw, double *out /* [1 + nq + nw] */) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double uniform = 1.0 / (2.0 * M_PI * nq);
  double tot = 0.0;
  for (int k = 0; k < nw; ++k) out[1 + nq + k] = 0.0;
  for (int q = 0; q < nq; ++q) {
    const double pref = w_q ? w_q[q] / (2.0 * M_PI) : uniform;
    double sq = 0.0;
    for (int k = 0; k < nw; ++k) {
      const double f = pref * w_omega[k] * (lndet[q * nw + k] + trace[q * nw + k]);
      sq += f;
      out[1 + nq + k] += f;
    }
    out[1 + q] = sq;
    tot += sq;
  }
  out[0] = tot;
}

// Sliced-operand scratch of the tensor-core route.
struct TcScratch {
  oz::Sliced pa, pb;      // panel of the trailing updates (as A' and as B'^T)
  oz::Sliced pi;          // L_pp^{-H} of the panel solves (as B'^T)
  double2 *inv = nullptr; // [matrix][NB][NB]: L_pp^{-1} of every matrix's current diagonal block
  int *err = nullptr;
  int S = 0;
};

// Blocked Cholesky of `mats` (n x n, lower, in place, uniform stride when tc != nullptr), in step.
// inv_panel (tensor-core route, matrices whose diagonal blocks are well conditioned, such as
// I - L^H chi0 L >= I): the panel solve X L_pp^H = B as the product X = B L_pp^{-H} on the tensor
// cores, with L_pp^{-1} from the diagonal-block kernel; otherwise by substitution (FP64).
void potrf_batched(Handle &h, double2 *const *d_mats, const std::vector<double2 *> &mats, int n, int ld,
                   double *lndet, int *info, TcScratch *tc, bool inv_panel = false) {
  cudaStream_t s = h.stream;
  const int B = (int)mats.size();
  const size_t smem = (size_t)NB * (NB + 1) * sizeof(double2);
  const bool use_inv = tc && inv_panel && tc->inv;
  LR_CUDA(cudaFuncSetAttribute(k_potrf_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * smem)));
  LR_CUDA(cudaFuncSetAttribute(k_trsm_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * smem)));
  const long long bstride = B > 1 ? (long long)(mats[1] - mats[0]) : 0;
  for (int p0 = 0; p0 < n; p0 += NB) {
    const int nb = std::min(NB, n - p0), rest = n - p0 - nb;
    const bool inv_now = use_inv && rest > 0;
    k_potrf_diag<<<B, 256, inv_now ? 2 * smem : smem, s>>>(d_mats, n, ld, p0, lndet, info,
                                                          inv_now ? tc->inv : nullptr);
    ++launch_counter();
    if (rest <= 0) break;
    if (inv_now) {
      // X = B L_pp^{-H}: stacked real GEMM over the B matrices, K' = 2 nb, written over B
      double2 *P = mats[0] + (size_t)(p0 + nb) * ld + p0;
      oz::sliced_bind(tc->pa, tc->pa.digits, 2 * rest * B, 2 * nb, tc->S);
      oz::sliced_bind(tc->pi, tc->pi.digits, nb * B, 2 * nb, tc->S);
      oz::split_complex(P, ld, oz::OP_N, true, rest, nb, B, bstride, tc->pa, s);
      oz::split_complex(tc->inv, NB, oz::OP_H, false, nb, nb, B, (long long)NB * NB, tc->pi, s);
      oz::Out o;
      o.C = (double *)P;
      o.ldc = ld;
      o.batch_stride = bstride;
      o.mode = 1;
      o.alpha = 1.0;
      o.beta = 0.0;
      Handle::Timed tm{nullptr, nullptr, 8.0 * B * rest * 0.5 * nb * nb, 1};
      LR_CUDA(cudaEventCreate(&tm.a));
      LR_CUDA(cudaEventCreate(&tm.b));
      LR_CUDA(cudaEventRecord(tm.a, s));
      oz::gemm(tc->pa, tc->pi, 2 * rest, nb, B, o, 0, 0, 0, tc->err, s, h);
      LR_CUDA(cudaEventRecord(tm.b, s));
      h.timed.push_back(tm);
    } else {
      dim3 g((unsigned)((rest + 63) / 64), (unsigned)B);
      k_trsm_panel<<<g, 64, 2 * smem, s>>>(d_mats, n, ld, p0);
      ++launch_counter();
    }
    // algorithmic work: the lower triangle (with diagonal) of a rest x rest update of rank nb
    const double fl = 8.0 * B * (0.5 * rest * (rest + 1.0)) * nb;
    if (tc) {
      // A22 -= P P^H with P = A[p0+nb.., p0..p0+nb): stacked real GEMM, K' = 2 nb
      const double2 *P = mats[0] + (size_t)(p0 + nb) * ld + p0;
      oz::sliced_bind(tc->pa, tc->pa.digits, 2 * rest * B, 2 * nb, tc->S);
      oz::sliced_bind(tc->pb, tc->pb.digits, rest * B, 2 * nb, tc->S);
      oz::split_complex(P, ld, oz::OP_N, true, rest, nb, B, bstride, tc->pa, s);
      oz::split_complex(P, ld, oz::OP_H, false, rest, nb, B, bstride, tc->pb, s);
      oz::Out o;
      o.C = (double *)(mats[0] + (size_t)(p0 + nb) * ld + p0 + nb);
      o.ldc = ld;
      o.batch_stride = bstride;
      o.mode = 1;
      o.alpha = -1.0;
      o.beta = 1.0;
      Handle::Timed tm{nullptr, nullptr, fl, 1};
      LR_CUDA(cudaEventCreate(&tm.a));
      LR_CUDA(cudaEventCreate(&tm.b));
      LR_CUDA(cudaEventRecord(tm.a, s));
      oz::gemm(tc->pa, tc->pb, 2 * rest, rest, B, o, 0, 0, 2, tc->err, s, h);
      LR_CUDA(cudaEventRecord(tm.b, s));
      h.timed.push_back(tm);
      continue;
    }
    std::vector<ZGemm> batch;
    for (int b = 0; b < B; ++b) {
      ZGemm z{};
      double2 *M = mats[b];
      z.A = M + (size_t)(p0 + nb) * ld + p0;
      z.B = z.A;
      z.C = M + (size_t)(p0 + nb) * ld + p0 + nb;
      z.M = rest;
      z.N = rest;
      z.K = nb;
      z.lda = ld;
      z.ldb = ld;
      z.ldc = ld;
      z.alpha = make_double2(-1.0, 0.0);
      z.beta = make_double2(1.0, 0.0);
      batch.push_back(z);
    }
    ZGemmFlags f;
    f.transB = true;
    f.conjB = true;
    f.lower_only = true;
    zgemm_batched(batch, f, s, h, 1, fl);
  }
  LR_CUDA(cudaGetLastError());
}

// Batched real GEMMs (k_dgemm_tri) of one launch.  shape: 0 = every output tile, 1 = tiles on or
// above the diagonal (n0 >= m0), 2 = on or below (n0 <= m0); kfrom_row: K starts at the tile's
// first row (A zero left of its diagonal).  flops: algorithmic count for the stats.
void rgemm_batched(Handle &h, const std::vector<RGemm> &gs, int shape, bool kfrom_row, double flops) {
  constexpr int T = 64;
  std::vector<RTile> tiles;
  for (int e = 0; e < (int)gs.size(); ++e)
    for (int m0 = 0; m0 < gs[e].M; m0 += T)
      for (int n0 = 0; n0 < gs[e].N; n0 += T) {
        if ((shape == 1 && n0 < m0) || (shape == 2 && n0 > m0)) continue;
        tiles.push_back({e, m0, n0, kfrom_row ? m0 : 0});
      }
  if (tiles.empty()) return;
  const size_t b1 = gs.size() * sizeof(RGemm), b2 = tiles.size() * sizeof(RTile);
  const size_t off2 = (b1 + 255) / 256 * 256;
  static thread_local std::vector<char> host;
  host.resize(off2 + b2);
  std::memcpy(host.data(), gs.data(), b1);
  std::memcpy(host.data() + off2, tiles.data(), b2);
  h.ensure(h.rgemm_args, off2 + b2);
  cudaStream_t s = h.stream;
  LR_CUDA(cudaMemcpyAsync(h.rgemm_args.p, host.data(), off2 + b2, cudaMemcpyHostToDevice, s));
  const RGemm *dg = reinterpret_cast<const RGemm *>(h.rgemm_args.p);
  const RTile *dt = reinterpret_cast<const RTile *>((const char *)h.rgemm_args.p + off2);
  Handle::Timed tm{nullptr, nullptr, flops, 1};
  LR_CUDA(cudaEventCreate(&tm.a));
  LR_CUDA(cudaEventCreate(&tm.b));
  LR_CUDA(cudaEventRecord(tm.a, s));
  for (size_t t0 = 0; t0 < tiles.size(); t0 += 1u << 30) {
    const unsigned nb = (unsigned)std::min<size_t>(tiles.size() - t0, 1u << 30);
    k_dgemm_tri<<<nb, 128, 0, s>>>(dg, dt + t0);
    ++launch_counter();
  }
  LR_CUDA(cudaEventRecord(tm.b, s));
  h.timed.push_back(tm);
  LR_CUDA(cudaGetLastError());
}

// Blocked real Cholesky of `mats` (n x n, lower, in place), in step (as potrf_batched).
// Real blocked Cholesky (lower, in place).  tc (tensor-core route, uniform matrix stride): the
// trailing updates as digit-plane GEMMs; otherwise FP64 DMMA.
void potrf_batched_r(Handle &h, double *const *d_mats, const std::vector<double *> &mats, int n, int ld,
                     double *lndet, int *info, TcScratch *tc = nullptr) {
  cudaStream_t s = h.stream;
  const int B = (int)mats.size();
  const size_t smem = (size_t)NB * (NB + 1) * sizeof(double);
  LR_CUDA(cudaFuncSetAttribute(k_potrf_diag_r, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LR_CUDA(cudaFuncSetAttribute(k_trsm_panel_r, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * smem)));
  const long long bstride = B > 1 ? (long long)(mats[1] - mats[0]) : 0;
  for (int p0 = 0; p0 < n; p0 += NB) {
    k_potrf_diag_r<<<B, 256, smem, s>>>(d_mats, n, ld, p0, lndet, info);
    ++launch_counter();
    const int nb = std::min(NB, n - p0), rest = n - p0 - nb;
    if (rest <= 0) break;
    dim3 g((unsigned)((rest + 63) / 64), (unsigned)B);
    k_trsm_panel_r<<<g, 64, 2 * smem, s>>>(d_mats, n, ld, p0);
    ++launch_counter();
    const double fl = 2.0 * B * (0.5 * rest * (rest + 1.0)) * nb;
    if (tc) {
      // A22 -= P P^T on the lower tiles, P = A[p0+nb.., p0..p0+nb): one operand in both roles
      const double *P = mats[0] + (size_t)(p0 + nb) * ld + p0;
      oz::sliced_bind(tc->pa, tc->pa.digits, rest * B, nb, tc->S);
      oz::split_real(P, ld, false, rest, nb, B, bstride, tc->pa, s);
      oz::Out o;
      o.C = mats[0] + (size_t)(p0 + nb) * ld + p0 + nb;
      o.ldc = ld;
      o.batch_stride = bstride;
      o.mode = 0;
      o.alpha = -1.0;
      o.beta = 1.0;
      Handle::Timed tm{nullptr, nullptr, fl, 1};
      LR_CUDA(cudaEventCreate(&tm.a));
      LR_CUDA(cudaEventCreate(&tm.b));
      LR_CUDA(cudaEventRecord(tm.a, s));
      oz::gemm(tc->pa, tc->pa, rest, rest, B, o, 0, 0, 1, tc->err, s, h);
      LR_CUDA(cudaEventRecord(tm.b, s));
      tm.exec_flops = h.oz_exec_flops;
      h.timed.push_back(tm);
      continue;
    }
    // A22 -= P P^T on the lower tiles, P = A[p0+nb.., p0..p0+nb)
    std::vector<RGemm> batch;
    for (int b = 0; b < B; ++b) {
      double *M = mats[b];
      const double *P = M + (size_t)(p0 + nb) * ld + p0;
      batch.push_back(RGemm{P, P, M + (size_t)(p0 + nb) * ld + p0 + nb, rest, rest, nb, ld, ld, ld, -1.0, 1.0});
    }
    rgemm_batched(h, batch, 2, false, fl);
  }
  LR_CUDA(cudaGetLastError());
}

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// Workspace of the ln det stage: L[nq], W[nw], A[nw] (complex n x n), pointer tables,
// lndet/trace/info, output, and for the tensor-core route the digit planes.
struct EcLayout {
  size_t o_L, o_W, o_A, o_ptr, o_ld, o_tr, o_ldc, o_trc, o_inf, o_out, o_wo, o_wq, o_err;
  size_t o_sx = 0, o_sw = 0, o_sl = 0, o_slh = 0, o_pa = 0, o_pb = 0, o_inv = 0, o_pi = 0;
  size_t total = 0;
};

// q points factorised together: the q <= -q of the mesh (all q are computed in chunks of this
// size when V(q) turns out not to pair)
int ec_chunk(const Handle &h) {
  int c = 0;
  for (int q = 0; q < h.mesh.size(); ++q) c += q <= h.mesh.neg(q);
  return c;
}

EcLayout ec_layout(const Handle &h) {
  const int n = h.naux, nq = h.mesh.size(), nw = h.ntau, S = h.ec_S, nc = ec_chunk(h);
  const size_t n2 = (size_t)n * n, mat = n2 * sizeof(double2);
  const int bmax = std::max(nq, nc * nw);
  EcLayout l;
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += al256(bytes); return o; };
  l.o_L = take(nq * mat);
  l.o_W = take(nw * mat);
  l.o_A = take((size_t)nc * nw * mat);   // the (q, omega) of a chunk are factorised in one batch
  l.o_ptr = take(((size_t)nq + (size_t)nc * nw + 8) * 8);
  l.o_ld = take(((size_t)nq * nw + nq) * 8);
  l.o_tr = take((size_t)nq * nw * 8);
  l.o_ldc = take((size_t)nq * nw * 8);
  l.o_trc = take((size_t)nq * nw * 8);
  l.o_inf = take((size_t)(nq + nq * nw) * 4);
  l.o_out = take((size_t)(1 + nq + nw) * 8);
  l.o_wo = take((size_t)nw * 8);
  l.o_wq = take((size_t)nq * 8);
  l.o_err = take(4);
  if (S >= 0) {
    l.o_sx = take(oz::sliced_bytes(nw * 2 * n, 2 * n, S));
    l.o_sw = take(oz::sliced_bytes(nw * n, 2 * n, S));
    l.o_sl = take(oz::sliced_bytes(n, 2 * n, S));
    l.o_slh = take(oz::sliced_bytes(2 * n, 2 * n, S));
    l.o_pa = take(oz::sliced_bytes(bmax * 2 * n, 2 * NB, S));
    l.o_pb = take(oz::sliced_bytes(bmax * n, 2 * NB, S));
    l.o_inv = take((size_t)bmax * NB * NB * sizeof(double2));
    l.o_pi = take(oz::sliced_bytes(bmax * NB, 2 * NB, S));
  }
  l.total = off;
  return l;
}

}  // namespace

size_t ec_work_bytes(const Handle &h) { return ec_layout(h).total; }

int ec_run(Handle &h, double *ec, double *ec_q, double *ec_w) {
  const int n = h.naux, nq = h.mesh.size(), nw = h.ntau, S = h.ec_S;
  const size_t n2 = (size_t)n * n;
  cudaStream_t s = h.stream;
  const size_t mat = n2 * sizeof(double2);
  const int nc = ec_chunk(h), bmax = std::max(nq, nc * nw);
  const EcLayout lay = ec_layout(h);
  const size_t o_L = lay.o_L, o_W = lay.o_W, o_A = lay.o_A, o_ptr = lay.o_ptr, o_ld = lay.o_ld, o_tr = lay.o_tr,
               o_inf = lay.o_inf, o_out = lay.o_out, o_wo = lay.o_wo, o_err = lay.o_err, o_sx = lay.o_sx,
               o_sw = lay.o_sw, o_sl = lay.o_sl, o_slh = lay.o_slh, o_pa = lay.o_pa, o_pb = lay.o_pb;
  h.ensure(h.work, lay.total);
  char *w = (char *)h.work.p;
  double2 *Lq = (double2 *)(w + o_L), *Wm = (double2 *)(w + o_W), *Am = (double2 *)(w + o_A);
  double2 **ptrs = (double2 **)(w + o_ptr);
  double *lndet = (double *)(w + o_ld), *trace = (double *)(w + o_tr), *out = (double *)(w + o_out);
  double *wo = (double *)(w + o_wo);
  int *info = (int *)(w + o_inf);
  int *err = (int *)(w + o_err);
  double *lndet_v = lndet + (size_t)nq * nw;   // scratch for the V(q) factorisations
  LR_CUDA(cudaMemsetAsync(lndet, 0, ((size_t)nq * nw + nq) * 8, s));
  LR_CUDA(cudaMemsetAsync(info, 0, (size_t)(nq + nq * nw) * 4, s));
  LR_CUDA(cudaMemsetAsync(err, 0, 4, s));
  LR_CUDA(cudaMemcpyAsync(wo, h.w_omega.data(), (size_t)nw * 8, cudaMemcpyHostToDevice, s));
  // per-q weights of the q sum (set_q_weights), else 1 / N_q; q of zero weight are not computed
  const bool weighted = !h.wq.empty();
  double *wqd = weighted ? (double *)(w + lay.o_wq) : nullptr;
  if (weighted) LR_CUDA(cudaMemcpyAsync(wqd, h.wq.data(), (size_t)nq * 8, cudaMemcpyHostToDevice, s));
  auto weight = [&](int q) { return weighted ? h.wq[q] : 1.0; };
  TcScratch tcs;
  TcScratch *tc = nullptr;
  oz::Sliced sx, sw, sl, slh;
  if (S >= 0) {
    tcs.S = S;
    tcs.err = err;
    oz::sliced_bind(tcs.pa, w + o_pa, bmax * 2 * n, 2 * NB, S);
    oz::sliced_bind(tcs.pb, w + o_pb, bmax * n, 2 * NB, S);
    oz::sliced_bind(tcs.pi, w + lay.o_pi, bmax * NB, 2 * NB, S);
    tcs.inv = (double2 *)(w + lay.o_inv);
    oz::sliced_bind(sx, w + o_sx, nw * 2 * n, 2 * n, S);
    oz::sliced_bind(sw, w + o_sw, nw * n, 2 * n, S);
    oz::sliced_bind(sl, w + o_sl, n, 2 * n, S);
    oz::sliced_bind(slh, w + o_slh, 2 * n, 2 * n, S);
    tc = &tcs;
  }
  // q <-> -q: chi0(R) is real, so chi0(-q) = conj chi0(q); when also V(-q) = conj V(q) (to 1e-12
  // of max |V|), the integrand of -q equals that of q (ln det and trace of complex-conjugate
  // matrices), and only q <= -q is computed.  The check runs once per set of V(q).
  // The same check gives the real route (section above) its condition: V(q) real at q = -q.
  if (h.vq_sym < 0 || h.vq_real < 0) {
    // 24 bytes at lndet (its region is at least 256 bytes long; it is cleared again below)
    unsigned long long *res = (unsigned long long *)(w + o_ld);
    LR_CUDA(cudaMemsetAsync(res, 0, 24, s));
    k_conj_check<<<dim3(64, (unsigned)nq), 256, 0, s>>>((const double2 *)h.d_vq.p, n, h.mesh.n1, h.mesh.n2,
                                                        h.mesh.n3, res);
    ++launch_counter();
    LR_CUDA(cudaGetLastError());
    double dm[3] = {0, 0, 0};
    LR_CUDA(cudaMemcpyAsync(dm, res, 24, cudaMemcpyDeviceToHost, s));
    LR_CUDA(cudaStreamSynchronize(s));
    h.vq_sym = dm[0] <= 1e-12 * dm[1] ? 1 : 0;
    h.vq_real = dm[2] <= 1e-12 * dm[1] ? 1 : 0;
    LR_CUDA(cudaMemsetAsync(lndet, 0, 24, s));
  }
  std::vector<int> qlist;
  for (int q = 0; q < nq; ++q) {
    const int p = h.mesh.neg(q);
    if (h.vq_sym == 1 ? q <= p && (weight(q) > 0 || weight(p) > 0) : weight(q) > 0) qlist.push_back(q);
  }
  const int nql = (int)qlist.size();
  // positions in qlist, the complex ones first, then those of the real route: the per-(q, omega)
  // ln det and trace are kept in this order until the end
  std::vector<int> order;
  auto real_q = [&](int q) { return h.vq_real == 1 && q == h.mesh.neg(q); };
  for (int qi = 0; qi < nql; ++qi)
    if (!real_q(qlist[qi])) order.push_back(qi);
  const int nx = (int)order.size();
  for (int qi = 0; qi < nql; ++qi)
    if (real_q(qlist[qi])) order.push_back(qi);
  // Cholesky of every V(q) computed, packed in qlist order (the batched factorisation needs a
  // uniform stride)
  std::vector<double2 *> lp(nql);
  for (int i = 0; i < nql; ++i) {
    lp[i] = Lq + (size_t)i * n2;
    LR_CUDA(cudaMemcpyAsync(lp[i], (const char *)h.d_vq.p + (size_t)qlist[i] * mat, mat, cudaMemcpyDeviceToDevice, s));
  }
  LR_CUDA(cudaMemcpyAsync(ptrs, lp.data(), nql * 8, cudaMemcpyHostToDevice, s));
  potrf_batched(h, ptrs, lp, n, n, lndet_v, info, tc);
  {
    dim3 g((unsigned)((n2 + 255) / 256), (unsigned)nql);
    k_zero_upper<<<g, 256, 0, s>>>(ptrs, n, n);
    ++launch_counter();
  }
  const double2 *chi = (const double2 *)h.d_chi_qw.p;
  // A(q, omega) of the q of a chunk, packed: A[(pos - c0) * nw + k]; each chunk is factorised in
  // one lockstep batch
  double2 **aptr = ptrs + nq;
  double *lndet_c = (double *)(w + lay.o_ldc), *trace_c = (double *)(w + lay.o_trc);
  LR_CUDA(cudaMemsetAsync(lndet_c, 0, (size_t)nql * nw * 8, s));
  // algorithmic work (8 flops per complex MAC): A = -L^H W on the lower triangle,
  // sum_{i >= j} (n - i) MACs per matrix
  const double dn = n;
  const double fl_a = 8.0 * nw * (dn * (dn + 1) * (dn + 2) / 6);
  // A needs W only on and below its diagonal tiles (j >= k), sum_k (n - k)^2 MACs
  const double fl_w_lower = 8.0 * nw * (dn * (dn + 1) * (2 * dn + 1) / 6);
  for (int c0 = 0; c0 < nx; c0 += nc) {
    const int c1 = std::min(nx, c0 + nc);
    std::vector<double2 *> ap((size_t)(c1 - c0) * nw);
    for (size_t b = 0; b < ap.size(); ++b) ap[b] = Am + b * n2;
    LR_CUDA(cudaMemcpyAsync(aptr, ap.data(), ap.size() * 8, cudaMemcpyHostToDevice, s));
    for (int pos = c0; pos < c1; ++pos) {
      const int qi = order[pos], q = qlist[qi];
      double2 *Aq = Am + (size_t)(pos - c0) * nw * n2;
      if (S >= 0) {
        const double2 *L = Lq + (size_t)qi * n2;
        oz::split_complex(L, n, oz::OP_N, false, n, n, 1, 0, sl, s);     // B'^T of W = chi0 L
        oz::split_complex(L, n, oz::OP_H, true, n, n, 1, 0, slh, s);     // A' of L^H W
        oz::split_complex(chi + (size_t)q * nw * n2, n, oz::OP_N, true, n, n, nw, (long long)n2, sx, s);
        // W^T, so that the second GEMM reads W column by column as rows.  A = -L^H W reads W only on
        // and below its diagonal tiles (k >= j): the tiles above are not computed and stay zero
        // (the digit planes of W's rows see zeros there)
        LR_CUDA(cudaMemsetAsync(Wm, 0, (size_t)nw * mat, s));
        oz::Out o1;
        o1.C = (double *)Wm;
        o1.ldc = n;
        o1.batch_stride = (long long)n2;
        o1.mode = 2;
        Handle::Timed t1{nullptr, nullptr, fl_w_lower, 1};
        LR_CUDA(cudaEventCreate(&t1.a));
        LR_CUDA(cudaEventCreate(&t1.b));
        LR_CUDA(cudaEventRecord(t1.a, s));
        oz::gemm(sx, sl, 2 * n, n, nw, o1, 0, 2, 2, err, s, h);
        LR_CUDA(cudaEventRecord(t1.b, s));
        t1.exec_flops = h.oz_exec_flops;
        h.timed.push_back(t1);
        oz::split_complex(Wm, n, oz::OP_T, false, n, n, nw, (long long)n2, sw, s);   // B'^T rows j: W[k][j]
        oz::Out o2;
        o2.C = (double *)Aq;
        o2.ldc = n;
        o2.batch_stride = (long long)n2;
        o2.mode = 1;
        o2.alpha = -1.0;
        Handle::Timed t2{nullptr, nullptr, fl_a, 1};
        LR_CUDA(cudaEventCreate(&t2.a));
        LR_CUDA(cudaEventCreate(&t2.b));
        LR_CUDA(cudaEventRecord(t2.a, s));
        oz::gemm(slh, sw, 2 * n, n, nw, o2, 1, 0, 2, err, s, h);
        LR_CUDA(cudaEventRecord(t2.b, s));
        t2.exec_flops = h.oz_exec_flops;
        h.timed.push_back(t2);
      } else {
        // W = chi0(q, omega) L_q  (L lower triangular: k >= j)
        std::vector<ZGemm> b1, b2;
        for (int k = 0; k < nw; ++k) {
          ZGemm z{};
          z.A = chi + ((size_t)q * nw + k) * n2;
          z.B = Lq + (size_t)qi * n2;
          z.C = Wm + k * n2;
          z.M = z.N = z.K = n;
          z.lda = z.ldb = z.ldc = n;
          z.alpha = make_double2(1.0, 0.0);
          z.beta = make_double2(0.0, 0.0);
          b1.push_back(z);
          ZGemm y{};
          y.A = Lq + (size_t)qi * n2;     // op(A) = L^H: stored [K][M], conjugated
          y.B = Wm + k * n2;
          y.C = Aq + k * n2;
          y.M = y.N = y.K = n;
          y.lda = y.ldb = y.ldc = n;
          y.alpha = make_double2(-1.0, 0.0);
          y.beta = make_double2(0.0, 0.0);
          b2.push_back(y);
        }
        ZGemmFlags f1;
        f1.kfrom = 2;
        f1.lower_only = true;   // the second GEMM reads W only on and below the diagonal tiles
        zgemm_batched(b1, f1, s, h, 1, fl_w_lower);
        ZGemmFlags f2;
        f2.transA = true;
        f2.conjA = true;
        f2.kfrom = 1;
        f2.lower_only = true;
        zgemm_batched(b2, f2, s, h, 1, fl_a);
      }
    }
    // A = I - L^H chi0 L of the chunk's (q, omega): trace, then one lockstep Cholesky of all
    k_diag_shift<<<(unsigned)ap.size(), 256, 0, s>>>(aptr, n, n, trace_c + (size_t)c0 * nw);
    ++launch_counter();
    potrf_batched(h, aptr, ap, n, n, lndet_c + (size_t)c0 * nw, info + nq + (size_t)c0 * nw, tc, true);
  }
  if (nql > nx) {
    // real route, all its (q, omega) in one lockstep batch, in the A region (real matrices take
    // half the room of complex ones): Ar[B] then Lt; W's region holds Re chi0 and W^T of one q
    const int nr = nql - nx;
    const size_t B = (size_t)nr * nw;
    double *Ar = (double *)Am, *Lt = Ar + B * n2;
    double *Xr = (double *)Wm, *WT = Xr + (size_t)nw * n2;
    std::vector<double *> ar(B);
    for (size_t b = 0; b < B; ++b) ar[b] = Ar + b * n2;
    double **rptr = reinterpret_cast<double **>(aptr);
    LR_CUDA(cudaMemcpyAsync(rptr, ar.data(), B * 8, cudaMemcpyHostToDevice, s));
    const unsigned nt = (unsigned)((n + 31) / 32);
    for (int r = 0; r < nr; ++r) {
      const int qi = order[nx + r], q = qlist[qi];
      k_real_transpose<<<dim3(nt, nt), dim3(32, 8), 0, s>>>(Lq + (size_t)qi * n2, n, Lt);
      const size_t cnt = (size_t)nw * n2;
      k_real_part<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(chi + (size_t)q * nw * n2, cnt, Xr);
      launch_counter() += 2;
      LR_CUDA(cudaGetLastError());
      if (S >= 0) {
        // W = Xr L on and below the diagonal tiles (W[k][j] = sum_l Xr[k][l] Lt[j][l], l >= j; the
        // tiles above stay zero), then A = -L^T W = -(Lt rows) . (W^T rows), l >= i, lower tiles
        double *Wr = WT;
        LR_CUDA(cudaMemsetAsync(Wr, 0, (size_t)nw * n2 * sizeof(double), s));
        oz::Sliced slt = sl, sxr = sx, swt = sw;
        oz::sliced_bind(slt, sl.digits, n, n, S);
        oz::sliced_bind(sxr, sx.digits, nw * n, n, S);
        oz::sliced_bind(swt, sw.digits, nw * n, n, S);
        oz::split_real(Lt, n, false, n, n, 1, 0, slt, s);
        oz::split_real(Xr, n, false, n, n, nw, (long long)n2, sxr, s);
        oz::Out o1;
        o1.C = Wr;
        o1.ldc = n;
        o1.batch_stride = (long long)n2;
        o1.mode = 0;
        Handle::Timed t1{nullptr, nullptr, fl_w_lower / 4, 1};
        LR_CUDA(cudaEventCreate(&t1.a));
        LR_CUDA(cudaEventCreate(&t1.b));
        LR_CUDA(cudaEventRecord(t1.a, s));
        oz::gemm(sxr, slt, n, n, nw, o1, 0, 1, 1, err, s, h);
        LR_CUDA(cudaEventRecord(t1.b, s));
        t1.exec_flops = h.oz_exec_flops;
        h.timed.push_back(t1);
        oz::split_real(Wr, n, true, n, n, nw, (long long)n2, swt, s);
        oz::Out o2;
        o2.C = Ar + (size_t)r * nw * n2;
        o2.ldc = n;
        o2.batch_stride = (long long)n2;
        o2.mode = 0;
        o2.alpha = -1.0;
        Handle::Timed t2{nullptr, nullptr, fl_a / 4, 1};
        LR_CUDA(cudaEventCreate(&t2.a));
        LR_CUDA(cudaEventCreate(&t2.b));
        LR_CUDA(cudaEventRecord(t2.a, s));
        oz::gemm(slt, swt, n, n, nw, o2, 1, 0, 1, err, s, h);
        LR_CUDA(cudaEventRecord(t2.b, s));
        t2.exec_flops = h.oz_exec_flops;
        h.timed.push_back(t2);
        continue;
      }
      // W^T = Lt Xr^T (= (chi0 L)^T) on and above the diagonal tiles; A = -Lt (W^T)^T = -L^T W on
      // and below them; Lt is upper triangular, so K starts at the tile's first row
      std::vector<RGemm> g1, g2;
      for (int k = 0; k < nw; ++k) {
        g1.push_back(RGemm{Lt, Xr + (size_t)k * n2, WT + (size_t)k * n2, n, n, n, n, n, n, 1.0, 0.0});
        g2.push_back(RGemm{Lt, WT + (size_t)k * n2, Ar + ((size_t)r * nw + k) * n2, n, n, n, n, n, n, -1.0, 0.0});
      }
      rgemm_batched(h, g1, 1, true, fl_w_lower / 4);
      rgemm_batched(h, g2, 2, true, fl_a / 4);
    }
    k_diag_shift_r<<<(unsigned)B, 256, 0, s>>>(rptr, n, n, trace_c + (size_t)nx * nw);
    ++launch_counter();
    potrf_batched_r(h, rptr, ar, n, n, lndet_c + (size_t)nx * nw, info + nq + (size_t)nx * nw, tc);
  }
  for (int pos = 0; pos < nql; ++pos) {   // to the flat (q, omega) order
    const int q = qlist[order[pos]];
    LR_CUDA(cudaMemcpyAsync(lndet + (size_t)q * nw, lndet_c + (size_t)pos * nw, nw * 8, cudaMemcpyDeviceToDevice, s));
    LR_CUDA(cudaMemcpyAsync(trace + (size_t)q * nw, trace_c + (size_t)pos * nw, nw * 8, cudaMemcpyDeviceToDevice, s));
  }
  for (int q : qlist) {   // the integrands of -q
    const int p = h.mesh.neg(q);
    if (p == q || h.vq_sym != 1) continue;
    LR_CUDA(cudaMemcpyAsync(lndet + (size_t)p * nw, lndet + (size_t)q * nw, nw * 8, cudaMemcpyDeviceToDevice, s));
    LR_CUDA(cudaMemcpyAsync(trace + (size_t)p * nw, trace + (size_t)q * nw, nw * 8, cudaMemcpyDeviceToDevice, s));
  }
  k_energy<<<1, 1, 0, s>>>(lndet, trace, wo, wqd, nq, nw, out);
  ++launch_counter();
  LR_CUDA(cudaGetLastError());
  std::vector<double> res(1 + nq + nw);
  std::vector<int> inf(nq + (size_t)nq * nw);
  int e_host = 0;
  LR_CUDA(cudaMemcpyAsync(res.data(), out, res.size() * 8, cudaMemcpyDeviceToHost, s));
  LR_CUDA(cudaMemcpyAsync(inf.data(), info, inf.size() * 4, cudaMemcpyDeviceToHost, s));
  LR_CUDA(cudaMemcpyAsync(&e_host, err, 4, cudaMemcpyDeviceToHost, s));
  LR_CUDA(cudaStreamSynchronize(s));
  if (e_host) return LIBRPA_E_TIMEOUT;
  for (int v : inf)
    if (v) return LIBRPA_E_NOT_PD;
  *ec = res[0];
  if (ec_q)
    for (int q = 0; q < nq; ++q) ec_q[q] = res[1 + q];
  if (ec_w)
    for (int k = 0; k < nw; ++k) ec_w[k] = res[1 + nq + k];
  // flop count of this stage (complex MAC = 8 real flops, real MAC = 2): per q (4/3 n^3 real for
  // the Cholesky of V), per (q, omega): W = chi0 L on the tiles A needs (n^3/3 MAC), L^H W lower
  // (n^3/6 MAC), Cholesky (n^3/6 MAC)
  const double n3 = (double)n * n * n;
  const double macs = n3 / 3 + n3 / 6 + n3 / 6;
  h.stats.flop_ec = nql * (8.0 * n3 / 6.0) + (double)nx * nw * 8.0 * macs + (double)(nql - nx) * nw * 2.0 * macs;
  return LIBRPA_OK;
}

}  // namespace librpa
