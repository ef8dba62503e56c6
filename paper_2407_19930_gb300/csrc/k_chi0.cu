// K2: chi0_{mu nu}(R, tau) by the atom-pair contraction of Algorithm 1 (Sec. 2).
//
// Per (R, tau) point, with A = G^vir (the paper's G(i tau)) and B = G^occ (G(-i tau)):
//
//   N^{B,nu}_{jk}(K R1) = sum_{(L,R2') in N[V]} sum_l C[V,L,R2']_{nu j l} B_{lk}(R1 - R - R2')
//   X^{A,nu}_{ij}       = sum_{(L,R2') in N[V]} sum_l C[V,L,R2']_{nu j l} A_{il}(R + R2')
//   O^nu_{ik}(K R1)     = sum_{j in V} A_ij(R) N^{B,nu}_jk + B_ij(R) N^{A,nu}_jk
//                                  + B_jk(R1 - R) X^{A,nu}_ij + A_jk(R1 - R) X^{B,nu}_ij
//   chi0_{mu nu}(R, tau) = -s sum_{(K,R1) in N[U]} sum_{ik} C[U,K,R1]_{mu i k} O^nu_{ik}(K R1)
//
// i.e. Algorithm 1's M + M*(-i tau) + Z + Z*(-i tau) with the paper's -i factors taken out
// (real convention: G(i tau) = +i G^vir, G(-i tau) = -i G^occ).  Two exact restructurings
// of the loop nest: N depends on (V, R, K R1) but not on U, so it is computed once per V for
// every (K, R1) in the union of all N[U]; X depends on (V, R) only, so it is computed once
// per V for every NAO i of the home cell.  All contractions are then dense GEMMs:
//
//   N-step  (per V, per G):  N_V = Cpack_V [n_aux_V n_V x m_V]  .  Bg_V^T  [m_V x M_all]
//   X-step  (per V, per G):  X_V = Ag_V [n_ao x m_V]            .  Cpack_V^T [m_V x n_aux_V n_V]
//   final   (per U):         chi0[U rows] = -s Cpack_U [n_aux_U x n_U m_U] . O_U^T [n_U m_U x N_aux]
//
// where Cpack_U[mu][i][(K,R1,k)] packs the blocks C[U,K,R1] side by side, Bg_V and Ag_V are
// G blocks gathered at the lattice vectors above, and O_U[nu][(i,(K,R1,k))] is assembled by a
// dedicated kernel.  The GEMMs run on the FP64 tensor cores (mma.sync m8n8k4 .f64).
#include <algorithm>
#include <cstring>
#include <functional>
#include <set>
#include <vector>

#include "internal.h"
#include "ozgemm.h"

namespace librpa {
namespace {

// ---------------------------------------------------------------------------------------
// batched FP64 "NT" GEMM on the tensor cores: C[m][n] = alpha sum_k A[m][k] B[n][k] + beta C
struct DGemm {
  const double *A, *B;
  double *C;
  int M, N, K, lda, ldb, ldc;
  double alpha, beta;
};
// An output tile; c_n >= 0: only the K chunks (of GK) listed at chunks[c_off .. + c_n) are summed
// (block-sparse operands under Green's-function screening: the others multiply exact zeros).
struct DTile {
  int e, m0, n0, c_off, c_n;
};

constexpr int GK = 16, GPAD = GK + 1;

__device__ __forceinline__ void dmma_m8n8k4(double &c0, double &c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

// CTA tile (32 WM) x (32 WN), one 32 x 32 warp tile per warp, K staged 16 at a time through
// shared memory.  Every variant accumulates each output element over K in the same order
// (chunks of 16, m8n8k4 steps of 4), so the tile shape never changes the result.
template <int WM, int WN>
__global__ void __launch_bounds__(32 * WM * WN) k_dgemm_nt(const DGemm *__restrict__ gs,
                                                           const DTile *__restrict__ tiles,
                                                           const int *__restrict__ chunks) {
  constexpr int BM = 32 * WM, BN = 32 * WN, NT = 32 * WM * WN;
  const DTile t = tiles[blockIdx.x];
  const DGemm g = gs[t.e];
  __shared__ double As[BM][GPAD];
  __shared__ double Bs[BN][GPAD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp / WN, wn = warp % WN;
  const int gid = lane >> 2, tig = lane & 3;
  double acc[4][4][2];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c][0] = acc[r][c][1] = 0.0;
  const int nch = t.c_n < 0 ? (g.K + GK - 1) / GK : t.c_n;
  for (int ci = 0; ci < nch; ++ci) {
    const int k0 = (t.c_n < 0 ? ci : chunks[t.c_off + ci]) * GK;
#pragma unroll
    for (int e = tid; e < BM * GK; e += NT) {
      const int row = e / GK, k = e % GK, gm = t.m0 + row, gk = k0 + k;
      As[row][k] = (gm < g.M && gk < g.K) ? g.A[(size_t)gm * g.lda + gk] : 0.0;
    }
#pragma unroll
    for (int e = tid; e < BN * GK; e += NT) {
      const int row = e / GK, k = e % GK, gn = t.n0 + row, gk = k0 + k;
      Bs[row][k] = (gn < g.N && gk < g.K) ? g.B[(size_t)gn * g.ldb + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; kk += 4) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[wm * 32 + r * 8 + gid][kk + tig];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[wn * 32 + c * 8 + gid][kk + tig];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) dmma_m8n8k4(acc[r][c][0], acc[r][c][1], a[r], b[c]);
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
      for (int h = 0; h < 2; ++h) {
        const int gn = t.n0 + wn * 32 + c * 8 + tig * 2 + h;
        if (gn >= g.N) continue;
        double *p = g.C + (size_t)gm * g.ldc + gn;
        const double v = g.alpha * acc[r][c][h];
        *p = g.beta == 0.0 ? v : v + g.beta * *p;
      }
  }
}

// tile variants {WM, WN}: 64x64 first (the default before tuning)
constexpr int kNumVariants = 5;
constexpr int kVarWM[kNumVariants] = {2, 1, 2, 1, 4};
constexpr int kVarWN[kNumVariants] = {2, 2, 1, 1, 2};

void launch_dgemm_variant(int v, unsigned ntiles, const DGemm *g, const DTile *t, const int *c, cudaStream_t s) {
  switch (v) {
    case 0: k_dgemm_nt<2, 2><<<ntiles, 128, 0, s>>>(g, t, c); break;
    case 1: k_dgemm_nt<1, 2><<<ntiles, 64, 0, s>>>(g, t, c); break;
    case 2: k_dgemm_nt<2, 1><<<ntiles, 64, 0, s>>>(g, t, c); break;
    case 3: k_dgemm_nt<1, 1><<<ntiles, 32, 0, s>>>(g, t, c); break;
    default: k_dgemm_nt<4, 2><<<ntiles, 256, 0, s>>>(g, t, c); break;
  }
}

// K chunks a tile of entry e must sum: chunk_fn(e, m0, rows, n0, cols, chunk size, K, out) appends the
// needed chunk indices (ascending) and returns true, or returns false for every chunk.
using ChunkFn = std::function<bool(int, int, int, int, int, int, int, std::vector<int> &)>;

// ---------------------------------------------------------------------------------------
// gathers.  Column tables hold 6 ints per column: {atom, R0, R1, R2, orbital, ao(atom)+orbital}.
struct Point {
  int iR, itau;
  int R[3];
};

// G of the spin channel being contracted ([spin][g][tau][R][i][j]) and the spin factor of chi0 per
// channel: 2 for the single unpolarised channel, 1 per channel when nspins = 2 (chi0 = sum over
// channels; the second channel's final GEMM accumulates, beta = 1)
const double *g_spin(const Handle &h) {
  return (const double *)h.d_g.p + (size_t)h.cur_spin * 2 * h.ntau * h.mesh.size() * h.nao * h.nao;
}
double spin_factor(const Handle &h) { return h.nspins == 1 ? 2.0 : 1.0; }

// Bg[p][g][V][kappa][lambda] = G^g(tau_p)[bvk(R1_kappa - R_p - R2'_lambda)][ao_lambda][ao_kappa]
__global__ void k_gather_bg(const double *__restrict__ G, size_t g_gstride, const Point *__restrict__ pts,
                            const int *__restrict__ uni, const int *__restrict__ lam, const long long *lam_off,
                            const int *m, const long long *bg_off, int natoms, int m_all, int nR_stride,
                            int nao, int n1, int n2, int n3, long long bg_sz_g, long long bg_sz_p, double *Bg) {
  const int V = blockIdx.y % natoms;
  const int g = (blockIdx.y / natoms) % 2;
  const int p = blockIdx.y / (2 * natoms);
  const int mV = m[V];
  const long long n = (long long)m_all * mV;
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  const int kap = (int)(x / mV), l = (int)(x % mV);
  const int *u = uni + 6 * kap;
  const int *c = lam + 6 * (lam_off[V] + l);
  const Point pt = pts[p];
  auto fold = [](int a, int nn) { int r = a % nn; return r < 0 ? r + nn : r; };
  const int iR = (fold(u[1] - pt.R[0] - c[1], n1) * n2 + fold(u[2] - pt.R[1] - c[2], n2)) * n3 +
                 fold(u[3] - pt.R[2] - c[3], n3);
  const double *Gp = G + g * g_gstride + ((size_t)pt.itau * nR_stride + iR) * nao * nao;
  Bg[p * bg_sz_p + g * bg_sz_g + bg_off[V] + x] = Gp[(size_t)c[5] * nao + u[5]];
}

// Ag[p][g][V][i][lambda] = G^g(tau_p)[bvk(R_p + R2'_lambda)][i][ao_lambda]
__global__ void k_gather_ag(const double *__restrict__ G, size_t g_gstride, const Point *__restrict__ pts,
                            const int *__restrict__ lam, const long long *lam_off, const int *m,
                            const long long *ag_off, int natoms, int nR_stride, int nao, int n1, int n2, int n3,
                            long long ag_sz_g, long long ag_sz_p, double *Ag) {
  const int V = blockIdx.y % natoms;
  const int g = (blockIdx.y / natoms) % 2;
  const int p = blockIdx.y / (2 * natoms);
  const int mV = m[V];
  const long long n = (long long)nao * mV;
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  const int i = (int)(x / mV), l = (int)(x % mV);
  const int *c = lam + 6 * (lam_off[V] + l);
  const Point pt = pts[p];
  auto fold = [](int a, int nn) { int r = a % nn; return r < 0 ? r + nn : r; };
  const int iR = (fold(pt.R[0] + c[1], n1) * n2 + fold(pt.R[1] + c[2], n2)) * n3 + fold(pt.R[2] + c[3], n3);
  const double *Gp = G + g * g_gstride + ((size_t)pt.itau * nR_stride + iR) * nao * nao;
  Ag[p * ag_sz_p + g * ag_sz_g + ag_off[V] + x] = Gp[(size_t)i * nao + c[5]];
}

// ---------------------------------------------------------------------------------------
// O assembly: O^nu_{ik}(K R1) for every (point, U, V), written as O_U[nu][(i, kap)].
struct OArgs {
  const double *G;       // [2][ntau][nR][nao][nao]
  size_t g_gstride;
  int nR_stride, nao, natoms, naux, n1, n2, n3;
  const Point *pts;
  const int *n_ao, *n_aux, *ao_off, *aux_off, *m;
  const int *kap;            // per-U column table {K, R0, R1, R2, ao(K)+k, union column}
  const long long *kap_off;
  const double *N;           // [P][2][sum_V n_aux_V n_V M_all]
  const long long *n_off;
  long long n_sz_g, n_sz_p;
  int m_all;
  const double *X;           // [P][2][sum_V nao n_aux_V n_V]
  const long long *x_off;
  long long x_sz_g, x_sz_p;
  double *O;                 // [P][sum_U naux n_U m_U]
  const long long *o_off;
  long long o_sz_p;
  // under screening: 1 where the CTA's O block is exactly zero ([P][U][V][64-column chunk]), else NULL
  const unsigned char *zero;
  // 3-plane tensor-core kernel: the row exponents of O's digit planes (rows (p, U, nu); atomicMax
  // of the largest biased FP64 exponent minus 1022), or NULL
  int *rexp;
};

// Arithmetic of the O assembly.  ArD: FP64 (FP64 modes).  ArF: FP32, for the mixed modes whose
// contraction GEMMs keep at most ~23 bits.  ArDF: unevaluated sums of two FP32 numbers (about 48
// significant bits; the product of the high parts split exactly with an FMA, sums by Knuth's
// two-sum) for the FP64-accurate tensor-core mode: it runs on the FP32 pipe, whose rate on GB300
// is ~70x that of the FP64 pipe.
struct ArD {
  using T = double;
  __device__ static T from(double x) { return x; }
  __device__ static T load(const double *p) { return *p; }
  __device__ static double to(T x) { return x; }
  __device__ static T zero() { return 0.0; }
  __device__ static T mad(T a, T b, T c) { return fma(a, b, c); }
};
struct ArF {
  using T = float;
  __device__ static T from(double x) { return (float)x; }
  // N and X arrive from their GEMMs as (hi, lo) FP32 pairs in 8-byte slots: the hi part
  __device__ static T load(const double *p) { return reinterpret_cast<const float2 *>(p)->x; }
  __device__ static double to(T x) { return (double)x; }
  __device__ static T zero() { return 0.f; }
  __device__ static T mad(T a, T b, T c) { return fmaf(a, b, c); }
};
struct ArDF {
  using T = float2;   // value x + y; operands normalised (|y| <= ulp(x) / 2), accumulators not
  __device__ static T from(double v) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
  }
  __device__ static double to(T v) { return (double)v.x + (double)v.y; }
  __device__ static T zero() { return make_float2(0.f, 0.f); }
  // N and X arrive from their GEMMs already as (hi, lo) pairs in 8-byte slots
  __device__ static T load(const double *p) { return *reinterpret_cast<const float2 *>(p); }
  // c + a b: the high parts' rounded product joins c.x by an exact two-sum; the product's
  // rounding error, the cross terms and the two-sum error collect in c.y, which is never
  // renormalised (its own rounding is ~2^-24 of terms of size ulp(c.x): ~n 2^-48 overall)
  __device__ static T mad(T a, T b, T c) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);   // a.x b.x = p + e exactly
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float s = c.x + p;        // s + t = c.x + p exactly
    const float bv = s - c.x;
    const float t = (c.x - (s - bv)) + (p - bv);
    return make_float2(s, c.y + (t + e));
  }
};

// row-block sizes of the O assembly: atoms with up to 5, 9, 13 and more NAOs (13: carbon-like,
// 5 / 9: light and intermediate species of the workloads)
constexpr int kOasmRows[4] = {5, 9, 13, 16};
int oasm_group(int n_ao) { return n_ao <= 5 ? 0 : n_ao <= 9 ? 1 : n_ao <= 13 ? 2 : 3; }

// One CTA per (point, U, V, 64-column chunk of U's packed columns), for the atoms U listed in ulist
// (those whose NAO count the row block ROWS suits: a launch per such group); 64 x NL threads = 64
// columns x NL lanes over nu; every thread computes all rows i < n_U of U for its (nu, column),
// ROWS at a time (ROWS = n_U for the 5, 9 and 13 NAOs of the workloads).  Shared
// memory (type T): Lm[n_U][2 n_V] = [A_UV(R) | B_UV(R)], RG[2 n_V][64] = [B_{V,kap}(R1-R);
// A_{V,kap}(R1-R)], LX[NL][n_U][2 n_V] = [X^A_nu | X^B_nu] (rows of U) for the NL nu of a step.
template <class Ar, int ROWS>
__global__ void __launch_bounds__(256, 2) k_oassemble(OArgs a, int NL, const int *__restrict__ ulist, int nlist) {
  using T = typename Ar::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *sm = reinterpret_cast<T *>(smraw);
  const int V = blockIdx.y % a.natoms;
  const int U = ulist[(blockIdx.y / a.natoms) % nlist];
  const int p = blockIdx.y / (a.natoms * nlist);
  const int mU = a.m[U];
  const int c0 = blockIdx.x * 64;
  if (c0 >= mU) return;
  const int nU = a.n_ao[U], nV = a.n_ao[V], two = 2 * nV;
  if (a.zero && a.zero[((size_t)(p * a.natoms + U) * a.natoms + V) * gridDim.x + blockIdx.x]) {
    // every term of this block multiplies a dropped G block or an exactly zero N / X block
    double *Ob = a.O + p * a.o_sz_p + a.o_off[U];
    const int w = min(64, mU - c0), nauxV = a.n_aux[V];
    for (long long e = threadIdx.x; e < (long long)nauxV * nU * 64; e += blockDim.x) {
      const int col = (int)(e % 64);
      if (col >= w) continue;
      const long long r = e / 64;
      Ob[(size_t)(a.aux_off[V] + r / nU) * nU * mU + (size_t)(r % nU) * mU + c0 + col] = 0.0;
    }
    return;
  }
  T *Lm = sm;                  // [nU][two]
  T *RG = Lm + nU * two;       // [two][64]
  T *LX = RG + two * 64;       // [NL][nU][two]
  const Point pt = a.pts[p];
  const int tid = threadIdx.x, col = tid & 63, nl = tid >> 6, nthr = 64 * NL;
  const size_t n2 = (size_t)a.nao * a.nao;
  const double *GB = a.G + ((size_t)pt.itau * a.nR_stride) * n2;                 // G^occ(tau)
  const double *GA = a.G + a.g_gstride + ((size_t)pt.itau * a.nR_stride) * n2;   // G^vir(tau)
  const int aoU = a.ao_off[U], aoV = a.ao_off[V];
  for (int e = tid; e < nU * two; e += nthr) {
    const int i = e / two, t = e % two;
    const double *Gs = t < nV ? GA : GB;
    Lm[e] = Ar::from(Gs[((size_t)pt.iR) * n2 + (size_t)(aoU + i) * a.nao + aoV + (t % nV)]);
  }
  const int kc = c0 + col;
  const bool live = kc < mU;
  const int *kp = a.kap + 6 * (a.kap_off[U] + (live ? kc : 0));
  const int ucol = kp[5];
  {
    auto fold = [](int x, int nn) { int r = x % nn; return r < 0 ? r + nn : r; };
    const int iR = (fold(kp[1] - pt.R[0], a.n1) * a.n2 + fold(kp[2] - pt.R[1], a.n2)) * a.n3 +
                   fold(kp[3] - pt.R[2], a.n3);
    for (int t = nl; t < two; t += NL) {
      const double *Gs = t < nV ? GB : GA;
      RG[t * 64 + col] = live ? Ar::from(Gs[(size_t)iR * n2 + (size_t)(aoV + (t % nV)) * a.nao + kp[4]]) : Ar::zero();
    }
  }
  const int nauxV = a.n_aux[V];
  const double *NB = a.N + p * a.n_sz_p + a.n_off[V];                 // N[G^occ]: g = 0
  const double *NA = a.N + p * a.n_sz_p + a.n_sz_g + a.n_off[V];      // N[G^vir]: g = 1
  const double *XB = a.X + p * a.x_sz_p + a.x_off[V];                 // X[G^occ]
  const double *XA = a.X + p * a.x_sz_p + a.x_sz_g + a.x_off[V];      // X[G^vir]
  const int ldx = nauxV * nV;
  double *Ob = a.O + p * a.o_sz_p + a.o_off[U];
  const int ldo = nU * mU;
  for (int nu0 = 0; nu0 < nauxV; nu0 += NL) {
    __syncthreads();   // previous LX consumed; Lm and RG written
    for (int e = tid; e < NL * nU * two; e += nthr) {
      const int q = e / (nU * two), r = e % (nU * two), i = r / two, t = r % two;
      const int nu = nu0 + q;
      LX[e] = nu < nauxV ? Ar::load((t < nV ? XA : XB) + (size_t)(aoU + i) * ldx + nu * nV + (t % nV)) : Ar::zero();
    }
    __syncthreads();
    const int nu = nu0 + nl;
    if (!live || nu >= nauxV) continue;
    const T *lx = LX + nl * nU * two;
    double *orow = Ob + (size_t)(a.aux_off[V] + nu) * ldo;
    for (int i0 = 0; i0 < nU; i0 += ROWS) {
      T acc[ROWS];
#pragma unroll
      for (int r = 0; r < ROWS; ++r) acc[r] = Ar::zero();
      // the two halves of t (N[G^occ] with A_UV, then N[G^vir] with B_UV) without a select per t
#pragma unroll 1
      for (int hlf = 0; hlf < 2; ++hlf) {
        const double *Nh = (hlf == 0 ? NB : NA) + (size_t)nu * nV * a.m_all + ucol;
#pragma unroll 2
        for (int j = 0; j < nV; ++j) {
          const int t = hlf * nV + j;
          const T rn = Ar::load(Nh + (size_t)j * a.m_all);
          const T rgv = RG[t * 64 + col];
#pragma unroll
          for (int r = 0; r < ROWS; ++r) {
            const int i = i0 + r;
            if (i >= nU) break;   // rows beyond U's NAOs (ROWS is the group's largest n_U)
            acc[r] = Ar::mad(Lm[i * two + t], rn, Ar::mad(lx[i * two + t], rgv, acc[r]));
          }
        }
      }
#pragma unroll
      for (int r = 0; r < ROWS; ++r)
        if (i0 + r < nU) orow[(size_t)(i0 + r) * mU + kc] = Ar::to(acc[r]);
    }
  }
}

// ------------------------------------------------------------ O assembly on the tensor cores
// The same O = M + M* + Z + Z* for the tensor-core modes, as exact digit-plane products on the
// BF16 tensor cores (mma.sync m16n8k16, FP32 accumulators).  Per nu of V, O_nu[i][kc] is the sum
// of two products over K = 2 n_V:
//   term 1:  Lm[i][t] . Nt_nu[t][kc]   Lm = [A_UV(R) | B_UV(R)],  Nt = [N[G^occ]; N[G^vir]] at ucol(kc)
//   term 2:  LX_nu[i][t] . RG[t][kc]   LX = [X^A_nu | X^B_nu] (rows of U),  RG = [B_{V,kap}; A_{V,kap}]
// Each row of an A operand (i, over t) and each column of a B operand (kc, over t) is scaled by a
// power of two 2^-E (E: its largest |value| < 2^E) and cut into S balanced base-256 digits
// x = sum_s d_s 2^{-7-8(s-1)}, |d_s| <= 128 (exact in BF16); the digit products of one diagonal
// s + t are summed exactly on the tensor cores (|sum| <= 5 * 32 * 2^14 < 2^22 for K <= 32), the
// diagonals folded into one int64 per term, the two terms aligned to the larger scale and
// converted to FP64 once.  Inputs: N and X as (hi, lo) FP32 pairs, G as FP64 turned into pairs;
// the low part joins the digits after the second (error below 2^-39 of the row or column
// maximum).  One CTA of 4 warps per (point, U, V, 64-column chunk of U); warp w owns columns
// c0 + 16 w .. + 16 (two n8 tiles) and runs over every nu.  Needs n_U, n_V <= 16.
constexpr int kTcKP = 40;   // row pitch of a digit plane in BF16 elements (80 bytes: ldmatrix rows
                            // of 8 consecutive planes rows fall in distinct 16-byte bank groups)
constexpr float kRintMagic = 12582912.0f;   // 1.5 * 2^23: (x + M) - M rounds |x| < 2^22 to an integer

__host__ __device__ constexpr int oasm_tc_smem(int S) {
  // Lm, LX [S][16][KP]; RG [S][64][KP]; N [4][S][16][KP] (BF16); exponents: e1[16], e2[16], f2[64], f1[4][16]
  return (S * 16 * kTcKP * 2 + S * 64 * kTcKP + 4 * S * 16 * kTcKP) * 2 + (16 + 16 + 64 + 64) * 4;
}

// E with max |value| < 2^E from the largest |hi| (0 for an all-zero row), kept in [-100, 100]
__device__ __forceinline__ int tc_expo(float m) {
  if (!(m > 0.f)) return 0;
  const int be = (__float_as_int(m) >> 23) & 0xff;
  return min(100, max(-100, be - 126));
}
__device__ __forceinline__ float tc_pow2(int k) { return __int_as_float((k + 127) << 23); }   // |k| <= 126

// S digits of (h + l) 2^-E into d[] (sc7 = 2^{7-E}, sc15 = 2^{15-E})
template <int S>
__device__ __forceinline__ void tc_digits(float h, float l, float sc7, float sc15, float *d) {
  float t = h * sc7;
  float dd = (t + kRintMagic) - kRintMagic;
  float r = t - dd;
  d[0] = dd;
#pragma unroll
  for (int s = 1; s < S; ++s) {
    if (s == 2) r = fmaf(l, sc15, r);   // the low part, in units of the third digit
    t = r * 256.f;
    dd = (t + kRintMagic) - kRintMagic;
    r = t - dd;
    d[s] = dd;
  }
}

__device__ __forceinline__ unsigned pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);   // small integers: exact
  return *reinterpret_cast<unsigned *>(&v);
}
__device__ __forceinline__ float2 g_pair(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float *c, const unsigned *a, unsigned b0, unsigned b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};\n"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Digit products of one term for the warp's two n8 tiles: A planes [S][16][KP] (rows i), B planes
// [S][..][KP] (rows kc, from brow0), ks_n k-steps of 16; acc[d][nt][4] for the diagonals d = sa + sb.
template <int S>
__device__ __forceinline__ void tc_term(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int bplane, int brow0,
                                        int ks_n, int lane, float (*acc)[2][4]) {
#pragma unroll
  for (int d = 0; d < S; ++d)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[d][nt][r] = 0.f;
  const int arow = lane & 15, acol = (lane >> 4) * 8;
  const int brow = brow0 + (lane & 7) + ((lane >> 4) << 3), bcol = ((lane >> 3) & 1) * 8;
  for (int ks = 0; ks < ks_n; ++ks) {
    unsigned a[S][4], b[S][4];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      ldsm_x4(smem_u32(A + (s * 16 + arow) * kTcKP + ks * 16 + acol), a[s][0], a[s][1], a[s][2], a[s][3]);
      ldsm_x4(smem_u32(B + s * bplane + brow * kTcKP + ks * 16 + bcol), b[s][0], b[s][1], b[s][2], b[s][3]);
    }
#pragma unroll
    for (int sa = 0; sa < S; ++sa)
#pragma unroll
      for (int sb = 0; sb < S - sa; ++sb) {
        mma_bf16(acc[sa + sb][0], a[sa], b[sb][0], b[sb][1]);
        mma_bf16(acc[sa + sb][1], a[sa], b[sb][2], b[sb][3]);
      }
  }
}

// sum_d A_d 2^{8(S-1-d)} of exact integer-valued FP32 diagonal sums (|A_d| < 2^22)
template <int S>
__device__ __forceinline__ long long tc_fold(const float *a) {
  int v[S];
#pragma unroll
  for (int d = 0; d < S; ++d) v[d] = (int)((unsigned)__float_as_int(a[d] + kRintMagic) - 0x4B400000u);
  if constexpr (S == 5) {   // v0 2^8 + v1 and v3 2^8 + v4 stay below 2^31
    return ((long long)(v[0] * 256 + v[1]) << 24) + ((long long)v[2] << 16) + (long long)(v[3] * 256 + v[4]);
  } else if constexpr (S == 3) {
    return ((long long)v[0] << 16) + (long long)(v[1] * 256 + v[2]);
  } else {
    long long T = 0;
#pragma unroll
    for (int d = 0; d < S; ++d) T = T * 256 + v[d];
    return T;
  }
}

template <int S>
__global__ void __launch_bounds__(128) k_oassemble_tc(OArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __nv_bfloat16 *sLm = reinterpret_cast<__nv_bfloat16 *>(smraw);   // [S][16][KP]
  __nv_bfloat16 *sLX = sLm + S * 16 * kTcKP;                        // [S][16][KP]
  __nv_bfloat16 *sRG = sLX + S * 16 * kTcKP;                        // [S][64][KP]
  __nv_bfloat16 *sN = sRG + S * 64 * kTcKP;                         // [4][S][16][KP]
  int *sE1 = reinterpret_cast<int *>(sN + 4 * S * 16 * kTcKP);      // [16]
  int *sE2 = sE1 + 16;                                              // [16]
  int *sF2 = sE2 + 16;                                              // [64]
  int *sF1 = sF2 + 64;                                              // [4][16]
  const int V = blockIdx.y % a.natoms;
  const int U = (blockIdx.y / a.natoms) % a.natoms;
  const int p = blockIdx.y / (a.natoms * a.natoms);
  const int mU = a.m[U];
  const int c0 = blockIdx.x * 64;
  if (c0 >= mU) return;
  const int nU = a.n_ao[U], nV = a.n_ao[V], two = 2 * nV, nauxV = a.n_aux[V];
  double *Ob = a.O + p * a.o_sz_p + a.o_off[U];
  const int ldo = nU * mU;
  if (a.zero && a.zero[((size_t)(p * a.natoms + U) * a.natoms + V) * gridDim.x + blockIdx.x]) {
    const int w = min(64, mU - c0);
    for (long long e = threadIdx.x; e < (long long)nauxV * nU * 64; e += blockDim.x) {
      const int col = (int)(e % 64);
      if (col >= w) continue;
      const long long r = e / 64;
      Ob[(size_t)(a.aux_off[V] + r / nU) * ldo + (size_t)(r % nU) * mU + c0 + col] = 0.0;
    }
    return;
  }
  const Point pt = a.pts[p];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t n2 = (size_t)a.nao * a.nao;
  const double *GB = a.G + ((size_t)pt.itau * a.nR_stride) * n2;                 // G^occ(tau)
  const double *GA = a.G + a.g_gstride + ((size_t)pt.itau * a.nR_stride) * n2;   // G^vir(tau)
  const int aoU = a.ao_off[U], aoV = a.ao_off[V];
  const int ks_n = (two + 15) / 16;
  // Lm digits (A of term 1): thread = (row i, 4 t); row exponent over the 8 lanes of the row
  {
    const int i = tid >> 3, t0 = (tid & 7) * 4;
    float2 v[4];
    float m = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int t = t0 + q;
      v[q] = make_float2(0.f, 0.f);
      if (i < nU && t < two) {
        const double *Gs = t < nV ? GA : GB;
        v[q] = g_pair(Gs[((size_t)pt.iR) * n2 + (size_t)(aoU + i) * a.nao + aoV + (t < nV ? t : t - nV)]);
      }
      m = fmaxf(m, fabsf(v[q].x));
    }
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
    const int E = tc_expo(m);
    if ((tid & 7) == 0) sE1[i] = E;
    const float sc7 = tc_pow2(7 - E), sc15 = tc_pow2(15 - E);
    float d[4][S];
#pragma unroll
    for (int q = 0; q < 4; ++q) tc_digits<S>(v[q].x, v[q].y, sc7, sc15, d[q]);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      uint2 w2 = make_uint2(pack_bf16(d[0][s], d[1][s]), pack_bf16(d[2][s], d[3][s]));
      *reinterpret_cast<uint2 *>(sLm + (s * 16 + i) * kTcKP + t0) = w2;
    }
  }
  // RG digits (B of term 2, stored [kc][t]): thread = (column, 16 t); column exponent over 2 lanes
  {
    const int col = tid >> 1, t0 = (tid & 1) * 16;
    const int kc = c0 + col;
    const bool live = kc < mU;
    const int *kp = a.kap + 6 * (a.kap_off[U] + (live ? kc : 0));
    auto fold = [](int x, int nn) { int r = x % nn; return r < 0 ? r + nn : r; };
    const int iR = (fold(kp[1] - pt.R[0], a.n1) * a.n2 + fold(kp[2] - pt.R[1], a.n2)) * a.n3 +
                   fold(kp[3] - pt.R[2], a.n3);
    float2 v[16];
    float m = 0.f;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int t = t0 + q;
      v[q] = make_float2(0.f, 0.f);
      if (live && t < two) {
        const double *Gs = t < nV ? GB : GA;
        v[q] = g_pair(Gs[(size_t)iR * n2 + (size_t)(aoV + (t < nV ? t : t - nV)) * a.nao + kp[4]]);
      }
      m = fmaxf(m, fabsf(v[q].x));
    }
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    const int E = tc_expo(m);
    if ((tid & 1) == 0) sF2[col] = E;
    const float sc7 = tc_pow2(7 - E), sc15 = tc_pow2(15 - E);
#pragma unroll
    for (int q0 = 0; q0 < 16; q0 += 8) {
      float d[8][S];
#pragma unroll
      for (int q = 0; q < 8; ++q) tc_digits<S>(v[q0 + q].x, v[q0 + q].y, sc7, sc15, d[q]);
#pragma unroll
      for (int s = 0; s < S; ++s) {
        uint4 w4 = make_uint4(pack_bf16(d[0][s], d[1][s]), pack_bf16(d[2][s], d[3][s]), pack_bf16(d[4][s], d[5][s]),
                              pack_bf16(d[6][s], d[7][s]));
        *reinterpret_cast<uint4 *>(sRG + (s * 64 + col) * kTcKP + t0 + q0) = w4;
      }
    }
  }
  // this lane's column of the N operand: (column = lane & 15 of the warp's 16, t half = lane >> 4)
  const int ncol = lane & 15, nt0 = (lane >> 4) * 16;
  const int nkc = c0 + warp * 16 + ncol;
  const bool nlive = nkc < mU;
  const int ucol = a.kap[6 * (a.kap_off[U] + (nlive ? nkc : 0)) + 5];
  const double *NB = a.N + p * a.n_sz_p + a.n_off[V];                 // N[G^occ]: g = 0
  const double *NA = a.N + p * a.n_sz_p + a.n_sz_g + a.n_off[V];      // N[G^vir]: g = 1
  const double *XB = a.X + p * a.x_sz_p + a.x_off[V];                 // X[G^occ]
  const double *XA = a.X + p * a.x_sz_p + a.x_sz_g + a.x_off[V];      // X[G^vir]
  const int ldx = nauxV * nV;
  __nv_bfloat16 *sNw = sN + warp * S * 16 * kTcKP;
  const int g = lane >> 2, tig = lane & 3;
  for (int nu = 0; nu < nauxV; ++nu) {
    // LX digits (A of term 2), shared by the 4 warps
    {
      const int i = tid >> 3, t0 = (tid & 7) * 4;
      float2 v[4];
      float m = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int t = t0 + q;
        v[q] = make_float2(0.f, 0.f);
        if (i < nU && t < two)
          v[q] = *reinterpret_cast<const float2 *>(t < nV ? XA + (size_t)(aoU + i) * ldx + nu * nV + t
                                                          : XB + (size_t)(aoU + i) * ldx + nu * nV + (t - nV));
        m = fmaxf(m, fabsf(v[q].x));
      }
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
      const int E = tc_expo(m);
      if ((tid & 7) == 0) sE2[i] = E;
      const float sc7 = tc_pow2(7 - E), sc15 = tc_pow2(15 - E);
      float d[4][S];
#pragma unroll
      for (int q = 0; q < 4; ++q) tc_digits<S>(v[q].x, v[q].y, sc7, sc15, d[q]);
#pragma unroll
      for (int s = 0; s < S; ++s) {
        uint2 w2 = make_uint2(pack_bf16(d[0][s], d[1][s]), pack_bf16(d[2][s], d[3][s]));
        *reinterpret_cast<uint2 *>(sLX + (s * 16 + i) * kTcKP + t0) = w2;
      }
    }
    // N digits (B of term 1) of the warp's 16 columns, stored [kc][t]
    {
      const double *Nn = NB + (size_t)nu * nV * a.m_all + ucol;
      const double *Na = NA + (size_t)nu * nV * a.m_all + ucol;
      float2 v[16];
      float m = 0.f;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int t = nt0 + q;
        v[q] = make_float2(0.f, 0.f);
        if (nlive && t < two)
          v[q] = *reinterpret_cast<const float2 *>(t < nV ? Nn + (size_t)t * a.m_all : Na + (size_t)(t - nV) * a.m_all);
        m = fmaxf(m, fabsf(v[q].x));
      }
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));
      const int E = tc_expo(m);
      if (lane < 16) sF1[warp * 16 + ncol] = E;
      const float sc7 = tc_pow2(7 - E), sc15 = tc_pow2(15 - E);
#pragma unroll
      for (int q0 = 0; q0 < 16; q0 += 8) {
        float d[8][S];
#pragma unroll
        for (int q = 0; q < 8; ++q) tc_digits<S>(v[q0 + q].x, v[q0 + q].y, sc7, sc15, d[q]);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          uint4 w4 = make_uint4(pack_bf16(d[0][s], d[1][s]), pack_bf16(d[2][s], d[3][s]),
                                pack_bf16(d[4][s], d[5][s]), pack_bf16(d[6][s], d[7][s]));
          *reinterpret_cast<uint4 *>(sNw + (s * 16 + ncol) * kTcKP + nt0 + q0) = w4;
        }
      }
    }
    __syncthreads();   // LX, N and (first pass) Lm, RG digits and exponents written
    float acc[S][2][4];
    long long T1[2][4];
    tc_term<S>(sLm, sNw, 16 * kTcKP, 0, ks_n, lane, acc);
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        float av[S];
#pragma unroll
        for (int d = 0; d < S; ++d) av[d] = acc[d][nt][r];
        T1[nt][r] = tc_fold<S>(av);
      }
    tc_term<S>(sLX, sRG, 64 * kTcKP, warp * 16, ks_n, lane, acc);
    double *orow = Ob + (size_t)(a.aux_off[V] + nu) * ldo;
    int emax = 0;   // largest biased exponent among this lane's stored outputs
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = g + (r >> 1) * 8, cw = nt * 8 + 2 * tig + (r & 1), kc = c0 + warp * 16 + cw;
        float av[S];
#pragma unroll
        for (int d = 0; d < S; ++d) av[d] = acc[d][nt][r];
        const long long T2 = tc_fold<S>(av);
        const int E1 = sE1[i] + sF1[warp * 16 + cw], E2 = sE2[i] + sF2[warp * 16 + cw];
        long long T;
        int E;
        if (E1 >= E2) {
          const int sh = E1 - E2;
          T = T1[nt][r] + (sh == 0 ? T2 : sh >= 62 ? 0 : (T2 + (1LL << (sh - 1))) >> sh);
          E = E1;
        } else {
          const int sh = E2 - E1;
          T = T2 + (sh >= 62 ? 0 : (T1[nt][r] + (1LL << (sh - 1))) >> sh);
          E = E2;
        }
        double o = (double)T;
        if (T != 0) {
          const long long bits = __double_as_longlong(o);
          const int k = E - 14 - 8 * (S - 1);
          const int ex = (int)((bits >> 52) & 0x7ff) + k;
          o = ex <= 0 ? 0.0 : __longlong_as_double(bits + ((long long)k << 52));
        }
        if (i < nU && kc < mU) {
          orow[(size_t)i * mU + kc] = o;
          emax = max(emax, (int)((__double_as_longlong(o) >> 52) & 0x7FF));
        }
      }
    if (S < 4 && a.rexp) {   // the row (p, U, nu) of the final contraction's O operand
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, off));
      if (lane == 0 && emax > 0)
        atomicMax(a.rexp + ((size_t)p * a.natoms + U) * a.naux + a.aux_off[V] + nu, emax - 1022);
    }
    __syncthreads();   // every warp done with LX and the exponents before the next nu
  }
}

template <class T>
T *upload(Handle &h, DevBuf &b, const std::vector<T> &v) {
  h.ensure(b, std::max<size_t>(1, v.size()) * sizeof(T));
  if (!v.empty()) LR_CUDA(cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return (T *)b.p;
}

// Descriptors and tiles of one grouped FP64 GEMM launch, resident on the device, so that the
// launch can be repeated or captured in a CUDA graph.
struct DLaunch {
  const DGemm *g = nullptr;
  const DTile *t = nullptr;
  const int *c = nullptr;
  unsigned ntiles = 0;
  int v = 0;
  double flops = 0;
};

// Descriptors, tiles and (with chunk_fn) each tile's K chunks, resident on the device.  flops:
// the algorithmic flops of what the tiles sum (2 M N K per entry, or per tile over its chunks).
DLaunch dgemm_prepare(Handle &h, const std::vector<DGemm> &batch, int v, cudaStream_t s, DevBuf &args,
                      const ChunkFn *chunk_fn = nullptr) {
  const int BM = 32 * kVarWM[v], BN = 32 * kVarWN[v];
  std::vector<DTile> tiles;
  std::vector<int> chunks, cl;
  DLaunch L;
  L.v = v;
  for (int e = 0; e < (int)batch.size(); ++e) {
    const DGemm &g = batch[e];
    for (int m0 = 0; m0 < g.M; m0 += BM)
      for (int n0 = 0; n0 < g.N; n0 += BN) {
        const int rows = std::min(BM, g.M - m0), cols = std::min(BN, g.N - n0);
        cl.clear();
        if (chunk_fn && (*chunk_fn)(e, m0, rows, n0, cols, GK, g.K, cl)) {
          if (cl.empty()) {   // nothing to sum: a K = 0 entry writes its zeros
            tiles.push_back({e, m0, n0, 0, 0});
            continue;
          }
          double kk = 0;
          for (int c : cl) kk += std::min(GK, g.K - c * GK);
          L.flops += 2.0 * rows * cols * kk;
          tiles.push_back({e, m0, n0, (int)chunks.size(), (int)cl.size()});
          chunks.insert(chunks.end(), cl.begin(), cl.end());
        } else {
          L.flops += 2.0 * rows * cols * g.K;
          tiles.push_back({e, m0, n0, 0, -1});
        }
      }
  }
  if (tiles.empty()) return L;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t b1 = batch.size() * sizeof(DGemm), off2 = al(b1), b2 = tiles.size() * sizeof(DTile),
               off3 = off2 + al(b2), b3 = std::max<size_t>(1, chunks.size()) * sizeof(int);
  std::vector<char> host(off3 + b3);
  std::memcpy(host.data(), batch.data(), b1);
  std::memcpy(host.data() + off2, tiles.data(), b2);
  if (!chunks.empty()) std::memcpy(host.data() + off3, chunks.data(), chunks.size() * sizeof(int));
  h.upload_async(args, host.data(), off3 + b3);
  L.g = (const DGemm *)args.p;
  L.t = (const DTile *)((const char *)args.p + off2);
  L.c = (const int *)((const char *)args.p + off3);
  L.ntiles = (unsigned)tiles.size();
  return L;
}

void dgemm_launch(Handle &h, const DLaunch &L, cudaStream_t s, bool timed) {
  if (!L.ntiles) return;
  Handle::Timed t{nullptr, nullptr, L.flops, 0};
  if (timed) {
    LR_CUDA(cudaEventCreate(&t.a));
    LR_CUDA(cudaEventCreate(&t.b));
    LR_CUDA(cudaEventRecord(t.a, s));
  }
  launch_dgemm_variant(L.v, L.ntiles, L.g, L.t, L.c, s);
  ++launch_counter();
  LR_CUDA(cudaGetLastError());
  if (timed) {
    LR_CUDA(cudaEventRecord(t.b, s));
    h.timed.push_back(t);
  }
}

int dgemm_autotune(Handle &h, const std::vector<DGemm> &batch, cudaStream_t s, DevBuf &args,
                   const ChunkFn *chunk_fn = nullptr) {
  for (const DGemm &g : batch)
    if (g.beta != 0.0) return 0;   // repeated runs would accumulate into C
  int best = 0;
  float best_ms = 1e30f;
  cudaEvent_t a, b;
  LR_CUDA(cudaEventCreate(&a));
  LR_CUDA(cudaEventCreate(&b));
  for (int v = 0; v < kNumVariants; ++v) {
    const DLaunch L = dgemm_prepare(h, batch, v, s, args, chunk_fn);
    LR_CUDA(cudaEventRecord(a, s));
    dgemm_launch(h, L, s, false);
    LR_CUDA(cudaEventRecord(b, s));
    LR_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    LR_CUDA(cudaEventElapsedTime(&ms, a, b));
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

// returns the algorithmic flops of the launch
double dgemm_batched(Handle &h, const std::vector<DGemm> &batch, cudaStream_t s, DevBuf &args, int *var,
                     const ChunkFn *chunk_fn = nullptr) {
  if (*var < 0) *var = dgemm_autotune(h, batch, s, args, chunk_fn);
  const DLaunch L = dgemm_prepare(h, batch, *var, s, args, chunk_fn);
  dgemm_launch(h, L, s, true);
  return L.flops;
}

}  // namespace

void chi0_shape(const Handle &h, Chi0Plan &P) {
  const int nat = h.natoms;
  P.natoms = nat;
  P.nao = h.nao;
  P.naux = h.naux;
  P.n_ao = h.n_ao;
  P.n_aux = h.n_aux;
  P.ao_off = h.ao_off;
  P.aux_off = h.aux_off;
  P.nb.assign(nat, {});
  for (auto &kv : h.lri) {
    int I, K, r0, r1, r2;
    std::tie(I, K, r0, r1, r2) = kv.first;
    NbEntry e{K, {r0, r1, r2}, 0, 0};
    P.nb[I].push_back(e);
  }
  std::set<std::tuple<int, int, int, int>> uni;
  P.m.assign(nat, 0);
  for (int U = 0; U < nat; ++U) {
    // std::map iteration already orders by (K, R)
    int col = 0;
    for (auto &e : P.nb[U]) {
      e.col = col;
      col += h.n_ao[e.K];
      uni.insert(std::make_tuple(e.K, e.R[0], e.R[1], e.R[2]));
    }
    P.m[U] = col;
  }
  P.uni.assign(uni.begin(), uni.end());
  P.uni_col.resize(P.uni.size());
  int mc = 0;
  std::map<std::tuple<int, int, int, int>, int> ucol;
  for (size_t b = 0; b < P.uni.size(); ++b) {
    P.uni_col[b] = mc;
    ucol[P.uni[b]] = mc;
    mc += h.n_ao[std::get<0>(P.uni[b])];
  }
  P.m_all = mc;
  for (int U = 0; U < nat; ++U)
    for (auto &e : P.nb[U]) e.ucol = ucol[std::make_tuple(e.K, e.R[0], e.R[1], e.R[2])];
  // packed coefficients
  P.cp_off.assign(nat + 1, 0);
  for (int U = 0; U < nat; ++U) P.cp_off[U + 1] = P.cp_off[U] + (long long)h.n_aux[U] * h.n_ao[U] * P.m[U];
  P.cp_total = P.cp_off[nat];
  // workspace offsets (elements, per point and per Green's function)
  P.bg_off.assign(nat + 1, 0);
  P.ag_off.assign(nat + 1, 0);
  P.n_off.assign(nat + 1, 0);
  P.x_off.assign(nat + 1, 0);
  P.o_off.assign(nat + 1, 0);
  double fl = 0;
  for (int V = 0; V < nat; ++V) {
    const long long rowsV = (long long)h.n_aux[V] * h.n_ao[V];
    P.bg_off[V + 1] = P.bg_off[V] + (long long)P.m_all * P.m[V];
    P.ag_off[V + 1] = P.ag_off[V] + (long long)h.nao * P.m[V];
    P.n_off[V + 1] = P.n_off[V] + rowsV * P.m_all;
    P.x_off[V + 1] = P.x_off[V] + (long long)h.nao * rowsV;
    P.o_off[V + 1] = P.o_off[V] + (long long)h.naux * h.n_ao[V] * P.m[V];
    fl += 2.0 * 2.0 * rowsV * P.m[V] * P.m_all;    // N-step, both G
    fl += 2.0 * 2.0 * h.nao * P.m[V] * rowsV;      // X-step, both G
  }
  P.flop_nx_per_point = fl;
  P.flop_fin_per_point = 0;
  for (int U = 0; U < nat; ++U) {
    const double cols = (double)h.n_ao[U] * P.m[U];
    for (int V = 0; V < nat; ++V) fl += 2.0 * h.n_aux[V] * cols * 4.0 * h.n_ao[V];   // O assembly
    fl += 2.0 * h.n_aux[U] * cols * h.naux;                                        // final
    P.flop_fin_per_point += 2.0 * h.n_aux[U] * cols * h.naux;
  }
  P.flop_per_point = fl;
  P.bg_sz = P.bg_off[nat];
  P.ag_sz = P.ag_off[nat];
  P.n_sz = P.n_off[nat];
  P.x_sz = P.x_off[nat];
  P.o_sz = P.o_off[nat];
  P.max_m = P.max_nm = 0;
  P.cpnx_off.assign(nat + 1, 0);
  for (int a = 0; a < nat; ++a) {
    P.max_m = std::max(P.max_m, P.m[a]);
    P.max_nm = std::max(P.max_nm, h.n_ao[a] * P.m[a]);
    P.cpnx_off[a + 1] = P.cpnx_off[a] + h.n_aux[a] * h.n_ao[a];
  }
  P.cpnx_rows = P.cpnx_off[nat];
  P.tc_S = h.chi0_S;
}

void chi0_plan(Handle &h) {
  Chi0Plan &P = h.plan;
  chi0_shape(h, P);
  P.var_nx = P.var_fin = -1;
  ++P.gen;
  const int nat = h.natoms;
  std::vector<double> cp(P.cp_total, 0.0);
  for (int U = 0; U < nat; ++U) {
    const int nU = h.n_ao[U], mU = P.m[U];
    for (auto &e : P.nb[U]) {
      const std::vector<double> &C = h.lri.at(std::make_tuple(U, e.K, e.R[0], e.R[1], e.R[2]));
      const int nK = h.n_ao[e.K];
      for (int mu = 0; mu < h.n_aux[U]; ++mu)
        for (int i = 0; i < nU; ++i)
          for (int k = 0; k < nK; ++k)
            cp[P.cp_off[U] + ((size_t)mu * nU + i) * mU + e.col + k] = C[((size_t)mu * nU + i) * nK + k];
    }
  }
  upload(h, h.d_cpack, cp);
  // column tables
  std::vector<int> lam, kap, un;
  P.lam_off.assign(nat + 1, 0);
  P.kap_off.assign(nat + 1, 0);
  for (int U = 0; U < nat; ++U) {
    P.lam_off[U] = (long long)lam.size() / 6;
    P.kap_off[U] = (long long)kap.size() / 6;
    for (auto &e : P.nb[U])
      for (int k = 0; k < h.n_ao[e.K]; ++k) {
        const int row[6] = {e.K, e.R[0], e.R[1], e.R[2], k, h.ao_off[e.K] + k};
        lam.insert(lam.end(), row, row + 6);
        const int krow[6] = {e.K, e.R[0], e.R[1], e.R[2], h.ao_off[e.K] + k, e.ucol + k};
        kap.insert(kap.end(), krow, krow + 6);
      }
  }
  P.lam_off[nat] = (long long)lam.size() / 6;
  P.kap_off[nat] = (long long)kap.size() / 6;
  for (size_t b = 0; b < P.uni.size(); ++b) {
    const int K = std::get<0>(P.uni[b]);
    for (int k = 0; k < h.n_ao[K]; ++k) {
      const int row[6] = {K, std::get<1>(P.uni[b]), std::get<2>(P.uni[b]), std::get<3>(P.uni[b]), k,
                          h.ao_off[K] + k};
      un.insert(un.end(), row, row + 6);
    }
  }
  upload(h, P.d_lam, lam);
  upload(h, P.d_kap, kap);
  upload(h, P.d_uni, un);
  upload(h, P.t_n_ao, h.n_ao);
  upload(h, P.t_n_aux, h.n_aux);
  upload(h, P.t_ao_off, h.ao_off);
  upload(h, P.t_aux_off, h.aux_off);
  upload(h, P.t_m, P.m);
  upload(h, P.t_lam_off, P.lam_off);
  upload(h, P.t_kap_off, P.kap_off);
  upload(h, P.t_bg_off, P.bg_off);
  upload(h, P.t_ag_off, P.ag_off);
  upload(h, P.t_n_off, P.n_off);
  upload(h, P.t_x_off, P.x_off);
  upload(h, P.t_o_off, P.o_off);
  {   // atoms by the O assembly's row-block size
    std::vector<int> ug;
    P.ugroup_off.assign(5, 0);
    for (int gi = 0; gi < 4; ++gi) {
      P.ugroup_off[gi] = (int)ug.size();
      for (int a = 0; a < nat; ++a)
        if (oasm_group(h.n_ao[a]) == gi) ug.push_back(a);
    }
    P.ugroup_off[4] = (int)ug.size();
    upload(h, P.t_ugroups, ug);
  }
  // tensor-core route: digit planes of the packed coefficients, split once per plan
  if (P.tc_S >= 0) {
    const int S = P.tc_S;
    const double *Cp = (const double *)h.d_cpack.p;
    oz::Sliced cpnx, cpf;
    h.ensure(P.cp_nx, oz::sliced_bytes(P.cpnx_rows, P.max_m, S));
    h.ensure(P.cp_f, oz::sliced_bytes(h.naux, P.max_nm, S));
    oz::sliced_bind(cpnx, P.cp_nx.p, P.cpnx_rows, P.max_m, S);
    oz::sliced_bind(cpf, P.cp_f.p, h.naux, P.max_nm, S);
    for (int a = 0; a < nat; ++a) {
      const int nm = h.n_ao[a] * P.m[a];
      // rows (nu, j) of atom a, K = m_a (N and X steps)
      oz::split_real(Cp + P.cp_off[a], P.m[a], false, h.n_aux[a] * h.n_ao[a], P.m[a], 1, 0, cpnx, h.stream,
                     P.cpnx_off[a]);
      // rows mu of atom a, K = n_a m_a (final contraction)
      oz::split_real(Cp + P.cp_off[a], nm, false, h.n_aux[a], nm, 1, 0, cpf, h.stream, h.aux_off[a]);
    }
    LR_CUDA(cudaStreamSynchronize(h.stream));
  }
}

namespace {

// O = M + M* + Z + Z* for the np points of a batch (FP64 pipe).  zero: device flags of the CTAs
// whose O block is exactly zero under screening ([np][U][V][64-column chunk]), or NULL.
template <class Ar>
void set_oasm_smem_limits(int bytes) {
  LR_CUDA(cudaFuncSetAttribute(k_oassemble<Ar, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  LR_CUDA(cudaFuncSetAttribute(k_oassemble<Ar, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  LR_CUDA(cudaFuncSetAttribute(k_oassemble<Ar, 13>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  LR_CUDA(cudaFuncSetAttribute(k_oassemble<Ar, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
}

template <class Ar>
void launch_oasm(int gi, dim3 grid, int threads, size_t smem, cudaStream_t s, const OArgs &oa, int NL, const int *ul,
                 int cnt) {
  switch (kOasmRows[gi]) {
    case 5: k_oassemble<Ar, 5><<<grid, threads, smem, s>>>(oa, NL, ul, cnt); break;
    case 9: k_oassemble<Ar, 9><<<grid, threads, smem, s>>>(oa, NL, ul, cnt); break;
    case 13: k_oassemble<Ar, 13><<<grid, threads, smem, s>>>(oa, NL, ul, cnt); break;
    default: k_oassemble<Ar, 16><<<grid, threads, smem, s>>>(oa, NL, ul, cnt); break;
  }
}

// 64-column chunks of the widest packed-column list (the O assembly's grid.x)
int oasm_chunks(const Handle &h) {
  int c = 0;
  for (int a = 0; a < h.natoms; ++a) c = std::max(c, (h.plan.m[a] + 63) / 64);
  return c;
}

// rexp (may be NULL): row exponents of the O operand's digit planes, built by atomicMax (initialised
// to -1022) in the 3-plane tensor-core kernel only: in the 5-plane kernel the atomics cost more
// than the exponent pass they save.  Returns true when the kernel that builds them ran.
bool run_oassemble(Handle &h, const Point *dpts, int np, double *Nw, double *Xw, double *Ow,
                   const unsigned char *zero = nullptr, int *rexp = nullptr) {
  Chi0Plan &P = h.plan;
  const int nat = h.natoms;
  int maxn = 0, max_chunks = 0;
  for (int a = 0; a < nat; ++a) {
    maxn = std::max(maxn, h.n_ao[a]);
    max_chunks = std::max(max_chunks, (P.m[a] + 63) / 64);
  }
  // arithmetic: FP64 pipes for the FP64 mode, FP32 for the mixed modes, FP32 pairs (~48 bits)
  // for the FP64-accurate tensor-core mode
  const int ar = h.chi0_S < 0 ? 0 : (h.chi0_S >= 4 && h.chi0_S <= oz::SMAX) ? 2 : 1;
  const size_t esz = ar == 1 ? sizeof(float) : 8;
  int NL = 4;
  auto smem_for = [&](int nl) { return (size_t)(maxn * 2 * maxn + 2 * maxn * 64 + nl * maxn * 2 * maxn) * esz; };
  while (NL > 1 && smem_for(NL) > 200 * 1024) NL /= 2;
  const size_t osmem = smem_for(NL);
  // the limit is the same fixed bound for every handle: handles on other host threads (batched
  // and serving workers) set it concurrently, and a per-handle value could undercut a launch
  // in flight on another thread
  constexpr int kOasmSmemLimit = 200 * 1024;
  if (osmem > (size_t)kOasmSmemLimit) throw Error{LIBRPA_E_ARG, "O assembly: atoms with too many NAOs"};
  set_oasm_smem_limits<ArD>(kOasmSmemLimit);
  set_oasm_smem_limits<ArF>(kOasmSmemLimit);
  set_oasm_smem_limits<ArDF>(kOasmSmemLimit);
  OArgs oa;
  oa.G = g_spin(h);
  oa.g_gstride = (size_t)h.ntau * h.mesh.size() * h.nao * h.nao;
  oa.nR_stride = h.mesh.size();
  oa.nao = h.nao;
  oa.natoms = nat;
  oa.naux = h.naux;
  oa.n1 = h.mesh.n1;
  oa.n2 = h.mesh.n2;
  oa.n3 = h.mesh.n3;
  oa.pts = dpts;
  oa.n_ao = (const int *)P.t_n_ao.p;
  oa.n_aux = (const int *)P.t_n_aux.p;
  oa.ao_off = (const int *)P.t_ao_off.p;
  oa.aux_off = (const int *)P.t_aux_off.p;
  oa.m = (const int *)P.t_m.p;
  oa.kap = (const int *)P.d_kap.p;
  oa.kap_off = (const long long *)P.t_kap_off.p;
  oa.N = Nw;
  oa.n_off = (const long long *)P.t_n_off.p;
  oa.n_sz_g = P.n_sz;
  oa.n_sz_p = 2 * P.n_sz;
  oa.m_all = P.m_all;
  oa.X = Xw;
  oa.x_off = (const long long *)P.t_x_off.p;
  oa.x_sz_g = P.x_sz;
  oa.x_sz_p = 2 * P.x_sz;
  oa.O = Ow;
  oa.o_off = (const long long *)P.t_o_off.p;
  oa.o_sz_p = P.o_sz;
  oa.zero = zero;
  oa.rexp = nullptr;
  if (ar != 0 && maxn <= 16) {
    oa.rexp = ar == 1 ? rexp : nullptr;
    // tensor-core modes: digit-plane products on the tensor cores, one launch over every (U, V);
    // 5 planes (~39 bits) for the FP64-accurate mode, 3 (~23 bits, as FP32) for the mixed modes
    dim3 og((unsigned)max_chunks, (unsigned)(np * nat * nat));
    if (ar == 2) {
      constexpr int kSmem = oasm_tc_smem(5);
      static_assert(kSmem <= kOasmSmemLimit, "O assembly (tensor cores): shared memory");
      LR_CUDA(cudaFuncSetAttribute(k_oassemble_tc<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
      k_oassemble_tc<5><<<og, 128, kSmem, h.stream>>>(oa);
    } else {
      constexpr int kSmem = oasm_tc_smem(3);
      LR_CUDA(cudaFuncSetAttribute(k_oassemble_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
      k_oassemble_tc<3><<<og, 128, kSmem, h.stream>>>(oa);
    }
    ++launch_counter();
    LR_CUDA(cudaGetLastError());
    return oa.rexp != nullptr;
  }
  // one launch per row-block size: the atoms U of each group (listed in the plan's table).  The
  // FP64 arithmetic is bound by the FP64 pipe, where rows beyond n_U cost nothing: one launch over
  // every atom with 16-row blocks (no tail of a second, small launch).
  for (int gi = ar == 0 ? 3 : 0; gi < 4; ++gi) {
    const int cnt = ar == 0 ? nat : P.ugroup_off[gi + 1] - P.ugroup_off[gi];
    if (!cnt) continue;
    const int *ul = (const int *)P.t_ugroups.p + (ar == 0 ? 0 : P.ugroup_off[gi]);
    dim3 og((unsigned)max_chunks, (unsigned)(np * cnt * nat));
    if (ar == 0)
      launch_oasm<ArD>(gi, og, 64 * NL, osmem, h.stream, oa, NL, ul, cnt);
    else if (ar == 1)
      launch_oasm<ArF>(gi, og, 64 * NL, osmem, h.stream, oa, NL, ul, cnt);
    else
      launch_oasm<ArDF>(gi, og, 64 * NL, osmem, h.stream, oa, NL, ul, cnt);
    ++launch_counter();
    LR_CUDA(cudaGetLastError());
  }
  return false;
}

// Points of the (R, tau) grid in flat order: point idx = itau * nR + iR.
// chi0(-R, tau) = chi0(R, tau)^T for the lattice vectors left out of the point list (the pair
// symmetry of Sec. 2: chi0_{VU}(-R) = chi0_{UV}(R)^T, from G^occ and G^vir being real and
// symmetric in (r, r')).  One 32 x 32 tile per CTA, staged through shared memory.
__global__ void k_fill_partner(double *chi, int naux, int n1, int n2, int n3) {
  __shared__ double t[32][33];
  const int nR = n1 * n2 * n3;
  const int iR = blockIdx.z % nR, itau = blockIdx.z / nR;
  const int a = iR / (n2 * n3), b = (iR / n3) % n2, c = iR % n3;
  const int pR = (((n1 - a) % n1) * n2 + (n2 - b) % n2) * n3 + (n3 - c) % n3;
  if (iR <= pR) return;   // computed directly
  const double *src = chi + ((size_t)itau * nR + pR) * naux * naux;
  double *dst = chi + ((size_t)itau * nR + iR) * naux * naux;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int gr = r0 + r, gc = c0 + threadIdx.x;
    if (gr < naux && gc < naux) t[r][threadIdx.x] = src[(size_t)gr * naux + gc];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int gr = c0 + r, gc = r0 + threadIdx.x;   // dst[gr][gc] = src[gc][gr]
    if (gr < naux && gc < naux) dst[(size_t)gr * naux + gc] = t[threadIdx.x][r];
  }
}

void fill_partners(Handle &h) {
  const int nR = h.mesh.size(), naux = h.naux;
  if ((int)chi0_r_list(h.mesh).size() == nR) return;
  const unsigned nt = (unsigned)((naux + 31) / 32);
  dim3 g(nt, nt, (unsigned)(h.ntau * nR));
  k_fill_partner<<<g, dim3(32, 8), 0, h.stream>>>((double *)h.d_chi_tau.p, naux, h.mesh.n1, h.mesh.n2, h.mesh.n3);
  ++launch_counter();
  LR_CUDA(cudaGetLastError());
}

std::vector<Point> make_points(Handle &h, const std::vector<int> &rl, long long p0, int np) {
  const int nr = (int)rl.size();
  std::vector<Point> pts(np);
  for (int q = 0; q < np; ++q) {
    const long long idx = p0 + q;
    pts[q].itau = (int)(idx / nr);
    pts[q].iR = rl[idx % nr];
    h.mesh.split(pts[q].iR, pts[q].R[0], pts[q].R[1], pts[q].R[2]);
  }
  return pts;
}

// Point selection under Green's-function screening (Sec. 5), from the kept-block mask of the
// screened G.  For the point (R_p, tau) and one Green's function g, the contraction reads:
//   N-step of V:  blocks (L, K) at R1 - R_p - R2, for (L, R2) in N[V] and (K, R1) in the union list;
//   X-step of V:  blocks (I, L) at R_p + R2, every atom I;
//   O assembly:   blocks (U, V) at R_p, and (V, K) at R1 - R_p for (K, R1) in the union list.
// Every term of chi0 pairs a G^occ factor with a G^vir factor (M = G^vir N[G^occ] and
// G^occ N[G^vir], Z = X[G^vir] G^occ and X[G^occ] G^vir), so chi0(R_p, tau) is exactly zero when
// one Green's function has no kept block among those it contributes there: such points are not
// contracted.  An N- or X-step operand with no kept block is exactly zero.
struct ScreenSel {
  std::vector<Point> pts;                // points to contract, in (tau, R) order
  std::vector<unsigned char> nzN, nzX;   // [point][g][V]: the operand holds a kept block
  long long skipped = 0;
};

ScreenSel screen_select(const Handle &h, const std::vector<int> &rl) {
  const Chi0Plan &P = h.plan;
  const int nat = h.natoms, nR = h.mesh.size(), ntau = h.ntau, nr = (int)rl.size();
  const bool on = h.g_screen > 0 && !h.gmask.empty();
  ScreenSel sel;
  auto point = [&](int it, int iR) {
    Point pt;
    pt.itau = it;
    pt.iR = iR;
    h.mesh.split(iR, pt.R[0], pt.R[1], pt.R[2]);
    return pt;
  };
  if (!on) {
    for (int it = 0; it < ntau; ++it)
      for (int r = 0; r < nr; ++r) sel.pts.push_back(point(it, rl[r]));
    sel.nzN.assign(sel.pts.size() * 2 * nat, 1);
    sel.nzX.assign(sel.pts.size() * 2 * nat, 1);
    return sel;
  }
  // per V: distinct (L, K, R1 - R2) of the N-step and distinct (L, R2) of the X-step
  struct Key { int L, K, d[3]; };
  std::vector<std::vector<Key>> dn(nat), dx(nat);
  for (int V = 0; V < nat; ++V) {
    std::set<std::tuple<int, int, int, int, int>> sn, sx;
    for (const NbEntry &l : P.nb[V]) {
      sx.insert(std::make_tuple(l.K, 0, l.R[0], l.R[1], l.R[2]));
      for (const auto &u : P.uni)
        sn.insert(std::make_tuple(l.K, std::get<0>(u), std::get<1>(u) - l.R[0], std::get<2>(u) - l.R[1],
                                  std::get<3>(u) - l.R[2]));
    }
    for (auto &t : sn) dn[V].push_back(Key{std::get<0>(t), std::get<1>(t), {std::get<2>(t), std::get<3>(t), std::get<4>(t)}});
    for (auto &t : sx) dx[V].push_back(Key{std::get<0>(t), 0, {std::get<2>(t), std::get<3>(t), std::get<4>(t)}});
  }
  const size_t nn = (size_t)nat * nat;
  std::vector<unsigned char> col(nR * nat), any_r(nR);   // per (R, J): a kept block (*, J); per R: any
  for (int it = 0; it < ntau; ++it) {
    std::vector<unsigned char> nz(nr * 4 * nat, 0), anyg(nr * 2, 0);   // [r][N/X][g][V], [r][g]
    for (int g = 0; g < 2; ++g) {
      const unsigned char *M = h.gmask.data() + ((size_t)(h.cur_spin * 2 + g) * ntau + it) * nR * nn;
      std::fill(col.begin(), col.end(), 0);
      std::fill(any_r.begin(), any_r.end(), 0);
      for (int iR = 0; iR < nR; ++iR)
        for (int I = 0; I < nat; ++I)
          for (int J = 0; J < nat; ++J)
            if (M[(size_t)iR * nn + (size_t)I * nat + J]) col[iR * nat + J] = any_r[iR] = 1;
      for (int r = 0; r < nr; ++r) {
        int R[3];
        h.mesh.split(rl[r], R[0], R[1], R[2]);
        bool any = any_r[rl[r]];
        for (const auto &u : P.uni)
          if (!any && col[h.mesh.index(std::get<1>(u) - R[0], std::get<2>(u) - R[1], std::get<3>(u) - R[2]) * nat +
                          std::get<0>(u)])
            any = true;
        for (int V = 0; V < nat; ++V) {
          bool n_any = false, x_any = false;
          for (const Key &k : dn[V])
            if (M[(size_t)h.mesh.index(k.d[0] - R[0], k.d[1] - R[1], k.d[2] - R[2]) * nn + (size_t)k.L * nat + k.K]) {
              n_any = true;
              break;
            }
          for (const Key &k : dx[V])
            if (col[h.mesh.index(R[0] + k.d[0], R[1] + k.d[1], R[2] + k.d[2]) * nat + k.L]) {
              x_any = true;
              break;
            }
          nz[((size_t)r * 2 + 0) * 2 * nat + g * nat + V] = n_any;
          nz[((size_t)r * 2 + 1) * 2 * nat + g * nat + V] = x_any;
          any = any || n_any || x_any;
        }
        anyg[r * 2 + g] = any;
      }
    }
    for (int r = 0; r < nr; ++r) {
      if (!(anyg[r * 2] && anyg[r * 2 + 1])) {
        ++sel.skipped;
        continue;
      }
      sel.pts.push_back(point(it, rl[r]));
      const unsigned char *a = nz.data() + (size_t)r * 4 * nat;
      sel.nzN.insert(sel.nzN.end(), a, a + 2 * nat);
      sel.nzX.insert(sel.nzX.end(), a + 2 * nat, a + 4 * nat);
    }
  }
  return sel;
}

// returns the algorithmic flops of the launch (over the K stages summed)
double timed_grouped(Handle &h, const oz::Sliced &a, const oz::Sliced &b, const std::vector<oz::Entry> &es, int *err,
                     DevBuf &args, const oz::StageFn *stage_fn = nullptr) {
  Handle::Timed t{nullptr, nullptr, 0, 0};
  LR_CUDA(cudaEventCreate(&t.a));
  LR_CUDA(cudaEventCreate(&t.b));
  LR_CUDA(cudaEventRecord(t.a, h.stream));
  oz::gemm_grouped(a, b, es, err, h.stream, h, args, stage_fn);
  LR_CUDA(cudaEventRecord(t.b, h.stream));
  t.flops = h.oz_alg_flops;
  t.exec_flops = h.oz_exec_flops;
  h.timed.push_back(t);
  return t.flops;
}

// Block structure of the contraction of a batch of points under Green's-function screening (Sec. 5's
// threshold; Sec. 2: the decay of G limits what contributes).  For point q:
//   n(q, g, V, b, l): the N-step block of V for union block b (K, R1) and neighbour l (L, R2) of V
//                     multiplies the kept G^g block (L, K) at R1 - R_q - R2;
//   x(q, g, V, I, l): the X-step block of V for atom I and neighbour l multiplies the kept G^g block
//                     (I, L) at R_q + R2;
//   o(q, U, V, b'):   the O block of (U, V) on U's neighbour b' (K, R1) can be nonzero: one of its four
//                     terms pairs a kept G block with an N or X block that is not exactly zero,
//                     G^vir_UV(R_q) N[G^occ] + G^occ_UV(R_q) N[G^vir] + X[G^vir] G^occ_VK(R1 - R_q)
//                     + X[G^occ] G^vir_VK(R1 - R_q).
// The GEMM tiles then sum only the K chunks that meet such blocks, and O blocks without one are
// written as zeros: every skipped product is an exact zero, so the result is that of the dense
// contraction on the screened G, and the cost follows the kept blocks inside a point.
struct BlockSparse {
  int nat = 0, nuni = 0, maxnb = 1, np = 0;
  std::vector<int> ublock_of_col;   // union block index at its first union column, -1 elsewhere
  std::vector<unsigned char> n, x, o;
  size_t in(int q, int g, int V, int b, int l) const { return ((((size_t)q * 2 + g) * nat + V) * nuni + b) * maxnb + l; }
  size_t ix(int q, int g, int V, int I, int l) const { return ((((size_t)q * 2 + g) * nat + V) * nat + I) * maxnb + l; }
  size_t io(int q, int U, int V, int b) const { return (((size_t)q * nat + U) * nat + V) * maxnb + b; }
};

BlockSparse block_sparse(const Handle &h, const std::vector<Point> &pts) {
  const Chi0Plan &P = h.plan;
  const int nat = h.natoms, nR = h.mesh.size(), ntau = h.ntau;
  const size_t nn = (size_t)nat * nat;
  BlockSparse B;
  B.nat = nat;
  B.nuni = (int)P.uni.size();
  B.np = (int)pts.size();
  for (int a = 0; a < nat; ++a) B.maxnb = std::max(B.maxnb, (int)P.nb[a].size());
  B.ublock_of_col.assign(P.m_all + 1, -1);
  for (int b = 0; b < B.nuni; ++b) B.ublock_of_col[P.uni_col[b]] = b;
  B.n.assign((size_t)B.np * 2 * nat * B.nuni * B.maxnb, 0);
  B.x.assign((size_t)B.np * 2 * nat * nat * B.maxnb, 0);
  B.o.assign((size_t)B.np * nat * nat * B.maxnb, 0);
  auto kept = [&](int g, int it, int iR, int I, int J) {
    return h.gmask[(((size_t)(h.cur_spin * 2 + g) * ntau + it) * nR + iR) * nn + (size_t)I * nat + J];
  };
  std::vector<unsigned char> nnz(2 * (size_t)nat * B.nuni), xnz(2 * nn);
  for (int q = 0; q < B.np; ++q) {
    const Point &pt = pts[q];
    const int *R = pt.R, it = pt.itau;
    std::fill(nnz.begin(), nnz.end(), 0);
    std::fill(xnz.begin(), xnz.end(), 0);
    for (int g = 0; g < 2; ++g)
      for (int V = 0; V < nat; ++V) {
        const std::vector<NbEntry> &nbV = P.nb[V];
        for (int b = 0; b < B.nuni; ++b) {
          const auto &u = P.uni[b];
          for (int l = 0; l < (int)nbV.size(); ++l) {
            const unsigned char v = kept(g, it, h.mesh.index(std::get<1>(u) - R[0] - nbV[l].R[0], std::get<2>(u) - R[1] - nbV[l].R[1],
                                                             std::get<3>(u) - R[2] - nbV[l].R[2]),
                                         nbV[l].K, std::get<0>(u));
            B.n[B.in(q, g, V, b, l)] = v;
            nnz[((size_t)g * nat + V) * B.nuni + b] |= v;
          }
        }
        for (int l = 0; l < (int)nbV.size(); ++l) {
          const int iR = h.mesh.index(R[0] + nbV[l].R[0], R[1] + nbV[l].R[1], R[2] + nbV[l].R[2]);
          for (int I = 0; I < nat; ++I) {
            const unsigned char v = kept(g, it, iR, I, nbV[l].K);
            B.x[B.ix(q, g, V, I, l)] = v;
            xnz[((size_t)g * nat + V) * nat + I] |= v;
          }
        }
      }
    for (int U = 0; U < nat; ++U)
      for (int V = 0; V < nat; ++V) {
        const bool vir_uv = kept(1, it, pt.iR, U, V), occ_uv = kept(0, it, pt.iR, U, V);
        const bool xv = xnz[((size_t)1 * nat + V) * nat + U], xo = xnz[((size_t)0 * nat + V) * nat + U];
        for (int b = 0; b < (int)P.nb[U].size(); ++b) {
          const NbEntry &e = P.nb[U][b];
          const int ub = B.ublock_of_col[e.ucol];
          const int iRk = h.mesh.index(e.R[0] - R[0], e.R[1] - R[1], e.R[2] - R[2]);
          const bool nz = (vir_uv && nnz[((size_t)0 * nat + V) * B.nuni + ub]) ||
                          (occ_uv && nnz[((size_t)1 * nat + V) * B.nuni + ub]) ||
                          (xv && kept(0, it, iRk, V, e.K)) || (xo && kept(1, it, iRk, V, e.K));
          B.o[B.io(q, U, V, b)] = nz;
        }
      }
  }
  return B;
}

// chunk lists computed once per (entry, tile row or column, chunk size) and reused by the other tiles
// that share them
struct ChunkMemo {
  std::map<std::tuple<int, int, int>, std::vector<int>> m;
  template <class F>
  void get(int e, int pos, int cs, std::vector<int> &out, F &&make) {
    auto it = m.find(std::make_tuple(e, pos, cs));
    if (it == m.end()) {
      std::vector<int> v;
      make(v);
      it = m.emplace(std::make_tuple(e, pos, cs), std::move(v)).first;
    }
    out.insert(out.end(), it->second.begin(), it->second.end());
  }
};

// the needed chunks of [0, K) in units of cs, given which of `blocks` (start, width) are live
void chunks_from_blocks(const std::vector<std::pair<int, int>> &blocks, const std::vector<char> &live, int cs, int K,
                        std::vector<int> &out) {
  std::vector<int> pre(K + 1, 0);   // prefix count of live columns
  std::vector<char> col(K, 0);
  for (size_t l = 0; l < blocks.size(); ++l)
    if (live[l])
      for (int c = blocks[l].first; c < std::min(K, blocks[l].first + blocks[l].second); ++c) col[c] = 1;
  for (int c = 0; c < K; ++c) pre[c + 1] = pre[c] + col[c];
  for (int c = 0; c * cs < K; ++c)
    if (pre[std::min(K, (c + 1) * cs)] > pre[c * cs]) out.push_back(c);
}

// N-step tile of (q, g, V): columns [n0, n0 + cols) of the union list, K = V's packed columns
void chunks_n(const Handle &h, const BlockSparse &B, int q, int g, int V, int n0, int cols, int cs, int K,
              std::vector<int> &out) {
  const Chi0Plan &P = h.plan;
  const std::vector<NbEntry> &nbV = P.nb[V];
  std::vector<std::pair<int, int>> blocks;
  std::vector<char> live(nbV.size(), 0);
  const int b0 = (int)(std::upper_bound(P.uni_col.begin(), P.uni_col.end(), n0) - P.uni_col.begin()) - 1;
  for (int l = 0; l < (int)nbV.size(); ++l) {
    blocks.push_back({nbV[l].col, h.n_ao[nbV[l].K]});
    for (int b = std::max(0, b0); b < B.nuni && P.uni_col[b] < n0 + cols; ++b)
      if (B.n[B.in(q, g, V, b, l)]) {
        live[l] = 1;
        break;
      }
  }
  chunks_from_blocks(blocks, live, cs, K, out);
}

// X-step tile of (q, g, V): rows [m0, m0 + rows) of all NAOs, K = V's packed columns
void chunks_x(const Handle &h, const BlockSparse &B, int q, int g, int V, int m0, int rows, int cs, int K,
              std::vector<int> &out) {
  const Chi0Plan &P = h.plan;
  const std::vector<NbEntry> &nbV = P.nb[V];
  std::vector<std::pair<int, int>> blocks;
  std::vector<char> live(nbV.size(), 0);
  for (int l = 0; l < (int)nbV.size(); ++l) {
    blocks.push_back({nbV[l].col, h.n_ao[nbV[l].K]});
    for (int I = 0; I < B.nat; ++I)
      if (h.ao_off[I] < m0 + rows && h.ao_off[I] + h.n_ao[I] > m0 && B.x[B.ix(q, g, V, I, l)]) {
        live[l] = 1;
        break;
      }
  }
  chunks_from_blocks(blocks, live, cs, K, out);
}

// final-contraction tile of (q, U): nu in [n0, n0 + cols) (its rows in the tensor-core route, where
// the product is O_U . Cpack_U^T; its columns on the FP64 route), K = (i, k) over U's n_U x m_U.
// Whether a K index is live depends on k only (its block of U's packed columns), so one prefix
// count over the m_U columns answers every chunk.
void chunks_f(const Handle &h, const BlockSparse &B, int q, int U, int n0, int cols, int cs, int K,
              std::vector<int> &out) {
  const Chi0Plan &P = h.plan;
  const std::vector<NbEntry> &nbU = P.nb[U];
  const int mU = P.m[U];
  std::vector<int> pre(mU + 1, 0);
  for (int b = 0; b < (int)nbU.size(); ++b) {
    bool live = false;
    for (int V = 0; V < B.nat && !live; ++V)
      live = h.aux_off[V] < n0 + cols && h.aux_off[V] + h.n_aux[V] > n0 && B.o[B.io(q, U, V, b)];
    if (live)
      for (int k = nbU[b].col; k < nbU[b].col + h.n_ao[nbU[b].K]; ++k) pre[k + 1] = 1;
  }
  for (int k = 0; k < mU; ++k) pre[k + 1] += pre[k];
  auto live_in = [&](int lo, int hi) {   // any live column among K indices [lo, hi)
    while (lo < hi) {
      const int i = lo / mU, k0 = lo - i * mU, k1 = std::min(mU, hi - i * mU);
      if (pre[k1] > pre[k0]) return true;
      lo = (i + 1) * mU;
    }
    return false;
  };
  for (int c = 0; c * cs < K; ++c)
    if (live_in(c * cs, std::min(K, (c + 1) * cs))) out.push_back(c);
}

// O-assembly flags [q][U][V][64-column chunk]: 1 where the block is exactly zero; and the
// algorithmic flops of the blocks that are not
std::vector<unsigned char> ozero_flags(const Handle &h, const BlockSparse &B, int max_chunks, double *flops) {
  const Chi0Plan &P = h.plan;
  const int nat = B.nat;
  std::vector<unsigned char> z((size_t)B.np * nat * nat * max_chunks, 1);
  *flops = 0;
  for (int q = 0; q < B.np; ++q)
    for (int U = 0; U < nat; ++U)
      for (int V = 0; V < nat; ++V)
        for (int b = 0; b < (int)P.nb[U].size(); ++b) {
          if (!B.o[B.io(q, U, V, b)]) continue;
          const NbEntry &e = P.nb[U][b];
          for (int c = e.col / 64; c <= (e.col + h.n_ao[e.K] - 1) / 64; ++c)
            z[(((size_t)q * nat + U) * nat + V) * max_chunks + c] = 0;
          *flops += 8.0 * h.n_aux[V] * h.n_ao[U] * h.n_ao[V] * h.n_ao[e.K];
        }
  return z;
}

// FP64 route, one batch of np points whose workspace starts at P.ws: gathered G operands Bg, Ag,
// the N- and X-step results, and O.
struct Fp64Ws {
  double *Bg, *Ag, *Nw, *Xw, *Ow;
};

Fp64Ws fp64_ws(Handle &h, long long npb) {
  const Chi0Plan &P = h.plan;
  Fp64Ws w;
  w.Bg = (double *)P.ws.p;
  w.Ag = w.Bg + npb * 2 * P.bg_sz;
  w.Nw = w.Ag + npb * 2 * P.ag_sz;
  w.Xw = w.Nw + npb * 2 * P.n_sz;
  w.Ow = w.Xw + npb * 2 * P.x_sz;
  return w;
}

void fp64_gather(Handle &h, const Point *dpts, int np, const Fp64Ws &w) {
  const Chi0Plan &P = h.plan;
  const int nat = h.natoms, nR = h.mesh.size(), nao = h.nao;
  const size_t g_gstride = (size_t)h.ntau * nR * nao * nao;
  int max_m = 0;
  for (int a = 0; a < nat; ++a) max_m = std::max(max_m, P.m[a]);
  dim3 grid((unsigned)(((long long)P.m_all * max_m + 255) / 256), (unsigned)(np * 2 * nat));
  k_gather_bg<<<grid, 256, 0, h.stream>>>(g_spin(h), g_gstride, dpts, (const int *)P.d_uni.p,
                                          (const int *)P.d_lam.p, (const long long *)P.t_lam_off.p,
                                          (const int *)P.t_m.p, (const long long *)P.t_bg_off.p, nat, P.m_all, nR,
                                          nao, h.mesh.n1, h.mesh.n2, h.mesh.n3, P.bg_sz, 2 * P.bg_sz, w.Bg);
  dim3 grid2((unsigned)(((long long)nao * max_m + 255) / 256), (unsigned)(np * 2 * nat));
  k_gather_ag<<<grid2, 256, 0, h.stream>>>(g_spin(h), g_gstride, dpts, (const int *)P.d_lam.p,
                                           (const long long *)P.t_lam_off.p, (const int *)P.t_m.p,
                                           (const long long *)P.t_ag_off.p, nat, nR, nao, h.mesh.n1, h.mesh.n2,
                                           h.mesh.n3, P.ag_sz, 2 * P.ag_sz, w.Ag);
  launch_counter() += 2;
  LR_CUDA(cudaGetLastError());
}

// N- and X-step descriptors of np points (appended to b).  nzN / nzX ([point][g][V], nullable):
// an operand without a kept G block under screening is exactly zero, and its GEMM runs with
// K = 0, which writes zeros.  Returns the algorithmic flops of the descriptors.
double fp64_nx(Handle &h, int np, const Fp64Ws &w, std::vector<DGemm> &b, const unsigned char *nzN = nullptr,
               const unsigned char *nzX = nullptr) {
  const Chi0Plan &P = h.plan;
  const double *Cp = (const double *)h.d_cpack.p;
  const int nat = h.natoms;
  double fl = 0;
  for (int q = 0; q < np; ++q)
    for (int g = 0; g < 2; ++g)
      for (int V = 0; V < nat; ++V) {
        const int rowsV = h.n_aux[V] * h.n_ao[V], mV = P.m[V];
        const size_t e = ((size_t)q * 2 + g) * nat + V;
        const int kn = !nzN || nzN[e] ? mV : 0, kx = !nzX || nzX[e] ? mV : 0;
        DGemm dn{Cp + P.cp_off[V], w.Bg + (size_t)q * 2 * P.bg_sz + g * P.bg_sz + P.bg_off[V],
                 w.Nw + (size_t)q * 2 * P.n_sz + g * P.n_sz + P.n_off[V], rowsV, P.m_all, kn, mV, mV, P.m_all,
                 1.0, 0.0};
        b.push_back(dn);
        DGemm dx{w.Ag + (size_t)q * 2 * P.ag_sz + g * P.ag_sz + P.ag_off[V], Cp + P.cp_off[V],
                 w.Xw + (size_t)q * 2 * P.x_sz + g * P.x_sz + P.x_off[V], h.nao, rowsV, kx, mV, mV, rowsV, 1.0, 0.0};
        b.push_back(dx);
        fl += 2.0 * rowsV * P.m_all * kn + 2.0 * h.nao * rowsV * kx;
      }
  return fl;
}

// final contraction chi0(R, tau)[U rows] = -s Cpack_U O_U^T of the points (appended to b)
void fp64_final(Handle &h, const std::vector<Point> &pts, const Fp64Ws &w, std::vector<DGemm> &b) {
  const Chi0Plan &P = h.plan;
  const double *Cp = (const double *)h.d_cpack.p;
  const int naux = h.naux, nR = h.mesh.size();
  const double spin = spin_factor(h), beta = h.cur_spin > 0 ? 1.0 : 0.0;
  for (size_t q = 0; q < pts.size(); ++q) {
    double *chi = (double *)h.d_chi_tau.p + ((size_t)pts[q].itau * nR + pts[q].iR) * naux * naux;
    for (int U = 0; U < h.natoms; ++U) {
      const int K = h.n_ao[U] * P.m[U];
      DGemm df{Cp + P.cp_off[U], w.Ow + q * P.o_sz + P.o_off[U], chi + (size_t)h.aux_off[U] * naux, h.n_aux[U],
               naux, K, K, K, naux, -spin, beta};
      b.push_back(df);
    }
  }
}

// Workspace of the tensor-core route for a batch of npb points: FP64 N, X, O and the digit planes
// of Bg, Ag and O (bounded by 2 GiB, at least one point).
struct TcWs {
  long long npb;
  size_t b_n, b_x, b_o, b_bg, b_ag, b_od, total;
};

TcWs tc_ws(const Handle &h, const Chi0Plan &P) {
  const int nat = h.natoms, S = h.chi0_S;
  const int rows_bg = 2 * nat * P.m_all, rows_ag = 2 * nat * h.nao, rows_o = nat * h.naux;
  const size_t fp = 8 * (size_t)(2 * P.n_sz + 2 * P.x_sz + P.o_sz);
  const size_t per_point = fp + oz::sliced_bytes(rows_bg, P.max_m, S) + oz::sliced_bytes(rows_ag, P.max_m, S) +
                           oz::sliced_bytes(rows_o, P.max_nm, S) + 4096;
  const long long total_pts = (long long)h.ntau * chi0_r_list(h.mesh).size();
  TcWs w;
  w.npb = std::min(std::max<long long>(1, (2LL << 30) / (long long)per_point), total_pts);
  w.b_n = 8 * (size_t)w.npb * 2 * P.n_sz;
  w.b_x = 8 * (size_t)w.npb * 2 * P.x_sz;
  w.b_o = 8 * (size_t)w.npb * P.o_sz;
  w.b_bg = oz::sliced_bytes((int)w.npb * rows_bg, P.max_m, S);
  w.b_ag = oz::sliced_bytes((int)w.npb * rows_ag, P.max_m, S);
  w.b_od = oz::sliced_bytes((int)w.npb * rows_o, P.max_nm, S);
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  w.total = al(w.b_n) + al(w.b_x) + al(w.b_o) + al(w.b_bg) + al(w.b_ag) + al(w.b_od) + 256;
  return w;
}

// Workspace of the FP64 route: gathered G operands, N, X and O for npb points (2^27 doubles,
// at least one point).
struct DpWs {
  long long npb, per_point;
  size_t total;
};

DpWs dp_ws(const Handle &h, const Chi0Plan &P, long long cap_doubles = 1LL << 27) {
  DpWs w;
  w.per_point = 2 * (P.bg_sz + P.ag_sz + P.n_sz + P.x_sz) + P.o_sz;
  const long long total_pts = (long long)h.ntau * chi0_r_list(h.mesh).size();
  w.npb = std::min(std::max<long long>(1, cap_doubles / std::max<long long>(1, w.per_point)), total_pts);
  w.total = (size_t)w.npb * w.per_point * sizeof(double);
  return w;
}

// One point batch of the tensor-core route of a handle: views of its workspace (FP64 N, X, O and the
// digit planes of Bg, Ag and O), the split operands and the GEMM entries of the three steps.
struct TcRound {
  std::vector<Point> pts;
  int np = 0;
  double *Nw = nullptr, *Xw = nullptr, *Ow = nullptr;
  char *wbg = nullptr, *wag = nullptr, *wod = nullptr;
  int *err = nullptr;
  oz::Sliced cpnx, cpf, sbg, sag, sod;
  std::vector<oz::Entry> en, ex, ef;
};

// workspace of h for its point batches (allocated), the error flag cleared; returns the views
TcRound tc_views(Handle &h, long long *npb) {
  Chi0Plan &P = h.plan;
  const TcWs tw = tc_ws(h, P);
  *npb = tw.npb;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  h.ensure(h.d_chi_tau, (size_t)h.ntau * h.mesh.size() * h.naux * h.naux * sizeof(double));
  h.ensure(P.ws, tw.total);
  TcRound r;
  char *w = (char *)P.ws.p;
  r.Nw = (double *)w;
  r.Xw = (double *)(w + al(tw.b_n));
  r.Ow = (double *)(w + al(tw.b_n) + al(tw.b_x));
  r.wbg = w + al(tw.b_n) + al(tw.b_x) + al(tw.b_o);
  r.wag = r.wbg + al(tw.b_bg);
  r.wod = r.wag + al(tw.b_ag);
  r.err = (int *)(r.wod + al(tw.b_od));
  LR_CUDA(cudaMemsetAsync(r.err, 0, 4, h.stream));
  oz::sliced_bind(r.cpnx, P.cp_nx.p, P.cpnx_rows, P.max_m, h.chi0_S);
  oz::sliced_bind(r.cpf, P.cp_f.p, h.naux, P.max_nm, h.chi0_S);
  return r;
}

// points r.pts: upload them, split the gathered Green's-function operands into digit planes and
// build the N- and X-step entries
void tc_gather(Handle &h, TcRound &r) {
  Chi0Plan &P = h.plan;
  const int nat = h.natoms, nR = h.mesh.size(), nao = h.nao, S = h.chi0_S;
  const int np = r.np = (int)r.pts.size();
  cudaStream_t s = h.stream;
  h.upload_async(P.t_pts, r.pts.data(), np * sizeof(Point));
  oz::GatherSrc gs;
  gs.kind = 0;
  gs.G = g_spin(h);
  gs.g_gstride = (long long)h.ntau * nR * nao * nao;
  gs.nR = nR;
  gs.nao = nao;
  gs.n1 = h.mesh.n1;
  gs.n2 = h.mesh.n2;
  gs.n3 = h.mesh.n3;
  gs.natoms = nat;
  gs.rows_per_entry = P.m_all;
  gs.pts = (const int *)P.t_pts.p;
  gs.uni = (const int *)P.d_uni.p;
  gs.lam = (const int *)P.d_lam.p;
  gs.lam_off = (const long long *)P.t_lam_off.p;
  gs.m = (const int *)P.t_m.p;
  const int rows_bg = 2 * nat * P.m_all, rows_ag = 2 * nat * nao, rows_o = nat * h.naux;
  oz::sliced_bind(r.sbg, r.wbg, np * rows_bg, P.max_m, S);
  oz::sliced_bind(r.sag, r.wag, np * rows_ag, P.max_m, S);
  oz::sliced_bind(r.sod, r.wod, np * rows_o, P.max_nm, S);
  oz::split_gather(gs, np * rows_bg, P.max_m, r.sbg, s);
  gs.kind = 1;
  gs.rows_per_entry = nao;
  oz::split_gather(gs, np * rows_ag, P.max_m, r.sag, s);
  // N-step: N_V = Cpack_V Bg_V^T;  X-step: X_V = Ag_V Cpack_V^T, both as FP32 pairs (hi, lo): the O
  // assembly reads the pair (FP32-pair arithmetic) or its hi part (FP32 arithmetic)
  const bool pairs = true;
  (void)S;
  r.en.clear();
  r.ex.clear();
  for (int q = 0; q < np; ++q)
    for (int g = 0; g < 2; ++g)
      for (int V = 0; V < nat; ++V) {
        const int rowsV = h.n_aux[V] * h.n_ao[V], e = (q * 2 + g) * nat + V;
        oz::Entry a{};
        a.a_row0 = P.cpnx_off[V];
        a.b_row0 = e * P.m_all;
        a.M = rowsV;
        a.N = P.m_all;
        a.K = P.m[V];
        a.C = r.Nw + (size_t)q * 2 * P.n_sz + g * P.n_sz + P.n_off[V];
        a.ldc = P.m_all;
        a.alpha = 1.0;
        a.mode = pairs ? 3 : 0;
        r.en.push_back(a);
        oz::Entry b{};
        b.a_row0 = e * nao;
        b.b_row0 = P.cpnx_off[V];
        b.M = nao;
        b.N = rowsV;
        b.K = P.m[V];
        b.C = r.Xw + (size_t)q * 2 * P.x_sz + g * P.x_sz + P.x_off[V];
        b.mode = pairs ? 3 : 0;
        b.ldc = rowsV;
        b.alpha = 1.0;
        r.ex.push_back(b);
      }
}

// O = M + M* + Z + Z* of the round (zero: screening flags or NULL), its digit planes (rows nu per
// (point, U), K = n_U m_U), and the final-contraction entries
void tc_assemble(Handle &h, TcRound &r, const unsigned char *zero) {
  Chi0Plan &P = h.plan;
  const int nat = h.natoms, nR = h.mesh.size(), naux = h.naux, np = r.np;
  // the 3-plane kernel builds the row exponents when O is split into at most 3 digit planes (the
  // plain BF16 / TF32 operands have none)
  int *rexp = h.chi0_S >= 1 && h.chi0_S <= 3 ? r.sod.expo : nullptr;
  if (rexp) oz::expo_init(r.sod, np * nat * naux, h.stream);
  const bool expo_given = run_oassemble(h, (const Point *)P.t_pts.p, np, r.Nw, r.Xw, r.Ow, zero, rexp);
  std::vector<long long> off(np * nat);
  std::vector<int> ke(np * nat);
  for (int q = 0; q < np; ++q)
    for (int U = 0; U < nat; ++U) {
      off[q * nat + U] = (long long)q * P.o_sz + P.o_off[U];
      ke[q * nat + U] = h.n_ao[U] * P.m[U];
    }
  h.upload_async(P.t_oe_off, off.data(), off.size() * 8);
  h.upload_async(P.t_oe_k, ke.data(), ke.size() * 4);
  oz::split_ragged(r.Ow, (const long long *)P.t_oe_off.p, (const int *)P.t_oe_k.p, naux, np * nat, P.max_nm, r.sod,
                   h.stream, expo_given);
  const double spin = spin_factor(h);
  r.ef.clear();
  for (int q = 0; q < np; ++q) {
    double *chi = (double *)h.d_chi_tau.p + ((size_t)r.pts[q].itau * nR + r.pts[q].iR) * naux * naux;
    for (int U = 0; U < nat; ++U) {
      // chi0[U rows]^T = O_U . Cpack_U^T: rows nu (N_aux of them fill the 128-row tiles), columns
      // mu of U, stored transposed into chi0[mu][nu]
      oz::Entry f{};
      f.a_row0 = (q * nat + U) * naux;
      f.b_row0 = h.aux_off[U];
      f.M = naux;
      f.N = h.n_aux[U];
      f.K = h.n_ao[U] * P.m[U];
      f.C = chi + (size_t)h.aux_off[U] * naux;
      f.ldc = naux;
      f.mode = 4;
      f.alpha = -spin;
      f.beta = h.cur_spin > 0 ? 1.0 : 0.0;
      r.ef.push_back(f);
    }
  }
}

void tc_check(Handle &h, const int *err) {
  int e_host = 0;
  LR_CUDA(cudaMemcpyAsync(&e_host, err, 4, cudaMemcpyDeviceToHost, h.stream));
  LR_CUDA(cudaStreamSynchronize(h.stream));
  if (e_host) throw Error{LIBRPA_E_TIMEOUT, "chi0: a bounded wait in the tensor-core GEMM ran out"};
}

// Tensor-core route: the N, X and final GEMMs on digit planes (S = h.chi0_S).
void chi0_run_tc(Handle &h) {
  Chi0Plan &P = h.plan;
  const int nat = h.natoms, nR = h.mesh.size(), ntau = h.ntau, naux = h.naux;
  const bool scr = h.g_screen > 0;
  cudaStream_t s = h.stream;
  const std::vector<int> rl = chi0_r_list(h.mesh);
  long long npb = 1;
  TcRound r = tc_views(h, &npb);
  // under screening, points left out keep chi0 = 0 (the second spin channel accumulates)
  if (scr) LR_CUDA(cudaMemsetAsync(h.d_chi_tau.p, 0, (size_t)ntau * nR * naux * naux * sizeof(double), s));
  h.flop_chi0_run = 0;
  for (h.cur_spin = 0; h.cur_spin < h.nspins; ++h.cur_spin) {
    const ScreenSel sel = screen_select(h, rl);
    const long long total_pts = (long long)sel.pts.size();
    h.stats.n_points_chi0 += total_pts;
    h.stats.n_points_skipped += sel.skipped;
    for (long long p0 = 0; p0 < total_pts; p0 += npb) {
      const int np = (int)std::min(npb, total_pts - p0);
      r.pts.assign(sel.pts.begin() + p0, sel.pts.begin() + p0 + np);
      tc_gather(h, r);
      // screening: tiles sum only the K stages that meet kept G blocks, O blocks without a kept
      // contribution are written as zeros (see BlockSparse)
      BlockSparse B;
      if (scr) B = block_sparse(h, r.pts);
      ChunkMemo memo_n, memo_x, memo_f;
      const oz::StageFn fn_n = [&](int e, int, int, int n0, int cols, int cs, int K, std::vector<int> &out) {
        memo_n.get(e, n0, cs, out, [&](std::vector<int> &o) {
          chunks_n(h, B, e / (2 * nat), (e / nat) % 2, e % nat, n0, cols, cs, K, o);
        });
        return true;
      };
      const oz::StageFn fn_x = [&](int e, int m0, int rows, int, int, int cs, int K, std::vector<int> &out) {
        memo_x.get(e, m0, cs, out, [&](std::vector<int> &o) {
          chunks_x(h, B, e / (2 * nat), (e / nat) % 2, e % nat, m0, rows, cs, K, o);
        });
        return true;
      };
      const oz::StageFn fn_f = [&](int e, int m0, int rows, int, int, int cs, int K, std::vector<int> &out) {
        memo_f.get(e, m0, cs, out, [&](std::vector<int> &o) { chunks_f(h, B, e / nat, e % nat, m0, rows, cs, K, o); });
        return true;
      };
      h.flop_chi0_run += timed_grouped(h, r.cpnx, r.sbg, r.en, r.err, P.gargs1, scr ? &fn_n : nullptr);
      h.flop_chi0_run += timed_grouped(h, r.sag, r.cpnx, r.ex, r.err, P.gargs2, scr ? &fn_x : nullptr);
      std::vector<unsigned char> zf;
      if (scr) {
        double fo = 0;
        zf = ozero_flags(h, B, oasm_chunks(h), &fo);
        h.upload_async(P.t_ozero, zf.data(), zf.size());
        h.flop_chi0_run += fo;
      } else {
        h.flop_chi0_run += np * (P.flop_per_point - P.flop_nx_per_point - P.flop_fin_per_point);
      }
      tc_assemble(h, r, scr ? (const unsigned char *)P.t_ozero.p : nullptr);
      h.flop_chi0_run += timed_grouped(h, r.sod, r.cpf, r.ef, r.err, P.gargs3, scr ? &fn_f : nullptr);
    }
  }
  h.cur_spin = 0;
  fill_partners(h);
  tc_check(h, r.err);
}

// the same for several handles at once, on hs[0]'s stream (see chi0_run_tc_merged)
void tc_merged(std::vector<Handle *> &hs) {
  Handle &h0 = *hs[0];
  const size_t nh = hs.size();
  std::vector<TcRound> rs(nh);
  std::vector<long long> npb(nh);
  std::vector<std::vector<Point>> pts(nh);
  int rounds = 0;
  for (size_t i = 0; i < nh; ++i) {
    Handle &h = *hs[i];
    h.cur_spin = 0;
    rs[i] = tc_views(h, &npb[i]);
    const std::vector<int> rl = chi0_r_list(h.mesh);
    pts[i] = make_points(h, rl, 0, (int)(h.ntau * rl.size()));
    h.stats.n_points_chi0 = (long long)pts[i].size();
    h.flop_chi0_run = pts[i].size() * h.plan.flop_per_point;
    rounds = std::max(rounds, (int)((pts[i].size() + npb[i] - 1) / npb[i]));
  }
  auto launch = [&](int step) {   // 0: N, 1: X, 2: final; every handle's entries in one launch
    std::vector<std::pair<const oz::Sliced *, const oz::Sliced *>> ops;
    std::vector<oz::Entry> es;
    for (size_t i = 0; i < nh; ++i) {
      TcRound &r = rs[i];
      if (!r.np) continue;
      const int pair = (int)ops.size();
      if (step == 0) ops.push_back({&r.cpnx, &r.sbg});
      if (step == 1) ops.push_back({&r.sag, &r.cpnx});
      if (step == 2) ops.push_back({&r.sod, &r.cpf});
      for (oz::Entry e : step == 0 ? r.en : step == 1 ? r.ex : r.ef) {
        e.pair = pair;
        es.push_back(e);
      }
    }
    Handle::Timed t{nullptr, nullptr, 0, 0};
    LR_CUDA(cudaEventCreate(&t.a));
    LR_CUDA(cudaEventCreate(&t.b));
    LR_CUDA(cudaEventRecord(t.a, h0.stream));
    DevBuf &args = step == 0 ? h0.plan.gargs1 : step == 1 ? h0.plan.gargs2 : h0.plan.gargs3;
    oz::gemm_multi(ops, es, rs[0].err, h0.stream, h0, args);
    LR_CUDA(cudaEventRecord(t.b, h0.stream));
    t.flops = h0.oz_alg_flops;
    t.exec_flops = h0.oz_exec_flops;
    h0.timed.push_back(t);
  };
  for (int r = 0; r < rounds; ++r) {
    for (size_t i = 0; i < nh; ++i) {
      const long long p0 = (long long)r * npb[i];
      const long long np = std::max<long long>(0, std::min<long long>(npb[i], (long long)pts[i].size() - p0));
      rs[i].pts.assign(pts[i].begin() + p0, pts[i].begin() + p0 + np);
      rs[i].np = (int)np;
      if (np) tc_gather(*hs[i], rs[i]);
    }
    launch(0);
    launch(1);
    for (size_t i = 0; i < nh; ++i)
      if (rs[i].np) tc_assemble(*hs[i], rs[i], nullptr);
    launch(2);
  }
  for (size_t i = 0; i < nh; ++i) fill_partners(*hs[i]);
  tc_check(h0, rs[0].err);
}

}  // namespace

void chi0_run(Handle &h, double *ms_gemm) {
  if (ms_gemm) *ms_gemm = 0;
  if (h.chi0_S >= 0) {
    chi0_run_tc(h);
    return;
  }
  Chi0Plan &P = h.plan;
  const int nR = h.mesh.size(), ntau = h.ntau, naux = h.naux;
  cudaStream_t s = h.stream;
  h.ensure(h.d_chi_tau, (size_t)ntau * nR * naux * naux * sizeof(double));
  const std::vector<int> rl = chi0_r_list(h.mesh);
  const DpWs dw = dp_ws(h, P);
  const long long npb = dw.npb;
  h.ensure(P.ws, dw.total);
  const Fp64Ws w = fp64_ws(h, npb);
  const bool scr = h.g_screen > 0;
  // under screening, points left out keep chi0 = 0 (the second spin channel accumulates)
  if (scr) LR_CUDA(cudaMemsetAsync(h.d_chi_tau.p, 0, (size_t)ntau * nR * naux * naux * sizeof(double), s));
  h.flop_chi0_run = 0;
  for (h.cur_spin = 0; h.cur_spin < h.nspins; ++h.cur_spin) {
    const ScreenSel sel = screen_select(h, rl);
    const long long total_pts = (long long)sel.pts.size();
    h.stats.n_points_chi0 += total_pts;
    h.stats.n_points_skipped += sel.skipped;
    for (long long p0 = 0; p0 < total_pts; p0 += npb) {
      const int np = (int)std::min(npb, total_pts - p0);
      std::vector<Point> pts(sel.pts.begin() + p0, sel.pts.begin() + p0 + np);
      h.upload_async(P.t_pts, pts.data(), np * sizeof(Point));
      const Point *dpts = (const Point *)P.t_pts.p;
      fp64_gather(h, dpts, np, w);
      std::vector<DGemm> b1, b2;
      const size_t z = (size_t)p0 * 2 * h.natoms;
      if (!scr) {
        h.flop_chi0_run += fp64_nx(h, np, w, b1);
        h.flop_chi0_run += np * (P.flop_per_point - P.flop_nx_per_point);
        dgemm_batched(h, b1, s, P.gargs1, &P.var_nx);
        run_oassemble(h, dpts, np, w.Nw, w.Xw, w.Ow);
        fp64_final(h, pts, w, b2);
        dgemm_batched(h, b2, s, P.gargs2, &P.var_fin);
        continue;
      }
      // screening: the GEMM tiles sum only the K chunks that meet kept G blocks, and O blocks with
      // no kept contribution are written as zeros
      const BlockSparse B = block_sparse(h, pts);
      const int nat = h.natoms;
      // an N-step tile's chunks depend on its columns only, an X-step tile's on its rows, a final
      // tile's on its columns: one list per (entry, tile column or row)
      ChunkMemo memo_nx, memo_f;
      const ChunkFn fnx = [&](int e, int m0, int rows, int n0, int cols, int cs, int K, std::vector<int> &out) {
        const int r = e / 2, V = r % nat, g = (r / nat) % 2, q = r / (2 * nat);
        memo_nx.get(e, e % 2 == 0 ? n0 : m0, cs, out, [&](std::vector<int> &o) {
          if (e % 2 == 0)
            chunks_n(h, B, q, g, V, n0, cols, cs, K, o);
          else
            chunks_x(h, B, q, g, V, m0, rows, cs, K, o);
        });
        return true;
      };
      const ChunkFn ff = [&](int e, int, int, int n0, int cols, int cs, int K, std::vector<int> &out) {
        memo_f.get(e, n0, cs, out, [&](std::vector<int> &o) { chunks_f(h, B, e / nat, e % nat, n0, cols, cs, K, o); });
        return true;
      };
      fp64_nx(h, np, w, b1, sel.nzN.data() + z, sel.nzX.data() + z);
      h.flop_chi0_run += dgemm_batched(h, b1, s, P.gargs1, &P.var_nx, &fnx);
      double fo = 0;
      const std::vector<unsigned char> zf = ozero_flags(h, B, oasm_chunks(h), &fo);
      h.upload_async(P.t_ozero, zf.data(), zf.size());
      run_oassemble(h, dpts, np, w.Nw, w.Xw, w.Ow, (const unsigned char *)P.t_ozero.p);
      h.flop_chi0_run += fo;
      fp64_final(h, pts, w, b2);
      h.flop_chi0_run += dgemm_batched(h, b2, s, P.gargs2, &P.var_fin, &ff);
    }
  }
  h.cur_spin = 0;
  fill_partners(h);
  LR_CUDA(cudaStreamSynchronize(s));
  if (ms_gemm) *ms_gemm = 0;
}

bool chi0_run_merged(std::vector<Handle *> &hs, MergedChi0 &m) {
  if (hs.empty()) return false;
  Handle &h0 = *hs[0];
  cudaStream_t s = h0.stream;
  const size_t nh = hs.size();
  bool fresh = m.gens.size() != nh;
  for (size_t i = 0; i < nh && !fresh; ++i) fresh = m.gens[i] != hs[i]->plan.gen || m.hs[i] != hs[i];
  for (Handle *h : hs) h->cur_spin = 0;   // one channel (nspins = 1 handles only)
  if (fresh) {
    if (!m.hs.empty() && m.hs[0] != hs[0]) {   // descriptor buffers belong to the old first handle
      for (DevBuf &d : m.nx_args) m.hs[0]->release(d);
      for (DevBuf &d : m.fin_args) m.hs[0]->release(d);
      m.nx_args.clear();
      m.fin_args.clear();
    }
    m.reset();
    m.hs = hs;
    m.gens.clear();
    for (Handle *h : hs) m.gens.push_back(h->plan.gen);
  }
  // per handle: chi0(R, tau), a workspace for npb points (at most 16 GiB over the batch), all its
  // points resident, and the number of rounds it takes
  const long long cap = std::max<long long>(1LL << 24, std::min<long long>(1LL << 27, (2LL << 30) / (long long)nh));
  std::vector<Fp64Ws> ws(nh);
  std::vector<std::vector<Point>> pts(nh);
  std::vector<long long> npb(nh);
  int rounds = 0;
  for (size_t i = 0; i < nh; ++i) {
    Handle &h = *hs[i];
    Chi0Plan &P = h.plan;
    h.ensure(h.d_chi_tau, (size_t)h.ntau * h.mesh.size() * h.naux * h.naux * sizeof(double));
    const DpWs dw = dp_ws(h, P, cap);
    h.ensure(P.ws, dw.total);
    ws[i] = fp64_ws(h, dw.npb);
    npb[i] = dw.npb;
    const std::vector<int> rl = chi0_r_list(h.mesh);
    pts[i] = make_points(h, rl, 0, (int)(h.ntau * rl.size()));
    h.stats.n_points_chi0 = (long long)pts[i].size();
    h.flop_chi0_run = pts[i].size() * P.flop_per_point;
    rounds = std::max(rounds, (int)((pts[i].size() + npb[i] - 1) / npb[i]));
    if (fresh) {
      h.ensure(P.t_pts, pts[i].size() * sizeof(Point));
      LR_CUDA(cudaMemcpyAsync(P.t_pts.p, pts[i].data(), pts[i].size() * sizeof(Point), cudaMemcpyHostToDevice, s));
    }
  }
  if (m.exec) {   // replay the captured sequence
    LR_CUDA(cudaGraphLaunch(m.exec, s));
    launch_counter() += m.nodes;
    LR_CUDA(cudaStreamSynchronize(s));
    return true;
  }
  // descriptors of every round: round r takes points [r npb_i, (r + 1) npb_i) of handle i
  auto slice = [&](size_t i, int r, long long &p0, int &np) {
    p0 = (long long)r * npb[i];
    np = (int)std::max<long long>(0, std::min<long long>(npb[i], (long long)pts[i].size() - p0));
  };
  std::vector<std::vector<DGemm>> b1(rounds), b2(rounds);
  for (int r = 0; r < rounds; ++r)
    for (size_t i = 0; i < nh; ++i) {
      long long p0;
      int np;
      slice(i, r, p0, np);
      if (!np) continue;
      fp64_nx(*hs[i], np, ws[i], b1[r]);
      fp64_final(*hs[i], std::vector<Point>(pts[i].begin() + p0, pts[i].begin() + p0 + np), ws[i], b2[r]);
    }
  m.nx_args.resize(rounds);
  m.fin_args.resize(rounds);
  std::vector<DLaunch> L1(rounds), L2(rounds);
  // the whole sequence; tile variants are tuned on the first pass (eagerly), then the same
  // launches are captured into a graph for the next calls
  auto sequence = [&](bool first) {
    for (int r = 0; r < rounds; ++r) {
      for (size_t i = 0; i < nh; ++i) {
        long long p0;
        int np;
        slice(i, r, p0, np);
        if (np) fp64_gather(*hs[i], (const Point *)hs[i]->plan.t_pts.p + p0, np, ws[i]);
      }
      if (first) {
        if (m.var_nx < 0) m.var_nx = dgemm_autotune(h0, b1[r], s, m.nx_args[r]);
        L1[r] = dgemm_prepare(h0, b1[r], m.var_nx, s, m.nx_args[r]);
      }
      dgemm_launch(h0, L1[r], s, first);
      for (size_t i = 0; i < nh; ++i) {
        long long p0;
        int np;
        slice(i, r, p0, np);
        if (np) run_oassemble(*hs[i], (const Point *)hs[i]->plan.t_pts.p + p0, np, ws[i].Nw, ws[i].Xw, ws[i].Ow);
      }
      if (first) {
        if (m.var_fin < 0) m.var_fin = dgemm_autotune(h0, b2[r], s, m.fin_args[r]);
        L2[r] = dgemm_prepare(h0, b2[r], m.var_fin, s, m.fin_args[r]);
      }
      dgemm_launch(h0, L2[r], s, first);
    }
    for (Handle *h : hs) fill_partners(*h);
  };
  sequence(true);
  LR_CUDA(cudaStreamSynchronize(s));
  if (m.graph_failed) return false;
  const long long c1 = launch_counter();
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    m.graph_failed = true;
    return false;
  }
  bool ok = true;
  try {
    sequence(false);
  } catch (const Error &) {
    ok = false;
  }
  if (cudaStreamEndCapture(s, &g) != cudaSuccess || !ok || !g ||
      cudaGraphInstantiate(&m.exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    m.exec = nullptr;
    m.graph_failed = true;
  }
  if (g) cudaGraphDestroy(g);
  m.nodes = launch_counter() - c1;
  launch_counter() = c1;   // captured launches did not run
  return false;
}

bool chi0_fits_one_batch(const Handle &h) { return h.chi0_S < 0 && h.nspins == 1 && !(h.g_screen > 0); }

bool chi0_fits_tc_batch(const Handle &h) { return h.chi0_S >= 0 && h.nspins == 1 && !(h.g_screen > 0); }

void chi0_run_tc_merged(std::vector<Handle *> &hs) {
  if (hs.empty()) return;
  for (Handle *h : hs)
    if (!chi0_fits_tc_batch(*h) || h->chi0_S != hs[0]->chi0_S || h->stream != hs[0]->stream)
      throw Error{LIBRPA_E_ARG, "chi0_run_tc_merged: handles of different kinds or streams"};
  tc_merged(hs);
}

void MergedChi0::reset() {
  if (exec) cudaGraphExecDestroy(exec);
  exec = nullptr;
  graph_failed = false;
  nodes = 0;
}

size_t chi0_device_bytes(const Handle &h, const Chi0Plan &P) {
  size_t b = (size_t)P.cp_total * 8;                                    // packed C
  b += (size_t)h.ntau * h.mesh.size() * h.naux * h.naux * 8;            // chi0(R, tau)
  b += h.chi0_S >= 0 ? tc_ws(h, P).total : dp_ws(h, P).total;           // batch workspace
  if (h.chi0_S >= 0)                                                    // digit planes of C
    b += oz::sliced_bytes(P.cpnx_rows, P.max_m, h.chi0_S) + oz::sliced_bytes(h.naux, P.max_nm, h.chi0_S);
  // column tables and per-atom tables
  size_t cols = 0;
  for (int a = 0; a < h.natoms; ++a) cols += P.m[a];
  b += (2 * cols + (size_t)P.m_all) * 6 * sizeof(int) + 16 * (size_t)(h.natoms + 1) * 8 + 12 * 256;
  return b;
}

std::vector<int> chi0_r_list(const Mesh &m) {
  std::vector<int> rl;
  for (int i = 0; i < m.size(); ++i)
    if (i <= m.neg(i)) rl.push_back(i);
  return rl;
}

}  // namespace librpa
