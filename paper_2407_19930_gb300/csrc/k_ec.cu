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
#include <cmath>
#include <vector>

#include "internal.h"
#include "ozgemm.h"

namespace librpa {
namespace {

constexpr int NB = 64;

// Factor the NB x NB diagonal block at p0 of every matrix in place (lower triangle).  One CTA per
// matrix.  Adds 2 sum ln d_jj to lndet[b]; sets info[b] = 1 on a non-positive pivot.
__global__ void __launch_bounds__(256) k_potrf_diag(double2 *const *mats, int n, int ld, int p0, double *lndet,
                                                    int *info) {
  extern __shared__ double2 a[];   // [NB][NB + 1]
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

// Largest |V(-q) - conj V(q)| over the pairs q < -q (res[0]) and largest |V(q)| (res[1]), as the
// bit patterns of non-negative doubles (ordered like the values) for atomicMax.
__global__ void k_conj_check(const double2 *V, int n, int n1, int n2, int n3, unsigned long long *res) {
  const int q = blockIdx.y;
  const int a = q / (n2 * n3), b = (q / n3) % n2, c = q % n3;
  const int p = (((n1 - a) % n1) * n2 + (n2 - b) % n2) * n3 + (n3 - c) % n3;
  if (p <= q) return;
  const size_t nn = (size_t)n * n;
  const double2 *Vq = V + nn * q, *Vp = V + nn * p;
  double d = 0.0, m = 0.0;
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < nn; x += (size_t)gridDim.x * blockDim.x) {
    const double2 u = Vq[x], v = Vp[x];
    d = fmax(d, fmax(fabs(v.x - u.x), fabs(v.y + u.y)));
    m = fmax(m, fmax(fabs(u.x), fabs(u.y)));
    if (isnan(u.x + u.y + v.x + v.y)) d = INFINITY;
  }
  for (int o = 16; o > 0; o >>= 1) {
    d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(res, (unsigned long long)__double_as_longlong(d));
    atomicMax(res + 1, (unsigned long long)__double_as_longlong(m));
  }
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

// K6: E_c, per-q and per-omega parts from the per-(q, omega) ln det and trace.
__global__ void k_energy(const double *lndet, const double *trace, const double *w_omega, int nq, int nw,
                         double *out /* [1 + nq + nw] */) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double pref = 1.0 / (2.0 * M_PI * nq);
  double tot = 0.0;
  for (int k = 0; k < nw; ++k) out[1 + nq + k] = 0.0;
  for (int q = 0; q < nq; ++q) {
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
  int *err = nullptr;
  int S = 0;
};

// Blocked Cholesky of `mats` (n x n, lower, in place, uniform stride when tc != nullptr), in step.
void potrf_batched(Handle &h, double2 *const *d_mats, const std::vector<double2 *> &mats, int n, int ld,
                   double *lndet, int *info, TcScratch *tc) {
  cudaStream_t s = h.stream;
  const int B = (int)mats.size();
  const size_t smem = (size_t)NB * (NB + 1) * sizeof(double2);
  LR_CUDA(cudaFuncSetAttribute(k_potrf_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LR_CUDA(cudaFuncSetAttribute(k_trsm_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * smem)));
  const long long bstride = B > 1 ? (long long)(mats[1] - mats[0]) : 0;
  for (int p0 = 0; p0 < n; p0 += NB) {
    k_potrf_diag<<<B, 256, smem, s>>>(d_mats, n, ld, p0, lndet, info);
    ++launch_counter();
    const int nb = std::min(NB, n - p0), rest = n - p0 - nb;
    if (rest <= 0) break;
    dim3 g((unsigned)((rest + 63) / 64), (unsigned)B);
    k_trsm_panel<<<g, 64, 2 * smem, s>>>(d_mats, n, ld, p0);
    ++launch_counter();
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

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// Workspace of the ln det stage: L[nq], W[nw], A[nw] (complex n x n), pointer tables,
// lndet/trace/info, output, and for the tensor-core route the digit planes.
struct EcLayout {
  size_t o_L, o_W, o_A, o_ptr, o_ld, o_tr, o_ldc, o_trc, o_inf, o_out, o_wo, o_err;
  size_t o_sx = 0, o_sw = 0, o_sl = 0, o_slh = 0, o_pa = 0, o_pb = 0;
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
  l.o_err = take(4);
  if (S >= 0) {
    l.o_sx = take(oz::sliced_bytes(nw * 2 * n, 2 * n, S));
    l.o_sw = take(oz::sliced_bytes(nw * n, 2 * n, S));
    l.o_sl = take(oz::sliced_bytes(n, 2 * n, S));
    l.o_slh = take(oz::sliced_bytes(2 * n, 2 * n, S));
    l.o_pa = take(oz::sliced_bytes(bmax * 2 * n, 2 * NB, S));
    l.o_pb = take(oz::sliced_bytes(bmax * n, 2 * NB, S));
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
  TcScratch tcs;
  TcScratch *tc = nullptr;
  oz::Sliced sx, sw, sl, slh;
  if (S >= 0) {
    tcs.S = S;
    tcs.err = err;
    oz::sliced_bind(tcs.pa, w + o_pa, bmax * 2 * n, 2 * NB, S);
    oz::sliced_bind(tcs.pb, w + o_pb, bmax * n, 2 * NB, S);
    oz::sliced_bind(sx, w + o_sx, nw * 2 * n, 2 * n, S);
    oz::sliced_bind(sw, w + o_sw, nw * n, 2 * n, S);
    oz::sliced_bind(sl, w + o_sl, n, 2 * n, S);
    oz::sliced_bind(slh, w + o_slh, 2 * n, 2 * n, S);
    tc = &tcs;
  }
  // q <-> -q: chi0(R) is real, so chi0(-q) = conj chi0(q); when also V(-q) = conj V(q) (to 1e-12
  // of max |V|), the integrand of -q equals that of q (ln det and trace of complex-conjugate
  // matrices), and only q <= -q is computed.  The check runs once per set of V(q).
  if (h.vq_sym < 0) {
    unsigned long long *res = (unsigned long long *)(w + o_ld);   // lndet is cleared again below
    LR_CUDA(cudaMemsetAsync(res, 0, 16, s));
    k_conj_check<<<dim3(64, (unsigned)nq), 256, 0, s>>>((const double2 *)h.d_vq.p, n, h.mesh.n1, h.mesh.n2,
                                                        h.mesh.n3, res);
    ++launch_counter();
    LR_CUDA(cudaGetLastError());
    double dm[2] = {0, 0};
    LR_CUDA(cudaMemcpyAsync(dm, res, 16, cudaMemcpyDeviceToHost, s));
    LR_CUDA(cudaStreamSynchronize(s));
    h.vq_sym = dm[0] <= 1e-12 * dm[1] ? 1 : 0;
    LR_CUDA(cudaMemsetAsync(lndet, 0, 16, s));
  }
  std::vector<int> qlist;
  for (int q = 0; q < nq; ++q)
    if (h.vq_sym != 1 || q <= h.mesh.neg(q)) qlist.push_back(q);
  const int nql = (int)qlist.size();
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
  // A(q, omega) of the q of a chunk, packed: A[(qi - c0) * nw + k]; each chunk is factorised in
  // one lockstep batch
  double2 **aptr = ptrs + nq;
  double *lndet_c = (double *)(w + lay.o_ldc), *trace_c = (double *)(w + lay.o_trc);
  LR_CUDA(cudaMemsetAsync(lndet_c, 0, (size_t)nql * nw * 8, s));
  // algorithmic work (8 flops per complex MAC): W = chi0 L with L lower triangular,
  // sum_j (n - j) = n (n + 1) / 2 MACs per row; A = -L^H W on the lower triangle,
  // sum_{i >= j} (n - i) MACs per matrix
  const double dn = n;
  const double fl_w = 8.0 * nw * dn * (dn * (dn + 1) / 2), fl_a = 8.0 * nw * (dn * (dn + 1) * (dn + 2) / 6);
  // FP64 route: A needs W only on and below its diagonal tiles (j >= k), sum_k (n - k)^2 MACs
  const double fl_w_lower = 8.0 * nw * (dn * (dn + 1) * (2 * dn + 1) / 6);
  for (int c0 = 0; c0 < nql; c0 += nc) {
    const int c1 = std::min(nql, c0 + nc);
    std::vector<double2 *> ap((size_t)(c1 - c0) * nw);
    for (size_t b = 0; b < ap.size(); ++b) ap[b] = Am + b * n2;
    LR_CUDA(cudaMemcpyAsync(aptr, ap.data(), ap.size() * 8, cudaMemcpyHostToDevice, s));
    for (int qi = c0; qi < c1; ++qi) {
      const int q = qlist[qi];
      double2 *Aq = Am + (size_t)(qi - c0) * nw * n2;
      if (S >= 0) {
        const double2 *L = Lq + (size_t)qi * n2;
        oz::split_complex(L, n, oz::OP_N, false, n, n, 1, 0, sl, s);     // B'^T of W = chi0 L
        oz::split_complex(L, n, oz::OP_H, true, n, n, 1, 0, slh, s);     // A' of L^H W
        oz::split_complex(chi + (size_t)q * nw * n2, n, oz::OP_N, true, n, n, nw, (long long)n2, sx, s);
        oz::Out o1;   // W^T, so that the second GEMM reads W column by column as rows
        o1.C = (double *)Wm;
        o1.ldc = n;
        o1.batch_stride = (long long)n2;
        o1.mode = 2;
        Handle::Timed t1{nullptr, nullptr, fl_w, 1};
        LR_CUDA(cudaEventCreate(&t1.a));
        LR_CUDA(cudaEventCreate(&t1.b));
        LR_CUDA(cudaEventRecord(t1.a, s));
        oz::gemm(sx, sl, 2 * n, n, nw, o1, 0, 2, 0, err, s, h);
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
    potrf_batched(h, aptr, ap, n, n, lndet_c + (size_t)c0 * nw, info + nq + (size_t)c0 * nw, tc);
  }
  for (int qi = 0; qi < nql; ++qi) {   // to the flat (q, omega) order
    const int q = qlist[qi];
    LR_CUDA(cudaMemcpyAsync(lndet + (size_t)q * nw, lndet_c + (size_t)qi * nw, nw * 8, cudaMemcpyDeviceToDevice, s));
    LR_CUDA(cudaMemcpyAsync(trace + (size_t)q * nw, trace_c + (size_t)qi * nw, nw * 8, cudaMemcpyDeviceToDevice, s));
  }
  for (int q : qlist) {   // the integrands of -q
    const int p = h.mesh.neg(q);
    if (p == q || h.vq_sym != 1) continue;
    LR_CUDA(cudaMemcpyAsync(lndet + (size_t)p * nw, lndet + (size_t)q * nw, nw * 8, cudaMemcpyDeviceToDevice, s));
    LR_CUDA(cudaMemcpyAsync(trace + (size_t)p * nw, trace + (size_t)q * nw, nw * 8, cudaMemcpyDeviceToDevice, s));
  }
  k_energy<<<1, 1, 0, s>>>(lndet, trace, wo, nq, nw, out);
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
  // flop count of this stage (complex MAC = 8 real flops): per q (4/3 n^3 real for the Cholesky of
  // V), per (q, omega): W = chi0 L (n^3/2 MAC), L^H W lower (n^3/6 MAC), Cholesky (n^3/6 MAC)
  const double n3 = (double)n * n * n;
  h.stats.flop_ec = nql * (8.0 * n3 / 6.0) + (double)nql * nw * 8.0 * ((S >= 0 ? n3 / 2 : n3 / 3) + n3 / 6 + n3 / 6);
  return LIBRPA_OK;
}

}  // namespace librpa
