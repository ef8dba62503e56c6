// K1: real-space imaginary-time Green's functions (Sec. 2, Eq. green_mat):
//
//   G^occ_ij(R, tau) = (1/N_k) sum_{k,n} f_nk       c_in(k) c*_jn(k) e^{-ik.R} e^{-(mu - e_nk) tau}
//   G^vir_ij(R, tau) = (1/N_k) sum_{k,n} (1 - f_nk) c_in(k) c*_jn(k) e^{-ik.R} e^{-(e_nk - mu) tau}
//
// (the paper's two branches with the factors -i, +i taken out; tau >= 0 in both).  For each
// tau: P^g_k = C_k diag(w^g(tau)) C_k^H as one batched complex GEMM over (g, k) restricted to
// the bands with non-zero weight, then G^g(R) = (1/N_k) Re sum_k e^{-ik.R} P^g_k.  The
// exponentials are evaluated in FP64 on the device.  For time-reversal-symmetric input
// G is real; the largest |Im| relative to the largest |Re| is returned as a check.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "ozgemm.h"

namespace librpa {
namespace {

// digit planes of the G build in the tensor-core modes (FP64-accurate products)
constexpr int kGreenS = 5;

// Y[g][k][n][i] = sqrt(w[g][k][n]) c_in(k) (the weights are >= 0), so that P^g_k = Y^T conj(Y)
__global__ void k_scale_bands(const double2 *wfc, const double *w, int nk, int nb, int nao, double2 *Y) {
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t per_g = (size_t)nk * nb * nao;
  if (x >= 2 * per_g) return;
  const int g = (int)(x / per_g);
  const size_t kni = x % per_g;
  const size_t kn = kni / nao;
  const double sw = sqrt(w[(size_t)g * nk * nb + kn]);
  const double2 c = wfc[kni];
  Y[x] = make_double2(sw * c.x, sw * c.y);
}

// w[g][k][n] for one tau: g = 0 occupied weight f e^{-(mu - e) tau}, g = 1 virtual weight
// (1 - f) e^{-(e - mu) tau}
__global__ void k_weights(const double *eig, const double *occ, double mu, double tau, int nkb, double *w) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nkb) return;
  const double e = eig[x], f = occ[x];
  w[x] = f > 0.0 ? f * exp(-(mu - e) * tau) : 0.0;
  w[nkb + x] = f < 1.0 ? (1.0 - f) * exp(-(e - mu) * tau) : 0.0;
}

// G[g][R][i][j] (slab of one tau) from the lower triangles of P[g][k] (Hermitian).
// One thread per (g, i, j); twiddle[k][R] = e^{-i 2 pi k.R}.
__global__ void k_phase_sum(const double2 *P, const double2 *twiddle, int nk, int nR, int nao,
                            double inv_nk, double *G, size_t g_stride, unsigned long long *maxabs) {
  const size_t n2 = (size_t)nao * nao;
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= 2 * n2) return;
  const int g = (int)(x / n2);
  const size_t ij = x % n2;
  const int i = (int)(ij / nao), j = (int)(ij % nao);
  const bool lower = i >= j;
  const size_t src = lower ? ij : (size_t)j * nao + i;
  double mre = 0.0, mim = 0.0;
  for (int R = 0; R < nR; ++R) {
    double re = 0.0, im = 0.0;
    for (int k = 0; k < nk; ++k) {
      double2 p = P[((size_t)g * nk + k) * n2 + src];
      if (!lower) p.y = -p.y;
      const double2 t = twiddle[(size_t)k * nR + R];
      re = fma(p.x, t.x, re);
      re = fma(-p.y, t.y, re);
      im = fma(p.x, t.y, im);
      im = fma(p.y, t.x, im);
    }
    re *= inv_nk;
    im *= inv_nk;
    G[(size_t)g * g_stride + (size_t)R * n2 + ij] = re;
    mre = fmax(mre, fabs(re));
    mim = fmax(mim, fabs(im));
  }
  // non-negative doubles order like their bit patterns
  atomicMax(&maxabs[0], __double_as_longlong(mre));
  atomicMax(&maxabs[1], __double_as_longlong(mim));
}

// Green's-function block screening (Sec. 5): the atom-pair block G^g_{IJ}(R, tau) is zeroed when
// its largest |element| is below theta, and kept[b] = 1 for the blocks that stay.  One warp per
// block; blocks flat over [spin][g][tau][R][I][J], the order of G's slabs and of the mask.
__global__ void k_screen(double *G, const int *tab, int natoms, int nao, long long nblocks, double theta,
                         unsigned char *kept) {
  const long long b = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= nblocks) return;   // the same for every lane of the warp
  const int J = (int)(b % natoms), I = (int)((b / natoms) % natoms);
  const long long slab = b / ((long long)natoms * natoms);
  const int *n_ao = tab, *ao_off = tab + natoms;
  double *blk = G + (size_t)slab * nao * nao + (size_t)ao_off[I] * nao + ao_off[J];
  const int nj = n_ao[J], n = n_ao[I] * nj;
  double mx = 0.0;
  for (int e = lane; e < n; e += 32) mx = fmax(mx, fabs(blk[(size_t)(e / nj) * nao + e % nj]));
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const bool keep = mx >= theta;
  if (lane == 0) kept[b] = keep ? 1 : 0;
  if (!keep)
    for (int e = lane; e < n; e += 32) blk[(size_t)(e / nj) * nao + e % nj] = 0.0;
}

// Screens every spin channel's G in place (h.g_screen > 0) and keeps the block mask on the host
// for the point selection of the contraction.
void green_screen(Handle &h) {
  const int nat = h.natoms, nR = h.mesh.size();
  const long long nblocks = (long long)h.nspins * 2 * h.ntau * nR * nat * nat;
  h.stats.n_blocks_total = nblocks;
  if (!(h.g_screen > 0)) {
    h.gmask.clear();
    h.stats.n_blocks_kept = nblocks;
    return;
  }
  cudaStream_t s = h.stream;
  std::vector<int> tab(2 * nat);
  for (int a = 0; a < nat; ++a) {
    tab[a] = h.n_ao[a];
    tab[nat + a] = h.ao_off[a];
  }
  h.ensure(h.d_screen_tab, tab.size() * sizeof(int));
  h.ensure(h.d_gmask, (size_t)nblocks);
  LR_CUDA(cudaMemcpyAsync(h.d_screen_tab.p, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  const long long threads = nblocks * 32;
  k_screen<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>((double *)h.d_g.p, (const int *)h.d_screen_tab.p, nat,
                                                             h.nao, nblocks, h.g_screen,
                                                             (unsigned char *)h.d_gmask.p);
  ++launch_counter();
  LR_CUDA(cudaGetLastError());
  h.gmask.resize((size_t)nblocks);
  LR_CUDA(cudaMemcpyAsync(h.gmask.data(), h.d_gmask.p, (size_t)nblocks, cudaMemcpyDeviceToHost, s));
  LR_CUDA(cudaStreamSynchronize(s));   // tab is a host temporary; the mask is read on the host next
  long long kept = 0;
  for (unsigned char c : h.gmask) kept += c;
  h.stats.n_blocks_kept = kept;
}

}  // namespace

size_t green_work_bytes(const Handle &h) {
  const size_t nk = h.mesh.size(), nR = nk, nb = h.nao, n2 = (size_t)h.nao * h.nao;
  const size_t b_e = nk * nb * 8, b_w = 2 * b_e, b_p = 2 * nk * n2 * 16, b_t = nk * nR * 16;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  size_t b = al(b_w) + al(b_p) + al(b_t) + 256;
  if (h.chi0_S >= 0)   // tensor-core modes: Y and the digit planes of both GEMM roles
    b += al(b_p) + oz::sliced_bytes((int)(2 * nk * 2 * h.nao), (int)(2 * nb), kGreenS) +
         oz::sliced_bytes((int)(2 * nk * h.nao), (int)(2 * nb), kGreenS) + 256;
  return b;
}

double green_build(Handle &h) {
  const int nk = h.mesh.size(), nR = nk, nao = h.nao, nb = h.nao, ntau = h.ntau;
  const size_t n2 = (size_t)nao * nao;
  const double mu = h.efermi_k[0];
  cudaStream_t s = h.stream;
  h.ensure(h.d_g, (size_t)h.nspins * 2 * ntau * nR * n2 * sizeof(double));   // [spin][g][tau][R][i][j]
  // workspace: weights, P, twiddles, max; the KS data is already on the device
  const size_t b_e = (size_t)nk * nb * 8, b_w = 2 * b_e, b_p = 2 * (size_t)nk * n2 * 16,
               b_t = (size_t)nk * nR * 16;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t o_w = 0, o_p = o_w + al(b_w), o_t = o_p + al(b_p), o_m = o_t + al(b_t);
  // tensor-core modes: P^g_k = Y^T conj(Y) as one batched digit-plane GEMM per tau (FP64-accurate)
  const bool tc = h.chi0_S >= 0;
  const size_t o_y = o_m + 256, o_sa = o_y + al(b_p),
               o_sb = o_sa + oz::sliced_bytes(2 * nk * 2 * nao, 2 * nb, kGreenS),
               o_err = o_sb + oz::sliced_bytes(2 * nk * nao, 2 * nb, kGreenS);
  h.ensure(h.work, green_work_bytes(h));
  char *wk = (char *)h.work.p;
  double2 *d_Y = tc ? (double2 *)(wk + o_y) : nullptr;
  int *d_err = tc ? (int *)(wk + o_err) : nullptr;
  oz::Sliced sa, sb;
  if (tc) {
    oz::sliced_bind(sa, wk + o_sa, 2 * nk * 2 * nao, 2 * nb, kGreenS);
    oz::sliced_bind(sb, wk + o_sb, 2 * nk * nao, 2 * nb, kGreenS);
    LR_CUDA(cudaMemsetAsync(d_err, 0, 4, s));
  }
  const double2 *d_wfc0 = (const double2 *)h.d_wfc.p;
  const double *d_eig0 = (const double *)h.d_eig.p, *d_occ0 = (const double *)h.d_occ.p;
  double *d_w = (double *)(wk + o_w);
  double2 *d_P = (double2 *)(wk + o_p), *d_tw = (double2 *)(wk + o_t);
  unsigned long long *d_max = (unsigned long long *)(wk + o_m);
  std::vector<double2> tw((size_t)nk * nR);
  for (int k = 0; k < nk; ++k) {
    int a, b, c;
    h.mesh.split(k, a, b, c);
    for (int R = 0; R < nR; ++R) {
      int x, y, z;
      h.mesh.split(R, x, y, z);
      // k.R in units of 2 pi with exact rational reduction
      const long long num = (long long)a * x * h.mesh.n2 * h.mesh.n3 + (long long)b * y * h.mesh.n1 * h.mesh.n3 +
                            (long long)c * z * h.mesh.n1 * h.mesh.n2;
      const long long den = (long long)h.mesh.n1 * h.mesh.n2 * h.mesh.n3;
      const double th = 2.0 * M_PI * (double)(num % den) / (double)den;
      tw[(size_t)k * nR + R] = make_double2(std::cos(th), -std::sin(th));
    }
  }
  LR_CUDA(cudaMemcpyAsync(d_tw, tw.data(), b_t, cudaMemcpyHostToDevice, s));
  LR_CUDA(cudaStreamSynchronize(s));   // tw is a host temporary
  LR_CUDA(cudaMemsetAsync(d_max, 0, 16, s));
  const size_t g_stride = (size_t)ntau * nR * n2;
  for (int sp = 0; sp < h.nspins; ++sp) {   // one spin channel at a time, own KS data, own G
    const double2 *d_wfc = d_wfc0 + (size_t)sp * nk * nb * nao;
    const double *d_eig = d_eig0 + (size_t)sp * nk * nb, *d_occ = d_occ0 + (size_t)sp * nk * nb;
    double *d_gs = (double *)h.d_g.p + (size_t)sp * 2 * g_stride;
    // band ranges with non-zero occupied / virtual weight per k
    std::vector<int> olo(nk, nb), ohi(nk, 0), vlo(nk, nb), vhi(nk, 0);
    for (int k = 0; k < nk; ++k)
      for (int n = 0; n < nb; ++n) {
        const double f = h.occ[((size_t)sp * nk + k) * nb + n];
        if (f > 0) { olo[k] = std::min(olo[k], n); ohi[k] = n + 1; }
        if (f < 1) { vlo[k] = std::min(vlo[k], n); vhi[k] = n + 1; }
      }
    for (int it = 0; it < ntau; ++it) {
      k_weights<<<(nk * nb + 255) / 256, 256, 0, s>>>(d_eig, d_occ, mu, h.tau[it], nk * nb, d_w);
      ++launch_counter();
      if (tc) {
        // every band enters with its weight (zero outside the occupied / virtual range)
        const size_t ny = 2 * (size_t)nk * nb * nao;
        k_scale_bands<<<(unsigned)((ny + 255) / 256), 256, 0, s>>>(d_wfc, d_w, nk, nb, nao, d_Y);
        ++launch_counter();
        oz::split_complex(d_Y, nao, oz::OP_T, true, nao, nb, 2 * nk, (long long)nb * nao, sa, s);
        oz::split_complex(d_Y, nao, oz::OP_C, false, nao, nb, 2 * nk, (long long)nb * nao, sb, s);
        oz::Out o;
        o.C = (double *)d_P;
        o.ldc = nao;
        o.batch_stride = (long long)n2;
        o.mode = 1;
        oz::gemm(sa, sb, 2 * nao, nao, 2 * nk, o, 0, 0, 2, d_err, s, h);
        const size_t nthr = 2 * n2;
        k_phase_sum<<<(unsigned)((nthr + 255) / 256), 256, 0, s>>>(d_P, d_tw, nk, nR, nao, 1.0 / nk,
                                                                  d_gs + (size_t)it * nR * n2, g_stride, d_max);
        ++launch_counter();
        LR_CUDA(cudaGetLastError());
        continue;
      }
      std::vector<ZGemm> batch;
      for (int g = 0; g < 2; ++g)
        for (int k = 0; k < nk; ++k) {
          const int lo = g == 0 ? olo[k] : vlo[k], hi = g == 0 ? ohi[k] : vhi[k];
          ZGemm z{};
          z.A = d_wfc + ((size_t)k * nb + lo) * nao;
          z.B = z.A;
          z.C = d_P + ((size_t)g * nk + k) * n2;
          z.kscale = d_w + (size_t)g * nk * nb + (size_t)k * nb + lo;
          z.M = nao;
          z.N = nao;
          z.K = hi > lo ? hi - lo : 0;
          z.lda = z.ldb = nao;
          z.ldc = nao;
          z.alpha = make_double2(1.0, 0.0);
          z.beta = make_double2(0.0, 0.0);
          if (z.K == 0) {
            LR_CUDA(cudaMemsetAsync(z.C, 0, n2 * 16, s));
            continue;
          }
          batch.push_back(z);
        }
      ZGemmFlags f;
      f.transA = true;   // A stored [band][i]
      f.conjB = true;    // B = conj(wfc) stored [band][j]
      f.lower_only = true;
      zgemm_batched(batch, f, s, h);
      const size_t nthr = 2 * n2;
      k_phase_sum<<<(unsigned)((nthr + 255) / 256), 256, 0, s>>>(d_P, d_tw, nk, nR, nao, 1.0 / nk,
                                                                d_gs + (size_t)it * nR * n2, g_stride, d_max);
      ++launch_counter();
      LR_CUDA(cudaGetLastError());
    }
  }
  unsigned long long mx[2];
  int e_host = 0;
  LR_CUDA(cudaMemcpyAsync(mx, d_max, 16, cudaMemcpyDeviceToHost, s));
  if (tc) LR_CUDA(cudaMemcpyAsync(&e_host, d_err, 4, cudaMemcpyDeviceToHost, s));
  LR_CUDA(cudaStreamSynchronize(s));
  if (e_host) throw Error{LIBRPA_E_TIMEOUT, "Green's function: a bounded wait in the tensor-core GEMM ran out"};
  green_screen(h);   // after the imaginary-part check's maxima: they describe the unscreened G
  double mre, mim;
  std::memcpy(&mre, &mx[0], 8);
  std::memcpy(&mim, &mx[1], 8);
  return mre > 0 ? mim / mre : mim;
}

}  // namespace librpa
