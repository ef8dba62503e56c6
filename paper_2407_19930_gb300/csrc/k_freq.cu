// K3 + K4: chi0(R, tau) -> chi0(R, i omega) -> chi0(q, i omega) (Sec. 2):
//
//   chi0(R, i omega_k) = sum_j Gamma_kj chi0(R, tau_j)        (cosine transform; Gamma real)
//   chi0(q, i omega)   = sum_{R in BvK} e^{+i q.R} chi0(R, i omega)
//
// Both are per-element linear maps over whole N_aux^2 matrices: one thread per matrix element
// keeps its tau (or R) vector in registers, the small transform matrices sit in shared memory,
// and consecutive threads touch consecutive elements, so every load and store is coalesced.
#include <vector>

#include "internal.h"

namespace librpa {
namespace {

template <int NT>
__global__ void __launch_bounds__(256) k_tau_to_omega(const double *__restrict__ in, double *__restrict__ out,
                                                      const double *__restrict__ gamma, int ntau, int nR,
                                                      size_t n2) {
  __shared__ double gs[NT * NT];
  for (int e = threadIdx.x; e < ntau * ntau; e += blockDim.x) gs[e] = gamma[e];
  __syncthreads();
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int R = blockIdx.y;
  if (x >= n2) return;
  double v[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) v[j] = j < ntau ? in[((size_t)j * nR + R) * n2 + x] : 0.0;
#pragma unroll 1
  for (int k = 0; k < ntau; ++k) {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < NT; ++j)
      if (j < ntau) acc = fma(gs[k * ntau + j], v[j], acc);
    out[((size_t)k * nR + R) * n2 + x] = acc;
  }
}

// chi0(q, i omega_k) for the nsel selected q (qidx: their mesh indices; ph: their phases, [qi][R])
template <int NR>
__global__ void __launch_bounds__(256) k_r_to_q(const double *__restrict__ in, double2 *__restrict__ out,
                                                const double2 *__restrict__ ph, const int *__restrict__ qidx,
                                                int nR, int nsel, int nw, size_t n2) {
  __shared__ double2 ps[NR * NR];
  __shared__ int qs[NR];
  for (int e = threadIdx.x; e < nsel * nR; e += blockDim.x) ps[e] = ph[e];
  for (int e = threadIdx.x; e < nsel; e += blockDim.x) qs[e] = qidx[e];
  __syncthreads();
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (x >= n2) return;
  double y[NR];
#pragma unroll
  for (int R = 0; R < NR; ++R) y[R] = R < nR ? in[((size_t)k * nR + R) * n2 + x] : 0.0;
#pragma unroll 1
  for (int qi = 0; qi < nsel; ++qi) {
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int R = 0; R < NR; ++R)
      if (R < nR) {
        const double2 p = ps[qi * nR + R];
        re = fma(p.x, y[R], re);
        im = fma(p.y, y[R], im);
      }
    out[((size_t)qs[qi] * nw + k) * n2 + x] = make_double2(re, im);
  }
}

// chi0(q) = conj chi0(-q) for the q not computed (chi0(R) is real); pairs[2 i] = q, pairs[2 i + 1] = -q
__global__ void __launch_bounds__(256) k_conj_fill(double2 *__restrict__ chi, const int *__restrict__ pairs, int nw,
                                                   size_t per_q) {
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= per_q) return;
  const int q = pairs[2 * blockIdx.y], p = pairs[2 * blockIdx.y + 1];
  const double2 z = chi[(size_t)p * per_q + x];
  chi[(size_t)q * per_q + x] = make_double2(z.x, -z.y);
}

template <int NT>
void launch_tw(const double *in, double *out, const double *gamma, int ntau, int nR, size_t n2, cudaStream_t s) {
  dim3 g((unsigned)((n2 + 255) / 256), (unsigned)nR);
  k_tau_to_omega<NT><<<g, 256, 0, s>>>(in, out, gamma, ntau, nR, n2);
}

template <int NR>
void launch_rq(const double *in, double2 *out, const double2 *ph, const int *qidx, int nR, int nsel, int nw,
               size_t n2, cudaStream_t s) {
  dim3 g((unsigned)((n2 + 255) / 256), (unsigned)nw);
  k_r_to_q<NR><<<g, 256, 0, s>>>(in, out, ph, qidx, nR, nsel, nw, n2);
}

}  // namespace

size_t freq_work_bytes(const Handle &h) {
  const size_t nR = h.mesh.size(), n2 = (size_t)h.naux * h.naux;
  const size_t b_rw = (size_t)h.ntau * nR * n2 * 8, b_g = (size_t)h.ntau * h.ntau * 8, b_p = nR * nR * 16;
  return b_rw + 256 + b_g + 256 + b_p + 256 + 3 * nR * 4;
}

void freq_transform(Handle &h) {
  const int ntau = h.ntau, nR = h.mesh.size(), nq = nR;
  const size_t n2 = (size_t)h.naux * h.naux;
  cudaStream_t s = h.stream;
  if (nR > 64) throw Error{LIBRPA_E_ARG, "k-mesh with more than 64 points is not supported"};
  h.ensure(h.d_chi_qw, (size_t)nq * ntau * n2 * 16);
  // workspace: chi0(R, i omega) plus the two small matrices
  const size_t b_rw = (size_t)ntau * nR * n2 * 8, b_g = (size_t)ntau * ntau * 8, b_p = (size_t)nq * nR * 16;
  h.ensure(h.work, freq_work_bytes(h));
  char *w = (char *)h.work.p;
  double *rw = (double *)w;
  double *dg = (double *)(w + (b_rw + 255) / 256 * 256);
  double2 *dp = (double2 *)((char *)dg + (b_g + 255) / 256 * 256);
  int *di = (int *)((char *)dp + (b_p + 255) / 256 * 256);   // [nq] selected q, then [nq][2] pairs
  // only q <= -q is transformed; the others are conj chi0(-q) (chi0(R) is real)
  std::vector<int> qsel, pairs;
  for (int q = 0; q < nq; ++q) {
    const int p = h.mesh.neg(q);
    if (q <= p)
      qsel.push_back(q);
    else
      pairs.insert(pairs.end(), {q, p});
  }
  const int nsel = (int)qsel.size();
  std::vector<double2> ph((size_t)nsel * nR);
  for (int qi = 0; qi < nsel; ++qi) {
    const int q = qsel[qi];
    int a, b, c;
    h.mesh.split(q, a, b, c);
    for (int R = 0; R < nR; ++R) {
      int x, y, z;
      h.mesh.split(R, x, y, z);
      const long long den = (long long)h.mesh.n1 * h.mesh.n2 * h.mesh.n3;
      const long long num = (long long)a * x * h.mesh.n2 * h.mesh.n3 + (long long)b * y * h.mesh.n1 * h.mesh.n3 +
                            (long long)c * z * h.mesh.n1 * h.mesh.n2;
      const double th = 2.0 * M_PI * (double)(num % den) / (double)den;
      ph[(size_t)qi * nR + R] = make_double2(std::cos(th), std::sin(th));
    }
  }
  std::vector<int> ints(qsel);
  ints.insert(ints.end(), pairs.begin(), pairs.end());
  LR_CUDA(cudaMemcpyAsync(dg, h.gamma.data(), b_g, cudaMemcpyHostToDevice, s));
  LR_CUDA(cudaMemcpyAsync(dp, ph.data(), ph.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
  LR_CUDA(cudaMemcpyAsync(di, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  const double *in = (const double *)h.d_chi_tau.p;
  if (ntau <= 16)
    launch_tw<16>(in, rw, dg, ntau, nR, n2, s);
  else if (ntau <= 32)
    launch_tw<32>(in, rw, dg, ntau, nR, n2, s);
  else
    launch_tw<64>(in, rw, dg, ntau, nR, n2, s);
  double2 *out = (double2 *)h.d_chi_qw.p;
  if (nR <= 16)
    launch_rq<16>(rw, out, dp, di, nR, nsel, ntau, n2, s);
  else if (nR <= 32)
    launch_rq<32>(rw, out, dp, di, nR, nsel, ntau, n2, s);
  else
    launch_rq<64>(rw, out, dp, di, nR, nsel, ntau, n2, s);
  launch_counter() += 2;
  if (!pairs.empty()) {
    const size_t per_q = (size_t)ntau * n2;
    dim3 g((unsigned)((per_q + 255) / 256), (unsigned)(pairs.size() / 2));
    k_conj_fill<<<g, 256, 0, s>>>(out, di + nsel, ntau, per_q);
    ++launch_counter();
  }
  LR_CUDA(cudaGetLastError());
}

}  // namespace librpa
