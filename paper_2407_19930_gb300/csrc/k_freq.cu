// K3 + K4: chi0(R, tau) -> chi0(R, i omega) -> chi0(q, i omega) (Sec. 2):
//
//   chi0(R, i omega_k) = sum_j Gamma_kj chi0(R, tau_j)        (cosine transform; Gamma real)
//   chi0(q, i omega)   = sum_{R in BvK} e^{+i q.R} chi0(R, i omega)
//
// Both are per-element linear maps over whole N_aux^2 matrices: one thread per matrix element
// keeps its tau (or R) vector in registers, the small transform matrices sit in shared memory,
// and consecutive threads touch consecutive elements, so every load and store is coalesced.  The
// R -> q map runs for q <= -q only and stores conj chi0(q) at -q as well (chi0(R) is real).
#include <vector>

#include "internal.h"

namespace librpa {
namespace {

// Arithmetic of the two maps: double, or float in LIBRPA_SPLIT_FAST, whose chi0(R, tau) carries
// ~23 bits, so that FP32 rounding is of the size of chi0's own error and the FP64 pipe's flops
// (~60 ms per energy on the graphene slab) give way to the HBM traffic.
template <class A>
struct Cplx;
template <>
struct Cplx<double> {
  using T = double2;
  static __host__ __device__ T make(double x, double y) { return make_double2(x, y); }
};
template <>
struct Cplx<float> {
  using T = float2;
  static __host__ __device__ T make(float x, float y) { return make_float2(x, y); }
};
__device__ __forceinline__ double fma_a(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_a(float a, float b, float c) { return fmaf(a, b, c); }

template <int NT, class A>
__global__ void __launch_bounds__(256) k_tau_to_omega(const double *__restrict__ in, A *__restrict__ out,
                                                      const A *__restrict__ gamma, int ntau, int nR, size_t n2) {
  __shared__ A gs[NT * NT];
  for (int e = threadIdx.x; e < ntau * ntau; e += blockDim.x) gs[e] = gamma[e];
  __syncthreads();
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int R = blockIdx.y;
  if (x >= n2) return;
  A v[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) v[j] = j < ntau ? (A)in[((size_t)j * nR + R) * n2 + x] : A(0);
#pragma unroll 1
  for (int k = 0; k < ntau; ++k) {
    A acc = 0;
#pragma unroll
    for (int j = 0; j < NT; ++j)
      if (j < ntau) acc = fma_a(gs[k * ntau + j], v[j], acc);
    out[((size_t)k * nR + R) * n2 + x] = acc;
  }
}

// chi0(q, i omega_k) for the nsel selected q (qidx: their mesh indices; ph: their phases, [qi][R]);
// where qneg[qi] >= 0, chi0(-q) = conj chi0(q) (chi0(R) is real) is written there as well
template <int NR, class A>
__global__ void __launch_bounds__(256) k_r_to_q(const A *__restrict__ in, double2 *__restrict__ out,
                                                const typename Cplx<A>::T *__restrict__ ph,
                                                const int *__restrict__ qidx, const int *__restrict__ qneg, int nR,
                                                int nsel, int nw, size_t n2) {
  // nsel <= nR / 2 + 4: q = -q for at most 2 values per mesh dimension (checked on the host)
  __shared__ typename Cplx<A>::T ps[NR * (NR / 2 + 4)];
  __shared__ int qs[NR], qn[NR];
  for (int e = threadIdx.x; e < nsel * nR; e += blockDim.x) ps[e] = ph[e];
  for (int e = threadIdx.x; e < nsel; e += blockDim.x) {
    qs[e] = qidx[e];
    qn[e] = qneg[e];
  }
  __syncthreads();
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (x >= n2) return;
  A y[NR];
#pragma unroll
  for (int R = 0; R < NR; ++R) y[R] = R < nR ? in[((size_t)k * nR + R) * n2 + x] : A(0);
#pragma unroll 1
  for (int qi = 0; qi < nsel; ++qi) {
    A re = 0, im = 0;
#pragma unroll
    for (int R = 0; R < NR; ++R)
      if (R < nR) {
        const typename Cplx<A>::T p = ps[qi * nR + R];
        re = fma_a(p.x, y[R], re);
        im = fma_a(p.y, y[R], im);
      }
    out[((size_t)qs[qi] * nw + k) * n2 + x] = make_double2(re, im);
    if (qn[qi] >= 0) out[((size_t)qn[qi] * nw + k) * n2 + x] = make_double2(re, -(double)im);
  }
}

template <class A>
void launch_tw(const double *in, A *out, const A *gamma, int ntau, int nR, size_t n2, cudaStream_t s) {
  dim3 g((unsigned)((n2 + 255) / 256), (unsigned)nR);
  if (ntau <= 16)
    k_tau_to_omega<16, A><<<g, 256, 0, s>>>(in, out, gamma, ntau, nR, n2);
  else if (ntau <= 32)
    k_tau_to_omega<32, A><<<g, 256, 0, s>>>(in, out, gamma, ntau, nR, n2);
  else
    k_tau_to_omega<64, A><<<g, 256, 0, s>>>(in, out, gamma, ntau, nR, n2);
}

template <class A>
void launch_rq(const A *in, double2 *out, const typename Cplx<A>::T *ph, const int *qidx, const int *qneg, int nR,
               int nsel, int nw, size_t n2, cudaStream_t s) {
  dim3 g((unsigned)((n2 + 255) / 256), (unsigned)nw);
  if (nR <= 16)
    k_r_to_q<16, A><<<g, 256, 0, s>>>(in, out, ph, qidx, qneg, nR, nsel, nw, n2);
  else if (nR <= 32)
    k_r_to_q<32, A><<<g, 256, 0, s>>>(in, out, ph, qidx, qneg, nR, nsel, nw, n2);
  else
    k_r_to_q<64, A><<<g, 256, 0, s>>>(in, out, ph, qidx, qneg, nR, nsel, nw, n2);
}

// the two maps in arithmetic A; gamma [ntau][ntau] and the phases [nsel][nR] in double on the host
template <class A>
void transform_as(Handle &h, const std::vector<double> &gamma, const std::vector<double2> &ph,
                  const std::vector<int> &ints, int nsel, char *w, size_t b_rw, size_t b_g, size_t b_p) {
  const int ntau = h.ntau, nR = h.mesh.size();
  const size_t n2 = (size_t)h.naux * h.naux;
  cudaStream_t s = h.stream;
  A *rw = (A *)w;
  A *dg = (A *)(w + (b_rw + 255) / 256 * 256);
  auto *dp = (typename Cplx<A>::T *)((char *)dg + (b_g + 255) / 256 * 256);
  int *di = (int *)((char *)dp + (b_p + 255) / 256 * 256);   // [nsel] selected q, then [nsel] their -q
  std::vector<A> ga(gamma.begin(), gamma.end());
  std::vector<typename Cplx<A>::T> pa(ph.size());
  for (size_t i = 0; i < ph.size(); ++i) pa[i] = Cplx<A>::make((A)ph[i].x, (A)ph[i].y);
  // pageable sources: the copies are complete (staged) when cudaMemcpyAsync returns
  LR_CUDA(cudaMemcpyAsync(dg, ga.data(), ga.size() * sizeof(A), cudaMemcpyHostToDevice, s));
  LR_CUDA(cudaMemcpyAsync(dp, pa.data(), pa.size() * sizeof(pa[0]), cudaMemcpyHostToDevice, s));
  LR_CUDA(cudaMemcpyAsync(di, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  launch_tw<A>((const double *)h.d_chi_tau.p, rw, dg, ntau, nR, n2, s);
  launch_rq<A>(rw, (double2 *)h.d_chi_qw.p, dp, di, di + nsel, nR, nsel, ntau, n2, s);
  launch_counter() += 2;
  LR_CUDA(cudaGetLastError());
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
  if (nR > 64) throw Error{LIBRPA_E_ARG, "k-mesh with more than 64 points is not supported"};
  h.ensure(h.d_chi_qw, (size_t)nq * ntau * n2 * 16);
  // workspace: chi0(R, i omega) plus the two small matrices (sized for double)
  const size_t b_rw = (size_t)ntau * nR * n2 * 8, b_g = (size_t)ntau * ntau * 8, b_p = (size_t)nq * nR * 16;
  h.ensure(h.work, freq_work_bytes(h));
  // only q <= -q is transformed; -q, where it differs, gets conj chi0(q) (chi0(R) is real)
  std::vector<int> qsel, qneg;
  for (int q = 0; q < nq; ++q) {
    const int p = h.mesh.neg(q);
    if (q <= p) {
      qsel.push_back(q);
      qneg.push_back(p == q ? -1 : p);
    }
  }
  const int nsel = (int)qsel.size();
  if (nsel > nR / 2 + 4) throw Error{LIBRPA_E_ARG, "k-mesh: more self-inverse q than a mesh can have"};
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
  ints.insert(ints.end(), qneg.begin(), qneg.end());
  char *w = (char *)h.work.p;
  if (h.freq_f32)
    transform_as<float>(h, h.gamma, ph, ints, nsel, w, b_rw, b_g, b_p);
  else
    transform_as<double>(h, h.gamma, ph, ints, nsel, w, b_rw, b_g, b_p);
}

}  // namespace librpa
