// librpa_gpu_ec_noalloc: the ln det stage for one q and a set of frequencies, with its scratch
// in a static device array instead of memory obtained from an allocator.
//
// For whom: callers that cannot call cudaMalloc -- host codes that hand all of the GPU's
// memory to their own pool at start-up (so a further cudaMalloc fails or fragments it), and
// callers whose loop must not stall other streams (cudaMalloc and cudaFree may synchronise
// the device).  They pass device inputs and outputs only; the library allocates nothing.
//
// Per frequency k, with V = L L^H (Cholesky) and A_k = I - L^H chi_k L:
//   out[k] = ln det(I - chi_k V) + Re Tr(chi_k V) = 2 sum_i ln (L_A)_ii + sum_i Re (1 - A_k,ii)
// (Sylvester's identity: det(I - chi L L^H) = det(I - L^H chi L); the same reading of the
// integrand of the E_c formula in Sec. 2 as the handle-based ln det stage, computed here by one
// fused kernel instead of the blocked, batched one.)
//
// Scratch: a file-scope __device__ array of LIBRPA_NOALLOC_SCRATCH_BYTES, split into slots of
// 3 naux^2 complex values (L, T = chi L, A) per CTA.  Every value a CTA reads from its slot is
// written earlier in the same call, so nothing needs clearing; the array keeps the last call's
// contents.  All calls share it: calls that overlap on the GPU race.  The device creates the
// array when it loads this file's module: with lazy module loading (the CUDA default) that is
// the first call made with the device current, which therefore takes 16 MiB of device memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/librpa_gpu.h"

namespace {

constexpr size_t kScratchElems = LIBRPA_NOALLOC_SCRATCH_BYTES / sizeof(double2);
static_assert(3ull * LIBRPA_NOALLOC_MAX_NAUX * LIBRPA_NOALLOC_MAX_NAUX <= kScratchElems,
              "one slot of the largest size must fit the scratch array");
constexpr int kThreads = 256;
constexpr int kTile = 32;
constexpr int kMaxDevices = 64;

}  // namespace

// The scratch itself.  In host code this name is a host-side stand-in; the device address
// comes from cudaGetSymbolAddress.
static __device__ __align__(256) double2 noalloc_scratch[kScratchElems];

namespace {

__device__ __forceinline__ double2 cmul_conj_b(double2 a, double2 b) {   // a * conj(b)
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {   // a * b + c
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// In-place lower Cholesky M = L L^H of an n x n Hermitian matrix (row-major, only the lower
// triangle read), right-looking, one column per step.  Returns sum_i ln L_ii on thread 0, NaN
// on every thread if a pivot is not positive (or not a number).
__device__ double cta_cholesky(double2 *M, int n, double2 *col, double *s_piv) {
  const int tid = threadIdx.x;
  double lsum = 0.0;
  for (int j = 0; j < n; ++j) {
    __syncthreads();   // previous trailing update complete
    if (tid == 0) *s_piv = M[(size_t)j * n + j].x;
    __syncthreads();
    const double d = *s_piv;
    if (!(d > 0.0)) return NAN;
    const double r = sqrt(d), ri = 1.0 / r;
    for (int i = j + tid; i < n; i += kThreads) {
      double2 v = M[(size_t)i * n + j];
      v = i == j ? make_double2(r, 0.0) : make_double2(v.x * ri, v.y * ri);
      M[(size_t)i * n + j] = v;
      col[i] = v;
    }
    if (tid == 0) lsum += log(r);
    __syncthreads();
    // trailing update of the lower triangle only: one warp per row, lanes along the row
    const int warp = tid >> 5, lane = tid & 31;
    for (int ii = j + 1 + warp; ii < n; ii += kThreads / 32) {
      const double2 ci = col[ii];
      for (int kk = j + 1 + lane; kk <= ii; kk += 32) {
        double2 &x = M[(size_t)ii * n + kk];
        const double2 p = cmul_conj_b(ci, col[kk]);
        x = make_double2(x.x - p.x, x.y - p.y);
      }
    }
  }
  return lsum;
}

// One CTA per slot; CTA b factors V once into its slot, then takes frequencies b, b + grid, ...
__global__ void __launch_bounds__(kThreads) k_ec_noalloc(double2 *scratch, int n, int nomega,
                                                         const double2 *__restrict__ V,
                                                         const double2 *__restrict__ chi, double *out) {
  __shared__ double2 As[kTile][kTile + 1];
  __shared__ double2 Bs[kTile][kTile + 1];
  __shared__ double2 col[LIBRPA_NOALLOC_MAX_NAUX];
  __shared__ double s_piv;
  const int tid = threadIdx.x, tx = tid % kTile, ty = tid / kTile;   // ty in 0..7
  const size_t n2 = (size_t)n * n;
  double2 *Lm = scratch + 3 * n2 * blockIdx.x;
  double2 *T = Lm + n2;
  double2 *A = T + n2;
  for (size_t e = tid; e < n2; e += kThreads) Lm[e] = V[e];
  const double lv = cta_cholesky(Lm, n, col, &s_piv);
  const bool v_ok = !isnan(lv);   // uniform: NaN is returned on every thread
  const int nt = (n + kTile - 1) / kTile;
  for (int k = blockIdx.x; k < nomega; k += gridDim.x) {
    if (!v_ok) {
      if (tid == 0) out[k] = NAN;
      continue;
    }
    const double2 *X = chi + n2 * k;
    // T = chi_k L (L lower: L_jc = 0 for j < c, so the j tiles start at the column tile)
    for (int t = 0; t < nt * nt; ++t) {
      const int ti = t / nt, tc = t % nt;
      double2 acc[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) acc[s] = make_double2(0.0, 0.0);
      for (int tj = tc; tj < nt; ++tj) {
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int r = ty + 8 * s;
          const int gi = ti * kTile + r, gj = tj * kTile + tx;
          As[r][tx] = (gi < n && gj < n) ? X[(size_t)gi * n + gj] : make_double2(0.0, 0.0);
          const int lj = tj * kTile + r, lc = tc * kTile + tx;
          Bs[r][tx] = (lj < n && lc < n && lj >= lc) ? Lm[(size_t)lj * n + lc] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 8
        for (int jj = 0; jj < kTile; ++jj) {
          const double2 b = Bs[jj][tx];
#pragma unroll
          for (int s = 0; s < 4; ++s) acc[s] = cfma(As[ty + 8 * s][jj], b, acc[s]);
        }
      }
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int gi = ti * kTile + ty + 8 * s, gc = tc * kTile + tx;
        if (gi < n && gc < n) T[(size_t)gi * n + gc] = acc[s];
      }
    }
    // A = I - L^H T on the lower tiles (L^H_ij = conj(L_ji), zero for j < i)
    for (int t = 0; t < nt * nt; ++t) {
      const int ti = t / nt, tc = t % nt;
      if (tc > ti) continue;
      double2 acc[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) acc[s] = make_double2(0.0, 0.0);
      for (int tj = ti; tj < nt; ++tj) {
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int r = ty + 8 * s;
          // As[i][j] = conj(L[j][i]): read L row j = tj*32 + r, column i = ti*32 + tx (coalesced)
          const int lj = tj * kTile + r, li = ti * kTile + tx;
          const double2 v = (lj < n && li < n && lj >= li) ? Lm[(size_t)lj * n + li] : make_double2(0.0, 0.0);
          As[tx][r] = make_double2(v.x, -v.y);
          const int gj = tj * kTile + r, gc = tc * kTile + tx;
          Bs[r][tx] = (gj < n && gc < n) ? T[(size_t)gj * n + gc] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 8
        for (int jj = 0; jj < kTile; ++jj) {
          const double2 b = Bs[jj][tx];
#pragma unroll
          for (int s = 0; s < 4; ++s) acc[s] = cfma(As[ty + 8 * s][jj], b, acc[s]);
        }
      }
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int gi = ti * kTile + ty + 8 * s, gc = tc * kTile + tx;
        if (gi < n && gc < n) A[(size_t)gi * n + gc] = make_double2((gi == gc ? 1.0 : 0.0) - acc[s].x, -acc[s].y);
      }
    }
    __syncthreads();
    double tr = 0.0;   // Re Tr(chi V) = sum_i Re (1 - A_ii), on thread 0
    if (tid == 0)
      for (int i = 0; i < n; ++i) tr += 1.0 - A[(size_t)i * n + i].x;
    const double la = cta_cholesky(A, n, col, &s_piv);
    if (tid == 0) out[k] = isnan(la) ? NAN : 2.0 * la + tr;
    __syncthreads();   // thread 0's reads of A done before the next frequency rewrites the slot
  }
}

int fail(char *msg, size_t msg_len, int code, const char *text) {
  if (msg && msg_len) {
    std::strncpy(msg, text, msg_len - 1);
    msg[msg_len - 1] = '\0';
  }
  return code;
}

int fail_cuda(char *msg, size_t msg_len, const char *what, cudaError_t e) {
  char buf[256];
  std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  return fail(msg, msg_len, LIBRPA_E_CUDA, buf);
}

std::mutex g_mu;
void *g_scratch[kMaxDevices] = {};

}  // namespace

extern "C" int librpa_gpu_ec_noalloc(int naux, int nomega, const double *V, const double *chi, double *out,
                                     void *stream, char *msg, size_t msg_len) {
  if (msg && msg_len) msg[0] = '\0';
  char buf[256];
  if (naux < 1 || naux > LIBRPA_NOALLOC_MAX_NAUX) {
    std::snprintf(buf, sizeof buf,
                  "librpa_gpu_ec_noalloc: naux = %d outside 1..%d (the static scratch holds %d MiB)", naux,
                  LIBRPA_NOALLOC_MAX_NAUX, (int)(LIBRPA_NOALLOC_SCRATCH_BYTES >> 20));
    return fail(msg, msg_len, LIBRPA_E_ARG, buf);
  }
  if (nomega < 0) return fail(msg, msg_len, LIBRPA_E_ARG, "librpa_gpu_ec_noalloc: nomega < 0");
  if (nomega > 0 && (!V || !chi || !out))
    return fail(msg, msg_len, LIBRPA_E_ARG, "librpa_gpu_ec_noalloc: NULL V, chi or out");
  if (((uintptr_t)V | (uintptr_t)chi) % 16 || (uintptr_t)out % 8)
    return fail(msg, msg_len, LIBRPA_E_ARG,
                "librpa_gpu_ec_noalloc: V and chi must be 16-byte aligned, out 8-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_cuda(msg, msg_len, "cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) return fail(msg, msg_len, LIBRPA_E_ARG, "librpa_gpu_ec_noalloc: device index >= 64");
  void *base = nullptr;
  {
    // set-up, once per device, on the first call made with that device current.  Under lazy
    // module loading (the CUDA default) this is also when the device creates the static array:
    // its memory is taken here, so this lookup can fail for lack of device memory.
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
      e = cudaGetSymbolAddress(&g_scratch[dev], noalloc_scratch);
      if (e != cudaSuccess) {
        g_scratch[dev] = nullptr;
        if (e == cudaErrorMemoryAllocation) {
          cudaGetLastError();
          std::snprintf(buf, sizeof buf,
                        "librpa_gpu_ec_noalloc: out of device memory while the device created the %d MiB "
                        "static scratch array (first call on device %d); make the first call, e.g. with "
                        "nomega = 0, before other code claims the device's memory",
                        (int)(LIBRPA_NOALLOC_SCRATCH_BYTES >> 20), dev);
          return fail(msg, msg_len, LIBRPA_E_NOMEM, buf);
        }
        return fail_cuda(msg, msg_len, "cudaGetSymbolAddress(noalloc_scratch)", e);
      }
    }
    base = g_scratch[dev];
  }
  if (nomega == 0) return LIBRPA_OK;   // set-up only
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail_cuda(msg, msg_len, "cudaDeviceGetAttribute", e);
  const size_t slot = 3 * (size_t)naux * naux;
  int grid = (int)std::min<size_t>(kScratchElems / slot, (size_t)nomega);
  grid = std::min(grid, 2 * sms);
  k_ec_noalloc<<<grid, kThreads, 0, (cudaStream_t)stream>>>(
      (double2 *)base, naux, nomega, (const double2 *)V, (const double2 *)chi, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(msg, msg_len, "k_ec_noalloc launch", e);
  return LIBRPA_OK;
}
