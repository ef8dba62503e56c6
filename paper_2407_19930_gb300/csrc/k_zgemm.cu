// Batched complex FP64 GEMM: C = alpha op(A) diag(kscale) op(B) + beta C.
//
// Used by the Green's-function build (P_k = C_k diag(w) C_k^H, Eq. green_mat) and by the
// correlation-energy stage (W = chi0 L, A = I - L^H W and the Cholesky trailing updates).
// FP64 on GB300 runs at the same rate on the DFMA and DMMA pipes, so this kernel uses
// DFMA with 4x4 register tiles; one CTA computes a 64 x 64 tile, K in chunks of 8.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

namespace librpa {
namespace {

constexpr int TM = 64, TN = 64, TK = 8, NT = 256;

struct Tile {
  int e, m0, n0;
};

struct Args {
  const ZGemm *g;
  const Tile *tiles;
  ZGemmFlags f;
};

__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}

__global__ void __launch_bounds__(NT) k_zgemm(Args args) {
  const Tile t = args.tiles[blockIdx.x];
  const ZGemm g = args.g[t.e];
  const ZGemmFlags f = args.f;
  __shared__ double2 As[TK][TM];
  __shared__ double2 Bs[TK][TN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  double2 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_double2(0.0, 0.0);
  int kbeg = 0;
  if (f.kfrom == 1) kbeg = t.m0;
  if (f.kfrom == 2) kbeg = t.n0;
  for (int k0 = kbeg; k0 < g.K; k0 += TK) {
#pragma unroll
    for (int s = 0; s < (TM * TK) / NT; ++s) {
      const int e = tid + NT * s;
      int m, k;
      if (f.transA) { m = e % TM; k = e / TM; } else { m = e / TK; k = e % TK; }
      const int gm = t.m0 + m, gk = k0 + k;
      double2 v = make_double2(0.0, 0.0);
      if (gm < g.M && gk < g.K) {
        v = f.transA ? g.A[(size_t)gk * g.lda + gm] : g.A[(size_t)gm * g.lda + gk];
        if (f.conjA) v.y = -v.y;
        if (g.kscale) { const double sc = g.kscale[gk]; v.x *= sc; v.y *= sc; }
      }
      As[k][m] = v;
    }
#pragma unroll
    for (int s = 0; s < (TN * TK) / NT; ++s) {
      const int e = tid + NT * s;
      int n, k;
      if (f.transB) { n = e / TK; k = e % TK; } else { n = e % TN; k = e / TN; }
      const int gn = t.n0 + n, gk = k0 + k;
      double2 v = make_double2(0.0, 0.0);
      if (gn < g.N && gk < g.K) {
        v = f.transB ? g.B[(size_t)gn * g.ldb + gk] : g.B[(size_t)gk * g.ldb + gn];
        if (f.conjB) v.y = -v.y;
      }
      Bs[k][n] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      double2 a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[k][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[k][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = cfma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
  const bool beta0 = g.beta.x == 0.0 && g.beta.y == 0.0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gm = t.m0 + ty + 16 * r;
    if (gm >= g.M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gn = t.n0 + tx + 16 * c;
      if (gn >= g.N) continue;
      double2 *p = g.C + (size_t)gm * g.ldc + gn;
      double2 v;
      v.x = g.alpha.x * acc[r][c].x - g.alpha.y * acc[r][c].y;
      v.y = g.alpha.x * acc[r][c].y + g.alpha.y * acc[r][c].x;
      if (!beta0) {
        const double2 o = *p;
        v.x += g.beta.x * o.x - g.beta.y * o.y;
        v.y += g.beta.x * o.y + g.beta.y * o.x;
      }
      *p = v;
    }
  }
}

}  // namespace

void zgemm_batched(const std::vector<ZGemm> &batch, const ZGemmFlags &f, cudaStream_t s, Handle &h,
                   int timed_kind, double flops) {
  std::vector<Tile> tiles;
  for (int e = 0; e < (int)batch.size(); ++e) {
    const ZGemm &g = batch[e];
    if (g.M <= 0 || g.N <= 0) continue;
    for (int m0 = 0; m0 < g.M; m0 += TM)
      for (int n0 = 0; n0 < g.N; n0 += TN) {
        if (f.lower_only && n0 > m0) continue;
        tiles.push_back({e, m0, n0});
      }
  }
  if (tiles.empty()) return;
  // one device buffer holds the descriptors followed by the tile list
  const size_t b1 = batch.size() * sizeof(ZGemm), b2 = tiles.size() * sizeof(Tile);
  const size_t off2 = (b1 + 255) / 256 * 256;
  static thread_local std::vector<char> host;
  host.resize(off2 + b2);
  std::memcpy(host.data(), batch.data(), b1);
  std::memcpy(host.data() + off2, tiles.data(), b2);
  DevBuf &args = h.zgemm_args;
  h.ensure(args, off2 + b2);
  LR_CUDA(cudaMemcpyAsync(args.p, host.data(), off2 + b2, cudaMemcpyHostToDevice, s));
  Args a;
  a.g = reinterpret_cast<const ZGemm *>(args.p);
  a.tiles = reinterpret_cast<const Tile *>((const char *)args.p + off2);
  a.f = f;
  Handle::Timed tm{nullptr, nullptr, flops, timed_kind};
  if (timed_kind >= 0) {
    LR_CUDA(cudaEventCreate(&tm.a));
    LR_CUDA(cudaEventCreate(&tm.b));
    LR_CUDA(cudaEventRecord(tm.a, s));
  }
  // the grid is a flat list of tiles; it may exceed 2^31 - 1 only for absurd sizes
  for (size_t t0 = 0; t0 < tiles.size(); t0 += 1u << 30) {
    const unsigned nb = (unsigned)std::min<size_t>(tiles.size() - t0, 1u << 30);
    Args aa = a;
    aa.tiles = a.tiles + t0;
    k_zgemm<<<nb, NT, 0, s>>>(aa);
    ++launch_counter();
  }
  if (timed_kind >= 0) {
    LR_CUDA(cudaEventRecord(tm.b, s));
    h.timed.push_back(tm);
  }
  LR_CUDA(cudaGetLastError());
}

}  // namespace librpa
