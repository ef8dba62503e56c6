// FP64-accurate GEMM on the BF16 tensor cores of sm_103a (see ozgemm.h for the scheme).
//
// Operands are split once into BF16 digit planes (k_row_expo + k_digits, or k_plain for plain
// BF16); the GEMM kernel streams them with TMA (cp.async.bulk.tensor) into a shared-memory ring
// and multiplies every digit pair with tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128,
// N = 64, K = 16) into the TMEM accumulator of its diagonal; flush groups (the largest K range
// whose FP32 sums stay exact) are moved into exact int64 register sums, scaled by
// 2^(E_A + E_B - 14 - 8(S-1)) into FP64 at the end.  Every wait on an mbarrier is bounded by the
// global timer; on a timeout the kernel records the failure in *err, waits (bounded) for its own
// copies in flight, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "internal.h"
#include "ozgemm.h"

namespace librpa {
namespace oz {
namespace {

// ------------------------------------------------------------------ splitting

__device__ __forceinline__ int biased_exp(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7FF); }

// balanced base-256 digits of x = v 2^-E (|x| < 1): x ~ sum_s d_s 2^{-7-8(s-1)}, |d_s| <= 128
template <int S>
__device__ __forceinline__ void make_digits(double v, int E, int (&d)[S]) {
  const long long bits = __double_as_longlong(v);
  const int ex = (int)((bits >> 52) & 0x7FF);
#pragma unroll
  for (int s = 0; s < S; ++s) d[s] = 0;
  if (ex == 0) return;   // zero (subnormals are far below any row scale of interest)
  const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
  const int r = 1075 + E - 7 - 8 * (S - 1) - ex;   // W = mant 2^-r, r > 0 since |x| < 1
  long long W = 0;
  if (r <= 0)
    W = mant << (-r);
  else if (r < 62)
    W = (mant + (1LL << (r - 1))) >> r;
  if (bits < 0) W = -W;
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    const long long dg = ((W + 128) & 255) - 128;
    d[s] = (int)dg;
    W = (W - dg) >> 8;
  }
  d[0] = (int)W;
}

struct RealSrc {
  const double *p;
  long long ld, bstride;
  int rows_pb;
  bool trans;
  __device__ double get(int r, int k) const {
    const int b = r / rows_pb, rr = r % rows_pb;
    const double *q = p + b * bstride;
    return trans ? q[(long long)k * ld + rr] : q[(long long)rr * ld + k];
  }
};

struct CplxSrc {
  const double2 *p;
  long long ld, bstride;
  int rows_pb, op;
  bool as_a;
  __device__ double2 opget(const double2 *q, int i, int k) const {
    if (op == OP_N) return q[(long long)i * ld + k];
    if (op == OP_C) {
      const double2 z = q[(long long)i * ld + k];
      return make_double2(z.x, -z.y);
    }
    double2 z = q[(long long)k * ld + i];
    if (op == OP_H) z.y = -z.y;
    return z;
  }
  __device__ double get(int r, int kk) const {
    const int b = r / rows_pb, rr = r % rows_pb;
    const double2 *q = p + b * bstride;
    const int k = kk >> 1, cp = kk & 1;
    if (as_a) {
      const int i = rr >> 1, c = rr & 1;
      const double2 z = opget(q, i, k);
      return c == cp ? z.x : (c == 0 ? -z.y : z.y);
    }
    const double2 z = opget(q, k, rr);
    return cp ? z.y : z.x;
  }
};

struct GatherDev {
  GatherSrc g;
  __device__ static int fold(int a, int n) {
    const int r = a % n;
    return r < 0 ? r + n : r;
  }
  __device__ double get(int r, int k) const {
    const int e = r / g.rows_per_entry, rr = r % g.rows_per_entry;
    const int V = e % g.natoms, gg = (e / g.natoms) % 2, p = e / (2 * g.natoms);
    if (k >= g.m[V]) return 0.0;
    const int *pt = g.pts + 5 * p;
    const int *c = g.lam + 6 * (g.lam_off[V] + k);
    int iR, row, col;
    if (g.kind == 0) {
      const int *u = g.uni + 6 * rr;
      iR = (fold(u[1] - pt[2] - c[1], g.n1) * g.n2 + fold(u[2] - pt[3] - c[2], g.n2)) * g.n3 +
           fold(u[3] - pt[4] - c[3], g.n3);
      row = c[5];
      col = u[5];
    } else {
      iR = (fold(pt[2] + c[1], g.n1) * g.n2 + fold(pt[3] + c[2], g.n2)) * g.n3 + fold(pt[4] + c[3], g.n3);
      row = rr;
      col = c[5];
    }
    const double *Gp = g.G + gg * g.g_gstride + ((long long)pt[1] * g.nR + iR) * g.nao * g.nao;
    return Gp[(long long)row * g.nao + col];
  }
};

struct RaggedSrc {
  const double *base;
  const long long *off;
  const int *Ke;
  int rows_pe;
  __device__ double get(int r, int k) const {
    const int e = r / rows_pe, rr = r % rows_pe;
    const int K = Ke[e];
    return k < K ? base[off[e] + (long long)rr * K + k] : 0.0;
  }
};

// exponent of each row: one warp per row
template <class Src>
__global__ void k_row_expo(Src src, int rows, int K, int row0, int *expo) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= rows) return;
  int m = 0;
  for (int k = lane; k < K; k += 32) m = max(m, biased_exp(src.get(w, k)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) expo[row0 + w] = m - 1022;
}

// one row per blockIdx.x, 4 consecutive k per thread (kpad is a multiple of 8): the row's scale and
// source offsets are fetched once, each plane is written 8 bytes per thread
template <int S, class Src>
__global__ void __launch_bounds__(256) k_digits(Src src, int K, int kpad, int row0, long long plane, const int *expo,
                                                __nv_bfloat16 *dig) {
  const int r = blockIdx.x;
  const int k0 = (blockIdx.y * 256 + threadIdx.x) * 4;
  if (k0 >= kpad) return;
  const int E = expo[row0 + r];
  int d[4][S];
#pragma unroll
  for (int q = 0; q < 4; ++q) make_digits<S>(k0 + q < K ? src.get(r, k0 + q) : 0.0, E, d[q]);
  const long long o = ((long long)row0 + r) * kpad + k0;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    __nv_bfloat162 lo = __floats2bfloat162_rn((float)d[0][s], (float)d[1][s]);
    __nv_bfloat162 hi = __floats2bfloat162_rn((float)d[2][s], (float)d[3][s]);
    uint2 w;
    w.x = *reinterpret_cast<unsigned *>(&lo);
    w.y = *reinterpret_cast<unsigned *>(&hi);
    *reinterpret_cast<uint2 *>(dig + s * plane + o) = w;
  }
}

template <class Src>
__global__ void k_plain(Src src, int rows, int K, int kpad, int row0, __nv_bfloat16 *dig) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (long long)rows * kpad) return;
  const int r = (int)(x / kpad), k = (int)(x % kpad);
  dig[(long long)row0 * kpad + x] = __double2bfloat16(k < K ? src.get(r, k) : 0.0);
}

__device__ __forceinline__ float to_tf32(float f) {   // round to nearest, ties away
  uint32_t t;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(f));
  return __uint_as_float(t);
}

// 3xTF32 split: plane 0 = tf32(x), plane 1 = tf32(x - plane 0)
template <class Src>
__global__ void k_split_tf32x3(Src src, int rows, int K, int kpad, int row0, long long plane, float *dig) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (long long)rows * kpad) return;
  const int r = (int)(x / kpad), k = (int)(x % kpad);
  const double v = k < K ? src.get(r, k) : 0.0;
  const float hi = to_tf32((float)v);
  const long long o = (long long)row0 * kpad + x;
  dig[o] = hi;
  dig[plane + o] = to_tf32((float)(v - (double)hi));
}

// plain TF32: the FP32 value rounded to the 10-bit TF32 mantissa (round to nearest, ties away)
template <class Src>
__global__ void k_plain_tf32(Src src, int rows, int K, int kpad, int row0, float *dig) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (long long)rows * kpad) return;
  const int r = (int)(x / kpad), k = (int)(x % kpad);
  dig[(long long)row0 * kpad + x] = to_tf32((float)(k < K ? src.get(r, k) : 0.0));
}

template <class Src>
void split_any(const Src &src, int rows, int K, int row0, Sliced &o, cudaStream_t s, bool expo_given = false) {
  if (row0 < 0 || row0 + rows > o.rows || K > o.kpad) throw Error{LIBRPA_E_ARG, "split: rows or K exceed the operand"};
  if (rows <= 0) return;
  const int kpad = o.kpad;
  const long long plane = (long long)o.rows * kpad;
  const long long n = (long long)rows * kpad;
  const unsigned g = (unsigned)((n + 255) / 256);
  if (o.S == S_TF32X3) {
    k_split_tf32x3<Src><<<g, 256, 0, s>>>(src, rows, K, kpad, row0, plane, (float *)o.digits);
    ++launch_counter();
    LR_CUDA(cudaGetLastError());
    return;
  }
  if (o.S == 0 || o.S == S_TF32) {
    if (o.S == 0)
      k_plain<Src><<<g, 256, 0, s>>>(src, rows, K, kpad, row0, (__nv_bfloat16 *)o.digits);
    else
      k_plain_tf32<Src><<<g, 256, 0, s>>>(src, rows, K, kpad, row0, (float *)o.digits);
    ++launch_counter();
    LR_CUDA(cudaGetLastError());
    return;
  }
  __nv_bfloat16 *dig = (__nv_bfloat16 *)o.digits;
  if (!expo_given) {
    k_row_expo<Src><<<(unsigned)(((long long)rows * 32 + 255) / 256), 256, 0, s>>>(src, rows, K, row0, o.expo);
    ++launch_counter();
  }
  const dim3 gd((unsigned)rows, (unsigned)((kpad + 1023) / 1024));
  switch (o.S) {
    case 1: k_digits<1, Src><<<gd, 256, 0, s>>>(src, K, kpad, row0, plane, o.expo, dig); break;
    case 2: k_digits<2, Src><<<gd, 256, 0, s>>>(src, K, kpad, row0, plane, o.expo, dig); break;
    case 3: k_digits<3, Src><<<gd, 256, 0, s>>>(src, K, kpad, row0, plane, o.expo, dig); break;
    case 4: k_digits<4, Src><<<gd, 256, 0, s>>>(src, K, kpad, row0, plane, o.expo, dig); break;
    default: k_digits<5, Src><<<gd, 256, 0, s>>>(src, K, kpad, row0, plane, o.expo, dig); break;
  }
  ++launch_counter();
  LR_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------ tcgen05 / TMA / mbarrier

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait: false after ~limit_ns, or as soon as *abort is set (abort may be NULL: the
// waits that drain a CTA's own copies and MMAs before it exits never give up early)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns,
                                          const volatile int *abort = nullptr) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (abort && *abort) return false;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}


// instruction descriptors: D = F32, A and B K-major, M = 128, N = BN; A/B format 1 = BF16
// (kind::f16) or 2 = TF32 (kind::tf32)
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
constexpr uint32_t IDESC_TF32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d), "l"(a), "l"(b), "r"(IDESC), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d), "l"(a), "l"(b), "r"(IDESC_TF32), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// An output tile; c_n >= 0: only the K stages listed at chunks[c_off .. + c_n) (in units of the
// stage's K) are summed -- block-sparse operands, the others multiply exact zeros.
struct Tile {
  int e, m0, n0, c_off, c_n;
};

// ------------------------------------------------------------------ epilogue conversions
// The FP64 pipe of GB300 runs at about 1/64 of its FP32 rate, so the epilogue builds its FP64 (and
// FP32-pair) outputs from the exact int64 digit sums with integer instructions: normalise by the
// leading-one position, round to nearest even, and put the scale 2^sh into the exponent field.
// Results outside the normal range take the FP64 route (rare).

// a 2^sh as FP64, rounded to nearest even
__device__ __forceinline__ double i64_to_f64(long long a, int sh) {
  if (a == 0) return 0.0;
  const unsigned long long neg = a < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long m = a < 0 ? 0ull - (unsigned long long)a : (unsigned long long)a;
  const int lz = __clzll((long long)m);
  m <<= lz;                                    // leading one at bit 63
  unsigned long long mant = m >> 11;           // 53 significant bits
  const unsigned rem = (unsigned)(m & 0x7FFull);
  int e = 1086 - lz + sh;                      // biased exponent: 1023 + (63 - lz) + sh
  if (rem > 0x400u || (rem == 0x400u && (mant & 1ull))) {
    ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++e;
    }
  }
  if (e <= 0 || e >= 2047) return ldexp((double)a, sh);
  return __longlong_as_double((long long)(neg | ((unsigned long long)e << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// u 2^sh as FP32 (u < 2^63), rounded to nearest even; *ok = false outside the normal range
__device__ __forceinline__ float u64_to_f32(unsigned long long u, int sh, bool *ok) {
  if (u == 0) return 0.f;
  const int lz = __clzll((long long)u);
  u <<= lz;
  unsigned mant = (unsigned)(u >> 40);         // 24 significant bits
  const unsigned long long rem = u & 0xFFFFFFFFFFull;
  int e = 190 - lz + sh;                       // biased exponent: 127 + (63 - lz) + sh
  if (rem > 0x8000000000ull || (rem == 0x8000000000ull && (mant & 1u))) {
    ++mant;
    if (mant >> 24) {
      mant >>= 1;
      ++e;
    }
  }
  if (e <= 0 || e >= 255) {
    *ok = false;
    return 0.f;
  }
  return __uint_as_float(((unsigned)e << 23) | (mant & 0x7FFFFFu));
}

// a 2^sh as an unevaluated pair of FP32 numbers (hi, lo): hi = the value rounded to 24 bits, lo =
// the remainder rounded to 24 bits (about 48 significant bits)
__device__ __forceinline__ float2 i64_to_f32x2(long long a, int sh) {
  if (a == 0) return make_float2(0.f, 0.f);
  const bool neg = a < 0;
  unsigned long long m = neg ? 0ull - (unsigned long long)a : (unsigned long long)a;
  const int lz = __clzll((long long)m);
  m <<= lz;                                    // leading one at bit 63; value = m 2^(sh - lz)
  unsigned long long hm = m >> 40;
  long long r = (long long)(m & 0xFFFFFFFFFFull);
  if (r > 0x8000000000ll || (r == 0x8000000000ll && (hm & 1ull))) {
    ++hm;
    r -= 0x10000000000ll;                      // the remainder of the rounded-up hi is negative
  }
  bool ok = true;
  float hi = u64_to_f32(hm, sh - lz + 40, &ok);   // hm <= 2^24: exact
  float lo = u64_to_f32((unsigned long long)(r < 0 ? -r : r), sh - lz, &ok);
  if (!ok) {   // outside the FP32 normal range: through FP64
    const double v = ldexp((double)a, sh);
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
  }
  if (r < 0) lo = -lo;
  return neg ? make_float2(-hi, -lo) : make_float2(hi, lo);
}

template <int S>
__host__ __device__ constexpr uint32_t tmem_cols() {
  return S * BN <= 64 ? 64 : S * BN <= 128 ? 128 : S * BN <= 256 ? 256 : 512;
}
constexpr uint64_t WAIT_NS = 2000000000ull;   // 2 s

// Pipelined, warp-specialised kernel (one CTA = one 128 x 64 output tile of one GEMM entry):
//   warp EW (one lane): TMA producer over a ring of NST shared-memory stages, each holding the
//     NP digit planes of a 128 x 32 A slice and a 64 x 32 B slice (SWIZZLE_64B, K-major);
//   warp EW + 1 (one lane): tcgen05.mma issuer; commits free a stage when its MMAs complete
//     and, at the end of a flush group, signal the epilogue;
//   warps 0..EW-1: epilogue; warp w owns TMEM lanes 32 (w % 4) .. + 31 (= tile rows).  With
//     EW = 8 (digit planes) warp w takes columns 32 (w / 4) .. + 31: after each flush group it
//     moves the diagonal accumulators into exact int64 register sums (32 per thread) and hands
//     the TMEM columns back to the issuer.  With EW = 4 (plain BF16 / TF32, one drain at the
//     end) each warp takes all 64 columns.
constexpr int PBK = 32;   // K per stage: one 64-byte swizzle row of BF16 (16 TF32 values)
constexpr int NST = 3;    // pipeline depth
// epilogue warps of the S variant
__host__ __device__ constexpr int epi_warps(int S) { return (S == 0 || S == S_TF32 || S == S_TF32X3) ? 4 : 8; }

// shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 bytes apart
__device__ __forceinline__ uint64_t smem_desc64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(16 >> 4) << 16;     // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)4 << 61;             // SWIZZLE_64B
  return d;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Operands of the entries of one launch that share them: tensor maps of the A and B digit planes
// (global memory, 128-byte aligned) and their row exponents.
struct alignas(128) MapPair {
  CUtensorMap a, b;
  const int *ea, *eb;
};

// Pipelined, warp-specialised kernel: CTA c takes tiles c, c + gridDim.x, ... (128 x 64 output
// tiles of the launch's entries, sorted by decreasing K range on the host), keeping its barriers and
// TMEM across them (one CTA per tile, or a persistent grid of one CTA per SM: see gemm_multi).
//   warp EW (one lane): TMA producer over a ring of NST shared-memory stages (each the NP digit
//     planes of a 128 x 32 A slice and a 64 x 32 B slice, SWIZZLE_64B, K-major); the ring runs on
//     across tiles, so the next tile's loads overlap this tile's MMAs and epilogue;
//   warp EW + 1 (one lane): tcgen05.mma issuer; commits free a stage when its MMAs complete and, at
//     the end of a flush group, signal the epilogue; the next group (of this or the next tile)
//     starts once the epilogue has drained the accumulators;
//   warps 0..EW-1: epilogue; warp w owns TMEM lanes 32 (w % 4) .. + 31 (= tile rows).  With EW = 8
//     (digit planes) warp w takes columns 32 (w / 4) .. + 31 and after each flush group moves the
//     diagonal accumulators into exact int64 register sums (32 per thread); with EW = 4 (plain
//     BF16 / TF32, one group) each warp takes all 64 columns into registers.  The TMEM columns go
//     back to the issuer before the values are converted and stored, so conversion and stores
//     overlap the next tile's MMAs.
// stall_ns > 0 (testing only): the MMA issuer first waits that long on an mbarrier nothing arrives
// at, so the CTA takes the bounded-wait failure path.  On any failure the CTA sets *err, stops
// issuing, waits (with the full limit) for the TMA copies and MMAs it has already issued, frees its
// TMEM and returns.
template <int S>
__global__ void __launch_bounds__(32 * (epi_warps(S) + 2), 1)
    k_ozgemm(const MapPair *__restrict__ maps, const Entry *__restrict__ entries, const Tile *__restrict__ tiles,
             const int *__restrict__ chunks, int ntiles, int *err, uint64_t stall_ns, int stage_in_ring) {
  constexpr bool TF = S == S_TF32 || S == S_TF32X3;   // kind::tf32
  constexpr bool PLAIN = S == 0 || TF;                 // one FP32 accumulator over all K
  constexpr int NP = S == S_TF32X3 ? 2 : PLAIN ? 1 : S;   // planes per operand
  constexpr int KS = TF ? PBK / 2 : PBK;               // K elements per stage (64 bytes per row)
  constexpr uint32_t A_BYTES = BM * 64, B_BYTES = BN * 64;
  constexpr uint32_t STAGE = NP * (A_BYTES + B_BYTES);
  // K steps per flush group: NP pairs x (32 G) x 2^14 <= 2^24 keeps the FP32 sums exact; plain
  // forms accumulate over the whole K in FP32
  constexpr int G = PLAIN ? (1 << 30) : 32 / NP;
  constexpr int EPI_WARPS = epi_warps(S), HALF = BN * 4 / EPI_WARPS;   // HALF: columns per epilogue warp
  constexpr uint32_t TMEM_COLS = tmem_cols<PLAIN ? 1 : NP>();
  constexpr int SPITCH = 17;   // staging: 32 rows x 16 columns (+1) of 8-byte values per epilogue warp
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[NST], empty[NST], tfull, tempty, mdone, never;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // the epilogue's staging area: in the pipeline's stages when the CTA has a single tile (they are
  // idle once its last MMA completed), else after them
  double *stage_out = reinterpret_cast<double *>(stage_in_ring ? smem : smem + NST * STAGE);
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&tfull, 1);
    mbar_init(&tempty, EPI_WARPS);
    mbar_init(&mdone, 1);
    mbar_init(&never, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_slot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  // K range of a tile: from (m0 km + n0 kn) rounded down to the stage size (triangular operands),
  // or the tile's list of stages
  auto steps_of = [&](const Entry &en, const Tile &tl, int &kbeg) {
    kbeg = (tl.m0 * en.km + tl.n0 * en.kn) / KS * KS;
    if (tl.c_n >= 0) return tl.c_n;
    return en.K > kbeg ? (en.K - kbeg + KS - 1) / KS : 0;
  };
  auto k_of = [&](const Tile &tl, int kbeg, int i) { return tl.c_n >= 0 ? chunks[tl.c_off + i] * KS : kbeg + i * KS; };
  if (warp == EPI_WARPS) {
    if (lane == 0) {
      long long it = 0;   // stages issued so far (all tiles)
      for (int t = blockIdx.x; t < ntiles && !abort_flag; t += gridDim.x) {
        const Tile tl = tiles[t];
        const Entry en = entries[tl.e];
        const MapPair *mp = maps + en.pair;
        int kbeg;
        const int nsteps = steps_of(en, tl, kbeg);
        const int arow = en.a_row0 + tl.m0, brow = en.b_row0 + tl.n0;
        for (int i = 0; i < nsteps; ++i, ++it) {
          const int st = (int)(it % NST);
          if (abort_flag || !mbar_wait(&empty[st], (uint32_t)(((it / NST) & 1) ^ 1), WAIT_NS, &abort_flag)) {
            abort_flag = 1;
            break;
          }
          mbar_expect_tx(&full[st], STAGE);
          uint8_t *sa = smem + st * STAGE, *sb = sa + NP * A_BYTES;
          const int k0 = k_of(tl, kbeg, i);
#pragma unroll
          for (int p = 0; p < NP; ++p) tma_load_3d(sa + p * A_BYTES, &mp->a, &full[st], k0, arow, p);
#pragma unroll
          for (int p = 0; p < NP; ++p) tma_load_3d(sb + p * B_BYTES, &mp->b, &full[st], k0, brow, p);
        }
      }
      // after a failure: the copies of the last NST issued stages may still be in flight (earlier
      // ones were consumed); wait for each to land before the CTA exits
      if (abort_flag)
        for (long long i = it > NST ? it - NST : 0; i < it; ++i)
          mbar_wait(&full[i % NST], (uint32_t)((i / NST) & 1), WAIT_NS);
    }
  } else if (warp == EPI_WARPS + 1) {
    if (lane == 0) {
      if (stall_ns) {   // testing only: a barrier nothing arrives at
        mbar_wait(&never, 0, stall_ns, &abort_flag);
        abort_flag = 1;
      }
      long long it = 0, g = 0;   // stages consumed, flush groups committed (all tiles)
      for (int t = blockIdx.x; t < ntiles && !abort_flag; t += gridDim.x) {
        const Tile tl = tiles[t];
        const Entry en = entries[tl.e];
        int kbeg;
        const int nsteps = steps_of(en, tl, kbeg);
        for (int i = 0; i < nsteps; ++i, ++it) {
          const int st = (int)(it % NST), c = i % G;
          // a new group needs the accumulators drained by the epilogue (previous group, any tile)
          if (c == 0 && g > 0 && (abort_flag || !mbar_wait(&tempty, (uint32_t)((g - 1) & 1), WAIT_NS, &abort_flag))) {
            abort_flag = 1;
            break;
          }
          if (abort_flag || !mbar_wait(&full[st], (uint32_t)((it / NST) & 1), WAIT_NS, &abort_flag)) {
            abort_flag = 1;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + st * STAGE), sb = sa + NP * A_BYTES;
#pragma unroll
          for (int s = 1; s <= NP; ++s)
#pragma unroll
            for (int u = 1; u + s <= NP + 1; ++u)
#pragma unroll
              for (int j = 0; j < 2; ++j) {   // two MMAs of 32 bytes of K per 64-byte row
                const uint64_t da = smem_desc64(sa + (s - 1) * A_BYTES + 32 * j);
                const uint64_t db = smem_desc64(sb + (u - 1) * B_BYTES + 32 * j);
                // digit planes: one accumulator per diagonal s + u; plain forms: one for all
                const uint32_t col = PLAIN ? 0u : (uint32_t)(s + u - 2) * BN;
                const uint32_t accum = (c == 0 && j == 0 && s == 1 && (!PLAIN || u == 1)) ? 0u : 1u;
                if constexpr (TF)
                  umma_tf32(tmem + col, da, db, accum);
                else
                  umma(tmem + col, da, db, accum);
              }
          umma_commit(&empty[st]);
          if (c == G - 1 || i == nsteps - 1) {
            umma_commit(&tfull);
            ++g;
          }
        }
      }
      // after a failure: wait until every MMA this thread issued has completed (they read the
      // shared-memory stages and write TMEM)
      if (abort_flag) {
        umma_commit(&mdone);
        mbar_wait(&mdone, 0, WAIT_NS);
      }
    }
  } else {
    const int quad = warp & 3, half = warp >> 2;   // TMEM lane quadrant, column half
    double *stg = stage_out + (size_t)warp * 32 * SPITCH;
    long long g = 0;   // flush groups drained (all tiles)
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const Tile tl = tiles[t];
      const Entry en = entries[tl.e];
      int kbeg;
      const int nsteps = steps_of(en, tl, kbeg);
      const int ngroups = (nsteps + G - 1) / G;
      const int m0 = tl.m0, n0 = tl.n0;
      long long acc[HALF];       // digit planes: exact int64 sums of the diagonals, or (fpath) an FP32 pair
      uint32_t fa[PLAIN ? HALF : 1];   // plain forms: the FP32 accumulators
#pragma unroll
      for (int j = 0; j < HALF; ++j) acc[j] = 0;
      // FP32-pair outputs of a tile with a single flush group (the short-K GEMMs of the chi0 steps):
      // the diagonal sums, exact integers below 2^24 times their powers of two, are summed into an
      // unevaluated FP32 pair (hi, lo) by exact two-sums, held in the int64 slot's two halves --
      // FP32 arithmetic instead of the int64 sum and its conversion
      const bool fpath = !PLAIN && ngroups == 1 && en.mode == 3 && en.alpha_shift != kNoShift;
      bool ok_all = true;
      for (int gi = 0; gi < ngroups; ++gi, ++g) {
        bool ok = !abort_flag && mbar_wait(&tfull, (uint32_t)(g & 1), WAIT_NS, &abort_flag);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
          abort_flag = 1;
          ok_all = false;
          break;
        }
        tc_fence_after();
        if constexpr (!PLAIN) {
          if (fpath) {
#pragma unroll 1
            for (int d = 2; d <= S + 1; ++d) {
              const float mulf = __uint_as_float((uint32_t)(127 + 8 * (S + 1 - d)) << 23);   // 2^(8(S+1-d))
#pragma unroll
              for (int cb = 0; cb < HALF / 16; ++cb) {
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(d - 2) * BN + half * HALF + cb * 16, r);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                  const int c = cb * 16 + j;
                  const float t = __uint_as_float(r[j]) * mulf;   // exact
                  const float hi = __int_as_float((int)(acc[c] & 0xFFFFFFFFll));
                  float lo = __int_as_float((int)(acc[c] >> 32));
                  const float sm = hi + t, bb = sm - hi;
                  lo += (hi - (sm - bb)) + (t - bb);
                  acc[c] = ((long long)__float_as_int(lo) << 32) | (long long)(uint32_t)__float_as_int(sm);
                }
              }
            }
          } else {
#pragma unroll 1
            for (int d = 2; d <= S + 1; ++d) {
              const long long mul = 1LL << (8 * (S + 1 - d));
#pragma unroll
              for (int cb = 0; cb < HALF / 16; ++cb) {
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(d - 2) * BN + half * HALF + cb * 16, r);
#pragma unroll
                for (int j = 0; j < 16; ++j)
                  acc[cb * 16 + j] += (long long)__float2int_rn(__uint_as_float(r[j])) * mul;
              }
            }
          }
        } else {
#pragma unroll
          for (int cb = 0; cb < HALF / 16; ++cb) {
            uint32_t r[16];
            tmem_ld16(tmem + ((uint32_t)(32 * quad) << 16) + half * HALF + cb * 16, r);
#pragma unroll
            for (int j = 0; j < 16; ++j) fa[cb * 16 + j] = r[j];
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty);   // the accumulators may be overwritten now
      }
      if (!ok_all) break;
      if constexpr (PLAIN) {
        // plain forms: one FP32 sum per element, scaled in FP64 and stored from the registers,
        // thread = tile row
        const int row = m0 + 32 * quad + lane;
        if (row < en.M) {
#pragma unroll
          for (int c = 0; c < HALF; ++c) {
            const int col = n0 + half * HALF + c;
            if (col >= en.N) break;
            if (en.mode == 3 && en.alpha_shift != kNoShift) {   // the FP32 sum times +-2^k: exact in FP32
              const float f = nsteps > 0 ? __uint_as_float(fa[c]) * (float)en.alpha : 0.f;
              reinterpret_cast<float2 *>(en.C)[(long long)row * en.ldc + col] = make_float2(f, 0.f);
              continue;
            }
            const double v = nsteps > 0 ? en.alpha * (double)__uint_as_float(fa[c]) : 0.0;
            if (en.mode == 3) {   // real, as an unevaluated pair of FP32 numbers (hi, lo)
              const float hi = __double2float_rn(v);
              reinterpret_cast<float2 *>(en.C)[(long long)row * en.ldc + col] =
                  make_float2(hi, __double2float_rn(v - (double)hi));
              continue;
            }
            double *p = en.mode == 0   ? en.C + (long long)row * en.ldc + col
                        : en.mode == 1 ? en.C + 2 * ((long long)(row >> 1) * en.ldc + col) + (row & 1)
                        : en.mode == 4 ? en.C + (long long)col * en.ldc + row
                                       : en.C + 2 * ((long long)col * en.ldc + (row >> 1)) + (row & 1);
            *p = en.beta == 0.0 ? v : v + en.beta * *p;
          }
        }
        continue;
      }
      // Digit planes: values are formed with thread = tile row (the TMEM lane layout).  Row-major outputs
      // (modes 0, 1, 3) go through a per-warp staging area, 16 columns at a time, and are written
      // with lanes along the row (two rows of 16 columns per warp store); the transposed outputs
      // (modes 2, 4) are consecutive along rows already and are stored directly.
      const int row = m0 + 32 * quad + lane;
      const bool row_ok = row < en.M;
      const int ea = (!PLAIN && row_ok) ? maps[en.pair].ea[en.a_row0 + row] : 0;
      const int *eb = maps[en.pair].eb;
      const int cbase = n0 + half * HALF;
      const bool pow2 = en.alpha_shift != kNoShift;   // alpha = +-2^alpha_shift: folded into the exponent
      const int ash = pow2 ? en.alpha_shift : 0;
      const bool aneg = pow2 && en.alpha < 0.0;
      const bool staged = en.mode != 2 && en.mode != 4;
#pragma unroll
      for (int cb = 0; cb < HALF / 16; ++cb) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = cb * 16 + j, col = cbase + c;
          const bool ok = row_ok && col < en.N;
          double v = 0.0;
          float2 pr = make_float2(0.f, 0.f);
          if (ok) {
            {
              const int sh = ea + eb[en.b_row0 + col] - 14 - 8 * (S - 1) + ash;
              const long long a = aneg ? -acc[c] : acc[c];
              if (fpath) {
                // renormalise the pair, then scale it by 2^sh (exact in the normal range)
                float hi = __int_as_float((int)(acc[c] & 0xFFFFFFFFll)), lo = __int_as_float((int)(acc[c] >> 32));
                const float sm = hi + lo;
                lo = lo - (sm - hi);
                hi = sm;
                if (aneg) {
                  hi = -hi;
                  lo = -lo;
                }
                const int eh = (int)((__float_as_uint(hi) >> 23) & 0xFF);
                if (sh >= -126 && sh <= 127 && (hi == 0.f || (eh + sh >= 1 && eh + sh <= 254))) {
                  const float sc = __uint_as_float((uint32_t)(sh + 127) << 23);
                  pr = make_float2(hi * sc, lo * sc);
                } else {   // outside the FP32 range of a direct scaling: through FP64
                  const double dv = ldexp((double)hi + (double)lo, sh);
                  pr.x = __double2float_rn(dv);
                  pr.y = __double2float_rn(dv - (double)pr.x);
                }
              } else if (en.mode == 3 && pow2) {
                pr = i64_to_f32x2(a, sh);
              } else {
                v = i64_to_f64(a, sh);
                if (!pow2) v *= en.alpha;
                if (en.mode == 3) {
                  pr.x = __double2float_rn(v);
                  pr.y = __double2float_rn(v - (double)pr.x);
                }
              }
            }
          }
          if (en.mode == 3)
            v = __longlong_as_double(
                (long long)(((unsigned long long)__float_as_uint(pr.y) << 32) | __float_as_uint(pr.x)));
          if (staged) {
            stg[lane * SPITCH + j] = v;
          } else if (ok) {
            double *p = en.mode == 4 ? en.C + (long long)col * en.ldc + row
                                     : en.C + 2 * ((long long)col * en.ldc + (row >> 1)) + (row & 1);
            *p = en.beta == 0.0 ? v : v + en.beta * *p;
          }
        }
        if (staged) {
          __syncwarp();
          const int cl = lane & 15, col = cbase + cb * 16 + cl;
          for (int rr = lane >> 4; rr < 32; rr += 2) {
            const int grow = m0 + 32 * quad + rr;
            if (grow < en.M && col < en.N) {
              const double v = stg[rr * SPITCH + cl];
              if (en.mode == 3) {   // the 8 bytes already hold the pair (hi, lo)
                reinterpret_cast<double *>(en.C)[(long long)grow * en.ldc + col] = v;
              } else {
                double *p = en.mode == 0 ? en.C + (long long)grow * en.ldc + col
                                         : en.C + 2 * ((long long)(grow >> 1) * en.ldc + col) + (grow & 1);
                *p = en.beta == 0.0 ? v : v + en.beta * *p;
              }
            }
          }
          __syncwarp();
        }
      }
    }
  }
  __syncthreads();
  if (abort_flag && tid == 0) atomicExch(err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}


PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

CUtensorMap make_map(const Sliced &o, int box_rows) {
  CUtensorMap m;
  const cuuint64_t eb = (cuuint64_t)elem_bytes(o.S);
  const cuuint64_t dims[3] = {(cuuint64_t)o.kpad, (cuuint64_t)o.rows, (cuuint64_t)planes(o.S)};
  const cuuint64_t strides[2] = {(cuuint64_t)o.kpad * eb, (cuuint64_t)o.kpad * eb * (cuuint64_t)o.rows};
  const cuuint32_t box[3] = {(cuuint32_t)(64 / eb), (cuuint32_t)box_rows, 1};   // 64-byte rows
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType dt = eb == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const CUresult r = g_encode(&m, dt, 3, o.digits, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error{LIBRPA_E_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r)};
  return m;
}

template <int S>
void launch(const MapPair *mp, const Entry *e, const Tile *t, const int *c, int ntiles, int grid, int *err,
            uint64_t stall_ns, cudaStream_t s) {
  // the pipeline's stages and the epilogue's staging area (32 rows x 17 doubles per epilogue warp),
  // overlapping when every CTA has one tile (the shared memory, and so the CTAs an SM holds at
  // once, stay those of the stages alone)
  const int ring = NST * planes(S) * (BM + BN) * 64, staging = epi_warps(S) * 32 * 17 * 8;
  const int in_ring = grid >= ntiles ? 1 : 0;
  const int smem = (in_ring ? std::max(ring, staging) : ring + staging) + 1024;
  LR_CUDA(cudaFuncSetAttribute(k_ozgemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  k_ozgemm<S><<<grid, 32 * (epi_warps(S) + 2), smem, s>>>(mp, e, t, c, ntiles, err, stall_ns, in_ring);
}

}  // namespace

void init() {
  static std::once_flag once;   // handles on several host threads (the serving loop) share it
  std::call_once(once, [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e == cudaSuccess && q == cudaDriverEntryPointSuccess && fn) g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  if (!g_encode) throw Error{LIBRPA_E_CUDA, "cuTensorMapEncodeTiled entry point not available"};
}

size_t sliced_bytes(int rows, int K, int S) {
  const size_t kpad = ((size_t)K + 7) / 8 * 8;
  const size_t dig = ((size_t)planes(S) * rows * kpad * elem_bytes(S) + 255) / 256 * 256;
  return dig + ((size_t)rows * 4 + 255) / 256 * 256;
}

void sliced_bind(Sliced &o, void *mem, int rows, int K, int S) {
  o.rows = rows;
  o.K = K;
  o.kpad = (K + 7) / 8 * 8;
  o.S = S;
  o.digits = mem;
  const size_t dig = ((size_t)planes(S) * rows * o.kpad * elem_bytes(S) + 255) / 256 * 256;
  o.expo = (int *)((char *)mem + dig);
}

void split_real(const double *src, long long ld, bool trans, int rows, int K, int batch, long long batch_stride,
                Sliced &out, cudaStream_t s, int row0) {
  RealSrc r{src, ld, batch_stride, rows, trans};
  split_any(r, rows * batch, K, row0, out, s);
}

void split_complex(const double2 *src, long long ld, Op op, bool as_a, int n_out, int n_k, int batch,
                   long long batch_stride, Sliced &out, cudaStream_t s) {
  const int rows_pb = as_a ? 2 * n_out : n_out;
  CplxSrc c{src, ld, batch_stride, rows_pb, (int)op, as_a};
  split_any(c, rows_pb * batch, 2 * n_k, 0, out, s);
}

void split_gather(const GatherSrc &src, int rows, int K, Sliced &out, cudaStream_t s) {
  GatherDev g{src};
  split_any(g, rows, K, 0, out, s);
}

void split_ragged(const double *base, const long long *off, const int *Ke, int rows_per_entry, int n_entries,
                  int Kmax, Sliced &out, cudaStream_t s, bool expo_given) {
  RaggedSrc r{base, off, Ke, rows_per_entry};
  split_any(r, rows_per_entry * n_entries, Kmax, 0, out, s, expo_given);
}

// out.expo[r] = -1022 (the exponent of an all-zero row) for rows [0, rows)
__global__ void k_expo_init(int *expo, int rows) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < rows) expo[r] = -1022;
}
void expo_init(Sliced &out, int rows, cudaStream_t s) {
  if (rows <= 0) return;
  k_expo_init<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(out.expo, rows);
  ++launch_counter();
  LR_CUDA(cudaGetLastError());
}

long long gemm_multi(const std::vector<std::pair<const Sliced *, const Sliced *>> &ops, const std::vector<Entry> &entries,
                     int *err, cudaStream_t s, Handle &h, DevBuf &args, const StageFn *stage_fn) {
  if (ops.empty()) return 0;
  const int S = ops[0].first->S;
  for (const auto &o : ops)
    if (o.first->S != S || o.second->S != S || S < 0 || (S > SMAX && S != S_TF32 && S != S_TF32X3))
      throw Error{LIBRPA_E_ARG, "oz::gemm: operand mismatch"};
  init();
  // tiles with their K range in stages; MMA flops issued: per tile BM x BN x (K rounded up to the
  // K step) per digit-plane product
  const double prods = (S == 0 || S == S_TF32) ? 1.0 : S == S_TF32X3 ? 3.0 : S * (S + 1) / 2.0;
  const int ks = elem_bytes(S) == 4 ? PBK / 2 : PBK;   // K elements per pipeline stage
  std::vector<std::pair<int, Tile>> tk;
  std::vector<int> chunks, cl;
  double exec = 0;
  h.oz_exec_flops = 0;
  h.oz_alg_flops = 0;
  for (int e = 0; e < (int)entries.size(); ++e) {
    const Entry &en = entries[e];
    if (en.M <= 0 || en.N <= 0) continue;
    if (en.pair < 0 || en.pair >= (int)ops.size()) throw Error{LIBRPA_E_ARG, "oz::gemm: entry without operands"};
    const Sliced &a = *ops[en.pair].first, &b = *ops[en.pair].second;
    if (en.K > a.kpad || en.K > b.kpad || en.a_row0 < 0 || en.b_row0 < 0 || en.a_row0 + en.M > a.rows ||
        en.b_row0 + en.N > b.rows)
      throw Error{LIBRPA_E_ARG, "oz::gemm: entry outside its operands"};
    for (int m0 = 0; m0 < en.M; m0 += BM)
      for (int n0 = 0; n0 < en.N; n0 += BN) {
        // strictly above the diagonal: every column of the tile beyond every row (in output rows,
        // lower_div stacked rows per output row)
        if (en.lower_div > 0 && (long long)n0 * en.lower_div >= (long long)m0 + BM) continue;
        const int rows = std::min(BM, en.M - m0), cols = std::min(BN, en.N - n0);
        cl.clear();
        if (stage_fn && (*stage_fn)(e, m0, rows, n0, cols, ks, en.K, cl)) {
          double kk = 0;
          for (int c : cl) kk += std::min(ks, en.K - c * ks);
          h.oz_alg_flops += 2.0 * rows * cols * kk;
          tk.push_back({(int)cl.size(), Tile{e, m0, n0, (int)chunks.size(), (int)cl.size()}});
          chunks.insert(chunks.end(), cl.begin(), cl.end());
          exec += 2.0 * BM * BN * (double)cl.size() * ks * prods;
          continue;
        }
        const int kbeg = (m0 * en.km + n0 * en.kn) / ks * ks;   // as in the kernel
        const int nst = en.K > kbeg ? (en.K - kbeg + ks - 1) / ks : 0;
        tk.push_back({nst, Tile{e, m0, n0, 0, -1}});
        h.oz_alg_flops += 2.0 * rows * cols * std::max(0, en.K - kbeg);
        exec += 2.0 * BM * BN * (double)nst * ks * prods;
      }
  }
  if (tk.empty()) return 0;
  // the longest K ranges first: CTAs take tiles round-robin, so this evens out their work
  std::stable_sort(tk.begin(), tk.end(), [](const std::pair<int, Tile> &x, const std::pair<int, Tile> &y) {
    return x.first > y.first;
  });
  std::vector<MapPair> mp(ops.size());
  for (size_t i = 0; i < ops.size(); ++i) {
    mp[i].a = make_map(*ops[i].first, BM);
    mp[i].b = make_map(*ops[i].second, BN);
    mp[i].ea = ops[i].first->expo;
    mp[i].eb = ops[i].second->expo;
  }
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t b0 = mp.size() * sizeof(MapPair), off1 = al(b0), b1 = entries.size() * sizeof(Entry),
               off2 = off1 + al(b1), b2 = tk.size() * sizeof(Tile), off3 = off2 + al(b2),
               b3 = std::max<size_t>(1, chunks.size()) * sizeof(int);
  std::vector<char> host(off3 + b3);
  std::memcpy(host.data(), mp.data(), b0);
  std::memcpy(host.data() + off1, entries.data(), b1);
  // alpha = +-2^k goes into the epilogue's exponent arithmetic (every GEMM of the path), other
  // values are multiplied in FP64
  for (size_t e = 0; e < entries.size(); ++e) {
    Entry &en = reinterpret_cast<Entry *>(host.data() + off1)[e];
    int ex = 0;
    const double fr = std::frexp(std::fabs(en.alpha), &ex);
    en.alpha_shift = (en.alpha != 0.0 && fr == 0.5) ? ex - 1 : kNoShift;
  }
  Tile *ht = reinterpret_cast<Tile *>(host.data() + off2);
  for (size_t i = 0; i < tk.size(); ++i) ht[i] = tk[i].second;
  if (!chunks.empty()) std::memcpy(host.data() + off3, chunks.data(), chunks.size() * sizeof(int));
  if (s != h.stream) throw Error{LIBRPA_E_ARG, "oz::gemm: launch on a stream other than the handle's"};
  h.upload_async(args, host.data(), off3 + b3);
  const MapPair *dm = (const MapPair *)args.p;
  const Entry *de = (const Entry *)((const char *)args.p + off1);
  const Tile *dt = (const Tile *)((const char *)args.p + off2);
  const int *dc = (const int *)((const char *)args.p + off3);
  // Grid: when two CTAs' stages fit in an SM's shared memory (fewer than 4 digit planes, the plain
  // forms), one CTA per tile, so that several CTAs per SM hide each other's TMA waits and
  // epilogues; with 4 or 5 planes only one CTA fits, and a persistent grid of one CTA per SM, its
  // ring running on across tiles, was measured faster on GB300 (3.5 % on the chi0 GEMMs).
  const int ring = NST * planes(S) * (BM + BN) * 64;
  int nsm = 0;
  LR_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h.opts.device));
  const int nt = (int)tk.size(), grid = 2 * (ring + 1024) > 227 * 1024 ? std::min(nt, nsm) : nt;
  // testing only: the handle's first opts.test_stall_gemms launches take the failure path
  uint64_t stall = 0;
  if (h.stalls_left > 0) {
    --h.stalls_left;
    stall = 100000;   // 100 us per CTA
  }
  switch (S) {
    case 0: launch<0>(dm, de, dt, dc, nt, grid, err, stall, s); break;
    case 1: launch<1>(dm, de, dt, dc, nt, grid, err, stall, s); break;
    case 2: launch<2>(dm, de, dt, dc, nt, grid, err, stall, s); break;
    case 3: launch<3>(dm, de, dt, dc, nt, grid, err, stall, s); break;
    case 4: launch<4>(dm, de, dt, dc, nt, grid, err, stall, s); break;
    case S_TF32: launch<S_TF32>(dm, de, dt, dc, nt, grid, err, stall, s); break;
    case S_TF32X3: launch<S_TF32X3>(dm, de, dt, dc, nt, grid, err, stall, s); break;
    default: launch<5>(dm, de, dt, dc, nt, grid, err, stall, s); break;
  }
  ++launch_counter();
  LR_CUDA(cudaGetLastError());
  h.oz_exec_flops = exec;
  return nt;
}

long long gemm_grouped(const Sliced &a, const Sliced &b, const std::vector<Entry> &entries, int *err,
                       cudaStream_t s, Handle &h, DevBuf &args, const StageFn *stage_fn) {
  std::vector<Entry> es(entries);
  for (Entry &e : es) e.pair = 0;
  return gemm_multi({{&a, &b}}, es, err, s, h, args, stage_fn);
}

long long gemm(const Sliced &a, const Sliced &b, int M, int N, int batch, const Out &out, int km, int kn,
               int lower_div, int *err, cudaStream_t s, Handle &h) {
  if (a.K != b.K) throw Error{LIBRPA_E_ARG, "oz::gemm: K mismatch"};
  // an operand holding a single entry is shared by every batch entry
  const int a_pb = (batch > 1 && a.rows == M) ? 0 : a.rows / batch;
  const int b_pb = (batch > 1 && b.rows == N) ? 0 : b.rows / batch;
  std::vector<Entry> es(batch);
  for (int i = 0; i < batch; ++i) {
    Entry &e = es[i];
    e.a_row0 = i * a_pb;
    e.b_row0 = i * b_pb;
    e.M = M;
    e.N = N;
    e.K = a.K;
    e.km = km;
    e.kn = kn;
    e.lower_div = lower_div;
    e.C = out.C + (long long)i * out.batch_stride * (out.mode == 0 || out.mode == 4 ? 1 : 2);
    e.ldc = out.ldc;
    e.mode = out.mode;
    e.alpha = out.alpha;
    e.beta = out.beta;
  }
  return gemm_grouped(a, b, es, err, s, h, h.oz_args);
}

}  // namespace oz
}  // namespace librpa
