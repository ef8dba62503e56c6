// FP64-accurate GEMM on the BF16 tensor cores of sm_103a (see ozgemm.h for the scheme).
//
// Kernel structure (one CTA = one 128 x 64 output tile, 4 warps):
//   * thread 0 issues TMA loads (cp.async.bulk.tensor, SWIZZLE_128B, K-major) of the S digit
//     planes of the A tile (128 x 64) and of the B tile (64 x 64) for each 64-wide K step, then
//     the tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128, N = 64, K = 16) of every digit
//     pair into the TMEM accumulator of its diagonal, and commits to an mbarrier;
//   * after a flush group of K steps (the largest group whose FP32 sums stay exact) all four
//     warps read the accumulators (tcgen05.ld 32x32b, warp w owns TMEM lanes 32w..32w+31 = tile
//     rows), convert them to integers and add them into exact int64 register sums;
//   * the final int64 sums are scaled by 2^(E_A + E_B - 14 - 8(S-1)) into FP64.
// Every wait on an mbarrier is bounded by the global timer; on a timeout the kernel records the
// failure in *err, waits (bounded) for its own copies in flight, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <string>

#include "internal.h"
#include "ozgemm.h"

namespace librpa {
namespace oz {
namespace {

// ------------------------------------------------------------------ splitting

__device__ __forceinline__ int biased_exp(double v) {
  return (int)((__double_as_longlong(v) >> 52) & 0x7FF);
}

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

// exponent of each row: one warp per row
template <class Src>
__global__ void k_row_expo(Src src, int rows, int K, int *expo) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= rows) return;
  int m = 0;
  for (int k = lane; k < K; k += 32) m = max(m, biased_exp(src.get(w, k)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) expo[w] = m - 1022;
}

template <int S, class Src>
__global__ void k_digits(Src src, int rows, int K, int kpad, const int *expo, __nv_bfloat16 *dig) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (long long)rows * kpad) return;
  const int r = (int)(x / kpad), k = (int)(x % kpad);
  int d[S];
  make_digits<S>(k < K ? src.get(r, k) : 0.0, expo[r], d);
  const long long plane = (long long)rows * kpad;
#pragma unroll
  for (int s = 0; s < S; ++s) dig[s * plane + x] = __float2bfloat16_rn((float)d[s]);
}

template <class Src>
void split_any(const Src &src, Sliced &o, cudaStream_t s) {
  const int rows = o.rows, K = o.K, kpad = o.kpad;
  k_row_expo<Src><<<(unsigned)(((long long)rows * 32 + 255) / 256), 256, 0, s>>>(src, rows, K, o.expo);
  const long long n = (long long)rows * kpad;
  const unsigned g = (unsigned)((n + 255) / 256);
  switch (o.S) {
    case 1: k_digits<1, Src><<<g, 256, 0, s>>>(src, rows, K, kpad, o.expo, o.digits); break;
    case 2: k_digits<2, Src><<<g, 256, 0, s>>>(src, rows, K, kpad, o.expo, o.digits); break;
    case 3: k_digits<3, Src><<<g, 256, 0, s>>>(src, rows, K, kpad, o.expo, o.digits); break;
    case 4: k_digits<4, Src><<<g, 256, 0, s>>>(src, rows, K, kpad, o.expo, o.digits); break;
    default: k_digits<5, Src><<<g, 256, 0, s>>>(src, rows, K, kpad, o.expo, o.digits); break;
  }
  launch_counter() += 2;
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
// bounded wait: false after ~limit_ns
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
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

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(16 >> 4) << 16;     // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // SWIZZLE_128B
  return d;
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = BN
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d), "l"(a), "l"(b), "r"(IDESC), "r"(acc)
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

struct KArgs {
  int M, N, K;
  int a_rows_pb, b_rows_pb;   // rows of one batch entry in the A / B digit planes
  const int *ea, *eb;
  Out out;
  int km, kn, lower_div;
  int *err;
};

template <int S>
__host__ __device__ constexpr uint32_t tmem_cols() {
  return S * BN <= 64 ? 64 : S * BN <= 128 ? 128 : S * BN <= 256 ? 256 : 512;
}
constexpr uint64_t WAIT_NS = 2000000000ull;   // 2 s

template <int S>
__global__ void __launch_bounds__(128, 1)
    k_ozgemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const KArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM, bz = blockIdx.z;
  if (a.lower_div > 0 && n0 > m0 / a.lower_div) return;
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *sA = smem;                    // S planes of 128 x 64 BF16 (16 KB each)
  uint8_t *sB = smem + S * BM * BK * 2;  // S planes of  64 x 64 BF16 ( 8 KB each)
  constexpr uint32_t TX = S * (BM + BN) * BK * 2;
  constexpr int G = 16 / S;              // K steps per flush: S pairs x (64 G) x 2^14 <= 2^24
  if (tid == 0) {
    mbar_init(&bar_tma, 1);
    mbar_init(&bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  constexpr uint32_t TMEM_COLS = tmem_cols<S>();
  if (warp == 0) tmem_alloc(&tmem_slot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  long long acc[BN];
#pragma unroll
  for (int j = 0; j < BN; ++j) acc[j] = 0;
  int kbeg = m0 * a.km + n0 * a.kn;
  kbeg = kbeg / BK * BK;
  const int nsteps = a.K > kbeg ? (a.K - kbeg + BK - 1) / BK : 0;
  uint32_t ph_tma = 0, ph_mma = 0;
  const int arow = bz * a.a_rows_pb + m0, brow = bz * a.b_rows_pb + n0;
  bool failed = false;
  for (int g0 = 0; g0 < nsteps && !failed; g0 += G) {
    const int gn = min(G, nsteps - g0);
    for (int c = 0; c < gn; ++c) {
      const int k0 = kbeg + (g0 + c) * BK;
      if (tid == 0) {
        mbar_expect_tx(&bar_tma, TX);
#pragma unroll
        for (int s = 0; s < S; ++s) tma_load_3d(sA + s * BM * BK * 2, &tmA, &bar_tma, k0, arow, s);
#pragma unroll
        for (int s = 0; s < S; ++s) tma_load_3d(sB + s * BN * BK * 2, &tmB, &bar_tma, k0, brow, s);
      }
      bool ok = mbar_wait(&bar_tma, ph_tma, WAIT_NS);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      ph_tma ^= 1;
      if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int s = 1; s <= S; ++s)
#pragma unroll
          for (int t = 1; t + s <= S + 1; ++t) {
            const uint32_t dt = tmem + (uint32_t)(s + t - 2) * BN;
            const uint32_t abase = smem_u32(sA + (s - 1) * BM * BK * 2);
            const uint32_t bbase = smem_u32(sB + (t - 1) * BN * BK * 2);
#pragma unroll
            for (int j = 0; j < BK / 16; ++j)
              umma(dt, smem_desc(abase + 32 * j), smem_desc(bbase + 32 * j), (c == 0 && j == 0 && s == 1) ? 0u : 1u);
          }
        umma_commit(&bar_mma);
      }
      ok = mbar_wait(&bar_mma, ph_mma, WAIT_NS);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      ph_mma ^= 1;
    }
    if (failed) break;
    tc_fence_after();
    // flush the diagonals of this group into the int64 sums
#pragma unroll
    for (int d = 2; d <= S + 1; ++d) {
      const long long mul = 1LL << (8 * (S + 1 - d));
#pragma unroll
      for (int cb = 0; cb < BN / 16; ++cb) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(d - 2) * BN + cb * 16, r);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[cb * 16 + j] += (long long)__float2int_rn(__uint_as_float(r[j])) * mul;
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  if (failed) {
    if (tid == 0) atomicExch(a.err, 1);
    // let copies and MMAs already issued land before the CTA gives up its memory
    mbar_wait(&bar_tma, ph_tma, WAIT_NS);
    mbar_wait(&bar_mma, ph_mma, WAIT_NS);
  } else {
    const int row = m0 + 32 * warp + lane;
    if (row < a.M) {
      const int ea = a.ea[(long long)bz * a.a_rows_pb + row];
      const Out &o = a.out;
#pragma unroll
      for (int j = 0; j < BN; ++j) {
        const int col = n0 + j;
        if (col >= a.N) break;
        const int e = ea + a.eb[(long long)bz * a.b_rows_pb + col] - 14 - 8 * (S - 1);
        const double v = o.alpha * ldexp((double)acc[j], e);
        double *p;
        if (o.mode == 0)
          p = o.C + (long long)bz * o.batch_stride + (long long)row * o.ldc + col;
        else if (o.mode == 1)
          p = o.C + 2 * ((long long)bz * o.batch_stride + (long long)(row >> 1) * o.ldc + col) + (row & 1);
        else
          p = o.C + 2 * ((long long)bz * o.batch_stride + (long long)col * o.ldc + (row >> 1)) + (row & 1);
        *p = o.beta == 0.0 ? v : v + o.beta * *p;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

CUtensorMap make_map(const Sliced &o, int box_rows) {
  CUtensorMap m;
  const cuuint64_t dims[3] = {(cuuint64_t)o.kpad, (cuuint64_t)o.rows, (cuuint64_t)o.S};
  const cuuint64_t strides[2] = {(cuuint64_t)o.kpad * 2, (cuuint64_t)o.kpad * 2 * (cuuint64_t)o.rows};
  const cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = g_encode(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)o.digits, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error{LIBRPA_E_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r)};
  return m;
}

template <int S>
void launch(const CUtensorMap &ma, const CUtensorMap &mb, const KArgs &ka, dim3 grid, cudaStream_t s) {
  const int smem = S * (BM + BN) * BK * 2 + 1024;
  LR_CUDA(cudaFuncSetAttribute(k_ozgemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  k_ozgemm<S><<<grid, 128, smem, s>>>(ma, mb, ka);
}

}  // namespace

void init() {
  if (g_encode) return;
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
    throw Error{LIBRPA_E_CUDA, "cuTensorMapEncodeTiled entry point not available"};
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
}

size_t sliced_bytes(int rows, int K, int S) {
  const size_t kpad = ((size_t)K + 7) / 8 * 8;
  const size_t dig = ((size_t)S * rows * kpad * 2 + 255) / 256 * 256;
  return dig + ((size_t)rows * 4 + 255) / 256 * 256;
}

void sliced_bind(Sliced &o, void *mem, int rows, int K, int S) {
  o.rows = rows;
  o.K = K;
  o.kpad = (K + 7) / 8 * 8;
  o.S = S;
  o.digits = (__nv_bfloat16 *)mem;
  const size_t dig = ((size_t)S * rows * o.kpad * 2 + 255) / 256 * 256;
  o.expo = (int *)((char *)mem + dig);
}

void split_real(const double *src, long long ld, bool trans, int rows, int K, int batch, long long batch_stride,
                Sliced &out, cudaStream_t s) {
  RealSrc r{src, ld, batch_stride, rows, trans};
  if (out.rows != rows * batch || out.K != K) throw Error{LIBRPA_E_ARG, "split_real: operand shape mismatch"};
  split_any(r, out, s);
}

void split_complex(const double2 *src, long long ld, Op op, bool as_a, int n_out, int n_k, int batch,
                   long long batch_stride, Sliced &out, cudaStream_t s) {
  const int rows_pb = as_a ? 2 * n_out : n_out;
  CplxSrc c{src, ld, batch_stride, rows_pb, (int)op, as_a};
  if (out.rows != rows_pb * batch || out.K != 2 * n_k) throw Error{LIBRPA_E_ARG, "split_complex: operand shape mismatch"};
  split_any(c, out, s);
}

long long gemm(const Sliced &a, const Sliced &b, int M, int N, int batch, const Out &out, int km, int kn,
               int lower_div, int *err, cudaStream_t s) {
  if (a.S != b.S || a.K != b.K || a.S < 1 || a.S > SMAX) throw Error{LIBRPA_E_ARG, "oz::gemm: operand mismatch"};
  init();
  const CUtensorMap ma = make_map(a, BM), mb = make_map(b, BN);
  KArgs ka;
  ka.M = M;
  ka.N = N;
  ka.K = a.K;
  // an operand holding a single entry is shared by every batch entry
  ka.a_rows_pb = (batch > 1 && a.rows == M) ? 0 : a.rows / batch;
  ka.b_rows_pb = (batch > 1 && b.rows == N) ? 0 : b.rows / batch;
  ka.ea = a.expo;
  ka.eb = b.expo;
  ka.out = out;
  ka.km = km;
  ka.kn = kn;
  ka.lower_div = lower_div;
  ka.err = err;
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), (unsigned)batch);
  switch (a.S) {
    case 1: launch<1>(ma, mb, ka, grid, s); break;
    case 2: launch<2>(ma, mb, ka, grid, s); break;
    case 3: launch<3>(ma, mb, ka, grid, s); break;
    case 4: launch<4>(ma, mb, ka, grid, s); break;
    default: launch<5>(ma, mb, ka, grid, s); break;
  }
  ++launch_counter();
  LR_CUDA(cudaGetLastError());
  return (long long)grid.x * grid.y * grid.z;
}

}  // namespace oz
}  // namespace librpa
