// FP64 matrix products on the BF16 tensor cores by error-free splitting of the
// operands (the Ozaki scheme: Ozaki, Ogita, Oishi & Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012; integer
// slices as in Ootomo, Ozaki & Yokota, IJHPCA 2024).
//
//   C[b] = alpha X[b] Y[b]^T + beta C0[b]      X: M x K, Y: N x K, C: M x N (FP64, row-major)
//
// This GPU runs FP64 FMA at 2 per clock per SM, so the library's FP64 dense
// products go to the BF16 tensor cores instead:
//   * Split (ozaki_split_kernel, integer arithmetic only): every row r of an
//     operand gets the power of two 2^e_r above its largest magnitude, and each
//     entry x = 2^e_r * 2^-6 * sum_{a<8} s_a 2^{-7a} + (rounding below 2^{e_r-61}),
//     with integer digits |s_a| <= 64 (exact in BF16) taken from round(x 2^{55-e_r}).
//   * Product: with t_b the digits of Y's rows,
//       X Y^T = 2^{e_r + e_c - 12} sum_L 2^{-7L} P_L,   P_L = sum_{a+b=L} S_a T_b^T,
//     truncated at L <= 7 (36 digit products; the dropped terms are below
//     2^-55 of the row and column maxima).  Each P_L accumulates in FP32 in its
//     own 64-column block of tensor memory: for K <= 1024 every partial sum of
//     P_0..P_3 is an integer of magnitude <= (L+1) K 2^12 <= 2^24, so FP32
//     holds it exactly; P_4..P_7 may round, 2^-24 of terms already 2^-28
//     below the leading one.
//   * Combination (once per 1024 of K): P_0..P_3 as one exact 64-bit integer,
//     P_4..P_7 summed in FP32, then three FP64 operations per output entry (the
//     scaling by powers of two and the conversions are integer operations).
// One CTA computes one 128 x 64 tile of C: 4 warps; thread 0 issues the TMA
// copies (two 96 KB stages: the 8 digit slices of a 128 x 32 slab of X and a
// 64 x 32 slab of Y, 64-byte swizzle) and the MMAs (tcgen05.mma kind::f16, BF16
// inputs, M = 128, N = 64, K = 16; 72 per stage); every thread reads its TMEM
// lane (one row of the tile) for the combination.  Every mbarrier wait is
// bounded (inla_set_wait_limit); a wait that runs out marks the point
// INLA_ERR_TIMEOUT, skips the rest, waits with the full bound for its copies
// and MMAs in flight, releases the tensor memory and returns.
#include <cuda_bf16.h>

#include <cstdint>
#include <mutex>
#include <stdexcept>
#include <string>

#include "inla_internal.cuh"
#include "tc_common.cuh"

namespace inla {
namespace {

using tc::mbar_expect_tx;
using tc::mbar_init;
using tc::mbar_wait;
using tc::mma_commit;
using tc::smem_addr;
using tc::tma_load_4d;
using tc::tmem_ld16;
using tc::WAIT_NS;

constexpr int OZ_M = 128, OZ_N = 64, OZ_KS = 32;             // tile rows, tile columns, K per stage
constexpr int OZ_THREADS = 128;
constexpr int OZ_XBOX = OZ_M * OZ_KS * 2;                    // 8 KB: one digit slice of a 128 x 32 slab
constexpr int OZ_YBOX = OZ_N * OZ_KS * 2;                    // 4 KB
constexpr int OZ_STAGE = OZ_SLICES * (OZ_XBOX + OZ_YBOX);    // 96 KB
constexpr int OZ_SMEM = 2 * OZ_STAGE + 1024;                 // two stages + alignment slack
constexpr int OZ_KSUPER = 1024;                              // K per accumulation in tensor memory
constexpr uint32_t OZ_TMEM_COLS = 512;                       // 8 levels x 64 columns
// Instruction descriptor of kind::f16: D in F32 (bits 4-5 = 1), A and B in BF16
// (bits 7-9 and 10-12 = 1), both K-major, N / 8 in bits 17-22, M / 16 in bits 24-28.
constexpr uint32_t OZ_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_N >> 3) << 17) |
                              ((uint32_t)(OZ_M >> 4) << 24);

// Shared-memory matrix descriptor of a K-major operand in the 64-byte swizzle:
// start address / 16, leading byte offset 1 (unused), stride byte offset
// 512 B / 16 between 8-row groups, the fixed 0b001 in bits 46-48, layout
// type 4 (64-byte swizzle) in bits 61-63.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(tmem), "l"(a), "l"(b), "r"(OZ_IDESC), "r"(accumulate)
      : "memory");
}

// Row r of point b: the exponent e_r (|x| < 2^e_r on the row) and the 8 digit
// slices, stored as S[b][a][r][k] (BF16) and E[b][r].  One warp per row, 8 rows
// per block; up to two operands per launch (rows of both are multiples of 8).
struct SplitJob {
  const double *X;
  int64_t ldx, sX;
  int rows, K;
  uint16_t *S;
  int64_t sS;
  int32_t *E;
  int64_t sE;
};

__global__ void __launch_bounds__(256) ozaki_split_kernel(SplitJob j0, SplitJob j1, int blocks0, const int *active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const bool second = (int)blockIdx.x >= blocks0;
  const SplitJob &J = second ? j1 : j0;
  const int r = ((int)blockIdx.x - (second ? blocks0 : 0)) * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= J.rows) return;
  const int K = J.K;
  const double *xr = J.X + b * J.sX + (int64_t)r * J.ldx;
  int fmax = 0;   // largest biased exponent field of the row (0: zero and subnormal entries only)
  for (int k = lane; k < K; k += 32) {
    const int f = (int)((__double_as_longlong(xr[k]) >> 52) & 0x7FF);
    if (f != 0x7FF) fmax = max(fmax, f);
  }
  for (int o = 16; o > 0; o >>= 1) fmax = max(fmax, __shfl_xor_sync(0xffffffffu, fmax, o));
  const int e = (fmax == 0 ? 1 : fmax) - 1022;   // |x| < 2^e for every normal entry of the row
  if (lane == 0) J.E[b * J.sE + r] = e;
  uint16_t *sr = J.S + b * J.sS + (int64_t)r * K;
  const int64_t plane = (int64_t)J.rows * K;
  for (int k = lane; k < K; k += 32) {
    const int64_t bits = __double_as_longlong(xr[k]);
    const int f = (int)((bits >> 52) & 0x7FF);
    int64_t T = 0;   // round(x 2^(55 - e)), |T| < 2^55
    if (f != 0 && f != 0x7FF) {
      const int64_t m = (bits & ((1ll << 52) - 1)) | (1ll << 52);   // x = +-m 2^(f - 1075)
      const int sh = f - 1075 + 55 - e;                              // <= 2
      if (sh >= 0) T = m << sh;
      else if (sh > -62) T = (m + (1ll << (-sh - 1))) >> (-sh);
      if (bits < 0) T = -T;
    }
    int d[OZ_SLICES];
#pragma unroll
    for (int a = OZ_SLICES - 1; a >= 1; --a) {   // signed base-128 digits in [-64, 63] from the bottom
      const int64_t q = ((T + 64) & 127) - 64;
      d[a] = (int)q;
      T = (T - q) >> 7;
    }
    d[0] = (int)T;   // |d_0| <= 64
#pragma unroll
    for (int a = 0; a < OZ_SLICES; ++a) sr[a * plane + k] = __bfloat16_as_ushort(__float2bfloat16_rn((float)d[a]));
  }
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    ozaki_gemm_kernel(const __grid_constant__ CUtensorMap mX, const __grid_constant__ CUtensorMap mY,
                      const int32_t *__restrict__ Xe, int64_t sXe, const int32_t *__restrict__ Ye, int64_t sYe, int N,
                      int K, double *C, int64_t ldc, int64_t sC, double alpha, const double *C0, int64_t ldc0,
                      int64_t sC0, double beta, int lower_only, const int *active, int *status, uint64_t wait_ns) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  int ti, tj;
  if (lower_only) {   // tiles with tj * 64 < (ti + 1) * 128: row ti holds 2 ti + 2 of them
    const int t = blockIdx.x;
    ti = (int)((sqrtf(4.0f * t + 1.0f) - 1.0f) * 0.5f);
    while ((ti + 1) * (ti + 2) <= t) ++ti;
    while (ti * (ti + 1) > t) --ti;
    tj = t - ti * (ti + 1);
  } else {
    const int nt = N / OZ_N;
    ti = blockIdx.x / nt;
    tj = blockIdx.x % nt;
  }
  const int i0 = ti * OZ_M, j0 = tj * OZ_N;

  extern __shared__ uint8_t smraw[];
  __shared__ uint64_t full[2], done[2];
  __shared__ uint32_t tmem_slot;
  const uint32_t raw = smem_addr(smraw);
  uint8_t *base = smraw + (((raw + 1023u) & ~1023u) - raw);   // 1024-aligned for the swizzle atoms
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_addr(&full[i]), 1u);
      mbar_init(smem_addr(&done[i]), 1u);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  const int nch = K / OZ_KS;
  auto issue = [&](int c) {   // thread 0: the 16 slabs of chunk c into stage c % 2
    const int s = c & 1;
    const uint32_t st = smem_addr(base + s * OZ_STAGE), bar = smem_addr(&full[s]);
    mbar_expect_tx(bar, (uint32_t)OZ_STAGE);
#pragma unroll
    for (int a = 0; a < OZ_SLICES; ++a) tma_load_4d(st + a * OZ_XBOX, &mX, c * OZ_KS, i0, a, b, bar);
#pragma unroll
    for (int a = 0; a < OZ_SLICES; ++a) tma_load_4d(st + OZ_SLICES * OZ_XBOX + a * OZ_YBOX, &mY, c * OZ_KS, j0, a, b, bar);
  };
  if (tid == 0) {
    issue(0);
    if (nch > 1) issue(1);
  }
  int issued = nch > 1 ? 2 : 1;   // chunks whose copies were issued
  int consumed = 0;               // chunks whose copies have landed
  int last = -1;                  // last chunk whose MMAs were committed
  bool aborted = false, first = true;
  const int row = i0 + 32 * warp + lane;   // TMEM lane = row of the tile
  const uint32_t lane_addr = (uint32_t)(32 * warp) << 16;
  const int32_t er = Xe[b * sXe + row];
  const bool unit_alpha = alpha == 1.0 || alpha == -1.0, neg = unit_alpha && alpha < 0.0;
  double *crow = C + b * sC + (int64_t)row * ldc + j0;
  const double *c0row = C0 ? C0 + b * sC0 + (int64_t)row * ldc0 + j0 : nullptr;

  for (int c = 0; c < nch; ++c) {
    const int s = c & 1;
    bool ok = mbar_wait(smem_addr(&full[s]), (uint32_t)(c >> 1) & 1u, wait_ns);
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    consumed = c + 1;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const bool fresh = (c % (OZ_KSUPER / OZ_KS)) == 0;
      const uint32_t xs = smem_addr(base + s * OZ_STAGE), ys = xs + OZ_SLICES * OZ_XBOX;
#pragma unroll
      for (int kk = 0; kk < OZ_KS / 16; ++kk)   // K = 16 BF16 = 32 bytes per MMA
#pragma unroll
        for (int a = 0; a < OZ_SLICES; ++a)
#pragma unroll
          for (int d = 0; a + d < OZ_LEVELS; ++d)
            mma_bf16(tmem + (uint32_t)(OZ_N * (a + d)), sw64_desc(xs + a * OZ_XBOX + 32 * kk),
                     sw64_desc(ys + d * OZ_YBOX + 32 * kk), (fresh && kk == 0 && a == 0) ? 0u : 1u);
      mma_commit(smem_addr(&done[s]));
    }
    last = c;
    if (c >= 1 && c + 1 < nch) {
      // stage (c + 1) % 2 held chunk c - 1: refill it once those MMAs are done
      ok = mbar_wait(smem_addr(&done[(c - 1) & 1]), (uint32_t)((c - 1) >> 1) & 1u, wait_ns);
      if (__syncthreads_or(!ok)) {
        aborted = true;
        break;
      }
      if (tid == 0) issue(c + 1);
      issued = c + 2;
    }
    if ((c + 1) % (OZ_KSUPER / OZ_KS) == 0 || c + 1 == nch) {
      // combine the levels of this part of K into C (all threads, one row each)
      ok = mbar_wait(smem_addr(&done[s]), (uint32_t)(c >> 1) & 1u, wait_ns);
      if (__syncthreads_or(!ok)) {
        aborted = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
      for (int g = 0; g < OZ_N / 16; ++g) {
        int64_t I[16];
        float F[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          I[q] = 0;
          F[q] = 0.0f;
        }
#pragma unroll
        for (int L = 0; L < OZ_LEVELS; ++L) {
          uint32_t v[16];
          tmem_ld16(tmem + lane_addr + (uint32_t)(OZ_N * L + 16 * g), v);
          if (L < 4) {
#pragma unroll
            for (int q = 0; q < 16; ++q) I[q] += (int64_t)__float2int_rn(__uint_as_float(v[q])) << (7 * (3 - L));
          } else {
            const float w = L == 4 ? 1.0f : (L == 5 ? 0x1p-7f : (L == 6 ? 0x1p-14f : 0x1p-21f));
#pragma unroll
            for (int q = 0; q < 16; ++q) F[q] = fmaf(__uint_as_float(v[q]), w, F[q]);
          }
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int j = j0 + 16 * g + q;
          // Three FP64 operations per entry (the FP64 pipe does 2 per clock per SM): the
          // sign of alpha = +-1, the power of two and the float -> double conversion of F
          // are integer operations on the bit patterns.
          int64_t Iq = I[q];
          float Fq = F[q];
          if (neg) {
            Iq = -Iq;
            Fq = -Fq;
          }
          // |I| < 2^51: exact through the 2^52 + 2^51 bias
          const double dI = __longlong_as_double(0x4338000000000000ll + Iq) - 6755399441055744.0;
          // F 2^-7 as a double: exponent rebiased (127 -> 1023, minus 7), mantissa widened
          const uint32_t fb = __float_as_uint(Fq);
          const uint32_t fe = (fb >> 23) & 0xFFu;
          const double dF = fe == 0u ? 0.0
                                     : __longlong_as_double(((int64_t)(fb >> 31) << 63) |
                                                            ((int64_t)(fe + 1023u - 127u - 7u) << 52) |
                                                            ((int64_t)(fb & 0x7FFFFFu) << 29));
          double v = dI + dF;
          if (!unit_alpha) v *= alpha;
          const int k = er + Ye[b * sYe + j] - 33;   // C = 2^k (I + 2^-7 F)
          const int64_t vb = __double_as_longlong(v);
          const int ve = (int)((vb >> 52) & 0x7FF);
          double o;
          if (ve == 0) o = 0.0;
          else if (ve + k > 0 && ve + k < 2047) o = __longlong_as_double(vb + ((int64_t)k << 52));
          else o = ldexp(v, k);
          if (first) {
            if (c0row) o = fma(beta, c0row[16 * g + q], o);
          } else {
            o += crow[16 * g + q];
          }
          crow[16 * g + q] = o;
        }
      }
      first = false;
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();   // the next MMAs overwrite the accumulators
    }
  }
  if (aborted) {
    // wait (with the full bound, whatever the caller's limit) for the copies and the
    // MMAs in flight before the shared and tensor memory are released
    for (int c = consumed; c < issued; ++c) mbar_wait(smem_addr(&full[c & 1]), (uint32_t)(c >> 1) & 1u, WAIT_NS);
    if (last >= 0) mbar_wait(smem_addr(&done[last & 1]), (uint32_t)(last >> 1) & 1u, WAIT_NS);
    if (tid == 0 && status) status[b] = INLA_ERR_TIMEOUT;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
  }
}

// P operands of `rows` x K digit slices (each point's 8 planes contiguous, points
// point_stride elements apart): dims (K, rows, 8, P), one box = 32 x box_rows.
CUtensorMap slice_map(const uint16_t *base, int rows, int K, int P, int64_t point_stride, int box_rows) {
  CUtensorMap m;
  const cuuint64_t dims[4] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)OZ_SLICES, (cuuint64_t)P};
  const cuuint64_t strides[3] = {(cuuint64_t)K * 2u, (cuuint64_t)rows * K * 2u, (cuuint64_t)point_stride * 2u};
  const cuuint32_t box[4] = {(cuuint32_t)OZ_KS, (cuuint32_t)box_rows, 1u, 1u};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  if (point_stride < (int64_t)OZ_SLICES * rows * K) throw std::runtime_error("digit slices overlap");
  const CUresult r = tc::encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<uint16_t *>(base), dims,
                                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw std::runtime_error("cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return m;
}

}  // namespace

void ozaki_prepare() {
  static std::mutex mu;
  static bool done[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  cudaFuncSetAttribute(ozaki_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
  prefer_shared(ozaki_gemm_kernel);
  prefer_shared(ozaki_split_kernel);
  done[dev] = true;
}

void ozaki_split(Launch &L, int P, int rows, int K, const double *X, int64_t ldx, int64_t sX, uint16_t *S,
                 int64_t sS, int32_t *E, int64_t sE, const int *active) {
  const SplitJob j{X, ldx, sX, rows, K, S, sS, E, sE};
  const int blocks = (rows + 7) / 8;
  ozaki_split_kernel<<<dim3(blocks, P), 256, 0, L.st>>>(j, j, blocks, active);
  L.tick();
}

void ozaki_split2(Launch &L, int P, int rows0, int K0, const double *X0, int64_t ldx0, int64_t sX0, uint16_t *S0,
                  int32_t *E0, int rows1, int K1, const double *X1, int64_t ldx1, int64_t sX1, uint16_t *S1,
                  int32_t *E1, int64_t sS, int64_t sE, const int *active) {
  const SplitJob j0{X0, ldx0, sX0, rows0, K0, S0, sS, E0, sE}, j1{X1, ldx1, sX1, rows1, K1, S1, sS, E1, sE};
  const int b0 = (rows0 + 7) / 8, b1 = (rows1 + 7) / 8;
  ozaki_split_kernel<<<dim3(b0 + b1, P), 256, 0, L.st>>>(j0, j1, b0, active);
  L.tick();
}

void gemm_nt_ozaki(Launch &L, int P, int M, int N, int K, const uint16_t *Xs, int64_t sXs, const int32_t *Xe,
                   int64_t sXe, const uint16_t *Ys, int64_t sYs, const int32_t *Ye, int64_t sYe, double *C,
                   int64_t ldc, int64_t sC, double alpha, const double *C0, int64_t ldc0, int64_t sC0, double beta,
                   bool lower_only, const int *active, int *status) {
  if (M % OZ_M || N % OZ_N || K % OZ_KS || (lower_only && M != N))
    throw std::runtime_error("gemm_nt_ozaki: M % 128, N % 64 and K % 32 must be 0 (M == N for lower_only)");
  ozaki_prepare();
  const CUtensorMap mX = slice_map(Xs, M, K, P, sXs, OZ_M), mY = slice_map(Ys, N, K, P, sYs, OZ_N);
  const int tm = M / OZ_M;
  const int tiles = lower_only ? tm * (tm + 1) : tm * (N / OZ_N);
  // units: 64^3 tile products of the algorithmic FP64 product (2 M N K flops)
  L.start(KID_GEMM, (double)P * tiles * OZ_M * OZ_N * (double)K / (64.0 * 64.0 * 64.0));
  ozaki_gemm_kernel<<<dim3(tiles, P), OZ_THREADS, OZ_SMEM, L.st>>>(mX, mY, Xe, sXe, Ye, sYe, N, K, C, ldc, sC, alpha,
                                                                   C0, ldc0, sC0, beta, lower_only ? 1 : 0, active,
                                                                   status, wait_limit_ns());
  L.stop();
  L.tick();
}

}  // namespace inla

// C[b] = X[b] Y[b]^T for a batch of n x n row-major FP64 matrices through the
// digit slices and the BF16 tensor cores; see include/inla_gpu.h.
namespace {
inline size_t rup256(size_t x) { return (x + 255) / 256 * 256; }
}  // namespace

extern "C" size_t inla_gemm_f64_workspace_bytes(int n, int batch) {
  if (n <= 0 || batch <= 0) return 0;
  const size_t slices = (size_t)inla::OZ_SLICES * n * n * 2, exps = (size_t)n * 4;
  return 2 * rup256(slices * batch) + 2 * rup256(exps * batch);
}

extern "C" int inla_gemm_f64(int n, int batch, const double *X, const double *Y, double *C, void *work,
                             size_t work_bytes, int32_t *status, void *stream) {
  if (n <= 0 || n % 128 != 0 || batch <= 0 || !X || !Y || !C || !work) {
    inla::set_error("inla_gemm_f64: n must be a positive multiple of 128, batch > 0, X, Y, C, work non-NULL");
    return INLA_ERR_ARG;
  }
  if (work_bytes < inla_gemm_f64_workspace_bytes(n, batch) || (reinterpret_cast<uintptr_t>(work) & 255u)) {
    inla::set_error("inla_gemm_f64: work must be 256-byte aligned and hold inla_gemm_f64_workspace_bytes(n, batch)");
    return INLA_ERR_ARG;
  }
  try {
    inla::Launch L{static_cast<cudaStream_t>(stream), nullptr};
    const int64_t nn = (int64_t)n * n, ss = (int64_t)inla::OZ_SLICES * nn;
    char *p = static_cast<char *>(work);
    uint16_t *Xs = reinterpret_cast<uint16_t *>(p);
    p += rup256((size_t)ss * 2 * batch);
    uint16_t *Ys = reinterpret_cast<uint16_t *>(p);
    p += rup256((size_t)ss * 2 * batch);
    int32_t *Xe = reinterpret_cast<int32_t *>(p);
    p += rup256((size_t)n * 4 * batch);
    int32_t *Ye = reinterpret_cast<int32_t *>(p);
    if (status) cudaMemsetAsync(status, 0, sizeof(int32_t) * batch, L.st);
    inla::ozaki_split(L, batch, n, n, X, n, nn, Xs, ss, Xe, n, nullptr);
    inla::ozaki_split(L, batch, n, n, Y, n, nn, Ys, ss, Ye, n, nullptr);
    inla::gemm_nt_ozaki(L, batch, n, n, n, Xs, ss, Xe, n, Ys, ss, Ye, n, C, n, nn, 1.0, nullptr, 0, 0, 0.0, false,
                        nullptr, status);
  } catch (const std::exception &e) {
    inla::set_error(e.what());
    return INLA_ERR_CUDA;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    inla::set_error(cudaGetErrorString(e));
    return INLA_ERR_CUDA;
  }
  return INLA_OK;
}
