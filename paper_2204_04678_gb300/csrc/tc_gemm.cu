// Split-product (3xTF32) GEMM on the fifth-generation tensor cores.
//
//   C[b] = alpha X[b] Y[b]^T + beta C0[b]      (C: n x n, row-major FP32, n % 128 == 0;
//                                               X, Y: n x K, row stride ldx, K % 32 == 0)
//
// It serves two products.  (1) The FP32 selected inversion (K = ldx = n).
// (2) The rank-64 update of the FP32 block sweep, A_IJ -= C_I O_J^T over the
// lower tiles (K = ldx = 64, C = C0 = A, alpha = -1, beta = 1), where the
// 64 x 64 sub-tiles of the pivot row and column, the upper sub-tiles of the
// diagonal 128-blocks and the next pivot's sub-tile (which another kernel
// updates and inverts) are computed but not stored.
//
// Used by the FP32 selected inversion (the Takahashi products of Eq.
// sel_inv_cov on n_s x n_s blocks), where both operands are read along their
// rows: X Y^T with X and Y row-major is a product of two K-major operands.
// Each FP32 value x is split into two TF32 values, x_hi = tf32(x) and
// x_lo = tf32(x - x_hi) (round to nearest, ties away), and
//   X Y^T ~ X_lo Y_hi^T + X_hi Y_lo^T + X_hi Y_hi^T
// is accumulated in FP32 in tensor memory (the X_lo Y_lo^T term is below
// FP32 rounding).  One CTA computes one 128 x 128 tile of C:
//   * all 256 threads load a 128 x 32 slab of X and of Y per stage (coalesced
//     float4 loads, issued one stage ahead), split it, and store the four
//     TF32 slabs into shared memory in the 128-byte swizzled K-major layout;
//   * one thread issues the MMAs (tcgen05.mma kind::tf32, M = N = 128, K = 8;
//     12 per stage) and commits them to the stage's mbarrier, which guards
//     the stage's reuse two stages later (double buffering);
//   * each stage's partial product goes to a pair of 128 x 128 FP32
//     accumulators in tensor memory (X_hi Y_hi^T in one, the two cross terms
//     in the other; two stages x two = all 512 columns), which the threads
//     read back with tcgen05.ld two stages later (each warp its 32-lane
//     quarter, half of the columns) and add into registers.  The tensor
//     cores' own accumulation loses about one FP32 unit in the last place per
//     addition (an error that grows linearly with K: 4.5e-5 relative at
//     K = 1024 when one accumulator took the whole sum), so the large hi*hi
//     partial takes only the 4 MMAs of one 32-deep stage, the small cross
//     terms never round it, and the sum over stages runs in FP32 arithmetic.
// Every mbarrier wait is bounded (2 s of %globaltimer by default; the limit is
// a kernel argument, set process-wide by inla_set_wait_limit); a wait that runs
// out marks the point INLA_ERR_TIMEOUT, skips the epilogue, waits with the full
// 2 s bound for its own copies and MMAs in flight, releases the tensor memory
// and returns.
#include <atomic>
#include <cstdint>
#include <mutex>
#include <stdexcept>
#include <string>

#include "inla_internal.cuh"
#include "tc_common.cuh"

namespace inla {
namespace {

using tc::global_ns;
using tc::mbar_expect_tx;
using tc::mbar_wait;
using tc::smem_addr;
using tc::tmem_ld32;
using tc::WAIT_NS;

constexpr int TCM = 128;                              // tile rows = tile columns
constexpr int TCK = 32;                               // K per stage (one 128-byte swizzle row)
constexpr int TC_THREADS = 256;
constexpr int SLAB_BYTES = TCM * TCK * 4;             // 16 KB per operand slab
constexpr int STAGE_BYTES = 4 * SLAB_BYTES;           // X_hi, X_lo, Y_hi, Y_lo
constexpr int TC_SMEM = 2 * STAGE_BYTES + 1024;       // two stages + alignment slack
constexpr uint32_t TMEM_COLS = 512;                   // 2 stages x {hi*hi, cross terms} x 128 columns

// Instruction descriptor of kind::tf32: D in F32 (bits 4-5 = 1), A and B in
// TF32 (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), N / 8 in
// bits 17-22, M / 16 in bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TCM >> 3) << 17) |
                           ((uint32_t)(TCM >> 4) << 24);

// Shared-memory matrix descriptor: start address / 16 (bits 0-13), leading
// byte offset / 16 (bits 16-29; unused by swizzled K-major operands, set to
// 1), stride byte offset / 16 (bits 32-45: 1024 B between 8-row groups),
// the fixed 0b001 in bits 46-48, swizzle mode 2 = 128-byte in bits 61-63.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(tmem), "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
      : "memory");
}

// Split four FP32 values into TF32 hi / lo parts and store them at byte
// offset `off` of the hi and lo slabs.
__device__ __forceinline__ void split_store(uint8_t *hi, uint8_t *lo, uint32_t off, float4 v) {
  uint4 h, l;
  h.x = tf32_rna(v.x);
  h.y = tf32_rna(v.y);
  h.z = tf32_rna(v.z);
  h.w = tf32_rna(v.w);
  l.x = tf32_rna(v.x - __uint_as_float(h.x));
  l.y = tf32_rna(v.y - __uint_as_float(h.y));
  l.z = tf32_rna(v.z - __uint_as_float(h.z));
  l.w = tf32_rna(v.w - __uint_as_float(h.w));
  *reinterpret_cast<uint4 *>(hi + off) = h;
  *reinterpret_cast<uint4 *>(lo + off) = l;
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    gemm_tf32x3_kernel(int n, int K, int ldx, const float *__restrict__ X, int64_t sX, const float *__restrict__ Y,
                       int64_t sY, float *C, int64_t sC, float alpha, const float *C0, int64_t sC0, float beta,
                       int lower_only, int sweep_pivot, int sweep_next, const int *active, int *status,
                       uint64_t wait_ns) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  int ti, tj;
  if (lower_only) {
    const int t = blockIdx.x;
    ti = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    while (ti * (ti + 1) / 2 > t) --ti;
    tj = t - ti * (ti + 1) / 2;
  } else {
    const int nt = n / TCM;
    ti = blockIdx.x / nt;
    tj = blockIdx.x % nt;
  }
  const int i0 = ti * TCM, j0 = tj * TCM;
  const float *Xb = X + b * sX + (int64_t)i0 * ldx;
  const float *Yb = Y + b * sY + (int64_t)j0 * ldx;

  extern __shared__ uint8_t smraw[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const uint32_t raw = smem_addr(smraw);
  uint8_t *base = smraw + (((raw + 1023u) & ~1023u) - raw);   // 1024-aligned for the swizzle atoms
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar[0])), "r"(1u) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar[1])), "r"(1u) : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  // thread -> (row, 16-byte chunk) of a 128 x 32 slab, four slots per operand
  float4 xv[4], yv[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int idx = tid + TC_THREADS * it, r = idx >> 3, q = idx & 7;
      xv[it] = __ldg(reinterpret_cast<const float4 *>(Xb + (int64_t)r * ldx + k0 + 4 * q));
      yv[it] = __ldg(reinterpret_cast<const float4 *>(Yb + (int64_t)r * ldx + k0 + 4 * q));
    }
  };
  const int nch = K / TCK;
  // This thread's 64 entries of the C tile: row 32 * quarter + lane, columns
  // 64 * half .. 64 * half + 63 (a warp reads only its own 32-lane quarter of TMEM).
  const int quarter = warp & 3, half = warp >> 2;
  const uint32_t lane_addr = (uint32_t)(32 * quarter) << 16;
  float racc[64];
#pragma unroll
  for (int e = 0; e < 64; ++e) racc[e] = 0.0f;
  // add the stage's partial product (TMEM accumulator s) into the registers
  auto drain = [&](int s) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      uint32_t big[32], small[32];
      const uint32_t col = (uint32_t)(2 * s * TCM + half * 64 + cc * 32);
      tmem_ld32(tmem + lane_addr + col, big);
      tmem_ld32(tmem + lane_addr + col + TCM, small);
#pragma unroll
      for (int e = 0; e < 32; ++e) racc[cc * 32 + e] += __uint_as_float(big[e]) + __uint_as_float(small[e]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  };
  load(0);
  bool aborted = false;
  int last = -1;   // last stage whose MMAs were committed
  for (int c = 0; c < nch; ++c) {
    const int s = c & 1;
    if (c >= 2) {
      // stage s and accumulator s are free once the MMAs of chunk c - 2 completed
      const bool ok = mbar_wait(smem_addr(&mbar[s]), (uint32_t)((c - 2) >> 1) & 1u, wait_ns);
      if (__syncthreads_or(!ok)) {
        aborted = true;
        break;
      }
      drain(s);
    }
    uint8_t *st = base + s * STAGE_BYTES;
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int idx = tid + TC_THREADS * it, r = idx >> 3, q = idx & 7;
      const uint32_t off = (uint32_t)(r * 128 + ((q ^ (r & 7)) << 4));
      split_store(st, st + SLAB_BYTES, off, xv[it]);
      split_store(st + 2 * SLAB_BYTES, st + 3 * SLAB_BYTES, off, yv[it]);
    }
    if (c + 1 < nch) load((c + 1) * TCK);   // next slab in flight during this stage's MMAs
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t xh = smem_addr(st), xl = xh + SLAB_BYTES, yh = xh + 2 * SLAB_BYTES, yl = xh + 3 * SLAB_BYTES;
      const uint32_t big = tmem + (uint32_t)(2 * s * TCM), small = big + TCM;
#pragma unroll
      for (int ks = 0; ks < TCK / 8; ++ks) {   // K = 8 TF32 = 32 bytes per MMA
        const uint32_t o = 32u * ks, acc = ks > 0 ? 1u : 0u;
        mma_tf32(small, sw128_desc(xl + o), sw128_desc(yh + o), acc);
        mma_tf32(small, sw128_desc(xh + o), sw128_desc(yl + o), 1u);
        mma_tf32(big, sw128_desc(xh + o), sw128_desc(yh + o), acc);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(&mbar[s]))
                   : "memory");
    }
    last = c;
  }
  if (!aborted) {
    // the last two stages' partial products
    for (int c = nch >= 2 ? nch - 2 : 0; c < nch; ++c) {
      const bool ok = mbar_wait(smem_addr(&mbar[c & 1]), (uint32_t)(c >> 1) & 1u, wait_ns);
      if (__syncthreads_or(!ok)) {
        aborted = true;
        break;
      }
      drain(c & 1);
    }
  }
  if (aborted && last >= 0) {
    // wait (with the full bound, whatever the caller's limit) for the MMAs in flight
    // before the tensor memory is released
    mbar_wait(smem_addr(&mbar[last & 1]), (uint32_t)(last >> 1) & 1u, WAIT_NS);
  }
  // sweep update: this thread's 64 columns lie in one 64 x 64 sub-tile (si, sj)
  const int si = (i0 + 32 * quarter) >> 6, sj = (j0 >> 6) + half;
  const bool skip = sweep_pivot >= 0 && (si == sweep_pivot || sj == sweep_pivot || si < sj ||
                                         (si == sweep_next && sj == sweep_next));
  if (!aborted && !skip) {
    const int row = i0 + 32 * quarter + lane;
    float *crow = C + b * sC + (int64_t)row * n + j0 + half * 64;
    const float *c0row = C0 ? C0 + b * sC0 + (int64_t)row * n + j0 + half * 64 : nullptr;
#pragma unroll
    for (int e = 0; e < 64; e += 4) {
      float4 o = make_float4(alpha * racc[e], alpha * racc[e + 1], alpha * racc[e + 2], alpha * racc[e + 3]);
      if (c0row) {
        const float4 z = *reinterpret_cast<const float4 *>(c0row + e);
        o.x += beta * z.x;
        o.y += beta * z.y;
        o.z += beta * z.z;
        o.w += beta * z.w;
      }
      *reinterpret_cast<float4 *>(crow + e) = o;
    }
  } else if (aborted && tid == 0 && status) {
    status[b] = INLA_ERR_TIMEOUT;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ------------------------------------------------------------------ TMA-fed variant
//
// The selected inversion's two products with operands split into TF32 hi / lo
// parts once in global memory (split_tf32_kernel, and the first product's
// epilogue for its output), so that each stage's four 128 x 32 slabs arrive
// by TMA (cp.async.bulk.tensor, 128-byte swizzle: the K-major layout the MMA
// descriptors read) instead of being loaded, split and stored by the CTA's
// threads.  Three stages of shared memory; the copies of chunk c + 1 are
// issued as soon as the MMAs of chunk c - 2 (the stage's previous user) have
// completed, so that they overlap the MMAs of chunk c - 1 and the drain of
// chunk c - 2.  The MMAs, accumulators, drains and epilogue are those of
// gemm_tf32x3_kernel, in the same order, so the results are the same.
constexpr int TMA_STAGES = 3;
constexpr int TMA_SMEM = TMA_STAGES * STAGE_BYTES + 1024;

__device__ __forceinline__ void tma_load_slab(uint32_t dst, const CUtensorMap *map, int k0, int row0, int b,
                                              uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(k0), "r"(row0), "r"(b), "r"(bar)
      : "memory");
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    gemm_tf32x3_tma_kernel(const __grid_constant__ CUtensorMap mXh, const __grid_constant__ CUtensorMap mXl,
                           const __grid_constant__ CUtensorMap mYh, const __grid_constant__ CUtensorMap mYl, int N,
                           int K, float *C, int64_t ldc, int64_t sC, float alpha, const float *C0, int64_t ldc0,
                           int64_t sC0, float beta, float *Chi, float *Clo, int lower_only, const int *active,
                           int *status, uint64_t wait_ns) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  int ti, tj;
  if (lower_only) {
    const int t = blockIdx.x;
    ti = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    while (ti * (ti + 1) / 2 > t) --ti;
    tj = t - ti * (ti + 1) / 2;
  } else {
    const int nt = N / TCM;
    ti = blockIdx.x / nt;
    tj = blockIdx.x % nt;
  }
  const int i0 = ti * TCM, j0 = tj * TCM;

  extern __shared__ uint8_t smraw[];
  __shared__ uint64_t full[TMA_STAGES];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const uint32_t raw = smem_addr(smraw);
  uint8_t *base = smraw + (((raw + 1023u) & ~1023u) - raw);   // 1024-aligned for the swizzle atoms
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < TMA_STAGES; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&full[i])), "r"(1u) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar[0])), "r"(1u) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar[1])), "r"(1u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  const int nch = K / TCK;
  // the four slabs of chunk c into stage c % TMA_STAGES (thread 0)
  auto issue = [&](int c) {
    const int s = c % TMA_STAGES;
    const uint32_t st = smem_addr(base + s * STAGE_BYTES), bar = smem_addr(&full[s]);
    mbar_expect_tx(bar, (uint32_t)STAGE_BYTES);
    tma_load_slab(st, &mXh, c * TCK, i0, b, bar);
    tma_load_slab(st + SLAB_BYTES, &mXl, c * TCK, i0, b, bar);
    tma_load_slab(st + 2 * SLAB_BYTES, &mYh, c * TCK, j0, b, bar);
    tma_load_slab(st + 3 * SLAB_BYTES, &mYl, c * TCK, j0, b, bar);
  };
  if (tid == 0)
    for (int c = 0; c < TMA_STAGES && c < nch; ++c) issue(c);
  int issued = nch < TMA_STAGES ? nch : TMA_STAGES;   // chunks whose copies were issued

  const int quarter = warp & 3, half = warp >> 2;
  const uint32_t lane_addr = (uint32_t)(32 * quarter) << 16;
  float racc[64];
#pragma unroll
  for (int e = 0; e < 64; ++e) racc[e] = 0.0f;
  auto drain = [&](int s) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      uint32_t big[32], small[32];
      const uint32_t col = (uint32_t)(2 * s * TCM + half * 64 + cc * 32);
      tmem_ld32(tmem + lane_addr + col, big);
      tmem_ld32(tmem + lane_addr + col + TCM, small);
#pragma unroll
      for (int e = 0; e < 32; ++e) racc[cc * 32 + e] += __uint_as_float(big[e]) + __uint_as_float(small[e]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  };
  bool aborted = false;
  int last = -1;     // last chunk whose MMAs were committed
  int consumed = 0;  // chunks whose copies were waited for
  for (int c = 0; c < nch; ++c) {
    const int a = c & 1, s = c % TMA_STAGES;
    if (c >= 2) {
      // accumulator pair a and the stage of chunk c - 2 are free once its MMAs completed
      const bool ok = mbar_wait(smem_addr(&mbar[a]), (uint32_t)((c - 2) >> 1) & 1u, wait_ns);
      if (__syncthreads_or(!ok)) {
        aborted = true;
        break;
      }
      if (tid == 0 && c + 1 < nch) issue(c + 1);
      if (c + 1 < nch) issued = c + 2;
      drain(a);
    }
    const bool ok = mbar_wait(smem_addr(&full[s]), (uint32_t)(c / TMA_STAGES) & 1u, wait_ns);
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    consumed = c + 1;   // only once the copies of chunk c have landed
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t xh = smem_addr(base + s * STAGE_BYTES), xl = xh + SLAB_BYTES, yh = xh + 2 * SLAB_BYTES,
                     yl = xh + 3 * SLAB_BYTES;
      const uint32_t big = tmem + (uint32_t)(2 * a * TCM), small = big + TCM;
#pragma unroll
      for (int ks = 0; ks < TCK / 8; ++ks) {   // K = 8 TF32 = 32 bytes per MMA
        const uint32_t o = 32u * ks, acc = ks > 0 ? 1u : 0u;
        mma_tf32(small, sw128_desc(xl + o), sw128_desc(yh + o), acc);
        mma_tf32(small, sw128_desc(xh + o), sw128_desc(yl + o), 1u);
        mma_tf32(big, sw128_desc(xh + o), sw128_desc(yh + o), acc);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(&mbar[a]))
                   : "memory");
    }
    last = c;
  }
  if (!aborted) {
    for (int c = nch >= 2 ? nch - 2 : 0; c < nch; ++c) {
      const bool ok = mbar_wait(smem_addr(&mbar[c & 1]), (uint32_t)(c >> 1) & 1u, wait_ns);
      if (__syncthreads_or(!ok)) {
        aborted = true;
        break;
      }
      drain(c & 1);
    }
  }
  if (aborted) {
    // wait (with the full bound, whatever the caller's limit) for the copies and the
    // MMAs in flight before the shared and tensor memory are released
    for (int c = consumed; c < issued; ++c)
      mbar_wait(smem_addr(&full[c % TMA_STAGES]), (uint32_t)(c / TMA_STAGES) & 1u, WAIT_NS);
    if (last >= 0) mbar_wait(smem_addr(&mbar[last & 1]), (uint32_t)(last >> 1) & 1u, WAIT_NS);
  }
  if (!aborted) {
    const int row = i0 + 32 * quarter + lane;
    const int64_t off = (int64_t)row * ldc + j0 + half * 64;
    const float *c0row = C0 ? C0 + b * sC0 + (int64_t)row * ldc0 + j0 + half * 64 : nullptr;
#pragma unroll
    for (int e = 0; e < 64; e += 4) {
      float4 o = make_float4(alpha * racc[e], alpha * racc[e + 1], alpha * racc[e + 2], alpha * racc[e + 3]);
      if (c0row) {
        const float4 z = *reinterpret_cast<const float4 *>(c0row + e);
        o.x += beta * z.x;
        o.y += beta * z.y;
        o.z += beta * z.z;
        o.w += beta * z.w;
      }
      if (Chi) {   // the result split for use as the next product's operand
        uint4 h, l;
        h.x = tf32_rna(o.x);
        h.y = tf32_rna(o.y);
        h.z = tf32_rna(o.z);
        h.w = tf32_rna(o.w);
        l.x = tf32_rna(o.x - __uint_as_float(h.x));
        l.y = tf32_rna(o.y - __uint_as_float(h.y));
        l.z = tf32_rna(o.z - __uint_as_float(h.z));
        l.w = tf32_rna(o.w - __uint_as_float(h.w));
        *reinterpret_cast<uint4 *>(Chi + b * sC + off + e) = h;
        *reinterpret_cast<uint4 *>(Clo + b * sC + off + e) = l;
      } else {
        *reinterpret_cast<float4 *>(C + b * sC + off + e) = o;
      }
    }
  } else if (tid == 0 && status) {
    status[b] = INLA_ERR_TIMEOUT;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// hi = tf32(x), lo = tf32(x - hi) for every entry of P matrices of `count` floats.
__global__ void split_tf32_kernel(const float *__restrict__ src, int64_t ssrc, float *__restrict__ hi,
                                  float *__restrict__ lo, int64_t sdst, int64_t count, const int *active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (q >= count) return;
  const float4 v = *reinterpret_cast<const float4 *>(src + b * ssrc + q);
  split_store(reinterpret_cast<uint8_t *>(hi + b * sdst + q), reinterpret_cast<uint8_t *>(lo + b * sdst + q), 0u,
              v);
}

// hi / lo parts of the rows x K block at src (leading dimension lds) of P
// points into compact rows x K arrays (point stride sdst).  K % 4 == 0.
__global__ void split_tf32_2d_kernel(const float *__restrict__ src, int64_t lds, int64_t ssrc, int rows, int K,
                                     float *__restrict__ hi, float *__restrict__ lo, int64_t sdst, const int *active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int q4 = K / 4;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)rows * q4) return;
  const int r = (int)(q / q4), c = (int)(q % q4) * 4;
  const float4 v = *reinterpret_cast<const float4 *>(src + b * ssrc + (int64_t)r * lds + c);
  const int64_t o = b * sdst + (int64_t)r * K + c;
  split_store(reinterpret_cast<uint8_t *>(hi + o), reinterpret_cast<uint8_t *>(lo + o), 0u, v);
}

// P row-major rows x K FP32 matrices, `point_stride` floats apart; one box is a
// 128-row x 32-float slab (128 bytes per row, 128-byte swizzle).
CUtensorMap slab_map(const float *base, int rows, int K, int P, int64_t point_stride) {
  CUtensorMap m;
  const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)P};
  const cuuint64_t strides[2] = {(cuuint64_t)K * 4u, (cuuint64_t)point_stride * 4u};
  const cuuint32_t box[3] = {(cuuint32_t)TCK, (cuuint32_t)TCM, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUresult r = tc::encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box,
                               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw std::runtime_error("cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return m;
}

}  // namespace

namespace tc {
EncodeTiled lookup_encoder() {
  void *p = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
    throw std::runtime_error("the driver does not provide cuTensorMapEncodeTiled");
  return reinterpret_cast<EncodeTiled>(p);
}

EncodeTiled encoder() {
  static const EncodeTiled fn = lookup_encoder();   // initialised once, thread-safe
  return fn;
}
}  // namespace tc

// Bound on one mbarrier wait of the tensor-core kernels (inla_set_wait_limit),
// read at each launch and passed to the kernel.
static std::atomic<uint64_t> g_wait_ns{tc::WAIT_NS};
uint64_t wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }
void set_wait_limit_ns(uint64_t ns) { g_wait_ns.store(ns, std::memory_order_relaxed); }

// Kernel attributes belong to the device's context: set once per device.
void tc_prepare() {
  static std::mutex mu;
  static bool done[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  cudaFuncSetAttribute(gemm_tf32x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  cudaFuncSetAttribute(gemm_tf32x3_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TMA_SMEM);
  prefer_shared(gemm_tf32x3_kernel);
  prefer_shared(gemm_tf32x3_tma_kernel);
  prefer_shared(split_tf32_kernel);
  prefer_shared(split_tf32_2d_kernel);
  done[dev] = true;
}

void split_tf32(Launch &L, int P, const float *src, int64_t ssrc, float *hi, float *lo, int64_t sdst, int64_t count,
                const int *active) {
  const int64_t quads = count / 4;
  split_tf32_kernel<<<dim3((unsigned)((quads + 255) / 256), P), 256, 0, L.st>>>(src, ssrc, hi, lo, sdst, count,
                                                                                 active);
  L.tick();
}

void split_tf32_2d(Launch &L, int P, int rows, int K, const float *src, int64_t lds, int64_t ssrc, float *hi,
                   float *lo, int64_t sdst, const int *active) {
  const int64_t quads = (int64_t)rows * (K / 4);
  split_tf32_2d_kernel<<<dim3((unsigned)((quads + 255) / 256), P), 256, 0, L.st>>>(src, lds, ssrc, rows, K, hi, lo,
                                                                                   sdst, active);
  L.tick();
}

void gemm_nt_tf32x3_split(Launch &L, int P, int M, int N, int K, const float *Xh, const float *Xl, int64_t sX,
                          const float *Yh, const float *Yl, int64_t sY, float *C, int64_t ldc, int64_t sC, float alpha,
                          const float *C0, int64_t ldc0, int64_t sC0, float beta, float *Chi, float *Clo,
                          bool lower_only, const int *active, int *status) {
  if (M % TCM || N % TCM || K % TCK || (lower_only && M != N))
    throw std::runtime_error("gemm_nt_tf32x3_split: M, N % 128 and K % 32 must be 0 (M == N for lower_only)");
  tc_prepare();
  const CUtensorMap mXh = slab_map(Xh, M, K, P, sX), mXl = slab_map(Xl, M, K, P, sX);
  const CUtensorMap mYh = slab_map(Yh, N, K, P, sY), mYl = slab_map(Yl, N, K, P, sY);
  const int tm = M / TCM, tn = N / TCM;
  const int tiles = lower_only ? tm * (tm + 1) / 2 : tm * tn;
  L.start(KID_GEMM, (double)P * tiles * 8.0 * (K / 128.0));   // 8 units of 64^3 per 128 x 128 x 128
  gemm_tf32x3_tma_kernel<<<dim3(tiles, P), TC_THREADS, TMA_SMEM, L.st>>>(
      mXh, mXl, mYh, mYl, N, K, C, ldc, sC, alpha, C0, ldc0, sC0, beta, Chi, Clo, lower_only ? 1 : 0, active, status,
      wait_limit_ns());
  L.stop();
  L.tick();
}

void gemm_nt_tf32x3(Launch &L, int P, int n, const float *X, int64_t sX, const float *Y, int64_t sY, float *C,
                    int64_t sC, float alpha, const float *C0, int64_t sC0, float beta, bool lower_only,
                    const int *active, int *status) {
  tc_prepare();
  const int nt = n / TCM;
  const int tiles = lower_only ? nt * (nt + 1) / 2 : nt * nt;
  L.start(KID_GEMM, (double)P * tiles * nt * 8.0);   // 8 units of 64^3 per 128^3 tile product
  gemm_tf32x3_kernel<<<dim3(tiles, P), TC_THREADS, TC_SMEM, L.st>>>(n, n, n, X, sX, Y, sY, C, sC, alpha, C0, sC0,
                                                                     beta, lower_only ? 1 : 0, -1, -1, active,
                                                                     status, wait_limit_ns());
  L.stop();
  L.tick();
}

void sweep_update_tf32x3(Launch &L, int P, int n_p, float *A, int64_t sA, const float *Cbuf, const float *Obuf,
                         int64_t sCO, int pivot, int next, const int *active, int *status) {
  tc_prepare();
  const int nt2 = n_p / TCM, nt = n_p / 64;
  const int tiles = nt2 * (nt2 + 1) / 2;
  // stored 64^3 sub-tile products: the lower tiles minus the pivot row and column and the next pivot
  const double units = (double)P * (nt * (nt + 1) / 2 - nt - (next >= 0 ? 1 : 0));
  L.start(KID_GJ_UPDATE32, units);
  gemm_tf32x3_kernel<<<dim3(tiles, P), TC_THREADS, TC_SMEM, L.st>>>(n_p, 64, 64, Cbuf, sCO, Obuf, sCO, A, sA, -1.0f,
                                                                     A, sA, 1.0f, 1, pivot, next, active, status,
                                                                     wait_limit_ns());
  L.stop();
  L.tick();
}

}  // namespace inla

// C[b] = X[b] Y[b]^T for a batch of n x n row-major FP32 matrices on the
// tensor cores (3xTF32); see include/inla_gpu.h.
extern "C" int inla_gemm_tf32x3(int n, int batch, const float *X, const float *Y, float *C, int32_t *status,
                                void *stream) {
  if (n <= 0 || n % 128 != 0 || batch <= 0 || !X || !Y || !C) {
    inla::set_error("inla_gemm_tf32x3: n must be a positive multiple of 128, batch > 0, X, Y, C non-NULL");
    return INLA_ERR_ARG;
  }
  if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y) | reinterpret_cast<uintptr_t>(C)) & 15u) {
    inla::set_error("inla_gemm_tf32x3: X, Y and C must be 16-byte aligned");
    return INLA_ERR_ARG;
  }
  inla::Launch L{static_cast<cudaStream_t>(stream), nullptr};
  const int64_t s = (int64_t)n * n;
  if (status) cudaMemsetAsync(status, 0, sizeof(int32_t) * batch, L.st);
  inla::gemm_nt_tf32x3(L, batch, n, X, s, Y, s, C, s, 1.0f, nullptr, 0, 0.0f, false, nullptr, status);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    inla::set_error(cudaGetErrorString(e));
    return INLA_ERR_CUDA;
  }
  return INLA_OK;
}
