// Dense kernels on n_p x n_p blocks (n_p a multiple of 64), batched over the
// evaluation points of a wave (blockIdx.y = point).  The storage type R of the
// blocks is double (FP64 path) or float (mixed path); pivot-block inversions
// and log-determinants are always computed in double.
//
// 1. Symmetric positive-definite inversion by the block sweep (Gauss-Jordan)
//    operator.  The block factorisation of Q_c used here is the block form of
//    Q = V D V^T (Sec. 2.4.2, Eq. takahashi_identity) with D = blockdiag(D_t):
//    every step needs D_t^-1 and log|D_t|.  Sweeping pivot block K of a
//    symmetric A replaces
//        A_KK -> -A_KK^-1,  A_IK -> A_IK A_KK^-1,  A_IJ -> A_IJ - A_IK A_KK^-1 A_KJ,
//    and after all pivot blocks A holds -A^-1; the pivots are the successive
//    Schur complements, so log|A| = sum_K log|pivot_K| and a non-positive
//    pivot means A is not positive definite.  Each sweep step is one small
//    (32 x 32) pivot inversion followed by a rank-32 update of the whole
//    lower triangle, which spreads over every SM (no triangular solves on
//    the critical path).  Work: n^3 flops, the same as Cholesky + inverse.
// 2. C = alpha A B + beta C0 for the selected-inversion products.
//
// In FP64 the kernels are bound by the FP64 pipe; all operand traffic is
// staged through shared memory with conflict-free access (padded rows).
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "inla_internal.cuh"

namespace inla {

// defined with the blocked inversion below; declared here for ensure_attrs
template <typename R>
__global__ void transpose_kernel(const R *__restrict__ src, int64_t lds, int64_t ss, R *__restrict__ dst,
                                 int64_t ldd, int64_t sd, int rows, int cols, const int *active);

namespace {

constexpr int T = TILE;     // 64
constexpr int LDS = T + 1;  // padded shared-memory row

// Row and column of the x-th lower tile.  Single-precision square root plus an
// integer correction: no instruction of this lands on the FP64 pipe, which
// the tile products saturate.
__device__ __forceinline__ void tri_index(int x, int &I, int &J) {
  int i = (int)((sqrtf(8.0f * (float)x + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= x) ++i;
  while (i * (i + 1) / 2 > x) --i;
  I = i;
  J = x - i * (i + 1) / 2;
}

// ---------------------------------------------------------------- block sweep
// Pivot blocks and update tiles are G x G: G = 32 in FP64 (128 threads, 2 x 4
// outputs per thread) and G = 64 in FP32 (256 threads, 4 x 4 outputs per
// thread).  One update launch has P * nt(nt+1)/2 blocks that balance well over
// the 152 SMs.
template <int G>
struct Sweep {
  static constexpr int LD = G + 1;                         // padded shared-memory row
  static constexpr int TX = G / 4;                         // threads along a tile row
  static constexpr int THREADS = 4 * G;                    // 16 rows of threads
  static constexpr int MI = G / 16;                        // output rows per thread
  static constexpr int TRI = G * (G + 1) / 2;              // lower entries
  static constexpr int PER = (TRI + THREADS - 1) / THREADS;
  static constexpr int SMEM_ELEMS = G * LD + 16 * 17 + 2 * G * 16 + G;   // sweep workspace (both forms)
  static constexpr int SHIFT = G == 32 ? 5 : 6;
};

// Inversion of a G x G SPD block held (lower triangle) in shared memory, by the
// same sweep applied recursively: for each 16-wide sub-pivot, one warp sweeps
// the 16 x 16 sub-pivot element by element (warp-synchronous), then all
// threads form the sub-panel C = A_iK P_K and apply the rank-16 update to the
// whole block.  On return Pout holds A^-1 (full symmetric tile) and *logdet
// has gained log|A| = sum of log pivots (accumulated in double); a non-positive
// pivot sets *status.  Arithmetic in the storage type R.  Called by all
// Sweep<G>::THREADS threads; shared workspace Sweep<G>::SMEM_ELEMS elements.
constexpr int SB = 16;
template <typename R, int G>
__device__ void sweep_tile_blocked(R *sm, R *Pout, double *logdet, int *status) {
  using S = Sweep<G>;
  constexpr int LD = S::LD;
  R *a = sm;                          // [G][LD]   full symmetric working copy
  R *sp = sm + G * LD;                // [SB][SB+1] sub-pivot, then its inverse
  R *Cp = sp + SB * (SB + 1);         // [G][SB]   sub-panel C = A_iK P
  R *Op = Cp + G * SB;                // [SB][G]   old column block A_iK, transposed
  R *pv = Op + G * SB;                // [G]       scalar pivots
  __shared__ int s_bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // mirror the lower triangle so that the working copy is full
  for (int e = tid; e < G * G; e += S::THREADS) {
    const int i = e >> S::SHIFT, j = e & (G - 1);
    if (j > i) a[i * LD + j] = a[j * LD + i];
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int kb = 0; kb < G / SB; ++kb) {
    const int K0 = kb * SB;
    if (warp == 0) {
      // 1. scalar sweep of the 16 x 16 sub-pivot by one warp, in registers:
      //    lane l holds entries (2 q + l / 16, l % 16), q < 8; the pivot row and
      //    column reach every lane by shuffles, so a pivot step is a short
      //    dependency chain (shuffle, reciprocal, one FMA) with no shared memory
      R v[8];
      const int hi = lane >> 4, j = lane & 15;
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = a[(K0 + 2 * q + hi) * LD + K0 + j];
      bool bad = false;
#pragma unroll
      for (int p = 0; p < SB; ++p) {
        const int qp = p >> 1, lp = ((p & 1) << 4);
        const R piv = __shfl_sync(0xffffffffu, v[qp], lp + p);
        const bool ok = (piv > R(0)) && (piv < R(INFINITY));
        if (!ok) bad = true;
        const R inv = ok ? R(1) / piv : R(0);
        const R pj = __shfl_sync(0xffffffffu, v[qp], lp + j);        // entry (p, j)
        R ip[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) ip[q] = __shfl_sync(0xffffffffu, v[q], (lane & 16) + p);   // entry (i, p)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = 2 * q + hi;
          if (i == p) v[q] = (j == p) ? -inv : pj * inv;
          else if (j == p) v[q] = ip[q] * inv;
          else v[q] = fma(-ip[q] * inv, pj, v[q]);
        }
        if (lane == 0) pv[K0 + p] = ok ? piv : R(1);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) sp[(2 * q + hi) * (SB + 1) + j] = v[q];
      if (bad && lane == 0) s_bad = 1;
      // sp now holds -P, P = (sub-pivot)^-1
    }
    __syncthreads();
    // 2. sub-panel C_i = A_iK P for rows i outside the sub-pivot; keep the old
    //    A_iK, transposed (OpT[c][i]) so that step 3 reads it without bank conflicts
    for (int e = tid; e < G * SB; e += S::THREADS) {
      const int i = e / SB, c = e % SB;
      if (i >= K0 && i < K0 + SB) continue;
      R acc = 0;
#pragma unroll
      for (int k = 0; k < SB; ++k) acc = fma(a[i * LD + K0 + k], -sp[k * (SB + 1) + c], acc);
      Cp[i * SB + c] = acc;
      Op[c * G + i] = a[i * LD + K0 + c];
    }
    __syncthreads();
    // 3. rank-SB update of everything outside the sub-pivot rows/columns (each
    //    thread a MI x 4 patch: rows ty + 16 i, columns tx + TX j, the product
    //    summed first and subtracted once); the sub-pivot row/column become C,
    //    the sub-pivot block -P
    {
      const int tx = tid % S::TX, ty = tid / S::TX;
      R u[S::MI][4];
#pragma unroll
      for (int i = 0; i < S::MI; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) u[i][j] = R(0);
#pragma unroll
      for (int c = 0; c < SB; ++c) {
        R cv[S::MI], ov[4];
#pragma unroll
        for (int i = 0; i < S::MI; ++i) cv[i] = Cp[(ty + 16 * i) * SB + c];
#pragma unroll
        for (int j = 0; j < 4; ++j) ov[j] = Op[c * G + tx + S::TX * j];
#pragma unroll
        for (int i = 0; i < S::MI; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) u[i][j] = fma(cv[i], ov[j], u[i][j]);
      }
      R w[S::MI][4];
#pragma unroll
      for (int i = 0; i < S::MI; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int r = ty + 16 * i, c = tx + S::TX * j;
          const bool ik = r >= K0 && r < K0 + SB, jk = c >= K0 && c < K0 + SB;
          if (ik && jk) w[i][j] = sp[(r - K0) * (SB + 1) + (c - K0)];
          else if (jk) w[i][j] = Cp[r * SB + (c - K0)];
          else if (ik) w[i][j] = Cp[c * SB + (r - K0)];
          else w[i][j] = a[r * LD + c] - u[i][j];
        }
      __syncthreads();   // every read of the old block is done
#pragma unroll
      for (int i = 0; i < S::MI; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) a[(ty + 16 * i) * LD + tx + S::TX * j] = w[i][j];
    }
    __syncthreads();
  }
  for (int e = tid; e < G * G; e += S::THREADS) {
    const int i = e >> S::SHIFT, j = e & (G - 1);
    Pout[e] = -a[i * LD + j];
  }
  if (tid < 32) {
    double l = 0.0;
    for (int p = tid; p < G; p += 32) l += log((double)pv[p]);
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if (tid == 0) {
      *logdet += l;
      if (s_bad) *status = INLA_ERR_NOT_SPD;
    }
  }
}

// Scalar sweep of the lower triangle: G steps, each one FMA per lower entry;
// the fewest FP64 instructions, which matters when the fused sweep shares an
// SM whose FP64 pipe the update blocks saturate.
template <typename R, int G>
__device__ void sweep_tile_scalar(R *sm, R *Pout, double *logdet, int *status) {
  using S = Sweep<G>;
  R *a = sm;                       // [G][LD]
  R *colp = sm + G * S::LD;        // [G]  column p of the current state
  R *cinv = colp + G;              // [G]  column p divided by the pivot
  R *pivs = cinv + G;              // [G]  pivots
  __shared__ R s_inv;
  __shared__ int s_bad;
  __shared__ double s_log[2];
  const int tid = threadIdx.x;
  int ei[S::PER], ej[S::PER];
  int ne = 0;
  for (int e = tid; e < S::TRI; e += S::THREADS) {
    int i = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    while (i * (i + 1) / 2 > e) --i;
    ei[ne] = i;
    ej[ne] = e - i * (i + 1) / 2;
    ++ne;
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int p = 0; p < G; ++p) {
    if (tid == 0) {
      const R piv = a[p * S::LD + p];
      const bool ok = (piv > R(0)) && (piv < R(INFINITY));
      pivs[p] = ok ? piv : R(1);
      s_inv = ok ? R(1) / piv : R(0);
      if (!ok) s_bad = 1;
    }
    __syncthreads();
    if (tid < G) {
      const R c = (tid >= p) ? a[tid * S::LD + p] : a[p * S::LD + tid];
      colp[tid] = c;
      cinv[tid] = c * s_inv;
    }
    __syncthreads();
    // every operand of this thread's entries is read before any entry is written (the
    // arrays share one buffer, so reads interleaved with writes would run one entry at
    // a time); the step's critical path is this phase's latency, not its FMAs
    R nv[S::PER];
    const R inv = s_inv;
#pragma unroll
    for (int k = 0; k < S::PER; ++k) {
      if (k < ne) {
        const int i = ei[k], j = ej[k];
        const R ci = cinv[i], cj = cinv[j], pj = colp[j], old = a[i * S::LD + j];
        nv[k] = (i == p) ? ((j == p) ? -inv : cj) : ((j == p) ? ci : fma(-ci, pj, old));
      }
    }
#pragma unroll
    for (int k = 0; k < S::PER; ++k)
      if (k < ne) a[ei[k] * S::LD + ej[k]] = nv[k];
    __syncthreads();
  }
  for (int e = tid; e < G * G; e += S::THREADS) {
    const int i = e >> S::SHIFT, j = e & (G - 1);
    Pout[e] = -((j <= i) ? a[i * S::LD + j] : a[j * S::LD + i]);
  }
  if (tid < G) {
    double l = log((double)pivs[tid]);
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((tid & 31) == 0) s_log[tid >> 5] = l;
  }
  __syncthreads();
  if (tid == 0) {
    *logdet += s_log[0] + (G > 32 ? s_log[1] : 0.0);
    if (s_bad) *status = INLA_ERR_NOT_SPD;
  }
}

// FP64: the element-by-element sweep (one FMA per lower entry per step, the
// fewest FP64 instructions: the two-level form does ~3x as many FP64 FMAs and
// measured slower on the 128 x 128 base blocks); FP32: the two-level sweep
// (12 block barriers instead of 192).
template <typename R, int G>
__device__ void sweep_tile(R *sm, R *Pout, double *logdet, int *status) {
  if (sizeof(R) == 4) sweep_tile_blocked<R, G>(sm, Pout, logdet, status);
  else sweep_tile_scalar<R, G>(sm, Pout, logdet, status);
}

// Pivot block 0 of an inversion (later pivots are inverted by the update
// kernel of the previous step).  Pbuf holds two G x G slots per point.
template <typename R, int G>
__global__ void __launch_bounds__(Sweep<G>::THREADS) gj_pivot_kernel(R *A, int64_t sA, int n_p, int K, R *Pbuf,
                                                                    double *logdet, int ld_stride, int *status,
                                                                    const int *active) {
  using S = Sweep<G>;
  const int b = blockIdx.x;
  if (active && !active[b]) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  R *sm = reinterpret_cast<R *>(smraw);
  const R *src = A + b * sA + (int64_t)(K * G) * n_p + K * G;
  for (int e = threadIdx.x; e < G * G; e += S::THREADS) {
    const int i = e >> S::SHIFT, j = e & (G - 1);
    if (j <= i) sm[i * S::LD + j] = src[(int64_t)i * n_p + j];
  }
  __syncthreads();
  sweep_tile<R, G>(sm, Pbuf + ((int64_t)b * 2 + (K & 1)) * G * G, logdet + (int64_t)b * ld_stride, status + b);
}

// C_I = A_IK P for every row tile I != K; the old A_IK is kept in Obuf.
template <typename R, int G>
__global__ void __launch_bounds__(Sweep<G>::THREADS) gj_panel_kernel(const R *A, int64_t sA, int n_p, int K,
                                                                    const R *Pbuf, R *Cbuf, R *Obuf,
                                                                    int64_t sCO, const int *active) {
  using S = Sweep<G>;
  const int I = blockIdx.x, b = blockIdx.y;
  if (I == K || (active && !active[b])) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  R *Os = reinterpret_cast<R *>(smraw);   // [G][LD]  O[r][k]
  R *Ps = Os + G * S::LD;                 // [G][LD]  P[k][c]
  const R *Ab = A + b * sA;
  if (I > K) {
    const R *src = Ab + (int64_t)(I * G) * n_p + K * G;
    for (int e = threadIdx.x; e < G * G; e += S::THREADS) {
      const int r = e >> S::SHIFT, c = e & (G - 1);
      Os[r * S::LD + c] = src[(int64_t)r * n_p + c];
    }
  } else {  // upper tile (I, K) = transpose of the stored lower tile (K, I)
    const R *src = Ab + (int64_t)(K * G) * n_p + I * G;
    for (int e = threadIdx.x; e < G * G; e += S::THREADS) {
      const int c = e >> S::SHIFT, r = e & (G - 1);
      Os[r * S::LD + c] = src[(int64_t)c * n_p + r];
    }
  }
  const R *Pb = Pbuf + ((int64_t)b * 2 + (K & 1)) * G * G;
  for (int e = threadIdx.x; e < G * G; e += S::THREADS) Ps[(e >> S::SHIFT) * S::LD + (e & (G - 1))] = Pb[e];
  __syncthreads();
  const int tx = threadIdx.x % S::TX, ty = threadIdx.x / S::TX;   // rows ty + 16 i, cols tx + TX j
  R acc[S::MI][4] = {};
#pragma unroll 8
  for (int k = 0; k < G; ++k) {
    R av[S::MI], bv[4];
#pragma unroll
    for (int i = 0; i < S::MI; ++i) av[i] = Os[(ty + 16 * i) * S::LD + k];
#pragma unroll
    for (int j = 0; j < 4; ++j) bv[j] = Ps[k * S::LD + tx + S::TX * j];
#pragma unroll
    for (int i = 0; i < S::MI; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
  }
  R *Cb = Cbuf + b * sCO + (int64_t)(I * G) * G;
  R *Ob = Obuf + b * sCO + (int64_t)(I * G) * G;
#pragma unroll
  for (int i = 0; i < S::MI; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) Cb[(ty + 16 * i) * G + tx + S::TX * j] = acc[i][j];
  for (int e = threadIdx.x; e < G * G; e += S::THREADS) Ob[e] = Os[(e >> S::SHIFT) * S::LD + (e & (G - 1))];
}

// Rank-G update of one lower tile (I, J): A_IJ -= C_I O_J^T for I, J != K; the
// pivot row/column become C (resp. C^T) and the pivot block -P.  next_pivot: the
// tile is (K+1, K+1), which is then inverted as the next pivot (slot (K+1)&1 of
// Pbuf).  Cs / Os: the block's shared workspace.  Called by all threads of a block.
template <typename R, int G>
__device__ void update_tile(R *A, int64_t sA, int n_p, int K, int I, int J, bool next_pivot, R *Pbuf,
                            const R *Cbuf, const R *Obuf, int64_t sCO, double *logdet, int ld_stride, int *status,
                            int b, R *Cs, R *Os) {
  using S = Sweep<G>;
  R *dst = A + b * sA + (int64_t)(I * G) * n_p + J * G;
  const R *Cb = Cbuf + b * sCO;
  if (I == K && J == K) {
    const R *Pb = Pbuf + ((int64_t)b * 2 + (K & 1)) * G * G;
    for (int e = threadIdx.x; e < G * G; e += S::THREADS)
      dst[(int64_t)(e >> S::SHIFT) * n_p + (e & (G - 1))] = -Pb[e];
    return;
  }
  if (J == K) {  // tile (I, K), I > K
    const R *src = Cb + (int64_t)(I * G) * G;
    for (int e = threadIdx.x; e < G * G; e += S::THREADS)
      dst[(int64_t)(e >> S::SHIFT) * n_p + (e & (G - 1))] = src[e];
    return;
  }
  if (I == K) {  // tile (K, J), J < K: transpose of C_J
    const R *src = Cb + (int64_t)(J * G) * G;
    for (int e = threadIdx.x; e < G * G; e += S::THREADS) {
      const int c = e >> S::SHIFT, r = e & (G - 1);
      dst[(int64_t)r * n_p + c] = src[c * G + r];
    }
    return;
  }
  R *sm = Cs;   // the fused pivot sweep's workspace
  const R *ci = Cb + (int64_t)(I * G) * G;
  const R *oj = Obuf + b * sCO + (int64_t)(J * G) * G;
  for (int e = threadIdx.x; e < G * G; e += S::THREADS) {
    Cs[(e >> S::SHIFT) * S::LD + (e & (G - 1))] = ci[e];
    Os[(e >> S::SHIFT) * S::LD + (e & (G - 1))] = oj[e];
  }
  const int tx = threadIdx.x % S::TX, ty = threadIdx.x / S::TX;
  // FP64: the accumulator starts at A_IJ and each step subtracts with one FMA.
  // FP32: the rank-G product is summed from zero and added to A_IJ once, so
  // the tile takes one rounding per block step instead of G (a sequential
  // FP32 accumulation loses about ten times more accuracy in log|D| and in
  // the selected inverse at n_s ~ 1000).
  constexpr bool kSumFirst = std::is_same<R, float>::value;
  R acc[S::MI][4];
#pragma unroll
  for (int i = 0; i < S::MI; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = kSumFirst ? R(0) : dst[(int64_t)(ty + 16 * i) * n_p + tx + S::TX * j];
  __syncthreads();
#pragma unroll 8
  for (int k = 0; k < G; ++k) {
    R av[S::MI], bv[4];
#pragma unroll
    for (int i = 0; i < S::MI; ++i) av[i] = -Cs[(ty + 16 * i) * S::LD + k];
#pragma unroll
    for (int j = 0; j < 4; ++j) bv[j] = Os[(tx + S::TX * j) * S::LD + k];
#pragma unroll
    for (int i = 0; i < S::MI; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
  }
  __syncthreads();   // every read of Cs / Os is done (they are rewritten next)
#pragma unroll
  for (int i = 0; i < S::MI; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = ty + 16 * i, c = tx + S::TX * j;
      if (kSumFirst) acc[i][j] += dst[(int64_t)r * n_p + c];
      dst[(int64_t)r * n_p + c] = acc[i][j];
      if (next_pivot && c <= r) sm[r * S::LD + c] = acc[i][j];
    }
  if (next_pivot) {
    __syncthreads();
    sweep_tile<R, G>(sm, Pbuf + ((int64_t)b * 2 + ((K + 1) & 1)) * G * G, logdet + (int64_t)b * ld_stride,
                     status + b);
  }
}

// Rank-G update of every lower tile of the block sweep at pivot K.  Grid (points,
// blocks per point), points fastest.  With lookahead (K + 1 < nt) block 0 of each
// point takes only tile (K+1, K+1) and, once updated, inverts it as the next pivot,
// so no separate pivot launch sits on the critical path; the other blocks take the
// remaining tiles in turn.  The launch sizes the blocks per point so that the whole
// grid is about one block per SM: the lookahead block, whose serial pivot sweep sets
// the launch length, then shares its SM's FP64 pipe with as few update blocks as
// possible (one tile per block packed 2-3 blocks on each SM, and the lookahead
// blocks ran at a fraction of the pipe).
template <typename R, int G>
__global__ void __launch_bounds__(Sweep<G>::THREADS) gj_update_kernel(R *A, int64_t sA, int n_p, int K, int nt,
                                                                     R *Pbuf, const R *Cbuf, const R *Obuf,
                                                                     int64_t sCO, double *logdet, int ld_stride,
                                                                     int *status, const int *active) {
  using S = Sweep<G>;
  const int b = blockIdx.x;
  if (active && !active[b]) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  R *Cs = reinterpret_cast<R *>(smraw);   // [G][LD]  C_I[r][k]
  R *Os = Cs + G * S::LD;                 // [G][LD]  O_J[c][k]
  const bool look = K + 1 < nt;
  const int ntri = nt * (nt + 1) / 2;
  const int nxt = (K + 1) * (K + 2) / 2 + (K + 1);   // linear index of tile (K+1, K+1)
  int I, J;
  if (look && blockIdx.y == 0) {
    tri_index(nxt, I, J);
    update_tile<R, G>(A, sA, n_p, K, I, J, true, Pbuf, Cbuf, Obuf, sCO, logdet, ld_stride, status, b, Cs, Os);
    return;
  }
  const int nrem = look ? ntri - 1 : ntri;
  const int workers = look ? (int)gridDim.y - 1 : (int)gridDim.y;
  for (int r = look ? (int)blockIdx.y - 1 : (int)blockIdx.y; r < nrem; r += workers) {
    tri_index((look && r >= nxt) ? r + 1 : r, I, J);
    update_tile<R, G>(A, sA, n_p, K, I, J, false, Pbuf, Cbuf, Obuf, sCO, logdet, ld_stride, status, b, Cs, Os);
    __syncthreads();   // the next tile rewrites Cs / Os
  }
}

// Pivot panel C_I = A_IK P for every row tile I != K, split in four G/4-row
// quarters per tile so that a launch has 4 (nt - 1) blocks per point instead
// of nt - 1 (one tile per block left most SMs idle).  4G threads; thread t
// computes row (G/4) q + t / 16 and G/16 consecutive columns from 16 (t % 16).
template <typename R, int G>
__global__ void __launch_bounds__(4 * G) gj_panel_q_kernel(const R *A, int64_t sA, int n_p, int K, const R *Pbuf,
                                                          R *Cbuf, R *Obuf, int64_t sCO, const int *active) {
  constexpr int QR = G / 4, OPT = G / 16, THREADS = 4 * G;
  const int I = blockIdx.x >> 2, q = blockIdx.x & 3, b = blockIdx.y;
  if (I == K || (active && !active[b])) return;
  __shared__ __align__(16) R As[QR][G];   // rows QR q .. QR q + QR - 1 of A_IK
  __shared__ __align__(16) R Ps[G][G];    // P (symmetric)
  const R *Ab = A + b * sA;
  const int tid = threadIdx.x;
  if (I > K) {
    const R *src = Ab + (int64_t)(I * G + QR * q) * n_p + K * G;
    for (int e = tid; e < QR * G; e += THREADS) As[e / G][e % G] = src[(int64_t)(e / G) * n_p + (e % G)];
  } else {  // upper tile (I, K) = transpose of the stored lower tile (K, I)
    const R *src = Ab + (int64_t)(K * G) * n_p + I * G + QR * q;
    for (int e = tid; e < QR * G; e += THREADS) {
      const int c = e / QR, r = e % QR;
      As[r][c] = src[(int64_t)c * n_p + r];
    }
  }
  const R *Pb = Pbuf + ((int64_t)b * 2 + (K & 1)) * G * G;
  constexpr int P16 = G * G * (int)sizeof(R) / 16;   // P in 16-byte chunks (slots are 16-byte aligned)
  for (int e = tid; e < P16; e += THREADS)
    reinterpret_cast<uint4 *>(&Ps[0][0])[e] = reinterpret_cast<const uint4 *>(Pb)[e];
  __syncthreads();
  const int r = tid / 16, c0 = (tid % 16) * OPT;
  R acc[OPT];
#pragma unroll
  for (int o = 0; o < OPT; ++o) acc[o] = R(0);
#pragma unroll 8
  for (int k = 0; k < G; ++k) {
    const R a = As[r][k];
    R pk[OPT];
    if constexpr (OPT * sizeof(R) == 16) {   // one 16-byte shared-memory read (the configurations in use)
      const uint4 u = *reinterpret_cast<const uint4 *>(&Ps[k][c0]);
      memcpy(pk, &u, 16);
    } else {
#pragma unroll
      for (int o = 0; o < OPT; ++o) pk[o] = Ps[k][c0 + o];
    }
#pragma unroll
    for (int o = 0; o < OPT; ++o) acc[o] = fma(a, pk[o], acc[o]);
  }
  const int64_t off = (int64_t)(I * G + QR * q + r) * G + c0;
#pragma unroll
  for (int o = 0; o < OPT; ++o) {
    Cbuf[b * sCO + off + o] = acc[o];
    Obuf[b * sCO + off + o] = As[r][c0 + o];
  }
}

// FP32 rank-64 update (G = 64): the same tiles and lookahead as
// gj_update_kernel, with the three 16 KB tiles (C_I, O_J and the old A_IJ)
// staged by asynchronous 16-byte copies issued together, so that their
// latencies overlap, and the product read from shared memory four k at a time
// (rows padded to 68 floats: 16-byte aligned, conflict-free along a quarter
// warp).  The rank-64 product is summed from zero and subtracted from A_IJ once.
constexpr int U32_LD = 68;
constexpr int U32_SMEM = (2 * 64 * U32_LD + 64 * 64) * 4;   // C_I, O_J, old A_IJ

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}

// special_only: only the lookahead tile and the tiles of the pivot row and
// column (grid.y = [1 +] nt), while the tensor cores update the other tiles
// (sweep_update_tf32x3).
__global__ void __launch_bounds__(256, 3) gj_update_f32_kernel(float *A, int64_t sA, int n_p, int K, int nt,
                                                           float *Pbuf, const float *Cbuf, const float *Obuf,
                                                           int64_t sCO, double *logdet, int ld_stride, int *status,
                                                           const int *active, int special_only) {
  constexpr int G = 64;
  using S = Sweep<G>;
  const int b = blockIdx.x;   // points fastest: every point's lookahead tile is among the first blocks
  if (active && !active[b]) return;
  const bool look = K + 1 < nt;
  int I, J;
  if (special_only) {
    const int y = (int)blockIdx.y - (look ? 1 : 0);   // -1: lookahead; then (K, 0..K-1), (K, K), (K+1..nt-1, K)
    if (y < 0) { I = K + 1; J = K + 1; }
    else if (y < K) { I = K; J = y; }
    else if (y == K) { I = K; J = K; }
    else { I = y; J = K; }
  } else if (look) {
    const int nxt = (K + 1) * (K + 2) / 2 + (K + 1);   // linear index of tile (K+1, K+1)
    int x = blockIdx.y;
    if (x == 0) x = nxt;
    else if (x <= nxt) x = x - 1;
    tri_index(x, I, J);
  } else {
    tri_index(blockIdx.y, I, J);
  }
  float *dst = A + b * sA + (int64_t)(I * G) * n_p + J * G;
  const float *Cb = Cbuf + b * sCO;
  if (I == K && J == K) {
    const float *Pb = Pbuf + ((int64_t)b * 2 + (K & 1)) * G * G;
    for (int e = threadIdx.x; e < G * G; e += 256) dst[(int64_t)(e >> 6) * n_p + (e & 63)] = -Pb[e];
    return;
  }
  if (J == K) {  // tile (I, K), I > K
    const float *src = Cb + (int64_t)(I * G) * G;
    for (int e = threadIdx.x; e < G * G; e += 256) dst[(int64_t)(e >> 6) * n_p + (e & 63)] = src[e];
    return;
  }
  if (I == K) {  // tile (K, J), J < K: transpose of C_J
    const float *src = Cb + (int64_t)(J * G) * G;
    for (int e = threadIdx.x; e < G * G; e += 256) {
      const int c = e >> 6, r = e & 63;
      dst[(int64_t)r * n_p + c] = src[c * G + r];
    }
    return;
  }
  extern __shared__ __align__(16) float u32s[];
  float *Cs = u32s;                 // [64][68]  C_I[r][k]
  float *Os = Cs + G * U32_LD;      // [64][68]  O_J[c][k]
  float *Ds = Os + G * U32_LD;      // [64][64]  old A_IJ
  const float *ci = Cb + (int64_t)(I * G) * G;
  const float *oj = Obuf + b * sCO + (int64_t)(J * G) * G;
#pragma unroll
  for (int it = 0; it < 4; ++it) {   // 1024 16-byte chunks per tile, 4 per thread
    const int q = threadIdx.x + 256 * it, r = q >> 4, c4 = (q & 15) * 4;
    cp_async16(Cs + r * U32_LD + c4, ci + r * G + c4);
    cp_async16(Os + r * U32_LD + c4, oj + r * G + c4);
    cp_async16(Ds + r * G + c4, dst + (int64_t)r * n_p + c4);
  }
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // rows ty + 16 i, columns tx + 16 j
  float acc[4][4] = {};
#pragma unroll 4
  for (int k = 0; k < G; k += 4) {
    float4 a[4], o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = *reinterpret_cast<const float4 *>(Cs + (ty + 16 * i) * U32_LD + k);
#pragma unroll
    for (int j = 0; j < 4; ++j) o[j] = *reinterpret_cast<const float4 *>(Os + (tx + 16 * j) * U32_LD + k);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[i][j] = fmaf(a[i].x, o[j].x, acc[i][j]);
        acc[i][j] = fmaf(a[i].y, o[j].y, acc[i][j]);
        acc[i][j] = fmaf(a[i].z, o[j].z, acc[i][j]);
        acc[i][j] = fmaf(a[i].w, o[j].w, acc[i][j]);
      }
  }
  const bool next_pivot = look && I == K + 1 && J == K + 1;
  float out[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[i][j] = Ds[(ty + 16 * i) * G + tx + 16 * j] - acc[i][j];
  if (next_pivot) __syncthreads();   // the staged tiles are reused as the sweep's workspace
  float *sm = u32s;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;
      dst[(int64_t)r * n_p + c] = out[i][j];
      if (next_pivot && c <= r) sm[r * S::LD + c] = out[i][j];
    }
  if (next_pivot) {
    __syncthreads();
    sweep_tile<float, G>(sm, Pbuf + ((int64_t)b * 2 + ((K + 1) & 1)) * G * G, logdet + (int64_t)b * ld_stride,
                         status + b);
  }
}

// A <- -A on the lower triangle, mirrored into the upper triangle.
template <typename R>
__global__ void gj_finalize_kernel(R *A, int64_t sA, int n_p, const int *active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  int I, J;
  tri_index(blockIdx.x, I, J);
  R *Ab = A + b * sA;
  for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
    int r = e >> 6, c = e & 63;
    if (I == J && c > r) continue;
    int64_t gi = I * T + r, gj = J * T + c;
    R v = -Ab[gi * n_p + gj];
    Ab[gi * n_p + gj] = v;
    Ab[gj * n_p + gi] = v;
  }
}

template <typename R>
__global__ void mirror_kernel(R *A, int64_t sA, int n_p, const int *active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  int I, J;
  tri_index(blockIdx.x, I, J);
  R *Ab = A + b * sA;
  for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
    int r = e >> 6, c = e & 63;
    if (I == J && c >= r) continue;
    int64_t gi = I * T + r, gj = J * T + c;
    Ab[gj * n_p + gi] = Ab[gi * n_p + gj];
  }
}

// C = alpha A B + beta C0 (row-major n x n), one 64 x 64 tile of C per block.
template <typename R>
__global__ void __launch_bounds__(256) gemm_nn_kernel(int n, const R *A, int64_t sA, const R *B,
                                                     int64_t sB, R *C, int64_t sC, R alpha,
                                                     const R *C0, int64_t sC0, R beta, int lower_only,
                                                     const int *active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int nt = n / T;
  int I, J;
  if (lower_only) tri_index(blockIdx.x, I, J);
  else { I = blockIdx.x / nt; J = blockIdx.x % nt; }
  extern __shared__ __align__(16) unsigned char smraw[];
  R *As = reinterpret_cast<R *>(smraw);   // [64][65]  A[r][k]
  R *Bs = As + T * LDS;                   // [64][65]  B[k][c]
  const R *Ab = A + b * sA + (int64_t)(I * T) * n;
  const R *Bb = B + b * sB + J * T;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  R acc[4][4] = {};
  for (int kk = 0; kk < nt; ++kk) {
    for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
      int r = e >> 6, c = e & 63;
      As[r * LDS + c] = Ab[(int64_t)r * n + kk * T + c];
      Bs[r * LDS + c] = Bb[(int64_t)(kk * T + r) * n + c];
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < T; ++k) {
      R av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[(ty + 16 * i) * LDS + k];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[k * LDS + tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  R *Cb = C + b * sC + (int64_t)(I * T) * n + J * T;
  const R *C0b = C0 ? C0 + b * sC0 + (int64_t)(I * T) * n + J * T : nullptr;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t off = (int64_t)(ty + 16 * i) * n + tx + 16 * j;
      R v = alpha * acc[i][j];
      if (C0b) v += beta * C0b[off];
      Cb[off] = v;
    }
}

// FP32 C = alpha A B + beta C0 with 128 x 128 tiles of C (n a multiple of 128):
// 256 threads, each owning an 8 x 8 block of outputs (rows ty*4+{0..3} and
// 64+ty*4+{0..3}, likewise for columns), operands staged through shared memory
// in 16-deep k slabs read as float4; the next slab is prefetched into
// registers while the current one is multiplied.
constexpr int G128 = 128, KC = 16, APAD = 4;
__global__ void __launch_bounds__(256, 2) gemm128_f32_kernel(int n, const float *A, int64_t sA, const float *B,
                                                         int64_t sB, float *C, int64_t sC, float alpha,
                                                         const float *C0, int64_t sC0, float beta, int lower_only,
                                                         const int *active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int nt = n / G128;
  int I, J;
  if (lower_only) tri_index(blockIdx.x, I, J);
  else { I = blockIdx.x / nt; J = blockIdx.x % nt; }
  __shared__ __align__(16) float As[KC][G128 + APAD];   // A transposed: As[k][row]
  __shared__ __align__(16) float Bs[KC][G128];          // Bs[k][col]
  const float *Ab = A + b * sA + (int64_t)(I * G128) * n;
  const float *Bb = B + b * sB + J * G128;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  float4 ra[2], rb[2];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int r = (tid >> 2) + 64 * q, c4 = tid & 3;
      ra[q] = *reinterpret_cast<const float4 *>(Ab + (int64_t)r * n + k0 + c4 * 4);
      const int kk = (tid >> 5) + 8 * q, cc = tid & 31;
      rb[q] = *reinterpret_cast<const float4 *>(Bb + (int64_t)(k0 + kk) * n + cc * 4);
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int r = (tid >> 2) + 64 * q, c4 = tid & 3;
      As[c4 * 4 + 0][r] = ra[q].x;
      As[c4 * 4 + 1][r] = ra[q].y;
      As[c4 * 4 + 2][r] = ra[q].z;
      As[c4 * 4 + 3][r] = ra[q].w;
      const int kk = (tid >> 5) + 8 * q, cc = tid & 31;
      *reinterpret_cast<float4 *>(&Bs[kk][cc * 4]) = rb[q];
    }
  };
  load(0);
  for (int k0 = 0; k0 < n; k0 += KC) {
    __syncthreads();
    store();
    __syncthreads();
    if (k0 + KC < n) load(k0 + KC);
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      const float4 a0 = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&As[k][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[k][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
  }
  float *Cb = C + b * sC + (int64_t)(I * G128) * n + J * G128;
  const float *C0b = C0 ? C0 + b * sC0 + (int64_t)(I * G128) * n + J * G128 : nullptr;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = h * 64 + tx * 4;
      float4 v = make_float4(alpha * acc[i][4 * h + 0], alpha * acc[i][4 * h + 1], alpha * acc[i][4 * h + 2],
                             alpha * acc[i][4 * h + 3]);
      if (C0b) {
        const float4 z = *reinterpret_cast<const float4 *>(C0b + (int64_t)r * n + c);
        v.x += beta * z.x;
        v.y += beta * z.y;
        v.z += beta * z.z;
        v.w += beta * z.w;
      }
      *reinterpret_cast<float4 *>(Cb + (int64_t)r * n + c) = v;
    }
  }
}

template <typename R>
constexpr size_t smem_gemm() { return 2 * T * LDS * sizeof(R); }
template <typename R, int G>
constexpr size_t smem_update() {
  return (2 * G * Sweep<G>::LD > Sweep<G>::SMEM_ELEMS ? 2 * G * Sweep<G>::LD : Sweep<G>::SMEM_ELEMS) * sizeof(R);
}
template <typename R, int G>
constexpr size_t smem_pivot() { return Sweep<G>::SMEM_ELEMS * sizeof(R); }

// Kernel attributes belong to the device's context: they are set once for
// every device the process uses (the first call with that device current).
template <typename R>
void ensure_attrs() {
  static std::mutex mu;
  static bool done[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  cudaFuncSetAttribute(gemm_nn_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_gemm<R>());
  // 64-wide FP64 tiles need more than the default 48 KB of dynamic shared memory
  cudaFuncSetAttribute(gj_update_kernel<R, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem_update<R, 64>());
  cudaFuncSetAttribute(gj_panel_kernel<R, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(2 * 64 * Sweep<64>::LD * sizeof(R)));
  cudaFuncSetAttribute(gj_pivot_kernel<R, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_pivot<R, 64>());
  if (sizeof(R) == 4)
    cudaFuncSetAttribute(gj_update_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, U32_SMEM);
  prefer_shared(gemm_nn_kernel<R>);
  prefer_shared(gj_pivot_kernel<R, 32>);
  prefer_shared(gj_pivot_kernel<R, 64>);
  prefer_shared(gj_panel_kernel<R, 32>);
  prefer_shared(gj_panel_kernel<R, 64>);
  prefer_shared(gj_panel_q_kernel<R, 32>);
  prefer_shared(gj_panel_q_kernel<R, 64>);
  prefer_shared(gj_update_kernel<R, 32>);
  prefer_shared(gj_update_kernel<R, 64>);
  prefer_shared(gj_finalize_kernel<R>);
  prefer_shared(mirror_kernel<R>);
  prefer_shared(transpose_kernel<R>);
  if (sizeof(R) == 4) {
    prefer_shared(gj_update_f32_kernel);
    prefer_shared(gemm128_f32_kernel);
  }
  done[dev] = true;
}

// Blocks per point of gj_update_kernel: about one block per SM over the grid, at
// most MAX_TILES_PER_BLOCK tiles per update block (fine enough to balance large
// batches), and the lookahead block on its own.
constexpr int MAX_TILES_PER_BLOCK = 4;
int update_blocks(int P, int ntri, bool look) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int tiles = look ? ntri - 1 : ntri;
  int per = std::max((sms + P - 1) / P - (look ? 1 : 0), (tiles + MAX_TILES_PER_BLOCK - 1) / MAX_TILES_PER_BLOCK);
  per = std::max(1, std::min(per, tiles));
  return per + (look ? 1 : 0);
}

// Block sweep inversion with G x G pivots (see the kernels above) of the
// nsub x nsub block at A (leading dimension ld; the kernels' n_p argument is
// the leading dimension).
template <typename R, int G>
void gj_invert_g(Launch &L, const DevModel &M, const Work &W, R *A, int64_t strideA, int ld, int nsub,
                 double *logdet_out, int logdet_slot_stride) {
  using S = Sweep<G>;
  const int n_p = ld, nt = nsub / G, P = W.P;
  const int ntri = nt * (nt + 1) / 2;
  const int64_t sCO = (int64_t)M.n_p * G;
  const int tnt = nsub / T, tntri = tnt * (tnt + 1) / 2;
  R *Pb = reinterpret_cast<R *>(W.gjP);
  R *Cb = reinterpret_cast<R *>(W.gjC);
  R *Ob = reinterpret_cast<R *>(W.gjO);
  const double unit = (double)G * G * G / (64.0 * 64.0 * 64.0);   // one tile product in 64^3 units
  const bool tensor_update =
      sizeof(R) == 4 && G == 64 && M.sweep_g32 == INLA_SWEEP_TF32X3 && n_p % 128 == 0 && nsub == ld;
  for (int K = 0; K < nt; ++K) {
    if (K == 0) {
      L.start(KID_GJ_PIVOT, (double)P);
      gj_pivot_kernel<R, G><<<P, S::THREADS, smem_pivot<R, G>(), L.st>>>(A, strideA, n_p, K, Pb, logdet_out,
                                                                          logdet_slot_stride, W.status, W.active);
      L.stop();
      L.tick();
    }
    if (nt > 1) {
      L.start(KID_GJ_PANEL, (double)P * (nt - 1) * unit);
      if (sizeof(R) == 8 && G == 64)   // 2 x 32 KB of static shared memory would exceed the limit
        gj_panel_kernel<R, G><<<dim3(nt, P), S::THREADS, 2 * G * S::LD * sizeof(R), L.st>>>(
            A, strideA, n_p, K, Pb, Cb, Ob, sCO, W.active);
      else
        gj_panel_q_kernel<R, G><<<dim3(4 * nt, P), 4 * G, 0, L.st>>>(A, strideA, n_p, K, Pb, Cb, Ob, sCO,
                                                                     W.active);
      L.stop();
      L.tick();
    }
    if (sizeof(R) == 4 && G == 64 && tensor_update) {
      // the lookahead tile (with the next pivot inversion) and the pivot row and column on the
      // CUDA cores, then every other lower tile on the tensor cores
      const int look = K + 1 < nt ? 1 : 0;
      L.start(KID_GJ_PIVOT, (double)P);
      gj_update_f32_kernel<<<dim3(P, look + nt), 256, U32_SMEM, L.st>>>(
          reinterpret_cast<float *>(A), strideA, n_p, K, nt, reinterpret_cast<float *>(Pb),
          reinterpret_cast<const float *>(Cb), reinterpret_cast<const float *>(Ob), sCO, logdet_out,
          logdet_slot_stride, W.status, W.active, 1);
      L.stop();
      L.tick();
      sweep_update_tf32x3(L, P, n_p, reinterpret_cast<float *>(A), strideA, reinterpret_cast<const float *>(Cb),
                          reinterpret_cast<const float *>(Ob), sCO, K, look ? K + 1 : -1, W.active, W.status);
      continue;
    }
    L.start(sizeof(R) == 4 ? KID_GJ_UPDATE32 : KID_GJ_UPDATE, (double)P * (ntri - nt) * unit);
    if (sizeof(R) == 4 && G == 64)
      gj_update_f32_kernel<<<dim3(P, ntri), 256, U32_SMEM, L.st>>>(
          reinterpret_cast<float *>(A), strideA, n_p, K, nt, reinterpret_cast<float *>(Pb),
          reinterpret_cast<const float *>(Cb), reinterpret_cast<const float *>(Ob), sCO, logdet_out,
          logdet_slot_stride, W.status, W.active, 0);
    else
      gj_update_kernel<R, G><<<dim3(P, update_blocks(P, ntri, K + 1 < nt)), S::THREADS, smem_update<R, G>(),
                               L.st>>>(A, strideA, n_p, K, nt, Pb, Cb, Ob, sCO, logdet_out, logdet_slot_stride,
                                       W.status, W.active);
    L.stop();
    L.tick();
  }
  gj_finalize_kernel<R><<<dim3(tntri, P), 256, 0, L.st>>>(A, strideA, n_p, W.active);
  L.tick();
}

}  // namespace

void dense_prepare() {
  ensure_attrs<double>();
  ensure_attrs<float>();
  tc_prepare();
  ozaki_prepare();
  bta_prepare();
}

// Tile width per precision from the model (defaults: 32 for FP64, where short
// pivot sweeps matter on the slow FP64 pipe; 64 for FP32, which gives each
// block 4x the work); inla_autotune may change them.
template <typename R>
void gj_invert_sub(Launch &L, const DevModel &M, const Work &W, R *A, int64_t strideA, int ld, int nsub,
                   double *logdet_out, int logdet_slot_stride) {
  ensure_attrs<R>();
  const int g = sizeof(R) == 4 ? M.sweep_g32 : M.sweep_g64;
  if (g == 64 || g == INLA_SWEEP_TF32X3 || g == INLA_INV_BLOCKED)
    gj_invert_g<R, 64>(L, M, W, A, strideA, ld, nsub, logdet_out, logdet_slot_stride);
  else
    gj_invert_g<R, 32>(L, M, W, A, strideA, ld, nsub, logdet_out, logdet_slot_stride);
}

// ---------------------------------------------------------------- blocked inversion on the tensor cores
//
// D^-1 and log|D| by 2 x 2 block recursion on multiples of 128, with
//   D = [A11 A21^T; A21 A22],  Wt = A21 A11^-1,  S = A22 - Wt A21^T,
//   D^-1 = [A11^-1 + Wt^T S^-1 Wt,  -(S^-1 Wt)^T;  -S^-1 Wt,  S^-1],
//   log|D| = log|A11| + log|S|
// (the block LDL^T of Sec. 2.4 applied inside one block).  Every product is an
// X Y^T of row-major operands on the tensor cores: FP64 blocks through BF16
// digit slices (ozaki.cu), FP32 blocks through the 3xTF32 split product
// (tc_gemm.cu).  Diagonal blocks of up to 256 rows are inverted by the block sweep
// (their pivots give the log-determinant and the positive-definiteness test).
// The four products per level cost (n/2)^3 (1 + 1/2 + 1 + 1/2) multiply-adds,
// n^3 flops over the recursion, as the sweep.  Scratch: W.S, W.SigN, W.SigC
// (free during a factorisation) for Wt, its transpose and the transpose of the
// new A21; two operand buffers: digit slices W.Zd/Ed and W.Zs/Es (FP64), TF32
// hi / lo parts W.Dh/Dl and W.Sh/Sl (FP32).
// Diagonal blocks of at most this size are inverted by the sweep: the sweep's
// launches on 128 x 128 blocks are latency-bound, and 256 measured faster per step
// in both precisions (FP64 at n_s = 1024: 206 against 217 ms; FP32 at n_s = 2500:
// 2.58 against 2.72 s).
template <typename R>
constexpr int inv_base() { return 256; }

template <typename R>
__global__ void transpose_kernel(const R *__restrict__ src, int64_t lds, int64_t ss, R *__restrict__ dst,
                                 int64_t ldd, int64_t sd, int rows, int cols, const int *active) {
  const int b = blockIdx.z;
  if (active && !active[b]) return;
  __shared__ R t[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[i][threadIdx.x] = src[b * ss + (int64_t)r * lds + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[b * sd + (int64_t)c * ldd + r] = t[threadIdx.x][i];
  }
}

template <typename R>
void transpose(Launch &L, int P, int rows, int cols, const R *src, int64_t lds, int64_t ss, R *dst, int64_t ldd,
               int64_t sd, const int *active) {
  transpose_kernel<R><<<dim3((cols + 31) / 32, (rows + 31) / 32, P), dim3(32, 8), 0, L.st>>>(src, lds, ss, dst, ldd,
                                                                                            sd, rows, cols, active);
  L.tick();
}

template <typename R>
void mirror_sub(Launch &L, int P, int n, int ld, R *A, int64_t sA, const int *active);

// Operand buffer `which` (0 or 1) of a tensor-core product: the rows x K block at
// src (leading dimension ld, point stride ss) in the product's input format.
void split_operand(Launch &L, const Work &W, int which, int rows, int K, const double *src, int64_t ld, int64_t ss) {
  ozaki_split(L, W.P, rows, K, src, ld, ss, which ? W.Zs : W.Zd, W.sZ, which ? W.Es : W.Ed, W.sE, W.active);
}
void split_operand(Launch &L, const Work &W, int which, int rows, int K, const float *src, int64_t ld, int64_t ss) {
  split_tf32_2d(L, W.P, rows, K, src, ld, ss, which ? W.Sh : W.Dh, which ? W.Sl : W.Dl, W.sMat, W.active);
}
// Both operand buffers at once: src0 into buffer 0, src1 into buffer 1.
void split_operands(Launch &L, const Work &W, int rows0, int K0, const double *src0, int64_t ld0, int64_t ss0,
                    int rows1, int K1, const double *src1, int64_t ld1, int64_t ss1) {
  ozaki_split2(L, W.P, rows0, K0, src0, ld0, ss0, W.Zd, W.Ed, rows1, K1, src1, ld1, ss1, W.Zs, W.Es, W.sZ, W.sE,
               W.active);
}
void split_operands(Launch &L, const Work &W, int rows0, int K0, const float *src0, int64_t ld0, int64_t ss0,
                    int rows1, int K1, const float *src1, int64_t ld1, int64_t ss1) {
  split_operand(L, W, 0, rows0, K0, src0, ld0, ss0);
  split_operand(L, W, 1, rows1, K1, src1, ld1, ss1);
}

// C = alpha X Y^T + beta C0 with X in operand buffer x and Y in buffer y.
void operand_gemm(Launch &L, const Work &W, int Mr, int Nr, int K, int x, int y, double *C, int64_t ldc, int64_t sC,
                  double alpha, const double *C0, int64_t ldc0, int64_t sC0, double beta, bool lower) {
  gemm_nt_ozaki(L, W.P, Mr, Nr, K, x ? W.Zs : W.Zd, W.sZ, x ? W.Es : W.Ed, W.sE, y ? W.Zs : W.Zd, W.sZ,
                y ? W.Es : W.Ed, W.sE, C, ldc, sC, alpha, C0, ldc0, sC0, beta, lower, W.active, W.status);
}
void operand_gemm(Launch &L, const Work &W, int Mr, int Nr, int K, int x, int y, float *C, int64_t ldc, int64_t sC,
                  float alpha, const float *C0, int64_t ldc0, int64_t sC0, float beta, bool lower) {
  gemm_nt_tf32x3_split(L, W.P, Mr, Nr, K, x ? W.Sh : W.Dh, x ? W.Sl : W.Dl, W.sMat, y ? W.Sh : W.Dh,
                       y ? W.Sl : W.Dl, W.sMat, C, ldc, sC, alpha, C0, ldc0, sC0, beta, nullptr, nullptr, lower,
                       W.active, W.status);
}

// woff: offset of this level's Wt in W.S.  Wt must survive the recursion on A22,
// which therefore places its own Wt after it (n^2 / 3 elements over all levels).
template <typename R>
void inv_rec(Launch &L, const DevModel &M, const Work &W, R *A, int64_t sA, int ld, int o, int n, double *logdet,
             int ldst, int64_t woff) {
  R *A11 = A + (int64_t)o * ld + o;
  if (n <= inv_base<R>()) {
    gj_invert_sub<R>(L, M, W, A11, sA, ld, n, logdet, ldst);
    return;
  }
  const int n1 = 128 * (n / 256), n2 = n - n1, P = W.P;
  R *A21 = A11 + (int64_t)n1 * ld, *A22 = A21 + n1;
  R *Wt = static_cast<R *>(W.S) + woff, *Wm = static_cast<R *>(W.SigN), *Vt = static_cast<R *>(W.SigC);
  const int64_t sM = W.sMat;
  inv_rec<R>(L, M, W, A, sA, ld, o, n1, logdet, ldst, woff);   // A11 <- A11^-1, full symmetric
  // Wt = A21 A11^-1 (n2 x n1)
  split_operands(L, W, n1, n1, A11, ld, sA, n2, n1, A21, ld, sA);
  operand_gemm(L, W, n2, n1, n1, 1, 0, Wt, n1, sM, R(1), nullptr, 0, 0, R(0), false);
  // A22 <- S = A22 - Wt A21^T (lower tiles; the sweep and the recursion read the lower triangle)
  split_operand(L, W, 0, n2, n1, Wt, n1, sM);
  operand_gemm(L, W, n2, n2, n1, 0, 1, A22, ld, sA, R(-1), A22, ld, sA, R(1), true);
  inv_rec<R>(L, M, W, A, sA, ld, o + n1, n2, logdet, ldst, woff + (int64_t)n1 * n2);   // A22 <- S^-1, full
  // A21 <- -S^-1 Wt = -(S^-1) (Wt^T)^T
  transpose<R>(L, P, n2, n1, Wt, n1, sM, Wm, n2, sM, W.active);   // Wm = Wt^T (n1 x n2)
  split_operands(L, W, n2, n2, A22, ld, sA, n1, n2, Wm, n2, sM);
  operand_gemm(L, W, n2, n1, n2, 0, 1, A21, ld, sA, R(-1), nullptr, 0, 0, R(0), false);
  // A11 <- A11^-1 + Wm S^-1 Wm^T = A11^-1 - A21^T Wm^T (A21 now -S^-1 Wt)
  transpose<R>(L, P, n2, n1, A21, ld, sA, Vt, n2, sM, W.active);   // Vt = A21^T (n1 x n2)
  split_operand(L, W, 0, n1, n2, Vt, n2, sM);
  operand_gemm(L, W, n1, n1, n2, 0, 1, A11, ld, sA, R(-1), A11, ld, sA, R(1), true);
  mirror_sub<R>(L, P, n, ld, A11, sA, W.active);   // upper triangle = lower (A12 = A21^T, A11 full)
}

// Whether D^-1 is formed by the blocked recursion with tensor-core products.
template <typename R>
bool blocked_inverse(const DevModel &M, const Work &W) {
  if (M.n_p % 128 || M.n_p <= inv_base<R>()) return false;
  if (sizeof(R) == 8) return M.f64_tensor && W.Zd;
  return M.sweep_g32 == INLA_INV_BLOCKED && W.Dh;
}

template <typename R>
void gj_invert(Launch &L, const DevModel &M, const Work &W, R *A, int64_t strideA, double *logdet_out,
               int logdet_slot_stride) {
  ensure_attrs<R>();
  if (blocked_inverse<R>(M, W)) {
    inv_rec<R>(L, M, W, A, strideA, M.n_p, 0, M.n_p, logdet_out, logdet_slot_stride, 0);
    return;
  }
  gj_invert_sub<R>(L, M, W, A, strideA, M.n_p, M.n_p, logdet_out, logdet_slot_stride);
}

template <typename R>
void gemm_nn(Launch &L, int P, int n, const R *A, int64_t sA, const R *B, int64_t sB, R *C, int64_t sC, R alpha,
             const R *C0, int64_t sC0, R beta, bool lower_only, const int *active, int tile) {
  ensure_attrs<R>();
  if (sizeof(R) == 4 && tile == 128 && n % G128 == 0) {
    const int nt = n / G128;
    const int tiles = lower_only ? nt * (nt + 1) / 2 : nt * nt;
    L.start(KID_GEMM, (double)P * tiles * nt * 8.0);   // 8 units of 64^3 per 128^3 tile product
    gemm128_f32_kernel<<<dim3(tiles, P), 256, 0, L.st>>>(
        n, reinterpret_cast<const float *>(A), sA, reinterpret_cast<const float *>(B), sB,
        reinterpret_cast<float *>(C), sC, (float)alpha, reinterpret_cast<const float *>(C0), sC0, (float)beta,
        lower_only ? 1 : 0, active);
    L.stop();
    L.tick();
    return;
  }
  const int nt = n / T;
  const int tiles = lower_only ? nt * (nt + 1) / 2 : nt * nt;
  // units: 64 x 64 x 64 tile products (2 * 64^3 flops each)
  L.start(KID_GEMM, (double)P * tiles * nt);
  gemm_nn_kernel<R><<<dim3(tiles, P), 256, smem_gemm<R>(), L.st>>>(n, A, sA, B, sB, C, sC, alpha, C0, sC0, beta,
                                                                    lower_only ? 1 : 0, active);
  L.stop();
  L.tick();
}

template <typename R>
void mirror_sub(Launch &L, int P, int n, int ld, R *A, int64_t sA, const int *active) {
  const int nt = n / T;
  mirror_kernel<R><<<dim3(nt * (nt + 1) / 2, P), 256, 0, L.st>>>(A, sA, ld, active);
  L.tick();
}

template <typename R>
void mirror_lower(Launch &L, int P, int n, R *A, int64_t sA, const int *active) {
  mirror_sub<R>(L, P, n, n, A, sA, active);
}

template void gj_invert<double>(Launch &, const DevModel &, const Work &, double *, int64_t, double *, int);
template void gj_invert<float>(Launch &, const DevModel &, const Work &, float *, int64_t, double *, int);
template void gemm_nn<double>(Launch &, int, int, const double *, int64_t, const double *, int64_t, double *, int64_t,
                              double, const double *, int64_t, double, bool, const int *, int);
template void gemm_nn<float>(Launch &, int, int, const float *, int64_t, const float *, int64_t, float *, int64_t,
                             float, const float *, int64_t, float, bool, const int *, int);
template void mirror_lower<double>(Launch &, int, int, double *, int64_t, const int *);
template void mirror_lower<float>(Launch &, int, int, float *, int64_t, const int *);

}  // namespace inla
