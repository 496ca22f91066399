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

#include "inla_internal.cuh"

namespace inla {

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
// Pivot blocks and update tiles are 32 x 32 (GT); a block of 128 threads
// owns one tile, so one update launch has P * nt(nt+1)/2 small blocks that
// balance well over 152 SMs (up to 16 resident blocks per SM).
constexpr int GT = 32;
constexpr int GLD = GT + 1;
constexpr int GTHREADS = 128;
constexpr int GTRI = GT * (GT + 1) / 2;                    // 528 lower entries
constexpr int GPER = (GTRI + GTHREADS - 1) / GTHREADS;     // entries per thread
constexpr int SWEEP_SMEM_DOUBLES = GT * GLD + 3 * GT;

// Scalar sweep of a 32 x 32 SPD block held (lower triangle) in shared memory:
// after 32 steps it holds -A^-1.  Writes P = A^-1 (full symmetric tile) to
// Pout and adds log|A| = sum_p log(pivot_p), accumulated in double, to
// *logdet; a non-positive pivot sets *status.  One FMA per lower entry and
// step; one reciprocal per step; the logarithms once at the end.  The sweep
// runs in the storage type R of the blocks.  Called by all GTHREADS threads.
template <typename R>
__device__ void sweep_tile(R *sm, R *Pout, double *logdet, int *status) {
  R *a = sm;                       // [32][33]
  R *colp = sm + GT * GLD;         // [32]  column p of the current state
  R *cinv = colp + GT;             // [32]  column p divided by the pivot
  R *pivs = cinv + GT;             // [32]  pivots
  __shared__ R s_inv;
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  int ei[GPER], ej[GPER];
  int ne = 0;
  for (int e = tid; e < GTRI; e += GTHREADS) {
    int i = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    while (i * (i + 1) / 2 > e) --i;
    ei[ne] = i;
    ej[ne] = e - i * (i + 1) / 2;
    ++ne;
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int p = 0; p < GT; ++p) {
    if (tid == 0) {
      const R piv = a[p * GLD + p];
      const bool ok = (piv > R(0)) && (piv < R(INFINITY));
      pivs[p] = ok ? piv : R(1);
      s_inv = ok ? R(1) / piv : R(0);
      if (!ok) s_bad = 1;
    }
    __syncthreads();
    if (tid < GT) {
      const R c = (tid >= p) ? a[tid * GLD + p] : a[p * GLD + tid];
      colp[tid] = c;
      cinv[tid] = c * s_inv;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GPER; ++k) {
      if (k >= ne) break;
      const int i = ei[k], j = ej[k];
      R *ap = &a[i * GLD + j];
      if (i == p) *ap = (j == p) ? -s_inv : cinv[j];
      else if (j == p) *ap = cinv[i];
      else *ap = fma(-cinv[i], colp[j], *ap);
    }
    __syncthreads();
  }
  for (int e = tid; e < GT * GT; e += GTHREADS) {
    const int i = e >> 5, j = e & 31;
    Pout[e] = -((j <= i) ? a[i * GLD + j] : a[j * GLD + i]);
  }
  if (tid < 32) {
    double l = log((double)pivs[tid]);
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if (tid == 0) {
      *logdet += l;
      if (s_bad) *status = INLA_ERR_NOT_SPD;
    }
  }
}

// Pivot block 0 of an inversion (later pivots are inverted by the update
// kernel of the previous step).  Pbuf holds two 32 x 32 slots per point.
template <typename R>
__global__ void __launch_bounds__(GTHREADS) gj_pivot_kernel(R *A, int64_t sA, int n_p, int K, R *Pbuf,
                                                           double *logdet, int ld_stride, int *status,
                                                           const int *active) {
  const int b = blockIdx.x;
  if (active && !active[b]) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  R *sm = reinterpret_cast<R *>(smraw);
  const R *src = A + b * sA + (int64_t)(K * GT) * n_p + K * GT;
  for (int e = threadIdx.x; e < GT * GT; e += GTHREADS) {
    const int i = e >> 5, j = e & 31;
    if (j <= i) sm[i * GLD + j] = src[(int64_t)i * n_p + j];
  }
  __syncthreads();
  sweep_tile(sm, Pbuf + ((int64_t)b * 2 + (K & 1)) * GT * GT, logdet + (int64_t)b * ld_stride, status + b);
}

// C_I = A_IK P for every row tile I != K; the old A_IK is kept in Obuf.
template <typename R>
__global__ void __launch_bounds__(GTHREADS) gj_panel_kernel(const R *A, int64_t sA, int n_p, int K,
                                                           const R *Pbuf, R *Cbuf, R *Obuf,
                                                           int64_t sCO, const int *active) {
  const int I = blockIdx.x, b = blockIdx.y;
  if (I == K || (active && !active[b])) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  R *Os = reinterpret_cast<R *>(smraw);   // [32][33]  O[r][k]
  R *Ps = Os + GT * GLD;                  // [32][33]  P[k][c]
  const R *Ab = A + b * sA;
  if (I > K) {
    const R *src = Ab + (int64_t)(I * GT) * n_p + K * GT;
    for (int e = threadIdx.x; e < GT * GT; e += GTHREADS) {
      const int r = e >> 5, c = e & 31;
      Os[r * GLD + c] = src[(int64_t)r * n_p + c];
    }
  } else {  // upper tile (I, K) = transpose of the stored lower tile (K, I)
    const R *src = Ab + (int64_t)(K * GT) * n_p + I * GT;
    for (int e = threadIdx.x; e < GT * GT; e += GTHREADS) {
      const int c = e >> 5, r = e & 31;
      Os[r * GLD + c] = src[(int64_t)c * n_p + r];
    }
  }
  const R *Pb = Pbuf + ((int64_t)b * 2 + (K & 1)) * GT * GT;
  for (int e = threadIdx.x; e < GT * GT; e += GTHREADS) Ps[(e >> 5) * GLD + (e & 31)] = Pb[e];
  __syncthreads();
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;   // rows ty + 16 i, cols tx + 8 j
  R acc[2][4] = {};
#pragma unroll 8
  for (int k = 0; k < GT; ++k) {
    R av[2], bv[4];
#pragma unroll
    for (int i = 0; i < 2; ++i) av[i] = Os[(ty + 16 * i) * GLD + k];
#pragma unroll
    for (int j = 0; j < 4; ++j) bv[j] = Ps[k * GLD + tx + 8 * j];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
  }
  R *Cb = Cbuf + b * sCO + (int64_t)(I * GT) * GT;
  R *Ob = Obuf + b * sCO + (int64_t)(I * GT) * GT;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) Cb[(ty + 16 * i) * GT + tx + 8 * j] = acc[i][j];
  for (int e = threadIdx.x; e < GT * GT; e += GTHREADS) Ob[e] = Os[(e >> 5) * GLD + (e & 31)];
}

// Rank-32 update of every lower tile (I, J): A_IJ -= C_I O_J^T for I, J != K;
// the pivot row/column become C (resp. C^T) and the pivot block -P.  With
// lookahead (K + 1 < nt) block 0 takes tile (K+1, K+1) and, once updated,
// inverts it as the next pivot (slot (K+1)&1 of Pbuf), so no separate pivot
// launch sits on the critical path.
template <typename R>
__global__ void __launch_bounds__(GTHREADS) gj_update_kernel(R *A, int64_t sA, int n_p, int K, int nt,
                                                            R *Pbuf, const R *Cbuf, const R *Obuf,
                                                            int64_t sCO, double *logdet, int ld_stride, int *status,
                                                            const int *active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const bool look = K + 1 < nt;
  int I, J;
  if (look) {
    const int nxt = (K + 1) * (K + 2) / 2 + (K + 1);   // linear index of tile (K+1, K+1)
    int x = blockIdx.x;
    if (x == 0) x = nxt;
    else if (x <= nxt) x = x - 1;
    tri_index(x, I, J);
  } else {
    tri_index(blockIdx.x, I, J);
  }
  R *dst = A + b * sA + (int64_t)(I * GT) * n_p + J * GT;
  const R *Cb = Cbuf + b * sCO;
  if (I == K && J == K) {
    const R *Pb = Pbuf + ((int64_t)b * 2 + (K & 1)) * GT * GT;
    for (int e = threadIdx.x; e < GT * GT; e += GTHREADS) dst[(int64_t)(e >> 5) * n_p + (e & 31)] = -Pb[e];
    return;
  }
  if (J == K) {  // tile (I, K), I > K
    const R *src = Cb + (int64_t)(I * GT) * GT;
    for (int e = threadIdx.x; e < GT * GT; e += GTHREADS) dst[(int64_t)(e >> 5) * n_p + (e & 31)] = src[e];
    return;
  }
  if (I == K) {  // tile (K, J), J < K: transpose of C_J
    const R *src = Cb + (int64_t)(J * GT) * GT;
    for (int e = threadIdx.x; e < GT * GT; e += GTHREADS) {
      const int c = e >> 5, r = e & 31;
      dst[(int64_t)r * n_p + c] = src[c * GT + r];
    }
    return;
  }
  extern __shared__ __align__(16) unsigned char smraw[];
  R *Cs = reinterpret_cast<R *>(smraw);   // [32][33]  C_I[r][k]
  R *Os = Cs + GT * GLD;                  // [32][33]  O_J[c][k]
  R *sm = Cs;                             // the fused pivot sweep's workspace
  const R *ci = Cb + (int64_t)(I * GT) * GT;
  const R *oj = Obuf + b * sCO + (int64_t)(J * GT) * GT;
  for (int e = threadIdx.x; e < GT * GT; e += GTHREADS) {
    Cs[(e >> 5) * GLD + (e & 31)] = ci[e];
    Os[(e >> 5) * GLD + (e & 31)] = oj[e];
  }
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  R acc[2][4];   // starts at A_IJ; each step subtracts with one FMA
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = dst[(int64_t)(ty + 16 * i) * n_p + tx + 8 * j];
  __syncthreads();
#pragma unroll 8
  for (int k = 0; k < GT; ++k) {
    R av[2], bv[4];
#pragma unroll
    for (int i = 0; i < 2; ++i) av[i] = -Cs[(ty + 16 * i) * GLD + k];
#pragma unroll
    for (int j = 0; j < 4; ++j) bv[j] = Os[(tx + 8 * j) * GLD + k];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
  }
  const bool next_pivot = look && I == K + 1 && J == K + 1;
  if (next_pivot) __syncthreads();   // Cs/Os are reused as the sweep's workspace
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = ty + 16 * i, c = tx + 8 * j;
      dst[(int64_t)r * n_p + c] = acc[i][j];
      if (next_pivot && c <= r) sm[r * GLD + c] = acc[i][j];
    }
  if (next_pivot) {
    __syncthreads();
    sweep_tile(sm, Pbuf + ((int64_t)b * 2 + ((K + 1) & 1)) * GT * GT, logdet + (int64_t)b * ld_stride,
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

template <typename R>
constexpr size_t smem_gemm() { return 2 * T * LDS * sizeof(R); }
template <typename R>
constexpr size_t smem_update() {
  return 2 * GT * GLD * sizeof(R) > SWEEP_SMEM_DOUBLES * sizeof(R) ? 2 * GT * GLD * sizeof(R)
                                                                     : SWEEP_SMEM_DOUBLES * sizeof(R);
}
constexpr size_t SMEM_PIV = SWEEP_SMEM_DOUBLES * sizeof(double);

template <typename R>
void ensure_attrs() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(gemm_nn_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_gemm<R>());
  cudaFuncSetAttribute(gj_pivot_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_PIV);
  done = true;
}

}  // namespace

void dense_prepare() {
  ensure_attrs<double>();
  ensure_attrs<float>();
}

template <typename R>
void gj_invert(Launch &L, const DevModel &M, const Work &W, R *A, int64_t strideA, double *logdet_out,
               int logdet_slot_stride) {
  ensure_attrs<R>();
  const int n_p = M.n_p, nt = n_p / GT, P = W.P;
  const int ntri = nt * (nt + 1) / 2;
  const int64_t sCO = (int64_t)n_p * GT;
  const int tnt = n_p / T, tntri = tnt * (tnt + 1) / 2;
  R *Pb = reinterpret_cast<R *>(W.gjP);
  R *Cb = reinterpret_cast<R *>(W.gjC);
  R *Ob = reinterpret_cast<R *>(W.gjO);
  for (int K = 0; K < nt; ++K) {
    if (K == 0) {
      L.start(KID_GJ_PIVOT, (double)P);
      gj_pivot_kernel<R><<<P, GTHREADS, SMEM_PIV, L.st>>>(A, strideA, n_p, K, Pb, logdet_out, logdet_slot_stride,
                                                           W.status, W.active);
      L.stop();
      L.tick();
    }
    if (nt > 1) {
      L.start(KID_GJ_PANEL, (double)P * (nt - 1) / 8.0);
      gj_panel_kernel<R><<<dim3(nt, P), GTHREADS, 2 * GT * GLD * sizeof(R), L.st>>>(A, strideA, n_p, K, Pb, Cb, Ob,
                                                                                   sCO, W.active);
      L.stop();
      L.tick();
    }
    // units: 64 x 64 x 64 tile products (2 * 64^3 flops); a 32-tile update is 1/8 of one
    L.start(KID_GJ_UPDATE, (double)P * (ntri - nt) / 8.0);
    gj_update_kernel<R><<<dim3(ntri, P), GTHREADS, smem_update<R>(), L.st>>>(
        A, strideA, n_p, K, nt, Pb, Cb, Ob, sCO, logdet_out, logdet_slot_stride, W.status, W.active);
    L.stop();
    L.tick();
  }
  gj_finalize_kernel<R><<<dim3(tntri, P), 256, 0, L.st>>>(A, strideA, n_p, W.active);
  L.tick();
}

template <typename R>
void gemm_nn(Launch &L, int P, int n, const R *A, int64_t sA, const R *B, int64_t sB, R *C, int64_t sC, R alpha,
             const R *C0, int64_t sC0, R beta, bool lower_only, const int *active) {
  ensure_attrs<R>();
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
void mirror_lower(Launch &L, int P, int n, R *A, int64_t sA, const int *active) {
  const int nt = n / T;
  mirror_kernel<R><<<dim3(nt * (nt + 1) / 2, P), 256, 0, L.st>>>(A, sA, n, active);
  L.tick();
}

template void gj_invert<double>(Launch &, const DevModel &, const Work &, double *, int64_t, double *, int);
template void gj_invert<float>(Launch &, const DevModel &, const Work &, float *, int64_t, double *, int);
template void gemm_nn<double>(Launch &, int, int, const double *, int64_t, const double *, int64_t, double *, int64_t,
                              double, const double *, int64_t, double, bool, const int *);
template void gemm_nn<float>(Launch &, int, int, const float *, int64_t, const float *, int64_t, float *, int64_t,
                             float, const float *, int64_t, float, bool, const int *);
template void mirror_lower<double>(Launch &, int, int, double *, int64_t, const int *);
template void mirror_lower<float>(Launch &, int, int, float *, int64_t, const int *);

}  // namespace inla
