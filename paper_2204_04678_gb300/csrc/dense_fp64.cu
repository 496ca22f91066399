// Dense FP64 kernels on n_p x n_p blocks (n_p a multiple of 64), batched over
// the evaluation points of a wave (blockIdx.y = point).
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
//    pivot inversion followed by a rank-64 update of the whole lower
//    triangle, which spreads over every SM (no triangular solves on the
//    critical path).  Work: n^3 flops, the same as Cholesky + inverse.
// 2. C = alpha A B + beta C0 for the selected-inversion products.
//
// The kernels are bound by the FP64 pipe; all operand traffic is staged
// through shared memory with conflict-free access (row stride 65 doubles).
#include <cmath>

#include "inla_internal.cuh"

namespace inla {

namespace {

constexpr int T = TILE;     // 64
constexpr int LDS = T + 1;  // padded shared-memory row

__device__ __forceinline__ void tri_index(int x, int &I, int &J) {
  int i = (int)((sqrt(8.0 * x + 1.0) - 1.0) * 0.5);
  while ((i + 1) * (i + 2) / 2 <= x) ++i;
  while (i * (i + 1) / 2 > x) --i;
  I = i;
  J = x - i * (i + 1) / 2;
}

// Scalar sweep of a 64 x 64 SPD block held (lower triangle) in shared memory `a`:
// after 64 steps `a` holds -A^-1.  Writes P = A^-1 (full symmetric tile) to Pout and
// adds log|A| = sum_p log(pivot_p) to *logdet; a non-positive pivot sets *status.
// One FMA per lower entry and step; the reciprocal of each pivot is formed once
// and the logarithms once at the end.  Called by all threads of the block.
constexpr int TRI = T * (T + 1) / 2;             // 2080 lower entries
constexpr int PIV_PER_THREAD = (TRI + 255) / 256;
constexpr int SWEEP_SMEM_DOUBLES = T * LDS + 3 * T;

__device__ void sweep_tile(double *sm, double *Pout, double *logdet, int *status) {
  double *a = sm;                 // [64][65]
  double *colp = sm + T * LDS;    // [64]  column p of the current state
  double *cinv = colp + T;        // [64]  column p divided by the pivot
  double *pivs = cinv + T;        // [64]  pivots, for the log-determinant
  __shared__ double s_inv;
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  int ei[PIV_PER_THREAD], ej[PIV_PER_THREAD];
  int ne = 0;
  for (int e = tid; e < TRI; e += blockDim.x) {
    int i = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    while (i * (i + 1) / 2 > e) --i;
    ei[ne] = i;
    ej[ne] = e - i * (i + 1) / 2;
    ++ne;
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int p = 0; p < T; ++p) {
    if (tid == 0) {
      const double piv = a[p * LDS + p];
      const bool ok = (piv > 0.0) && (piv < INFINITY);
      pivs[p] = ok ? piv : 1.0;
      s_inv = ok ? 1.0 / piv : 0.0;
      if (!ok) s_bad = 1;
    }
    __syncthreads();
    if (tid < T) {
      const double c = (tid >= p) ? a[tid * LDS + p] : a[p * LDS + tid];
      colp[tid] = c;
      cinv[tid] = c * s_inv;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PIV_PER_THREAD; ++k) {
      if (k >= ne) break;
      const int i = ei[k], j = ej[k];
      double *ap = &a[i * LDS + j];
      if (i == p) *ap = (j == p) ? -s_inv : cinv[j];
      else if (j == p) *ap = cinv[i];
      else *ap = fma(-cinv[i], colp[j], *ap);
    }
    __syncthreads();
  }
  for (int e = tid; e < T * T; e += blockDim.x) {
    int i = e >> 6, j = e & 63;
    Pout[e] = -((j <= i) ? a[i * LDS + j] : a[j * LDS + i]);
  }
  if (tid < 64) {
    double l = log(pivs[tid]);
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((tid & 31) == 0) colp[tid >> 5] = l;
  }
  __syncthreads();
  if (tid == 0) {
    *logdet += colp[0] + colp[1];
    if (s_bad) *status = INLA_ERR_NOT_SPD;
  }
}

__device__ __forceinline__ void load_lower_tile(double *a, const double *src, int n_p) {
  for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
    int i = e >> 6, j = e & 63;
    if (j <= i) a[i * LDS + j] = src[(int64_t)i * n_p + j];
  }
}

// Pivot block K (used for K = 0 only: later pivots are inverted by the update
// kernel of the previous step).  Pbuf holds two 64 x 64 slots per point.
__global__ void __launch_bounds__(256) gj_pivot_kernel(double *A, int64_t sA, int n_p, int K, double *Pbuf,
                                                      double *logdet, int ld_stride, int *status,
                                                      const int *active) {
  const int b = blockIdx.x;
  if (active && !active[b]) return;
  extern __shared__ double sm[];
  load_lower_tile(sm, A + b * sA + (int64_t)(K * T) * n_p + K * T, n_p);
  __syncthreads();
  sweep_tile(sm, Pbuf + ((int64_t)b * 2 + (K & 1)) * T * T, logdet + (int64_t)b * ld_stride, status + b);
}

// C_I = A_IK P for every row tile I != K; also keep the old A_IK in Obuf.
__global__ void __launch_bounds__(256) gj_panel_kernel(const double *A, int64_t sA, int n_p, int K,
                                                      const double *Pbuf, double *Cbuf, double *Obuf,
                                                      int64_t sCO, const int *active) {
  const int I = blockIdx.x, b = blockIdx.y;
  if (I == K || (active && !active[b])) return;
  extern __shared__ double sm[];
  double *Os = sm;              // [64][65]  O[r][k]
  double *Ps = sm + T * LDS;    // [64][65]  P[k][c]
  const double *Ab = A + b * sA;
  if (I > K) {
    const double *src = Ab + (int64_t)(I * T) * n_p + K * T;
    for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
      int r = e >> 6, c = e & 63;
      Os[r * LDS + c] = src[(int64_t)r * n_p + c];
    }
  } else {  // upper tile (I, K) = transpose of the stored lower tile (K, I)
    const double *src = Ab + (int64_t)(K * T) * n_p + I * T;
    for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
      int c = e >> 6, r = e & 63;
      Os[r * LDS + c] = src[(int64_t)c * n_p + r];
    }
  }
  const double *Pb = Pbuf + ((int64_t)b * 2 + (K & 1)) * T * T;
  for (int e = threadIdx.x; e < T * T; e += blockDim.x) Ps[(e >> 6) * LDS + (e & 63)] = Pb[e];
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
#pragma unroll 4
  for (int k = 0; k < T; ++k) {
    double av[4], bv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) av[i] = Os[(ty + 16 * i) * LDS + k];
#pragma unroll
    for (int j = 0; j < 4; ++j) bv[j] = Ps[k * LDS + tx + 16 * j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
  }
  double *Cb = Cbuf + b * sCO + (int64_t)(I * T) * T;
  double *Ob = Obuf + b * sCO + (int64_t)(I * T) * T;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) Cb[(ty + 16 * i) * T + tx + 16 * j] = acc[i][j];
  for (int e = threadIdx.x; e < T * T; e += blockDim.x) Ob[e] = Os[(e >> 6) * LDS + (e & 63)];
}

// Rank-64 update of every lower tile (I, J): A_IJ -= C_I O_J^T for I, J != K;
// the pivot row/column become C (resp. C^T) and the pivot block -P.  With
// lookahead (K + 1 < nt) block 0 takes tile (K+1, K+1) and, once updated,
// inverts it as the next pivot (slot (K+1)&1 of Pbuf), so no separate pivot
// launch sits on the critical path.
__global__ void __launch_bounds__(256) gj_update_kernel(double *A, int64_t sA, int n_p, int K, int nt,
                                                       double *Pbuf, const double *Cbuf, const double *Obuf,
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
  double *Ab = A + b * sA;
  double *dst = Ab + (int64_t)(I * T) * n_p + J * T;
  const double *Cb = Cbuf + b * sCO;
  if (I == K && J == K) {
    const double *Pb = Pbuf + ((int64_t)b * 2 + (K & 1)) * T * T;
    for (int e = threadIdx.x; e < T * T; e += blockDim.x) dst[(int64_t)(e >> 6) * n_p + (e & 63)] = -Pb[e];
    return;
  }
  if (J == K) {  // tile (I, K), I > K
    const double *src = Cb + (int64_t)(I * T) * T;
    for (int e = threadIdx.x; e < T * T; e += blockDim.x) dst[(int64_t)(e >> 6) * n_p + (e & 63)] = src[e];
    return;
  }
  if (I == K) {  // tile (K, J), J < K: transpose of C_J
    const double *src = Cb + (int64_t)(J * T) * T;
    for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
      int c = e >> 6, r = e & 63;  // read C_J[c][r] coalesced, write dst[r][c]
      dst[(int64_t)r * n_p + c] = src[c * T + r];
    }
    return;
  }
  extern __shared__ double sm[];
  double *Cs = sm;            // [64][65]  C_I[r][k]
  double *Os = sm + T * LDS;  // [64][65]  O_J[c][k]
  const double *ci = Cb + (int64_t)(I * T) * T;
  const double *oj = Obuf + b * sCO + (int64_t)(J * T) * T;
  for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
    Cs[(e >> 6) * LDS + (e & 63)] = ci[e];
    Os[(e >> 6) * LDS + (e & 63)] = oj[e];
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
#pragma unroll 4
  for (int k = 0; k < T; ++k) {
    double av[4], bv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) av[i] = Cs[(ty + 16 * i) * LDS + k];
#pragma unroll
    for (int j = 0; j < 4; ++j) bv[j] = Os[(tx + 16 * j) * LDS + k];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
  }
  const bool next_pivot = look && I == K + 1 && J == K + 1;
  if (next_pivot) __syncthreads();   // Cs/Os are reused as the sweep's workspace
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double *p = dst + (int64_t)(ty + 16 * i) * n_p + tx + 16 * j;
      const double v = *p - acc[i][j];
      *p = v;
      if (next_pivot && tx + 16 * j <= ty + 16 * i) sm[(ty + 16 * i) * LDS + tx + 16 * j] = v;
    }
  if (next_pivot) {
    __syncthreads();
    sweep_tile(sm, Pbuf + ((int64_t)b * 2 + ((K + 1) & 1)) * T * T, logdet + (int64_t)b * ld_stride, status + b);
  }
}

// A <- -A on the lower triangle, mirrored into the upper triangle.
__global__ void gj_finalize_kernel(double *A, int64_t sA, int n_p, const int *active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  int I, J;
  tri_index(blockIdx.x, I, J);
  double *Ab = A + b * sA;
  for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
    int r = e >> 6, c = e & 63;
    if (I == J && c > r) continue;
    int64_t gi = I * T + r, gj = J * T + c;
    double v = -Ab[gi * n_p + gj];
    Ab[gi * n_p + gj] = v;
    Ab[gj * n_p + gi] = v;
  }
}

__global__ void mirror_kernel(double *A, int64_t sA, int n_p, const int *active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  int I, J;
  tri_index(blockIdx.x, I, J);
  double *Ab = A + b * sA;
  for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
    int r = e >> 6, c = e & 63;
    if (I == J && c >= r) continue;
    int64_t gi = I * T + r, gj = J * T + c;
    Ab[gj * n_p + gi] = Ab[gi * n_p + gj];
  }
}

// C = alpha A B + beta C0 (row-major n x n), one 64 x 64 tile of C per block.
__global__ void __launch_bounds__(256) gemm_nn_kernel(int n, const double *A, int64_t sA, const double *B,
                                                     int64_t sB, double *C, int64_t sC, double alpha,
                                                     const double *C0, int64_t sC0, double beta, int lower_only,
                                                     const int *active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int nt = n / T;
  int I, J;
  if (lower_only) tri_index(blockIdx.x, I, J);
  else { I = blockIdx.x / nt; J = blockIdx.x % nt; }
  extern __shared__ double sm[];
  double *As = sm;            // [64][65]  A[r][k]
  double *Bs = sm + T * LDS;  // [64][65]  B[k][c]
  const double *Ab = A + b * sA + (int64_t)(I * T) * n;
  const double *Bb = B + b * sB + J * T;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int kk = 0; kk < nt; ++kk) {
    for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
      int r = e >> 6, c = e & 63;
      As[r * LDS + c] = Ab[(int64_t)r * n + kk * T + c];
      Bs[r * LDS + c] = Bb[(int64_t)(kk * T + r) * n + c];
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < T; ++k) {
      double av[4], bv[4];
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
  double *Cb = C + b * sC + (int64_t)(I * T) * n + J * T;
  const double *C0b = C0 ? C0 + b * sC0 + (int64_t)(I * T) * n + J * T : nullptr;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t off = (int64_t)(ty + 16 * i) * n + tx + 16 * j;
      double v = alpha * acc[i][j];
      if (C0b) v += beta * C0b[off];
      Cb[off] = v;
    }
}

constexpr size_t SMEM2 = 2 * T * LDS * sizeof(double);
constexpr size_t SMEM_PIV = SWEEP_SMEM_DOUBLES * sizeof(double);

bool g_attr_done = false;
void ensure_attrs() {
  if (g_attr_done) return;
  cudaFuncSetAttribute(gj_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM2);
  cudaFuncSetAttribute(gj_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM2);
  cudaFuncSetAttribute(gemm_nn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM2);
  cudaFuncSetAttribute(gj_pivot_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_PIV);
  g_attr_done = true;
}

}  // namespace

void gj_invert(Launch &L, const DevModel &M, const Work &W, double *A, int64_t strideA, double *logdet_out,
               int logdet_slot_stride) {
  ensure_attrs();
  const int n_p = M.n_p, nt = n_p / T, P = W.P;
  const int ntri = nt * (nt + 1) / 2;
  const int64_t sCO = (int64_t)n_p * T;
  for (int K = 0; K < nt; ++K) {
    if (K == 0) {
      L.start(KID_GJ_PIVOT, (double)P);
      gj_pivot_kernel<<<P, 256, SMEM_PIV, L.st>>>(A, strideA, n_p, K, W.gjP, logdet_out, logdet_slot_stride,
                                                   W.status, W.active);
      L.stop();
      L.tick();
    }
    if (nt > 1) {
      L.start(KID_GJ_PANEL, (double)P * (nt - 1));
      gj_panel_kernel<<<dim3(nt, P), 256, SMEM2, L.st>>>(A, strideA, n_p, K, W.gjP, W.gjC, W.gjO, sCO, W.active);
      L.stop();
      L.tick();
    }
    // units: rank-64 updates of one 64 x 64 tile (2 * 64^3 flops each)
    L.start(KID_GJ_UPDATE, (double)P * (ntri - nt));
    gj_update_kernel<<<dim3(ntri, P), 256, SMEM2, L.st>>>(A, strideA, n_p, K, nt, W.gjP, W.gjC, W.gjO, sCO,
                                                           logdet_out, logdet_slot_stride, W.status, W.active);
    L.stop();
    L.tick();
  }
  gj_finalize_kernel<<<dim3(ntri, P), 256, 0, L.st>>>(A, strideA, n_p, W.active);
  L.tick();
}

void gemm_nn(Launch &L, int P, int n, const double *A, int64_t sA, const double *B, int64_t sB, double *C,
             int64_t sC, double alpha, const double *C0, int64_t sC0, double beta, bool lower_only,
             const int *active) {
  ensure_attrs();
  const int nt = n / T;
  const int tiles = lower_only ? nt * (nt + 1) / 2 : nt * nt;
  // units: 64 x 64 x 64 tile products (2 * 64^3 flops each)
  L.start(KID_GEMM, (double)P * tiles * nt);
  gemm_nn_kernel<<<dim3(tiles, P), 256, SMEM2, L.st>>>(n, A, sA, B, sB, C, sC, alpha, C0, sC0, beta,
                                                        lower_only ? 1 : 0, active);
  L.stop();
  L.tick();
}

void mirror_lower(Launch &L, int P, int n, double *A, int64_t sA, const int *active) {
  const int nt = n / T;
  mirror_kernel<<<dim3(nt * (nt + 1) / 2, P), 256, 0, L.st>>>(A, sA, n, active);
  L.tick();
}

}  // namespace inla
