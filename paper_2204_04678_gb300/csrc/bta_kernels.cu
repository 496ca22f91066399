// Kernels of the block-tridiagonal-arrowhead path: hyperparameter maps,
// sparse assembly of the Schur-complement blocks, block substitution, the
// block Takahashi recursion's small pieces, contractions for the gradient,
// observation-space reductions and the final assembly of f and grad f.
//
// Notation (per evaluation point): Q_c has diagonal blocks A_t, sub-diagonal
// blocks B_t = q_off Q_s (block (t+1, t)), arrow blocks R_t and tip A_a.  The
// block LDL^T factorisation keeps D_t^-1 (Dinv_t) and R~_t:
//   D_0 = A_0,  D_t = A_t - q_off^2 Q_s D_{t-1}^-1 Q_s,
//   R~_0 = R_0, R~_t = R_t - q_off (R~_{t-1} D_{t-1}^-1) Q_s,
//   D_a = A_a - sum_t R~_t D_t^-1 R~_t^T,
// and log|Q_c| = sum_t log|D_t| + log|D_a| (Sec. 2.4: the log-determinant is
// read off the factorisation).  The sub-diagonal blocks stay sparse, so the
// only dense work per time step is one n_s x n_s inversion (dense_fp64.cu).
#include <cmath>

#include <cstring>
#include <mutex>

#include "inla_internal.cuh"

namespace inla {

namespace {

__device__ __forceinline__ double q_tt(const PointParams &p, int t, int n_t) {
  if (n_t == 1) return 1.0;
  return (t == 0 || t == n_t - 1) ? p.qd_end : p.qd_mid;
}
__device__ __forceinline__ double dq_tt(const PointParams &p, int t, int n_t) {
  if (n_t == 1) return 0.0;
  return (t == 0 || t == n_t - 1) ? p.dqd_end : p.dqd_mid;
}

// Sum over a block of 256 threads; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;
}

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}


// 16-byte vector access to R arrays (4 floats or 2 doubles); addresses 16-byte aligned.
template <typename R>
struct Vec16 {
  static constexpr int N = 16 / sizeof(R);
};
template <typename R>
__device__ __forceinline__ void ld16(R (&v)[16 / sizeof(R)], const R *p) {
  const uint4 u = *reinterpret_cast<const uint4 *>(p);
  memcpy(v, &u, 16);
}
template <typename R>
__device__ __forceinline__ void st16(R *p, const R (&v)[16 / sizeof(R)]) {
  uint4 u;
  memcpy(&u, v, 16);
  *reinterpret_cast<uint4 *>(p) = u;
}

// Likelihood part of the arrow block (a, t), row l, column i (scaled into Q_c).
__device__ __forceinline__ double lik_arrow(const DevModel &M, const Work &W, int mode, int b, int t, int l, int i) {
  if (mode != ASM_QC || M.n_b == 0) return 0.0;
  const int64_t k = ((int64_t)t * M.n_b + l) * M.n_s + i;
  if (M.lik == INLA_LIK_GAUSSIAN) return W.prm[b].tau_y * M.Arw[k];
  return W.Arwp[b * W.sArwp + k];
}

// ------------------------------------------------------------------ parameters

__global__ void params_kernel(DevModel M, Work W) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= W.P) return;
  const double *th = W.theta + 4 * b;
  PointParams p;
  for (int j = 0; j < 4; ++j) p.theta[j] = th[j];
  const bool gauss = M.lik == INLA_LIK_GAUSSIAN;
  p.tau_y = gauss ? exp(th[0]) : 0.0;
  p.tau_b = gauss ? M.tau_b_fixed : exp(th[0]);
  const double r = exp(th[1]), sigma = exp(th[2]);
  const double rho = 1.0 / (1.0 + exp(-th[3]));
  const double kappa = sqrt(8.0) / r;
  const double k2 = kappa * kappa;
  const double tau2 = 1.0 / (4.0 * M_PI * k2 * sigma * sigma);
  p.aC = tau2 * k2 * k2;
  p.aG = 2.0 * tau2 * k2;
  p.aH = tau2;
  p.rho = rho;
  const double s = 1.0 - rho * rho;
  const double drho = rho * (1.0 - rho);
  if (M.n_t == 1) {
    p.qd_end = p.qd_mid = 1.0;
    p.q_off = 0.0;
    p.dqd_end = p.dqd_mid = p.dq_off = 0.0;
  } else {
    p.qd_end = 1.0 / s;
    p.qd_mid = (1.0 + rho * rho) / s;
    p.q_off = -rho / s;
    p.dqd_end = 2.0 * rho / (s * s) * drho;
    p.dqd_mid = 4.0 * rho / (s * s) * drho;
    p.dq_off = -(1.0 + rho * rho) / (s * s) * drho;
  }
  double lp = 0.0;
  for (int j = 0; j < 4; ++j) {
    const double z = (th[j] - M.prior_mean[j]) / M.prior_sd[j];
    lp += -0.5 * log(2.0 * M_PI) - log(M.prior_sd[j]) - 0.5 * z * z;
    p.dlogprior[j] = -(th[j] - M.prior_mean[j]) / (M.prior_sd[j] * M.prior_sd[j]);
  }
  p.logprior = lp;
  W.prm[b] = p;
}

__global__ void qs_values_kernel(DevModel M, Work W) {
  const int b = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M.nnz) return;
  const PointParams &p = W.prm[b];
  W.qs[b * W.sNnz + e] = p.aC * M.vC[e] + p.aG * M.vG[e] + p.aH * M.vH[e];
}

__global__ void set_active_kernel(Work W, int mask) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= W.P) return;
  W.active[b] = (mask == 0) ? 1 : ((W.flags[b] & mask) ? 1 : 0);
}

// ------------------------------------------------------------------ factorisation pieces

// R~_t0 = R_t0 for the first block t0 of an elimination chain, and the tip
// D_a = A_a before the Schur updates (tip_init = 0: D_a = 0, the accumulator of
// a second chain's Schur updates).
__global__ void init_step0_kernel(DevModel M, Work W, int mode, int t0, int tip_init) {
  const int b = blockIdx.z;
  if (!W.active[b]) return;
  const int l = blockIdx.y;
  const int n_b = M.n_b, n_p = M.n_p;
  if (l < n_b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_p) return;
    W.Rt[b * W.sRt + ((int64_t)t0 * n_b + l) * n_p + i] = (i < M.n_s) ? lik_arrow(M, W, mode, b, t0, l, i) : 0.0;
    return;
  }
  if (blockIdx.x != 0) return;
  for (int e = threadIdx.x; e < n_b * n_b; e += blockDim.x) {
    const int r = e / n_b, c = e % n_b;
    double v = (r == c && tip_init) ? W.prm[b].tau_b : 0.0;
    if (mode == ASM_QC && tip_init) {
      if (M.lik == INLA_LIK_GAUSSIAN) v += W.prm[b].tau_y * M.Tip[e];
      else v += W.Tipp[b * W.sNb2 + e];
    }
    W.Da[b * W.sNb2 + e] = v;
  }
}

// Dense diagonal block: D_t = c_t Q_s + (likelihood block) - [schur] q_off^2 Q_s T1,
// with T1 = Dinv_{t-1} Q_s; identity in the padding.  mode ASM_QS builds Q_s alone.
// Only the lower 32-wide tiles are written: the block sweep (32- or 64-wide
// tiles) reads nothing else.  T1 is computed up to 64-wide tiles past the band.
constexpr int SWEEP_TILE = 32, SWEEP_TILE_MAX = 64;
// Row i of the lower 32-tiles of the diagonal block: the sparse part
// c Q_s + (likelihood) staged in a shared row buffer, minus (Schur update)
// q_off^2 (Q_s T1)_{i,:}, with T1 = D_{t-1}^-1 Q_s; identity in the padding.
// One block per (row, point); the row's pattern (<= ROW_PMAX entries) is staged
// in shared memory so that every thread streams 16-byte vectors of T1 rows.
template <typename R>
__global__ void __launch_bounds__(256) assemble_diag_kernel(DevModel M, Work W, int t, int mode, R *dst,
                                                           int64_t sdst, int schur) {
  constexpr int V = Vec16<R>::N;
  const int b = blockIdx.y, i = blockIdx.x;
  if (!W.active[b]) return;
  extern __shared__ double rowbuf[];     // [n_p]: the sparse part of row i
  __shared__ int pc[ROW_PMAX];
  __shared__ R pv[ROW_PMAX];
  const int n_p = M.n_p, n_s = M.n_s;
  const int jmax = min(n_p, (i / SWEEP_TILE + 1) * SWEEP_TILE);
  R *out = dst + b * sdst + (int64_t)i * n_p;
  if (i >= n_s) {
    for (int j = threadIdx.x; j < jmax; j += blockDim.x) out[j] = (i == j) ? R(1) : R(0);
    return;
  }
  const PointParams &p = W.prm[b];
  const double c = (mode == ASM_QS) ? 1.0 : q_tt(p, t, M.n_t);
  const double *qs = W.qs + b * W.sNnz;
  const double *lik = nullptr;
  double lik_scale = 0.0;
  if (mode == ASM_QC) {
    if (M.lik == INLA_LIK_GAUSSIAN) { lik = M.AtA + (int64_t)t * M.nnz; lik_scale = p.tau_y; }
    else { lik = W.AtAp + b * W.sAtAp + (int64_t)t * M.nnz; lik_scale = 1.0; }
  }
  const int e0 = M.prow[i], len = M.prow[i + 1] - e0;
  for (int j = threadIdx.x; j < jmax; j += blockDim.x) rowbuf[j] = 0.0;
  __syncthreads();
  for (int e = threadIdx.x; e < len; e += blockDim.x) {
    const int k = M.pcol[e0 + e];
    pc[e] = k;
    pv[e] = (R)qs[e0 + e];
    if (k < jmax) rowbuf[k] = c * qs[e0 + e] + (lik ? lik_scale * lik[e0 + e] : 0.0);
  }
  __syncthreads();
  const R *T1 = static_cast<const R *>(W.T1) + b * W.sMat;
  const R q2 = (R)(p.q_off * p.q_off);
  for (int j = threadIdx.x * V; j < jmax; j += blockDim.x * V) {
    R acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = R(0);
    if (schur) {
      int e = 0;
      for (; e + 2 <= len; e += 2) {
        R x0[V], x1[V];
        ld16<R>(x0, T1 + (int64_t)pc[e] * n_p + j);
        ld16<R>(x1, T1 + (int64_t)pc[e + 1] * n_p + j);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = fma(pv[e + 1], x1[v], fma(pv[e], x0[v], acc[v]));
      }
      if (e < len) {
        R x0[V];
        ld16<R>(x0, T1 + (int64_t)pc[e] * n_p + j);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = fma(pv[e], x0[v], acc[v]);
      }
    }
    R o[V];
#pragma unroll
    for (int v = 0; v < V; ++v) o[v] = (j + v < n_s) ? fma(-q2, acc[v], (R)rowbuf[j + v]) : R(0);
    st16<R>(out + j, o);
  }
}

// out[i][j] = coef * sum_k X[i][k] Q_s[k][j] + sum_l SigA[l][i] Rt[l][j]   (i, j < n_s; 0 elsewhere)
// lower_band: only columns j < (floor((i + pbw) / 32) + 1) * 32, the ones the
// lower-tile assembly of rows within the pattern bandwidth of i reads.
// Tiled form: a block computes 64 rows x 32 columns of the output.  The pattern
// rows of its 32 columns are staged once in shared memory (SR_PMAX entries
// each), so the CSR is read once per 64 output rows instead of once per row.
constexpr int SR_COLS = 32, SR_ROWS = 64, SR_PMAX = 32;
template <typename R>
__global__ void __launch_bounds__(256) sparse_right_tiled_kernel(DevModel M, Work W, const R *X, int64_t sX, R *outp,
                                                                int64_t sOut, int coef_qoff, const double *SigA,
                                                                const double *Rt_t, int lower_band) {
  const int b = blockIdx.z;
  if (!W.active[b]) return;
  __shared__ int pc[SR_COLS][SR_PMAX + 1];   // +1: consecutive columns in distinct banks
  __shared__ R pv[SR_COLS][SR_PMAX + 1];
  __shared__ int pn[SR_COLS];
  const int n_p = M.n_p, n_s = M.n_s;
  const int j0 = blockIdx.x * SR_COLS, i0 = blockIdx.y * SR_ROWS;
  const int tj = threadIdx.x & 31, ti = threadIdx.x >> 5;
  const double *qs = W.qs + b * W.sNnz;
  const R coef = coef_qoff ? (R)W.prm[b].q_off : R(1);
  for (int c = ti; c < SR_COLS; c += 8) {
    const int j = j0 + c;
    const int e0 = (j < n_s) ? M.prow[j] : 0, len = (j < n_s) ? M.prow[j + 1] - e0 : 0;
    if (tj == 0) pn[c] = len;
    if (tj < len) {
      pc[c][tj] = M.pcol[e0 + tj];
      pv[c][tj] = coef * (R)qs[e0 + tj];
    }
  }
  __syncthreads();
  const int j = j0 + tj;
  const int len = pn[tj];
  const double *sa = SigA ? SigA + b * W.sNbNp : nullptr;
  const double *rt = SigA ? Rt_t + b * W.sRt : nullptr;
  for (int r = 0; r < SR_ROWS / 8; ++r) {
    const int i = i0 + ti + 8 * r;
    if (i >= n_p || j >= n_p) continue;
    if (lower_band && j >= ((i + M.pbw) / SWEEP_TILE_MAX + 1) * SWEEP_TILE_MAX) continue;
    R *out = outp + b * sOut + (int64_t)i * n_p + j;
    if (i >= n_s || j >= n_s) { *out = R(0); continue; }
    const R *Xi = X + b * sX + (int64_t)i * n_p;
    R acc = 0;
    for (int e = 0; e < len; ++e) acc = fma(Xi[pc[tj][e]], pv[tj][e], acc);
    if (sa)
      for (int l = 0; l < M.n_b; ++l) acc = fma((R)sa[(int64_t)l * n_p + i], (R)rt[(int64_t)l * n_p + j], acc);
    *out = acc;
  }
}

template <typename R>
__global__ void sparse_right_kernel(DevModel M, Work W, const R *X, int64_t sX, R *outp, int64_t sOut,
                                    int coef_qoff, const double *SigA, const double *Rt_t, int lower_band) {
  const int b = blockIdx.z;
  if (!W.active[b]) return;
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_p = M.n_p, n_s = M.n_s;
  if (j >= n_p) return;
  if (lower_band && j >= ((i + M.pbw) / SWEEP_TILE_MAX + 1) * SWEEP_TILE_MAX) return;
  R *out = outp + b * sOut + (int64_t)i * n_p + j;
  if (i >= n_s || j >= n_s) { *out = R(0); return; }
  const R *Xi = X + b * sX + (int64_t)i * n_p;
  const double *qs = W.qs + b * W.sNnz;
  R acc = 0;
  for (int e = M.prow[j]; e < M.prow[j + 1]; ++e) acc = fma(Xi[M.pcol[e]], (R)qs[e], acc);
  if (coef_qoff) acc *= (R)W.prm[b].q_off;
  if (SigA) {
    const double *sa = SigA + b * W.sNbNp;
    const double *rt = Rt_t + b * W.sRt;
    for (int l = 0; l < M.n_b; ++l) acc = fma((R)sa[(int64_t)l * n_p + i], (R)rt[(int64_t)l * n_p + j], acc);
  }
  *out = acc;
}

// out[i][j] = [with_X] q_off * sum_k Q_s[i][k] X[k][j] + sum_l Rt[l][i] Y[l][j]
// One block per (row, point): the row's pattern is staged in shared memory and
// every thread streams 16-byte vectors of the pattern rows of X.
template <typename R>
__global__ void __launch_bounds__(256) sparse_left_kernel(DevModel M, Work W, const R *X, int64_t sX, R *outp,
                                                         int64_t sOut, int with_X, const double *Rt_t,
                                                         const double *Ymat) {
  constexpr int V = Vec16<R>::N;
  const int b = blockIdx.y, i = blockIdx.x;
  if (!W.active[b]) return;
  __shared__ int pc[ROW_PMAX];
  __shared__ R pv[ROW_PMAX];
  __shared__ R rv[MAX_NB];
  const int n_p = M.n_p, n_s = M.n_s;
  R *out = outp + b * sOut + (int64_t)i * n_p;
  if (i >= n_s) {
    R z[V];
#pragma unroll
    for (int v = 0; v < V; ++v) z[v] = R(0);
    for (int j = threadIdx.x * V; j < n_p; j += blockDim.x * V) st16<R>(out + j, z);
    return;
  }
  const int e0 = M.prow[i], len = with_X ? M.prow[i + 1] - e0 : 0;
  const R q = (R)W.prm[b].q_off;
  const double *qs = W.qs + b * W.sNnz;
  for (int e = threadIdx.x; e < len; e += blockDim.x) {
    pc[e] = M.pcol[e0 + e];
    pv[e] = q * (R)qs[e0 + e];
  }
  const int nb = Ymat ? M.n_b : 0;
  if (threadIdx.x < nb) rv[threadIdx.x] = (R)Rt_t[b * W.sRt + (int64_t)threadIdx.x * n_p + i];
  __syncthreads();
  const R *Xb = X + b * sX;
  const double *Y = Ymat ? Ymat + b * W.sNbNp : nullptr;
  for (int j = threadIdx.x * V; j < n_p; j += blockDim.x * V) {
    R acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = R(0);
    int e = 0;
    for (; e + 2 <= len; e += 2) {
      R x0[V], x1[V];
      ld16<R>(x0, Xb + (int64_t)pc[e] * n_p + j);
      ld16<R>(x1, Xb + (int64_t)pc[e + 1] * n_p + j);
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = fma(pv[e + 1], x1[v], fma(pv[e], x0[v], acc[v]));
    }
    if (e < len) {
      R x0[V];
      ld16<R>(x0, Xb + (int64_t)pc[e] * n_p + j);
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = fma(pv[e], x0[v], acc[v]);
    }
    for (int l = 0; l < nb; ++l)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = fma(rv[l], (R)Y[(int64_t)l * n_p + j + v], acc[v]);
#pragma unroll
    for (int v = 0; v < V; ++v)
      if (j + v >= n_s) acc[v] = R(0);
    st16<R>(out + j, acc);
  }
}

// out[i] = scale * sum_k Dinv[i][k] v[k]: the block GEMV of the substitutions,
// bound by streaming D_t^-1 from HBM.  The vector is staged once per block in
// shared memory (as R); each warp reads 2 rows of D_t^-1 in 16-byte vectors.
constexpr int GV_ROWS_PER_WARP = 2;
constexpr int GV_ROWS = 8 * GV_ROWS_PER_WARP;
template <typename R>
__global__ void __launch_bounds__(256) dinv_gemv_kernel(DevModel M, Work W, const R *Dinv_t, const double *vecs,
                                                       int64_t sVecs, double *outp, int64_t sOut, double scale) {
  constexpr int V = Vec16<R>::N;
  const int b = blockIdx.y;
  if (!W.active[b]) return;
  extern __shared__ __align__(16) unsigned char gv_raw[];
  R *vs = reinterpret_cast<R *>(gv_raw);
  const int n_p = M.n_p;
  const double *vb = vecs + b * sVecs;
  for (int k = threadIdx.x; k < n_p; k += blockDim.x) vs[k] = (R)vb[k];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * GV_ROWS + warp * GV_ROWS_PER_WARP;
  if (row0 >= n_p) return;
  const R *D0 = Dinv_t + b * W.sDinv + (int64_t)row0 * n_p;
  const R *D1 = D0 + n_p;   // row0 + 1 < n_p: n_p is a multiple of 64
  R a0 = R(0), a1 = R(0);
#pragma unroll 4
  for (int k = lane * V; k < n_p; k += 32 * V) {
    R d0[V], d1[V], x[V];
    ld16<R>(d0, D0 + k);
    ld16<R>(d1, D1 + k);
    ld16<R>(x, vs + k);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      a0 = fma(d0[v], x[v], a0);
      a1 = fma(d1[v], x[v], a1);
    }
  }
  a0 = warp_sum(a0);
  a1 = warp_sum(a1);
  if (lane == 0) {
    double *O = outp + b * sOut;
    O[row0] = scale * (double)a0;
    O[row0 + 1] = scale * (double)a1;
  }
}

// out[c][i] = scale * sum_k Dinv[i][k] vecs[c][k], c < nvec (Dinv symmetric).
constexpr int DA_ROWS_PER_WARP = 2;
constexpr int DA_ROWS = 8 * DA_ROWS_PER_WARP;
constexpr int DA_CHUNK = 256;
constexpr int DA_MAXV = 1 + MAX_NB;
// NV: the number of vectors the kernel is compiled for (1, or up to 1 + MAX_NB).
template <typename R, int NV>
__global__ void __launch_bounds__(256) dinv_apply_kernel(DevModel M, Work W, const R *Dinv_t, int nvec,
                                                        const double *vecs, int64_t sVecs, double *outp,
                                                        int64_t sOut, double scale) {
  const int b = blockIdx.y;
  if (!W.active[b]) return;
  __shared__ R vs[NV * DA_CHUNK];
  const int n_p = M.n_p;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * DA_ROWS + warp * DA_ROWS_PER_WARP;
  const R *D = Dinv_t + b * W.sDinv;
  const double *V = vecs + b * sVecs;
  R acc[DA_ROWS_PER_WARP][NV];
#pragma unroll
  for (int r = 0; r < DA_ROWS_PER_WARP; ++r)
#pragma unroll
    for (int c = 0; c < NV; ++c) acc[r][c] = 0;
  for (int k0 = 0; k0 < n_p; k0 += DA_CHUNK) {
    __syncthreads();
    for (int e = threadIdx.x; e < nvec * DA_CHUNK; e += blockDim.x) {
      const int c = e / DA_CHUNK, k = e % DA_CHUNK;
      vs[e] = (k0 + k < n_p) ? (R)V[(int64_t)c * n_p + k0 + k] : R(0);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < DA_ROWS_PER_WARP; ++r) {
      const int row = row0 + r;
      if (row >= n_p) continue;
      const R *Dr = D + (int64_t)row * n_p + k0;
      for (int q = lane; q < DA_CHUNK && k0 + q < n_p; q += 32) {
        const R d = Dr[q];
#pragma unroll
        for (int c = 0; c < NV; ++c)
          if (NV == 1 || c < nvec) acc[r][c] = fma(d, vs[c * DA_CHUNK + q], acc[r][c]);
      }
    }
  }
  double *O = outp + b * sOut;
#pragma unroll
  for (int r = 0; r < DA_ROWS_PER_WARP; ++r) {
    const int row = row0 + r;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      if (c >= nvec) break;
      const R s = warp_sum(acc[r][c]);
      if (lane == 0 && row < n_p) O[(int64_t)c * n_p + row] = scale * (double)s;
    }
  }
}

// R~_t = R_t - q_off V Q_s with V = R~_{t-1} Dinv_{t-1} (rows of W.wv).
__global__ void arrow_update_kernel(DevModel M, Work W, int t, int mode) {
  const int b = blockIdx.z;
  if (!W.active[b]) return;
  const int l = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_p = M.n_p;
  if (i >= n_p) return;
  double *out = W.Rt + b * W.sRt + ((int64_t)t * M.n_b + l) * n_p + i;
  if (i >= M.n_s) { *out = 0.0; return; }
  const double *V = W.wv + b * W.sWV + (int64_t)l * n_p;
  const double *qs = W.qs + b * W.sNnz;
  double acc = 0.0;
  for (int e = M.prow[i]; e < M.prow[i + 1]; ++e) acc = fma(qs[e], V[M.pcol[e]], acc);
  *out = lik_arrow(M, W, mode, b, t, l, i) - W.prm[b].q_off * acc;
}

// D_a -= V R~_{tprev}^T with V = R~_{tprev} Dinv_{tprev} (rows of W.wv).
__global__ void arrow_dots_kernel(DevModel M, Work W, int tprev) {
  const int b = blockIdx.y;
  if (!W.active[b]) return;
  __shared__ double red[32];
  const int l = blockIdx.x / M.n_b, l2 = blockIdx.x % M.n_b;
  const int n_p = M.n_p;
  const double *V = W.wv + b * W.sWV + (int64_t)l * n_p;
  const double *R = W.Rt + b * W.sRt + ((int64_t)tprev * M.n_b + l2) * n_p;
  double s = 0.0;
  for (int i = threadIdx.x; i < M.n_s; i += blockDim.x) s = fma(V[i], R[i], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) W.Da[b * W.sNb2 + l * M.n_b + l2] -= s;
}

// Tip: Cholesky of D_a (log-det), then D_a <- D_a^-1.
__global__ void tip_kernel(DevModel M, Work W, int ld_slot) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= W.P || !W.active[b]) return;
  const int nb = M.n_b;
  if (nb == 0) return;
  double a[MAX_NB * MAX_NB];
  double *Da = W.Da + b * W.sNb2;
  for (int e = 0; e < nb * nb; ++e) a[e] = Da[e];
  double ld = 0.0;
  bool ok = true;
  for (int j = 0; j < nb; ++j) {  // in-place lower Cholesky
    double s = a[j * nb + j];
    for (int k = 0; k < j; ++k) s -= a[j * nb + k] * a[j * nb + k];
    if (!(s > 0.0) || !(s < INFINITY)) { ok = false; s = 1.0; }
    const double d = sqrt(s);
    a[j * nb + j] = d;
    ld += 2.0 * log(d);
    for (int i = j + 1; i < nb; ++i) {
      double v = a[i * nb + j];
      for (int k = 0; k < j; ++k) v -= a[i * nb + k] * a[j * nb + k];
      a[i * nb + j] = v / d;
    }
  }
  double li[MAX_NB * MAX_NB];  // L^-1 (lower)
  for (int j = 0; j < nb; ++j) {
    for (int i = 0; i < nb; ++i) li[i * nb + j] = 0.0;
    li[j * nb + j] = 1.0 / a[j * nb + j];
    for (int i = j + 1; i < nb; ++i) {
      double v = 0.0;
      for (int k = j; k < i; ++k) v -= a[i * nb + k] * li[k * nb + j];
      li[i * nb + j] = v / a[i * nb + i];
    }
  }
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) {
      double v = 0.0;
      for (int k = (i > j ? i : j); k < nb; ++k) v += li[k * nb + i] * li[k * nb + j];
      Da[i * nb + j] = v;
    }
  W.sc[b * SC_COUNT + ld_slot] += ld;
  if (!ok) W.status[b] = INLA_ERR_NOT_SPD;
}

// ------------------------------------------------------------------ block substitution

// z_nbr -= q_off Q_s w_t;  z_a -= R~_t w_t   (w_t = Dinv_t z_t in W.wv row 0; nbr: the
// neighbour of t eliminated after it, t + 1 or t - 1, or -1 for none)
__global__ void fwd_update_kernel(DevModel M, Work W, int t, int nbr, double *z) {
  const int b = blockIdx.y;
  if (!W.active[b]) return;
  const int n_p = M.n_p;
  const int nblk = (n_p + blockDim.x - 1) / blockDim.x;
  const double *w = W.wv + b * W.sWV;
  double *zb = z + b * W.sVec;
  if ((int)blockIdx.x < nblk) {
    if (nbr < 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M.n_s) return;
    const double *qs = W.qs + b * W.sNnz;
    double acc = 0.0;
    for (int e = M.prow[i]; e < M.prow[i + 1]; ++e) acc = fma(qs[e], w[M.pcol[e]], acc);
    zb[(int64_t)nbr * n_p + i] -= W.prm[b].q_off * acc;
    return;
  }
  __shared__ double red[32];
  for (int l = 0; l < M.n_b; ++l) {
    const double *R = W.Rt + b * W.sRt + ((int64_t)t * M.n_b + l) * n_p;
    double s = 0.0;
    for (int i = threadIdx.x; i < M.n_s; i += blockDim.x) s = fma(R[i], w[i], s);
    s = block_sum(s, red);
    if (threadIdx.x == 0) zb[(int64_t)M.n_t * n_p + l] -= s;
  }
}

// x_a = Sigma_a z_a
__global__ void tip_solve_kernel(DevModel M, Work W, const double *z, double *x) {
  const int b = blockIdx.x;
  if (!W.active[b]) return;
  const int l = threadIdx.x;
  if (l >= M.n_b) return;
  const int64_t tail = (int64_t)M.n_t * M.n_p;
  const double *Da = W.Da + b * W.sNb2;
  double v = 0.0;
  for (int k = 0; k < M.n_b; ++k) v += Da[l * M.n_b + k] * z[b * W.sVec + tail + k];
  x[b * W.sVec + tail + l] = v;
}

// tmpv = z_t - q_off Q_s x_nbr - R~_t^T x_a   (nbr as in fwd_update_kernel)
__global__ void bwd_rhs_kernel(DevModel M, Work W, int t, int nbr, const double *z, const double *x) {
  const int b = blockIdx.y;
  if (!W.active[b]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_p = M.n_p;
  if (i >= n_p) return;
  double *out = W.tmpv + b * W.sVec + i;
  if (i >= M.n_s) { *out = 0.0; return; }
  const double *zb = z + b * W.sVec;
  const double *xb = x + b * W.sVec;
  double v = zb[(int64_t)t * n_p + i];
  if (nbr >= 0) {
    const double *qs = W.qs + b * W.sNnz;
    const double *xn = xb + (int64_t)nbr * n_p;
    double acc = 0.0;
    for (int e = M.prow[i]; e < M.prow[i + 1]; ++e) acc = fma(qs[e], xn[M.pcol[e]], acc);
    v -= W.prm[b].q_off * acc;
  }
  const double *R = W.Rt + b * W.sRt + (int64_t)t * M.n_b * n_p;
  const double *xa = xb + (int64_t)M.n_t * n_p;
  for (int l = 0; l < M.n_b; ++l) v -= R[(int64_t)l * n_p + i] * xa[l];
  *out = v;
}

// ------------------------------------------------------------------ joining two elimination chains
//
// The time chain split at a separator block k (nested dissection, Sec. 3.3): blocks
// 0..k-1 and n_t-1..k+1 are eliminated as two independent chains, each in its own
// scratch; these kernels add the second chain's contributions into the first's.

// dst += src over `count` elements per point (the Schur products D^-1 Q_s of the two
// neighbours of the separator; the arrow rows R~ D^-1 of the two chains).
template <typename R>
__global__ void add_into_kernel(R *dst, const R *src, int64_t stride, int64_t count, const int *active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  R *d = dst + b * stride;
  const R *s = src + b * stride;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    d[i] += s[i];
}

// D_a += D_a' (the second chain's Schur updates of the tip, accumulated from 0) and
// the second chain's log-determinant into the slot.
__global__ void join_tip_kernel(DevModel M, Work W, const double *Da1, const double *sc1, int ld_slot) {
  const int b = blockIdx.x;
  if (!W.active[b]) return;
  for (int e = threadIdx.x; e < M.n_b * M.n_b; e += blockDim.x) W.Da[b * W.sNb2 + e] += Da1[b * W.sNb2 + e];
  if (threadIdx.x == 0) W.sc[b * SC_COUNT + ld_slot] += sc1[b * SC_COUNT + ld_slot];
}

// Forward substitution: z_k and z_a receive both chains' updates; the second chain
// worked on its own copy z' of the right-hand side, so z += z' - rhs there.
__global__ void join_rhs_kernel(DevModel M, Work W, int k, double *z, const double *z1, const double *rhs) {
  const int b = blockIdx.y;
  if (!W.active[b]) return;
  const int n_p = M.n_p;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int64_t o;
  if (i < n_p) o = (int64_t)k * n_p + i;
  else if (i < n_p + M.n_b) o = (int64_t)M.n_t * n_p + (i - n_p);
  else return;
  o += b * W.sVec;
  z[o] += z1[o] - rhs[o];
}

// ------------------------------------------------------------------ selected inversion pieces

// Y = [has_next] Sigma_{a,t+1} B_t + Sigma_a R~_t    (n_b x n_s)
__global__ void selinv_Y_kernel(DevModel M, Work W, int t, int has_next) {
  const int b = blockIdx.z;
  if (!W.active[b]) return;
  const int l = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_p = M.n_p;
  if (j >= n_p) return;
  double *out = W.Y + b * W.sNbNp + (int64_t)l * n_p + j;
  if (j >= M.n_s) { *out = 0.0; return; }
  double acc = 0.0;
  if (has_next) {
    const double *sa = W.SigAn + b * W.sNbNp + (int64_t)l * n_p;
    const double *qs = W.qs + b * W.sNnz;
    for (int e = M.prow[j]; e < M.prow[j + 1]; ++e) acc = fma(sa[M.pcol[e]], qs[e], acc);
    acc *= W.prm[b].q_off;
  }
  const double *Sa = W.Da + b * W.sNb2;
  const double *R = W.Rt + b * W.sRt + (int64_t)t * M.n_b * n_p;
  for (int k = 0; k < M.n_b; ++k) acc = fma(Sa[l * M.n_b + k], R[(int64_t)k * n_p + j], acc);
  *out = acc;
}

// <Sigma_{s,t}, X> for X in {C, G, H} with Sigma_{s,t} = -N Dinv_t on the pattern, s the
// neighbour of t eliminated after it (t + 1, or t - 1 on the second chain of a split
// time chain); X is symmetric, so the pair's slot is min(s, t) either way.
constexpr int OFF_ENTRIES_PER_WARP = 4;
template <typename R>
__global__ void __launch_bounds__(256) contract_offdiag_kernel(DevModel M, Work W, int t) {
  const int b = blockIdx.y;
  if (!W.active[b]) return;
  __shared__ double red[32];
  const int n_p = M.n_p;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const R *N = static_cast<const R *>(W.T1) + b * W.sMat;
  const R *D = static_cast<const R *>(W.Dinv) + b * W.sDinv + (int64_t)t * n_p * n_p;
  double sC = 0.0, sG = 0.0, sH = 0.0;
  const int per_block = 8 * OFF_ENTRIES_PER_WARP;
  for (int e0 = blockIdx.x * per_block; e0 < M.nnz; e0 += gridDim.x * per_block) {
    for (int q = 0; q < OFF_ENTRIES_PER_WARP; ++q) {
      const int e = e0 + warp * OFF_ENTRIES_PER_WARP + q;
      if (e >= M.nnz) break;
      const R *Ni = N + (int64_t)M.prow_of[e] * n_p;
      const R *Dj = D + (int64_t)M.pcol[e] * n_p;
      R dd = 0;
      for (int k = lane; k < n_p; k += 32) dd = fma(Ni[k], Dj[k], dd);
      const double d = -(double)warp_sum(dd);
      if (lane == 0) {
        sC = fma(d, M.vC[e], sC);
        sG = fma(d, M.vG[e], sG);
        sH = fma(d, M.vH[e], sH);
      }
    }
  }
  double *part = W.part + ((int64_t)b * NPART + blockIdx.x) * PART_W;
  sC = block_sum(sC, red);
  if (threadIdx.x == 0) part[0] = sC;
  sG = block_sum(sG, red);
  if (threadIdx.x == 0) part[1] = sG;
  sH = block_sum(sH, red);
  if (threadIdx.x == 0) part[2] = sH;
}

// dst[b*stride + slot[c]] = sum of the first nparts partial sums of component c.
struct Slots {
  int n;
  int at[PART_W];
};
__global__ void reduce_parts_kernel(Work W, int nparts, Slots slots, double *dst, int64_t dstride) {
  const int b = blockIdx.x;
  if (!W.active[b]) return;
  __shared__ double red[32];
  for (int c = 0; c < slots.n; ++c) {
    double s = 0.0;
    for (int p = threadIdx.x; p < nparts; p += blockDim.x) s += W.part[((int64_t)b * NPART + p) * PART_W + c];
    s = block_sum(s, red);
    if (threadIdx.x == 0) dst[b * dstride + slots.at[c]] = s;
  }
}
Slots consecutive(int n, int first = 0) {
  Slots s{n, {}};
  for (int c = 0; c < n; ++c) s.at[c] = first + c;
  return s;
}

// <Sigma_tt, X> on the pattern, <Sigma_{a,t}, Z^T D A_t>, and diag(Sigma_tt) output.
// Grid-stride over the pattern entries across gridDim.x blocks per point; block
// partial sums (C, G, H, A^T A, arrow) go to W.part and reduce_parts_kernel.
template <typename R>
__global__ void __launch_bounds__(256) contract_diag_kernel(DevModel M, Work W, int t, int mode, double *mv,
                                                           const int *point_out, int64_t point_base) {
  const int b = blockIdx.y;
  if (!W.active[b]) return;
  __shared__ double red[32];
  const int n_p = M.n_p;
  const int stride = gridDim.x * blockDim.x, first = blockIdx.x * blockDim.x + threadIdx.x;
  const R *S = static_cast<const R *>(W.SigC) + b * W.sMat;
  const double *lik = nullptr;
  if (mode == ASM_QC)
    lik = (M.lik == INLA_LIK_GAUSSIAN) ? M.AtA + (int64_t)t * M.nnz : W.AtAp + b * W.sAtAp + (int64_t)t * M.nnz;
  double sC = 0.0, sG = 0.0, sH = 0.0, sA = 0.0;
  for (int e = first; e < M.nnz; e += stride) {
    const double s = (double)S[(int64_t)M.prow_of[e] * n_p + M.pcol[e]];
    sC = fma(s, M.vC[e], sC);
    sG = fma(s, M.vG[e], sG);
    sH = fma(s, M.vH[e], sH);
    if (lik) sA = fma(s, lik[e], sA);
  }
  double sR = 0.0;
  if (mode == ASM_QC && M.n_b > 0) {
    const double *arw = (M.lik == INLA_LIK_GAUSSIAN) ? M.Arw + (int64_t)t * M.n_b * M.n_s
                                                     : W.Arwp + b * W.sArwp + (int64_t)t * M.n_b * M.n_s;
    const double *sa = W.SigAc + b * W.sNbNp;
    for (int e = first; e < M.n_b * M.n_s; e += stride) {
      const int l = e / M.n_s, i = e % M.n_s;
      sR = fma(sa[(int64_t)l * n_p + i], arw[e], sR);
    }
  }
  if (mode == ASM_QC && mv && point_out) {
    const int o = point_out[point_base + b];
    if (o >= 0) {
      double *dst = mv + (int64_t)o * M.n + (int64_t)t * M.n_s;
      for (int i = first; i < M.n_s; i += stride) dst[i] = (double)S[(int64_t)i * n_p + i];
    }
  }
  double *part = W.part + ((int64_t)b * NPART + blockIdx.x) * PART_W;
  sC = block_sum(sC, red);
  if (threadIdx.x == 0) part[0] = sC;
  sG = block_sum(sG, red);
  if (threadIdx.x == 0) part[1] = sG;
  sH = block_sum(sH, red);
  if (threadIdx.x == 0) part[2] = sH;
  if (mode == ASM_QC) {
    sA = block_sum(sA, red);
    if (threadIdx.x == 0) part[3] = sA;
    sR = block_sum(sR, red);
    if (threadIdx.x == 0) part[4] = sR;
  }
}

__global__ void contract_tip_kernel(DevModel M, Work W, int mode, double *mv, const int *point_out,
                                    int64_t point_base) {
  const int b = blockIdx.x;
  if (!W.active[b] || threadIdx.x != 0) return;
  const int nb = M.n_b;
  const double *Sa = W.Da + b * W.sNb2;
  double tr = 0.0, ata = 0.0;
  for (int l = 0; l < nb; ++l) tr += Sa[l * nb + l];
  if (mode == ASM_QC) {
    const double *tip = (M.lik == INLA_LIK_GAUSSIAN) ? M.Tip : W.Tipp + b * W.sNb2;
    for (int e = 0; e < nb * nb; ++e) ata += Sa[e] * tip[e];
    W.sc[b * SC_COUNT + SC_TIP_TRSIG] = tr;
    W.sc[b * SC_COUNT + SC_TIP_ATA] = ata;
    if (mv && point_out) {
      const int o = point_out[point_base + b];
      if (o >= 0)
        for (int l = 0; l < nb; ++l) mv[(int64_t)o * M.n + (int64_t)M.n_t * M.n_s + l] = Sa[l * nb + l];
    }
  }
}

// Per time block: u_t^T X v_t and u_{t+1}^T X v_t + u_t^T X v_{t+1} for X in {C, G, H};
// the tip product u_a . v_a goes to sc[tip_slot].
__global__ void __launch_bounds__(256) quadforms_kernel(DevModel M, Work W, const double *u, const double *v,
                                                       int slot0, int tip_slot) {
  const int b = blockIdx.y, t = blockIdx.x;
  if (!W.active[b]) return;
  __shared__ double red[32];
  const int n_p = M.n_p;
  const double *ut = u + b * W.sVec + (int64_t)t * n_p;
  const double *vt = v + b * W.sVec + (int64_t)t * n_p;
  const bool nxt = t < M.n_t - 1;
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int e = threadIdx.x; e < M.nnz; e += blockDim.x) {
    const int i = M.prow_of[e], j = M.pcol[e];
    const double X[3] = {M.vC[e], M.vG[e], M.vH[e]};
    const double d = ut[i] * vt[j];
    const double o = nxt ? ut[n_p + i] * vt[j] + ut[i] * vt[n_p + j] : 0.0;
    for (int c = 0; c < 3; ++c) {
      s[c] = fma(X[c], d, s[c]);
      s[3 + c] = fma(X[c], o, s[3 + c]);
    }
  }
  double *pt = W.pt + (b * (int64_t)M.n_t + t) * PT_COUNT;
  for (int c = 0; c < 6; ++c) {
    const double r = block_sum(s[c], red);
    if (threadIdx.x == 0) pt[slot0 + c] = r;
  }
  if (t == 0 && threadIdx.x == 0) {
    const int64_t tail = (int64_t)M.n_t * n_p;
    double a = 0.0;
    for (int l = 0; l < M.n_b; ++l) a += u[b * W.sVec + tail + l] * v[b * W.sVec + tail + l];
    W.sc[b * SC_COUNT + tip_slot] = a;
  }
}

__global__ void rhs_gaussian_kernel(DevModel M, Work W) {
  const int b = blockIdx.y;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M.nv) return;
  W.rhs[b * W.sVec + k] = W.prm[b].tau_y * M.Aty[k];
}

__device__ __forceinline__ double obs_eta(const DevModel &M, const double *xb, int64_t i) {
  const int t = M.obs_t[i];
  const double *xt = xb + (int64_t)t * M.n_p;
  double eta = 0.0;
  for (int s = 0; s < MAX_SPATIAL; ++s) eta = fma(M.obs_w[i * MAX_SPATIAL + s], xt[M.obs_v[i * MAX_SPATIAL + s]], eta);
  const double *xa = xb + (int64_t)M.n_t * M.n_p;
  for (int l = 0; l < M.n_b; ++l) eta = fma(M.obs_z[i * M.n_b + l], xa[l], eta);
  return eta;
}

// kind 0: sum (y - eta)^2;  kind 1: sum y eta - E exp(eta)   (partial sums per block)
__global__ void __launch_bounds__(256) obs_reduce_kernel(DevModel M, Work W, int kind) {
  const int b = blockIdx.y;
  if (!W.active[b]) return;
  __shared__ double red[32];
  const double *xb = W.x + b * W.sVec;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M.m; i += (int64_t)gridDim.x * blockDim.x) {
    const double eta = obs_eta(M, xb, i);
    if (kind == 0) {
      const double r = M.y[i] - eta;
      s = fma(r, r, s);
    } else {
      s += M.y[i] * eta - glm_terms(M.lik, M.E[i], M.y[i], M.nb_size, eta).b;
    }
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) W.part[((int64_t)b * NPART + blockIdx.x) * PART_W] = s;
}

// Q_s(theta) = tau^2 (kappa^4 C + 2 kappa^2 G + G C^-1 G) depends on theta_2 (the
// range) through kappa alone and on theta_3 only through the factor tau^2, so
// points with the same theta_2 have Q_s equal up to a positive factor: a
// central-difference stencil has three distinct ranges among its nine points, a
// 25-point central composite design five.  Within each aligned chunk of
// QS_SHARE_CHUNK points of a wave, the first point with a given theta_2 is the
// representative; only representatives run the inversion.
constexpr int QS_SHARE_CHUNK = 256;
__global__ void qs_share_setup_kernel(Work W) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= W.P) return;
  const double k = W.theta[4 * b + 1];
  int r = b;
  for (int c = (b / QS_SHARE_CHUNK) * QS_SHARE_CHUNK; c < b; ++c)
    if (W.theta[4 * c + 1] == k) {   // a NaN range matches nothing and stays its own representative
      r = c;
      break;
    }
  W.qsrep[b] = r;
  W.active[b] = (r == b) ? 1 : 0;
}

// For a point that shares the representative r's Q_s with s = tau_b^2 / tau_r^2:
// log|Q_s,b| = log|Q_s,r| + n_s log s and tr(Q_s,b^-1 X) = tr(Q_s,r^-1 X) / s.
__global__ void qs_share_kernel(DevModel M, Work W) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= W.P) return;
  const int r = W.qsrep[b];
  if (r == b) return;
  const double s = W.prm[b].aH / W.prm[r].aH;   // aH = tau^2
  double *sb = W.sc + b * SC_COUNT;
  const double *sr = W.sc + r * SC_COUNT;
  sb[SC_LOGDET_QS] = sr[SC_LOGDET_QS] + M.n_s * log(s);
  sb[SC_TR_QSI_C] = sr[SC_TR_QSI_C] / s;
  sb[SC_TR_QSI_G] = sr[SC_TR_QSI_G] / s;
  sb[SC_TR_QSI_H] = sr[SC_TR_QSI_H] / s;
  if (W.status[r] != INLA_OK) W.status[b] = W.status[r];
}

// tr(Q_s^-1 X) for X in {C, G, H}, Q_s^-1 in T1.
__global__ void qs_traces_kernel(DevModel M, Work W) {
  const int b = blockIdx.x;
  if (!W.active[b]) return;
  __shared__ double red[32];
  const double *S = W.QsI + b * W.sMat;
  double sC = 0.0, sG = 0.0, sH = 0.0;
  for (int e = threadIdx.x; e < M.nnz; e += blockDim.x) {
    const double s = S[(int64_t)M.prow_of[e] * M.n_p + M.pcol[e]];
    sC = fma(s, M.vC[e], sC);
    sG = fma(s, M.vG[e], sG);
    sH = fma(s, M.vH[e], sH);
  }
  double *sc = W.sc + b * SC_COUNT;
  sC = block_sum(sC, red);
  if (threadIdx.x == 0) sc[SC_TR_QSI_C] = sC;
  sG = block_sum(sG, red);
  if (threadIdx.x == 0) sc[SC_TR_QSI_G] = sG;
  sH = block_sum(sH, red);
  if (threadIdx.x == 0) sc[SC_TR_QSI_H] = sH;
}

// ------------------------------------------------------------------ f and grad f

// d/dtheta_j of (q * a_X): dq_j * a_X + q * da_X_j (see the gradient formulas).
__device__ __forceinline__ void dcoef(const PointParams &p, int j, double q, double dq, double out[3]) {
  const double a[3] = {p.aC, p.aG, p.aH};
  if (j == 1) { out[0] = -2.0 * q * p.aC; out[1] = 0.0; out[2] = 2.0 * q * p.aH; return; }
  if (j == 2) { for (int c = 0; c < 3; ++c) out[c] = -2.0 * q * a[c]; return; }
  if (j == 3) { for (int c = 0; c < 3; ++c) out[c] = dq * a[c]; return; }
  out[0] = out[1] = out[2] = 0.0;
}

// sum over t of d(q a_X)/dtheta_j against diag slots and off-diagonal slots (x2 when offmul = 2).
__device__ double dsum(const DevModel &M, const PointParams &p, const double *pt, int j, int sd, int so,
                       double offmul) {
  double s = 0.0;
  for (int t = 0; t < M.n_t; ++t) {
    const double *q = pt + (int64_t)t * PT_COUNT;
    double c[3];
    dcoef(p, j, q_tt(p, t, M.n_t), dq_tt(p, t, M.n_t), c);
    for (int k = 0; k < 3; ++k) s += c[k] * q[sd + k];
    if (t < M.n_t - 1) {
      dcoef(p, j, p.q_off, p.dq_off, c);
      for (int k = 0; k < 3; ++k) s += offmul * c[k] * q[so + k];
    }
  }
  return s;
}

__global__ void finalize_kernel(DevModel M, Work W, int grad_mode, int prior_mode, int64_t point_base,
                                double *f_all, double *grad_all, int *status_all, int *iters_all) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= W.P) return;
  const PointParams &p = W.prm[b];
  const double *sc = W.sc + b * SC_COUNT;
  const double *pt = W.pt + (int64_t)b * M.n_t * PT_COUNT;
  const int n_t = M.n_t, n_s = M.n_s, n_b = M.n_b;
  const double m = (double)M.m;
  const bool gauss = M.lik == INLA_LIK_GAUSSIAN;
  const double rho = p.rho;
  double logdetQ;
  if (prior_mode == INLA_PRIOR_KRONECKER)
    logdetQ = n_s * (-(n_t - 1) * log1p(-rho * rho)) + n_t * sc[SC_LOGDET_QS] + n_b * log(p.tau_b);
  else
    logdetQ = sc[SC_LOGDET_Q];
  double xQx = p.tau_b * sc[SC_TIP_XX];
  for (int t = 0; t < n_t; ++t) {
    const double *q = pt + (int64_t)t * PT_COUNT;
    const double c = q_tt(p, t, n_t);
    xQx += c * (p.aC * q[PT_XD_C] + p.aG * q[PT_XD_G] + p.aH * q[PT_XD_H]);
    if (t < n_t - 1) xQx += p.q_off * (p.aC * q[PT_XO_C] + p.aG * q[PT_XO_G] + p.aH * q[PT_XO_H]);
  }
  double f = -p.logprior - 0.5 * logdetQ + 0.5 * xQx + 0.5 * sc[SC_LOGDET_QC];
  if (gauss) f += -0.5 * m * p.theta[0] + 0.5 * m * log(2.0 * M_PI) + 0.5 * p.tau_y * sc[SC_RES2];
  else f -= sc[SC_LOGLIK] + M.consts[2] - M.consts[1];
  int st = W.status[b];
  const int64_t g = point_base + b;
  if (st != INLA_OK) f = INFINITY;
  f_all[g] = f;
  status_all[g] = st;
  iters_all[g] = W.iters[b];
  if (grad_mode != INLA_GRAD_ADJOINT || !grad_all) return;
  // tr(Sigma_c (Q - tau_b I_tip)) = n - tr(Sigma_c A^T D A) - tau_b tr(Sigma_a)  (Sigma_c Q_c = I).
  // With dQ/dlog(sigma) = -2 (Q - tau_b I_tip) and dQ_s/dlog(range) = 2 Q_s - 4 aC C - 2 aG G this
  // removes the large, nearly cancelling Q_s and H parts of the prior and posterior traces.
  double liktr = sc[SC_TIP_ATA];
  for (int t = 0; t < n_t; ++t) liktr += pt[(int64_t)t * PT_COUNT + PT_FD_ATA] + 2.0 * pt[(int64_t)t * PT_COUNT + PT_FA_ATA];
  liktr *= gauss ? p.tau_y : 1.0;
  const double trQcQ = (double)M.n - liktr - p.tau_b * sc[SC_TIP_TRSIG];
  auto cg_part = [&](int sd, int so) {   // sum_t of q (4 aC <S, C> + 2 aG <S, G>) over diagonal and 2x off blocks
    double v = 0.0;
    for (int t = 0; t < n_t; ++t) {
      const double *q = pt + (int64_t)t * PT_COUNT;
      v += q_tt(p, t, n_t) * (4.0 * p.aC * q[sd + 0] + 2.0 * p.aG * q[sd + 1]);
      if (t < n_t - 1) v += 2.0 * p.q_off * (4.0 * p.aC * q[so + 0] + 2.0 * p.aG * q[so + 1]);
    }
    return v;
  };
  double gr[4];
  for (int j = 0; j < 4; ++j) {
    double trQ;
    if (prior_mode == INLA_PRIOR_KRONECKER) {
      if (j == 0) trQ = gauss ? 0.0 : (double)n_b;
      else if (j == 1) trQ = n_t * (2.0 * n_s - 4.0 * p.aC * sc[SC_TR_QSI_C] - 2.0 * p.aG * sc[SC_TR_QSI_G]);
      else if (j == 2) trQ = -2.0 * n_t * n_s;
      else trQ = n_s * rho * (1.0 - rho) * 2.0 * (n_t - 1) * rho / (1.0 - rho * rho);
    } else {
      if (j == 1) trQ = 2.0 * n_t * n_s - cg_part(PT_QD_C, PT_QO_C);
      else if (j == 2) trQ = -2.0 * n_t * n_s;
      else trQ = dsum(M, p, pt, j, PT_QD_C, PT_QO_C, 2.0) + ((j == 0 && !gauss) ? (double)n_b : 0.0);
    }
    double trQc;
    if (j == 1) trQc = 2.0 * trQcQ - cg_part(PT_FD_C, PT_FO_C);
    else if (j == 2) trQc = -2.0 * trQcQ;
    else trQc = dsum(M, p, pt, j, PT_FD_C, PT_FO_C, 2.0);
    double xdx = dsum(M, p, pt, j, PT_XD_C, PT_XO_C, 1.0);
    double v = -p.dlogprior[j] - 0.5 * trQ + 0.5 * xdx + 0.5 * trQc;
    if (gauss) {
      if (j == 0) {
        double ata = sc[SC_TIP_ATA];
        for (int t = 0; t < n_t; ++t) ata += pt[(int64_t)t * PT_COUNT + PT_FD_ATA] + 2.0 * pt[(int64_t)t * PT_COUNT + PT_FA_ATA];
        v += 0.5 * p.tau_y * ata - 0.5 * m + 0.5 * p.tau_y * sc[SC_RES2];
      }
    } else {
      double ldx = dsum(M, p, pt, j, PT_LD_C, PT_LO_C, 1.0);
      if (j == 0) {
        v += 0.5 * p.tau_b * sc[SC_TIP_XX] + 0.5 * p.tau_b * sc[SC_TIP_TRSIG];
        ldx += p.tau_b * sc[SC_TIP_LX];
      }
      v -= ldx;
    }
    gr[j] = v;
  }
  for (int j = 0; j < 4; ++j) grad_all[g * 4 + j] = (st != INLA_OK) ? NAN : gr[j];
}

__global__ void copy_mode_kernel(DevModel M, Work W, double *x_out, const int *point_out, int64_t point_base) {
  const int b = blockIdx.y;
  const int o = point_out[point_base + b];
  if (o < 0) return;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M.n) return;
  const int64_t Ns = (int64_t)M.n_t * M.n_s;
  const int64_t src = (k < Ns) ? (k / M.n_s) * M.n_p + (k % M.n_s) : (int64_t)M.n_t * M.n_p + (k - Ns);
  const double v = W.x[b * W.sVec + src];
  x_out[(int64_t)o * M.n + k] = (W.status[b] == INLA_OK) ? v : NAN;
}

// Difference stencils per centre: central (per = 9) centre, +e_0, -e_0, +e_1, ...;
// forward (per = 5) centre, +e_0, +e_1, +e_2, +e_3 (steps eps).
__global__ void fd_points_kernel(int B, int per, const double *theta, double eps, double *pts) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * per) return;
  const int c = idx / per, k = idx % per;
  for (int j = 0; j < 4; ++j) {
    double v = theta[c * 4 + j];
    if (per == 9 && k > 0 && (k - 1) / 2 == j) v += ((k - 1) % 2 == 0) ? eps : -eps;
    if (per == 5 && k == j + 1) v += eps;
    pts[idx * 4 + j] = v;
  }
}

__global__ void outputs_kernel(int B, int per, double eps, int d, const double *f_all, const double *grad_all,
                               const int *status_all, const int *iters_all, double *f, double *grad, int *status,
                               int *iters) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= B) return;
  int st = INLA_OK;
  for (int k = 0; k < per; ++k)
    if (status_all[c * per + k] != INLA_OK && st == INLA_OK) st = status_all[c * per + k];
  status[c] = st;
  f[c] = (st == INLA_OK) ? f_all[c * per] : INFINITY;
  if (iters) iters[c] = iters_all[c * per];
  if (!grad) return;
  for (int j = 0; j < d; ++j) {
    double g;
    if (per == 1) g = grad_all ? grad_all[c * d + j] : NAN;
    else if (per == 9) g = (f_all[c * per + 1 + 2 * j] - f_all[c * per + 2 + 2 * j]) / (2.0 * eps);
    else g = (f_all[c * per + 1 + j] - f_all[c * per]) / eps;
    grad[c * d + j] = (st == INLA_OK) ? g : NAN;
  }
}

// ------------------------------------------------------------------ Poisson pieces

__global__ void poisson_eta_kernel(DevModel M, Work W, const double *x) {
  const int b = blockIdx.y;
  if (!W.active[b]) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M.m) return;
  const double eta = obs_eta(M, x + b * W.sVec, i);
  W.eta[b * W.sM + i] = eta;
  W.mu[b * W.sM + i] = glm_terms(M.lik, M.E[i], M.y[i], M.nb_size, eta).weight;
}

__device__ __forceinline__ double obs_r(const DevModel &M, const double *r, int64_t sR, bool r_newton,
                                        const double *mu, int64_t sMu, const double *eta, int b, int64_t i) {
  if (r_newton) {   // Newton right-hand side per observation: y - b'(eta) + b''(eta) eta
    const double e = eta[b * sMu + i];
    return M.y[i] - glm_terms(M.lik, M.E[i], M.y[i], M.nb_size, e).mean + mu[b * sMu + i] * e;
  }
  return r[b * sR + i];
}

// Spatial pattern part of A_t^T diag(mu) A_t.
__global__ void obs_assemble_pattern_kernel(DevModel M, const int *active, const double *mu, int64_t sMu,
                                            double *AtA, int64_t sAtA) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)M.n_t * M.nnz) return;
  double s = 0.0;
  for (int64_t c = M.sp_ptr[k]; c < M.sp_ptr[k + 1]; ++c) {
    const int i = M.sp_obs[c];
    s = fma(mu ? mu[b * sMu + i] : 1.0, M.sp_w[c], s);
  }
  AtA[b * sAtA + k] = s;
}

// Arrow part Z^T diag(mu) A_t (per (t, vertex)) and the spatial part of A^T r.
__global__ void obs_assemble_vertex_kernel(DevModel M, const int *active, const double *mu, int64_t sMu,
                                           const double *r, int64_t sR, int r_newton, const double *eta,
                                           double *Arw, int64_t sArw, double *rhs, int64_t sRhs) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)M.n_t * M.n_s) return;
  const int t = (int)(k / M.n_s), v = (int)(k % M.n_s);
  double arw[MAX_NB];
  for (int l = 0; l < M.n_b; ++l) arw[l] = 0.0;
  double sr = 0.0;
  for (int64_t c = M.vt_ptr[k]; c < M.vt_ptr[k + 1]; ++c) {
    const int i = M.vt_obs[c];
    const double w = M.vt_w[c];
    if (Arw) {
      const double u = (mu ? mu[b * sMu + i] : 1.0) * w;
      for (int l = 0; l < M.n_b; ++l) arw[l] = fma(u, M.obs_z[(int64_t)i * M.n_b + l], arw[l]);
    }
    if (rhs) sr = fma(w, obs_r(M, r, sR, r_newton, mu, sMu, eta, b, i), sr);
  }
  if (Arw)
    for (int l = 0; l < M.n_b; ++l) Arw[b * sArw + ((int64_t)t * M.n_b + l) * M.n_s + v] = arw[l];
  if (rhs) rhs[b * sRhs + (int64_t)t * M.n_p + v] = sr;
}

// Per time block partial sums of Z^T diag(mu) Z and Z^T r (warp-split components).
__global__ void __launch_bounds__(256) obs_assemble_tip_kernel(DevModel M, const int *active, const double *mu,
                                                              int64_t sMu, const double *r, int64_t sR, int r_newton,
                                                              const double *eta, int want_tip, int want_rhs,
                                                              double *tippart) {
  const int b = blockIdx.y, t = blockIdx.x;
  if (active && !active[b]) return;
  const int nb = M.n_b;
  const int ncomp = nb * nb + nb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double *out = tippart + ((int64_t)b * M.n_t + t) * ncomp;
  for (int c = warp; c < ncomp; c += 8) {
    const bool tipc = c < nb * nb;
    if ((tipc && !want_tip) || (!tipc && !want_rhs)) {
      if (lane == 0) out[c] = 0.0;
      continue;
    }
    const int l1 = tipc ? c / nb : c - nb * nb, l2 = tipc ? c % nb : 0;
    double s = 0.0;
    for (int64_t i = M.obs_ptr[t] + lane; i < M.obs_ptr[t + 1]; i += 32) {
      const double *z = M.obs_z + i * nb;
      if (tipc) s = fma((mu ? mu[b * sMu + i] : 1.0) * z[l1], z[l2], s);
      else s = fma(z[l1], obs_r(M, r, sR, r_newton, mu, sMu, eta, b, i), s);
    }
    s = warp_sum(s);
    if (lane == 0) out[c] = s;
  }
}

__global__ void obs_assemble_tip_sum_kernel(DevModel M, const int *active, const double *tippart, double *Tip,
                                            int64_t sTip, double *rhs, int64_t sRhs) {
  const int b = blockIdx.y, c = blockIdx.x;
  if (active && !active[b]) return;
  const int nb = M.n_b, ncomp = nb * nb + nb;
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int t = 0; t < M.n_t; ++t) s += tippart[((int64_t)b * M.n_t + t) * ncomp + c];
  if (c < nb * nb) {
    if (Tip) Tip[b * sTip + c] = s;
  } else if (rhs) {
    rhs[b * sRhs + (int64_t)M.n_t * M.n_p + (c - nb * nb)] = s;
  }
}

// ||x - xprev||_2 < tol ends the iteration of a point; xprev <- x.
__global__ void poisson_step_kernel(DevModel M, Work W, double tol, int iter_host, int max_iter,
                                    const int *iter_dev) {
  const int b = blockIdx.x;
  if (!W.active[b]) return;
  const int iter = iter_dev ? *iter_dev + 1 : iter_host;   // the graph path counts on the device
  __shared__ double red[32];
  double *x = W.x + b * W.sVec;
  double *xp = W.xprev + b * W.sVec;
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < M.nv; k += blockDim.x) {
    const double d = x[k] - xp[k];
    s = fma(d, d, s);
  }
  s = block_sum(s, red);
  __syncthreads();
  for (int64_t k = threadIdx.x; k < M.nv; k += blockDim.x) xp[k] = x[k];
  if (threadIdx.x == 0) {
    W.sc[b * SC_COUNT + SC_STEP2] = s;
    const bool bad = !(s < INFINITY);
    if (sqrt(s) < tol) {
      W.active[b] = 0;
      W.iters[b] = iter;
    } else if (iter >= max_iter || bad) {
      W.active[b] = 0;
      W.iters[b] = iter;
      W.status[b] = INLA_ERR_NO_CONVERGENCE;
    } else {
      *W.any_active = 1;
    }
  }
}

// a_i^T Sigma_c a_i for the observations of time block t (pattern entries only).
template <typename R>
__global__ void poisson_qobs_kernel(DevModel M, Work W, int t) {
  const int b = blockIdx.y;
  if (!W.active[b]) return;
  const int64_t i = M.obs_ptr[t] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M.obs_ptr[t + 1]) return;
  const int n_p = M.n_p, nb = M.n_b;
  const R *S = static_cast<const R *>(W.SigC) + b * W.sMat;
  const double *Sa = W.SigAc + b * W.sNbNp;
  const double *St = W.Da + b * W.sNb2;
  const double *w = M.obs_w + i * MAX_SPATIAL;
  const int *v = M.obs_v + i * MAX_SPATIAL;
  const double *z = M.obs_z + i * nb;
  double q = 0.0;
  for (int s1 = 0; s1 < MAX_SPATIAL; ++s1)
    for (int s2 = 0; s2 < MAX_SPATIAL; ++s2) q += w[s1] * w[s2] * (double)S[(int64_t)v[s1] * n_p + v[s2]];
  for (int s1 = 0; s1 < MAX_SPATIAL; ++s1)
    for (int l = 0; l < nb; ++l) q += 2.0 * w[s1] * z[l] * Sa[(int64_t)l * n_p + v[s1]];
  for (int l = 0; l < nb; ++l)
    for (int l2 = 0; l2 < nb; ++l2) q += z[l] * z[l2] * St[l * nb + l2];
  W.qobs[b * W.sM + i] = q;
}

__global__ void poisson_wobs_kernel(DevModel M, Work W) {
  const int b = blockIdx.y;
  if (!W.active[b]) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M.m) return;
  W.wobs[b * W.sM + i] = 0.5 * W.qobs[b * W.sM + i] * glm_terms(M.lik, M.E[i], M.y[i], M.nb_size, W.eta[b * W.sM + i]).third;
}

// r = b - Q_c x in FP64 from the sparse blocks (iterative refinement of the
// mode in the mixed-precision path): per time block
//   (Q_c x)_t = q_tt Q_s x_t + q_off Q_s (x_{t-1} + x_{t+1}) + L_t x_t + Arw_t^T x_a,
//   (Q_c x)_a = (tau_b I + L_a) x_a + sum_t Arw_t x_t.
__global__ void qc_residual_kernel(DevModel M, Work W, const double *x, const double *bvec, double *r) {
  const int b = blockIdx.z;
  if (!W.active[b]) return;
  const int t = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_p = M.n_p, n_s = M.n_s, n_b = M.n_b, n_t = M.n_t;
  if (i >= n_p) return;
  const int64_t o = b * W.sVec + (int64_t)t * n_p + i;
  if (i >= n_s) { r[o] = 0.0; return; }
  const PointParams &p = W.prm[b];
  const double *xb = x + b * W.sVec;
  const double *qs = W.qs + b * W.sNnz;
  const double *lik = (M.lik == INLA_LIK_GAUSSIAN) ? M.AtA + (int64_t)t * M.nnz
                                                   : W.AtAp + b * W.sAtAp + (int64_t)t * M.nnz;
  const double ls = (M.lik == INLA_LIK_GAUSSIAN) ? p.tau_y : 1.0;
  const double c = q_tt(p, t, n_t);
  const double *xt = xb + (int64_t)t * n_p;
  double y = 0.0;
  for (int e = M.prow[i]; e < M.prow[i + 1]; ++e) {
    const int k = M.pcol[e];
    double xn = 0.0;
    if (t > 0) xn += xt[k - n_p];
    if (t < n_t - 1) xn += xt[k + n_p];
    y += (c * qs[e] + ls * lik[e]) * xt[k] + p.q_off * qs[e] * xn;
  }
  const double *xa = xb + (int64_t)n_t * n_p;
  for (int l = 0; l < n_b; ++l) {
    const int64_t ka = ((int64_t)t * n_b + l) * n_s + i;
    const double a = (M.lik == INLA_LIK_GAUSSIAN) ? p.tau_y * M.Arw[ka] : W.Arwp[b * W.sArwp + ka];
    y += a * xa[l];
  }
  r[o] = (bvec ? bvec[o] : 0.0) - y;
}

// Tail rows of the residual: one block per point.
__global__ void qc_residual_tail_kernel(DevModel M, Work W, const double *x, const double *bvec, double *r) {
  const int b = blockIdx.x;
  if (!W.active[b]) return;
  __shared__ double red[32];
  const int n_p = M.n_p, n_s = M.n_s, n_b = M.n_b, n_t = M.n_t;
  const PointParams &p = W.prm[b];
  const double *xb = x + b * W.sVec;
  const double *xa = xb + (int64_t)n_t * n_p;
  const bool gauss = M.lik == INLA_LIK_GAUSSIAN;
  for (int l = 0; l < n_b; ++l) {
    double s = 0.0;
    for (int64_t k = threadIdx.x; k < (int64_t)n_t * n_s; k += blockDim.x) {
      const int t = (int)(k / n_s), i = (int)(k % n_s);
      const int64_t ka = ((int64_t)t * n_b + l) * n_s + i;
      const double a = gauss ? p.tau_y * M.Arw[ka] : W.Arwp[b * W.sArwp + ka];
      s = fma(a, xb[(int64_t)t * n_p + i], s);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
      for (int l2 = 0; l2 < n_b; ++l2) {
        const double tip = gauss ? p.tau_y * M.Tip[l * n_b + l2] : W.Tipp[b * W.sNb2 + l * n_b + l2];
        s += ((l == l2) ? p.tau_b : 0.0) * xa[l2] + tip * xa[l2];
      }
      const int64_t o = b * W.sVec + (int64_t)n_t * n_p + l;
      r[o] = (bvec ? bvec[o] : 0.0) - s;
    }
  }
}

__global__ void axpy_kernel(DevModel M, Work W, double *x, const double *d) {
  const int b = blockIdx.y;
  if (!W.active[b]) return;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < M.nv) x[b * W.sVec + k] += d[b * W.sVec + k];
}

__global__ void zero_kernel(double *p, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) p[k] = 0.0;
}

inline unsigned blocks(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

// ------------------------------------------------------------------ launch wrappers

void k_params(Launch &L, const DevModel &M, const Work &W) {
  params_kernel<<<blocks(W.P, 64), 64, 0, L.st>>>(M, W);
  L.tick();
}
void k_qs_values(Launch &L, const DevModel &M, const Work &W) {
  qs_values_kernel<<<dim3(blocks(M.nnz, 256), W.P), 256, 0, L.st>>>(M, W);
  L.tick();
}
void k_set_active(Launch &L, const Work &W, int mask) {
  set_active_kernel<<<blocks(W.P, 64), 64, 0, L.st>>>(W, mask);
  L.tick();
}
void k_init_step0(Launch &L, const DevModel &M, const Work &W, int mode, int t0, bool tip_init) {
  init_step0_kernel<<<dim3(blocks(M.n_p, 128), M.n_b + 1, W.P), 128, 0, L.st>>>(M, W, mode, t0, tip_init ? 1 : 0);
  L.tick();
}
template <typename R>
void k_assemble_diag(Launch &L, const DevModel &M, const Work &W, int t, int mode, R *dst, int64_t sdst,
                     bool schur) {
  assemble_diag_kernel<R><<<dim3(M.n_p, W.P), 256, sizeof(double) * M.n_p, L.st>>>(M, W, t, mode, dst, sdst,
                                                                                   schur ? 1 : 0);
  L.tick();
}
template <typename R>
void k_sparse_right(Launch &L, const DevModel &M, const Work &W, const R *X, int64_t sX, R *out, int64_t sOut,
                    bool coef_qoff, const double *SigA, const double *Rt_t, bool lower_band) {
  if (M.pmax <= SR_PMAX) {
    sparse_right_tiled_kernel<R><<<dim3(blocks(M.n_p, SR_COLS), blocks(M.n_p, SR_ROWS), W.P), 256, 0, L.st>>>(
        M, W, X, sX, out, sOut, coef_qoff ? 1 : 0, SigA, Rt_t, lower_band ? 1 : 0);
    L.tick();
    return;
  }
  sparse_right_kernel<R><<<dim3(blocks(M.n_p, 128), M.n_p, W.P), 128, 0, L.st>>>(M, W, X, sX, out, sOut,
                                                                               coef_qoff ? 1 : 0, SigA, Rt_t,
                                                                               lower_band ? 1 : 0);
  L.tick();
}
template <typename R>
void k_sparse_left(Launch &L, const DevModel &M, const Work &W, const R *X, int64_t sX, R *out, int64_t sOut,
                   bool with_X, const double *Rt_t, const double *Ymat) {
  sparse_left_kernel<R><<<dim3(M.n_p, W.P), 256, 0, L.st>>>(M, W, X, sX, out, sOut, with_X ? 1 : 0, Rt_t, Ymat);
  L.tick();
}
template <typename R>
void k_dinv_apply(Launch &L, const DevModel &M, const Work &W, const R *Dinv_t, int nvec, const double *vecs,
                  int64_t sVecs, double *out, int64_t sOut, double scale) {
  if (nvec <= 0) return;
  if (nvec == 1)
    dinv_gemv_kernel<R><<<dim3(blocks(M.n_p, GV_ROWS), W.P), 256, sizeof(R) * M.n_p, L.st>>>(M, W, Dinv_t, vecs,
                                                                                           sVecs, out, sOut, scale);
  else
    dinv_apply_kernel<R, DA_MAXV><<<dim3(blocks(M.n_p, DA_ROWS), W.P), 256, 0, L.st>>>(M, W, Dinv_t, nvec, vecs,
                                                                                     sVecs, out, sOut, scale);
  L.tick();
}
void k_arrow_update(Launch &L, const DevModel &M, const Work &W, int t, int mode) {
  if (M.n_b == 0) return;
  arrow_update_kernel<<<dim3(blocks(M.n_p, 128), M.n_b, W.P), 128, 0, L.st>>>(M, W, t, mode);
  L.tick();
}
void k_arrow_dots(Launch &L, const DevModel &M, const Work &W, int tprev) {
  if (M.n_b == 0) return;
  arrow_dots_kernel<<<dim3(M.n_b * M.n_b, W.P), 256, 0, L.st>>>(M, W, tprev);
  L.tick();
}
void k_tip(Launch &L, const DevModel &M, const Work &W, int ld_slot) {
  if (M.n_b == 0) return;
  tip_kernel<<<blocks(W.P, 32), 32, 0, L.st>>>(M, W, ld_slot);
  L.tick();
}
void k_fwd_update(Launch &L, const DevModel &M, const Work &W, int t, int nbr, double *z) {
  const int nblk = (int)blocks(M.n_p, 128);
  fwd_update_kernel<<<dim3(nblk + (M.n_b > 0 ? 1 : 0), W.P), 128, 0, L.st>>>(M, W, t, nbr, z);
  L.tick();
}
void k_tip_solve(Launch &L, const DevModel &M, const Work &W, const double *z, double *x) {
  if (M.n_b == 0) return;
  tip_solve_kernel<<<W.P, 32, 0, L.st>>>(M, W, z, x);
  L.tick();
}
void k_bwd_rhs(Launch &L, const DevModel &M, const Work &W, int t, int nbr, const double *z, const double *x) {
  bwd_rhs_kernel<<<dim3(blocks(M.n_p, 128), W.P), 128, 0, L.st>>>(M, W, t, nbr, z, x);
  L.tick();
}
template <typename R>
void k_add_into(Launch &L, int P, R *dst, const R *src, int64_t stride, int64_t count, const int *active) {
  const int nb = (int)std::min<int64_t>(blocks(count, 256), 1024);
  add_into_kernel<R><<<dim3(nb, P), 256, 0, L.st>>>(dst, src, stride, count, active);
  L.tick();
}
template void k_add_into<float>(Launch &, int, float *, const float *, int64_t, int64_t, const int *);
template void k_add_into<double>(Launch &, int, double *, const double *, int64_t, int64_t, const int *);
void k_join_tip(Launch &L, const DevModel &M, const Work &W, const double *Da1, const double *sc1, int ld_slot) {
  join_tip_kernel<<<W.P, 64, 0, L.st>>>(M, W, Da1, sc1, ld_slot);
  L.tick();
}
void k_join_rhs(Launch &L, const DevModel &M, const Work &W, int k, double *z, const double *z1, const double *rhs) {
  join_rhs_kernel<<<dim3(blocks(M.n_p + M.n_b, 128), W.P), 128, 0, L.st>>>(M, W, k, z, z1, rhs);
  L.tick();
}
void k_selinv_Y(Launch &L, const DevModel &M, const Work &W, int t, bool has_next) {
  if (M.n_b == 0) return;
  selinv_Y_kernel<<<dim3(blocks(M.n_p, 128), M.n_b, W.P), 128, 0, L.st>>>(M, W, t, has_next ? 1 : 0);
  L.tick();
}
template <typename R>
void k_contract_offdiag(Launch &L, const DevModel &M, const Work &W, int t, int pair, int slot0) {
  int nparts = (int)blocks(M.nnz, 8 * OFF_ENTRIES_PER_WARP);
  if (nparts > NPART) nparts = NPART;
  contract_offdiag_kernel<R><<<dim3(nparts, W.P), 256, 0, L.st>>>(M, W, t);
  L.tick();
  reduce_parts_kernel<<<W.P, 256, 0, L.st>>>(W, nparts, consecutive(3, slot0), W.pt + (int64_t)pair * PT_COUNT,
                                            (int64_t)M.n_t * PT_COUNT);
  L.tick();
}
template <typename R>
void k_contract_diag(Launch &L, const DevModel &M, const Work &W, int t, int mode, double *marg_var,
                     const int *point_out, int64_t point_base, int slot0) {
  int nparts = (int)blocks(M.nnz, 1024);
  if (nparts > 64) nparts = 64;
  contract_diag_kernel<R><<<dim3(nparts, W.P), 256, 0, L.st>>>(M, W, t, mode, marg_var, point_out, point_base);
  L.tick();
  Slots sl = consecutive(3, slot0);
  if (mode == ASM_QC) {
    sl.n = 5;
    sl.at[3] = PT_FD_ATA;
    sl.at[4] = PT_FA_ATA;
  }
  reduce_parts_kernel<<<W.P, 256, 0, L.st>>>(W, nparts, sl, W.pt + (int64_t)t * PT_COUNT, (int64_t)M.n_t * PT_COUNT);
  L.tick();
}
void k_contract_tip(Launch &L, const DevModel &M, const Work &W, int mode, double *marg_var, const int *point_out,
                    int64_t point_base) {
  contract_tip_kernel<<<W.P, 32, 0, L.st>>>(M, W, mode, marg_var, point_out, point_base);
  L.tick();
}
void k_quadforms(Launch &L, const DevModel &M, const Work &W, const double *u, const double *v, int slot0,
                 int tip_slot) {
  quadforms_kernel<<<dim3(M.n_t, W.P), 256, 0, L.st>>>(M, W, u, v, slot0, tip_slot);
  L.tick();
}
void k_rhs_gaussian(Launch &L, const DevModel &M, const Work &W) {
  rhs_gaussian_kernel<<<dim3(blocks(M.nv, 256), W.P), 256, 0, L.st>>>(M, W);
  L.tick();
}
void k_obs_reduce(Launch &L, const DevModel &M, const Work &W, int kind) {
  int nparts = (int)blocks(M.m, 256);
  if (nparts > NPART) nparts = NPART;
  obs_reduce_kernel<<<dim3(nparts, W.P), 256, 0, L.st>>>(M, W, kind);
  L.tick();
  reduce_parts_kernel<<<W.P, 256, 0, L.st>>>(W, nparts, consecutive(1), W.sc + (kind == 0 ? SC_RES2 : SC_LOGLIK),
                                            SC_COUNT);
  L.tick();
}
void k_qs_share_setup(Launch &L, const Work &W) {
  qs_share_setup_kernel<<<blocks(W.P, 64), 64, 0, L.st>>>(W);
  L.tick();
}
void k_qs_share(Launch &L, const DevModel &M, const Work &W) {
  qs_share_kernel<<<blocks(W.P, 64), 64, 0, L.st>>>(M, W);
  L.tick();
}
void k_qs_traces(Launch &L, const DevModel &M, const Work &W) {
  qs_traces_kernel<<<W.P, 256, 0, L.st>>>(M, W);
  L.tick();
}
void k_finalize(Launch &L, const DevModel &M, const Work &W, int grad_mode, int prior_mode, int64_t point_base,
                double *f_all, double *grad_all, int *status_all, int *iters_all) {
  finalize_kernel<<<blocks(W.P, 64), 64, 0, L.st>>>(M, W, grad_mode, prior_mode, point_base, f_all, grad_all,
                                                    status_all, iters_all);
  L.tick();
}
void k_copy_mode(Launch &L, const DevModel &M, const Work &W, double *x_out, const int *point_out,
                 int64_t point_base) {
  copy_mode_kernel<<<dim3(blocks(M.n, 256), W.P), 256, 0, L.st>>>(M, W, x_out, point_out, point_base);
  L.tick();
}
void k_fd_points(Launch &L, int B, int per, const double *theta, double eps, double *pts) {
  fd_points_kernel<<<blocks(B * per, 64), 64, 0, L.st>>>(B, per, theta, eps, pts);
  L.tick();
}
void k_outputs(Launch &L, int B, int per, double eps, int d, const double *f_all, const double *grad_all,
               const int *status_all, const int *iters_all, double *f, double *grad, int *status, int *iters) {
  outputs_kernel<<<blocks(B, 64), 64, 0, L.st>>>(B, per, eps, d, f_all, grad_all, status_all, iters_all, f, grad,
                                                 status, iters);
  L.tick();
}
void k_poisson_eta(Launch &L, const DevModel &M, const Work &W, const double *x) {
  poisson_eta_kernel<<<dim3(blocks(M.m, 256), W.P), 256, 0, L.st>>>(M, W, x);
  L.tick();
}
void k_obs_assemble(Launch &L, const DevModel &M, int P, const int *active, const double *mu, int64_t sMu,
                    const double *r, int64_t sR, bool r_newton, const double *eta, double *AtA, int64_t sAtA,
                    double *Arw, int64_t sArw, double *Tip, int64_t sTip, double *rhs, int64_t sRhs,
                    double *tippart) {
  if (AtA) {
    obs_assemble_pattern_kernel<<<dim3(blocks((int64_t)M.n_t * M.nnz, 256), P), 256, 0, L.st>>>(M, active, mu, sMu,
                                                                                              AtA, sAtA);
    L.tick();
  }
  if (Arw || rhs) {
    obs_assemble_vertex_kernel<<<dim3(blocks((int64_t)M.n_t * M.n_s, 128), P), 128, 0, L.st>>>(
        M, active, mu, sMu, r, sR, r_newton ? 1 : 0, eta, M.n_b ? Arw : nullptr, sArw, rhs, sRhs);
    L.tick();
  }
  if (M.n_b > 0 && (Tip || rhs)) {
    obs_assemble_tip_kernel<<<dim3(M.n_t, P), 256, 0, L.st>>>(M, active, mu, sMu, r, sR, r_newton ? 1 : 0, eta,
                                                              Tip ? 1 : 0, rhs ? 1 : 0, tippart);
    L.tick();
    obs_assemble_tip_sum_kernel<<<dim3(M.n_b * M.n_b + M.n_b, P), 32, 0, L.st>>>(M, active, tippart, Tip, sTip,
                                                                               rhs, sRhs);
    L.tick();
  }
}
// Largest change of the linear predictor a full Newton step would make:
// max_i |(A x)_i - eta_i| over the observations (eta = A xprev), per point.
__global__ void __launch_bounds__(256) newton_deta_kernel(DevModel M, Work W) {
  const int b = blockIdx.y;
  if (!W.active[b]) return;
  __shared__ double red[32];
  const double *xb = W.x + b * W.sVec;
  double mx = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M.m; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = fabs(obs_eta(M, xb, i) - W.eta[b * W.sM + i]);
    mx = (d > mx || d != d) ? d : mx;   // a NaN wins, so that it reaches the step test
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double v = __shfl_down_sync(0xffffffffu, mx, o);
    mx = (v > mx || v != v) ? v : mx;
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = (red[k] > m || red[k] != red[k]) ? red[k] : m;
    W.part[((int64_t)b * NPART + blockIdx.x) * PART_W] = m;
  }
}

// x <- xprev + a (x - xprev) with a = min(1, NEWTON_DETA / max change); one block per point.
__global__ void newton_cap_kernel(DevModel M, Work W, int nparts) {
  const int b = blockIdx.x;
  if (!W.active[b]) return;
  __shared__ double s_a;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int p = 0; p < nparts; ++p) {
      const double v = W.part[((int64_t)b * NPART + p) * PART_W];
      m = (v > m || v != v) ? v : m;
    }
    s_a = (m > NEWTON_DETA) ? NEWTON_DETA / m : 1.0;   // a NaN change keeps a = 1 (the step test fails it)
    W.sc[b * SC_COUNT + SC_DETA] = m;
  }
  __syncthreads();
  const double a = s_a;
  if (a == 1.0) return;
  double *x = W.x + b * W.sVec;
  const double *xp = W.xprev + b * W.sVec;
  for (int64_t k = threadIdx.x; k < M.nv; k += blockDim.x) x[k] = fma(a, x[k] - xp[k], xp[k]);
}
void k_newton_cap(Launch &L, const DevModel &M, const Work &W) {
  int nparts = (int)blocks(M.m, 256);
  if (nparts > 64) nparts = 64;
  newton_deta_kernel<<<dim3(nparts, W.P), 256, 0, L.st>>>(M, W);
  L.tick();
  newton_cap_kernel<<<W.P, 256, 0, L.st>>>(M, W, nparts);
  L.tick();
}

// Newton iterations of a captured evaluation: the while-node's body ends here.
__global__ void newton_continue_kernel(cudaGraphConditionalHandle h, const int *any_active, int *ctr) {
  ++*ctr;
  cudaGraphSetConditional(h, *any_active ? 1u : 0u);
}
void k_newton_continue(Launch &L, cudaGraphConditionalHandle h, const int *any_active, int *ctr) {
  newton_continue_kernel<<<1, 1, 0, L.st>>>(h, any_active, ctr);
  L.tick();
}
void k_poisson_step(Launch &L, const DevModel &M, const Work &W, double tol, int iter, int max_iter,
                    const int *iter_dev) {
  poisson_step_kernel<<<W.P, 256, 0, L.st>>>(M, W, tol, iter, max_iter, iter_dev);
  L.tick();
}
template <typename R>
void k_poisson_qobs(Launch &L, const DevModel &M, const Work &W, int t) {
  if (M.max_mt == 0) return;
  poisson_qobs_kernel<R><<<dim3(blocks(M.max_mt, 128), W.P), 128, 0, L.st>>>(M, W, t);
  L.tick();
}
void k_poisson_wobs(Launch &L, const DevModel &M, const Work &W) {
  poisson_wobs_kernel<<<dim3(blocks(M.m, 256), W.P), 256, 0, L.st>>>(M, W);
  L.tick();
}
void k_qc_residual(Launch &L, const DevModel &M, const Work &W, const double *x, const double *b, double *r) {
  qc_residual_kernel<<<dim3(blocks(M.n_p, 128), M.n_t, W.P), 128, 0, L.st>>>(M, W, x, b, r);
  L.tick();
  if (M.n_b > 0) {
    qc_residual_tail_kernel<<<W.P, 256, 0, L.st>>>(M, W, x, b, r);
    L.tick();
  }
}
void k_axpy(Launch &L, const DevModel &M, const Work &W, double *x, const double *d) {
  axpy_kernel<<<dim3(blocks(M.nv, 256), W.P), 256, 0, L.st>>>(M, W, x, d);
  L.tick();
}

#define INLA_INSTANTIATE(R)                                                                                     \
  template void k_assemble_diag<R>(Launch &, const DevModel &, const Work &, int, int, R *, int64_t, bool);     \
  template void k_sparse_right<R>(Launch &, const DevModel &, const Work &, const R *, int64_t, R *, int64_t,  \
                                  bool, const double *, const double *, bool);                                \
  template void k_sparse_left<R>(Launch &, const DevModel &, const Work &, const R *, int64_t, R *, int64_t,   \
                                 bool, const double *, const double *);                                       \
  template void k_dinv_apply<R>(Launch &, const DevModel &, const Work &, const R *, int, const double *,      \
                                int64_t, double *, int64_t, double);                                          \
  template void k_contract_offdiag<R>(Launch &, const DevModel &, const Work &, int, int, int);               \
  template void k_contract_diag<R>(Launch &, const DevModel &, const Work &, int, int, double *, const int *,  \
                                   int64_t, int);                                                             \
  template void k_poisson_qobs<R>(Launch &, const DevModel &, const Work &, int);
INLA_INSTANTIATE(double)
INLA_INSTANTIATE(float)
#undef INLA_INSTANTIATE

void k_zero(Launch &L, double *p, int64_t n) {
  if (n <= 0) return;
  zero_kernel<<<blocks(n, 256), 256, 0, L.st>>>(p, n);
  L.tick();
}

template <typename R>
void bta_prepare_r() {
  prefer_shared(assemble_diag_kernel<R>);
  prefer_shared(sparse_right_tiled_kernel<R>);
  prefer_shared(sparse_right_kernel<R>);
  prefer_shared(sparse_left_kernel<R>);
  prefer_shared(dinv_gemv_kernel<R>);
  prefer_shared(dinv_apply_kernel<R, DA_MAXV>);
  prefer_shared(add_into_kernel<R>);
  prefer_shared(contract_offdiag_kernel<R>);
  prefer_shared(contract_diag_kernel<R>);
  prefer_shared(poisson_qobs_kernel<R>);
}

void bta_prepare() {
  static std::mutex mu;
  static bool done[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  bta_prepare_r<double>();
  bta_prepare_r<float>();
  prefer_shared(params_kernel);
  prefer_shared(qs_values_kernel);
  prefer_shared(set_active_kernel);
  prefer_shared(init_step0_kernel);
  prefer_shared(arrow_update_kernel);
  prefer_shared(arrow_dots_kernel);
  prefer_shared(tip_kernel);
  prefer_shared(fwd_update_kernel);
  prefer_shared(tip_solve_kernel);
  prefer_shared(bwd_rhs_kernel);
  prefer_shared(join_tip_kernel);
  prefer_shared(join_rhs_kernel);
  prefer_shared(selinv_Y_kernel);
  prefer_shared(reduce_parts_kernel);
  prefer_shared(contract_tip_kernel);
  prefer_shared(quadforms_kernel);
  prefer_shared(rhs_gaussian_kernel);
  prefer_shared(obs_reduce_kernel);
  prefer_shared(qs_share_setup_kernel);
  prefer_shared(qs_share_kernel);
  prefer_shared(qs_traces_kernel);
  prefer_shared(finalize_kernel);
  prefer_shared(copy_mode_kernel);
  prefer_shared(fd_points_kernel);
  prefer_shared(outputs_kernel);
  prefer_shared(poisson_eta_kernel);
  prefer_shared(obs_assemble_pattern_kernel);
  prefer_shared(obs_assemble_vertex_kernel);
  prefer_shared(obs_assemble_tip_kernel);
  prefer_shared(obs_assemble_tip_sum_kernel);
  prefer_shared(poisson_step_kernel);
  prefer_shared(poisson_wobs_kernel);
  prefer_shared(qc_residual_kernel);
  prefer_shared(qc_residual_tail_kernel);
  prefer_shared(axpy_kernel);
  prefer_shared(zero_kernel);
  prefer_shared(newton_deta_kernel);
  prefer_shared(newton_cap_kernel);
  prefer_shared(newton_continue_kernel);
  done[dev] = true;
}

}  // namespace inla
