// Internal declarations shared by the library's translation units.
//
// Layout in HBM (per evaluation point b of a wave of P points):
//   Dinv   [P][n_t][n_p][n_p]  inverses of the Schur-complement diagonal blocks
//                              D_t of the block LDL^T factorisation of Q_c,
//                              padded to n_p = roundup(n_s, 64) with an identity
//                              in the padding, full symmetric row-major storage
//   Rt     [P][n_t][n_b][n_p]  arrow blocks after the Schur updates (R~_t)
//   vectors in "padded latent" layout [n_t][n_p] followed by the n_b tail
//   scratch [P][n_p][n_p] matrices for the assembly and the selected inversion
// Sparse theta-free matrices live on one union pattern (CSR over n_s rows):
//   vC, vG, vH (C, G, H = G C^-1 G) and per time block the spatial part of
//   A^T D A.  Q_s(theta) on the pattern is aC*vC + aG*vG + aH*vH.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/inla_gpu.h"

namespace inla {

constexpr int TILE = 64;        // dense tile edge (pivot blocks, GEMM tiles)
constexpr int MAX_NB = 16;      // fixed effects supported by the small kernels
constexpr int MAX_SPATIAL = 3;  // spatial entries per observation row
constexpr int NPART = 256;      // partial sums per point for long reductions
constexpr int PART_W = 8;       // components per partial sum
// Longest row of the sparse pattern (Q_s and A^T A on one time block) that the
// row kernels stage in shared memory; the 2-ring SPDE stencil of a triangle
// mesh has ~19 entries per row.
constexpr int ROW_PMAX = 64;

// Scalars of one evaluation point, computed on the device from theta.
struct PointParams {
  double tau_y;                     // Gaussian noise precision (0 for Poisson)
  double tau_b;                     // fixed-effect prior precision
  double aC, aG, aH;                // Q_s = aC C + aG G + aH H
  double rho;
  double qd_end, qd_mid, q_off;     // AR(1) precision entries
  double dqd_end, dqd_mid, dq_off;  // their derivatives wrt theta_4
  double logprior;
  double dlogprior[4];
  double theta[4];
};

// Index structures and theta-free values of a model (device pointers).
struct DevModel {
  int n_t, n_s, n_b, n_p, lik, nnz;
  int max_mt;                    // largest number of observations in one time block
  int pbw;                       // bandwidth of the pattern: max |column - row|
  int pmax;                      // longest pattern row
  int sweep_g64, sweep_g32;      // sweep tile width for FP64 / FP32 blocks (32 or 64; autotuned)
  int gemm_t32;                  // FP32 GEMM tile (64 or 128; autotuned)
  int f64_tensor;                // FP64 selected-inversion products on the BF16 tensor cores (n_p % 128 == 0)
  int64_t m, n, nv;              // nv = n_t*n_p + n_b (padded latent length)
  const int *prow, *pcol;        // union pattern, CSR [n_s+1], [nnz]
  const int *prow_of;            // [nnz] row of each pattern entry
  const double *vC, *vG, *vH;    // [nnz]
  const int64_t *obs_ptr;        // [n_t+1] observations of block t (sorted by time)
  const int *obs_t;              // [m] time block of each observation
  const int *obs_v;              // [m][3] local vertex of each spatial entry
  const double *obs_w;           // [m][3] weights (0 for unused entries)
  const double *obs_z;           // [m][n_b] covariates
  const double *y, *E;           // [m]
  const int64_t *sp_ptr;         // [n_t*nnz+1] pair contributions of each pattern entry
  const int *sp_obs;             //   observation index
  const double *sp_w;            //   product of the two weights
  const int64_t *vt_ptr;         // [n_t*n_s+1] contributions of each (t, vertex)
  const int *vt_obs;
  const double *vt_w;
  const double *AtA;             // Gaussian: [n_t][nnz] spatial A_t^T A_t
  const double *Arw;             // Gaussian: [n_t][n_b][n_s] Z^T A_t
  const double *Tip;             // Gaussian: [n_b][n_b] Z^T Z
  const double *Aty;             // Gaussian: [nv] A^T y (padded latent layout)
  const double *consts;          // [4]: y^T y, sum lgamma(y+1), sum y log E
  double prior_mean[4], prior_sd[4];
  double tau_b_fixed;
  double nb_size;                // negative binomial size r (0 for the other likelihoods)
  int point_groups;              // 2: a Gaussian wave's factorisation and mode run as two point
                                 // groups on two stream pairs (1: one group)
  int time_parts;                // 2: factorisations without a selected inversion split the time
                                 // chain at its middle block into two chains (1: one chain)
};

// Per-wave workspace (device) with per-point strides (in elements).  The dense
// n_p x n_p blocks (Dinv, T1, S, SigN, SigC and the sweep scratch) have storage
// type R = double (rb = 8) or float (rb = 4, mixed precision); everything else is
// double.
struct Work {
  int P;
  int rb;                // bytes per element of the dense blocks
  int64_t sDinv, sMat, sRt, sVec, sNb2, sWV, sNbNp, sNnz, sPt, sM, sAtAp, sArwp;
  double *theta;         // [P][4]
  PointParams *prm;      // [P]
  double *qs;            // [P][nnz]     Q_s values on the pattern
  void *Dinv;            // [P][n_t][n_p][n_p]  (R)
  double *Rt;            // [P][n_t][n_b][n_p]
  double *Da;            // [P][n_b][n_b]  tip Schur complement, then its inverse
  double *rhs, *zf, *x, *xprev, *tmpv;  // [P][nv]
  double *rvec, *dvec;                   // [P][nv]  refinement residual and correction
  double *wv;            // [P][1+n_b][n_p]  Dinv_t times vectors
  void *T1, *S, *SigN, *SigC;            // [P][n_p][n_p]  (R)
  float *Dh, *Dl, *Sh, *Sl, *Uh, *Ul;    // [P][n_p][n_p]  TF32 hi / lo parts of the tensor-core products' operands
                                         //                (FP32 blocks with n_p % 128 == 0 only)
  uint16_t *Zd, *Zs;                     // [P][OZ_SLICES][n_p][n_p]  BF16 digit slices of the FP64 tensor-core
  int32_t *Ed, *Es;                      // [P][n_p]  products' operands and their row exponents
                                         //           (FP64 blocks with n_p % 128 == 0 only)
  int64_t sZ, sE;
  double *SigAn, *SigAc, *Y;             // [P][n_b][n_p]
  void *gjP, *gjC, *gjO;                 // [P][2][32*32], [P][n_p*32], [P][n_p*32]  (R; sized for double)
  double *QsI;                           // [P][n_p][n_p]  Q_s^-1 (Kronecker prior), always FP64
  double *sc;            // [P][SC_COUNT] per-point scalars
  double *pt;            // [P][n_t][PT_COUNT] per-time-block contractions
  double *part;          // [P][NPART][PART_W] partial sums
  double *tippart;       // [P][n_t][n_b*n_b + n_b] per-time-block partial sums
  int *status;           // [P]
  int *active;           // [P]  1 = this point takes part in the current pass
  int *flags;            // [P]  bit 0: selected inversion, bit 1: adjoint gradient
  int *iters;            // [P]
  int *qsrep;            // [P]  earlier point of the wave whose Q_s this point shares (or itself)
  int *any_active;       // [1]
  int *grp0, *grp1;      // [P]  activity masks of two point groups factorised concurrently
  int lo, hi;            // points [lo, hi) that a pass's whole-array copies cover (hi = 0: all)
  // Poisson
  double *eta, *mu, *qobs, *wobs;        // [P][m] eta, weight b''(eta), a_i^T Sigma a_i, adjoint weights
  double *AtAp;          // [P][n_t][nnz]
  double *Arwp;          // [P][n_t][n_b][n_s]
  double *Tipp;          // [P][n_b][n_b]
  // Scratch of the second elimination chain of a time chain split at a separator
  // block (null when the workspace has none); same shapes and strides as above.
  struct Chain2 {
    void *T1, *S, *SigN, *SigC;
    float *Dh, *Dl, *Sh, *Sl, *Uh, *Ul;
    uint16_t *Zd, *Zs;
    int32_t *Ed, *Es;
    double *wv, *Da, *sc, *zf, *tmpv;
    void *gjP, *gjC, *gjO;
    double *SigAn, *SigAc, *Y, *part;
  } c2;
};

enum {
  SC_LOGDET_QC = 0, SC_LOGDET_Q, SC_LOGDET_QS, SC_TR_QSI_C, SC_TR_QSI_G, SC_TR_QSI_H,
  SC_RES2, SC_LOGLIK, SC_TIP_XX, SC_TIP_LX, SC_TIP_TRSIG, SC_TIP_ATA, SC_STEP2, SC_DETA,
  SC_COUNT = 16
};
enum {
  PT_FD_C = 0, PT_FD_G, PT_FD_H, PT_FD_ATA,   // <Sigma_tt, X>
  PT_FO_C, PT_FO_G, PT_FO_H,                  // <Sigma_{t+1,t}, X>
  PT_FA_ATA,                                  // <Sigma_{a,t}, Z^T A_t>
  PT_XD_C, PT_XD_G, PT_XD_H,                  // x_t^T X x_t
  PT_XO_C, PT_XO_G, PT_XO_H,                  // x_{t+1}^T X x_t + x_t^T X x_{t+1}
  PT_LD_C, PT_LD_G, PT_LD_H,                  // lambda_t^T X x_t
  PT_LO_C, PT_LO_G, PT_LO_H,                  // lambda_{t+1}^T X x_t + lambda_t^T X x_{t+1}
  PT_QD_C, PT_QD_G, PT_QD_H,                  // prior (BTA mode): <Sigma_Q,tt, X>
  PT_QO_C, PT_QO_G, PT_QO_H,                  //                   <Sigma_Q,{t+1,t}, X>
  PT_COUNT = 32
};

// Which matrix an assembly builds.
enum { ASM_QC = 0, ASM_Q = 1, ASM_QS = 2 };

// Optional CUDA-event timing of selected kernels (inla_profile_*).
constexpr int kMaxDevices = 256;   // device indices the per-device caches cover
enum { KID_GJ_UPDATE = 0, KID_GEMM = 1, KID_GJ_PIVOT = 2, KID_GJ_PANEL = 3, KID_GJ_UPDATE32 = 4, KID_COUNT = 5 };
struct Profiler {
  int enabled = 0;      // 0 = off, k >= 1: time every k-th launch of each kernel
  int64_t seen[KID_COUNT] = {};
  std::vector<cudaEvent_t> pool;
  size_t next = 0;
  struct Rec { int id; double units; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  cudaEvent_t get() {
    if (next == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[next++];
  }
  void reset() {
    next = 0;
    recs.clear();
    for (auto &c : seen) c = 0;
  }
  ~Profiler() { for (auto e : pool) cudaEventDestroy(e); }
};

struct Launch {
  cudaStream_t st;
  int64_t *counter;
  Profiler *prof = nullptr;
  bool capturing = false;   // being recorded into a CUDA graph (no host synchronisation allowed)
  // second stream for the second elimination chain, and the events that fork it
  // from st and join it back (null: no second chain)
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // the second point group's stream pair and events, and the events that fork it from st
  // and join it back (null: one group)
  cudaStream_t gst = nullptr, gst2 = nullptr;
  cudaEvent_t gev_fork = nullptr, gev_join = nullptr, gev_gfork = nullptr, gev_gjoin = nullptr;
  int cur_id = -1;
  double cur_units = 0.0;
  cudaEvent_t cur_a = nullptr;
  void tick() { if (counter) ++*counter; }
  // bracket one launch of kernel `id` processing `units` algorithmic units
  void start(int id, double units) {
    if (!prof || !prof->enabled) return;
    if (prof->seen[id]++ % prof->enabled != 0) return;
    cur_id = id;
    cur_units = units;
    cur_a = prof->get();
    cudaEventRecord(cur_a, st);
  }
  void stop() {
    if (!prof || !prof->enabled || cur_id < 0) return;
    cudaEvent_t b = prof->get();
    cudaEventRecord(b, st);
    prof->recs.push_back({cur_id, cur_units, cur_a, b});
    cur_id = -1;
  }
};

// Likelihood terms per observation: y eta - b is the log-likelihood up to
// theta-free constants, y - mean its derivative in eta (the score), weight the
// Newton weight -d^2 log p / d eta^2, third the derivative of the weight
// (adjoint gradient).  Canonical links: Poisson b = E exp(eta) (mean, weight and
// third all equal b); binomial b = N log(1 + exp(eta)), p = logistic(eta), mean
// N p, weight N p (1 - p), third N p (1 - p) (1 - 2 p).  Negative binomial with
// the log link (mu = E exp(eta), size r; not canonical): b = (y + r) log(mu + r),
// mean (y + r) mu / (mu + r), weight (y + r) r mu / (mu + r)^2 (the observed
// information), third (y + r) r mu (r - mu) / (mu + r)^3.
struct GlmTerms {
  double b, mean, weight, third;
};
__device__ __forceinline__ GlmTerms glm_terms(int lik, double E, double y, double r, double eta) {
  GlmTerms g;
  if (lik == INLA_LIK_NEGBINOMIAL) {
    const double mu = E * exp(eta), s = mu + r, a = (y + r) * mu / s;
    g.b = (y + r) * log(s);
    g.mean = a;
    g.weight = a * r / s;
    g.third = g.weight * (r - mu) / s;
    return g;
  }
  if (lik == INLA_LIK_BINOMIAL) {
    const double p = 1.0 / (1.0 + exp(-eta));
    const double q = 1.0 / (1.0 + exp(eta));   // 1 - p without cancellation
    g.b = E * (eta > 0.0 ? eta + log1p(exp(-eta)) : log1p(exp(eta)));
    g.mean = E * p;
    g.weight = E * p * q;
    g.third = g.weight * (q - p);
  } else {
    const double mu = E * exp(eta);
    g.b = g.mean = g.weight = g.third = mu;
  }
  return g;
}

// Every kernel of the library asks for the largest shared-memory share of the SM's
// unified L1 / shared storage (the tensor-core products need it anyway), so that
// consecutive kernels, and the kernels of the two elimination chains that share the
// SMs, do not make the SMs switch the split between launches (measured: 3.5% of the
// FP64 stencil step).  Set once per device by the *_prepare functions.
template <typename K>
inline void prefer_shared(K *kernel) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

// dense_blocks.cu (R = double or float)
void dense_prepare();   // one-time kernel attributes of every source file (call before a stream capture)
void bta_prepare();     // bta_kernels.cu's kernel attributes
template <typename R>
void gj_invert(Launch &L, const DevModel &M, const Work &W, R *A, int64_t strideA, double *logdet, int ld_stride);
template <typename R>
void gemm_nn(Launch &L, int P, int n, const R *A, int64_t sA, const R *B, int64_t sB, R *C, int64_t sC, R alpha,
             const R *C0, int64_t sC0, R beta, bool lower_only, const int *active, int tile = 128);
template <typename R>
void mirror_lower(Launch &L, int P, int n, R *A, int64_t sA, const int *active);

// tc_gemm.cu: C = alpha X Y^T + beta C0 in 3xTF32 on the tensor cores (n % 128 == 0)
void tc_prepare();
// ozaki.cu: FP64 products C = alpha X Y^T + beta C0 on the BF16 tensor cores by
// error-free splitting into OZ_SLICES digit slices per entry (X: M x K, Y: N x K;
// M % 128, N % 64, K % 32 == 0).  ozaki_split writes the slices of P row blocks
// (S[b][a][r][k] BF16, point stride sS = OZ_SLICES rows K) and their exponents
// (E[b][r], point stride sE).
constexpr int OZ_SLICES = 8;   // digit slices per FP64 entry
constexpr int OZ_LEVELS = 8;   // digit products s_a t_b with a + b < OZ_LEVELS
void ozaki_prepare();
void ozaki_split(Launch &L, int P, int rows, int K, const double *X, int64_t ldx, int64_t sX, uint16_t *S,
                 int64_t sS, int32_t *E, int64_t sE, const int *active);
// two operands in one launch (same point strides of the slices and exponents)
void ozaki_split2(Launch &L, int P, int rows0, int K0, const double *X0, int64_t ldx0, int64_t sX0, uint16_t *S0,
                  int32_t *E0, int rows1, int K1, const double *X1, int64_t ldx1, int64_t sX1, uint16_t *S1,
                  int32_t *E1, int64_t sS, int64_t sE, const int *active);
void gemm_nt_ozaki(Launch &L, int P, int M, int N, int K, const uint16_t *Xs, int64_t sXs, const int32_t *Xe,
                   int64_t sXe, const uint16_t *Ys, int64_t sYs, const int32_t *Ye, int64_t sYe, double *C,
                   int64_t ldc, int64_t sC, double alpha, const double *C0, int64_t ldc0, int64_t sC0, double beta,
                   bool lower_only, const int *active, int *status);

// bound (ns of %globaltimer) on one mbarrier wait of the tensor-core kernels
uint64_t wait_limit_ns();
void set_wait_limit_ns(uint64_t ns);
void gemm_nt_tf32x3(Launch &L, int P, int n, const float *X, int64_t sX, const float *Y, int64_t sY, float *C,
                    int64_t sC, float alpha, const float *C0, int64_t sC0, float beta, bool lower_only,
                    const int *active, int *status);
// The same product with operands already split into TF32 hi / lo parts (P
// compact M x K and N x K matrices, sX / sY floats apart; M, N % 128 == 0,
// K % 32 == 0), fed by TMA, into C (leading dimension ldc); with Chi != nullptr
// the result is stored split (Chi / Clo, leading dimension ldc) instead of to C.
void gemm_nt_tf32x3_split(Launch &L, int P, int M, int N, int K, const float *Xh, const float *Xl, int64_t sX,
                          const float *Yh, const float *Yl, int64_t sY, float *C, int64_t ldc, int64_t sC, float alpha,
                          const float *C0, int64_t ldc0, int64_t sC0, float beta, float *Chi, float *Clo,
                          bool lower_only, const int *active, int *status);
// hi / lo parts of the rows x K block at src (leading dimension lds) into compact arrays (K % 4 == 0).
void split_tf32_2d(Launch &L, int P, int rows, int K, const float *src, int64_t lds, int64_t ssrc, float *hi,
                   float *lo, int64_t sdst, const int *active);
// hi = tf32(x), lo = tf32(x - hi) for P matrices of `count` floats (count % 4 == 0).
void split_tf32(Launch &L, int P, const float *src, int64_t ssrc, float *hi, float *lo, int64_t sdst, int64_t count,
                const int *active);
// A -= C O^T over the lower 64 x 64 sub-tiles of the FP32 block sweep at pivot
// `pivot` (rank 64, 3xTF32 on the tensor cores; n_p % 128 == 0), leaving out the
// pivot row and column and the sub-tile (next, next) (next < 0: none).
void sweep_update_tf32x3(Launch &L, int P, int n_p, float *A, int64_t sA, const float *Cbuf, const float *Obuf,
                         int64_t sCO, int pivot, int next, const int *active, int *status);

// bta_kernels.cu
void k_params(Launch &L, const DevModel &M, const Work &W);
void k_qs_values(Launch &L, const DevModel &M, const Work &W);
void k_set_active(Launch &L, const Work &W, int mask);
void k_init_step0(Launch &L, const DevModel &M, const Work &W, int mode, int t0, bool tip_init);
template <typename R>
void k_assemble_diag(Launch &L, const DevModel &M, const Work &W, int t, int mode, R *dst, int64_t sdst,
                     bool schur);
// lower_band: compute only the columns that the lower-tile assembly of the
// next diagonal block reads (the factorisation); false = the full matrix.
template <typename R>
void k_sparse_right(Launch &L, const DevModel &M, const Work &W, const R *X, int64_t sX, R *out, int64_t sOut,
                    bool coef_qoff, const double *SigA, const double *Rt_t, bool lower_band = false);
template <typename R>
void k_sparse_left(Launch &L, const DevModel &M, const Work &W, const R *X, int64_t sX, R *out, int64_t sOut,
                   bool with_X, const double *Rt_t, const double *Ymat);
template <typename R>
void k_dinv_apply(Launch &L, const DevModel &M, const Work &W, const R *Dinv_t, int nvec, const double *vecs,
                  int64_t sVecs, double *out, int64_t sOut, double scale);
void k_arrow_update(Launch &L, const DevModel &M, const Work &W, int t, int mode);
void k_arrow_dots(Launch &L, const DevModel &M, const Work &W, int tprev);
void k_tip(Launch &L, const DevModel &M, const Work &W, int ld_slot);
void k_fwd_update(Launch &L, const DevModel &M, const Work &W, int t, int nbr, double *z);
void k_tip_solve(Launch &L, const DevModel &M, const Work &W, const double *z, double *x);
void k_bwd_rhs(Launch &L, const DevModel &M, const Work &W, int t, int nbr, const double *z, const double *x);
// joining two elimination chains of the time chain at a separator block
template <typename R>
void k_add_into(Launch &L, int P, R *dst, const R *src, int64_t stride, int64_t count, const int *active);
void k_join_tip(Launch &L, const DevModel &M, const Work &W, const double *Da1, const double *sc1, int ld_slot);
void k_join_rhs(Launch &L, const DevModel &M, const Work &W, int k, double *z, const double *z1, const double *rhs);
void k_selinv_Y(Launch &L, const DevModel &M, const Work &W, int t, bool has_next);
template <typename R>
void k_contract_offdiag(Launch &L, const DevModel &M, const Work &W, int t, int pair, int slot0);
template <typename R>
void k_contract_diag(Launch &L, const DevModel &M, const Work &W, int t, int mode, double *marg_var,
                     const int *point_out, int64_t point_base, int slot0);
void k_contract_tip(Launch &L, const DevModel &M, const Work &W, int mode, double *marg_var,
                    const int *point_out, int64_t point_base);
void k_quadforms(Launch &L, const DevModel &M, const Work &W, const double *u, const double *v, int slot0,
                 int tip_slot);
void k_rhs_gaussian(Launch &L, const DevModel &M, const Work &W);
void k_obs_reduce(Launch &L, const DevModel &M, const Work &W, int kind);
void k_qs_traces(Launch &L, const DevModel &M, const Work &W);   // tr(Q_s^-1 X) from W.QsI
// Kronecker prior: points with the same range parameter share one inversion of Q_s
void k_qs_share_setup(Launch &L, const Work &W);                  // W.qsrep; active = representatives
void k_qs_share(Launch &L, const DevModel &M, const Work &W);     // log|Q_s| and traces of the others
// y = Q_c x (mode ASM_QC) in FP64 from the sparse blocks; r = b - y when b != nullptr
void k_qc_residual(Launch &L, const DevModel &M, const Work &W, const double *x, const double *b, double *r);
void k_axpy(Launch &L, const DevModel &M, const Work &W, double *x, const double *d);
void k_finalize(Launch &L, const DevModel &M, const Work &W, int grad_mode, int prior_mode, int64_t point_base,
                double *f_all, double *grad_all, int *status_all, int *iters_all);
void k_copy_mode(Launch &L, const DevModel &M, const Work &W, double *x_out, const int *point_out,
                 int64_t point_base);
void k_fd_points(Launch &L, int B, int per, const double *theta, double eps, double *pts);
// evaluation points per centre of a gradient mode: 9 (central), 5 (forward), else 1
inline int fd_points_per_centre(int grad) {
  return grad == INLA_GRAD_FD_CENTRAL ? 9 : (grad == INLA_GRAD_FD_FORWARD ? 5 : 1);
}
void k_outputs(Launch &L, int B, int per, double eps, int d, const double *f_all, const double *grad_all,
               const int *status_all, const int *iters_all, double *f, double *grad, int *status, int *iters);
void k_poisson_eta(Launch &L, const DevModel &M, const Work &W, const double *x);
// A^T diag(mu) A pieces and A^T r.  mu == nullptr means mu = 1; r_newton
// uses r = y - mu + mu*eta from the workspace.  Any output may be nullptr.
void k_obs_assemble(Launch &L, const DevModel &M, int P, const int *active, const double *mu, int64_t sMu,
                    const double *r, int64_t sR, bool r_newton, const double *eta, double *AtA, int64_t sAtA,
                    double *Arw, int64_t sArw, double *Tip, int64_t sTip, double *rhs, int64_t sRhs,
                    double *tippart);
void k_poisson_step(Launch &L, const DevModel &M, const Work &W, double tol, int iter, int max_iter,
                    const int *iter_dev = nullptr);
// Newton step cap: x <- xprev + a (x - xprev), a = min(1, NEWTON_DETA / max_i |(A (x - xprev))_i|)
constexpr double NEWTON_DETA = 2.0;
void k_newton_cap(Launch &L, const DevModel &M, const Work &W);
// graph body: count the Newton iteration and continue the while-node while any point is active
void k_newton_continue(Launch &L, cudaGraphConditionalHandle h, const int *any_active, int *ctr);
template <typename R>
void k_poisson_qobs(Launch &L, const DevModel &M, const Work &W, int t);
void k_poisson_wobs(Launch &L, const DevModel &M, const Work &W);
void k_zero(Launch &L, double *p, int64_t n);

// setup_kernels.cu
void setup_theta_free(cudaStream_t st, DevModel &M, const int64_t *d_hptr, const int *d_hk, const int *d_hik,
                      const int *d_hkj, const double *d_Gval, const double *d_Cdiag, const int *d_gpos,
                      double *vC, double *vG, double *vH);
void setup_gaussian(cudaStream_t st, DevModel &M, double *AtA, double *Arw, double *Tip, double *Aty,
                    double *tippart);
void setup_consts(cudaStream_t st, DevModel &M, double *consts);

void set_error(const std::string &msg);

}  // namespace inla
