// C ABI (include/inla_gpu.h): model construction on the host (index
// structures only; every value is computed by device kernels), workspace
// management and the orchestration of one batched evaluation.
//
// One evaluation of a wave of P points runs, per point (all points of the
// wave advance together, one kernel launch per step):
//   1. theta -> model scalars; Q_s(theta) on the sparse pattern.
//   2. log|Q|: Kronecker form n_s log|Q_t| + n_t log|Q_s| + n_b log tau_b with one
//      dense inversion of Q_s, or the same block factorisation as Q_c.
//   3. Block factorisation of Q_c along the time chain (Sec. 2.4): per t the
//      Schur complement D_t is assembled from the sparse blocks and inverted
//      (block sweep, log|D_t| from its pivots); the arrow is updated; the tip
//      D_a is factored last (arrow last: no fill, Fig. arrowhead_matrices).
//   4. Mode: block forward/backward substitution (Gaussian), or the Newton
//      iteration of Sec. 2.2 (Poisson) with a factorisation per iteration and
//      a refactorisation at the mode.
//   5. f = -log pi~(theta|y) from the log-determinants and quadratic forms
//      (Eq. post_theta_approx, Sec. 3.1).
//   6. Selected inversion (block Takahashi recursion, Eq. takahashi_recursion
//      in block form) for diag(Q_c^-1) and the traces of the adjoint gradient;
//      Poisson adds one adjoint solve.  Central differences (Eq. central_diff)
//      instead evaluate 2d+1 points per centre.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <stdexcept>
#include <string>
#include <vector>

#include "inla_internal.cuh"

using namespace inla;

namespace inla {
static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
const char *get_error() { return g_err.c_str(); }
}  // namespace inla

namespace {

struct ApiError : std::runtime_error {
  int code;
  ApiError(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define CUDA_OK(call)                                                                               \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      throw ApiError(e_ == cudaErrorMemoryAllocation ? INLA_ERR_OOM : INLA_ERR_CUDA,                \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                           \
  } while (0)

inline int64_t rup(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

__global__ void point_out_kernel(int P, int per, int *out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  out[p] = (per == 1) ? p : ((p % per == 0) ? p / per : -1);
}

__global__ void flags_kernel(Work W, int64_t w0, int per, int centre_flags) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= W.P) return;
  const int64_t g = w0 + b;
  W.flags[b] = (per == 1 || g % per == 0) ? centre_flags : 0;
}

// A point whose status is not OK gets NaN marginal variances (its selected
// inverse may be incomplete, e.g. after a timed-out tensor-core product).
__global__ void mask_failed_kernel(Work W, int64_t n, double *mv, const int *point_out, int64_t point_base) {
  const int b = blockIdx.y;
  if (W.status[b] == INLA_OK) return;
  const int o = point_out[point_base + b];
  if (o < 0) return;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    mv[(int64_t)o * n + k] = NAN;
}

__global__ void zero_slot_kernel(Work W, int slot) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < W.P && W.active[b]) W.sc[b * SC_COUNT + slot] = 0.0;
}

}  // namespace

struct inla_model {
  int device = 0;
  DevModel M{};
  std::vector<void *> allocs;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  int ws_points = 0;
  void *bb = nullptr;
  size_t bb_bytes = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t stream2 = nullptr;   // the second elimination chain of a split time chain
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaStream_t stream3 = nullptr, stream4 = nullptr;   // the second point group's two chains
  cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr, ev_gfork = nullptr, ev_gjoin = nullptr;
  cudaEvent_t done = nullptr;   // end of the last evaluation (orders calls across streams)
  bool done_valid = false;
  int64_t launches = 0;
  Profiler prof;
  struct GraphEntry {
    int B, grad, prior, precision, want_mode, want_marg_var, max_newton, time_parts, point_groups;
    double fd_eps, newton_tol;
    void *ws, *bb;                 // workspace the graph was captured on
    cudaGraphExec_t exec = nullptr;
    void *stage = nullptr;         // theta in, outputs out (device)
    double *theta, *f, *grad_out, *x, *mv;
    int *status, *iters;
    int64_t launches = 0;
  };
  std::vector<GraphEntry> graphs;
  // host-API staging buffers (device)
  void *hb = nullptr;
  size_t hb_bytes = 0;

  template <class T>
  T *dalloc(size_t count) {
    void *p = nullptr;
    if (count == 0) count = 1;
    CUDA_OK(cudaMalloc(&p, count * sizeof(T)));
    allocs.push_back(p);
    return static_cast<T *>(p);
  }
  template <class T>
  T *upload(const std::vector<T> &v) {
    T *p = dalloc<T>(v.size());
    if (!v.empty()) CUDA_OK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
  }
  ~inla_model() {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(device);
    if (done && done_valid) cudaEventSynchronize(done);   // the last evaluation has finished
    for (void *p : allocs) cudaFree(p);
    if (ws) cudaFree(ws);
    if (bb) cudaFree(bb);
    if (hb) cudaFree(hb);
    if (stream) cudaStreamDestroy(stream);
    if (stream2) cudaStreamDestroy(stream2);
    for (cudaStream_t q : {stream3, stream4})
      if (q) cudaStreamDestroy(q);
    for (cudaEvent_t e : {ev_fork2, ev_join2, ev_gfork, ev_gjoin})
      if (e) cudaEventDestroy(e);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (done) cudaEventDestroy(done);
    for (auto &g : graphs) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.stage) cudaFree(g.stage);
    }
    cudaSetDevice(cur);
  }
};

namespace {

void *static_scratch(int device);   // the no-allocation entry point's array (defined below)

// ------------------------------------------------------------------ model construction

void validate(const inla_model_desc *d) {
  auto bad = [](const std::string &m) { throw ApiError(INLA_ERR_ARG, m); };
  if (!d) bad("desc is NULL");
  if (d->n_t < 1 || d->n_s < 1) bad("n_t and n_s must be >= 1");
  if (d->n_b < 0 || d->n_b > MAX_NB) bad("n_b must be in [0, 16]");
  if (d->m < 1 || d->m > (int64_t)INT32_MAX) bad("m must be in [1, 2^31)");
  if (d->lik != INLA_LIK_GAUSSIAN && d->lik != INLA_LIK_POISSON && d->lik != INLA_LIK_BINOMIAL &&
      d->lik != INLA_LIK_NEGBINOMIAL)
    bad("unknown likelihood");
  if (d->lik == INLA_LIK_NEGBINOMIAL && !(d->nb_size > 0.0 && std::isfinite(d->nb_size)))
    bad("negative binomial size must be positive and finite");
  if (!d->C_diag || !d->G_rowptr || !d->G_col || !d->G_val || !d->A_rowptr || !d->A_col || !d->A_val || !d->y)
    bad("a required array is NULL");
  if ((d->lik == INLA_LIK_POISSON || d->lik == INLA_LIK_NEGBINOMIAL) && !d->E) bad("this likelihood needs exposures E");
  if (d->lik == INLA_LIK_BINOMIAL && !d->E) bad("binomial likelihood needs the numbers of trials in E");
  if (d->lik == INLA_LIK_GAUSSIAN && !(d->tau_b > 0.0)) bad("tau_b must be > 0");
  for (int j = 0; j < 4; ++j)
    if (!(d->prior_sd[j] > 0.0) || !std::isfinite(d->prior_mean[j])) bad("hyperprior sd must be > 0");
  const int64_t n_s = d->n_s;
  for (int64_t i = 0; i < n_s; ++i)
    if (!(d->C_diag[i] > 0.0) || !std::isfinite(d->C_diag[i])) bad("C_diag must be positive and finite");
  if (d->G_rowptr[0] != 0) bad("G_rowptr[0] must be 0");
  for (int64_t i = 0; i < n_s; ++i) {
    if (d->G_rowptr[i + 1] < d->G_rowptr[i]) bad("G_rowptr not monotone");
    for (int p = d->G_rowptr[i]; p < d->G_rowptr[i + 1]; ++p) {
      if (d->G_col[p] < 0 || d->G_col[p] >= n_s) bad("G column index out of range");
      if (p > d->G_rowptr[i] && d->G_col[p] <= d->G_col[p - 1]) bad("G columns must be sorted and unique");
      if (!std::isfinite(d->G_val[p])) bad("G value not finite");
    }
  }
  if (d->A_rowptr[0] != 0) bad("A_rowptr[0] must be 0");
  const int64_t N = (int64_t)d->n_t * n_s, n = N + d->n_b;
  for (int64_t r = 0; r < d->m; ++r) {
    if (d->A_rowptr[r + 1] < d->A_rowptr[r]) bad("A_rowptr not monotone");
    int nsp = 0;
    int64_t tb = -1;
    for (int64_t p = d->A_rowptr[r]; p < d->A_rowptr[r + 1]; ++p) {
      const int64_t c = d->A_col[p];
      if (c < 0 || c >= n) bad("A column index out of range");
      if (p > d->A_rowptr[r] && c <= d->A_col[p - 1]) bad("A columns must be sorted and unique within a row");
      if (!std::isfinite(d->A_val[p])) bad("A value not finite");
      if (c < N) {
        if (tb >= 0 && c / n_s != tb) bad("spatial entries of an A row must lie in one time block");
        tb = c / n_s;
        ++nsp;
      }
    }
    if (nsp < 1 || nsp > MAX_SPATIAL) bad("each A row needs 1 to 3 spatial entries");
    if (!std::isfinite(d->y[r])) bad("y not finite");
    if (d->lik == INLA_LIK_POISSON || d->lik == INLA_LIK_NEGBINOMIAL) {
      if (!(d->E[r] > 0.0) || !std::isfinite(d->E[r])) bad("E must be positive");
      if (d->y[r] < 0.0 || d->y[r] != std::floor(d->y[r])) bad("count data y must be non-negative integers");
    }
    if (d->lik == INLA_LIK_BINOMIAL) {
      if (!(d->E[r] >= 1.0) || d->E[r] != std::floor(d->E[r]) || d->E[r] > 1e9)
        bad("binomial numbers of trials must be positive integers");
      if (d->y[r] < 0.0 || d->y[r] > d->E[r] || d->y[r] != std::floor(d->y[r]))
        bad("binomial y must be integers in [0, N]");
    }
  }
}

inla_model *create_model(const inla_model_desc *d, int device) {
  validate(d);
  int ndev = 0;
  CUDA_OK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) throw ApiError(INLA_ERR_ARG, "device index out of range");
  CUDA_OK(cudaSetDevice(device));
  auto *mdl = new inla_model();
  mdl->device = device;
  try {
    const int n_t = d->n_t, n_s = d->n_s, n_b = d->n_b;
    const int64_t m = d->m, N = (int64_t)n_t * n_s;
    DevModel &M = mdl->M;
    M.n_t = n_t; M.n_s = n_s; M.n_b = n_b; M.lik = d->lik; M.m = m;
    M.n_p = (int)rup(n_s, TILE);
    M.n = N + n_b;
    M.nv = (int64_t)n_t * M.n_p + n_b;
    for (int j = 0; j < 4; ++j) { M.prior_mean[j] = d->prior_mean[j]; M.prior_sd[j] = d->prior_sd[j]; }
    M.tau_b_fixed = d->tau_b;
    M.nb_size = d->lik == INLA_LIK_NEGBINOMIAL ? d->nb_size : 0.0;

    // observations: time block, vertices, weights, covariates; stable sort by time
    std::vector<int> ot(m);
    std::vector<int> ov(m * MAX_SPATIAL, 0);
    std::vector<double> ow(m * MAX_SPATIAL, 0.0), oz(m * (int64_t)n_b, 0.0);
    for (int64_t r = 0; r < m; ++r) {
      int s = 0;
      for (int64_t p = d->A_rowptr[r]; p < d->A_rowptr[r + 1]; ++p) {
        const int64_t c = d->A_col[p];
        if (c < N) {
          ot[r] = (int)(c / n_s);
          ov[r * MAX_SPATIAL + s] = (int)(c % n_s);
          ow[r * MAX_SPATIAL + s] = d->A_val[p];
          ++s;
        } else {
          oz[r * n_b + (c - N)] = d->A_val[p];
        }
      }
      for (; s < MAX_SPATIAL; ++s) ov[r * MAX_SPATIAL + s] = ov[r * MAX_SPATIAL];
    }
    std::vector<int64_t> obs_ptr(n_t + 1, 0);
    for (int64_t r = 0; r < m; ++r) obs_ptr[ot[r] + 1]++;
    for (int t = 0; t < n_t; ++t) obs_ptr[t + 1] += obs_ptr[t];
    std::vector<int64_t> perm(m), fill(obs_ptr.begin(), obs_ptr.end() - 1);
    for (int64_t r = 0; r < m; ++r) perm[fill[ot[r]]++] = r;
    std::vector<int> s_t(m), s_v(m * MAX_SPATIAL);
    std::vector<double> s_w(m * MAX_SPATIAL), s_z(m * (int64_t)n_b), s_y(m), s_E;
    if (d->lik != INLA_LIK_GAUSSIAN) s_E.resize(m);
    for (int64_t k = 0; k < m; ++k) {
      const int64_t r = perm[k];
      s_t[k] = ot[r];
      for (int s = 0; s < MAX_SPATIAL; ++s) {
        s_v[k * MAX_SPATIAL + s] = ov[r * MAX_SPATIAL + s];
        s_w[k * MAX_SPATIAL + s] = ow[r * MAX_SPATIAL + s];
      }
      for (int l = 0; l < n_b; ++l) s_z[k * n_b + l] = oz[r * n_b + l];
      s_y[k] = d->y[r];
      if (!s_E.empty()) s_E[k] = d->E[r];
    }
    int max_mt = 0;
    for (int t = 0; t < n_t; ++t) max_mt = std::max<int>(max_mt, (int)(obs_ptr[t + 1] - obs_ptr[t]));
    M.max_mt = max_mt;

    // union pattern: struct(G) + diag, struct(G)^2, and observation vertex pairs
    std::vector<std::vector<int>> gadj(n_s), pat(n_s);
    for (int i = 0; i < n_s; ++i) {
      gadj[i].push_back(i);
      for (int p = d->G_rowptr[i]; p < d->G_rowptr[i + 1]; ++p) gadj[i].push_back(d->G_col[p]);
      std::sort(gadj[i].begin(), gadj[i].end());
      gadj[i].erase(std::unique(gadj[i].begin(), gadj[i].end()), gadj[i].end());
    }
    for (int i = 0; i < n_s; ++i)
      for (int k : gadj[i])
        for (int j : gadj[k]) pat[i].push_back(j);
    for (int64_t k = 0; k < m; ++k)
      for (int a = 0; a < MAX_SPATIAL; ++a)
        for (int b = 0; b < MAX_SPATIAL; ++b) pat[s_v[k * MAX_SPATIAL + a]].push_back(s_v[k * MAX_SPATIAL + b]);
    std::vector<int> prow(n_s + 1, 0), pcol, prow_of;
    for (int i = 0; i < n_s; ++i) {
      auto &r = pat[i];
      std::sort(r.begin(), r.end());
      r.erase(std::unique(r.begin(), r.end()), r.end());
      prow[i + 1] = prow[i] + (int)r.size();
      for (int j : r) { pcol.push_back(j); prow_of.push_back(i); }
    }
    const int nnz = prow[n_s];
    M.nnz = nnz;
    int pbw = 0;
    for (int i = 0; i < n_s; ++i)
      for (int e = prow[i]; e < prow[i + 1]; ++e) pbw = std::max(pbw, std::abs(pcol[e] - i));
    M.pbw = pbw;
    int pmax = 0;
    for (int i = 0; i < n_s; ++i) pmax = std::max(pmax, prow[i + 1] - prow[i]);
    M.pmax = pmax;
    if (pmax > ROW_PMAX)
      throw ApiError(INLA_ERR_UNSUPPORTED, "a row of the pattern of G C^-1 G has more than 64 entries");
    M.sweep_g64 = 32;
    // the CUDA-core FP32 sweep update measured faster than the tensor-core one (INLA_SWEEP_TF32X3):
    // 29.4 vs 22.9 TFLOP/s at n_p = 2560, 33.0 vs 27.6 at n_p = 4096
    // FP32 blocks: the blocked inversion with tensor-core products measured ahead of the CUDA-core
    // sweep from 2560 rows on (and behind it at 1024), so it is the default from 2048 on
    M.sweep_g32 = (M.n_p % 128 == 0 && M.n_p >= 2048) ? INLA_INV_BLOCKED : 64;
    M.gemm_t32 = INLA_GEMM_TF32X3;   // tensor cores where n_p % 128 == 0, else 128-wide CUDA-core tiles
    M.f64_tensor = 1;                // FP64 selected inversion through BF16 digit slices where n_p % 128 == 0
    M.time_parts = 2;                // factorisations without a selected inversion: two chains
    M.point_groups = 2;              // Gaussian factorisations: two concurrent point groups
    auto find = [&](int i, int j) -> int {
      auto b = pcol.begin() + prow[i], e = pcol.begin() + prow[i + 1];
      auto it = std::lower_bound(b, e, j);
      if (it == e || *it != j) throw ApiError(INLA_ERR_ARG, "internal: pattern lookup failed");
      return (int)(it - pcol.begin());
    };
    // G must be structurally and numerically symmetric
    for (int i = 0; i < n_s; ++i)
      for (int p = d->G_rowptr[i]; p < d->G_rowptr[i + 1]; ++p) {
        const int j = d->G_col[p];
        const int *b = d->G_col + d->G_rowptr[j], *e = d->G_col + d->G_rowptr[j + 1];
        const int *it = std::lower_bound(b, e, i);
        if (it == e || *it != i) throw ApiError(INLA_ERR_ARG, "G pattern is not symmetric");
        const double v1 = d->G_val[p], v2 = d->G_val[it - d->G_col];
        if (std::fabs(v1 - v2) > 1e-12 * (std::fabs(v1) + std::fabs(v2)) + 1e-300)
          throw ApiError(INLA_ERR_ARG, "G is not symmetric");
      }
    // contribution lists of H = G C^-1 G on the pattern
    std::vector<int64_t> hcnt(nnz + 1, 0);
    for (int i = 0; i < n_s; ++i)
      for (int p1 = d->G_rowptr[i]; p1 < d->G_rowptr[i + 1]; ++p1) {
        const int k = d->G_col[p1];
        for (int p2 = d->G_rowptr[k]; p2 < d->G_rowptr[k + 1]; ++p2) hcnt[find(i, d->G_col[p2]) + 1]++;
      }
    for (int e = 0; e < nnz; ++e) hcnt[e + 1] += hcnt[e];
    std::vector<int> hk(hcnt[nnz]), hik(hcnt[nnz]), hkj(hcnt[nnz]);
    {
      std::vector<int64_t> f(hcnt.begin(), hcnt.end() - 1);
      for (int i = 0; i < n_s; ++i)
        for (int p1 = d->G_rowptr[i]; p1 < d->G_rowptr[i + 1]; ++p1) {
          const int k = d->G_col[p1];
          for (int p2 = d->G_rowptr[k]; p2 < d->G_rowptr[k + 1]; ++p2) {
            const int64_t c = f[find(i, d->G_col[p2])]++;
            hk[c] = k; hik[c] = p1; hkj[c] = p2;
          }
        }
    }
    std::vector<int> gpos(nnz, -1);
    for (int i = 0; i < n_s; ++i)
      for (int p = d->G_rowptr[i]; p < d->G_rowptr[i + 1]; ++p) gpos[find(i, d->G_col[p])] = p;
    // pair contributions (t, pattern entry) and vertex contributions (t, v)
    std::vector<int64_t> sp_ptr((int64_t)n_t * nnz + 1, 0), vt_ptr((int64_t)n_t * n_s + 1, 0);
    std::vector<int> pairpos(m * MAX_SPATIAL * MAX_SPATIAL);
    for (int64_t k = 0; k < m; ++k) {
      const int t = s_t[k];
      for (int a = 0; a < MAX_SPATIAL; ++a) {
        if (s_w[k * MAX_SPATIAL + a] == 0.0 && a > 0) continue;
        vt_ptr[(int64_t)t * n_s + s_v[k * MAX_SPATIAL + a] + 1]++;
        for (int b = 0; b < MAX_SPATIAL; ++b) {
          if (s_w[k * MAX_SPATIAL + b] == 0.0 && b > 0) continue;
          const int e = find(s_v[k * MAX_SPATIAL + a], s_v[k * MAX_SPATIAL + b]);
          pairpos[(k * MAX_SPATIAL + a) * MAX_SPATIAL + b] = e;
          sp_ptr[(int64_t)t * nnz + e + 1]++;
        }
      }
    }
    for (size_t e = 1; e < sp_ptr.size(); ++e) sp_ptr[e] += sp_ptr[e - 1];
    for (size_t e = 1; e < vt_ptr.size(); ++e) vt_ptr[e] += vt_ptr[e - 1];
    std::vector<int> sp_obs(sp_ptr.back()), vt_obs(vt_ptr.back());
    std::vector<double> sp_w(sp_ptr.back()), vt_w(vt_ptr.back());
    {
      std::vector<int64_t> fs(sp_ptr.begin(), sp_ptr.end() - 1), fv(vt_ptr.begin(), vt_ptr.end() - 1);
      for (int64_t k = 0; k < m; ++k) {
        const int t = s_t[k];
        for (int a = 0; a < MAX_SPATIAL; ++a) {
          if (s_w[k * MAX_SPATIAL + a] == 0.0 && a > 0) continue;
          const int64_t cv = fv[(int64_t)t * n_s + s_v[k * MAX_SPATIAL + a]]++;
          vt_obs[cv] = (int)k;
          vt_w[cv] = s_w[k * MAX_SPATIAL + a];
          for (int b = 0; b < MAX_SPATIAL; ++b) {
            if (s_w[k * MAX_SPATIAL + b] == 0.0 && b > 0) continue;
            const int e = pairpos[(k * MAX_SPATIAL + a) * MAX_SPATIAL + b];
            const int64_t c = fs[(int64_t)t * nnz + e]++;
            sp_obs[c] = (int)k;
            sp_w[c] = s_w[k * MAX_SPATIAL + a] * s_w[k * MAX_SPATIAL + b];
          }
        }
      }
    }
    // upload
    M.prow = mdl->upload(prow);
    M.pcol = mdl->upload(pcol);
    M.prow_of = mdl->upload(prow_of);
    M.obs_ptr = mdl->upload(obs_ptr);
    M.obs_t = mdl->upload(s_t);
    M.obs_v = mdl->upload(s_v);
    M.obs_w = mdl->upload(s_w);
    M.obs_z = mdl->upload(s_z);
    M.y = mdl->upload(s_y);
    M.E = s_E.empty() ? nullptr : mdl->upload(s_E);
    M.sp_ptr = mdl->upload(sp_ptr);
    M.sp_obs = mdl->upload(sp_obs);
    M.sp_w = mdl->upload(sp_w);
    M.vt_ptr = mdl->upload(vt_ptr);
    M.vt_obs = mdl->upload(vt_obs);
    M.vt_w = mdl->upload(vt_w);
    std::vector<double> Gval(d->G_val, d->G_val + d->G_rowptr[n_s]), Cd(d->C_diag, d->C_diag + n_s);
    const double *dG = mdl->upload(Gval);
    const double *dC = mdl->upload(Cd);
    const int *dgpos = mdl->upload(gpos);
    const int64_t *dhptr = mdl->upload(hcnt);
    const int *dhk = mdl->upload(hk), *dhik = mdl->upload(hik), *dhkj = mdl->upload(hkj);
    double *vC = mdl->dalloc<double>(nnz), *vG = mdl->dalloc<double>(nnz), *vH = mdl->dalloc<double>(nnz);
    M.vC = vC; M.vG = vG; M.vH = vH;
    double *consts = mdl->dalloc<double>(4);
    M.consts = consts;
    CUDA_OK(cudaStreamCreateWithFlags(&mdl->stream, cudaStreamNonBlocking));
    CUDA_OK(cudaStreamCreateWithFlags(&mdl->stream2, cudaStreamNonBlocking));
    CUDA_OK(cudaStreamCreateWithFlags(&mdl->stream3, cudaStreamNonBlocking));
    CUDA_OK(cudaStreamCreateWithFlags(&mdl->stream4, cudaStreamNonBlocking));
    for (cudaEvent_t *e : {&mdl->ev_fork2, &mdl->ev_join2, &mdl->ev_gfork, &mdl->ev_gjoin})
      CUDA_OK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    CUDA_OK(cudaEventCreateWithFlags(&mdl->ev_fork, cudaEventDisableTiming));
    CUDA_OK(cudaEventCreateWithFlags(&mdl->ev_join, cudaEventDisableTiming));
    CUDA_OK(cudaEventCreateWithFlags(&mdl->done, cudaEventDisableTiming));
    setup_theta_free(mdl->stream, M, dhptr, dhk, dhik, dhkj, dG, dC, dgpos, vC, vG, vH);
    setup_consts(mdl->stream, M, consts);
    if (d->lik == INLA_LIK_GAUSSIAN) {
      double *AtA = mdl->dalloc<double>((size_t)n_t * nnz);
      double *Arw = mdl->dalloc<double>((size_t)n_t * n_b * n_s);
      double *Tip = mdl->dalloc<double>((size_t)n_b * n_b);
      double *Aty = mdl->dalloc<double>((size_t)M.nv);
      double *tippart = mdl->dalloc<double>((size_t)n_t * (n_b * n_b + n_b));
      M.AtA = AtA; M.Arw = Arw; M.Tip = Tip; M.Aty = Aty;
      setup_gaussian(mdl->stream, M, AtA, Arw, Tip, Aty, tippart);
    }
    CUDA_OK(cudaGetLastError());
    CUDA_OK(cudaStreamSynchronize(mdl->stream));
    // Commit the no-allocation entry point's static array on this device now: with lazy
    // module loading its device memory is only backed when the address is first taken,
    // which must not happen inside inla_eval_batch_static.
    static_scratch(device);
    dense_prepare();
    prefer_shared(point_out_kernel);
    prefer_shared(flags_kernel);
    prefer_shared(mask_failed_kernel);
    prefer_shared(zero_slot_kernel);
    return mdl;
  } catch (...) {
    delete mdl;
    throw;
  }
}

// ------------------------------------------------------------------ workspace

struct Layout {
  int64_t per_point_bytes = 0;
  std::vector<std::pair<int64_t *, int64_t>> fields;  // (stride slot, count)
};

// Per-point element counts (doubles unless stated); each padded to 256 bytes.
struct Sizes {
  int64_t theta, prm, qs, Dinv, Rt, Da, vec, wv, mat, nbnp, gjP, gjCO, sc, pt, part, tippart;
  int64_t m, AtAp, Arwp, ints;
};

Sizes sizes_of(const DevModel &M) {  // element counts per point
  Sizes s{};
  const int64_t np = M.n_p, nb = M.n_b;
  s.theta = 32;
  s.prm = rup((int64_t)sizeof(PointParams), 256) / 8;
  s.qs = rup(M.nnz, 32);
  s.Dinv = (int64_t)M.n_t * np * np;
  s.Rt = rup((int64_t)M.n_t * nb * np, 32);
  s.Da = rup(nb * nb, 32) + 32;
  s.vec = rup(M.nv, 32);
  s.wv = rup((1 + nb) * np, 32);
  s.mat = np * np;
  s.nbnp = rup(nb * np, 32) + 32;
  s.gjP = 2 * TILE * TILE;
  s.gjCO = np * TILE;
  s.sc = 32;
  s.pt = rup((int64_t)M.n_t * PT_COUNT, 32);
  s.part = NPART * PART_W;
  s.tippart = rup((int64_t)M.n_t * (nb * nb + nb), 32) + 32;
  s.ints = 32;
  if (M.lik != INLA_LIK_GAUSSIAN) {
    s.m = rup(M.m, 32);
    s.AtAp = rup((int64_t)M.n_t * M.nnz, 32);
    s.Arwp = rup((int64_t)M.n_t * nb * M.n_s, 32) + 32;
  }
  return s;
}

// Scratch of the second elimination chain (Work::c2): the dense scratch blocks, the
// operand buffers of the tensor-core products, the sweep scratch, the arrow rows,
// the tip accumulator, the scalars, two vectors, the selected inversion's arrow
// blocks and partial sums.
int64_t chain2_bytes(const DevModel &M, int rb, bool mixed) {
  const Sizes s = sizes_of(M);
  const int64_t d = s.wv + s.Da + s.sc + 2 * s.vec + s.gjP + 2 * s.gjCO + 3 * s.nbnp + s.part;
  const int64_t split = (mixed && M.n_p % 128 == 0) ? 6 * s.mat * 4 : 0;
  const int64_t digits = (rb == 8 && M.n_p % 128 == 0) ? 2 * (OZ_SLICES * s.mat * 2 + 4 * (int64_t)M.n_p) : 0;
  return d * 8 + 4 * s.mat * rb + split + digits + 24 * 256;
}

// rb: bytes per element of the dense blocks' storage (8 = FP64, 4 = mixed
// precision; 8 also for mixed precision with an FP64 selected inversion);
// mixed: the TF32 hi / lo operand arrays of the FP32 tensor-core products exist;
// chain2: the scratch of a second elimination chain exists.
int64_t point_bytes(const DevModel &M, int rb, bool mixed, bool chain2) {
  const Sizes s = sizes_of(M);
  int64_t d = s.theta + s.prm + s.qs + s.Rt + 2 * s.Da + 7 * s.vec + s.wv + 3 * s.nbnp + s.sc + s.pt + s.part +
              s.tippart + 7 * s.ints + 1;
  if (M.lik != INLA_LIK_GAUSSIAN) d += 4 * s.m + s.AtAp + s.Arwp;
  d += s.gjP + 2 * s.gjCO + s.mat;   // sweep scratch (sized for double) and the FP64 Q_s^-1
  const int64_t split = (mixed && M.n_p % 128 == 0) ? 6 * s.mat * 4 : 0;   // TF32 hi / lo operands (bytes)
  const int64_t dense = s.Dinv + 4 * s.mat;
  // BF16 digit slices and row exponents of the FP64 tensor-core products' two operands
  const int64_t digits = (rb == 8 && M.n_p % 128 == 0) ? 2 * (OZ_SLICES * s.mat * 2 + 4 * (int64_t)M.n_p) : 0;
  return d * 8 + rup(dense * rb, 256) + split + digits + 64 * 256 +   // slack: each array starts on 256 bytes
         (chain2 ? chain2_bytes(M, rb, mixed) : 0);
}

Work carve(const DevModel &M, void *base, int Pw, int rb, bool mixed, bool chain2) {
  const Sizes s = sizes_of(M);
  Work W{};
  W.rb = rb;
  char *p = static_cast<char *>(base);
  auto take = [&](int64_t per) {
    char *r = p;
    p += rup((int64_t)per * Pw * 8, 256);
    return reinterpret_cast<double *>(r);
  };
  auto take_r = [&](int64_t per) {   // dense block storage, element size rb
    char *r = p;
    p += rup((int64_t)per * Pw * rb, 256);
    return static_cast<void *>(r);
  };
  W.theta = take(s.theta);
  W.prm = reinterpret_cast<PointParams *>(take(s.prm));
  W.qs = take(s.qs); W.sNnz = s.qs;
  W.Dinv = take_r(s.Dinv); W.sDinv = s.Dinv;
  W.Rt = take(s.Rt); W.sRt = s.Rt;
  W.Da = take(s.Da); W.sNb2 = s.Da;
  W.Tipp = take(s.Da);
  W.rhs = take(s.vec); W.zf = take(s.vec); W.x = take(s.vec); W.xprev = take(s.vec); W.tmpv = take(s.vec);
  W.rvec = take(s.vec); W.dvec = take(s.vec);
  W.sVec = s.vec;
  W.wv = take(s.wv); W.sWV = s.wv;
  W.T1 = take_r(s.mat); W.S = take_r(s.mat); W.SigN = take_r(s.mat); W.SigC = take_r(s.mat); W.sMat = s.mat;
  if (mixed && M.n_p % 128 == 0) {
    float **parts[6] = {&W.Dh, &W.Dl, &W.Sh, &W.Sl, &W.Uh, &W.Ul};
    for (float **q : parts) {
      *q = reinterpret_cast<float *>(p);
      p += rup((int64_t)s.mat * Pw * 4, 256);
    }
  }
  if (rb == 8 && M.n_p % 128 == 0) {
    auto take_b = [&](int64_t bytes) {   // bytes per point
      char *r = p;
      p += rup(bytes * Pw, 256);
      return static_cast<void *>(r);
    };
    W.sZ = OZ_SLICES * s.mat;
    W.sE = M.n_p;
    W.Zd = static_cast<uint16_t *>(take_b(W.sZ * 2));
    W.Zs = static_cast<uint16_t *>(take_b(W.sZ * 2));
    W.Ed = static_cast<int32_t *>(take_b(W.sE * 4));
    W.Es = static_cast<int32_t *>(take_b(W.sE * 4));
  }
  W.SigAn = take(s.nbnp); W.SigAc = take(s.nbnp); W.Y = take(s.nbnp); W.sNbNp = s.nbnp;
  W.gjP = take(s.gjP); W.gjC = take(s.gjCO); W.gjO = take(s.gjCO);
  W.QsI = take(s.mat);
  W.sc = take(s.sc);
  W.pt = take(s.pt); W.sPt = s.pt;
  W.part = take(s.part);
  W.tippart = take(s.tippart);
  W.status = reinterpret_cast<int *>(take(s.ints));
  W.active = reinterpret_cast<int *>(take(s.ints));
  W.flags = reinterpret_cast<int *>(take(s.ints));
  W.iters = reinterpret_cast<int *>(take(s.ints));
  W.qsrep = reinterpret_cast<int *>(take(s.ints));
  W.any_active = reinterpret_cast<int *>(take(1));
  W.grp0 = reinterpret_cast<int *>(take(s.ints));
  W.grp1 = reinterpret_cast<int *>(take(s.ints));
  if (M.lik != INLA_LIK_GAUSSIAN) {
    W.eta = take(s.m); W.mu = take(s.m); W.qobs = take(s.m); W.wobs = take(s.m); W.sM = s.m;
    W.AtAp = take(s.AtAp); W.sAtAp = s.AtAp;
    W.Arwp = take(s.Arwp); W.sArwp = s.Arwp;
  }
  if (chain2) {   // the same shapes and strides as the first chain's arrays
    Work::Chain2 &c = W.c2;
    c.T1 = take_r(s.mat); c.S = take_r(s.mat); c.SigN = take_r(s.mat); c.SigC = take_r(s.mat);
    if (mixed && M.n_p % 128 == 0) {
      float **parts[6] = {&c.Dh, &c.Dl, &c.Sh, &c.Sl, &c.Uh, &c.Ul};
      for (float **q : parts) {
        *q = reinterpret_cast<float *>(p);
        p += rup((int64_t)s.mat * Pw * 4, 256);
      }
    }
    if (rb == 8 && M.n_p % 128 == 0) {
      auto take_b = [&](int64_t bytes) {
        char *r = p;
        p += rup(bytes * Pw, 256);
        return static_cast<void *>(r);
      };
      c.Zd = static_cast<uint16_t *>(take_b(W.sZ * 2));
      c.Zs = static_cast<uint16_t *>(take_b(W.sZ * 2));
      c.Ed = static_cast<int32_t *>(take_b(W.sE * 4));
      c.Es = static_cast<int32_t *>(take_b(W.sE * 4));
    }
    c.wv = take(s.wv); c.Da = take(s.Da); c.sc = take(s.sc); c.zf = take(s.vec); c.tmpv = take(s.vec);
    c.gjP = take(s.gjP); c.gjC = take(s.gjCO); c.gjO = take(s.gjCO);
    c.SigAn = take(s.nbnp); c.SigAc = take(s.nbnp); c.Y = take(s.nbnp); c.part = take(s.part);
  }
  W.P = Pw;
  return W;
}

// The workspace of the second elimination chain: W with its scratch replaced by W.c2.
// Everything per time block (D_t^-1, R~_t) and per point (parameters, status) is shared:
// the two chains touch disjoint time blocks.
Work chain2_work(const Work &W) {
  Work V = W;
  const Work::Chain2 &c = W.c2;
  V.T1 = c.T1; V.S = c.S; V.SigN = c.SigN; V.SigC = c.SigC;
  V.Dh = c.Dh; V.Dl = c.Dl; V.Sh = c.Sh; V.Sl = c.Sl; V.Uh = c.Uh; V.Ul = c.Ul;
  V.Zd = c.Zd; V.Zs = c.Zs; V.Ed = c.Ed; V.Es = c.Es;
  V.wv = c.wv; V.Da = c.Da; V.sc = c.sc; V.zf = c.zf; V.tmpv = c.tmpv;
  V.gjP = c.gjP; V.gjC = c.gjC; V.gjO = c.gjO;
  V.SigAn = c.SigAn; V.SigAc = c.SigAc; V.Y = c.Y; V.part = c.part;
  return V;
}

// The per-point layout above uses stride = count for each array, so that the
// stride of point b is the count; sc, pt and Tipp use fixed strides.
static_assert(SC_COUNT <= 32, "sc slots");

int64_t point_bytes_for(const DevModel &M, const inla_eval_opts &o);

int wave_points(inla_model *mdl, int64_t P_total, const inla_eval_opts &o) {
  const int64_t per = point_bytes_for(mdl->M, o);
  size_t free_b = 0, total_b = 0;
  CUDA_OK(cudaMemGetInfo(&free_b, &total_b));
  const int64_t avail = (int64_t)free_b + (int64_t)mdl->ws_bytes - (int64_t)(2ll << 30);
  int64_t cap = avail / per;
  if (cap < 1) throw ApiError(INLA_ERR_OOM, "not enough device memory for one evaluation point");
  return (int)std::min<int64_t>(P_total, std::min<int64_t>(cap, 65535));
}

void ensure_workspace(inla_model *mdl, int Pw, const inla_eval_opts &o) {
  const size_t need = (size_t)point_bytes_for(mdl->M, o) * Pw;
  if (mdl->ws && mdl->ws_bytes >= need) return;
  if (mdl->ws) {
    CUDA_OK(cudaStreamSynchronize(mdl->stream));
    CUDA_OK(cudaDeviceSynchronize());
    cudaFree(mdl->ws);
    mdl->ws = nullptr;
    mdl->ws_bytes = 0;
  }
  CUDA_OK(cudaMalloc(&mdl->ws, need));
  mdl->ws_bytes = need;
  mdl->ws_points = Pw;
}

struct BatchBufs {
  double *theta_all, *f_all, *grad_all;
  int *point_out, *status_all, *iters_all;
};

BatchBufs batch_buffers(inla_model *mdl, int64_t P_total) {
  const int64_t per = rup(4 * 8, 256) + rup(8, 256) + rup(32, 256) + 3 * rup(4, 256);
  const size_t need = (size_t)per * P_total + 4096;
  if (!mdl->bb || mdl->bb_bytes < need) {
    if (mdl->bb) {
      CUDA_OK(cudaDeviceSynchronize());
      cudaFree(mdl->bb);
      mdl->bb = nullptr;
    }
    CUDA_OK(cudaMalloc(&mdl->bb, need));
    mdl->bb_bytes = need;
  }
  char *p = static_cast<char *>(mdl->bb);
  auto take = [&](int64_t bytes) {
    char *r = p;
    p += rup(bytes * P_total, 256);
    return r;
  };
  BatchBufs b;
  b.theta_all = reinterpret_cast<double *>(take(32));
  b.f_all = reinterpret_cast<double *>(take(8));
  b.grad_all = reinterpret_cast<double *>(take(32));
  b.point_out = reinterpret_cast<int *>(take(4));
  b.status_all = reinterpret_cast<int *>(take(4));
  b.iters_all = reinterpret_cast<int *>(take(4));
  return b;
}

// ------------------------------------------------------------------ phases

void zero_slot(Launch &L, const Work &W, int slot) {
  zero_slot_kernel<<<(W.P + 63) / 64, 64, 0, L.st>>>(W, slot);
  L.tick();
}

// The second elimination chain runs on L.st2, forked from L.st and joined back.
Launch chain2_launch(const Launch &L) {
  Launch L2 = L;
  L2.st = L.st2;
  L2.cur_id = -1;
  return L2;
}
void fork_chain2(const Launch &L) {
  CUDA_OK(cudaEventRecord(L.ev_fork, L.st));
  CUDA_OK(cudaStreamWaitEvent(L.st2, L.ev_fork, 0));
}
void join_chain2(const Launch &L) {
  CUDA_OK(cudaEventRecord(L.ev_join, L.st2));
  CUDA_OK(cudaStreamWaitEvent(L.st, L.ev_join, 0));
}

// One elimination step of the time chain: block t with its Schur complement from
// the neighbour `prev` eliminated just before it (-1: none), D_t^-1 and log|D_t|.
// R~_t = R_t - q_off (R~_prev D_prev^-1) Q_s and D_a -= (R~_prev D_prev^-1) R~_prev^T.
template <typename R>
void chain_step(Launch &L, const DevModel &M, const Work &W, int mode, int ld_slot, int t, int prev) {
  const int64_t np2 = (int64_t)M.n_p * M.n_p;
  const int64_t rtb = (int64_t)M.n_b * M.n_p;
  R *Dinv = static_cast<R *>(W.Dinv);
  R *Dt = Dinv + t * np2;
  if (prev >= 0) {
    const R *Dp = Dinv + prev * np2;
    if (M.n_b > 0) {
      k_dinv_apply(L, M, W, Dp, M.n_b, W.Rt + prev * rtb, W.sRt, W.wv, W.sWV, 1.0);
      k_arrow_update(L, M, W, t, mode);
      k_arrow_dots(L, M, W, prev);
    }
    k_sparse_right<R>(L, M, W, Dp, W.sDinv, static_cast<R *>(W.T1), W.sMat, false, nullptr, nullptr, true);
  }
  k_assemble_diag<R>(L, M, W, t, mode, Dt, W.sDinv, prev >= 0);
  gj_invert<R>(L, M, W, Dt, W.sDinv, W.sc + ld_slot, SC_COUNT);
}

// The contributions of the last block `last` of a chain to the separator: its arrow
// rows V = R~_last D_last^-1 (in W.wv) with D_a -= V R~_last^T, and T1 = D_last^-1 Q_s.
template <typename R>
void chain_close(Launch &L, const DevModel &M, const Work &W, int last) {
  const int64_t np2 = (int64_t)M.n_p * M.n_p;
  const int64_t rtb = (int64_t)M.n_b * M.n_p;
  const R *Dl = static_cast<const R *>(W.Dinv) + last * np2;
  if (M.n_b > 0) {
    k_dinv_apply(L, M, W, Dl, M.n_b, W.Rt + last * rtb, W.sRt, W.wv, W.sWV, 1.0);
    k_arrow_dots(L, M, W, last);
  }
  k_sparse_right<R>(L, M, W, Dl, W.sDinv, static_cast<R *>(W.T1), W.sMat, false, nullptr, nullptr, true);
}

// Separator block of a time chain split in two: the middle block.
inline int separator(const DevModel &M) { return M.n_t / 2; }

// Block LDL^T factorisation of Q_c (mode ASM_QC) or Q (ASM_Q) along the time chain.
// split: nested dissection of the chain at the middle block k (Sec. 3.3): blocks
// 0..k-1 and n_t-1..k+1 are eliminated as two independent chains, concurrently on two
// streams, each towards k; then k with the Schur complements of both neighbours,
//   D_k = A_k - q_off^2 Q_s (D_{k-1}^-1 + D_{k+1}^-1) Q_s,
// and the tip with the arrow updates of every block.  No fill: every block still has
// one later-eliminated neighbour in the chain (k has none), and log|Q_c| is the sum of
// the same log|D_t| over the new order.
template <typename R>
void factor(Launch &L, const DevModel &M, const Work &W, int mode, int ld_slot, bool split = false) {
  zero_slot(L, W, ld_slot);
  k_init_step0(L, M, W, mode, 0, true);
  if (!split) {
    for (int t = 0; t < M.n_t; ++t) chain_step<R>(L, M, W, mode, ld_slot, t, t - 1);
    if (M.n_b > 0) {
      const int64_t np2 = (int64_t)M.n_p * M.n_p;
      const int t = M.n_t - 1;
      k_dinv_apply<R>(L, M, W, static_cast<R *>(W.Dinv) + t * np2, M.n_b, W.Rt + t * (int64_t)M.n_b * M.n_p,
                      W.sRt, W.wv, W.sWV, 1.0);
      k_arrow_dots(L, M, W, t);
    }
    k_tip(L, M, W, ld_slot);
    return;
  }
  const int k = separator(M), last = M.n_t - 1;
  const Work W2 = chain2_work(W);
  Launch L2 = chain2_launch(L);
  fork_chain2(L);
  zero_slot(L2, W2, ld_slot);
  k_init_step0(L2, M, W2, mode, last, false);   // R~_{n_t-1} = R_{n_t-1}; the tip accumulator = 0
  for (int t = last; t > k; --t) chain_step<R>(L2, M, W2, mode, ld_slot, t, t < last ? t + 1 : -1);
  chain_close<R>(L2, M, W2, k + 1);
  for (int t = 0; t < k; ++t) chain_step<R>(L, M, W, mode, ld_slot, t, t - 1);
  chain_close<R>(L, M, W, k - 1);
  join_chain2(L);
  // the separator: both neighbours' Schur products and arrow rows
  k_add_into<R>(L, W.P, static_cast<R *>(W.T1), static_cast<const R *>(W2.T1), W.sMat, W.sMat, W.active);
  if (M.n_b > 0) {
    k_add_into<double>(L, W.P, W.wv, W2.wv, W.sWV, (int64_t)M.n_b * M.n_p, W.active);
    k_arrow_update(L, M, W, k, mode);
  }
  const int64_t np2 = (int64_t)M.n_p * M.n_p;
  R *Dk = static_cast<R *>(W.Dinv) + k * np2;
  k_assemble_diag<R>(L, M, W, k, mode, Dk, W.sDinv, true);
  gj_invert<R>(L, M, W, Dk, W.sDinv, W.sc + ld_slot, SC_COUNT);
  k_join_tip(L, M, W, W2.Da, W2.sc, ld_slot);
  if (M.n_b > 0) {
    k_dinv_apply<R>(L, M, W, Dk, M.n_b, W.Rt + k * (int64_t)M.n_b * M.n_p, W.sRt, W.wv, W.sWV, 1.0);
    k_arrow_dots(L, M, W, k);
  }
  k_tip(L, M, W, ld_slot);
}

// Forward and backward block substitution with the stored factorisation.  Block t's
// forward step w = D_t^-1 z_t, z_nbr -= q_off Q_s w, z_a -= R~_t w passes to the
// neighbour eliminated after t; the backward step x_t = D_t^-1 (z_t - q_off Q_s x_nbr -
// R~_t^T x_a) reads it.  split: the order of the split factorisation above (the two
// chains concurrently, the separator and the tip between the passes).
template <typename R>
void solve_once(Launch &L, const DevModel &M, const Work &W, const double *rhs, double *x, bool split) {
  const int64_t np2 = (int64_t)M.n_p * M.n_p;
  const R *Dinv = static_cast<const R *>(W.Dinv);
  // only the points of this pass: a concurrent pass of another point group owns the rest
  const int lo = W.hi > 0 ? W.lo : 0, hi = W.hi > 0 ? W.hi : W.P;
  const int64_t voff = (int64_t)lo * W.sVec;
  const size_t vbytes = sizeof(double) * W.sVec * (size_t)(hi - lo);
  CUDA_OK(cudaMemcpyAsync(W.zf + voff, rhs + voff, vbytes, cudaMemcpyDeviceToDevice, L.st));
  auto fwd = [&](Launch &Ls, const Work &Ws, int t, int nbr) {
    k_dinv_apply<R>(Ls, M, Ws, Dinv + t * np2, 1, Ws.zf + (int64_t)t * M.n_p, Ws.sVec, Ws.wv, Ws.sWV, 1.0);
    k_fwd_update(Ls, M, Ws, t, nbr, Ws.zf);
  };
  auto bwd = [&](Launch &Ls, const Work &Ws, int t, int nbr) {
    k_bwd_rhs(Ls, M, Ws, t, nbr, Ws.zf, x);
    k_dinv_apply<R>(Ls, M, Ws, Dinv + t * np2, 1, Ws.tmpv, Ws.sVec, x + (int64_t)t * M.n_p, Ws.sVec, 1.0);
  };
  if (!split) {
    for (int t = 0; t < M.n_t; ++t) fwd(L, W, t, t + 1 < M.n_t ? t + 1 : -1);
    k_tip_solve(L, M, W, W.zf, x);
    for (int t = M.n_t - 1; t >= 0; --t) bwd(L, W, t, t + 1 < M.n_t ? t + 1 : -1);
    return;
  }
  const int k = separator(M), last = M.n_t - 1;
  const Work W2 = chain2_work(W);
  Launch L2 = chain2_launch(L);
  fork_chain2(L);
  CUDA_OK(cudaMemcpyAsync(W2.zf + voff, rhs + voff, vbytes, cudaMemcpyDeviceToDevice, L2.st));
  for (int t = last; t > k; --t) fwd(L2, W2, t, t - 1);
  for (int t = 0; t < k; ++t) fwd(L, W, t, t + 1);
  join_chain2(L);
  k_join_rhs(L, M, W, k, W.zf, W2.zf, rhs);
  fwd(L, W, k, -1);
  k_tip_solve(L, M, W, W.zf, x);
  bwd(L, W, k, -1);
  fork_chain2(L);
  for (int t = k + 1; t <= last; ++t) bwd(L2, W2, t, t - 1);
  for (int t = k - 1; t >= 0; --t) bwd(L, W, t, t + 1);
  join_chain2(L);
}

// Q_c x = rhs.  With single-precision blocks the solution is refined with FP64
// residuals r = rhs - Q_c x computed from the sparse blocks (x += Q_c^-1 r).
constexpr int REFINE_STEPS = 3;
template <typename R>
void solve(Launch &L, const DevModel &M, const Work &W, const double *rhs, double *x, bool split = false) {
  solve_once<R>(L, M, W, rhs, x, split);
  if (sizeof(R) == sizeof(double)) return;
  for (int it = 0; it < REFINE_STEPS; ++it) {
    k_qc_residual(L, M, W, x, rhs, W.rvec);
    solve_once<R>(L, M, W, W.rvec, W.dvec, split);
    k_axpy(L, M, W, x, W.dvec);
  }
}

// The FP32 selected-inversion products run on the tensor cores when asked
// for and the padded block size is a multiple of their 128-wide tiles.
template <typename R>
bool tensor_gemm(const DevModel &M) {
  return sizeof(R) == sizeof(float) && M.gemm_t32 == INLA_GEMM_TF32X3 && M.n_p % 128 == 0;
}

// INLA_MIXED on meshes finer than this: the selected inversion (marginal
// variances, the adjoint's traces) runs on an FP64 factorisation at the mode,
// and the workspace is carved for FP64 blocks.  FP32 blocks carry errors of
// order kappa(D_t) 2^-24, and kappa(Q_s) of the alpha = 2 SPDE grows like h^-4:
// on the 64 x 64 mesh the FP32 selected inverse missed the mixed form's budget
// (gradient 3.4e-4, variances 1e-4) while f and the refined mode kept theirs.
constexpr int MIXED_FP64_SELINV_NS = 3000;

bool mixed_fp64_selinv(const DevModel &M, const inla_eval_opts &o) {
  return o.precision == INLA_MIXED && (o.want_marg_var || o.grad == INLA_GRAD_ADJOINT) &&
         M.n_s > MIXED_FP64_SELINV_NS;
}

// Bytes per element of the workspace's dense blocks for these options.
int workspace_rb(const DevModel &M, const inla_eval_opts &o) {
  return (o.precision == INLA_MIXED && !mixed_fp64_selinv(M, o)) ? 4 : 8;
}

// Whether this call's factorisations, substitutions and selected inversions split
// the time chain in two (nested dissection at the middle block).
bool split_chain(const DevModel &M, const inla_eval_opts &) {
  return M.time_parts >= 2 && M.n_t >= 3;
}

int64_t point_bytes_for(const DevModel &M, const inla_eval_opts &o) {
  return point_bytes(M, workspace_rb(M, o), o.precision == INLA_MIXED, split_chain(M, o));
}

Work carve_for(const DevModel &M, void *base, int Pw, const inla_eval_opts &o) {
  Work W = carve(M, base, Pw, workspace_rb(M, o), o.precision == INLA_MIXED, split_chain(M, o));
  W.rb = o.precision == INLA_MIXED ? 4 : 8;   // the dense blocks' arithmetic (an FP64-sized workspace may hold FP32 blocks)
  return W;
}

// The FP64 selected-inversion products run on the BF16 tensor cores (digit
// splitting, ozaki.cu) when enabled and the padded block size is a multiple of 128.
template <typename R>
bool digit_gemm(const DevModel &M) {
  return sizeof(R) == sizeof(double) && M.f64_tensor && M.n_p % 128 == 0;
}

// Block Takahashi recursion (Eq. takahashi_recursion in block form) in the reverse
// of the elimination order: one step for block t, whose neighbour eliminated after
// it is `next` (-1: none) with Sigma_{next,next} and Sigma_{a,next} in W.SigN and
// W.SigAn; Sigma_tt and Sigma_{a,t} land in W.SigC and W.SigAc, then the pairs swap.
template <typename R>
void selinv_step(Launch &L, const DevModel &M, Work &W, int mode, bool contractions, double *marg_var,
                 const int *point_out, int64_t point_base, bool poisson_q, int t, int next) {
  const int64_t np2 = (int64_t)M.n_p * M.n_p;
  const int64_t rtb = (int64_t)M.n_b * M.n_p;
  const int slotD = (mode == ASM_QC) ? PT_FD_C : PT_QD_C;
  const int slotO = (mode == ASM_QC) ? PT_FO_C : PT_QO_C;
  const R *Dinv = static_cast<const R *>(W.Dinv);
  R *T1 = static_cast<R *>(W.T1);
  R *S = static_cast<R *>(W.S);
  const R *Dt = Dinv + t * np2;
  const double *Rt_t = W.Rt + t * rtb;
  const bool nxt = next >= 0;
  R *SigN = static_cast<R *>(W.SigN), *SigC = static_cast<R *>(W.SigC);
  if (nxt) k_sparse_right<R>(L, M, W, SigN, W.sMat, T1, W.sMat, true, M.n_b ? W.SigAn : nullptr, Rt_t);
  k_selinv_Y(L, M, W, t, nxt);
  k_sparse_left<R>(L, M, W, T1, W.sMat, S, W.sMat, nxt, Rt_t, M.n_b ? W.Y : nullptr);
  if (contractions && nxt) k_contract_offdiag<R>(L, M, W, t, std::min(t, next), slotO);
  if (M.n_b > 0) k_dinv_apply<R>(L, M, W, Dt, M.n_b, W.Y, W.sNbNp, W.SigAc, W.sNbNp, -1.0);
  if (tensor_gemm<R>(M)) {
    // U = D^-1 S^T (= (S D^-1)^T, D^-1 symmetric), then Sigma_tt = D^-1 U^T + D^-1:
    // both products read their operands along rows (X Y^T), as the tensor-core kernel wants.
    // D^-1 and S are split into TF32 hi / lo parts once; U is stored split by the first product.
    const float *Df = reinterpret_cast<const float *>(Dt);
    split_tf32(L, W.P, Df, W.sDinv, W.Dh, W.Dl, W.sMat, np2, W.active);
    split_tf32(L, W.P, reinterpret_cast<const float *>(S), W.sMat, W.Sh, W.Sl, W.sMat, np2, W.active);
    const int n = M.n_p;
    gemm_nt_tf32x3_split(L, W.P, n, n, n, W.Dh, W.Dl, W.sMat, W.Sh, W.Sl, W.sMat, nullptr, n, W.sMat, 1.0f, nullptr,
                         n, 0, 0.0f, W.Uh, W.Ul, false, W.active, W.status);
    gemm_nt_tf32x3_split(L, W.P, n, n, n, W.Dh, W.Dl, W.sMat, W.Uh, W.Ul, W.sMat, reinterpret_cast<float *>(SigC), n,
                         W.sMat, 1.0f, Df, n, W.sDinv, 1.0f, nullptr, nullptr, true, W.active, W.status);
  } else if (digit_gemm<R>(M)) {
    // the same two products in FP64 through BF16 digit slices: U = D^-1 S^T into T1, then
    // Sigma_tt = D^-1 U^T + D^-1; D^-1 is split once, S's slices are replaced by U's
    const double *Dd = reinterpret_cast<const double *>(Dt);
    double *Ud = reinterpret_cast<double *>(T1);
    const int n = M.n_p;
    ozaki_split2(L, W.P, n, n, Dd, n, W.sDinv, W.Zd, W.Ed, n, n, reinterpret_cast<const double *>(S), n, W.sMat,
                 W.Zs, W.Es, W.sZ, W.sE, W.active);
    gemm_nt_ozaki(L, W.P, n, n, n, W.Zd, W.sZ, W.Ed, W.sE, W.Zs, W.sZ, W.Es, W.sE, Ud, n, W.sMat, 1.0, nullptr, 0,
                  0, 0.0, false, W.active, W.status);
    ozaki_split(L, W.P, n, n, Ud, n, W.sMat, W.Zs, W.sZ, W.Es, W.sE, W.active);
    gemm_nt_ozaki(L, W.P, n, n, n, W.Zd, W.sZ, W.Ed, W.sE, W.Zs, W.sZ, W.Es, W.sE,
                  reinterpret_cast<double *>(SigC), n, W.sMat, 1.0, Dd, n, W.sDinv, 1.0, true, W.active, W.status);
  } else {
    const int tile = M.gemm_t32 == INLA_GEMM_TF32X3 ? 128 : M.gemm_t32;   // CUDA-core fallback
    gemm_nn<R>(L, W.P, M.n_p, S, W.sMat, Dt, W.sDinv, T1, W.sMat, R(1), nullptr, 0, R(0), false, W.active, tile);
    gemm_nn<R>(L, W.P, M.n_p, Dt, W.sDinv, T1, W.sMat, SigC, W.sMat, R(1), Dt, W.sDinv, R(1), true, W.active,
               tile);
  }
  mirror_lower<R>(L, W.P, M.n_p, SigC, W.sMat, W.active);
  k_contract_diag<R>(L, M, W, t, mode, mode == ASM_QC ? marg_var : nullptr, point_out, point_base, slotD);
  if (poisson_q) k_poisson_qobs<R>(L, M, W, t);
  std::swap(W.SigN, W.SigC);
  std::swap(W.SigAn, W.SigAc);
}

// The selected inverse on the BTA pattern from the last-eliminated block outwards.
// split: the order of the split factorisation (Sec. 3.3: the separator's entries
// first, then the two independent parts concurrently): block k, then k-1..0 and
// k+1..n_t-1 on two streams, the second chain starting from a copy of Sigma_kk and
// Sigma_{a,k}.
template <typename R>
void selinv(Launch &L, const DevModel &M, const Work &W0, int mode, bool contractions, double *marg_var,
            const int *point_out, int64_t point_base, bool poisson_q, bool split = false) {
  Work W = W0;
  auto step = [&](Launch &Ls, Work &Ws, int t, int next) {
    selinv_step<R>(Ls, M, Ws, mode, contractions, marg_var, point_out, point_base, poisson_q, t, next);
  };
  if (!split) {
    for (int t = M.n_t - 1; t >= 0; --t) step(L, W, t, t + 1 < M.n_t ? t + 1 : -1);
  } else {
    const int k = separator(M), last = M.n_t - 1;
    step(L, W, k, -1);
    Work W2 = chain2_work(W);
    W2.Da = W.Da;   // Sigma_a (the second chain's scratch holds its factorisation's tip accumulator)
    CUDA_OK(cudaMemcpyAsync(W2.SigN, W.SigN, sizeof(R) * W.sMat * W.P, cudaMemcpyDeviceToDevice, L.st));
    if (M.n_b > 0)
      CUDA_OK(cudaMemcpyAsync(W2.SigAn, W.SigAn, sizeof(double) * W.sNbNp * W.P, cudaMemcpyDeviceToDevice, L.st));
    Launch L2 = chain2_launch(L);
    fork_chain2(L);
    for (int t = k + 1; t <= last; ++t) step(L2, W2, t, t - 1);
    for (int t = k - 1; t >= 0; --t) step(L, W, t, t + 1);
    join_chain2(L);
  }
  k_contract_tip(L, M, W, mode, mode == ASM_QC ? marg_var : nullptr, point_out, point_base);
}

// The model's second stream and fork / join events for the second elimination chain.
void with_chain2(inla_model *mdl, Launch &L) {
  L.st2 = mdl->stream2;
  L.ev_fork = mdl->ev_fork;
  L.ev_join = mdl->ev_join;
  L.gst = mdl->stream3;
  L.gst2 = mdl->stream4;
  L.gev_fork = mdl->ev_fork2;
  L.gev_join = mdl->ev_join2;
  L.gev_gfork = mdl->ev_gfork;
  L.gev_gjoin = mdl->ev_gjoin;
}

// Point groups: the first half of the wave's points in grp0, the rest in grp1 (each
// restricted to the points active now).
__global__ void group_mask_kernel(Work W) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= W.P) return;
  const int h = (W.P + 1) / 2, a = W.active[b];
  W.grp0[b] = (a && b < h) ? 1 : 0;
  W.grp1[b] = (a && b >= h) ? 1 : 0;
}

template <typename R>
void run_wave_t(inla_model *mdl, Launch &L, const Work &W, const inla_eval_opts &o, int64_t w0,
                const BatchBufs &bb, double *x_out, double *mv_out, int centre_flags) {
  const DevModel &M = mdl->M;
  const bool adj = o.grad == INLA_GRAD_ADJOINT;
  const bool need_sel = (centre_flags & 1) != 0;
  // mixed precision on a fine mesh: the selected inversion from an FP64 factorisation
  // at the mode, in the same (FP64-sized) workspace
  const bool esc = sizeof(R) == sizeof(float) && need_sel && mixed_fp64_selinv(M, o);
  const bool split = split_chain(M, o) && W.c2.T1 && L.st2;
  Work Wd = W;
  Wd.rb = 8;
  CUDA_OK(cudaMemsetAsync(W.sc, 0, sizeof(double) * 32 * W.P, L.st));
  CUDA_OK(cudaMemsetAsync(W.pt, 0, sizeof(double) * W.sPt * W.P, L.st));
  CUDA_OK(cudaMemsetAsync(W.status, 0, sizeof(int) * W.P, L.st));
  CUDA_OK(cudaMemsetAsync(W.iters, 0, sizeof(int) * W.P, L.st));
  CUDA_OK(cudaMemsetAsync(W.rhs, 0, sizeof(double) * W.sVec * W.P, L.st));
  flags_kernel<<<(W.P + 63) / 64, 64, 0, L.st>>>(W, w0, fd_points_per_centre(o.grad), centre_flags);
  L.tick();
  k_set_active(L, W, 0);
  k_params(L, M, W);
  k_qs_values(L, M, W);
  // prior log-determinant (and traces for the adjoint)
  if (o.prior_mode == INLA_PRIOR_KRONECKER) {
    // one n_s x n_s inversion per distinct range parameter: always in FP64
    k_qs_share_setup(L, W);
    k_assemble_diag<double>(L, M, W, 0, ASM_QS, W.QsI, W.sMat, false);
    gj_invert<double>(L, M, W, W.QsI, W.sMat, W.sc + SC_LOGDET_QS, SC_COUNT);
    if (adj) k_qs_traces(L, M, W);
    k_qs_share(L, M, W);
    k_set_active(L, W, 0);
  } else {
    factor<R>(L, M, W, ASM_Q, SC_LOGDET_Q, split);
    if (adj) {
      k_set_active(L, W, 2);
      if (esc) {
        factor<double>(L, M, Wd, ASM_Q, SC_LOGDET_Q, split);
        selinv<double>(L, M, Wd, ASM_Q, true, nullptr, nullptr, 0, false, split);
      } else {
        selinv<R>(L, M, W, ASM_Q, true, nullptr, nullptr, 0, false, split);
      }
      k_set_active(L, W, 0);
    }
  }
  if (M.lik == INLA_LIK_GAUSSIAN) {
    k_rhs_gaussian(L, M, W);
    if (M.point_groups >= 2 && W.P >= 2 && L.gst && L.capturing) {
      // two point groups, each factorised and solved on its own stream pair: the
      // launches are latency-bound, so two groups of half the points overlap.  Only in a
      // CUDA graph: the groups double the launches, which eager calls pay for on the host
      // (the FD step went from 184 to 254 ms eager while its graph went from 130 to 127 ms)
      group_mask_kernel<<<(W.P + 63) / 64, 64, 0, L.st>>>(W);
      L.tick();
      const int h = (W.P + 1) / 2;
      Work W0 = W, W1 = W;
      W0.active = W.grp0; W0.lo = 0; W0.hi = h;
      W1.active = W.grp1; W1.lo = h; W1.hi = W.P;
      Launch L1 = L;
      L1.st = L.gst; L1.st2 = L.gst2; L1.ev_fork = L.gev_fork; L1.ev_join = L.gev_join;
      L1.cur_id = -1;
      CUDA_OK(cudaEventRecord(L.gev_gfork, L.st));
      CUDA_OK(cudaStreamWaitEvent(L1.st, L.gev_gfork, 0));
      factor<R>(L1, M, W1, ASM_QC, SC_LOGDET_QC, split);
      solve<R>(L1, M, W1, W.rhs, W.x, split);
      factor<R>(L, M, W0, ASM_QC, SC_LOGDET_QC, split);
      solve<R>(L, M, W0, W.rhs, W.x, split);
      CUDA_OK(cudaEventRecord(L.gev_gjoin, L1.st));
      CUDA_OK(cudaStreamWaitEvent(L.st, L.gev_gjoin, 0));
    } else {
      factor<R>(L, M, W, ASM_QC, SC_LOGDET_QC, split);
      solve<R>(L, M, W, W.rhs, W.x, split);
    }
    k_obs_reduce(L, M, W, 0);
    k_quadforms(L, M, W, W.x, W.x, PT_XD_C, SC_TIP_XX);
    if (need_sel) {
      k_set_active(L, W, 1);
      if (esc) {
        factor<double>(L, M, Wd, ASM_QC, SC_LOGDET_QC, split);
        selinv<double>(L, M, Wd, ASM_QC, adj, mv_out, bb.point_out, w0, false, split);
      } else {
        selinv<R>(L, M, W, ASM_QC, adj, mv_out, bb.point_out, w0, false, split);
      }
      k_set_active(L, W, 0);
    }
  } else {
    const int max_it = o.max_newton > 0 ? o.max_newton : 50;
    const double tol = o.newton_tol > 0 ? o.newton_tol : 1e-8;
    CUDA_OK(cudaMemsetAsync(W.x, 0, sizeof(double) * W.sVec * W.P, L.st));
    CUDA_OK(cudaMemsetAsync(W.xprev, 0, sizeof(double) * W.sVec * W.P, L.st));
    auto newton_step = [&](Launch &Ls, int it, const int *it_dev) {
      k_poisson_eta(Ls, M, W, W.x);
      k_obs_assemble(Ls, M, W.P, W.active, W.mu, W.sM, nullptr, 0, true, W.eta, W.AtAp, W.sAtAp, W.Arwp,
                     W.sArwp, W.Tipp, W.sNb2, W.rhs, W.sVec, W.tippart);
      factor<R>(Ls, M, W, ASM_QC, SC_LOGDET_QC, split);
      solve<R>(Ls, M, W, W.rhs, W.x, split);
      k_newton_cap(Ls, M, W);   // no linear predictor moves by more than NEWTON_DETA in one step
      CUDA_OK(cudaMemsetAsync(W.any_active, 0, sizeof(int), Ls.st));
      k_poisson_step(Ls, M, W, tol, it, max_it, it_dev);
    };
    if (L.capturing) {
      // the Newton loop as a while-node of the graph: its body is one iteration for
      // every point of the wave, repeated on the device while any point is active
      int *ctr = W.any_active + 1;   // iterations done (the second int of the slot)
      CUDA_OK(cudaMemsetAsync(ctr, 0, sizeof(int), L.st));
      cudaStreamCaptureStatus cs;
      cudaGraph_t graph = nullptr;
      const cudaGraphNode_t *deps = nullptr;
      size_t ndeps = 0;
      CUDA_OK(cudaStreamGetCaptureInfo(L.st, &cs, nullptr, &graph, &deps, nullptr, &ndeps));
      cudaGraphConditionalHandle h;
      CUDA_OK(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams cp{};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t node;
      CUDA_OK(cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &cp));
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      // the body is captured from streams of its own (the model's second stream may
      // already belong to the enclosing capture)
      cudaStream_t bs, bs2;
      cudaEvent_t bf, bj;
      CUDA_OK(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
      CUDA_OK(cudaStreamCreateWithFlags(&bs2, cudaStreamNonBlocking));
      CUDA_OK(cudaEventCreateWithFlags(&bf, cudaEventDisableTiming));
      CUDA_OK(cudaEventCreateWithFlags(&bj, cudaEventDisableTiming));
      Launch Lb = L;
      Lb.st = bs;
      Lb.st2 = bs2;
      Lb.ev_fork = bf;
      Lb.ev_join = bj;
      cudaError_t e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        try {
          newton_step(Lb, 0, ctr);
          k_newton_continue(Lb, h, W.any_active, ctr);
        } catch (...) {
          cudaStreamEndCapture(bs, &body);
          cudaStreamDestroy(bs);
          cudaStreamDestroy(bs2);
          cudaEventDestroy(bf);
          cudaEventDestroy(bj);
          throw;
        }
        e = cudaStreamEndCapture(bs, &body);
      }
      cudaStreamDestroy(bs);
      cudaStreamDestroy(bs2);
      cudaEventDestroy(bf);
      cudaEventDestroy(bj);
      CUDA_OK(e);
      CUDA_OK(cudaStreamUpdateCaptureDependencies(L.st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    } else {
      for (int it = 1; it <= max_it; ++it) {
        newton_step(L, it, nullptr);
        int any = 0;
        CUDA_OK(cudaMemcpyAsync(&any, W.any_active, sizeof(int), cudaMemcpyDeviceToHost, L.st));
        CUDA_OK(cudaStreamSynchronize(L.st));
        if (!any) break;
      }
    }
    // refactorise at the mode
    k_set_active(L, W, 0);
    k_poisson_eta(L, M, W, W.x);
    k_obs_assemble(L, M, W.P, W.active, W.mu, W.sM, nullptr, 0, true, W.eta, W.AtAp, W.sAtAp, W.Arwp, W.sArwp,
                   W.Tipp, W.sNb2, nullptr, 0, W.tippart);
    factor<R>(L, M, W, ASM_QC, SC_LOGDET_QC, split);
    k_obs_reduce(L, M, W, 1);
    k_quadforms(L, M, W, W.x, W.x, PT_XD_C, SC_TIP_XX);
    if (need_sel) {
      k_set_active(L, W, 1);
      if (esc) {
        factor<double>(L, M, Wd, ASM_QC, SC_LOGDET_QC, split);   // Q_c at the mode, assembled above
        selinv<double>(L, M, Wd, ASM_QC, adj, mv_out, bb.point_out, w0, adj, split);
      } else {
        selinv<R>(L, M, W, ASM_QC, adj, mv_out, bb.point_out, w0, adj, split);
      }
      if (adj) {
        k_set_active(L, W, 2);
        k_poisson_wobs(L, M, W);
        CUDA_OK(cudaMemsetAsync(W.rhs, 0, sizeof(double) * W.sVec * W.P, L.st));
        k_obs_assemble(L, M, W.P, W.active, nullptr, 0, W.wobs, W.sM, false, nullptr, nullptr, 0, nullptr, 0,
                       nullptr, 0, W.rhs, W.sVec, W.tippart);
        if (esc) solve<double>(L, M, Wd, W.rhs, W.xprev, split);
        else solve<R>(L, M, W, W.rhs, W.xprev, split);
        k_quadforms(L, M, W, W.xprev, W.x, PT_LD_C, SC_TIP_LX);
      }
      k_set_active(L, W, 0);
    }
  }
  if (x_out) k_copy_mode(L, M, W, x_out, bb.point_out, w0);
  k_finalize(L, M, W, o.grad, o.prior_mode, w0, bb.f_all, bb.grad_all, bb.status_all, bb.iters_all);
  if (mv_out && need_sel) {
    mask_failed_kernel<<<dim3(64, W.P), 256, 0, L.st>>>(W, M.n, mv_out, bb.point_out, w0);
    L.tick();
  }
}

void run_wave(inla_model *mdl, Launch &L, const Work &W, const inla_eval_opts &o, int64_t w0,
              const BatchBufs &bb, double *x_out, double *mv_out, int centre_flags) {
  if (W.rb == 4) run_wave_t<float>(mdl, L, W, o, w0, bb, x_out, mv_out, centre_flags);
  else run_wave_t<double>(mdl, L, W, o, w0, bb, x_out, mv_out, centre_flags);
}

void enqueue_eval(inla_model *mdl, Launch &L, int B, const double *theta_dev, const inla_eval_opts *opts,
                  const inla_eval_out *out, const BatchBufs &bb, int Pw, int rb);
void replay_graph(inla_model *mdl, int B, const double *theta_dev, const inla_eval_opts *opts,
                  const inla_eval_out *out, cudaStream_t st, const BatchBufs &bb, int rb);

int64_t eval_impl(inla_model *mdl, int B, const double *theta_dev, const inla_eval_opts *opts,
                  const inla_eval_out *out, cudaStream_t st) {
  if (!mdl || !opts || !out || !theta_dev || B < 1) throw ApiError(INLA_ERR_ARG, "invalid arguments");
  if (!out->f_dev || !out->status_dev) throw ApiError(INLA_ERR_ARG, "f_dev and status_dev are required");
  if (opts->grad < INLA_GRAD_NONE || opts->grad > INLA_GRAD_FD_FORWARD) throw ApiError(INLA_ERR_ARG, "bad grad mode");
  if (opts->prior_mode != INLA_PRIOR_KRONECKER && opts->prior_mode != INLA_PRIOR_BTA)
    throw ApiError(INLA_ERR_ARG, "bad prior mode");
  if (opts->precision != INLA_FP64 && opts->precision != INLA_MIXED) throw ApiError(INLA_ERR_ARG, "bad precision");
  if (opts->grad != INLA_GRAD_NONE && !out->grad_dev) throw ApiError(INLA_ERR_ARG, "grad_dev required");
  if (opts->want_mode && !out->x_mode_dev) throw ApiError(INLA_ERR_ARG, "x_mode_dev required");
  if (opts->want_marg_var && !out->marg_var_dev) throw ApiError(INLA_ERR_ARG, "marg_var_dev required");
  const int rb = opts->precision == INLA_MIXED ? 4 : 8;
  CUDA_OK(cudaSetDevice(mdl->device));
  const int per = fd_points_per_centre(opts->grad);
  const int64_t P_total = (int64_t)B * per;
  mdl->launches = 0;
  // the workspace is shared by all calls on this model: order this call after the previous one
  if (mdl->done_valid) CUDA_OK(cudaStreamWaitEvent(st, mdl->done, 0));
  const int Pw = wave_points(mdl, P_total, *opts);
  ensure_workspace(mdl, Pw, *opts);
  BatchBufs bb = batch_buffers(mdl, P_total);
  if (opts->use_graph && Pw == P_total && !mdl->prof.enabled) {
    replay_graph(mdl, B, theta_dev, opts, out, st, bb, rb);
  } else {
    Launch L{st, &mdl->launches, &mdl->prof};
    with_chain2(mdl, L);
    enqueue_eval(mdl, L, B, theta_dev, opts, out, bb, Pw, rb);
  }
  CUDA_OK(cudaEventRecord(mdl->done, st));
  mdl->done_valid = true;
  CUDA_OK(cudaGetLastError());
  return mdl->launches;
}

// The whole evaluation of one call, enqueued on L.st (eager path and graph capture).
void enqueue_eval(inla_model *mdl, Launch &L, int B, const double *theta_dev, const inla_eval_opts *opts,
                  const inla_eval_out *out, const BatchBufs &bb, int Pw, int rb) {
  cudaStream_t st = L.st;
  const int per = fd_points_per_centre(opts->grad);
  const double eps = opts->fd_eps > 0 ? opts->fd_eps : 1e-3;
  const int64_t P_total = (int64_t)B * per;
  point_out_kernel<<<(unsigned)((P_total + 127) / 128), 128, 0, st>>>((int)P_total, per, bb.point_out);
  L.tick();
  if (per > 1) k_fd_points(L, B, per, theta_dev, eps, bb.theta_all);
  else CUDA_OK(cudaMemcpyAsync(bb.theta_all, theta_dev, sizeof(double) * 4 * B, cudaMemcpyDeviceToDevice, st));
  int centre_flags = 0;
  if (opts->want_marg_var || opts->grad == INLA_GRAD_ADJOINT) centre_flags |= 1;
  if (opts->grad == INLA_GRAD_ADJOINT) centre_flags |= 2;
  for (int64_t w0 = 0; w0 < P_total; w0 += Pw) {
    const int P = (int)std::min<int64_t>(Pw, P_total - w0);
    Work W = carve_for(mdl->M, mdl->ws, Pw, *opts);
    W.P = P;
    CUDA_OK(cudaMemcpyAsync(W.theta, bb.theta_all + 4 * w0, sizeof(double) * 4 * P, cudaMemcpyDeviceToDevice, st));
    // theta rows are read with stride 4 by the parameter kernel
    run_wave(mdl, L, W, *opts, w0, bb, opts->want_mode ? out->x_mode_dev : nullptr,
             opts->want_marg_var ? out->marg_var_dev : nullptr, centre_flags);
  }
  k_outputs(L, B, per, eps, 4, bb.f_all, opts->grad == INLA_GRAD_ADJOINT ? bb.grad_all : nullptr, bb.status_all,
            bb.iters_all, out->f_dev, opts->grad != INLA_GRAD_NONE ? out->grad_dev : nullptr, out->status_dev,
            out->newton_iters_dev);
}

// CUDA graph of the whole evaluation for one (batch size, options, workspace):
// captured once on the model's stream with model-owned input/output buffers,
// then replayed with one copy of theta in and one copy per output out.
void replay_graph(inla_model *mdl, int B, const double *theta_dev, const inla_eval_opts *opts,
                  const inla_eval_out *out, cudaStream_t st, const BatchBufs &bb, int rb) {
  const int64_t n = mdl->M.n;
  inla_model::GraphEntry *g = nullptr;
  for (auto &e : mdl->graphs)
    if (e.B == B && e.grad == opts->grad && e.prior == opts->prior_mode && e.precision == opts->precision &&
        e.want_mode == (opts->want_mode != 0) && e.want_marg_var == (opts->want_marg_var != 0) &&
        e.fd_eps == opts->fd_eps && e.max_newton == opts->max_newton && e.newton_tol == opts->newton_tol &&
        e.time_parts == mdl->M.time_parts && e.point_groups == mdl->M.point_groups && e.ws == mdl->ws &&
        e.bb == mdl->bb)
      g = &e;
  if (!g) {
    inla_model::GraphEntry e{};
    e.B = B; e.grad = opts->grad; e.prior = opts->prior_mode; e.precision = opts->precision;
    e.want_mode = opts->want_mode != 0; e.want_marg_var = opts->want_marg_var != 0; e.fd_eps = opts->fd_eps;
    e.max_newton = opts->max_newton; e.newton_tol = opts->newton_tol; e.time_parts = mdl->M.time_parts; e.point_groups = mdl->M.point_groups;
    e.ws = mdl->ws; e.bb = mdl->bb;
    const size_t bytes = rup(32 * B, 256) + rup(8 * B, 256) + rup(32 * B, 256) + 2 * rup(4 * B, 256) +
                         2 * rup(8 * n * B, 256);
    CUDA_OK(cudaDeviceSynchronize());
    CUDA_OK(cudaMalloc(&e.stage, bytes));
    char *p = static_cast<char *>(e.stage);
    auto take = [&](size_t b) { char *r = p; p += rup(b, 256); return r; };
    e.theta = reinterpret_cast<double *>(take(32 * B));
    e.f = reinterpret_cast<double *>(take(8 * B));
    e.grad_out = reinterpret_cast<double *>(take(32 * B));
    e.status = reinterpret_cast<int *>(take(4 * B));
    e.iters = reinterpret_cast<int *>(take(4 * B));
    e.x = reinterpret_cast<double *>(take(8 * n * B));
    e.mv = reinterpret_cast<double *>(take(8 * n * B));
    inla_eval_out so{};
    so.f_dev = e.f; so.grad_dev = e.grad_out; so.status_dev = e.status; so.newton_iters_dev = e.iters;
    so.x_mode_dev = e.x; so.marg_var_dev = e.mv;
    dense_prepare();
    int64_t count = 0;
    Launch L{mdl->stream, &count, nullptr};
    with_chain2(mdl, L);
    L.capturing = true;
    cudaGraph_t graph = nullptr;
    CUDA_OK(cudaStreamBeginCapture(mdl->stream, cudaStreamCaptureModeThreadLocal));
    try {
      enqueue_eval(mdl, L, B, e.theta, opts, &so, bb, (int)((int64_t)B * (fd_points_per_centre(opts->grad))),
                   rb);
    } catch (...) {
      cudaStreamEndCapture(mdl->stream, &graph);
      if (graph) cudaGraphDestroy(graph);
      cudaFree(e.stage);
      throw;
    }
    CUDA_OK(cudaStreamEndCapture(mdl->stream, &graph));
    cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      cudaFree(e.stage);
      throw ApiError(INLA_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
    }
    e.launches = count;
    mdl->graphs.push_back(e);
    g = &mdl->graphs.back();
  }
  CUDA_OK(cudaMemcpyAsync(g->theta, theta_dev, sizeof(double) * 4 * B, cudaMemcpyDeviceToDevice, st));
  CUDA_OK(cudaGraphLaunch(g->exec, st));
  CUDA_OK(cudaMemcpyAsync(out->f_dev, g->f, sizeof(double) * B, cudaMemcpyDeviceToDevice, st));
  CUDA_OK(cudaMemcpyAsync(out->status_dev, g->status, sizeof(int) * B, cudaMemcpyDeviceToDevice, st));
  if (out->newton_iters_dev)
    CUDA_OK(cudaMemcpyAsync(out->newton_iters_dev, g->iters, sizeof(int) * B, cudaMemcpyDeviceToDevice, st));
  if (opts->grad != INLA_GRAD_NONE)
    CUDA_OK(cudaMemcpyAsync(out->grad_dev, g->grad_out, sizeof(double) * 4 * B, cudaMemcpyDeviceToDevice, st));
  if (opts->want_mode)
    CUDA_OK(cudaMemcpyAsync(out->x_mode_dev, g->x, sizeof(double) * n * B, cudaMemcpyDeviceToDevice, st));
  if (opts->want_marg_var)
    CUDA_OK(cudaMemcpyAsync(out->marg_var_dev, g->mv, sizeof(double) * n * B, cudaMemcpyDeviceToDevice, st));
  mdl->launches = g->launches;
}

template <class F>
int guarded(F &&f) {
  try {
    f();
    set_error("");
    return INLA_OK;
  } catch (const ApiError &e) {
    set_error(e.what());
    return e.code;
  } catch (const std::bad_alloc &) {
    set_error("host allocation failed");
    return INLA_ERR_OOM;
  } catch (const std::exception &e) {
    set_error(e.what());
    return INLA_ERR_CUDA;
  }
}

}  // namespace

// ------------------------------------------------------------------ no-allocation variant
//
// inla_eval_batch_static runs the same evaluation with its workspace in this
// fixed array instead of memory from cudaMalloc.  Host code must not use the
// symbol as an address: the device address comes from cudaGetSymbolAddress,
// looked up once per device with that device current -- by inla_model_create,
// which thereby also makes the runtime back the array on that device (under
// lazy module loading that happens at the first use of the symbol), so that
// the entry point itself never triggers it.  Every GPU with a model holds the
// array until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[INLA_STATIC_SCRATCH_BYTES];

namespace {

std::mutex g_static_mu;
void *g_static_addr[256] = {};

void *static_scratch(int device) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (device < 0 || device >= 256) throw ApiError(INLA_ERR_ARG, "device index out of range");
  if (!g_static_addr[device]) {
    void *p = nullptr;
    CUDA_OK(cudaGetSymbolAddress(&p, g_static_scratch));
    g_static_addr[device] = p;
  }
  return g_static_addr[device];
}

int64_t eval_static_impl(inla_model *mdl, int B, const double *theta_dev, const inla_eval_opts *opts,
                         const inla_eval_out *out, cudaStream_t st) {
  if (!mdl || !opts || !out || !theta_dev || B < 1) throw ApiError(INLA_ERR_ARG, "invalid arguments");
  if (!out->f_dev || !out->status_dev) throw ApiError(INLA_ERR_ARG, "f_dev and status_dev are required");
  if (opts->grad < INLA_GRAD_NONE || opts->grad > INLA_GRAD_FD_FORWARD) throw ApiError(INLA_ERR_ARG, "bad grad mode");
  if (opts->prior_mode != INLA_PRIOR_KRONECKER && opts->prior_mode != INLA_PRIOR_BTA)
    throw ApiError(INLA_ERR_ARG, "bad prior mode");
  if (opts->precision != INLA_FP64 && opts->precision != INLA_MIXED) throw ApiError(INLA_ERR_ARG, "bad precision");
  if (opts->grad != INLA_GRAD_NONE && !out->grad_dev) throw ApiError(INLA_ERR_ARG, "grad_dev required");
  if (opts->want_mode && !out->x_mode_dev) throw ApiError(INLA_ERR_ARG, "x_mode_dev required");
  if (opts->want_marg_var && !out->marg_var_dev) throw ApiError(INLA_ERR_ARG, "marg_var_dev required");
  const int rb = opts->precision == INLA_MIXED ? 4 : 8;
  const int per = fd_points_per_centre(opts->grad);
  const double eps = opts->fd_eps > 0 ? opts->fd_eps : 1e-3;
  const int64_t P_total = (int64_t)B * per;
  // the whole batch is one wave: workspace, then the per-point batch arrays
  const int64_t ws_bytes = point_bytes_for(mdl->M, *opts) * P_total;
  const int64_t bb_bytes = rup(32 * P_total, 256) + rup(8 * P_total, 256) + rup(32 * P_total, 256) +
                           3 * rup(4 * P_total, 256);
  if (P_total > 65535 || ws_bytes + bb_bytes > (int64_t)INLA_STATIC_SCRATCH_BYTES)
    throw ApiError(INLA_ERR_ARG, "batch needs " + std::to_string(ws_bytes + bb_bytes) +
                                     " bytes of scratch; the static array holds " +
                                     std::to_string((long long)INLA_STATIC_SCRATCH_BYTES));
  CUDA_OK(cudaSetDevice(mdl->device));
  char *base = static_cast<char *>(static_scratch(mdl->device));
  mdl->launches = 0;
  Launch L{st, &mdl->launches, nullptr};
  with_chain2(mdl, L);
  if (mdl->done_valid) CUDA_OK(cudaStreamWaitEvent(st, mdl->done, 0));
  Work W0 = carve_for(mdl->M, base, (int)P_total, *opts);
  char *p = base + ws_bytes;
  auto take = [&](int64_t bytes) { char *r = p; p += rup(bytes, 256); return r; };
  BatchBufs bb;
  bb.theta_all = reinterpret_cast<double *>(take(32 * P_total));
  bb.f_all = reinterpret_cast<double *>(take(8 * P_total));
  bb.grad_all = reinterpret_cast<double *>(take(32 * P_total));
  bb.point_out = reinterpret_cast<int *>(take(4 * P_total));
  bb.status_all = reinterpret_cast<int *>(take(4 * P_total));
  bb.iters_all = reinterpret_cast<int *>(take(4 * P_total));
  point_out_kernel<<<(unsigned)((P_total + 127) / 128), 128, 0, st>>>((int)P_total, per, bb.point_out);
  L.tick();
  if (per > 1) k_fd_points(L, B, per, theta_dev, eps, bb.theta_all);
  else CUDA_OK(cudaMemcpyAsync(bb.theta_all, theta_dev, sizeof(double) * 4 * B, cudaMemcpyDeviceToDevice, st));
  int centre_flags = 0;
  if (opts->want_marg_var || opts->grad == INLA_GRAD_ADJOINT) centre_flags |= 1;
  if (opts->grad == INLA_GRAD_ADJOINT) centre_flags |= 2;
  Work W = W0;
  W.P = (int)P_total;
  CUDA_OK(cudaMemcpyAsync(W.theta, bb.theta_all, sizeof(double) * 4 * P_total, cudaMemcpyDeviceToDevice, st));
  run_wave(mdl, L, W, *opts, 0, bb, opts->want_mode ? out->x_mode_dev : nullptr,
           opts->want_marg_var ? out->marg_var_dev : nullptr, centre_flags);
  k_outputs(L, B, per, eps, 4, bb.f_all, opts->grad == INLA_GRAD_ADJOINT ? bb.grad_all : nullptr, bb.status_all,
            bb.iters_all, out->f_dev, opts->grad != INLA_GRAD_NONE ? out->grad_dev : nullptr, out->status_dev,
            out->newton_iters_dev);
  CUDA_OK(cudaEventRecord(mdl->done, st));
  mdl->done_valid = true;
  CUDA_OK(cudaGetLastError());
  return mdl->launches;
}

}  // namespace

extern "C" {

int inla_model_create(const inla_model_desc *desc, int device, inla_model **out) {
  return guarded([&] {
    if (!out) throw ApiError(INLA_ERR_ARG, "out is NULL");
    *out = nullptr;
    *out = create_model(desc, device);
  });
}

int inla_workspace_bytes(const inla_model *model, int B, const inla_eval_opts *opts, size_t *bytes) {
  return guarded([&] {
    if (!model || !opts || !bytes || B < 1) throw ApiError(INLA_ERR_ARG, "invalid arguments");
    const int per = fd_points_per_centre(opts->grad);
    *bytes = (size_t)point_bytes_for(model->M, *opts) * (size_t)B * per;
  });
}

int inla_eval_batch(inla_model *model, int B, const double *theta_dev, const inla_eval_opts *opts,
                    const inla_eval_out *out, void *stream) {
  return guarded([&] { eval_impl(model, B, theta_dev, opts, out, static_cast<cudaStream_t>(stream)); });
}

int inla_eval_batch_static(inla_model *model, int B, const double *theta_dev, const inla_eval_opts *opts,
                           const inla_eval_out *out, void *stream) {
  return guarded([&] { eval_static_impl(model, B, theta_dev, opts, out, static_cast<cudaStream_t>(stream)); });
}

int inla_set_tiles(inla_model *model, int sweep_fp64, int sweep_fp32, int gemm_fp32) {
  return guarded([&] {
    if (!model) throw ApiError(INLA_ERR_ARG, "model is NULL");
    if ((sweep_fp64 != 32 && sweep_fp64 != 64) ||
        (sweep_fp32 != 32 && sweep_fp32 != 64 && sweep_fp32 != INLA_SWEEP_TF32X3 && sweep_fp32 != INLA_INV_BLOCKED) ||
        (gemm_fp32 != 64 && gemm_fp32 != 128 && gemm_fp32 != INLA_GEMM_TF32X3))
      throw ApiError(INLA_ERR_ARG, "tile widths: FP64 sweep 32 or 64, FP32 sweep 32, 64, INLA_SWEEP_TF32X3 or "
                                   "INLA_INV_BLOCKED, FP32 GEMM 64, 128 or INLA_GEMM_TF32X3");
    CUDA_OK(cudaSetDevice(model->device));
    CUDA_OK(cudaDeviceSynchronize());
    model->M.sweep_g64 = sweep_fp64;
    model->M.sweep_g32 = sweep_fp32;
    model->M.gemm_t32 = gemm_fp32;
    for (auto &g : model->graphs) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.stage) cudaFree(g.stage);
    }
    model->graphs.clear();
  });
}

int inla_autotune(inla_model *model, int B, const double *theta_dev, const inla_eval_opts *opts, int32_t *choice) {
  return guarded([&] {
    if (!model || !opts || !theta_dev || B < 1) throw ApiError(INLA_ERR_ARG, "invalid arguments");
    CUDA_OK(cudaSetDevice(model->device));
    DevModel &M = model->M;
    const bool fp32 = opts->precision == INLA_MIXED;
    const int64_t n = M.n;
    // outputs of the trial evaluations (device, freed before returning)
    void *buf = nullptr;
    const size_t bytes = (size_t)B * (8 + 32 + 4 + 4 + 16 * n) + 4096;
    CUDA_OK(cudaMalloc(&buf, bytes));
    char *p = static_cast<char *>(buf);
    auto take = [&](size_t b) { char *r = p; p += rup(b, 256); return r; };
    inla_eval_out out{};
    out.f_dev = reinterpret_cast<double *>(take(8 * B));
    out.grad_dev = reinterpret_cast<double *>(take(32 * B));
    out.status_dev = reinterpret_cast<int *>(take(4 * B));
    out.newton_iters_dev = reinterpret_cast<int *>(take(4 * B));
    out.x_mode_dev = reinterpret_cast<double *>(take(8 * n * B));
    out.marg_var_dev = reinterpret_cast<double *>(take(8 * n * B));
    inla_eval_opts o = *opts;
    o.use_graph = 0;
    struct Cand { int g, t; };
    std::vector<Cand> cands;
    if (fp32) {
      cands = {{64, 128}, {32, 128}, {64, 64}, {32, 64}};
      if (M.n_p % 128 == 0) {
        cands.push_back({64, INLA_GEMM_TF32X3});
        cands.push_back({32, INLA_GEMM_TF32X3});
        cands.push_back({INLA_SWEEP_TF32X3, INLA_GEMM_TF32X3});
        cands.push_back({INLA_SWEEP_TF32X3, 128});
        cands.push_back({INLA_INV_BLOCKED, INLA_GEMM_TF32X3});
      }
    }
    else cands = {{32, M.gemm_t32}, {64, M.gemm_t32}};
    cudaEvent_t e0, e1;
    CUDA_OK(cudaEventCreate(&e0));
    CUDA_OK(cudaEventCreate(&e1));
    float best = 1e30f;
    Cand bc = cands[0];
    try {
      for (const Cand &c : cands) {
        if (fp32) { M.sweep_g32 = c.g; M.gemm_t32 = c.t; }
        else M.sweep_g64 = c.g;
        eval_impl(model, B, theta_dev, &o, &out, model->stream);   // warm-up (allocations, caches)
        CUDA_OK(cudaEventRecord(e0, model->stream));
        eval_impl(model, B, theta_dev, &o, &out, model->stream);
        CUDA_OK(cudaEventRecord(e1, model->stream));
        CUDA_OK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CUDA_OK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) { best = ms; bc = c; }
      }
    } catch (...) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      cudaFree(buf);
      throw;
    }
    if (fp32) { M.sweep_g32 = bc.g; M.gemm_t32 = bc.t; }
    else M.sweep_g64 = bc.g;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CUDA_OK(cudaFree(buf));
    for (auto &g : model->graphs) {          // graphs captured with other tiles are stale
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.stage) cudaFree(g.stage);
    }
    model->graphs.clear();
    if (choice) {
      choice[0] = M.sweep_g64;
      choice[1] = M.sweep_g32;
      choice[2] = M.gemm_t32;
    }
  });
}

int inla_eval_batch_host(inla_model *model, int B, const double *theta, const inla_eval_opts *opts,
                         const inla_eval_out_host *out) {
  return guarded([&] {
    if (!model || !opts || !out || !theta || B < 1 || !out->f || !out->status)
      throw ApiError(INLA_ERR_ARG, "invalid arguments");
    CUDA_OK(cudaSetDevice(model->device));
    const int64_t n = model->M.n;
    const size_t need = rup(32 * B, 256) + rup(8 * B, 256) + rup(32 * B, 256) + 2 * rup(4 * B, 256) +
                        2 * rup(8 * n * B, 256);
    if (!model->hb || model->hb_bytes < need) {
      if (model->hb) {
        CUDA_OK(cudaStreamSynchronize(model->stream));
        cudaFree(model->hb);
        model->hb = nullptr;
      }
      CUDA_OK(cudaMalloc(&model->hb, need));
      model->hb_bytes = need;
    }
    char *p = static_cast<char *>(model->hb);
    auto take = [&](size_t b) { char *r = p; p += rup(b, 256); return r; };
    double *th = reinterpret_cast<double *>(take(32 * B));
    inla_eval_out d{};
    d.f_dev = reinterpret_cast<double *>(take(8 * B));
    d.grad_dev = reinterpret_cast<double *>(take(32 * B));
    d.status_dev = reinterpret_cast<int *>(take(4 * B));
    d.newton_iters_dev = reinterpret_cast<int *>(take(4 * B));
    d.x_mode_dev = reinterpret_cast<double *>(take(8 * n * B));
    d.marg_var_dev = reinterpret_cast<double *>(take(8 * n * B));
    cudaStream_t st = model->stream;
    CUDA_OK(cudaMemcpyAsync(th, theta, sizeof(double) * 4 * B, cudaMemcpyHostToDevice, st));
    eval_impl(model, B, th, opts, &d, st);
    CUDA_OK(cudaMemcpyAsync(out->f, d.f_dev, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(out->status, d.status_dev, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
    if (out->grad && opts->grad != INLA_GRAD_NONE)
      CUDA_OK(cudaMemcpyAsync(out->grad, d.grad_dev, sizeof(double) * 4 * B, cudaMemcpyDeviceToHost, st));
    if (out->newton_iters)
      CUDA_OK(cudaMemcpyAsync(out->newton_iters, d.newton_iters_dev, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
    if (out->x_mode && opts->want_mode)
      CUDA_OK(cudaMemcpyAsync(out->x_mode, d.x_mode_dev, sizeof(double) * n * B, cudaMemcpyDeviceToHost, st));
    if (out->marg_var && opts->want_marg_var)
      CUDA_OK(cudaMemcpyAsync(out->marg_var, d.marg_var_dev, sizeof(double) * n * B, cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaStreamSynchronize(st));
  });
}

int inla_profile_enable(inla_model *model, int enable) {
  return guarded([&] {
    if (!model) throw ApiError(INLA_ERR_ARG, "model is NULL");
    CUDA_OK(cudaSetDevice(model->device));
    CUDA_OK(cudaDeviceSynchronize());
    model->prof.reset();
    model->prof.enabled = enable > 0 ? enable : 0;
  });
}

int inla_profile_read(inla_model *model, int kernel, double *total_ms, int64_t *launches, double *units) {
  return guarded([&] {
    if (!model || !total_ms || !launches || !units || kernel < 0 || kernel >= KID_COUNT)
      throw ApiError(INLA_ERR_ARG, "invalid arguments");
    CUDA_OK(cudaSetDevice(model->device));
    double ms = 0.0, u = 0.0;
    int64_t n = 0;
    for (auto &r : model->prof.recs) {
      if (r.id != kernel) continue;
      CUDA_OK(cudaEventSynchronize(r.b));
      float e = 0.f;
      CUDA_OK(cudaEventElapsedTime(&e, r.a, r.b));
      ms += e;
      u += r.units;
      ++n;
    }
    *total_ms = ms;
    *launches = n;
    *units = u;
  });
}

int inla_set_fp64_products(inla_model *model, int tensor) {
  return guarded([&] {
    if (!model || (tensor != 0 && tensor != 1)) throw ApiError(INLA_ERR_ARG, "model is NULL or tensor not 0 / 1");
    CUDA_OK(cudaSetDevice(model->device));
    CUDA_OK(cudaDeviceSynchronize());
    model->M.f64_tensor = tensor;
    for (auto &g : model->graphs) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.stage) cudaFree(g.stage);
    }
    model->graphs.clear();
  });
}

int inla_set_time_partition(inla_model *model, int parts) {
  return guarded([&] {
    if (!model || (parts != 1 && parts != 2)) throw ApiError(INLA_ERR_ARG, "model is NULL or parts not 1 / 2");
    model->M.time_parts = parts;   // the graph cache is keyed on it; the workspace grows on demand
  });
}

int inla_set_point_groups(inla_model *model, int groups) {
  return guarded([&] {
    if (!model || (groups != 1 && groups != 2)) throw ApiError(INLA_ERR_ARG, "model is NULL or groups not 1 / 2");
    model->M.point_groups = groups;
  });
}

int inla_set_wait_limit(double seconds) {
  return guarded([&] {
    if (!(seconds > 0.0) || !(seconds <= 2.0))
      throw ApiError(INLA_ERR_ARG, "the wait limit must be in (0, 2] seconds");
    set_wait_limit_ns((uint64_t)(seconds * 1e9));
  });
}

int64_t inla_model_latent_dim(const inla_model *model) { return model ? model->M.n : -1; }

int64_t inla_last_launch_count(const inla_model *model) { return model ? model->launches : -1; }

void inla_model_destroy(inla_model *model) { delete model; }

const char *inla_last_error(void) { return inla::get_error(); }

}  // extern "C"
