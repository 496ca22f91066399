// Theta-free values of a model, computed once at model creation:
//   C, G and H = G C^-1 G on the union pattern (the three pieces of
//   Q_s = tau^2 (kappa^4 C + 2 kappa^2 G + G C^-1 G)),
//   for a Gaussian likelihood A^T A by time block (spatial part, arrow Z^T A_t,
//   tip Z^T Z) and A^T y (Q_c = Q + tau_y A^T A, b = tau_y A^T y, Sec. 2.2),
//   and data constants (y^T y, sum log y!, sum y log E).
#include <cmath>

#include "inla_internal.cuh"

namespace inla {

namespace {

__global__ void fem_values_kernel(int nnz, const int *prow_of, const int *pcol, const int64_t *hptr, const int *hk,
                                  const int *hik, const int *hkj, const double *Gval, const double *Cdiag,
                                  const int *gpos, double *vC, double *vG, double *vH) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  const int i = prow_of[e], j = pcol[e];
  vC[e] = (i == j) ? Cdiag[i] : 0.0;
  vG[e] = gpos[e] >= 0 ? Gval[gpos[e]] : 0.0;
  double h = 0.0;
  for (int64_t c = hptr[e]; c < hptr[e + 1]; ++c) h += Gval[hik[c]] * Gval[hkj[c]] / Cdiag[hk[c]];
  vH[e] = h;
}

// consts[0] = y^T y; the theta-free part of the log-likelihood is
// consts[2] - consts[1]: Poisson sum(y log E) - sum(log y!), binomial
// sum(log N! - log (N - y)!) - sum(log y!) = sum log C(N, y), negative binomial
// sum(y log E + log Gamma(y + r) - log Gamma(r) + r log r) - sum(log y!).
__global__ void consts_kernel(int64_t m, const double *y, const double *E, int lik, double r, double *consts) {
  __shared__ double red[3][256];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    s0 += y[i] * y[i];
    if (lik == INLA_LIK_POISSON) {
      s1 += lgamma(y[i] + 1.0);
      s2 += y[i] * log(E[i]);
    } else if (lik == INLA_LIK_BINOMIAL) {
      s1 += lgamma(y[i] + 1.0);
      s2 += lgamma(E[i] + 1.0) - lgamma(E[i] - y[i] + 1.0);
    } else if (lik == INLA_LIK_NEGBINOMIAL) {
      s1 += lgamma(y[i] + 1.0);
      s2 += y[i] * log(E[i]) + lgamma(y[i] + r) - lgamma(r) + r * log(r);
    }
  }
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  red[2][threadIdx.x] = s2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    consts[0] = red[0][0];
    consts[1] = red[1][0];
    consts[2] = red[2][0];
    consts[3] = 0.0;
  }
}

}  // namespace

void setup_theta_free(cudaStream_t st, DevModel &M, const int64_t *d_hptr, const int *d_hk, const int *d_hik,
                      const int *d_hkj, const double *d_Gval, const double *d_Cdiag, const int *d_gpos, double *vC,
                      double *vG, double *vH) {
  fem_values_kernel<<<(M.nnz + 255) / 256, 256, 0, st>>>(M.nnz, M.prow_of, M.pcol, d_hptr, d_hk, d_hik, d_hkj,
                                                         d_Gval, d_Cdiag, d_gpos, vC, vG, vH);
}

void setup_consts(cudaStream_t st, DevModel &M, double *consts) {
  consts_kernel<<<1, 256, 0, st>>>(M.m, M.y, M.E, M.lik, M.nb_size, consts);
}

void setup_gaussian(cudaStream_t st, DevModel &M, double *AtA, double *Arw, double *Tip, double *Aty,
                    double *tippart) {
  Launch L{st, nullptr};
  // mu = 1, r = y: A^T A by blocks and A^T y in the padded latent layout.
  cudaMemsetAsync(Aty, 0, sizeof(double) * M.nv, st);
  k_obs_assemble(L, M, 1, nullptr, nullptr, 0, M.y, 0, false, nullptr, AtA, 0, Arw, 0, Tip, 0, Aty, 0, tippart);
}

}  // namespace inla
