// Synthetic spatio-temporal workloads in C++ (host code; inputs only, none of
// the method): the same recipe and random streams as the project's Python
// generator, so that a C caller can build the benchmark models without Python.
//
//  * random numbers: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) in counter
//    form, output k of stream (seed, id) = mix(base + (k + 1) * GAMMA); doubles
//    from the top 53 bits, normals by Box-Muller (both outputs of a pair),
//    Poisson counts by sequential CDF inversion (Devroye 1986, Sec. X.3.3);
//  * mesh: an nx x nx vertex grid of [0,1]^2, cells cut along (i,j)-(i+1,j+1),
//    P1 lumped mass C and stiffness G (every triangle edge stored);
//  * observations: uniform times and locations, barycentric weights of the
//    containing triangle plus n_b N(0,1) covariates per row of A;
//  * truth: a Matern(nu = 1) field by 128 random Fourier features per time
//    step with an AR(1) recursion in time, beta ~ N(0, 1) (Poisson N(0, 0.1^2)),
//    Gaussian y = A x + N(0, 1/tau_y), Poisson y ~ Pois(E exp(A x)), E ~ U(0.5, 2).
// Integer outputs (patterns, times, counts) match the Python generator exactly
// apart from Poisson draws that sit on a CDF boundary; floating outputs agree to
// rounding (libm and numpy may differ in the last bit of exp, log, cos, sin).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "inla_internal.cuh"

namespace {

constexpr uint64_t GAMMA = 0x9E3779B97F4A7C15ull;

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Stream {
  uint64_t base;
  uint64_t counter = 0;
  Stream(uint64_t seed, uint64_t id) {
    const uint64_t key = mix64(seed ^ (id * GAMMA));
    base = mix64(key + 0x632BE59BD9B4E019ull);
  }
  uint64_t bits() { return mix64(base + (++counter) * GAMMA); }
  double uniform() { return (double)(bits() >> 11) * (1.0 / 9007199254740992.0); }
  double uniform_open() { return ((double)(bits() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  int64_t integer(int64_t high) {
    const uint64_t top = bits() >> 32;
    return (int64_t)((top * (uint64_t)high) >> 32);
  }
  // n normals: pairs from (uniform_open, uniform) drawn as two blocks, as the
  // vectorised generator does (all first uniforms, then all second ones)
  std::vector<double> normal(int64_t n) {
    const int64_t h = (n + 1) / 2;
    std::vector<double> u1(h), u2(h), out(2 * h);
    for (int64_t i = 0; i < h; ++i) u1[i] = uniform_open();
    for (int64_t i = 0; i < h; ++i) u2[i] = uniform();
    for (int64_t i = 0; i < h; ++i) {
      const double r = std::sqrt(-2.0 * std::log(u1[i]));
      out[2 * i] = r * std::cos(2.0 * M_PI * u2[i]);
      out[2 * i + 1] = r * std::sin(2.0 * M_PI * u2[i]);
    }
    out.resize(n);
    return out;
  }
};

struct Owner {
  std::vector<double> C, G_val, A_val, y, E;
  std::vector<int32_t> G_rowptr, G_col, A_col;
  std::vector<int64_t> A_rowptr;
};

void grid_fem(int nx, Owner &o) {
  const int n_s = nx * nx;
  const double h = 1.0 / (nx - 1), area = 0.5 * h * h;
  o.C.assign(n_s, 0.0);
  // element matrices: (area grad_a) . grad_b for the two triangle shapes
  const double g1[3][2] = {{-1.0 / h, 0.0}, {1.0 / h, -1.0 / h}, {0.0, 1.0 / h}};
  const double g2[3][2] = {{0.0, -1.0 / h}, {1.0 / h, 0.0}, {-1.0 / h, 1.0 / h}};
  double K1[3][3], K2[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      K1[a][b] = (area * g1[a][0]) * g1[b][0] + (area * g1[a][1]) * g1[b][1];
      K2[a][b] = (area * g2[a][0]) * g2[b][0] + (area * g2[a][1]) * g2[b][1];
    }
  const int ncell = (nx - 1) * (nx - 1);
  std::vector<int64_t> key;
  std::vector<double> val;
  key.reserve((size_t)18 * ncell);
  val.reserve((size_t)18 * ncell);
  for (int shape = 0; shape < 2; ++shape) {
    const double(*K)[3] = shape == 0 ? K1 : K2;
    for (int a = 0; a < 3; ++a) {
      // cells in the order i fastest-major as meshgrid(..., indexing="ij").ravel(): c = i * (nx-1) + j
      for (int c = 0; c < ncell; ++c) {
        const int i = c / (nx - 1), j = c % (nx - 1);
        const int v00 = i + nx * j, v10 = (i + 1) + nx * j, v11 = (i + 1) + nx * (j + 1), v01 = i + nx * (j + 1);
        const int tri[3] = {v00, shape == 0 ? v10 : v11, shape == 0 ? v11 : v01};
        o.C[tri[a]] += area / 3.0;
      }
      for (int b = 0; b < 3; ++b)
        for (int c = 0; c < ncell; ++c) {
          const int i = c / (nx - 1), j = c % (nx - 1);
          const int v00 = i + nx * j, v10 = (i + 1) + nx * j, v11 = (i + 1) + nx * (j + 1),
                    v01 = i + nx * (j + 1);
          const int tri[3] = {v00, shape == 0 ? v10 : v11, shape == 0 ? v11 : v01};
          key.push_back((int64_t)tri[a] * n_s + tri[b]);
          val.push_back(K[a][b]);
        }
    }
  }
  std::vector<size_t> order(key.size());
  for (size_t e = 0; e < order.size(); ++e) order[e] = e;
  std::stable_sort(order.begin(), order.end(), [&](size_t p, size_t q) { return key[p] < key[q]; });
  o.G_rowptr.assign(n_s + 1, 0);
  o.G_col.clear();
  o.G_val.clear();
  for (size_t e = 0; e < order.size();) {
    const int64_t k = key[order[e]];
    double s = 0.0;
    size_t f = e;
    for (; f < order.size() && key[order[f]] == k; ++f) s += val[order[f]];
    o.G_col.push_back((int32_t)(k % n_s));
    o.G_val.push_back(s);
    ++o.G_rowptr[k / n_s + 1];
    e = f;
  }
  for (int r = 0; r < n_s; ++r) o.G_rowptr[r + 1] += o.G_rowptr[r];
}

void build(int n_t, int nx, int n_b, int64_t m, int lik, uint64_t seed, const double theta[4], double tau_b,
           inla_model_desc *d, Owner &o) {
  if (n_t < 1 || nx < 2 || n_b < 0 || n_b > inla::MAX_NB || m < 1 ||
      (lik != INLA_LIK_GAUSSIAN && lik != INLA_LIK_POISSON && lik != INLA_LIK_BINOMIAL))
    throw std::invalid_argument("invalid sizes or likelihood");
  const int n_s = nx * nx;
  grid_fem(nx, o);
  Stream s_time(seed, 0), s_loc(seed, 1), s_cov(seed, 2), s_field(seed, 3), s_beta(seed, 4), s_noise(seed, 5),
      s_exp(seed, 6);
  std::vector<int64_t> obs_t(m);
  for (int64_t i = 0; i < m; ++i) obs_t[i] = s_time.integer(n_t);
  std::vector<double> loc(2 * m);
  for (int64_t i = 0; i < 2 * m; ++i) loc[i] = s_loc.uniform();
  const std::vector<double> Z = n_b ? s_cov.normal(m * n_b) : std::vector<double>();
  // A: the three barycentric entries sorted by column, then the covariates
  const int nnz_row = 3 + n_b;
  o.A_rowptr.resize(m + 1);
  o.A_col.resize(m * nnz_row);
  o.A_val.resize(m * nnz_row);
  std::vector<int32_t> verts(3 * m);
  std::vector<double> wts(3 * m);
  const double h = 1.0 / (nx - 1);
  for (int64_t r = 0; r < m; ++r) {
    const double px = loc[2 * r], py = loc[2 * r + 1];
    const int64_t ci = std::min<int64_t>((int64_t)std::floor(px / h), nx - 2);
    const int64_t cj = std::min<int64_t>((int64_t)std::floor(py / h), nx - 2);
    const double dx = (px - ci * h) / h, dy = (py - cj * h) / h;
    const int32_t v00 = (int32_t)(ci + nx * cj), v10 = (int32_t)(ci + 1 + nx * cj),
                  v11 = (int32_t)(ci + 1 + nx * (cj + 1)), v01 = (int32_t)(ci + nx * (cj + 1));
    int32_t v[3];
    double w[3];
    if (dx >= dy) {
      v[0] = v00; v[1] = v10; v[2] = v11;
      w[0] = 1.0 - dx; w[1] = dx - dy; w[2] = dy;
    } else {
      v[0] = v00; v[1] = v11; v[2] = v01;
      w[0] = 1.0 - dy; w[1] = dx; w[2] = dy - dx;
    }
    int idx[3] = {0, 1, 2};
    std::stable_sort(idx, idx + 3, [&](int p, int q) { return v[p] < v[q]; });
    o.A_rowptr[r] = r * nnz_row;
    for (int k = 0; k < 3; ++k) {
      verts[3 * r + k] = v[idx[k]];
      wts[3 * r + k] = w[idx[k]];
      o.A_col[r * nnz_row + k] = (int32_t)(obs_t[r] * n_s + v[idx[k]]);
      o.A_val[r * nnz_row + k] = w[idx[k]];
    }
    for (int l = 0; l < n_b; ++l) {
      o.A_col[r * nnz_row + 3 + l] = n_t * n_s + l;
      o.A_val[r * nnz_row + 3 + l] = Z[r * n_b + l];
    }
  }
  o.A_rowptr[m] = m * nnz_row;
  // truth: Matern(nu = 1) field by random Fourier features, AR(1) in time
  const double range = std::exp(theta[1]), sigma = std::exp(theta[2]);
  const double rho = 1.0 / (1.0 + std::exp(-theta[3]));
  const double kappa = std::sqrt(8.0) / range;
  constexpr int NF = 128;
  std::vector<double> field((size_t)n_t * n_s), cur(n_s), prev(n_s);
  for (int t = 0; t < n_t; ++t) {
    double u[NF], ang[NF], phase[NF], wx[NF], wy[NF];
    for (int f = 0; f < NF; ++f) u[f] = s_field.uniform_open();
    for (int f = 0; f < NF; ++f) ang[f] = 2.0 * M_PI * s_field.uniform();
    for (int f = 0; f < NF; ++f) phase[f] = 2.0 * M_PI * s_field.uniform();
    for (int f = 0; f < NF; ++f) {
      const double r = kappa * std::sqrt(u[f] / (1.0 - u[f]));
      wx[f] = r * std::cos(ang[f]);
      wy[f] = r * std::sin(ang[f]);
    }
    const double amp = sigma * std::sqrt(2.0 / NF);
    for (int k = 0; k < n_s; ++k) {
      const double X = (k % nx) * h, Y = (k / nx) * h;
      double s = 0.0;
      for (int f = 0; f < NF; ++f) s += std::cos(X * wx[f] + Y * wy[f] + phase[f]);
      const double e = amp * s;
      cur[k] = t == 0 ? e : rho * prev[k] + std::sqrt(1.0 - rho * rho) * e;
    }
    std::copy(cur.begin(), cur.end(), field.begin() + (size_t)t * n_s);
    prev.swap(cur);
  }
  std::vector<double> beta = s_beta.normal(n_b);
  if (lik != INLA_LIK_GAUSSIAN)
    for (double &b : beta) b *= 0.1;   // Poisson and binomial
  std::vector<double> eta(m);
  for (int64_t r = 0; r < m; ++r) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s += wts[3 * r + k] * field[(size_t)obs_t[r] * n_s + verts[3 * r + k]];
    double zb = 0.0;
    for (int l = 0; l < n_b; ++l) zb += Z[r * n_b + l] * beta[l];
    eta[r] = s + zb;
  }
  o.y.resize(m);
  if (lik == INLA_LIK_GAUSSIAN) {
    const double tau_y = std::exp(theta[0]);
    const std::vector<double> e = s_noise.normal(m);
    for (int64_t r = 0; r < m; ++r) o.y[r] = eta[r] + e[r] / std::sqrt(tau_y);
  } else if (lik == INLA_LIK_BINOMIAL) {
    // N ~ 1 + U{0..9} trials, y ~ Bin(N, logistic(eta)) by inversion (one uniform each)
    o.E.resize(m);
    for (int64_t r = 0; r < m; ++r) o.E[r] = (double)(1 + s_exp.integer(10));
    for (int64_t r = 0; r < m; ++r) {
      const int64_t n = (int64_t)o.E[r];
      const double p = 1.0 / (1.0 + std::exp(-eta[r])), q = 1.0 - p;
      const double u = s_noise.uniform();
      int64_t k = 0;
      double pk = std::pow(q, (double)n), cdf = pk;
      while (u > cdf && k < n) {
        pk *= (double)(n - k) / ((double)k + 1.0) * (p / q);
        ++k;
        cdf += pk;
      }
      o.y[r] = (double)k;
    }
  } else {
    o.E.resize(m);
    for (int64_t r = 0; r < m; ++r) o.E[r] = 0.5 + 1.5 * s_exp.uniform();
    for (int64_t r = 0; r < m; ++r) {
      const double mean = o.E[r] * std::exp(eta[r]);
      if (mean > 700.0) throw std::invalid_argument("Poisson mean too large for inversion");
      const double u = s_noise.uniform();
      int64_t k = 0;
      double p = std::exp(-mean), cdf = p;
      while (u > cdf && p > 0.0) {
        ++k;
        p *= mean / (double)k;
        cdf += p;
      }
      o.y[r] = (double)k;
    }
  }
  std::memset(d, 0, sizeof(*d));
  d->n_t = n_t;
  d->n_s = n_s;
  d->n_b = n_b;
  d->lik = lik;
  d->m = m;
  d->C_diag = o.C.data();
  d->G_rowptr = o.G_rowptr.data();
  d->G_col = o.G_col.data();
  d->G_val = o.G_val.data();
  d->A_rowptr = o.A_rowptr.data();
  d->A_col = o.A_col.data();
  d->A_val = o.A_val.data();
  d->y = o.y.data();
  d->E = lik != INLA_LIK_GAUSSIAN ? o.E.data() : nullptr;
  d->tau_b = tau_b;
  d->nb_size = 0.0;
  for (int j = 0; j < 4; ++j) {
    d->prior_mean[j] = 0.0;
    d->prior_sd[j] = 10.0;
  }
  if (lik != INLA_LIK_GAUSSIAN) d->prior_mean[0] = std::log(1e-3);
}

}  // namespace

extern "C" int inla_synth_build(int32_t n_t, int32_t nx, int32_t n_b, int64_t m, int32_t lik, uint64_t seed,
                                const double *theta_true, inla_model_desc *desc, void **owner) {
  if (!desc || !owner) {
    inla::set_error("inla_synth_build: desc and owner must be non-NULL");
    return INLA_ERR_ARG;
  }
  *owner = nullptr;
  const double gauss[4] = {1.0, -1.0, 0.0, 1.5};
  const double pois[4] = {std::log(1e-3), -1.0, 0.0, 1.5};
  const double *th = theta_true ? theta_true : (lik != INLA_LIK_GAUSSIAN ? pois : gauss);
  try {
    std::unique_ptr<Owner> o(new Owner);
    build(n_t, nx, n_b, m, lik, seed, th, 1e-3, desc, *o);
    *owner = o.release();
    return INLA_OK;
  } catch (const std::bad_alloc &) {
    inla::set_error("inla_synth_build: out of host memory");
    return INLA_ERR_OOM;
  } catch (const std::exception &e) {
    inla::set_error(std::string("inla_synth_build: ") + e.what());
    return INLA_ERR_ARG;
  }
}

extern "C" int inla_synth_grid_model(int32_t cfg_id, uint64_t seed, inla_model_desc *desc, void **owner) {
  struct Cfg { int n_t, nx, n_b; int64_t m; int lik; };
  static const Cfg cfgs[5] = {{8, 8, 2, 2000, INLA_LIK_GAUSSIAN},
                              {50, 32, 4, 100000, INLA_LIK_GAUSSIAN},
                              {100, 45, 6, 400000, INLA_LIK_GAUSSIAN},
                              {200, 50, 6, 1000000, INLA_LIK_GAUSSIAN},
                              {100, 64, 8, 500000, INLA_LIK_POISSON}};
  if (cfg_id < 1 || cfg_id > 5) {
    inla::set_error("inla_synth_grid_model: cfg_id must be 1..5");
    return INLA_ERR_ARG;
  }
  const Cfg &c = cfgs[cfg_id - 1];
  return inla_synth_build(c.n_t, c.nx, c.n_b, c.m, c.lik, seed, nullptr, desc, owner);
}

extern "C" void inla_synth_free(void *owner) { delete static_cast<Owner *>(owner); }
