"""CPU oracle for the INLA hyperparameter-phase evaluation (TEST INFRASTRUCTURE).

This package is a plain, slow, float64 restatement of what the GPU library
computes for each hyperparameter point theta:

  f(theta) = -log pi~(theta | y)   (Eq. post_theta_approx and the definition
                                    of f in Sec. 3.1),
  its gradient, the latent mode x*(theta), and the marginal variances
  diag(Q_c(theta)^-1) (Sec. 2.3, Sec. 2.4.2).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline legs may import it.  The GPU library never does: the two share no
code besides the seeded input generators in ``synth``.

Modules
  model   hyperparameter maps, Q_s, Q_t, Q, Q_c, log prior        (readings)
  dense   the definition with dense n x n matrices (small n)
  bta     block-tridiagonal-arrowhead Cholesky, solves and block Takahashi
          selected inversion (Sec. 2.4, Eq. sel_inv_cov / takahashi_recursion)
  scalar  element-wise recursions on tiny matrices (Cholesky, Eq. backward_solve,
          Eq. sel_inv_cov, Eq. takahashi_recursion)
  fd      central differences (Eq. central_diff)
  tf32    the TF32 split product of the mixed path's tensor-core products (error model)

Parity status: every function is pinned by tests under tests/ against closed
forms, brute force and invariants; the Poisson Laplace value is pinned only
through its mode condition, the dense brute force of the same iteration and
the Gaussian special case ("parity partially pinned" for the Poisson f).
"""
