/* A plain C caller of the library (no Python, no PyTorch): builds the 8 x 8 x 8
 * Gaussian workload with the library's synthetic generator, creates the model
 * on CUDA device 0, evaluates f and its central-difference gradient at the
 * theta given on the command line through the host-buffer entry point, and
 * prints f, grad f and the status.  Exit code 0 on success, 1 on any non-OK
 * return (the message of inla_last_error goes to stderr). */
#include <stdio.h>
#include <stdlib.h>

#include "inla_gpu.h"

static int fail(const char *what) {
  fprintf(stderr, "%s: %s\n", what, inla_last_error());
  return 1;
}

int main(int argc, char **argv) {
  double theta[4] = {1.0, -1.0, 0.0, 1.5};
  for (int j = 0; j < 4 && j + 1 < argc; ++j) theta[j] = strtod(argv[j + 1], NULL);

  inla_model_desc desc;
  void *owner = NULL;
  if (inla_synth_grid_model(1, 0, &desc, &owner) != INLA_OK) return fail("inla_synth_grid_model");
  inla_model *model = NULL;
  const int rc = inla_model_create(&desc, 0, &model);
  inla_synth_free(owner); /* the model keeps its own device copies */
  if (rc != INLA_OK) return fail("inla_model_create");

  inla_eval_opts opts = {0};
  opts.grad = INLA_GRAD_FD_CENTRAL;
  opts.prior_mode = INLA_PRIOR_KRONECKER;
  opts.precision = INLA_FP64;
  double f = 0.0, grad[4] = {0.0, 0.0, 0.0, 0.0};
  int32_t status = -1, iters = -1;
  inla_eval_out_host out = {&f, grad, NULL, NULL, &status, &iters};
  if (inla_eval_batch_host(model, 1, theta, &opts, &out) != INLA_OK) {
    inla_model_destroy(model);
    return fail("inla_eval_batch_host");
  }
  printf("%.17g %.17g %.17g %.17g %.17g %d\n", f, grad[0], grad[1], grad[2], grad[3], (int)status);
  inla_model_destroy(model);
  return status == INLA_OK ? 0 : 1;
}
