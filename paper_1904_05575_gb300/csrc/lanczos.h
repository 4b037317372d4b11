// eps_M on a frequency grid by the Lanczos recursion (see lanczos.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/bse.h"

namespace bse {

// eps on the grid from the recursion on (A-B)(A+B); returns the steps taken,
// throws BSE_ERR_NO_CONV / NOT_PD / ARG.
int spectrum_lanczos(int n, const bse_c128* A, const bse_c128* B, int64_t ld, const bse_c128* rho,
                     double c_q, double vc, int n_omega, const double* omega, double delta,
                     double tol, int max_steps, int matvec_precision, bse_c128* eps_out,
                     cudaStream_t s);

}  // namespace bse
