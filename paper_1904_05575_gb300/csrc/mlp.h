// The learned preconditioner of the Davidson solver (see mlp.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace bse {

struct MlpNet;

// T[:, j] = g(features(alpha, E_j)) * R[:, j] for the n transitions and k
// columns, E on the device (k values), D = Re A_aa on the device.
void mlp_precondition(const MlpNet* net, int n, int k, const double* D, const double* E,
                      const double2* R, int64_t ldr, double2* T, int64_t ldt, cudaStream_t s);

}  // namespace bse
