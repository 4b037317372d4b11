// Batched FP64 complex GEMM on CUDA cores with user-defined operand access and
// epilogue, shared by the FP64 build and the Davidson solver.
#pragma once

#include <cuda_runtime.h>

#include "bse_internal.h"

namespace bse {
namespace {

struct cplx {
  double x, y;
};
__device__ __forceinline__ cplx cmake(double a, double b) { return {a, b}; }
__device__ __forceinline__ cplx ldc(const bse_c128* p) {
  double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ cplx conj(cplx a) { return {a.x, -a.y}; }

__device__ __forceinline__ double trans_energy(const double* e_v, const double* e_c, int nv,
                                               int nc, int64_t alpha) {
  int64_t k = alpha / (nv * nc);
  int v = (int)((alpha / nc) % nv);
  int c = (int)(alpha % nc);
  return e_c[k * nc + c] - e_v[k * nv + v];
}

// Batched complex GEMM C_b[m][n] = sum_k a(b, m, k) * b(b, n, k), result
// handed to P.store(b, m, n, value).  TM x TN tile per block, each thread
// RM x RN outputs, K staged through shared memory TK at a time.
template <int TM, int TN, int TK, int RM, int RN, class Prob>
__global__ void __launch_bounds__((TM / RM) * (TN / RN))
zgemm_batched(Prob P, int b0) {
  constexpr int NTM = TM / RM, NTN = TN / RN, NT = NTM * NTN;
  __shared__ double2 As[TK][TM];
  __shared__ double2 Bs[TK][TN];
  const int b = b0 + blockIdx.z;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int tid = threadIdx.x;
  const int tn = tid % NTN, tm = tid / NTN;
  double accx[RM][RN], accy[RM][RN];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < RN; ++j) accx[i][j] = accy[i][j] = 0.0;

  for (int k0 = 0; k0 < P.K; k0 += TK) {
    for (int i = tid; i < TM * TK; i += NT) {
      int mm = i / TK, kk = i % TK;
      cplx v = {0.0, 0.0};
      if (m0 + mm < P.M && k0 + kk < P.K) v = P.a(b, m0 + mm, k0 + kk);
      As[kk][mm] = make_double2(v.x, v.y);
    }
    for (int i = tid; i < TN * TK; i += NT) {
      int nn = i / TK, kk = i % TK;
      cplx v = {0.0, 0.0};
      if (n0 + nn < P.N && k0 + kk < P.K) v = P.b(b, n0 + nn, k0 + kk);
      Bs[kk][nn] = make_double2(v.x, v.y);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double2 av[RM], bv[RN];
#pragma unroll
      for (int i = 0; i < RM; ++i) av[i] = As[kk][tm + i * NTM];
#pragma unroll
      for (int j = 0; j < RN; ++j) bv[j] = Bs[kk][tn + j * NTN];
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) {
          accx[i][j] = fma(av[i].x, bv[j].x, accx[i][j]);
          accx[i][j] = fma(-av[i].y, bv[j].y, accx[i][j]);
          accy[i][j] = fma(av[i].x, bv[j].y, accy[i][j]);
          accy[i][j] = fma(av[i].y, bv[j].x, accy[i][j]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < RN; ++j) {
      int m = m0 + tm + i * NTM, n = n0 + tn + j * NTN;
      if (m < P.M && n < P.N) P.store(b, m, n, cmake(accx[i][j], accy[i][j]));
    }
}

template <class Prob>
void launch_zgemm(const Prob& P, int batch, cudaStream_t s) {
  // tile shape from the output shape; every config is 128 or 256 threads.
  // gridDim.z is capped at 65535, so large batches go in chunks.
  for (int b0 = 0; b0 < batch; b0 += 65535) {
    const int nb = batch - b0 < 65535 ? batch - b0 : 65535;
    if (P.M >= 48 && P.N >= 48) {
      dim3 grid((P.N + 63) / 64, (P.M + 63) / 64, nb);
      zgemm_batched<64, 64, 8, 4, 4, Prob><<<grid, 256, 0, s>>>(P, b0);
    } else if (P.M <= 16) {
      dim3 grid((P.N + 63) / 64, (P.M + 15) / 16, nb);
      zgemm_batched<16, 64, 16, 2, 4, Prob><<<grid, 128, 0, s>>>(P, b0);
    } else {
      dim3 grid((P.N + 31) / 32, (P.M + 31) / 32, nb);
      zgemm_batched<32, 32, 16, 2, 4, Prob><<<grid, 128, 0, s>>>(P, b0);
    }
    BSE_CUDA(cudaGetLastError());
    note_launches(1);
  }
}

// out[:, j] = H V[:, j], H Hermitian column-major: H[m][k] = conj(H[k + m ld])
struct MatvecProb {
  int M, N, K;
  const bse_c128* H;
  int64_t ld;
  const bse_c128* V;   // K x N, column-major, leading dimension ldv
  int64_t ldv;
  bse_c128* out;       // M x N, column-major, leading dimension ldo
  int64_t ldo;
  __device__ cplx a(int, int m, int k) const { return conj(ldc(H + (int64_t)m * ld + k)); }
  __device__ cplx b(int, int n, int k) const { return ldc(V + (int64_t)n * ldv + k); }
  __device__ void store(int, int m, int n, cplx v) const {
    reinterpret_cast<double2*>(out)[(int64_t)n * ldo + m] = make_double2(v.x, v.y);
  }
};

}  // namespace
}  // namespace bse
