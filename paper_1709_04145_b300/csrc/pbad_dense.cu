// The damped Gauss-Newton system of the LM step (Section 5) on its own: for
// a batch of square Jacobians, H = J^T J, the Cholesky factor of H + lambda I
// and dl = -(H + lambda I)^-1 g, one CTA per instance with the same device
// routines (pbad_cta.cuh) as the CTA-mode Newton rollout. Declared in
// include/pbad.h as pbad_damped_gram_solve.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "../../include/pbad.h"
#include "pbad_cta.cuh"
#include "pbad_kernels.cuh"

namespace pbad {
int set_error(int code, const char* msg);

namespace {
constexpr int kDenseThreads = 128;  // cta::syrk's thread layout

__global__ void __launch_bounds__(kDenseThreads) k_damped_gram_solve(
    const double* __restrict__ J, const double* __restrict__ g, int n, double lambda, double* H,
    double* L, double* dl, int32_t* status) {
  extern __shared__ double smem[];
  double* sa = smem;
  double* sc = sa + cta::kTile * cta::kPad;
  double* red = sc + cta::kTile * cta::kPad;
  double* vec = red + 32;
  const int64_t b = blockIdx.x, nn = (int64_t)n * n;
  cta::syrk(J + b * nn, H + b * nn, n, sa, sc);
  const bool ok =
      cta::factor_solve(H + b * nn, L + b * nn, g + b * n, dl + b * n, n, lambda, vec, red, sa, sc);
  if (threadIdx.x == 0) status[b] = ok ? PBAD_CONVERGED : PBAD_CHOL_FAIL;
}
}  // namespace
}  // namespace pbad

using namespace pbad;

extern "C" int pbad_damped_gram_solve(int64_t count, int32_t n, const double* J, const double* g,
                                      double lambda, double* H, double* L, double* dl,
                                      int32_t* status, void* stream) {
  if (count < 0 || count > 0x7fffffff) return set_error(PBAD_ERR_ARG, "count out of range");
  if (n < 1 || n > kNewtonCtaMaxSn) return set_error(PBAD_ERR_ARG, "n out of range (1..4096)");
  if (!std::isfinite(lambda)) return set_error(PBAD_ERR_ARG, "lambda must be finite");
  if (count == 0) return PBAD_OK;
  if (!J || !g || !H || !L || !dl || !status) return set_error(PBAD_ERR_ARG, "null array");
  const size_t smem = (2 * cta::kTile * cta::kPad + 32 + (size_t)n) * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (smem > 48 * 1024)
    e = cudaFuncSetAttribute(k_damped_gram_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  if (e == cudaSuccess) {
    k_damped_gram_solve<<<(unsigned)count, kDenseThreads, smem, (cudaStream_t)stream>>>(
        J, g, n, lambda, H, L, dl, status);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    char msg[160];
    std::snprintf(msg, sizeof(msg), "pbad_damped_gram_solve launch: %s", cudaGetErrorString(e));
    return set_error(PBAD_ERR_CUDA, msg);
  }
  return PBAD_OK;
}
