// Objective/gradient evaluation whose scratch lives in a fixed device array
// of this library instead of memory allocated by a batch. For callers that
// cannot call cudaMalloc when they evaluate: a host application whose device
// memory is wholly owned by its own allocator (a cudaMalloc from us would
// fail or fragment its pool), or a latency-bound control loop that cannot
// afford the implicit device synchronisation and unbounded latency of an
// allocation. Declared in include/pbad.h.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/pbad.h"
#include "pbad_kernels.cuh"

namespace pbad {
cudaError_t launch_eval(int S, const LaunchArgs& A, int grid, cudaStream_t s);
int fill_launch_single(const pbad_model* m, int S, double dt, double* ws, LaunchArgs* A, int* grid,
                       int64_t* lanes, int64_t* per_lane);
int model_device(const pbad_model* m);
int set_error(int code, const char* msg);
}  // namespace pbad

using namespace pbad;

// The scratch: PBAD_STATIC_SCRATCH_BYTES per GPU, held by every device that
// loads the library until the process exits. Its name is only a host-side
// stand-in; kernels get the device address from cudaGetSymbolAddress.
static __device__ __align__(256) double g_pbad_static_scratch[PBAD_STATIC_SCRATCH_BYTES / sizeof(double)];

namespace {
// Device address of the scratch in the current context. It is looked up on
// every call rather than cached: after cudaDeviceReset, or with another
// context current, the library's module is loaded again and the array may
// sit at another address, so a cached pointer could point at freed memory.
// Once the module is loaded in the context the lookup is a table read. The
// first call in a context loads the module, which is why that call has to
// come before any stream capture.
int scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_pbad_static_scratch);
  if (e != cudaSuccess || !p) {
    char msg[160];
    std::snprintf(msg, sizeof(msg), "cudaGetSymbolAddress of the static scratch: %s",
                  cudaGetErrorString(e));
    return set_error(PBAD_ERR_CUDA, msg);
  }
  *out = static_cast<double*>(p);
  return PBAD_OK;
}
}  // namespace

extern "C" int pbad_eval_objective_grad_static(const pbad_model* model, const double* q_star,
                                               const double* q_prev, const double* q_cur,
                                               const double* tau, double dt, int32_t stages,
                                               double* E, double* grad, double* resid,
                                               void* stream) {
  if (!model) return set_error(PBAD_ERR_ARG, "null model");
  if (stages < 1 || stages > PBAD_MAX_STAGES) return set_error(PBAD_ERR_ARG, "stages out of range");
  if (!(dt > 0.0)) return set_error(PBAD_ERR_ARG, "dt must be positive");
  if (!q_star || !q_prev || !q_cur || !E || !grad) return set_error(PBAD_ERR_ARG, "null array");
  const int dev = model_device(model);
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return set_error(PBAD_ERR_CUDA, "cudaGetDevice failed");
  if (prev != dev && cudaSetDevice(dev) != cudaSuccess)
    return set_error(PBAD_ERR_CUDA, "cudaSetDevice failed");
  int rc = PBAD_OK;
  double* scratch = nullptr;
  LaunchArgs A;
  int grid = 0;
  int64_t lanes = 0, per_lane = 0;
  rc = scratch_address(&scratch);
  if (rc == PBAD_OK) rc = fill_launch_single(model, stages, dt, scratch, &A, &grid, &lanes, &per_lane);
  if (rc == PBAD_OK && (double)lanes * per_lane * sizeof(double) > (double)PBAD_STATIC_SCRATCH_BYTES) {
    char msg[200];
    std::snprintf(msg, sizeof(msg),
                  "problem needs %lld bytes of scratch; the static scratch holds %lld bytes "
                  "(use pbad_eval_objective_grad with a batch)",
                  (long long)(lanes * per_lane * (int64_t)sizeof(double)),
                  (long long)PBAD_STATIC_SCRATCH_BYTES);
    rc = set_error(PBAD_ERR_ARG, msg);
  }
  if (rc == PBAD_OK) {
    A.q_prev0 = q_prev;
    A.q_cur0 = q_cur;
    A.tau = tau;
    A.q_star = q_star;
    A.E_out = E;
    A.grad_out = grad;
    A.resid_out = resid;
    A.n_steps = 1;
    const cudaError_t e = launch_eval(stages, A, grid, (cudaStream_t)stream);
    if (e != cudaSuccess) {
      char msg[160];
      std::snprintf(msg, sizeof(msg), "eval launch: %s", cudaGetErrorString(e));
      rc = set_error(PBAD_ERR_CUDA, msg);
    }
  }
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  return rc;
}
