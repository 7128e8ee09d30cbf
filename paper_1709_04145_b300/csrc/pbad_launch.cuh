// Launch-wide definitions shared by every kernel of the hot path: solver
// constants, step statuses, workspace and dense layouts, the launch
// arguments and the bucket lookup of a block.
#pragma once
#include "pbad_device.cuh"

namespace pbad {

constexpr int kMaxBuckets = 8;
constexpr double kLsC1 = 1e-4;     // Armijo constant
constexpr double kLsDelta = 0.1;   // approximate-Wolfe delta (Hager-Zhang)
constexpr double kLsEps = 1e-12;   // relative energy slack of approximate Wolfe
constexpr int kLsMax = 40;         // backtracking trials
constexpr double kCurvEps = 1e-14; // curvature-pair acceptance

enum Phase { kFirst = 1, kTrial = 2, kDone = 3 };
enum Status { kConverged = 0, kMaxIter = 1, kLsFail = 2, kCholFail = 3, kNonFinite = 4,
              kStalled = 5 };
// A step whose line search (or LM damping) cannot lower E while |r|_2 is at
// most kStallFactor times the rounding floor (Ctx::rnorm_floor) ends
// kStalled: solved as far as binary64 resolves r.
constexpr double kStallFactor = 1e3;

// Worst of two statuses in the order CONVERGED < STALLED < MAX_ITER <
// LS_FAIL < CHOL_FAIL < NONFINITE.
__host__ __device__ __forceinline__ int status_rank(int st) {
  return st == kStalled ? 1 : (st == kConverged ? 0 : st + 1);
}
__host__ __device__ __forceinline__ int status_worse(int a, int b) {
  return status_rank(b) > status_rank(a) ? b : a;
}

// Offsets (in doubles) of one lane's workspace.
struct WsLayout {
  int T, G, acc, axes, V, accd, C, Pb, ec, x, g, d, xt, gt, r, rt, qp, qc, sh, yh, rho;
  int u, jc;  // Jacobian-column scratch (present when Sd > 0)
  int tk;     // T(q_cur) per link: one-stage drag energy and contact (present when tk_region)
  int cg;     // 3 per contact point: adjoint load of the point at q_k (present with contact)
  int64_t total;
  __host__ __device__ void make(int N, int n, int m, int Sd = 0, int tk_region = 0, int nc = 0) {
    int o = 0;
    T = o; o += 12 * N;
    G = o; o += 12 * N;
    acc = o; o += 6 * N;
    axes = o; o += 9 * N;
    V = o; o += 6 * N;
    accd = o; o += 6 * N;
    C = o; o += 12 * N;
    Pb = o; o += 9 * N;
    ec = o; o += 4 * N;
    x = o; o += n;
    g = o; o += n;
    d = o; o += n;
    xt = o; o += n;
    gt = o; o += n;
    r = o; o += n;
    rt = o; o += n;
    qp = o; o += n;
    qc = o; o += n;
    sh = o; o += m * n;
    yh = o; o += m * n;
    rho = o; o += (m > 0 ? m : 1);
    u = o; o += (Sd ? n : 0);
    jc = o; o += (Sd ? n : 0);
    tk = o; o += (tk_region ? 12 * N : 0);
    cg = o; o += 3 * nc;
    total = o;
  }
};

// Per-instance dense storage of Newton and the adjoint (Sn = stages * n):
// J column-major [Sn][Sn] (column c contiguous; read row-major it is Jr^T),
// H and A row-major [Sn][Sn], then r, gg, dl, gb [Sn] each.
struct DenseLayout {
  int64_t J, H, A, r, gg, dl, gb, total;
  __host__ __device__ void make(int Sn) {
    const int64_t q = (int64_t)Sn * Sn;
    J = 0; H = q; A = 2 * q; r = 3 * q; gg = r + Sn; dl = gg + Sn; gb = dl + Sn; total = gb + Sn;
  }
};

struct LaunchArgs {
  int nb;
  int threads;             // threads per block (32, 64, 96 or 128)
  Bucket bk[kMaxBuckets];
  Colloc K;
  int history, max_iter, n_steps;
  int dense_stages;        // stages the dense Newton storage was sized for (0 = none)
  double tol;
  int64_t D;               // total DOFs of the batch (row length of DOF-packed arrays)
  const double* q_prev0;   // [D]
  const double* q_cur0;    // [D]
  const double* tau;       // [n_steps][D] or null
  const double* q_star;    // eval: [S*D] stage-packed
  double* E_out;           // eval: [instances]
  double* grad_out;        // eval: [S*D]
  double* resid_out;       // eval: [S*D] or null
  double* q_prev_out;      // [D] or null
  double* q_cur_out;       // [D] or null
  double* traj_prev;       // [n_steps][D] or null
  double* traj_cur;        // [n_steps][D] or null
  double* q_stages_out;    // [S*D] or null (last step's stages)
  double* stages_traj;     // [n_steps][S*D] or null (every step's stages)
  int* status;             // [instances] or null
  int* step_status;        // [n_steps][n_inst] each step's status, or null
  double* step_rnorm;      // [n_steps][n_inst] |r|_2 where each step ended, or null
  int64_t n_inst;          // instances of the launch (row length of the step logs)
  int df64;                // 1: the link-parallel evaluation's residual pass in double-float
  int cta_smem;            // dynamic shared memory of the rollout (CTA-mode Newton buckets)
  int* iters;              // [instances] or null
  int* evals;              // [instances] or null (objective evaluations)
  int* grads;              // [instances] or null (evaluations that formed dE/dq or Jr)
  // step backward (implicit-function adjoint)
  const double* g_bar;     // [S*D] dL/dq_* (stage-packed); segment adjoint: a_prev [D]
  const double* a_cur_in;  // segment adjoint: a_cur [D]
  double* gq_prev;         // [D]
  double* gq_cur;          // [D]
  double* gtau;            // [D]
  // link points
  int point_link[kMaxBuckets];  // link index per model
  const double* point_local;  // [instances][3] point in that link's frame
  double* point_pos;       // [instances][3]
  double* point_jac;       // [3 * D] per model block [count][3][n], or null
};

// Newton buckets with S n >= kNewtonCtaMin unknowns run one CTA of
// kNewtonCtaWarps warps per instance: the warps split the Jacobian columns
// and the whole CTA forms the Gram matrix and the Cholesky factor.
constexpr int kNewtonCtaWarps = 4;
constexpr int kNewtonCtaMin = 128;
constexpr int kNewtonCtaMaxSn = 4096;  // the vector of the solves sits in shared memory


// Bucket served by this block (buckets own consecutive block ranges).
__device__ __forceinline__ int find_bucket(const LaunchArgs& A) {
  int bk = 0;
  while (bk + 1 < A.nb && (int)blockIdx.x >= A.bk[bk + 1].block_begin) ++bk;
  return bk;
}

}  // namespace pbad
