// C ABI of the PBAD library (declarations and contracts: include/pbad.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pbad.h"
#include "pbad_kernels.cuh"
#include "pbad_lp.cuh"
#include "pbad_cta.cuh"

namespace pbad {
#define PBAD_DECL(S)                                                                \
  cudaError_t launch_eval_s##S(const LaunchArgs& A, int grid, cudaStream_t s);     \
  cudaError_t launch_rollout_s##S(const LaunchArgs& A, int grid, cudaStream_t s);  \
  int rollout_blocks_per_sm_s##S(const LaunchArgs& A, int threads);
#define PBAD_DECL_BWD(S)                                                                        \
  cudaError_t launch_backward_s##S(const LaunchArgs& A, int grid, cudaStream_t s);             \
  cudaError_t launch_segment_backward_s##S(const LaunchArgs& A, int grid, cudaStream_t s);     \
  cudaError_t launch_eval_lp_s##S(const LaunchArgs& A, int grid, size_t smem, cudaStream_t s); \
  cudaError_t launch_rollout_lp_s##S(const LaunchArgs& A, int grid, size_t smem, cudaStream_t s);
PBAD_DECL_BWD(1)
PBAD_DECL_BWD(2)
PBAD_DECL_BWD(3)
PBAD_DECL_BWD(4)
PBAD_DECL_BWD(5)
PBAD_DECL(1)
PBAD_DECL(2)
PBAD_DECL(3)
PBAD_DECL(4)
PBAD_DECL(5)
cudaError_t launch_fp64_peak(double* out, int blocks, int threads, int iters);
cudaError_t launch_dmma_peak(double* out, int blocks, int threads, int iters);
cudaError_t launch_link_points(const LaunchArgs& A, int grid, cudaStream_t s);

cudaError_t launch_eval(int S, const LaunchArgs& A, int grid, cudaStream_t s) {
  switch (S) {
    case 1: return launch_eval_s1(A, grid, s);
    case 2: return launch_eval_s2(A, grid, s);
    case 3: return launch_eval_s3(A, grid, s);
    case 4: return launch_eval_s4(A, grid, s);
    case 5: return launch_eval_s5(A, grid, s);
  }
  return cudaErrorInvalidValue;
}
cudaError_t launch_backward(int S, const LaunchArgs& A, int grid, cudaStream_t s) {
  switch (S) {
    case 1: return launch_backward_s1(A, grid, s);
    case 2: return launch_backward_s2(A, grid, s);
    case 3: return launch_backward_s3(A, grid, s);
    case 4: return launch_backward_s4(A, grid, s);
    case 5: return launch_backward_s5(A, grid, s);
  }
  return cudaErrorInvalidValue;
}
cudaError_t launch_segment_backward(int S, const LaunchArgs& A, int grid, cudaStream_t s) {
  switch (S) {
    case 1: return launch_segment_backward_s1(A, grid, s);
    case 2: return launch_segment_backward_s2(A, grid, s);
    case 3: return launch_segment_backward_s3(A, grid, s);
    case 4: return launch_segment_backward_s4(A, grid, s);
    case 5: return launch_segment_backward_s5(A, grid, s);
  }
  return cudaErrorInvalidValue;
}
cudaError_t launch_eval_lp(int S, const LaunchArgs& A, int grid, size_t smem, cudaStream_t s) {
  switch (S) {
    case 1: return launch_eval_lp_s1(A, grid, smem, s);
    case 2: return launch_eval_lp_s2(A, grid, smem, s);
    case 3: return launch_eval_lp_s3(A, grid, smem, s);
    case 4: return launch_eval_lp_s4(A, grid, smem, s);
    case 5: return launch_eval_lp_s5(A, grid, smem, s);
  }
  return cudaErrorInvalidValue;
}
cudaError_t launch_rollout_lp(int S, const LaunchArgs& A, int grid, size_t smem, cudaStream_t s) {
  switch (S) {
    case 1: return launch_rollout_lp_s1(A, grid, smem, s);
    case 2: return launch_rollout_lp_s2(A, grid, smem, s);
    case 3: return launch_rollout_lp_s3(A, grid, smem, s);
    case 4: return launch_rollout_lp_s4(A, grid, smem, s);
    case 5: return launch_rollout_lp_s5(A, grid, smem, s);
  }
  return cudaErrorInvalidValue;
}
int rollout_blocks_per_sm(int S, const LaunchArgs& A, int threads) {
  switch (S) {
    case 1: return rollout_blocks_per_sm_s1(A, threads);
    case 2: return rollout_blocks_per_sm_s2(A, threads);
    case 3: return rollout_blocks_per_sm_s3(A, threads);
    case 4: return rollout_blocks_per_sm_s4(A, threads);
    case 5: return rollout_blocks_per_sm_s5(A, threads);
  }
  return 0;
}
cudaError_t launch_rollout(int S, const LaunchArgs& A, int grid, cudaStream_t s) {
  switch (S) {
    case 1: return launch_rollout_s1(A, grid, s);
    case 2: return launch_rollout_s2(A, grid, s);
    case 3: return launch_rollout_s3(A, grid, s);
    case 4: return launch_rollout_s4(A, grid, s);
    case 5: return launch_rollout_s5(A, grid, s);
  }
  return cudaErrorInvalidValue;
}
}  // namespace pbad

using namespace pbad;

struct pbad_model {
  int N = 0, n = 0, device = 0, chain = 1;
  // 1 if every link's mass moment has Sxy = Sxz = Syz = mcx = mcy = 0 (a body
  // symmetric about its frame's z axis: rods, capsules)
  int axial = 1;
  int64_t count = 0;
  double drag = 0.0;  // drag coefficient c of Q_drag (Section 6.2)
  std::vector<int> parent, jtype, dof;
  double g[3] = {0, 0, 0};
  int* d_topo = nullptr;     // parent[N] | jtype[N] | dof[N] | rest_eye[N] | sub_end[N]
  double* d_axis = nullptr;  // [N][3]
  double* d_mm = nullptr;    // [N][10][count]
  double* d_rest = nullptr;  // [N][12][count]
  // penalty contact (Eq. FRI): points grouped by link
  int n_contact = 0;
  double c_z0 = 0.0, c_d1 = 0.0, c_d2 = 0.0;
  int* d_coff = nullptr;     // [N + 1]
  double* d_cpt = nullptr;   // [n_contact][3]
};

struct pbad_batch {
  int device = 0, max_stages = 0, max_history = 0, flags = 0;
  int threads = 32;  // threads per block of the solver kernels
  std::vector<pbad_model*> models;
  std::vector<int64_t> inst_off, dof_off, lanes, lane_doubles;
  std::vector<int> tk;         // per bucket: workspace holds T(q_cur) (one-stage drag / contact)
  std::vector<int> nc;         // per bucket: contact points the workspace was laid out for
  std::vector<size_t> ws_off;  // in doubles
  int64_t n_inst = 0, D = 0;
  double* d_ws = nullptr;
  size_t ws_doubles = 0;
  // dense Newton/adjoint storage (PBAD_BATCH_NEWTON): per bucket
  // count * dense_stride doubles from dense_off
  double* d_dense = nullptr;
  size_t dense_doubles = 0;
  std::vector<size_t> dense_off;
  std::vector<int64_t> dense_stride;
  // instance queue of the rollouts: one counter per bucket; queue_blocks = 0
  // caps the L-BFGS buckets at the blocks the GPU keeps resident, > 0 at that
  // many blocks, < 0 (the default) turns the queue off
  int* d_queue = nullptr;
  int queue_blocks = -1;
  int mapping = PBAD_MAP_STAGE;  // instance-to-lane mapping of the L-BFGS and eval kernels
  std::vector<int> bucket_mapping;  // per bucket for steps and rollouts (-1: the batch's mapping)
  int precision = PBAD_PRECISION_F64;  // arithmetic of pbad_eval_objective_grad's residual pass
  int newton_cta_min = kNewtonCtaMin;  // Newton buckets with S n at least this run a CTA per instance
  int newton_split = 1;  // one-warp Newton: trial residual passes spread over the replicas
};

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  return fail(PBAD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Legendre roots on [-1, 1] in closed form (degrees 0..4).
void legendre(int deg, double* x) {
  switch (deg) {
    case 1: x[0] = 0.0; break;
    case 2: x[0] = -1.0 / std::sqrt(3.0); x[1] = -x[0]; break;
    case 3: x[0] = -std::sqrt(0.6); x[1] = 0.0; x[2] = -x[0]; break;
    case 4: {
      const double a = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(1.2));
      const double b = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(1.2));
      x[0] = -b; x[1] = -a; x[2] = a; x[3] = b;
      break;
    }
    default: break;
  }
}

// nodes[S+2] and W[S][S+2] (1/dt^2 units): second derivative of the Lagrange
// basis polynomial l_j at stage node t_i, by the product rule:
//   l_j''(t) = sum_{a != j} sum_{b != j, a} prod_{p != j, a, b} (t - x_p)
//              / prod_{p != j} (x_j - x_p).
int colloc_table(int S, double* nodes, double* W) {
  if (S < 1 || S > kMaxStages) return -1;
  double alpha[kMaxStages + 1];
  double r[kMaxStages];
  legendre(S - 1, r);
  alpha[0] = 0.0;
  for (int k = 1; k < S; ++k) alpha[k] = 0.5 * (r[k - 1] + 1.0);
  alpha[S] = 1.0;
  const int P = S + 2;
  nodes[0] = alpha[S - 1] - 1.0;
  nodes[1] = 0.0;
  for (int k = 1; k <= S; ++k) nodes[1 + k] = alpha[k];
  for (int i = 0; i < S; ++i) {
    const double t = nodes[2 + i];
    for (int j = 0; j < P; ++j) {
      double den = 1.0;
      for (int p = 0; p < P; ++p)
        if (p != j) den *= nodes[j] - nodes[p];
      double num = 0.0;
      for (int a = 0; a < P; ++a) {
        if (a == j) continue;
        for (int b = 0; b < P; ++b) {
          if (b == j || b == a) continue;
          double pr = 1.0;
          for (int p = 0; p < P; ++p)
            if (p != j && p != a && p != b) pr *= t - nodes[p];
          num += pr;
        }
      }
      W[i * P + j] = num / den;
    }
  }
  return 0;
}

// First derivatives of the Lagrange basis over the same nodes at the stage
// nodes, l_j'(t) = sum_{a != j} prod_{p != j, a} (t - x_p) / prod_{p != j} (x_j - x_p);
// one stage uses the drag potential's backward difference [0, -1, 1]
// (Section 6.2) instead. V[i * (S+2) + j], dimensionless.
int colloc_vel_table(int S, const double* nodes, double* V) {
  const int P = S + 2;
  if (S == 1) {
    V[0] = 0.0;
    V[1] = -1.0;
    V[2] = 1.0;
    return 0;
  }
  for (int i = 0; i < S; ++i) {
    const double t = nodes[2 + i];
    for (int j = 0; j < P; ++j) {
      double den = 1.0;
      for (int p = 0; p < P; ++p)
        if (p != j) den *= nodes[j] - nodes[p];
      double num = 0.0;
      for (int a = 0; a < P; ++a) {
        if (a == j) continue;
        double pr = 1.0;
        for (int p = 0; p < P; ++p)
          if (p != j && p != a) pr *= t - nodes[p];
        num += pr;
      }
      V[i * P + j] = num / den;
    }
  }
  return 0;
}

// Gauss-Jordan inverse of a small dense matrix (n <= kMaxStages).
bool small_inverse(int n, const double* A_, double* X) {
  double A[kMaxStages * kMaxStages];
  std::memcpy(A, A_, sizeof(double) * n * n);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) X[r * n + c] = (r == c) ? 1.0 : 0.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
    for (int k = 0; k < n; ++k) {
      std::swap(A[c * n + k], A[piv * n + k]);
      std::swap(X[c * n + k], X[piv * n + k]);
    }
    const double d = A[c * n + c];
    for (int k = 0; k < n; ++k) {
      A[c * n + k] /= d;
      X[c * n + k] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[r * n + c];
      for (int k = 0; k < n; ++k) {
        A[r * n + k] -= f * A[c * n + k];
        X[r * n + k] -= f * X[c * n + k];
      }
    }
  }
  return true;
}

int make_colloc(int S, double dt, Colloc* K) {
  double nodes[kMaxStages + 2], W[kMaxStages * (kMaxStages + 2)];
  if (colloc_table(S, nodes, W) != 0) return fail(PBAD_ERR_ARG, "stages out of range");
  std::memset(K, 0, sizeof(Colloc));
  K->S = S;
  K->dt = dt;
  const int P = S + 2;
  const double idt2 = 1.0 / (dt * dt);
  double V[kMaxStages * (kMaxStages + 2)];
  colloc_vel_table(S, nodes, V);
  for (int k = 0; k < P; ++k) K->nodes[k] = nodes[k];
  for (int i = 0; i < S; ++i) {
    K->Wk[i][0] = W[i * P + 0] * idt2;
    K->Wk[i][1] = W[i * P + 1] * idt2;
    K->Vk[i][0] = V[i * P + 0] * idt2;
    K->Vk[i][1] = V[i * P + 1] * idt2;
    for (int j = 0; j < S; ++j) {
      K->Wu[i][j] = W[i * P + 2 + j] * idt2;
      K->Vu[i][j] = V[i * P + 2 + j] * idt2;
    }
  }
  // stage block of the L-BFGS initial inverse Hessian:
  //   S == 1: dt^2; S >= 2: (Wu^T Wu)^-1 / 2
  if (S == 1) {
    K->Ps[0][0] = dt * dt;
  } else {
    double G[kMaxStages * kMaxStages], X[kMaxStages * kMaxStages];
    for (int a = 0; a < S; ++a)
      for (int b = 0; b < S; ++b) {
        double s = 0;
        for (int i = 0; i < S; ++i) s += K->Wu[i][a] * K->Wu[i][b];
        G[a * S + b] = s;
      }
    if (!small_inverse(S, G, X)) return fail(PBAD_ERR_ARG, "singular collocation block");
    for (int a = 0; a < S; ++a)
      for (int b = 0; b < S; ++b) K->Ps[a][b] = 0.5 * X[a * S + b];
  }
  return PBAD_OK;
}

int groups_per_warp(int S) { return 32 / S; }

// Launch description over every bucket. Buckets solved by Newton (and every
// bucket when all_warp is set: the adjoint) use one warp per instance; the
// others one group of S lanes per instance, floor(32/S) instances per warp.
int fill_launch(pbad_batch* bt, int S, double dt, const int32_t* solvers, int history,
                LaunchArgs* A, int* grid, bool all_warp = false) {
  std::memset(A, 0, sizeof(LaunchArgs));
  int rc = make_colloc(S, dt, &A->K);
  if (rc != PBAD_OK) return rc;
  A->nb = (int)bt->models.size();
  A->D = bt->D;
  A->history = history;
  A->threads = bt->threads;
  A->dense_stages = (bt->flags & PBAD_BATCH_NEWTON) ? bt->max_stages : 0;
  // Newton buckets with S n >= kNewtonCtaMin run one CTA of kNewtonCtaWarps
  // warps per instance; the launch then uses blocks of that many warps
  int max_cta_sn = 0;
  if (!all_warp)
    for (int k = 0; k < (int)bt->models.size(); ++k) {
      const int sn = S * bt->models[k]->n;
      if (solvers && solvers[k] == PBAD_NEWTON && sn >= bt->newton_cta_min && sn <= kNewtonCtaMaxSn)
        max_cta_sn = std::max(max_cta_sn, sn);
    }
  if (max_cta_sn > 0) A->threads = 32 * kNewtonCtaWarps;
  A->cta_smem = max_cta_sn > 0 ? (int)((2 * cta::kTile * cta::kPad + 32 + max_cta_sn) * sizeof(double)) : 0;
  const int wpb = A->threads / 32;
  int blocks = 0;
  for (int k = 0; k < A->nb; ++k) {
    const pbad_model* m = bt->models[k];
    Bucket& B = A->bk[k];
    B.N = m->N;
    B.n = m->n;
    B.count = (int)m->count;
    B.parent = m->d_topo;
    B.jtype = m->d_topo + m->N;
    B.dof = m->d_topo + 2 * m->N;
    B.rest_eye = m->d_topo + 3 * m->N;
    B.sub_end = m->d_topo + 4 * m->N;
    B.axis = m->d_axis;
    B.mm = m->d_mm;
    B.rest = m->d_rest;
    for (int c = 0; c < 3; ++c) B.g[c] = m->g[c];
    B.inst_off = bt->inst_off[k];
    B.dof_off = bt->dof_off[k];
    B.ws = bt->d_ws + bt->ws_off[k];
    B.ws_lane = bt->lane_doubles[k];
    B.block_begin = blocks;
    B.solver = solvers ? solvers[k] : PBAD_LBFGS;
    B.chain = m->chain;
    B.axial = m->axial;
    B.dense = bt->d_dense ? bt->d_dense + bt->dense_off[k] : nullptr;
    B.dense_stride = bt->d_dense ? bt->dense_stride[k] : 0;
    B.drag = m->drag;
    B.tk = bt->tk[k];
    if (S == 1 && (m->drag != 0.0 || m->n_contact > 0) && !B.tk)
      return fail(PBAD_ERR_ARG, "the model's drag or contact was set after the batch was created "
                                "(one-stage drag and contact need storage reserved at batch creation)");
    if (m->n_contact != bt->nc[k])
      return fail(PBAD_ERR_ARG, "the model's contact points changed after the batch was created");
    if (m->n_contact > 0 && S != 1)
      return fail(PBAD_ERR_UNSUPPORTED, "the penalty contact (Eq. FRI) is defined for one stage");
    B.n_contact = m->n_contact;
    B.c_off = m->d_coff;
    B.c_pt = m->d_cpt;
    B.c_z0 = m->c_z0;
    B.c_d1 = m->c_d1;
    B.c_d2 = m->c_d2;
    const bool warp_map = all_warp || B.solver == PBAD_NEWTON;
    const int sn = S * m->n;
    B.cta = (!all_warp && B.solver == PBAD_NEWTON && sn >= bt->newton_cta_min && sn <= kNewtonCtaMaxSn)
                ? kNewtonCtaWarps : 1;
    B.split = bt->newton_split;
    const int64_t warps = warp_map ? m->count * B.cta
                                   : (m->count + groups_per_warp(S) - 1) / groups_per_warp(S);
    blocks += (int)((warps + wpb - 1) / wpb);
  }
  *grid = blocks;
  return PBAD_OK;
}

// Instance queue: when the L-BFGS buckets need more blocks than the cap, each
// gets a share of the cap (at least one block) and its groups, once done with
// an instance, take the next one of the bucket from its queue counter.
// Returns whether a queue is in use.
bool apply_queue(pbad_batch* bt, int S, LaunchArgs* A, int* grid) {
  const int nb = A->nb;
  for (int k = 0; k < nb; ++k) {
    A->bk[k].queue = nullptr;
    A->bk[k].first_dynamic = 0;
  }
  if (bt->queue_blocks < 0 || !bt->d_queue) return false;
  // the queue variants serve launches whose buckets all use one L-BFGS kind
  for (int k = 1; k < nb; ++k)
    if (A->bk[k].solver != A->bk[0].solver) return false;
  if (A->bk[0].solver == PBAD_NEWTON) return false;
  int blocks[kMaxBuckets];
  int64_t lb_total = 0, other = 0;
  int n_lb = 0;
  for (int k = 0; k < nb; ++k) {
    blocks[k] = (k + 1 < nb ? A->bk[k + 1].block_begin : *grid) - A->bk[k].block_begin;
    if (A->bk[k].solver == PBAD_NEWTON) {
      other += blocks[k];
    } else {
      lb_total += blocks[k];
      ++n_lb;
    }
  }
  if (n_lb == 0) return false;
  int64_t cap = bt->queue_blocks;
  if (cap == 0) {
    const int per_sm = rollout_blocks_per_sm(S, *A, A->threads);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, bt->device) != cudaSuccess)
      sms = 0;
    if (per_sm <= 0 || sms <= 0) return false;
    cap = (int64_t)per_sm * sms - other;
  }
  if (cap < n_lb) cap = n_lb;
  if (lb_total <= cap) return false;
  const int wpb = A->threads / 32;
  int begin = 0;
  for (int k = 0; k < nb; ++k) {
    int nbk = blocks[k];
    if (A->bk[k].solver != PBAD_NEWTON) {
      nbk = (int)std::max<int64_t>(1, (int64_t)blocks[k] * cap / lb_total);
      A->bk[k].queue = bt->d_queue + k;
      A->bk[k].first_dynamic = nbk * wpb * groups_per_warp(S);
    }
    A->bk[k].block_begin = begin;
    begin += nbk;
  }
  *grid = begin;
  return true;
}

// Link-parallel launch over every bucket (PBAD_MAP_LINK): each bucket must
// be a serial chain with S N <= 32 lanes per instance, solved by binary64
// L-BFGS (solvers may be null for an evaluation), and for one stage carry no
// drag or contact. On success *smem is the dynamic shared memory per block.
int lp_eligible(const pbad_model* m, int S, int solver);

int fill_launch_lp(pbad_batch* bt, int S, double dt, const int32_t* solvers, int history,
                   LaunchArgs* A, int* grid, size_t* smem) {
  int rc = fill_launch(bt, S, dt, solvers, history, A, grid);
  if (rc != PBAD_OK) return rc;
  const int wpb = bt->threads / 32;
  int blocks = 0;
  for (int k = 0; k < A->nb; ++k) {
    const pbad_model* m = bt->models[k];
    rc = lp_eligible(m, S, solvers ? solvers[k] : PBAD_LBFGS);
    if (rc != PBAD_OK) return rc;
    const int per_warp = 32 / (S * m->N);
    const int64_t warps = (m->count + per_warp - 1) / per_warp;
    A->bk[k].block_begin = blocks;
    A->bk[k].queue = nullptr;
    blocks += (int)((warps + wpb - 1) / wpb);
  }
  LpLayout L;
  L.make(history);
  *smem = (size_t)wpb * 32 * L.total * sizeof(double);
  *grid = blocks;
  return PBAD_OK;
}

// The link mapping's conditions for bucket k (PBAD_OK or PBAD_ERR_UNSUPPORTED).
int lp_eligible(const pbad_model* m, int S, int solver) {
  if (!m->chain) return fail(PBAD_ERR_UNSUPPORTED, "link-parallel mapping: the model is not a serial chain");
  if (S * m->N > 32)
    return fail(PBAD_ERR_UNSUPPORTED, "link-parallel mapping: stages x links exceeds the 32 lanes of a warp");
  if (solver != PBAD_LBFGS) return fail(PBAD_ERR_UNSUPPORTED, "link-parallel mapping: binary64 L-BFGS only");
  if (S == 1 && (m->drag != 0.0 || m->n_contact > 0))
    return fail(PBAD_ERR_UNSUPPORTED, "link-parallel mapping: no one-stage drag or contact");
  return PBAD_OK;
}

// A launch where only some buckets run the link mapping (want[k]): after
// fill_launch, those buckets are checked, flagged, and the block ranges and
// the dynamic shared memory (the larger of the link-mapped warps' tiles and
// the CTA-mode Newton scratch) recomputed.
int mark_lp_buckets(pbad_batch* bt, int S, const int32_t* solvers, int history,
                    const std::vector<int>& want, LaunchArgs* A, int* grid) {
  const int wpb = A->threads / 32;
  int blocks = 0;
  for (int k = 0; k < A->nb; ++k) {
    const pbad_model* m = bt->models[k];
    Bucket& B = A->bk[k];
    int64_t warps;
    if (want[k]) {
      const int rc = lp_eligible(m, S, solvers ? solvers[k] : PBAD_LBFGS);
      if (rc != PBAD_OK) return rc;
      B.lp = 1;
      const int per_warp = 32 / (S * m->N);
      warps = (m->count + per_warp - 1) / per_warp;
    } else if (B.solver == PBAD_NEWTON) {
      warps = m->count * B.cta;
    } else {
      warps = (m->count + groups_per_warp(S) - 1) / groups_per_warp(S);
    }
    B.block_begin = blocks;
    B.queue = nullptr;
    blocks += (int)((warps + wpb - 1) / wpb);
  }
  LpLayout L;
  L.make(history);
  A->cta_smem = std::max(A->cta_smem, (int)(wpb * 32 * L.total * sizeof(double)));
  *grid = blocks;
  return PBAD_OK;
}

// Workspace lanes a Newton bucket needs: one warp per instance, or one CTA
// of kNewtonCtaWarps warps when S n can reach cta_min (warps rounded up to a
// multiple of 12 so that every block size of 1..4 warps launches whole
// blocks inside the allocation).
int64_t newton_lanes(const pbad_model* m, int max_stages, int cta_min) {
  const int64_t per = max_stages * m->n >= cta_min ? kNewtonCtaWarps : 1;
  return ((m->count * per + 11) / 12) * 12 * 32;
}

int check_common(pbad_batch* bt, int32_t stages, double dt) {
  if (!bt) return fail(PBAD_ERR_ARG, "null batch");
  if (stages < 1 || stages > bt->max_stages)
    return fail(PBAD_ERR_ARG, "stages must be in 1..max_stages of the batch");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(PBAD_ERR_ARG, "dt must be positive and finite");
  return PBAD_OK;
}

int rollout_impl(pbad_batch* bt, const double* q_prev0, const double* q_cur0,
                 const double* tau_seq, int32_t n_steps, double dt, int32_t stages,
                 const int32_t* solvers, int32_t history, double tol, int32_t max_iter,
                 double* traj_prev, double* traj_cur, double* q_prev_out, double* q_cur_out,
                 double* q_stages_out, int32_t* status, int32_t* iters, int32_t* evals,
                 int32_t* grads, int32_t* step_status, double* step_rnorm, double* stages_traj,
                 void* stream) {
  int rc = check_common(bt, stages, dt);
  if (rc != PBAD_OK) return rc;
  if (!q_prev0 || !q_cur0) return fail(PBAD_ERR_ARG, "null state");
  if (n_steps < 1) return fail(PBAD_ERR_ARG, "n_steps must be positive");
  if (history < 0 || history > bt->max_history)
    return fail(PBAD_ERR_ARG, "history must be in 0..max_history of the batch");
  if (max_iter < 0) return fail(PBAD_ERR_ARG, "max_iter must be >= 0");
  if (!(tol >= 0.0)) return fail(PBAD_ERR_ARG, "tol must be >= 0");
  for (size_t k = 0; k < bt->models.size(); ++k) {
    const int sv = solvers ? solvers[k] : PBAD_LBFGS;
    if (sv != PBAD_LBFGS && sv != PBAD_NEWTON && sv != PBAD_LBFGS_F32)
      return fail(PBAD_ERR_ARG, "unknown solver");
    if (sv == PBAD_NEWTON && !(bt->flags & PBAD_BATCH_NEWTON))
      return fail(PBAD_ERR_ARG, "the Newton solver needs a batch created with PBAD_BATCH_NEWTON");
  }
  DeviceGuard dg(bt->device);
  LaunchArgs A;
  int grid = 0;
  size_t smem = 0;
  const int nb = (int)bt->models.size();
  std::vector<int> want(nb);
  int n_lp = 0;
  for (int k = 0; k < nb; ++k) {
    const int mk = (k < (int)bt->bucket_mapping.size() && bt->bucket_mapping[k] >= 0)
                       ? bt->bucket_mapping[k] : bt->mapping;
    want[k] = mk == PBAD_MAP_LINK;
    n_lp += want[k];
  }
  const bool lp = n_lp == nb;  // every bucket link-mapped: the pure kernel
  if (lp) {
    std::vector<int32_t> sv(nb, PBAD_LBFGS);
    if (solvers) sv.assign(solvers, solvers + nb);
    rc = fill_launch_lp(bt, stages, dt, sv.data(), history, &A, &grid, &smem);
  } else {
    rc = fill_launch(bt, stages, dt, solvers, history, &A, &grid);
    if (rc == PBAD_OK && n_lp > 0) rc = mark_lp_buckets(bt, stages, solvers, history, want, &A, &grid);
  }
  if (rc != PBAD_OK) return rc;
  A.q_prev0 = q_prev0;
  A.q_cur0 = q_cur0;
  A.tau = tau_seq;
  A.n_steps = n_steps;
  A.tol = tol;
  A.max_iter = max_iter;
  A.traj_prev = traj_prev;
  A.traj_cur = traj_cur;
  A.q_prev_out = q_prev_out;
  A.q_cur_out = q_cur_out;
  A.q_stages_out = q_stages_out;
  A.stages_traj = stages_traj;
  A.status = status;
  A.step_status = step_status;
  A.step_rnorm = step_rnorm;
  A.n_inst = bt->n_inst;
  A.iters = iters;
  A.evals = evals;
  A.grads = grads;
  cudaStream_t s = (cudaStream_t)stream;
  if (lp) {
    const cudaError_t e = launch_rollout_lp(stages, A, grid, smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "link-parallel rollout launch");
    return PBAD_OK;
  }
  if (n_lp == 0 && apply_queue(bt, stages, &A, &grid)) {
    const cudaError_t e = cudaMemsetAsync(bt->d_queue, 0, sizeof(int) * kMaxBuckets, s);
    if (e != cudaSuccess) return cuda_fail(e, "queue reset");
  }
  const cudaError_t e = launch_rollout(stages, A, grid, s);
  if (e != cudaSuccess) return cuda_fail(e, "rollout launch");
  return PBAD_OK;
}

}  // namespace

extern "C" {

int pbad_version(void) { return 200; }

const char* pbad_last_error(void) { return g_err.c_str(); }

int pbad_colloc(int32_t stages, double* nodes, double* W) {
  if (!nodes || !W) return fail(PBAD_ERR_ARG, "null output");
  if (colloc_table(stages, nodes, W) != 0) return fail(PBAD_ERR_ARG, "stages out of range");
  return PBAD_OK;
}

int pbad_model_create(int32_t n_links, const int32_t* parent, const int32_t* joint_type,
                      const double* axis, int64_t count, const double* mass_moment,
                      const double* rest, const double* gravity, int32_t device,
                      pbad_model** out) {
  if (!out) return fail(PBAD_ERR_ARG, "null out");
  *out = nullptr;
  if (n_links <= 0 || n_links > 4096) return fail(PBAD_ERR_ARG, "n_links must be in 1..4096");
  if (count <= 0 || count > (int64_t)1 << 30) return fail(PBAD_ERR_ARG, "count must be in 1..2^30");
  if (!parent || !joint_type || !axis || !mass_moment || !rest || !gravity)
    return fail(PBAD_ERR_ARG, "null model array");
  auto* m = new (std::nothrow) pbad_model();
  if (!m) return fail(PBAD_ERR_ALLOC, "host allocation");
  m->N = n_links;
  m->count = count;
  m->device = device;
  int off = 0;
  for (int l = 0; l < n_links; ++l) {
    if (parent[l] < -1 || parent[l] >= l) {
      delete m;
      return fail(PBAD_ERR_ARG, "parent[l] must be in -1..l-1");
    }
    if (joint_type[l] != PBAD_HINGE && joint_type[l] != PBAD_BALL &&
        joint_type[l] != PBAD_TRANSLATION) {
      delete m;
      return fail(PBAD_ERR_ARG, "unknown joint type");
    }
    m->parent.push_back(parent[l]);
    if (parent[l] != l - 1) m->chain = 0;
    m->jtype.push_back(joint_type[l]);
    m->dof.push_back(off);
    off += joint_type[l] == PBAD_HINGE ? 1 : 3;
  }
  m->n = off;
  for (int c = 0; c < 3; ++c) m->g[c] = gravity[c];
  DeviceGuard dg(device);
  if (!dg.ok) {
    delete m;
    return fail(PBAD_ERR_CUDA, "cudaSetDevice failed");
  }
  std::vector<int> topo(5 * n_links);
  // subtree end: link l's descendants are l + 1 .. sub_end[l] - 1 when the
  // order numbers each subtree contiguously (depth-first), else N
  std::vector<int> size(n_links, 1);
  for (int l = n_links - 1; l > 0; --l)
    if (m->parent[l] >= 0) size[m->parent[l]] += size[l];
  bool contiguous = true;
  for (int l = 0; l < n_links && contiguous; ++l)
    for (int c = l + 1; c < l + size[l]; ++c) {  // every link inside must descend from l
      int a = c;
      while (a > l) a = m->parent[a];
      if (a != l) {
        contiguous = false;
        break;
      }
    }
  for (int l = 0; l < n_links; ++l) topo[4 * n_links + l] = contiguous ? l + size[l] : n_links;
  for (int l = 0; l < n_links; ++l) {
    topo[l] = m->parent[l];
    topo[n_links + l] = m->jtype[l];
    topo[2 * n_links + l] = m->dof[l];
    // identity rest rotation in every instance (exact comparison)
    int eye = 1;
    for (int64_t b = 0; b < count && eye; ++b)
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
          if (rest[((size_t)b * n_links + l) * 12 + 4 * r + c] != (r == c ? 1.0 : 0.0)) eye = 0;
    topo[3 * n_links + l] = eye;
  }
  // SoA over instances: [l][k][instance]
  std::vector<double> mm((size_t)n_links * 10 * count), rs((size_t)n_links * 12 * count);
  for (int64_t b = 0; b < count; ++b)
    for (int l = 0; l < n_links; ++l) {
      for (int k = 0; k < 10; ++k) {
        const double v = mass_moment[((size_t)b * n_links + l) * 10 + k];
        mm[((size_t)l * 10 + k) * count + b] = v;
        if ((k == 1 || k == 2 || k == 4 || k == 6 || k == 7) && v != 0.0) m->axial = 0;
      }
      for (int k = 0; k < 12; ++k)
        rs[((size_t)l * 12 + k) * count + b] = rest[((size_t)b * n_links + l) * 12 + k];
    }
  cudaError_t e;
  if ((e = cudaMalloc(&m->d_topo, sizeof(int) * topo.size())) != cudaSuccess ||
      (e = cudaMalloc(&m->d_axis, sizeof(double) * 3 * n_links)) != cudaSuccess ||
      (e = cudaMalloc(&m->d_mm, sizeof(double) * mm.size())) != cudaSuccess ||
      (e = cudaMalloc(&m->d_rest, sizeof(double) * rs.size())) != cudaSuccess) {
    pbad_model_destroy(m);
    return fail(PBAD_ERR_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  if ((e = cudaMemcpy(m->d_topo, topo.data(), sizeof(int) * topo.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(m->d_axis, axis, sizeof(double) * 3 * n_links, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(m->d_mm, mm.data(), sizeof(double) * mm.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(m->d_rest, rs.data(), sizeof(double) * rs.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
    pbad_model_destroy(m);
    return cuda_fail(e, "cudaMemcpy");
  }
  *out = m;
  return PBAD_OK;
}

int pbad_model_destroy(pbad_model* m) {
  if (!m) return PBAD_OK;
  DeviceGuard dg(m->device);
  cudaFree(m->d_topo);
  cudaFree(m->d_axis);
  cudaFree(m->d_mm);
  cudaFree(m->d_rest);
  cudaFree(m->d_coff);
  cudaFree(m->d_cpt);
  delete m;
  return PBAD_OK;
}

int pbad_model_set_contact(pbad_model* m, int32_t n_points, const int32_t* link,
                           const double* point, double z0, double d1, double d2) {
  if (!m) return fail(PBAD_ERR_ARG, "null model");
  if (n_points < 0 || n_points > 65536) return fail(PBAD_ERR_ARG, "n_points must be in 0..65536");
  if (n_points > 0 && (!link || !point)) return fail(PBAD_ERR_ARG, "null contact arrays");
  if (!(d1 >= 0.0) || !(d2 >= 0.0) || !std::isfinite(d1) || !std::isfinite(d2) || !std::isfinite(z0))
    return fail(PBAD_ERR_ARG, "d1, d2 must be finite and >= 0, z0 finite");
  for (int k = 0; k < n_points; ++k)
    if (link[k] < 0 || link[k] >= m->N) return fail(PBAD_ERR_ARG, "contact link out of range");
  // group the points by link (stable)
  std::vector<int> off(m->N + 1, 0);
  for (int k = 0; k < n_points; ++k) off[link[k] + 1]++;
  for (int l = 0; l < m->N; ++l) off[l + 1] += off[l];
  std::vector<double> pts(3 * (size_t)n_points);
  std::vector<int> fill(off.begin(), off.end() - 1);
  for (int k = 0; k < n_points; ++k) {
    const int at = fill[link[k]]++;
    for (int c = 0; c < 3; ++c) pts[3 * at + c] = point[3 * k + c];
  }
  DeviceGuard dg(m->device);
  if (!dg.ok) return fail(PBAD_ERR_CUDA, "cudaSetDevice failed");
  cudaFree(m->d_coff);
  cudaFree(m->d_cpt);
  m->d_coff = nullptr;
  m->d_cpt = nullptr;
  m->n_contact = 0;
  if (n_points > 0) {
    if (cudaMalloc(&m->d_coff, sizeof(int) * (m->N + 1)) != cudaSuccess ||
        cudaMalloc(&m->d_cpt, sizeof(double) * 3 * n_points) != cudaSuccess) {
      cudaFree(m->d_coff);
      m->d_coff = nullptr;
      return fail(PBAD_ERR_ALLOC, "contact cudaMalloc");
    }
    if (cudaMemcpy(m->d_coff, off.data(), sizeof(int) * (m->N + 1), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(m->d_cpt, pts.data(), sizeof(double) * 3 * n_points, cudaMemcpyHostToDevice) !=
            cudaSuccess)
      return fail(PBAD_ERR_CUDA, "contact cudaMemcpy");
  }
  m->n_contact = n_points;
  m->c_z0 = z0;
  m->c_d1 = d1;
  m->c_d2 = d2;
  return PBAD_OK;
}

int pbad_model_set_drag(pbad_model* m, double c) {
  if (!m) return fail(PBAD_ERR_ARG, "null model");
  if (!(c >= 0.0) || !std::isfinite(c)) return fail(PBAD_ERR_ARG, "drag must be finite and >= 0");
  m->drag = c;
  return PBAD_OK;
}

int pbad_model_info(const pbad_model* m, int32_t* n_links, int32_t* n_dof, int64_t* count) {
  if (!m) return fail(PBAD_ERR_ARG, "null model");
  if (n_links) *n_links = m->N;
  if (n_dof) *n_dof = m->n;
  if (count) *count = m->count;
  return PBAD_OK;
}

int pbad_batch_create(int32_t n_models, pbad_model* const* models, int32_t max_stages,
                      int32_t max_history, int32_t flags, pbad_batch** out) {
  if (!out) return fail(PBAD_ERR_ARG, "null out");
  *out = nullptr;
  if (n_models < 1 || n_models > PBAD_MAX_MODELS || !models)
    return fail(PBAD_ERR_ARG, "n_models must be in 1..PBAD_MAX_MODELS");
  if (max_stages < 1 || max_stages > PBAD_MAX_STAGES)
    return fail(PBAD_ERR_ARG, "max_stages must be in 1..PBAD_MAX_STAGES");
  if (max_history < 0 || max_history > PBAD_MAX_HISTORY)
    return fail(PBAD_ERR_ARG, "max_history must be in 0..PBAD_MAX_HISTORY");
  auto* bt = new (std::nothrow) pbad_batch();
  if (!bt) return fail(PBAD_ERR_ALLOC, "host allocation");
  if (flags & ~PBAD_BATCH_NEWTON) {
    delete bt;
    return fail(PBAD_ERR_ARG, "unknown batch flags");
  }
  bt->max_stages = max_stages;
  bt->max_history = max_history;
  bt->flags = flags;
  size_t ws = 0;
  for (int k = 0; k < n_models; ++k) {
    pbad_model* m = models[k];
    if (!m) {
      delete bt;
      return fail(PBAD_ERR_ARG, "null model in batch");
    }
    if (k > 0 && m->device != bt->device) {
      delete bt;
      return fail(PBAD_ERR_ARG, "models of a batch must share one device");
    }
    bt->device = m->device;
    bt->models.push_back(m);
    bt->inst_off.push_back(bt->n_inst);
    bt->dof_off.push_back(bt->D);
    bt->n_inst += m->count;
    bt->D += m->count * m->n;
    // the widest lane layout over the admissible stage counts (group
    // mapping) and, for Newton batches, one warp per instance
    // (warps rounded up to a multiple of 12 so that every block size of 1..4
    // warps launches whole blocks inside the allocation)
    int64_t lanes = 0;
    for (int S = 1; S <= max_stages; ++S) {
      const int64_t warps = (m->count + groups_per_warp(S) - 1) / groups_per_warp(S);
      const int64_t l = ((warps + 11) / 12) * 12 * 32;
      if (l > lanes) lanes = l;
    }
    if (flags & PBAD_BATCH_NEWTON) {
      lanes = std::max(lanes, newton_lanes(m, max_stages, kNewtonCtaMin));
      DenseLayout DL;
      DL.make(max_stages * m->n);
      bt->dense_off.push_back(bt->dense_doubles);
      bt->dense_stride.push_back(DL.total);
      bt->dense_doubles += (size_t)m->count * DL.total;
    }
    WsLayout L;
    // one-stage drag energy and contact need T(q_cur) per link
    const int tk = m->drag != 0.0 || m->n_contact > 0;
    L.make(m->N, m->n, max_history, (flags & PBAD_BATCH_NEWTON) ? max_stages : 0, tk,
           m->n_contact);
    bt->tk.push_back(tk);
    bt->nc.push_back(m->n_contact);
    bt->lanes.push_back(lanes);
    bt->lane_doubles.push_back(L.total);
    bt->ws_off.push_back(ws);
    ws += (size_t)lanes * L.total;
  }
  DeviceGuard dg(bt->device);
  bt->ws_doubles = ws;
  cudaError_t e = cudaMalloc(&bt->d_ws, sizeof(double) * ws);
  if (e != cudaSuccess) {
    delete bt;
    return fail(PBAD_ERR_ALLOC, std::string("workspace cudaMalloc: ") + cudaGetErrorString(e));
  }
  e = cudaMemset(bt->d_ws, 0, sizeof(double) * ws);
  if (e != cudaSuccess) {
    cudaFree(bt->d_ws);
    delete bt;
    return cuda_fail(e, "cudaMemset");
  }
  e = cudaMalloc(&bt->d_queue, sizeof(int) * kMaxBuckets);
  if (e != cudaSuccess) {
    cudaFree(bt->d_ws);
    delete bt;
    return fail(PBAD_ERR_ALLOC, std::string("queue cudaMalloc: ") + cudaGetErrorString(e));
  }
  if (bt->dense_doubles) {
    e = cudaMalloc(&bt->d_dense, sizeof(double) * bt->dense_doubles);
    if (e == cudaSuccess) e = cudaMemset(bt->d_dense, 0, sizeof(double) * bt->dense_doubles);
    if (e != cudaSuccess) {
      cudaFree(bt->d_ws);
      cudaFree(bt->d_dense);
      cudaFree(bt->d_queue);
      delete bt;
      return fail(PBAD_ERR_ALLOC, std::string("dense cudaMalloc: ") + cudaGetErrorString(e));
    }
  }
  *out = bt;
  return PBAD_OK;
}

int pbad_batch_destroy(pbad_batch* bt) {
  if (!bt) return PBAD_OK;
  DeviceGuard dg(bt->device);
  cudaFree(bt->d_ws);
  cudaFree(bt->d_dense);
  cudaFree(bt->d_queue);
  delete bt;
  return PBAD_OK;
}

int pbad_batch_set_queue(pbad_batch* bt, int32_t max_blocks) {
  if (!bt) return fail(PBAD_ERR_ARG, "null batch");
  bt->queue_blocks = max_blocks;
  return PBAD_OK;
}

int pbad_batch_info(const pbad_batch* bt, int64_t* n_instances, int64_t* n_dof_total,
                    int64_t* workspace_bytes) {
  if (!bt) return fail(PBAD_ERR_ARG, "null batch");
  if (n_instances) *n_instances = bt->n_inst;
  if (n_dof_total) *n_dof_total = bt->D;
  if (workspace_bytes)
    *workspace_bytes = (int64_t)((bt->ws_doubles + bt->dense_doubles) * sizeof(double));
  return PBAD_OK;
}

int pbad_eval_objective_grad(pbad_batch* bt, const double* q_star, const double* q_prev,
                             const double* q_cur, const double* tau, double dt, int32_t stages,
                             double* E, double* grad, double* resid, void* stream) {
  int rc = check_common(bt, stages, dt);
  if (rc != PBAD_OK) return rc;
  if (!q_star || !q_prev || !q_cur || !E || !grad) return fail(PBAD_ERR_ARG, "null array");
  DeviceGuard dg(bt->device);
  LaunchArgs A;
  int grid = 0;
  size_t smem = 0;
  const bool lp = bt->mapping == PBAD_MAP_LINK;
  if (bt->precision == PBAD_PRECISION_DF64 && !lp)
    return fail(PBAD_ERR_UNSUPPORTED, "the double-float residual pass runs in the link-parallel mapping");
  if (lp) rc = fill_launch_lp(bt, stages, dt, nullptr, 0, &A, &grid, &smem);
  else rc = fill_launch(bt, stages, dt, nullptr, 0, &A, &grid);
  if (rc != PBAD_OK) return rc;
  A.df64 = bt->precision == PBAD_PRECISION_DF64;
  A.q_prev0 = q_prev;
  A.q_cur0 = q_cur;
  A.tau = tau;
  A.q_star = q_star;
  A.E_out = E;
  A.grad_out = grad;
  A.resid_out = resid;
  A.n_steps = 1;
  cudaStream_t s = (cudaStream_t)stream;
  const cudaError_t e = lp ? launch_eval_lp(stages, A, grid, smem, s) : launch_eval(stages, A, grid, s);
  if (e != cudaSuccess) return cuda_fail(e, "eval launch");
  return PBAD_OK;
}

int pbad_rollout(pbad_batch* bt, const double* q_prev0, const double* q_cur0,
                 const double* tau_seq, int32_t n_steps, double dt, int32_t stages,
                 const int32_t* solvers, int32_t history, double tol, int32_t max_iter,
                 double* traj_prev, double* traj_cur, double* q_prev_out, double* q_cur_out,
                 int32_t* status, int32_t* iters, int32_t* evals, int32_t* grad_evals,
                 int32_t* step_status, double* step_rnorm, double* stages_traj, void* stream) {
  return rollout_impl(bt, q_prev0, q_cur0, tau_seq, n_steps, dt, stages, solvers, history, tol,
                      max_iter, traj_prev, traj_cur, q_prev_out, q_cur_out, nullptr, status, iters,
                      evals, grad_evals, step_status, step_rnorm, stages_traj, stream);
}

int pbad_step(pbad_batch* bt, const double* q_prev, const double* q_cur, const double* tau,
              double dt, int32_t stages, const int32_t* solvers, int32_t history, double tol,
              int32_t max_iter, double* q_prev_out, double* q_cur_out, double* q_stages_out,
              int32_t* status, int32_t* iters, void* stream) {
  return rollout_impl(bt, q_prev, q_cur, tau, 1, dt, stages, solvers, history, tol, max_iter,
                      nullptr, nullptr, q_prev_out, q_cur_out, q_stages_out, status, iters,
                      nullptr, nullptr, nullptr, nullptr, nullptr, stream);
}

int pbad_step_backward(pbad_batch* bt, const double* q_prev, const double* q_cur,
                       const double* tau, const double* q_star, const double* g_bar, double dt,
                       int32_t stages, double* gq_prev, double* gq_cur, double* gtau,
                       int32_t* status, void* stream) {
  int rc = check_common(bt, stages, dt);
  if (rc != PBAD_OK) return rc;
  if (!q_prev || !q_cur || !q_star || !g_bar || !gq_prev || !gq_cur || !gtau)
    return fail(PBAD_ERR_ARG, "null array");
  if (!(bt->flags & PBAD_BATCH_NEWTON))
    return fail(PBAD_ERR_ARG, "the adjoint needs a batch created with PBAD_BATCH_NEWTON");
  DeviceGuard dg(bt->device);
  LaunchArgs A;
  int grid = 0;
  rc = fill_launch(bt, stages, dt, nullptr, 0, &A, &grid, true);
  if (rc != PBAD_OK) return rc;
  A.q_prev0 = q_prev;
  A.q_cur0 = q_cur;
  A.tau = tau;
  A.q_star = q_star;
  A.g_bar = g_bar;
  A.gq_prev = gq_prev;
  A.gq_cur = gq_cur;
  A.gtau = gtau;
  A.status = status;
  A.n_steps = 1;
  const cudaError_t e = launch_backward(stages, A, grid, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "backward launch");
  return PBAD_OK;
}

int pbad_rollout_backward(pbad_batch* bt, const double* q_prev0, const double* q_cur0,
                          const double* tau_seq, const double* stages_traj, int32_t n_steps,
                          double dt, int32_t stages, const double* a_prev, const double* a_cur,
                          double* a_prev_out, double* a_cur_out, double* g_tau, int32_t* status,
                          void* stream) {
  int rc = check_common(bt, stages, dt);
  if (rc != PBAD_OK) return rc;
  if (!q_prev0 || !q_cur0 || !stages_traj || !a_prev || !a_cur || !a_prev_out || !a_cur_out || !g_tau)
    return fail(PBAD_ERR_ARG, "null array");
  if (n_steps < 1) return fail(PBAD_ERR_ARG, "n_steps must be positive");
  if (!(bt->flags & PBAD_BATCH_NEWTON))
    return fail(PBAD_ERR_ARG, "the adjoint needs a batch created with PBAD_BATCH_NEWTON");
  DeviceGuard dg(bt->device);
  LaunchArgs A;
  int grid = 0;
  rc = fill_launch(bt, stages, dt, nullptr, 0, &A, &grid, true);
  if (rc != PBAD_OK) return rc;
  A.q_prev0 = q_prev0;
  A.q_cur0 = q_cur0;
  A.tau = tau_seq;
  A.stages_traj = const_cast<double*>(stages_traj);
  A.g_bar = a_prev;
  A.a_cur_in = a_cur;
  A.gq_prev = a_prev_out;
  A.gq_cur = a_cur_out;
  A.gtau = g_tau;
  A.status = status;
  A.n_steps = n_steps;
  const cudaError_t e = launch_segment_backward(stages, A, grid, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "segment backward launch");
  return PBAD_OK;
}

int pbad_link_points(pbad_batch* bt, const double* q, const int32_t* link,
                     const double* point_local, double* pos, double* jac, void* stream) {
  if (!bt) return fail(PBAD_ERR_ARG, "null batch");
  if (!q || !link || !point_local || !pos) return fail(PBAD_ERR_ARG, "null array");
  for (size_t k = 0; k < bt->models.size(); ++k)
    if (link[k] < 0 || link[k] >= bt->models[k]->N) return fail(PBAD_ERR_ARG, "link index out of range");
  DeviceGuard dg(bt->device);
  LaunchArgs A;
  int grid = 0;
  int rc = fill_launch(bt, 1, 1.0, nullptr, 0, &A, &grid);
  if (rc != PBAD_OK) return rc;
  static_assert(PBAD_MAX_MODELS <= kMaxBuckets, "bucket table");
  A.q_cur0 = q;
  A.point_local = point_local;
  A.point_pos = pos;
  A.point_jac = jac;
  for (size_t k = 0; k < bt->models.size(); ++k) A.point_link[k] = link[k];  // in the parameter block
  const cudaError_t e = launch_link_points(A, grid, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "points launch");
  return PBAD_OK;
}

int pbad_batch_set_mapping(pbad_batch* bt, int32_t mapping) {
  if (!bt) return fail(PBAD_ERR_ARG, "null batch");
  if (mapping != PBAD_MAP_STAGE && mapping != PBAD_MAP_LINK) return fail(PBAD_ERR_ARG, "unknown mapping");
  bt->mapping = mapping;
  return PBAD_OK;
}

int pbad_batch_set_bucket_mapping(pbad_batch* bt, const int32_t* mapping) {
  if (!bt) return fail(PBAD_ERR_ARG, "null batch");
  if (!mapping) {
    bt->bucket_mapping.clear();
    return PBAD_OK;
  }
  std::vector<int> v(bt->models.size());
  for (size_t k = 0; k < v.size(); ++k) {
    if (mapping[k] != -1 && mapping[k] != PBAD_MAP_STAGE && mapping[k] != PBAD_MAP_LINK)
      return fail(PBAD_ERR_ARG, "unknown mapping");
    v[k] = mapping[k];
  }
  bt->bucket_mapping = v;
  return PBAD_OK;
}

int pbad_batch_set_newton_split(pbad_batch* bt, int32_t on) {
  if (!bt) return fail(PBAD_ERR_ARG, "null batch");
  if (on != 0 && on != 1) return fail(PBAD_ERR_ARG, "on must be 0 or 1");
  bt->newton_split = on;
  return PBAD_OK;
}

int pbad_batch_set_newton_cta_min(pbad_batch* bt, int32_t min_sn) {
  if (!bt) return fail(PBAD_ERR_ARG, "null batch");
  if (min_sn < 1 || min_sn > kNewtonCtaMaxSn + 1) return fail(PBAD_ERR_ARG, "min_sn out of range");
  if (!(bt->flags & PBAD_BATCH_NEWTON)) {
    bt->newton_cta_min = min_sn;
    return PBAD_OK;
  }
  // grow the workspace where a bucket now needs a CTA's lanes per instance
  const int nb = (int)bt->models.size();
  std::vector<int64_t> lanes(bt->lanes);
  bool grow = false;
  for (int k = 0; k < nb; ++k) {
    const int64_t need = newton_lanes(bt->models[k], bt->max_stages, min_sn);
    if (need > lanes[k]) {
      lanes[k] = need;
      grow = true;
    }
  }
  if (grow) {
    std::vector<size_t> off(nb);
    size_t ws = 0;
    for (int k = 0; k < nb; ++k) {
      off[k] = ws;
      ws += (size_t)lanes[k] * bt->lane_doubles[k];
    }
    DeviceGuard dg(bt->device);
    double* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double) * ws);
    if (e != cudaSuccess)
      return fail(PBAD_ERR_ALLOC, std::string("workspace cudaMalloc: ") + cudaGetErrorString(e));
    e = cudaMemset(d, 0, sizeof(double) * ws);
    if (e != cudaSuccess) {
      cudaFree(d);
      return cuda_fail(e, "cudaMemset");
    }
    cudaFree(bt->d_ws);  // waits for the launches that still use it
    bt->d_ws = d;
    bt->ws_doubles = ws;
    bt->ws_off = off;
    bt->lanes = lanes;
  }
  bt->newton_cta_min = min_sn;
  return PBAD_OK;
}

int pbad_batch_set_precision(pbad_batch* bt, int32_t precision) {
  if (!bt) return fail(PBAD_ERR_ARG, "null batch");
  if (precision != PBAD_PRECISION_F64 && precision != PBAD_PRECISION_DF64)
    return fail(PBAD_ERR_ARG, "unknown precision");
  bt->precision = precision;
  return PBAD_OK;
}

int pbad_batch_set_threads(pbad_batch* bt, int32_t threads) {
  if (!bt) return fail(PBAD_ERR_ARG, "null batch");
  if (threads != 32 && threads != 64 && threads != 96 && threads != 128)
    return fail(PBAD_ERR_ARG, "threads per block must be 32, 64, 96 or 128");
  bt->threads = threads;
  return PBAD_OK;
}

int pbad_fp64_peak(int32_t device, double* gflops) {
  if (!gflops) return fail(PBAD_ERR_ARG, "null output");
  DeviceGuard dg(device);
  if (!dg.ok) return fail(PBAD_ERR_CUDA, "cudaSetDevice failed");
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return cuda_fail(e, "attribute");
  const int threads = 256, blocks = sms * 4, iters = 20000;
  double* d = nullptr;
  if ((e = cudaMalloc(&d, sizeof(double) * threads * blocks)) != cudaSuccess)
    return fail(PBAD_ERR_ALLOC, "probe buffer");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    launch_fp64_peak(d, blocks, threads, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "probe");
  *gflops = 2.0 * 8.0 * iters * (double)threads * blocks / (best * 1e-3) / 1e9;
  return PBAD_OK;
}

int pbad_fp64_mma_peak(int32_t device, double* gflops) {
  if (!gflops) return fail(PBAD_ERR_ARG, "null output");
  DeviceGuard dg(device);
  if (!dg.ok) return fail(PBAD_ERR_CUDA, "cudaSetDevice failed");
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return cuda_fail(e, "attribute");
  const int threads = 256, blocks = sms * 4, iters = 4000;
  double* d = nullptr;
  if ((e = cudaMalloc(&d, sizeof(double) * threads * blocks)) != cudaSuccess)
    return fail(PBAD_ERR_ALLOC, "probe buffer");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    launch_dmma_peak(d, blocks, threads, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "probe");
  // per warp and iteration: 8 mma of 8 x 8 x 4 FMA (2 flops each)
  const double warps = (double)threads / 32 * blocks;
  *gflops = 2.0 * 256.0 * 8.0 * iters * warps / (best * 1e-3) / 1e9;
  return PBAD_OK;
}

}  // extern "C"

// Launch description of one model with a caller-provided lane workspace, for
// entry points that do not own a batch. Returns PBAD_OK or an error code;
// on success *lanes and *per_lane give the workspace the launch touches
// (lanes * per_lane doubles from ws).
namespace pbad {
int fill_launch_single(const pbad_model* m, int S, double dt, double* ws, LaunchArgs* A, int* grid,
                       int64_t* lanes, int64_t* per_lane) {
  if (!m) return fail(PBAD_ERR_ARG, "null model");
  std::memset(A, 0, sizeof(LaunchArgs));
  int rc = make_colloc(S, dt, &A->K);
  if (rc != PBAD_OK) return rc;
  const int64_t warps = (m->count + groups_per_warp(S) - 1) / groups_per_warp(S);
  const int64_t blocks = (warps + 3) / 4;
  WsLayout L;
  const int tk = m->drag != 0.0 || m->n_contact > 0;
  if (m->n_contact > 0 && S != 1)
    return fail(PBAD_ERR_UNSUPPORTED, "the penalty contact (Eq. FRI) is defined for one stage");
  L.make(m->N, m->n, 0, 0, tk, m->n_contact);
  *lanes = blocks * 4 * 32;
  *per_lane = L.total;
  A->nb = 1;
  A->D = m->count * m->n;
  A->threads = 128;
  Bucket& B = A->bk[0];
  B.N = m->N;
  B.n = m->n;
  B.count = (int)m->count;
  B.parent = m->d_topo;
  B.jtype = m->d_topo + m->N;
  B.dof = m->d_topo + 2 * m->N;
  B.rest_eye = m->d_topo + 3 * m->N;
  B.sub_end = m->d_topo + 4 * m->N;
  B.axis = m->d_axis;
  B.mm = m->d_mm;
  B.rest = m->d_rest;
  for (int c = 0; c < 3; ++c) B.g[c] = m->g[c];
  B.ws = ws;
  B.ws_lane = L.total;
  B.block_begin = 0;
  B.chain = m->chain;
  B.axial = m->axial;
  B.drag = m->drag;
  B.tk = tk;
  B.n_contact = m->n_contact;
  B.c_off = m->d_coff;
  B.c_pt = m->d_cpt;
  B.c_z0 = m->c_z0;
  B.c_d1 = m->c_d1;
  B.c_d2 = m->c_d2;
  *grid = (int)blocks;
  return PBAD_OK;
}
int model_device(const pbad_model* m) { return m->device; }
int set_error(int code, const char* msg) { return fail(code, msg); }
}  // namespace pbad
