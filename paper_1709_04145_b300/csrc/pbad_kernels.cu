// Kernels of the PBAD hot path: batched objective/gradient evaluation and the
// persistent L-BFGS rollout. See pbad_kernels.cuh for the per-lane passes.
#include "pbad_kernels.cuh"

#ifndef PBAD_S
#error "compile with -DPBAD_S=<stages>"
#endif

namespace pbad {

}  // namespace pbad
#include "pbad_lp.cuh"
#include "pbad_cta.cuh"
namespace pbad {

// Lane identity inside a bucket: groups of S lanes, floor(32/S) groups per warp.
template <int S>
struct LaneId {
  int64_t lane_id;  // lane index inside the bucket's workspace
  int64_t inst;     // instance index inside the bucket (may be >= count)
  bool real;        // lane belongs to a full group
  __device__ LaneId(const Bucket& B) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)(blockIdx.x - B.block_begin) * blockDim.x + threadIdx.x) >> 5;
    constexpr int G = 32 / S;
    lane_id = warp * 32 + lane;
    real = lane < G * S;
    inst = warp * G + lane / S;
  }
};

// ------------------------------------------------------------------------
// E, r and dE/dq at given stage configurations (one evaluation per instance)
// ------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(128) k_eval(const __grid_constant__ LaunchArgs A) {
  const Bucket& B = A.bk[find_bucket(A)];
  const LaneId<S> id(B);
  const bool active = id.real && id.inst < B.count;
  const int b = active ? (int)id.inst : 0;
  Ctx<S> c(B, A.K, b, id.lane_id, 0);
  for (int d = 0; d < c.n; ++d) {
    c.ws[c.L.qp + d] = A.q_prev0[c.gdof(d)];
    c.ws[c.L.qc + d] = A.q_cur0[c.gdof(d)];
  }
  c.setup(true);
  for (int d = 0; d < c.n; ++d) c.ws[c.L.xt + d] = A.q_star[c.gstage(d)];
  const double E = c.evaluate(A.tau);
  if (active) {
    if (c.i == 0) A.E_out[B.inst_off + b] = E;
    for (int d = 0; d < c.n; ++d) {
      A.grad_out[c.gstage(d)] = c.ws[c.L.gt + d];
      if (A.resid_out) A.resid_out[c.gstage(d)] = c.ws[c.L.rt + d];
    }
  }
}

// ------------------------------------------------------------------------
// Persistent L-BFGS rollout: every group of S lanes integrates one instance
// for n_steps steps. Each loop trip evaluates E, r, dE/dq at every group's
// current trial point, then advances every group's state machine (line
// search, history update, convergence, next step) - the iteration-level
// scheduling of the paper's Fig. GPU, inside a warp. The whole trip is
// convergent: every vector sweep runs once per warp with per-group
// predicates, so groups in different phases share one pass over the
// workspace instead of taking turns through divergent branches.
// ------------------------------------------------------------------------
template <int S, bool F32, bool QUEUE>
__device__ __noinline__ void rollout_lbfgs(const LaunchArgs& A, const Bucket& B) {
  const LaneId<S> id(B);
  const bool active = id.real && id.inst < B.count;
  int b = active ? (int)id.inst : 0;
  const int m = A.history;
  constexpr bool f32 = F32;  // binary32 two-loop recursion (PBAD_LBFGS_F32)
  Ctx<S> c(B, A.K, b, id.lane_id, m);
  // c goes to the non-inlined passes; cv, a private copy used by the inline
  // helpers only, keeps the layout and lane fields in registers across the
  // workspace stores of the solver bookkeeping. Addresses of the group's
  // instance in the caller's arrays follow b (the queue may move it).
  const Ctx<S> cv(c);
  const int n = c.n;
  const WsLayout L = c.L;
  const Lane ws = c.ws;
  const int64_t D = A.D;
  constexpr unsigned kAll = 0xffffffffu;
  auto gdof = [&](int d) { return B.dof_off + (int64_t)b * n + d; };
  auto gstage = [&](int d) { return (int64_t)S * B.dof_off + ((int64_t)b * S + cv.i) * n + d; };

  for (int d = 0; d < n; ++d) {
    ws[L.qp + d] = A.q_prev0[gdof(d)];
    ws[L.qc + d] = A.q_cur0[gdof(d)];
  }
  int step = 0, phase = kFirst, k = 0, trials = 0, nh = 0, head = 0, step_evals = 0;
  int worst = kConverged, iters_total = 0, evals_total = 0, grads_total = 0;
  double E = 0.0, alpha = 1.0, gd = 0.0, gamma = 1.0;
  double rn_x = 0.0;  // |r|_2 at the current (last accepted) point
  double rstall = kStallFactor * c.rnorm_floor();
  const int max_evals = 4 * A.max_iter + kLsMax;  // evaluations per step
  c.setup(true);
  if (!active) phase = kDone;

  // outputs of the group's instance once its last step has ended
  auto finish_instance = [&]() {
    if (cv.i == 0) {
      if (A.status) A.status[B.inst_off + b] = worst;
      if (A.iters) A.iters[B.inst_off + b] = iters_total;
      if (A.evals) A.evals[B.inst_off + b] = evals_total;
      if (A.grads) A.grads[B.inst_off + b] = grads_total;
      for (int d = 0; d < n; ++d) {
        if (A.q_prev_out) A.q_prev_out[gdof(d)] = ws[L.qp + d];
        if (A.q_cur_out) A.q_cur_out[gdof(d)] = ws[L.qc + d];
      }
    }
  };
  // the next instance of the bucket's queue (group-uniform; the group's
  // lanes call it together): rebinds the context and loads its state
  auto next_instance = [&]() -> bool {
    if (!B.queue) return false;
    int nb = 0;
    if (cv.i == 0) nb = B.first_dynamic + atomicAdd(B.queue, 1);
    nb = __shfl_sync(cv.grp.mask, nb, cv.grp.src(0));
    if (nb >= B.count) return false;
    b = nb;
    c.b = nb;
    rstall = kStallFactor * c.rnorm_floor();
    for (int d = 0; d < n; ++d) {
      ws[L.qp + d] = A.q_prev0[gdof(d)];
      ws[L.qc + d] = A.q_cur0[gdof(d)];
    }
    step = 0;
    worst = kConverged;
    iters_total = evals_total = grads_total = 0;
    return true;
  };

  while (__any_sync(kAll, phase != kDone)) {
    const double* tau = A.tau ? A.tau + (int64_t)min(step, A.n_steps - 1) * D : nullptr;
    const double Et = c.evaluate_primal(tau);
    const bool live = phase != kDone;
    if (live) {
      ++evals_total;
      ++step_evals;
    }
    const bool first = live && phase == kFirst;
    const bool trial = live && phase == kTrial;
    // The gradient at xt is read by a step's first evaluation, by an accepted
    // trial (the next direction) and by the approximate-Wolfe test of a trial
    // whose energy lies within its band; a trial above both bounds is
    // rejected on E alone. The tangent pass (S >= 2) runs on the trips where
    // some group of the warp reads the gradient: the decisions are the same
    // as with a gradient at every trial.
    const bool need_g = first || (trial && isfinite(Et) &&
                                  (Et <= E + kLsEps * fabs(E) || Et <= E + kLsC1 * alpha * gd));
    if (need_g) ++grads_total;
    if (S == 1) {
      if (need_g)
        for (int d = 0; d < n; ++d) ws[L.gt + d] = ws[L.rt + d];
    } else if (__any_sync(kAll, need_g)) {
      c.tangent();
    }

    // (1) line-search test at xt = x + alpha d: Armijo or approximate Wolfe
    bool ok = false;
    if (__any_sync(kAll, trial)) {
      double gtd = 0.0, fin = 1.0;
      if (trial && need_g)
        for (int d0 = 0; d0 < n; d0 += Ctx<S>::kChunk) {
          double gv[Ctx<S>::kChunk], dv[Ctx<S>::kChunk];
#pragma unroll
          for (int k = 0; k < Ctx<S>::kChunk; ++k)
            if (d0 + k < n) {
              gv[k] = ws[L.gt + d0 + k];
              dv[k] = ws[L.d + d0 + k];
            }
#pragma unroll
          for (int k = 0; k < Ctx<S>::kChunk; ++k)
            if (d0 + k < n) {
              if (!isfinite(gv[k])) fin = 0.0;
              gtd = fma(gv[k], dv[k], gtd);
            }
        }
      fin = cv.grp.sum(fin);
      gtd = cv.grp.sum(gtd);
      if (trial && fin == (double)S && isfinite(Et)) {
        const bool armijo = Et <= E + kLsC1 * alpha * gd;
        const bool approx = (Et <= E + kLsEps * fabs(E)) && (gtd <= (1.0 - 2.0 * kLsDelta) * fabs(gd));
        ok = armijo || approx;
      }
    }
    int fin_st = -1;  // status of a step that ends on this trip
    if (trial && !ok) {
      if (step_evals >= max_evals) fin_st = kMaxIter;
      else if (++trials >= kLsMax) fin_st = rn_x <= rstall ? kStalled : kLsFail;
      else alpha *= 0.5;
    }
    const bool back = trial && !ok && fin_st < 0;  // next trial along the same d
    const bool acc = first || ok;                  // xt becomes the current point

    // (2) one sweep: accepted groups take (xt, gt, rt) and form the curvature
    // pair s = xt - x, y = gt - g (s into rt, y into gt and d, all dead now);
    // backtracking groups move xt = x + alpha d in the same sweep.
    double sy = 0.0, ss = 0.0, yy = 0.0, rr = 0.0, badg = 0.0;
    if (__any_sync(kAll, acc || back)) {
      constexpr int kC = Ctx<S>::kChunk;
      for (int d0 = 0; d0 < n; d0 += kC) {
        double xv[kC], gv[kC], rv[kC], xo[kC], go[kC];
#pragma unroll
        for (int k = 0; k < kC; ++k)
          if (d0 + k < n) {
            // back: xv = d, xo = x
            xv[k] = acc ? ws[L.xt + d0 + k] : (back ? ws[L.d + d0 + k] : 0.0);
            gv[k] = acc ? ws[L.gt + d0 + k] : 0.0;
            rv[k] = acc ? ws[L.rt + d0 + k] : 0.0;
            xo[k] = (ok || back) ? ws[L.x + d0 + k] : 0.0;
            go[k] = ok ? ws[L.g + d0 + k] : 0.0;
          }
#pragma unroll
        for (int k = 0; k < kC; ++k)
          if (d0 + k < n) {
            const int d = d0 + k;
            if (acc) {
              if (ok) {
                const double s_ = xv[k] - xo[k], y_ = gv[k] - go[k];
                sy = fma(s_, y_, sy);
                ss = fma(s_, s_, ss);
                yy = fma(y_, y_, yy);
                ws[L.rt + d] = s_;
                ws[L.gt + d] = y_;
                ws[L.d + d] = y_;
              }
              ws[L.x + d] = xv[k];
              ws[L.g + d] = gv[k];
              ws[L.r + d] = rv[k];
              rr = fma(rv[k], rv[k], rr);
              if (!isfinite(gv[k])) badg = 1.0;
            } else if (back) {
              ws[L.xt + d] = fma(alpha, xv[k], xo[k]);
            }
          }
      }
      sy = cv.grp.sum(sy);
      ss = cv.grp.sum(ss);
      yy = cv.grp.sum(yy);
      rr = cv.grp.sum(rr);
      badg = cv.grp.sum(badg);
    }

    // (3) curvature pair into the ring buffer: rho = 1/s^T y, gamma = s^T y / y^T P y
    const bool pair = ok && m > 0 && sy > kCurvEps * sqrt(ss) * sqrt(yy);
    if (__any_sync(kAll, pair)) {
      c.precond(pair ? L.d : L.gt);  // gt is dead for every other group
      double yPy = 0.0;
      if (pair) {
        constexpr int kC = Ctx<S>::kChunk;
        for (int d0 = 0; d0 < n; d0 += kC) {
          double yv[kC], pv[kC], sv[kC];
#pragma unroll
          for (int k = 0; k < kC; ++k)
            if (d0 + k < n) {
              yv[k] = ws[L.gt + d0 + k];
              pv[k] = ws[L.d + d0 + k];
              sv[k] = ws[L.rt + d0 + k];
            }
#pragma unroll
          for (int k = 0; k < kC; ++k)
            if (d0 + k < n) {
              yPy = fma(yv[k], pv[k], yPy);
              if constexpr (!f32) {
                ws[L.sh + head * n + d0 + k] = sv[k];
                ws[L.yh + head * n + d0 + k] = yv[k];
              }
            }
          if constexpr (f32) {  // packed binary32 pairs (kC even: d0 / 2 is a slot)
#pragma unroll
            for (int k = 0; k < kC; k += 2)
              if (d0 + k < n) {
                const bool two = d0 + k + 1 < n;
                const int o = (d0 + k) >> 1;
                ws[L.sh + head * n + o] = Ctx<S>::pack32(__double2float_rn(sv[k]),
                                                         two ? __double2float_rn(sv[k + 1]) : 0.0f);
                ws[L.yh + head * n + o] = Ctx<S>::pack32(__double2float_rn(yv[k]),
                                                         two ? __double2float_rn(yv[k + 1]) : 0.0f);
              }
          }
        }
      }
      yPy = cv.grp.sum(yPy);
      if (pair) {
        ws[L.rho + head] = 1.0 / sy;
        head = (head + 1) % m;
        if (nh < m) ++nh;
        gamma = sy / yPy;
      }
    }

    // (4) tests at the new current point
    bool start = false;
    if (acc) {
      E = Et;
      rn_x = sqrt(rr);
      if (first) {
        k = 0;
        nh = 0;
        head = 0;
        gamma = 1.0;
      } else {
        ++k;
        ++iters_total;
      }
      if (badg != 0.0 || !isfinite(E) || !isfinite(rr)) fin_st = kNonFinite;
      else if (sqrt(rr) < A.tol) fin_st = kConverged;
      else if (k >= A.max_iter || step_evals >= max_evals) fin_st = kMaxIter;
      else start = true;
    }

    // (5) steps that end: q_prev' = stage S-2 (q_cur when S = 1), q_cur' =
    // stage S-1, trajectory, then the next step's setup for every group
    // that goes on
    const bool fin = fin_st >= 0;
    if (__any_sync(kAll, fin)) {
      if (fin) {
        worst = status_worse(worst, fin_st);
        step_evals = 0;
        if (cv.i == 0) {
          const int64_t o = (int64_t)step * A.n_inst + B.inst_off + b;
          if (A.step_status) A.step_status[o] = fin_st;
          if (A.step_rnorm) A.step_rnorm[o] = rn_x;
        }
      }
      for (int d = 0; d < n; ++d) {
        const double xv = ws[L.x + d];
        const double xs = cv.grp.from(xv, S - 1);
        const double xp = (S == 1) ? ws[L.qc + d] : cv.grp.from(xv, S - 2);
        if (fin) {
          ws[L.qp + d] = xp;
          ws[L.qc + d] = xs;
          if (cv.i == 0) {
            if (A.traj_cur) A.traj_cur[(int64_t)step * D + gdof(d)] = xs;
            if (A.traj_prev) A.traj_prev[(int64_t)step * D + gdof(d)] = xp;
          }
          if (A.q_stages_out && step == A.n_steps - 1) A.q_stages_out[gstage(d)] = xv;
          if (A.stages_traj) A.stages_traj[(int64_t)step * S * D + gstage(d)] = xv;
        }
      }
      bool next = false;
      if (fin) {
        ++step;
        next = step < A.n_steps;
        if constexpr (QUEUE) {
          if (!next) {
            finish_instance();
            next = next_instance();
          }
        }
        phase = next ? kFirst : kDone;
      }
      if (__any_sync(kAll, next)) c.setup(next);
    }

    // (6) two-loop recursion with H0 = gamma P for the groups that start an
    // iteration (in binary32 on binary32 pairs for PBAD_LBFGS_F32); a
    // non-descent direction falls back to -P g, then to -g (binary64). Each
    // sweep applies one update and forms the next step's dot product.
    if (__any_sync(kAll, start)) {
      double gd0;
      if constexpr (f32) {
        gd0 = c.direction32(start, nh, head, gamma, m);
      } else {
        const int nh_w = __reduce_max_sync(kAll, start ? nh : 0);
        if (start) cv.vlin(L.d, -1.0, L.g, -1);
        auto slot = [&](int t) { return (head - 1 - t + 2 * m) % m; };
        double al[kMaxHistory];
        double a = 0.0;
        if (nh_w > 0) a = ws[L.rho + slot(0)] * cv.gdot(L.sh + slot(0) * n, L.d);
        for (int t = 0; t < nh_w; ++t) {
          const int j = slot(t);
          al[t] = a;
          const bool more = t + 1 < nh_w;
          const int jn = more ? slot(t + 1) : 0;
          const double dot = cv.axpy_dot(L.d, -a, L.yh + j * n, more ? L.sh + jn * n : -1, start && t < nh);
          if (more) a = ws[L.rho + jn] * dot;
        }
        c.precond(start ? L.d : L.gt);
        if (start) cv.vlin(L.d, gamma, L.d, -1);
        if (nh_w > 0) {
          double bta = ws[L.rho + slot(nh_w - 1)] * cv.gdot(L.yh + slot(nh_w - 1) * n, L.d);
          for (int t = nh_w - 1; t >= 0; --t) {
            const int j = slot(t);
            const int jn = t > 0 ? slot(t - 1) : 0;
            const double dot = cv.axpy_dot(L.d, al[t] - bta, L.sh + j * n, t > 0 ? L.yh + jn * n : L.g,
                                          start && t < nh);
            if (t > 0) bta = ws[L.rho + jn] * dot;
            else gd0 = dot;
          }
        } else {
          gd0 = cv.gdot(L.g, L.d);
        }
      }
      if (start) gd = gd0;
      const bool reset = start && !(gd < 0.0);
      if (__any_sync(kAll, reset)) {
        if (reset) {
          nh = 0;
          gamma = 1.0;
          cv.vlin(L.d, -1.0, L.g, -1);
        }
        c.precond(reset ? L.d : L.gt);
        const double gd1 = cv.gdot(L.g, L.d);
        if (reset) gd = gd1;
        // -P g not a descent direction either (P not positive definite in
        // rounding): steepest descent
        const bool sd = reset && !(gd < 0.0);
        if (__any_sync(kAll, sd)) {
          if (sd) cv.vlin(L.d, -1.0, L.g, -1);
          const double gd2 = cv.gdot(L.g, L.d);
          if (sd) gd = gd2;
        }
      }
      if (start) {
        alpha = 1.0;
        trials = 0;
        cv.vlin(L.xt, 1.0, L.d, L.x);
        phase = kTrial;
      }
    }
  }
  if constexpr (!QUEUE) {
    if (active) finish_instance();
  }
}

// ------------------------------------------------------------------------
// Persistent Newton (Levenberg-Marquardt) rollout, Section 5:
//   q <- q - [H + lambda I]^-1 g,  H = Jr^T Jr, g = Jr^T r   (S >= 2)
//                                  H = int dP/dq^T dP/dq / dt^2, g = dE/dq (S == 1)
// lambda starts at 1e-12 max diag(H) per step; a damped step that does not
// lower E is halved up to three times before lambda grows x10 (a failed
// Cholesky factorisation grows it at once); lambda shrinks x0.1 (floor 1e-20
// max diag) after a full damped step is accepted and stays after a halved
// one; a step is accepted when E decreases. One warp per instance:
// R = 32/S replicas of the stage group evaluate the same point and split the
// S n Jacobian columns; the Gram matrix, Cholesky and solves are shared by
// the warp's lanes (the paper's workgroup per trajectory, Fig. GPU).
// ------------------------------------------------------------------------
constexpr int kLmMaxTrials = 60;
constexpr int kLmHalvings = 3;  // halvings of a damped step before lambda grows

// Lane identity of the warp-per-instance mapping (cta = 1) or of the
// CTA-per-instance mapping of large Newton buckets (cta warps per instance,
// warp wid of the instance).
template <int S>
struct WarpId {
  int64_t lane_id, inst;
  int rep, R, wid;
  __device__ WarpId(const Bucket& B, int cta = 1) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)(blockIdx.x - B.block_begin) * blockDim.x + threadIdx.x) >> 5;
    lane_id = warp * 32 + lane;
    inst = warp / cta;
    wid = (int)(warp - inst * cta);
    R = 32 / S;
    rep = lane / S;  // rep == R: surplus lanes (S = 3, 5)
  }
};

__device__ __forceinline__ double bcast0(double v) { return __shfl_sync(0xffffffffu, v, 0); }

// Gram matrix of the CTA mode: H = Jr^T Jr and gg = Jr^T r (S >= 2, the
// syrk on the column-major Jacobian) or the Gauss-Newton matrix and gg = r
// (S == 1); returns max diag(H) on every thread.
template <int S>
__device__ double gram_cta(const Ctx<S>& c, double* D, const DenseLayout& DL, double* sa,
                           double* sc, double* red) {
  const int Sn = S * c.n;
  const int tid = threadIdx.x, nth = blockDim.x;
  if (S == 1) {
    for (int e = tid; e < Sn * Sn; e += nth) {
      const int a = e / Sn, cc = e - a * Sn;
      D[DL.H + e] = D[DL.J + (int64_t)cc * Sn + a];
    }
    for (int a = tid; a < Sn; a += nth) D[DL.gg + a] = D[DL.r + a];
    __syncthreads();
  } else {
    cta::syrk(D + DL.J, D + DL.H, Sn, sa, sc);
    // gg[a] = column a of Jr . r: one warp per column, lanes over the rows
    const int w = tid >> 5, lane = tid & 31, nw = nth >> 5;
    for (int a = w; a < Sn; a += nw) {
      double g = 0.0;
      for (int rr = lane; rr < Sn; rr += 32) g = fma(D[DL.J + (int64_t)a * Sn + rr], D[DL.r + rr], g);
      for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
      if (lane == 0) D[DL.gg + a] = g;
    }
    __syncthreads();
  }
  double hm = 0.0;
  for (int a = tid; a < Sn; a += nth) hm = fmax(hm, D[DL.H + (int64_t)a * Sn + a]);
  return cta::block_max(hm, red);
}

template <int S>
__device__ __noinline__ void rollout_newton(const LaunchArgs& A, const Bucket& B) {
  // CTA mode (B.cta > 1): the instance's warps run the same state machine on
  // the same values (each evaluates the residual pass itself), split the
  // Jacobian columns, and form the Gram matrix and the factor together.
  const int ncta = B.cta > 1 ? B.cta : 1;
  const WarpId<S> id(B, ncta);
  const bool active = id.inst < B.count;
  const int b = active ? (int)id.inst : 0;
  Ctx<S> c(B, A.K, b, id.lane_id, A.history, A.dense_stages);
  const int n = c.n;
  const auto& L = c.L;
  const Lane& ws = c.ws;
  const int64_t D = A.D;
  const bool writer = active && id.rep == 0 && id.wid == 0;  // one replica writes the outputs
  double* Dn = B.dense + (int64_t)b * B.dense_stride;
  DenseLayout DL;
  DL.make(S * n);
  extern __shared__ double dyn_smem[];  // CTA mode: syrk tiles, reduction scratch, a vector
  double* s_sa = dyn_smem;
  double* s_sc = s_sa + cta::kTile * cta::kPad;
  double* s_red = s_sc + cta::kTile * cta::kPad;
  double* s_vec = s_red + 32;
  // replica index and count over the whole CTA (surplus lanes stay surplus)
  const int rep_g = id.rep < id.R ? id.wid * id.R + id.rep : ncta * id.R;
  const int R_g = ncta * id.R;

  for (int d = 0; d < n; ++d) {
    ws[L.qp + d] = A.q_prev0[c.gdof(d)];
    ws[L.qc + d] = A.q_cur0[c.gdof(d)];
  }
  int step = 0, phase = kFirst, k = 0, trials = 0, halvings = 0;
  int worst = kConverged, iters_total = 0, evals_total = 0, grads_total = 0;
  double E = 0.0, lambda = -1.0, hmax = 0.0, alpha = 1.0;
  double rn_x = 0.0;  // |r|_2 at the current (last accepted) point
  const double rstall = kStallFactor * c.rnorm_floor();
  c.setup(true);
  if (!active) phase = kDone;  // warp-uniform

  auto gsum_bcast = [&](double v) {
    double t = 0.0;
#pragma unroll
    for (int j = 0; j < S; ++j) t += c.grp.from_full(v, j);
    return bcast0(t);
  };

  auto finish = [&](int st) {
    worst = status_worse(worst, st);
    if (writer && c.i == 0) {
      const int64_t o = (int64_t)step * A.n_inst + B.inst_off + b;
      if (A.step_status) A.step_status[o] = st;
      if (A.step_rnorm) A.step_rnorm[o] = rn_x;
    }
    for (int d = 0; d < n; ++d) {
      const double xs = c.grp.from_full(ws[L.x + d], S - 1);
      const double xp = (S == 1) ? ws[L.qc + d] : c.grp.from_full(ws[L.x + d], S - 2);
      ws[L.qp + d] = xp;
      ws[L.qc + d] = xs;
      if (writer && c.i == 0) {
        if (A.traj_cur) A.traj_cur[(int64_t)step * D + c.gdof(d)] = xs;
        if (A.traj_prev) A.traj_prev[(int64_t)step * D + c.gdof(d)] = xp;
      }
    }
    if (writer && A.q_stages_out && step == A.n_steps - 1)
      for (int d = 0; d < n; ++d) A.q_stages_out[c.gstage(d)] = ws[L.x + d];
    if (writer && A.stages_traj)
      for (int d = 0; d < n; ++d) A.stages_traj[(int64_t)step * S * D + c.gstage(d)] = ws[L.x + d];
    ++step;
    if (step >= A.n_steps) {
      phase = kDone;
    } else {
      c.setup(true);
      phase = kFirst;
    }
  };

  // trial points of the one-warp mode: residual pass spread over the replicas
  // (the same bits as every replica evaluating it; the Jacobian that follows
  // an accepted trial first completes the lanes' per-link arrays)
  const bool split_ok = ncta == 1 && S >= 2 && B.split;
  while (phase != kDone) {
    const double* tau = A.tau ? A.tau + (int64_t)min(step, A.n_steps - 1) * D : nullptr;
    const bool split = split_ok && phase == kTrial;
    const double Et = bcast0(split ? c.evaluate_primal_split(tau, id.rep, id.R)
                                   : c.evaluate_primal(tau));
    ++evals_total;
    double rrt = 0.0, fint = 1.0;
    for (int d = 0; d < n; ++d) {
      rrt = fma(ws[L.rt + d], ws[L.rt + d], rrt);
      if (!isfinite(ws[L.rt + d])) fint = 0.0;
    }
    rrt = gsum_bcast(rrt);
    fint = gsum_bcast(fint);
    int need = 0;  // 1: Jacobian at x, 2: new factorisation
    double rr = 0.0;
    if (phase == kFirst) {
      for (int d = 0; d < n; ++d) {
        ws[L.x + d] = ws[L.xt + d];
        ws[L.r + d] = ws[L.rt + d];
      }
      E = Et;
      rr = rrt;
      rn_x = sqrt(rr);
      k = 0;
      lambda = -1.0;
      need = 1;
    } else {
      double rr0 = 0.0;
      for (int d = 0; d < n; ++d) rr0 = fma(ws[L.r + d], ws[L.r + d], rr0);
      rr0 = gsum_bcast(rr0);
      const bool ok = fint == (double)S && isfinite(Et) &&
                      (Et < E || (S == 1 && Et <= E + kLsEps * fabs(E) && rrt < rr0));
      if (ok) {
        for (int d = 0; d < n; ++d) {
          ws[L.x + d] = ws[L.xt + d];
          ws[L.r + d] = ws[L.rt + d];
        }
        E = Et;
        rr = rrt;
        rn_x = sqrt(rr);
        if (alpha == 1.0) lambda = fmax(lambda * 0.1, 1e-20 * hmax);
        ++k;
        ++iters_total;
        need = 1;
      } else if (halvings < kLmHalvings) {
        // half of the damped step before a larger lambda
        ++halvings;
        alpha *= 0.5;
        for (int d = 0; d < n; ++d) ws[L.xt + d] = fma(alpha, Dn[DL.dl + c.i * n + d], ws[L.x + d]);
        __syncwarp();
      } else {
        lambda *= 10.0;
        if (++trials >= kLmMaxTrials) finish(rn_x <= rstall ? kStalled : kLsFail);
        else need = 2;
      }
    }
    if (need == 1) {
      if (fint != (double)S || !isfinite(E)) { finish(kNonFinite); need = 0; }
      else if (sqrt(rr) < A.tol) { finish(kConverged); need = 0; }
      else if (k >= A.max_iter) { finish(kMaxIter); need = 0; }
    }
    if (need == 1) {
      if (id.rep == 0 && id.wid == 0)
        for (int d = 0; d < n; ++d) Dn[DL.r + c.i * n + d] = ws[L.r + d];
      if (ncta > 1) {
        c.build_jacobian_warp(Dn, DL, rep_g, R_g, false);
        __syncthreads();
        hmax = gram_cta(c, Dn, DL, s_sa, s_sc, s_red);
      } else {
        __syncwarp();
        if (split) c.complete_split(id.R);
        c.build_jacobian_warp(Dn, DL, id.rep, id.R, false);
        hmax = c.gram_warp(Dn, DL);
      }
      ++grads_total;
      if (lambda < 0.0) lambda = 1e-12 * hmax;
      trials = 0;
      need = 2;
    }
    if (need == 2) {
      bool solved = false;
      while (!solved) {
        const bool f = ncta > 1 ? cta::factor_solve(Dn + DL.H, Dn + DL.A, Dn + DL.gg, Dn + DL.dl,
                                                   S * n, lambda, s_vec, s_red, s_sa, s_sc)
                               : c.factor_solve_warp(Dn, DL, lambda);
        if (f) {
          solved = true;
        } else {
          lambda *= 10.0;
          if (++trials >= kLmMaxTrials) break;
        }
      }
      if (!solved) {
        finish(kCholFail);
      } else {
        for (int d = 0; d < n; ++d) ws[L.xt + d] = ws[L.x + d] + Dn[DL.dl + c.i * n + d];
        alpha = 1.0;
        halvings = 0;
        phase = kTrial;
      }
      __syncwarp();
    }
  }
  if (writer && c.i == 0) {
    if (A.status) A.status[B.inst_off + b] = worst;
    if (A.iters) A.iters[B.inst_off + b] = iters_total;
    if (A.evals) A.evals[B.inst_off + b] = evals_total;
    if (A.grads) A.grads[B.inst_off + b] = grads_total;
    for (int d = 0; d < n; ++d) {
      if (A.q_prev_out) A.q_prev_out[c.gdof(d)] = ws[L.qp + d];
      if (A.q_cur_out) A.q_cur_out[c.gdof(d)] = ws[L.qc + d];
    }
  }
}

// One launch serves every bucket of the batch; each block runs the solver of
// its bucket (L-BFGS, Newton or L-BFGS with the binary32 direction) in the
// bucket's mapping, so an uneven batch with mixed solvers and mappings is a
// single persistent launch. SOLVERS selects the variant: 0 every bucket
// L-BFGS, 1 every bucket Newton, 3 every bucket binary32-direction L-BFGS, 2
// mixed (the only variant with link-mapped buckets next to others); 4 and 5
// are 0 and 3 with the instance queue. The single-solver variants carry only their own solver's
// code and registers (the queue's rebinding costs the others ~8% on large
// batches, hence its own variants).
template <int S, int SOLVERS>
__global__ void __maxnreg__(255) k_rollout(const __grid_constant__ LaunchArgs A) {
  const Bucket& B = A.bk[find_bucket(A)];
  if (SOLVERS == 2 && B.lp) rollout_lp<S>(A, B);  // a link-mapped bucket of a mixed launch
  else if (SOLVERS == 0) rollout_lbfgs<S, false, false>(A, B);
  else if (SOLVERS == 1) rollout_newton<S>(A, B);
  else if (SOLVERS == 3) rollout_lbfgs<S, true, false>(A, B);
  else if (SOLVERS == 4) rollout_lbfgs<S, false, true>(A, B);
  else if (SOLVERS == 5) rollout_lbfgs<S, true, true>(A, B);
  else if (B.solver == 1) rollout_newton<S>(A, B);
  else if (B.solver == 2) rollout_lbfgs<S, true, false>(A, B);
  else rollout_lbfgs<S, false, false>(A, B);
}

// ------------------------------------------------------------------------
// Implicit-function-theorem adjoint of one converged step. With
// r(q_*; q_prev, q_cur, tau) = 0 at the solution, dq_* = -Jr^-1 dr, so for a
// loss gradient gbar = dL/dq_*:  Jr^T mu = gbar, dL/dq_prev = -(dr/dq_prev)^T mu,
// dL/dq_cur = -(dr/dq_cur)^T mu, dL/dtau = sum_i mu_i. Jr is built exactly
// (S n tangent passes split over the warp's replicas; the exact Hessian of
// Eq. EQ for one stage) and solved by the warp's pivoted elimination; the
// known-node products are adjoint sweeps at q_prev and q_cur whose seeds come
// from the stage transforms' tangents along mu. One warp per instance.
// ------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(128) k_step_backward(const __grid_constant__ LaunchArgs A) {
  const Bucket& B = A.bk[find_bucket(A)];
  const WarpId<S> id(B);
  const bool active = id.inst < B.count;
  if (!active) return;  // warp-uniform
  const int b = (int)id.inst;
  Ctx<S> c(B, A.K, b, id.lane_id, 0, A.dense_stages);
  const int n = c.n;
  const auto& L = c.L;
  const Lane& ws = c.ws;
  const bool writer = id.rep == 0;
  double* Dn = B.dense + (int64_t)b * B.dense_stride;
  DenseLayout DL;
  DL.make(S * n);
  for (int d = 0; d < n; ++d) {
    ws[L.qp + d] = A.q_prev0[c.gdof(d)];
    ws[L.qc + d] = A.q_cur0[c.gdof(d)];
  }
  c.setup(true);
  for (int d = 0; d < n; ++d) ws[L.xt + d] = A.q_star[c.gstage(d)];
  if (writer)
    for (int d = 0; d < n; ++d) Dn[DL.gb + c.i * n + d] = A.g_bar[c.gstage(d)];
  c.primal(A.tau);
  __syncwarp();
  c.build_jacobian_warp(Dn, DL, id.rep, id.R, true);
  const bool ok = c.lu_solve_transposed_warp(Dn, DL);
  for (int d = 0; d < n; ++d) ws[L.x + d] = Dn[DL.dl + c.i * n + d];
  c.transform_tangents(L.x);
  c.known_node_vjp(0, L.qp, L.r);
  c.known_node_vjp(1, L.qc, L.rt);
  if (writer && c.i == 0) {
    for (int d = 0; d < n; ++d) {
      double gt = 0.0;
      for (int s = 0; s < S; ++s) gt += Dn[DL.dl + s * n + d];
      A.gq_prev[c.gdof(d)] = ok ? -ws[L.r + d] : NAN;
      A.gq_cur[c.gdof(d)] = ok ? -ws[L.rt + d] : NAN;
      A.gtau[c.gdof(d)] = ok ? gt : NAN;
    }
    if (A.status) A.status[B.inst_off + b] = ok ? kConverged : kCholFail;
  }
}

// ------------------------------------------------------------------------
// The same adjoint over n_steps consecutive steps of a rollout in one launch
// (a checkpoint segment of a differentiable rollout): from the loss
// gradients a_prev, a_cur of the state after the last step, the steps are
// taken in reverse; step t's stages come from stages_traj[t] (written by the
// recomputing rollout), the state before it from the stages of step t - 1
// (the segment's start state for its first step). Per step:
//   g_bar = a_cur on stage S-1 (+ a_prev on stage S-2 for S >= 2),
//   Jr^T mu = g_bar, a_prev' = -(dr/dq_prev)^T mu,
//   a_cur' = -(dr/dq_cur)^T mu (+ a_prev for one stage, whose q_prev' = q_cur),
//   dL/dtau_t = sum_i mu_i.
// a_prev and a_cur live in the lane workspace's g and d slices.
// ------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(128) k_segment_backward(const __grid_constant__ LaunchArgs A) {
  const Bucket& B = A.bk[find_bucket(A)];
  const WarpId<S> id(B);
  const bool active = id.inst < B.count;
  if (!active) return;  // warp-uniform
  const int b = (int)id.inst;
  Ctx<S> c(B, A.K, b, id.lane_id, 0, A.dense_stages);
  const int n = c.n;
  const auto& L = c.L;
  const Lane& ws = c.ws;
  const bool writer = id.rep == 0;
  const int64_t D = A.D;
  double* Dn = B.dense + (int64_t)b * B.dense_stride;
  DenseLayout DL;
  DL.make(S * n);
  // stage j of step t (stage-packed), instance b
  auto stage_of = [&](int t, int j, int d) {
    return A.stages_traj[(int64_t)t * S * D + (int64_t)S * B.dof_off + ((int64_t)b * S + j) * n + d];
  };
  for (int d = 0; d < n; ++d) {
    ws[L.g + d] = A.g_bar[c.gdof(d)];     // a_prev (dL/dq_prev after the last step)
    ws[L.d + d] = A.a_cur_in[c.gdof(d)];  // a_cur
  }
  int worst = kConverged;
  for (int t = A.n_steps - 1; t >= 0; --t) {
    for (int d = 0; d < n; ++d) {
      double qp, qc;
      if (t == 0) {
        qp = A.q_prev0[c.gdof(d)];
        qc = A.q_cur0[c.gdof(d)];
      } else if (S == 1) {
        qp = t == 1 ? A.q_cur0[c.gdof(d)] : stage_of(t - 2, 0, d);
        qc = stage_of(t - 1, 0, d);
      } else {
        qp = stage_of(t - 1, S - 2, d);
        qc = stage_of(t - 1, S - 1, d);
      }
      ws[L.qp + d] = qp;
      ws[L.qc + d] = qc;
    }
    c.setup(true);
    for (int d = 0; d < n; ++d) ws[L.xt + d] = stage_of(t, c.i, d);
    if (writer)
      for (int d = 0; d < n; ++d) {
        double gb = c.i == S - 1 ? ws[L.d + d] : 0.0;
        if (S >= 2 && c.i == S - 2) gb += ws[L.g + d];
        Dn[DL.gb + c.i * n + d] = gb;
      }
    const double* tau = A.tau ? A.tau + (int64_t)t * D : nullptr;
    c.primal(tau);
    __syncwarp();
    c.build_jacobian_warp(Dn, DL, id.rep, id.R, true);
    const bool ok = c.lu_solve_transposed_warp(Dn, DL);
    __syncwarp();
    for (int d = 0; d < n; ++d) ws[L.x + d] = Dn[DL.dl + c.i * n + d];
    c.transform_tangents(L.x);
    c.known_node_vjp(0, L.qp, L.r);
    c.known_node_vjp(1, L.qc, L.rt);
    if (!ok) worst = status_worse(worst, kCholFail);
    for (int d = 0; d < n; ++d) {
      double gt = 0.0;
      for (int j = 0; j < S; ++j) gt += Dn[DL.dl + j * n + d];
      const double ap = ok ? -ws[L.r + d] : NAN;
      const double ac = ok ? -ws[L.rt + d] + (S == 1 ? ws[L.g + d] : 0.0) : NAN;
      ws[L.g + d] = ap;
      ws[L.d + d] = ac;
      if (writer && c.i == 0) A.gtau[(int64_t)t * D + c.gdof(d)] = ok ? gt : NAN;
    }
    __syncwarp();
  }
  if (writer && c.i == 0) {
    for (int d = 0; d < n; ++d) {
      A.gq_prev[c.gdof(d)] = ws[L.g + d];
      A.gq_cur[c.gdof(d)] = ws[L.d + d];
    }
    if (A.status) A.status[B.inst_off + b] = worst;
  }
}

// ------------------------------------------------------------------------
// World position of one body point per instance and its Jacobian dp/dq
// (column d: w_d x (p - o_d) for the joints on the root-to-link path), from
// the forward kinematics of Section 5. One lane per instance.
// ------------------------------------------------------------------------
#if PBAD_S == 1
__global__ void __launch_bounds__(128) k_link_points(const __grid_constant__ LaunchArgs A) {
  int bk = 0;
  while (bk + 1 < A.nb && (int)blockIdx.x >= A.bk[bk + 1].block_begin) ++bk;
  const Bucket& B = A.bk[bk];
  const LaneId<1> id(B);
  const bool active = id.real && id.inst < B.count;
  const int b = active ? (int)id.inst : 0;
  Ctx<1> c(B, A.K, b, id.lane_id, 0);
  const int n = c.n;
  const auto& L = c.L;
  const Lane& ws = c.ws;
  for (int d = 0; d < n; ++d) ws[L.xt + d] = A.q_cur0[c.gdof(d)];
  for (int l = 0; l < c.N; ++l) {
    const int p = B.parent[l], d0 = B.dof[l], nd = c.ndof(l);
    double Tp[12], T[12], Jr[9], q3[3], w[9];
    if (p >= 0) c.load12(L.T + 12 * p, Tp);
    for (int k = 0; k < nd; ++k) q3[k] = ws[L.xt + d0 + k];
    c.link_fk(l, p >= 0 ? Tp : nullptr, q3, T, Jr);
    c.store12(L.T + 12 * l, T);
    c.link_axes(l, T, Jr, w);
    for (int k = 0; k < 3 * nd; ++k) ws[L.axes + 9 * l + k] = w[k];
  }
  if (!active) return;
  const int64_t g = B.inst_off + b;
  const int lk = A.point_link[bk];
  double T[12];
  c.load12(L.T + 12 * lk, T);
  const double* pl = A.point_local + 3 * g;
  double pw[3];
  for (int r = 0; r < 3; ++r) pw[r] = fma(T[4 * r], pl[0], fma(T[4 * r + 1], pl[1], fma(T[4 * r + 2], pl[2], T[4 * r + 3])));
  for (int r = 0; r < 3; ++r) A.point_pos[3 * g + r] = pw[r];
  if (A.point_jac) {
    double* Jp = A.point_jac + 3 * (B.dof_off + (int64_t)b * n);
    for (int k = 0; k < 3 * n; ++k) Jp[k] = 0.0;
    for (int a = lk; a >= 0; a = B.parent[a]) {
      const int d0 = B.dof[a], nd = c.ndof(a);
      const double o[3] = {ws[L.T + 12 * a + 3], ws[L.T + 12 * a + 7], ws[L.T + 12 * a + 11]};
      const double rel[3] = {pw[0] - o[0], pw[1] - o[1], pw[2] - o[2]};
      for (int k = 0; k < nd; ++k) {
        const double w[3] = {ws[L.axes + 9 * a + 3 * k], ws[L.axes + 9 * a + 3 * k + 1],
                             ws[L.axes + 9 * a + 3 * k + 2]};
        double v[3];
        cross(w, rel, v);
        for (int r = 0; r < 3; ++r) Jp[r * n + d0 + k] = B.jtype[a] == kTranslation ? w[r] : v[r];
      }
    }
  }
}
#endif

// ------------------------------------------------------------------------
// FP64 FMA throughput probe (roofline denominator): dependent chains, 8
// independent chains per thread.
// ------------------------------------------------------------------------
#if PBAD_S == 1
__global__ void k_fp64_peak(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}
#endif

// ------------------------------------------------------------------------
// FP64 tensor-core (DMMA) throughput probe: mma.sync m8n8k4 with binary64
// operands and accumulators, 8 independent accumulator tiles per warp, so
// that the decision whether to assemble the Newton Gram matrix Jr^T Jr on
// the tensor cores rests on a measured rate. One mma = 8*8*4 FMA per warp.
// ------------------------------------------------------------------------
#if PBAD_S == 1
__global__ void k_dmma_peak(double* out, int iters, double a0, double b0) {
  const int lane = threadIdx.x & 31;
  double a = a0 + 1e-3 * lane, b = b0 - 1e-3 * lane;
  double c[8][2];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    c[k][0] = 1e-3 * k;
    c[k][1] = -1e-3 * k;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c[k][0]), "+d"(c[k][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += c[k][0] + c[k][1];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}
#endif

// Host-side launchers for the stage count this translation unit is built for
// (PBAD_S): the library compiles this file once per stage count.
#define PBAD_CAT2(a, b) a##b
#define PBAD_CAT(a, b) PBAD_CAT2(a, b)
cudaError_t PBAD_CAT(launch_eval_s, PBAD_S)(const LaunchArgs& A, int grid, cudaStream_t s) {
  k_eval<PBAD_S><<<grid, A.threads, 0, s>>>(A);
  return cudaGetLastError();
}
cudaError_t PBAD_CAT(launch_backward_s, PBAD_S)(const LaunchArgs& A, int grid, cudaStream_t s) {
  k_step_backward<PBAD_S><<<grid, A.threads, 0, s>>>(A);
  return cudaGetLastError();
}
cudaError_t PBAD_CAT(launch_segment_backward_s, PBAD_S)(const LaunchArgs& A, int grid, cudaStream_t s) {
  k_segment_backward<PBAD_S><<<grid, A.threads, 0, s>>>(A);
  return cudaGetLastError();
}
cudaError_t PBAD_CAT(launch_rollout_s, PBAD_S)(const LaunchArgs& A, int grid, cudaStream_t s) {
  int kinds = 0;  // bit per solver present
  for (int k = 0; k < A.nb; ++k) kinds |= 1 << A.bk[k].solver;
  const bool queue = A.bk[0].queue != nullptr;  // set for single-kind L-BFGS launches only
  const size_t smem = A.cta_smem;  // CTA-mode Newton and link-mapped buckets
  bool any_lp = false;
  for (int k = 0; k < A.nb; ++k) any_lp = any_lp || A.bk[k].lp;
  void (*kern)(const LaunchArgs) = nullptr;
  size_t dyn = 0;
  if (any_lp) {  // link-mapped buckets beside others: the mixed variant
    kern = k_rollout<PBAD_S, 2>;
    dyn = smem;
  } else if (kinds == 1) {
    kern = queue ? k_rollout<PBAD_S, 4> : k_rollout<PBAD_S, 0>;
  } else if (kinds == 2) {
    kern = k_rollout<PBAD_S, 1>;
    dyn = smem;
  } else if (kinds == 4) {
    kern = queue ? k_rollout<PBAD_S, 5> : k_rollout<PBAD_S, 3>;
  } else {
    kern = k_rollout<PBAD_S, 2>;
    dyn = smem;
  }
  if (dyn > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, A.threads, dyn, s>>>(A);
  return cudaGetLastError();
}
// Link-parallel launches (every bucket a serial chain with S N <= 32): the
// dynamic shared memory is smem bytes per block.
cudaError_t PBAD_CAT(launch_eval_lp_s, PBAD_S)(const LaunchArgs& A, int grid, size_t smem,
                                              cudaStream_t s) {
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_eval_lp<PBAD_S>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_eval_lp<PBAD_S><<<grid, A.threads, smem, s>>>(A);
  return cudaGetLastError();
}
cudaError_t PBAD_CAT(launch_rollout_lp_s, PBAD_S)(const LaunchArgs& A, int grid, size_t smem,
                                                 cudaStream_t s) {
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_rollout_lp<PBAD_S>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_rollout_lp<PBAD_S><<<grid, A.threads, smem, s>>>(A);
  return cudaGetLastError();
}
// Blocks of the queue variant of the rollout kernel for these buckets (all
// binary64 or all binary32-direction L-BFGS) that one SM keeps resident at
// `threads` threads per block (0 on error or for other bucket mixes).
int PBAD_CAT(rollout_blocks_per_sm_s, PBAD_S)(const LaunchArgs& A, int threads) {
  int kinds = 0;
  for (int k = 0; k < A.nb; ++k) kinds |= 1 << A.bk[k].solver;
  int n = 0;
  cudaError_t e;
  if (kinds == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rollout<PBAD_S, 4>, threads, 0);
  else if (kinds == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rollout<PBAD_S, 5>, threads, 0);
  else return 0;
  return e == cudaSuccess ? n : 0;
}
#if PBAD_S == 1
cudaError_t launch_link_points(const LaunchArgs& A, int grid, cudaStream_t s) {
  k_link_points<<<grid, A.threads, 0, s>>>(A);
  return cudaGetLastError();
}
cudaError_t launch_fp64_peak(double* out, int blocks, int threads, int iters) {
  k_fp64_peak<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
  return cudaGetLastError();
}
cudaError_t launch_dmma_peak(double* out, int blocks, int threads, int iters) {
  k_dmma_peak<<<blocks, threads>>>(out, iters, 0.5, 1e-9);
  return cudaGetLastError();
}
#endif

}  // namespace pbad
