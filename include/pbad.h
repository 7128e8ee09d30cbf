/*
 * pbad.h - C ABI of the B300 position-based articulated dynamics library.
 *
 * The method is Pan & Manocha, "Time Integrating Articulated Body Dynamics
 * Using Position-Based Collocation Methods" (arXiv 1709.04145): every time
 * step solves for the S = K-1 unknown stage configurations of a K-th order
 * position-based collocation (Section 4.1) by minimising
 *   S == 1: the energy of Eq. EQ
 *             E(q) = sum_l tr(D_l M_l D_l^T)/(2 dt^2) - g.(T_l [mc; m]) - tau.q,
 *             D_l = T_l(q) - 2 T_l(q_cur) + T_l(q_prev),
 *   S >= 2: the squared stage residuals of Eq. EQHOC, E = sum_i |r_i|^2, with
 *             r_i = int dP(q_i)/dq_i^T [rho Pddot(t_i) - f] dp - tau  (Eq. HOC)
 * using L-BFGS or Newton (Levenberg-Marquardt), Section 5.
 *
 * Conventions shared by every entry point:
 *   - Links l = 0..N-1 are topologically sorted: parent[l] < l, -1 = world.
 *     The link frame origin is at its joint; T_l = T_parent * X_l * Rot(q_l)
 *     with X_l the 3x4 rest transform (row-major) and Rot a hinge rotation
 *     about a unit axis of the joint frame (1 DOF) or the exponential map of
 *     a 3-vector (ball, 3 DOF). Generalised torques tau are conjugate to q.
 *   - A model is one topology with `count` instances; each instance has its
 *     own mass moments and rest transforms. A batch is an ordered list of
 *     models (buckets of an uneven batch).
 *   - DOF-packed arrays (q, tau, ...) hold, model after model, `count` rows
 *     of that model's n DOFs: row-major [instance][dof] within each model
 *     block. Their total length is D = sum_m count_m * n_m.
 *   - Stage-packed arrays hold, model after model, [instance][stage][dof]:
 *     total length S * D.
 *   - Per-instance arrays (E, status, iters) hold one entry per instance in
 *     batch order.
 *   - Collocation nodes (units of dt, relative to t_k) are
 *     [k-1+alpha_{S-1}, k, k+alpha_1, ..., k+alpha_S], alpha_S = 1 and
 *     alpha_1..alpha_{S-1} the roots of L_{S-1}(2 alpha - 1). A step maps the
 *     state (q_prev at node k-1+alpha_{S-1}, q_cur at node k) to
 *     (stage S-1 (q_cur when S == 1), stage S).
 *   - All array arguments of the compute entry points are DEVICE pointers on
 *     the batch's device, owned by the caller, and must not alias outputs.
 *     Model set-up arrays are HOST pointers (copied). `stream` is a
 *     cudaStream_t (NULL = legacy default stream). The compute entry points
 *     only enqueue work: they allocate nothing, never synchronise the host and
 *     may be captured in a CUDA graph.
 *   - Every function returns PBAD_OK (0) or a negative PBAD_ERR_* code and
 *     then pbad_last_error() describes the failure (thread-local). Nothing
 *     aborts or throws across the ABI. Per-instance solver outcomes are
 *     reported through `status` (PBAD_CONVERGED ...), never as return codes.
 */
#ifndef PBAD_H
#define PBAD_H

#include <stdint.h>

#if defined(__GNUC__)
#define PBAD_API __attribute__((visibility("default")))
#else
#define PBAD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define PBAD_OK 0
#define PBAD_ERR_ARG (-1)         /* invalid argument (null, size, range) */
#define PBAD_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define PBAD_ERR_ALLOC (-3)       /* device or host allocation failed */
#define PBAD_ERR_UNSUPPORTED (-4) /* valid request outside what is built */

#define PBAD_HINGE 0
#define PBAD_BALL 1
/* Three prismatic coordinates along the joint frame's axes, J = [I | q]. A
 * massless link on a translation joint carrying a body on a ball joint at
 * the same origin is a free 6-DOF root (Section 6.2's swimmer and spider). */
#define PBAD_TRANSLATION 2

#define PBAD_LBFGS 0
#define PBAD_NEWTON 1
/* L-BFGS whose two-loop recursion runs in binary32 on binary32 curvature
 * pairs (H0 = gamma P still applied in binary64); the line search, the
 * convergence test and every evaluation of E, r and dE/dq stay binary64.
 * The solution of a converged step is the same fixed point of the step
 * equations; the iterates on the way differ from PBAD_LBFGS at the binary32
 * rounding level. A mixed-precision option, not the default. */
#define PBAD_LBFGS_F32 2

/* Per-step solver status. A rollout's per-instance `status` is the worst over
 * its steps in the order CONVERGED < STALLED < MAX_ITER < LS_FAIL <
 * CHOL_FAIL < NONFINITE. */
#define PBAD_CONVERGED 0  /* |r|_2 < tol */
#define PBAD_MAX_ITER 1   /* iteration cap reached */
#define PBAD_LS_FAIL 2    /* line search / damping could not decrease E */
#define PBAD_CHOL_FAIL 3  /* Newton system not factorable for any damping */
#define PBAD_NONFINITE 4  /* NaN or Inf in E, r or the gradient */
/* The line search / damping could not decrease E while |r|_2 was at most
 * 1e3 times the binary64 rounding floor of r: solved as far as binary64
 * resolves the step equations (the paper is silent on floors). The floor of
 * an instance, for S stages and step dt, is
 *   eps (What sum_l I_l + |g| sum_l (|m c_l| + m_l R_l)),
 * eps = 2^-52, What = max_i sum_j |W_ij + 2 c V_ij| / dt^2 over the S+2
 * nodes (acceleration and drag weights), R_l = sum of |t(X_a)| over the
 * joints a on the root-to-l path (rest translations), I_l = (sqrt(tr
 * Sigma_l) + sqrt(m_l) R_l)^2 from link l's mass moment. */
#define PBAD_STALLED 5

#define PBAD_BATCH_NEWTON 1 /* batch flag: reserve the dense Newton/adjoint workspace */

#define PBAD_MAX_STAGES 5
#define PBAD_MAX_HISTORY 16
#define PBAD_MAX_MODELS 8

typedef struct pbad_model pbad_model;
typedef struct pbad_batch pbad_batch;

/* Library version (major*10000 + minor*100 + patch). */
PBAD_API int pbad_version(void);

/* Message of the last failed call on this thread ("" if none). */
PBAD_API const char* pbad_last_error(void);

/* Collocation table of Section 4.1 for S stages (1..PBAD_MAX_STAGES):
 * nodes[S+2] as documented above; W[S][S+2] row-major, W[i][j] = l_j''(node
 * of stage i) of the Lagrange basis over all S+2 nodes, in units of 1/dt^2.
 * Host pointers. */
PBAD_API int pbad_colloc(int32_t stages, double* nodes, double* W);

/* Creates a model (one topology, `count` instances) on CUDA device `device`.
 *   parent[n_links], joint_type[n_links] (PBAD_HINGE/PBAD_BALL/
 *   PBAD_TRANSLATION), axis[n_links][3] (hinge axes in the joint frame, unit
 *   length; ignored for the other types), mass_moment[count][n_links][10] = Sxx Sxy Sxz Syy Syz Szz mcx mcy
 *   mcz m of int rho [p;1][p;1]^T dp in the link frame (Eq. ATOM),
 *   rest[count][n_links][12] (3x4 row-major), gravity[3].
 * All host pointers, copied. Errors: PBAD_ERR_ARG for a malformed tree,
 * unknown joint type, non-positive sizes or n_links > 4096. */
PBAD_API int pbad_model_create(int32_t n_links, const int32_t* parent, const int32_t* joint_type,
                      const double* axis, int64_t count, const double* mass_moment,
                      const double* rest, const double* gravity, int32_t device,
                      pbad_model** out);
PBAD_API int pbad_model_destroy(pbad_model* model);
PBAD_API int pbad_model_info(const pbad_model* model, int32_t* n_links, int32_t* n_dof, int64_t* count);

/* Drag potential of Section 6.2 (the swimmer's fluid drag) on every link of
 * the model: Q_drag = D |(P(q_{k+1}) - P(q_k))/dt|^2 integrated over the body,
 * with c = D / rho (per unit mass, >= 0; 0 = none). For one stage it adds
 * c/dt^2 tr((T_{k+1} - T_k) M (T_{k+1} - T_k)^T) to Eq. EQ (Appendix A); its
 * gradient, the force density -2 c rho v / dt, enters the residual. For
 * S >= 2 stages the same force law enters every stage residual of Eq. HOC with
 * v the velocity of the collocation polynomial at the stage node. Set it
 * before creating the batches that use the model (a batch reserves the
 * one-stage drag storage at creation; a one-stage call on a batch created
 * before the drag was set returns PBAD_ERR_ARG). Errors: PBAD_ERR_ARG for a
 * NULL model or a negative or non-finite c. */
PBAD_API int pbad_model_set_drag(pbad_model* model, double c);

/* Penalty frictional contact of Eq. FRI (Section 6.2, the spider) between
 * body points of the model and the ground: obstacle = the half-space
 * z < z0 (world), penetration depth d(P) = max(0, z0 - P_z), tangential
 * projection = the xy components, the body integral replaced by a sum over
 * n_points contact points (link[k], point[k][3] in that link's frame, the
 * same for every instance):
 *   Q = sum_k d1 d(P_k)^2 + d2 d(P_k)^2 |Pi (P_k(q_{k+1}) - P_k(q_k))/dt|^2,
 * added to Eq. EQ. Defined for one stage only: a call with stages >= 2 on a
 * model with contact points returns PBAD_ERR_UNSUPPORTED. n_points = 0
 * removes the contact. Host pointers, copied to the device. Set it before
 * creating the batches that use the model (like the drag). Errors:
 * PBAD_ERR_ARG (NULL model, n_points < 0 or > 65536, link out of range,
 * negative or non-finite d1/d2), PBAD_ERR_ALLOC. */
PBAD_API int pbad_model_set_contact(pbad_model* model, int32_t n_points, const int32_t* link,
                                    const double* point, double z0, double d1, double d2);

/* Creates a batch over 1..PBAD_MAX_MODELS models (same device) and allocates
 * the solver workspace for up to max_stages stages and L-BFGS history
 * max_history; flags = PBAD_BATCH_NEWTON also reserves the dense
 * (S n)^2 Newton storage per lane (needed by the Newton solver). The models
 * must outlive the batch. */
PBAD_API int pbad_batch_create(int32_t n_models, pbad_model* const* models, int32_t max_stages,
                      int32_t max_history, int32_t flags, pbad_batch** out);
PBAD_API int pbad_batch_destroy(pbad_batch* batch);
/* n_instances = sum count_m; n_dof_total = D; workspace_bytes = device bytes
 * the batch owns. Any output pointer may be NULL. */
PBAD_API int pbad_batch_info(const pbad_batch* batch, int64_t* n_instances, int64_t* n_dof_total,
                    int64_t* workspace_bytes);

/* Threads per block of the solver kernels (32, 64, 96 or 128; default 32):
 * one of the instance-to-warp mapping knobs the autotuner sets. */
PBAD_API int pbad_batch_set_threads(pbad_batch* batch, int32_t threads);

/* Instance-to-lane mappings of the evaluation and L-BFGS kernels (Section
 * 5.2, Fig. GPU: a group of GPU lanes per trajectory).
 *   PBAD_MAP_STAGE (default): one lane per collocation stage, S lanes per
 *     instance, floor(32/S) instances per warp; each lane walks the link tree
 *     in order (Algorithm DERIV, tree form). Every topology and solver.
 *   PBAD_MAP_LINK: one lane per stage and link, S N lanes per instance,
 *     floor(32/(S N)) instances per warp; forward kinematics and the subtree
 *     sums of Algorithm DERIV become shuffle scans across the links' lanes
 *     (the work-efficient counterpart of Algorithm DERIVP), and the solver
 *     state sits in shared memory. For buckets that are serial chains
 *     (parent[l] = l - 1) with S N <= 32, solved by PBAD_LBFGS (one stage:
 *     without drag or contact).
 * Results agree with the stage mapping to rounding (sums taken in another
 * order). pbad_step_backward and Newton always use one warp per instance.
 * With PBAD_MAP_LINK set, pbad_eval_objective_grad, pbad_step and
 * pbad_rollout return PBAD_ERR_UNSUPPORTED (nothing launched) when a
 * bucket does not qualify. Errors: PBAD_ERR_ARG for a null batch or an
 * unknown mapping. */
#define PBAD_MAP_STAGE 0
#define PBAD_MAP_LINK 1
PBAD_API int pbad_batch_set_mapping(pbad_batch* batch, int32_t mapping);

/* Newton (LM) buckets whose S n (stages x DOFs) is at least min_sn (and at
 * most 4096) run one CTA of four warps per instance: the warps split the
 * Jacobian columns and the CTA forms the Gram matrix and the Cholesky
 * factor together; smaller systems run one warp per instance. Default 128;
 * min_sn = 4097 keeps every bucket on one warp per instance. The batch's
 * workspace grows (cudaFree of the old one waits for the device) where a
 * bucket needs a CTA's lanes it was not created with. Errors: PBAD_ERR_ARG
 * (null batch, min_sn outside 1..4097), PBAD_ERR_ALLOC, PBAD_ERR_CUDA. */
PBAD_API int pbad_batch_set_newton_cta_min(pbad_batch* batch, int32_t min_sn);

/* One-warp Newton (LM) buckets with S >= 2 (Eq. EQHOC): on = 1 (the default)
 * spreads the residual pass at each trial point of the damping loop over the
 * warp's 32 / S replicas of the stage group (each replica takes every
 * (32 / S)-th link's joint rotation, axes, stage coupling, mass product,
 * seed and wrench; the forward kinematics and the subtree sums stay
 * sequential, in the order of the full pass); on = 0 has every replica
 * evaluate the whole pass. Both give the same bits: the setting changes
 * only the time of a trial, which matters for instances whose damping loop
 * rejects many trials (Section 5: lambda is raised until E decreases).
 * Errors: PBAD_ERR_ARG (null batch, on not 0 or 1). */
PBAD_API int pbad_batch_set_newton_split(pbad_batch* batch, int32_t on);

/* The damped Gauss-Newton system of one LM iteration (Section 5, LM with
 * J^T J), batched, on its own: for each instance b of count,
 *   H_b = J_b^T J_b,  L_b L_b^T = H_b + lambda I (Cholesky),
 *   dl_b = -(H_b + lambda I)^-1 g_b.
 * One CTA per instance with the routines of the CTA-mode Newton rollout
 * (tiled syrk, left-looking Cholesky, triangular solves).
 *   J:      device, [count][n][n], each instance column-major (column c of
 *           J_b at J + b n^2 + c n); read only.
 *   g:      device, [count][n] (for LM, J^T r); read only.
 *   H:      device, [count][n][n] out, row-major and symmetric.
 *   L:      device, [count][n][n] out, the factor column-major (L[r][c] at
 *           L + b n^2 + c n + r, r >= c; the upper part is left as is).
 *   dl:     device, [count][n] out.
 *   status: device, [count] out: PBAD_CONVERGED, or PBAD_CHOL_FAIL where a
 *           pivot was not positive (dl and the rest of L then undefined).
 * All buffers are caller-owned; nothing is allocated. Asynchronous on
 * `stream` (NULL: the default stream). 1 <= n <= 4096 and count < 2^31,
 * else PBAD_ERR_ARG (count 0 launches nothing); PBAD_ERR_ARG also for a
 * null array or a non-finite lambda; PBAD_ERR_CUDA if the launch fails. */
PBAD_API int pbad_damped_gram_solve(int64_t count, int32_t n, const double* J, const double* g,
                                    double lambda, double* H, double* L, double* dl,
                                    int32_t* status, void* stream);

/* Per-bucket mapping of pbad_step and pbad_rollout: mapping[n_models] (host)
 * of PBAD_MAP_STAGE, PBAD_MAP_LINK or -1 (the batch's mapping); NULL clears
 * it. A launch whose buckets mix the mappings stays one persistent launch:
 * each block runs its bucket's mapping (link-mapped buckets must qualify as
 * for pbad_batch_set_mapping, else PBAD_ERR_UNSUPPORTED). The instance queue
 * is not used in such launches. pbad_eval_objective_grad follows the
 * batch's mapping. Errors: PBAD_ERR_ARG for a null batch or an unknown
 * mapping value. */
PBAD_API int pbad_batch_set_bucket_mapping(pbad_batch* batch, const int32_t* mapping);

/* Arithmetic of the residual pass of pbad_eval_objective_grad (a
 * mixed-precision experiment; the paper states no precision):
 *   PBAD_PRECISION_F64 (default): binary64 throughout.
 *   PBAD_PRECISION_DF64: the joint rotations in binary64, everything after
 *     them (forward kinematics, seeds of Eq. HOC, wrenches, subtree sums,
 *     contraction: E and r) in double-float arithmetic, a value being the
 *     unevaluated sum of two binary32 numbers (about 48 significant bits),
 *     on the binary32 pipes; the gradient's tangent pass stays binary64.
 *     Needs PBAD_MAP_LINK (else PBAD_ERR_UNSUPPORTED). The residual's
 *     rounding floor is about 2^5 times the binary64 one.
 * Rollouts and steps always evaluate in binary64. Errors: PBAD_ERR_ARG for
 * a null batch or an unknown precision. */
#define PBAD_PRECISION_F64 0
#define PBAD_PRECISION_DF64 1
PBAD_API int pbad_batch_set_precision(pbad_batch* batch, int32_t precision);

/* Instance queue of pbad_step / pbad_rollout (Section 5.2's dynamic
 * assignment of work to the GPU's cores): when the L-BFGS buckets of a
 * launch would need more blocks than max_blocks, they get max_blocks blocks
 * in total (each bucket a share, at least one) and a group of lanes that has
 * finished all steps of its instance takes the bucket's next unstarted
 * instance from a device counter, so no lane idles while instances are left.
 * max_blocks = 0 uses the number of blocks of the rollout kernel that the
 * GPU keeps resident; max_blocks < 0 (the default) turns the queue off: one
 * group per instance, the hardware block scheduler starts blocks as others
 * finish. The queue serves launches whose buckets all use one L-BFGS solver
 * (PBAD_LBFGS or PBAD_LBFGS_F32); other launches ignore it. Results per
 * instance do not depend on it. Errors: PBAD_ERR_ARG for a null batch. */
PBAD_API int pbad_batch_set_queue(pbad_batch* batch, int32_t max_blocks);

/* Objective and gradient of one step at given stage configurations
 * (Eq. EQ / Eq. EQHOC; gradient by Algorithm DERIV in world coordinates and,
 * for S >= 2, its tangent sweep: grad = 2 Jr^T r in O(N)).
 *   q_star[S*D] stage-packed, q_prev[D], q_cur[D], tau[D] (NULL = zero),
 *   E[instances], grad[S*D], resid[S*D] (stage residuals r_i; NULL = skip).
 */
PBAD_API int pbad_eval_objective_grad(pbad_batch* batch, const double* q_star, const double* q_prev,
                             const double* q_cur, const double* tau, double dt, int32_t stages,
                             double* E, double* grad, double* resid, void* stream);

/* One time step for every instance: q_prev'/q_cur' [D] (either may be NULL),
 * q_stages_out[S*D] (NULL = skip), status/iters [instances] (NULL = skip).
 * solvers[n_models] (host, NULL = all PBAD_LBFGS): PBAD_LBFGS, PBAD_NEWTON or
 * PBAD_LBFGS_F32 per model; history <= max_history;
 * tol is the bound on |r|_2 (r = dE/dq for S == 1); max_iter >= 0. */
PBAD_API int pbad_step(pbad_batch* batch, const double* q_prev, const double* q_cur, const double* tau,
              double dt, int32_t stages, const int32_t* solvers, int32_t history, double tol,
              int32_t max_iter, double* q_prev_out, double* q_cur_out, double* q_stages_out,
              int32_t* status, int32_t* iters, void* stream);

/* n_steps steps in one persistent launch. tau_seq[n_steps][D] (NULL = zero),
 * traj_prev/traj_cur [n_steps][D] the state after each step (NULL = skip),
 * q_prev_out/q_cur_out [D] the final state (NULL = skip), status = worst
 * status over the steps, iters = total accepted iterations, evals = total
 * objective evaluations (E and r; line-search trials included), grad_evals =
 * the evaluations that also formed dE/dq (L-BFGS: a step's first point,
 * accepted trials and trials the approximate-Wolfe test had to read; a trial
 * rejected on E alone needs none) or Jr (Newton); each of
 * status/iters/evals/grad_evals [instances] may be NULL. step_status
 * [n_steps][instances] receives every step's own status and step_rnorm
 * [n_steps][instances] the |r|_2 of the point the step ended at (the
 * accepted point it returns); either may be NULL. stages_traj
 * [n_steps][S*D] (NULL = skip) receives every step's stages, stage-packed
 * (what pbad_rollout_backward reads). */
PBAD_API int pbad_rollout(pbad_batch* batch, const double* q_prev0, const double* q_cur0,
                 const double* tau_seq, int32_t n_steps, double dt, int32_t stages,
                 const int32_t* solvers, int32_t history, double tol, int32_t max_iter,
                 double* traj_prev, double* traj_cur, double* q_prev_out, double* q_cur_out,
                 int32_t* status, int32_t* iters, int32_t* evals, int32_t* grad_evals,
                 int32_t* step_status, double* step_rnorm, double* stages_traj, void* stream);

/* Implicit-function-theorem adjoint of one converged step (no counterpart
 * in the paper, which has no adjoint; it differentiates the stage equations
 * Eq. HOC, r(q_*; q_prev, q_cur, tau) = 0): given g_bar = dL/dq_*
 * [S*D] at the converged stages q_star [S*D], solves Jr^T mu = g_bar and
 * returns gq_prev = -(dr/dq_prev)^T mu, gq_cur = -(dr/dq_cur)^T mu and
 * gtau = sum_i mu_i [D each]. Jr is exact (for one stage: the Hessian of
 * Eq. EQ). status [instances] (NULL = skip): PBAD_CONVERGED, or
 * PBAD_CHOL_FAIL when Jr is singular (outputs NaN). Needs a batch created
 * with PBAD_BATCH_NEWTON. */
PBAD_API int pbad_step_backward(pbad_batch* batch, const double* q_prev, const double* q_cur,
                                const double* tau, const double* q_star, const double* g_bar,
                                double dt, int32_t stages, double* gq_prev, double* gq_cur,
                                double* gtau, int32_t* status, void* stream);

/* The implicit-function-theorem adjoint of n_steps consecutive steps in one
 * launch, in reverse (a checkpoint segment of a differentiable rollout; no
 * counterpart in the paper). stages_traj [n_steps][S*D] holds every step's
 * converged stages as pbad_rollout writes them from the segment's start
 * state (q_prev0, q_cur0 [D]); tau_seq [n_steps][D] (NULL = zero). From the
 * loss gradients a_prev, a_cur [D] of the state after the last step, each
 * step applies the adjoint of pbad_step_backward with g_bar = a_cur on stage
 * S-1 (+ a_prev on stage S-2 for S >= 2) and passes on a_prev' = -(dr/
 * dq_prev)^T mu, a_cur' = -(dr/dq_cur)^T mu (+ a_prev for one stage, whose
 * next q_prev is q_cur); g_tau [n_steps][D] receives dL/dtau of every step,
 * a_prev_out / a_cur_out [D] the gradients of the segment's start state.
 * status [instances] (NULL = skip): PBAD_CONVERGED, or PBAD_CHOL_FAIL when
 * some step's Jr is singular (that instance's outputs are NaN from there
 * on). The steps must have converged for the adjoint to hold (the caller's
 * check). Needs a batch created with PBAD_BATCH_NEWTON. Errors: PBAD_ERR_ARG
 * for null arrays, n_steps < 1, stages or dt out of range. */
PBAD_API int pbad_rollout_backward(pbad_batch* batch, const double* q_prev0, const double* q_cur0,
                                   const double* tau_seq, const double* stages_traj,
                                   int32_t n_steps, double dt, int32_t stages, const double* a_prev,
                                   const double* a_cur, double* a_prev_out, double* a_cur_out,
                                   double* g_tau, int32_t* status, void* stream);

/* World position of one body point per instance and its Jacobian:
 * link[n_models] (host) is the link carrying the point in each model,
 * point_local[instances][3] the point in that link's frame, q[D];
 * pos[instances][3]; jac (NULL = skip) holds, model after model,
 * [count][3][n] = dp/dq. */
PBAD_API int pbad_link_points(pbad_batch* batch, const double* q, const int32_t* link,
                              const double* point_local, double* pos, double* jac, void* stream);

/* Bytes of the fixed device scratch used by pbad_eval_objective_grad_static. */
#define PBAD_STATIC_SCRATCH_BYTES (8 * 1024 * 1024)

/* The same evaluation as pbad_eval_objective_grad for the instances of one
 * model, without a batch: its scratch is a fixed array of
 * PBAD_STATIC_SCRATCH_BYTES inside this library (every GPU that loads the
 * library holds it until the process exits), so the call allocates nothing.
 * The paper has no counterpart; this is for callers that cannot call
 * cudaMalloc when they evaluate - a host application whose device memory is
 * wholly owned by its own allocator, or a latency-bound control loop that
 * cannot afford an allocation's implicit synchronisation.
 *   Arrays as for pbad_eval_objective_grad with D = count * n of the model.
 *   Every call looks up the scratch's device address in the current
 *   context (the model's device is made current for the call), so the
 *   address stays right after cudaDeviceReset or under another context. The
 *   first call in a context also loads the library's device code there;
 *   make that first call before any stream capture.
 *   Every call shares the one scratch array and it keeps the last call's
 *   contents (each evaluation writes every scratch word before reading it,
 *   so nothing needs clearing); calls whose kernels overlap on the GPU race
 *   on it, so serialise them (one stream, or events).
 * Errors: PBAD_ERR_ARG when the model needs more scratch than
 * PBAD_STATIC_SCRATCH_BYTES (the message gives both sizes), or for the
 * argument errors of pbad_eval_objective_grad (null arrays, stages outside
 * 1..PBAD_MAX_STAGES, dt <= 0); PBAD_ERR_UNSUPPORTED for a model with
 * penalty contact points (Eq. FRI) and stages != 1; PBAD_ERR_CUDA when
 * selecting the model's device, the scratch address lookup or the launch
 * fails. */
PBAD_API int pbad_eval_objective_grad_static(const pbad_model* model, const double* q_star,
                                             const double* q_prev, const double* q_cur,
                                             const double* tau, double dt, int32_t stages,
                                             double* E, double* grad, double* resid, void* stream);

/* Measures the device's FP64 FMA throughput (GFLOP/s, FMA = 2 flops) with
 * the library's own probe kernel; synchronises the device. */
PBAD_API int pbad_fp64_peak(int32_t device, double* gflops);

/* Measures the device's FP64 tensor-core throughput (GFLOP/s) with the
 * library's own probe: warp-wide mma.sync m8n8k4 with binary64 operands,
 * eight independent accumulator tiles per warp. It decides whether dense
 * FP64 products (the Gram matrix Jr^T Jr of the Newton solver, Section 5)
 * would gain from the tensor cores; synchronises the device. */
PBAD_API int pbad_fp64_mma_peak(int32_t device, double* gflops);

#ifdef __cplusplus
}
#endif

#endif /* PBAD_H */
