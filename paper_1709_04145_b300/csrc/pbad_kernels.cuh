// The hot path of position-based articulated dynamics (Pan & Manocha):
//   - per-step setup (Section 4.1): known-node combination C_i and the
//     L-BFGS initial inverse Hessian from the joint-space mass matrix;
//   - objective/residual pass (Eq. EQ for one stage, Eq. HOC/EQHOC for
//     several): forward kinematics, per-link seeds, world wrench suffix sums
//     and joint contraction (Algorithm DERIV, tree form, world frame);
//   - tangent pass: d/de of the residual pass along r, giving
//     grad E = 2 Jr^T r for Eq. EQHOC in O(N) (Table 1's second-derivative
//     terms without forming any Hessian block);
//   - a persistent L-BFGS rollout (Section 5: one optimisation per step,
//     iteration-level scheduling of Fig. GPU inside each warp).
#pragma once
#include "pbad_launch.cuh"

namespace pbad {

// ------------------------------------------------------------------------
// per-lane context
// ------------------------------------------------------------------------
// The context is held by value: the hot passes below run on a private copy
// (see primal / tangent_pass / setup / precond), so that its fields live in
// registers instead of being reloaded from the caller's frame after every
// workspace store (a generic store could alias it).
template <int S>
struct Ctx {
  Bucket B;           // copy of the bucket descriptor
  const Colloc& K;
  Group<S> grp;
  WsLayout L;
  Lane ws;
  int b;              // instance within the bucket (always a valid index)
  int i;              // own stage
  int N, n;
  // seed weights of the own stage: acceleration plus the drag force,
  // W + 2 c V (units 1/dt^2); the preconditioner keeps the drag-free block
  double wk[2];       // known nodes: K.Wk[i][*] + 2c K.Vk[i][*]
  double wu_row[S];   // unknown stages: K.Wu[i][*] + 2c K.Vu[i][*]
  double wu_col[S];   // K.Wu[*][i] + 2c K.Vu[*][i]
  double ps_row[S];   // K.Ps[i][*]

  __device__ Ctx(const Bucket& B_, const Colloc& K_, int b_, int64_t lane_id, int m, int Sd = 0)
      : B(B_), K(K_), b(b_) {
    N = B.N;
    n = B.n;
    L.make(N, n, m, Sd, B.tk, B.n_contact);
    ws.p = B.ws + ((lane_id >> 5) * B.ws_lane) * Lane::kStride + (lane_id & 31);
    i = grp.stage;
    const double c2 = 2.0 * B.drag;
    wk[0] = fma(c2, K.Vk[i][0], K.Wk[i][0]);
    wk[1] = fma(c2, K.Vk[i][1], K.Wk[i][1]);
#pragma unroll
    for (int j = 0; j < S; ++j) {
      wu_row[j] = fma(c2, K.Vu[i][j], K.Wu[i][j]);
      wu_col[j] = fma(c2, K.Vu[j][i], K.Wu[j][i]);
      ps_row[j] = K.Ps[i][j];
    }
  }

  __device__ __forceinline__ double rest(int l, int k) const {
    return B.rest[((int64_t)l * 12 + k) * B.count + b];
  }
  __device__ __forceinline__ MassMoment mass(int l) const {
    MassMoment M;
#pragma unroll
    for (int k = 0; k < 10; ++k) M.s[k] = B.mm[((int64_t)l * 10 + k) * B.count + b];
    return M;
  }
  __device__ __forceinline__ int ndof(int l) const { return B.jtype[l] == 0 ? 1 : 3; }
  __device__ __forceinline__ int64_t gdof(int d) const { return B.dof_off + (int64_t)b * n + d; }
  __device__ __forceinline__ int64_t gstage(int d) const {
    return (int64_t)S * B.dof_off + ((int64_t)b * S + i) * n + d;
  }

  __device__ __forceinline__ void load12(int off, double* v) const {
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = ws[off + k];
  }
  __device__ __forceinline__ void store12(int off, const double* v) const {
#pragma unroll
    for (int k = 0; k < 12; ++k) ws[off + k] = v[k];
  }

  // T_l = T_parent * X_l * J(q_l), J = [Rot(q_l) | 0] or, for a translation
  // joint, [I | q_l]. Ball joints also return Jr(q_l) (translation: I).
  __device__ __forceinline__ void link_fk(int l, const double* Tp, const double* ql, double* T,
                                          double* Jr, ExpCoef* ec = nullptr) const {
    double R[9];
    const double u[3] = {B.axis[3 * l], B.axis[3 * l + 1], B.axis[3 * l + 2]};
    joint_rotation(B.jtype[l], u, ql, R, Jr, ec);
    link_fk_rot(l, Tp, ql, R, T);
  }
  // The same with the joint rotation R given.
  __device__ __forceinline__ void link_fk_rot(int l, const double* Tp, const double* ql,
                                              const double* R, double* T) const {
    double XJ[12];
    const int jt = B.jtype[l];
    if (B.rest_eye[l]) {
      // identity rest rotation: X_l J = [Rot | t_X] (translation: [I | t_X + q])
#pragma unroll
      for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int c = 0; c < 3; ++c) XJ[4 * r + c] = R[3 * r + c];
        XJ[4 * r + 3] = rest(l, 4 * r + 3);
      }
      if (jt == kTranslation) {  // uniform across the warp (same link on every lane)
#pragma unroll
        for (int r = 0; r < 3; ++r) XJ[4 * r + 3] += ql[r];
      }
    } else {
      double X[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) X[k] = rest(l, k);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          XJ[4 * r + c] = fma(X[4 * r], R[c], fma(X[4 * r + 1], R[3 + c], X[4 * r + 2] * R[6 + c]));
        XJ[4 * r + 3] = X[4 * r + 3];
      }
      if (jt == kTranslation) {
#pragma unroll
        for (int r = 0; r < 3; ++r)
          XJ[4 * r + 3] = fma(X[4 * r], ql[0], fma(X[4 * r + 1], ql[1], fma(X[4 * r + 2], ql[2], X[4 * r + 3])));
      }
    }
    if (Tp) compose(Tp, XJ, T);
    else {
#pragma unroll
      for (int k = 0; k < 12; ++k) T[k] = XJ[k];
    }
  }

  // World axes of the joint of link l: hinge w = R u; ball w_k = R Jr e_k.
  __device__ __forceinline__ void link_axes(int l, const double* T, const double* Jr, double* w) const {
    if (B.jtype[l] == 0) {
      const double u[3] = {B.axis[3 * l], B.axis[3 * l + 1], B.axis[3 * l + 2]};
#pragma unroll
      for (int r = 0; r < 3; ++r) w[r] = fma(T[4 * r], u[0], fma(T[4 * r + 1], u[1], T[4 * r + 2] * u[2]));
    } else {
      // column k of R Jr stored as w[3k..3k+2]
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int r = 0; r < 3; ++r)
          w[3 * k + r] = fma(T[4 * r], Jr[k], fma(T[4 * r + 1], Jr[3 + k], T[4 * r + 2] * Jr[6 + k]));
    }
  }

  // Rounding floor of |r|_2 for one step of this instance: binary64 cannot
  // resolve the stage residuals of Eq. HOC (or the gradient of Eq. EQ) below
  // about eps times the size of the terms that cancel in them. The bound:
  //   eps (What sum_l I_l + |g| sum_l (|m c_l| + m_l R_l)),
  // What = the largest stage row sum of |seed weights| (acceleration and
  // drag, over all S + 2 nodes), R_l = sum of |t(X_a)| over the joints on
  // the root-to-l path, I_l = (sqrt(tr Sigma_l) + sqrt(m_l) R_l)^2 (a bound
  // on int rho |P|^2 over link l about the root). Identical on the lanes of
  // a group (group-mask shuffles only).
  __device__ double rnorm_floor() const {
    double row = fabs(wk[0]) + fabs(wk[1]);
#pragma unroll
    for (int j = 0; j < S; ++j) row += fabs(wu_row[j]);
    double What = 0.0;
#pragma unroll
    for (int j = 0; j < S; ++j) What = fmax(What, grp.from(row, j));
    double sI = 0.0, sg = 0.0;
    for (int l = 0; l < N; ++l) {
      double R = 0.0;
      for (int a = l; a >= 0; a = B.parent[a]) {
        const double x = rest(a, 3), y = rest(a, 7), z = rest(a, 11);
        R += sqrt(x * x + y * y + z * z);
      }
      const MassMoment M = mass(l);
      const double tr = M.s[0] + M.s[3] + M.s[5], m = M.s[9];
      const double a = sqrt(fmax(tr, 0.0)) + sqrt(fmax(m, 0.0)) * R;
      sI += a * a;
      sg += sqrt(M.s[6] * M.s[6] + M.s[7] * M.s[7] + M.s[8] * M.s[8]) + m * R;
    }
    const double gn = sqrt(B.g[0] * B.g[0] + B.g[1] * B.g[1] + B.g[2] * B.g[2]);
    return 2.220446049250313e-16 * (What * sI + gn * sg);
  }

  // ----------------------------------------------------------- step setup
  // C_i,l = Wk[i][0] T_l(q_prev) + Wk[i][1] T_l(q_cur) for the own stage,
  // the preconditioner blocks at q_cur and the initial guess (linear
  // extrapolation through the two known nodes). q_prev/q_cur are read from
  // the lane's workspace copies. With commit = false the pass runs (so that a
  // warp can run it convergently) but leaves C, the blocks and the guess of
  // the lane untouched; T, G and the axes are scratch either way.
  __device__ __noinline__ void setup(bool commit) const {
    const Ctx self(*this);
    self.setup_body(commit);
  }
  __device__ __forceinline__ void setup_body(bool commit) const {
    double Tp[12], Tc[12], Jr[9], q3[3] = {0.0, 0.0, 0.0};
    // forward: FK at both known nodes; parents' transforms live in T (prev)
    // and G (cur) of the workspace during setup.
    for (int l = 0; l < N; ++l) {
      const int p = B.parent[l], d0 = B.dof[l], nd = ndof(l);
      double Pp[12], Pc[12];
      if (p >= 0) {
        load12(L.T + 12 * p, Pp);
        load12(L.G + 12 * p, Pc);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (k < nd) q3[k] = ws[L.qp + d0 + k];
      link_fk(l, p >= 0 ? Pp : nullptr, q3, Tp, nullptr);  // no Jr at q_prev
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (k < nd) q3[k] = ws[L.qc + d0 + k];
      link_fk(l, p >= 0 ? Pc : nullptr, q3, Tc, Jr);
      store12(L.T + 12 * l, Tp);
      store12(L.G + 12 * l, Tc);
      {  // joint axes at q_cur, for the preconditioner blocks below
        double w[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        link_axes(l, Tc, Jr, w);
#pragma unroll
        for (int k = 0; k < 9; ++k) ws[L.axes + 9 * l + k] = w[k];
      }
      if (S == 1 && commit && B.tk) store12(L.tk + 12 * l, Tc);  // drag energy, contact
      double C[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) C[k] = fma(wk[0], Tp[k], wk[1] * Tc[k]);
      if (S > 1) {
        // gravity folded into the seed: (A - g e4^T) M = A M - g [m c; m]^T,
        // since e4^T M is M's last row
#pragma unroll
        for (int r = 0; r < 3; ++r) C[4 * r + 3] -= B.g[r];
      }
      if (commit) store12(L.C + 12 * l, C);
    }
    // composite world mass moments at q_cur: [Sigma_w(6) h(3) m] per link in
    // the T region (no longer needed)
    for (int l = 0; l < N; ++l) {
      double T[12];
      load12(L.G + 12 * l, T);
      const MassMoment M = mass(l);
      const double* s = M.s;
      // R Sigma R^T, R mc
      double RS[9];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        RS[3 * r + 0] = fma(T[4 * r], s[0], fma(T[4 * r + 1], s[1], T[4 * r + 2] * s[2]));
        RS[3 * r + 1] = fma(T[4 * r], s[1], fma(T[4 * r + 1], s[3], T[4 * r + 2] * s[4]));
        RS[3 * r + 2] = fma(T[4 * r], s[2], fma(T[4 * r + 1], s[4], T[4 * r + 2] * s[5]));
      }
      double Rm[3], t[3] = {T[3], T[7], T[11]};
#pragma unroll
      for (int r = 0; r < 3; ++r) Rm[r] = fma(T[4 * r], s[6], fma(T[4 * r + 1], s[7], T[4 * r + 2] * s[8]));
      const double m = s[9];
      const int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const int r = ij[e][0], c = ij[e][1];
        const double rsr = fma(RS[3 * r], T[4 * c], fma(RS[3 * r + 1], T[4 * c + 1], RS[3 * r + 2] * T[4 * c + 2]));
        ws[L.T + 12 * l + e] = rsr + Rm[r] * t[c] + t[r] * Rm[c] + m * t[r] * t[c];
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) ws[L.T + 12 * l + 6 + r] = fma(m, t[r], Rm[r]);
      ws[L.T + 12 * l + 9] = m;
    }
    for (int l = N - 1; l >= 0; --l) {
      const int p = B.parent[l];
      if (p >= 0)
        for (int k = 0; k < 10; ++k) ws[L.T + 12 * p + k] += ws[L.T + 12 * l + k];
    }
    // joint blocks B_j = W^T I_o W, I_o = tr(Sig_o) I - Sig_o about the joint
    for (int l = 0; l < N; ++l) {
      double w[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) w[k] = ws[L.axes + 9 * l + k];
      const int nd = ndof(l), jt = B.jtype[l];
      double c[10];
      for (int k = 0; k < 10; ++k) c[k] = ws[L.T + 12 * l + k];
      const double o[3] = {ws[L.G + 12 * l + 3], ws[L.G + 12 * l + 7], ws[L.G + 12 * l + 11]};
      const double h[3] = {c[6], c[7], c[8]}, m = c[9];
      const int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
      double So[9];
      for (int e = 0; e < 6; ++e) {
        const int r = ij[e][0], q_ = ij[e][1];
        const double v = c[e] - h[r] * o[q_] - o[r] * h[q_] + m * o[r] * o[q_];
        So[3 * r + q_] = v;
        So[3 * q_ + r] = v;
      }
      const double tr = So[0] + So[4] + So[8];
      double Io[9];
      for (int k = 0; k < 9; ++k) Io[k] = -So[k];
      Io[0] += tr; Io[4] += tr; Io[8] += tr;
      double Bj[9], Pj[9], IW[9];
      // B = W Io W^T with the axes as the rows of W: IW = Io W^T, then W IW
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb)
          IW[3 * r + bb] = fma(Io[3 * r], w[3 * bb], fma(Io[3 * r + 1], w[3 * bb + 1], Io[3 * r + 2] * w[3 * bb + 2]));
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
          const double s = fma(w[3 * a], IW[bb], fma(w[3 * a + 1], IW[3 + bb], w[3 * a + 2] * IW[6 + bb]));
          // translation: the subtree mass along orthonormal axes
          Bj[3 * a + bb] = jt == kTranslation ? (a == bb ? c[9] : 0.0) : s;
          // (hinge: only Bj[0] is used, w[0..2] being its axis)
        }
      {
        // thin rods on ball joints have (near) singular blocks: add 1e-8 of
        // the mean diagonal; a zero-trace block (massless subtree) becomes I
        const double tr = nd == 1 ? Bj[0] : Bj[0] + Bj[4] + Bj[8];
        if (tr > 0.0) {
          const double lam = 1e-8 * tr / nd;
          Bj[0] += lam;
          Bj[4] += lam;
          Bj[8] += lam;
        } else {
#pragma unroll
          for (int k = 0; k < 9; ++k) Bj[k] = (k % 4 == 0) ? 1.0 : 0.0;
        }
      }
      if (nd == 1) {
        Pj[0] = 1.0 / Bj[0];
        if (S > 1) Pj[0] *= Pj[0];
      } else {
        const double a = Bj[0], b_ = Bj[1], c_ = Bj[2], d = Bj[3], e = Bj[4], f = Bj[5], g = Bj[6],
                     hh = Bj[7], ii = Bj[8];
        const double det = a * (e * ii - f * hh) - b_ * (d * ii - f * g) + c_ * (d * hh - e * g);
        const double id = 1.0 / det;
        double X[9] = {(e * ii - f * hh) * id, (c_ * hh - b_ * ii) * id, (b_ * f - c_ * e) * id,
                       (f * g - d * ii) * id,  (a * ii - c_ * g) * id,  (c_ * d - a * f) * id,
                       (d * hh - e * g) * id,  (b_ * g - a * hh) * id,  (a * e - b_ * d) * id};
        if (S > 1) {
          for (int r = 0; r < 3; ++r)
            for (int q_ = 0; q_ < 3; ++q_)
              Pj[3 * r + q_] = X[3 * r] * X[q_] + X[3 * r + 1] * X[3 + q_] + X[3 * r + 2] * X[6 + q_];
        } else {
          for (int k = 0; k < 9; ++k) Pj[k] = X[k];
        }
      }
      if (commit) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (k < nd * nd) ws[L.Pb + 9 * l + k] = Pj[k];
      }
    }
    // initial guess for the own stage
    const double sc = K.nodes[2 + i] / (0.0 - K.nodes[0]);
    if (commit)
      for (int d = 0; d < n; ++d) {
        const double qc = ws[L.qc + d], qp = ws[L.qp + d];
        ws[L.xt + d] = fma(sc, qc - qp, qc);
      }
  }

  // --------------------------------------------------- residual (primal)
  // Evaluates, at the own stage configuration xt: T, axes, seeds G and the
  // wrench suffix sums; r_i = contraction - tau into rt. Returns the lane's
  // share of E (energy for S = 1, |r_i|^2 otherwise); the caller sums over
  // the group. Must be called convergently by the whole warp.
  __device__ __noinline__ double primal(const double* tau) const {
    const Ctx self(*this);
    return self.primal_body(tau);
  }
  __device__ __forceinline__ double primal_body(const double* tau) const {
    double Eown = 0.0;
    const double dt2 = K.dt * K.dt;
    const bool chain = B.chain;
    double Tp[12];  // parent transform (kept in registers along a chain)
    // The joint rotation of link l + 1 (exponential map, Rodrigues) is
    // computed during link l: it does not depend on the chain, so it gives
    // the scheduler independent work next to link l's dependent products.
    double qn[3] = {0.0, 0.0, 0.0}, Rn[9], Jrn[9];
    ExpCoef ecn;
    auto joint_of = [&](int l) {
      const int nd = ndof(l), d0 = B.dof[l], jt = B.jtype[l];
#pragma unroll
      for (int k = 0; k < 3; ++k) qn[k] = k < nd ? ws[L.xt + d0 + k] : 0.0;
      const double u[3] = {B.axis[3 * l], B.axis[3 * l + 1], B.axis[3 * l + 2]};
      joint_rotation(jt, u, qn, Rn, Jrn, jt == kBall ? &ecn : nullptr);
    };
    joint_of(0);
    for (int l = 0; l < N; ++l) {
      const int p = B.parent[l], nd = ndof(l);
      double T[12], Jr[9], R[9], q3[3], w[9];
      const ExpCoef ec = ecn;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        R[k] = Rn[k];
        Jr[k] = Jrn[k];
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) q3[k] = qn[k];
      if (l + 1 < N) joint_of(l + 1);
      if (p >= 0 && !chain) load12(L.T + 12 * p, Tp);
      const int jt = B.jtype[l];
      link_fk_rot(l, p >= 0 ? Tp : nullptr, q3, R, T);
      if (jt == kBall) {  // cached for the tangent passes at this point
        ws[L.ec + 4 * l] = ec.c;
        ws[L.ec + 4 * l + 1] = ec.a;
        ws[L.ec + 4 * l + 2] = ec.b;
        ws[L.ec + 4 * l + 3] = ec.h;
      }
      store12(L.T + 12 * l, T);
      link_axes(l, T, Jr, w);
#pragma unroll
      for (int k = 0; k < 9; ++k)
        if (k < 3 * nd) ws[L.axes + 9 * l + k] = w[k];
      // A = C_i + sum_j Wu[i][j] T_j (stage coupling of Eq. HOC)
      double A[12];
      load12(L.C + 12 * l, A);
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const double wij = wu_row[j];
#pragma unroll
        for (int k = 0; k < 12; ++k) A[k] = fma(wij, grp.from_full(T[k], j), A[k]);
      }
      const MassMoment M = mass(l);
      double G[12];
      if (B.axial) mul_mass_axial(A, M, G);
      else mul_mass(A, M, G);
      const double mc4[4] = {M.s[6], M.s[7], M.s[8], M.s[9]};
      if (S == 1) {
        // Eq. EQ: tr(D M D^T)/(2 dt^2) with D = dt^2 A_kin, the drag potential
        // c tr(D' M D'^T)/dt^2 with D' = dt^2 V, V = (T - T(q_cur))/dt^2, and
        // -g.(T [mc; m]). A holds the seed's A_kin + 2c V and G = A M.
        double ek = 0.0, eg = 0.0, ed = 0.0;
        if (B.drag != 0.0) {
          double Tk[12], Vd[12], VM[12];
          load12(L.tk + 12 * l, Tk);
#pragma unroll
          for (int k = 0; k < 12; ++k) Vd[k] = fma(K.Vu[0][0], T[k], K.Vk[0][1] * Tk[k]);
          mul_mass(Vd, M, VM);
          const double c2 = 2.0 * B.drag;
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            ek = fma(fma(-c2, Vd[k], A[k]), fma(-c2, VM[k], G[k]), ek);
            ed = fma(Vd[k], VM[k], ed);
          }
        } else {
#pragma unroll
          for (int k = 0; k < 12; ++k) ek = fma(A[k], G[k], ek);
        }
#pragma unroll
        for (int r = 0; r < 3; ++r)
          eg = fma(B.g[r], fma(T[4 * r], mc4[0], fma(T[4 * r + 1], mc4[1], fma(T[4 * r + 2], mc4[2], T[4 * r + 3] * mc4[3]))), eg);
        Eown += 0.5 * dt2 * ek + B.drag * dt2 * ed - eg;
      }
      if (S == 1) {  // S > 1: gravity is folded into C (setup)
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) G[4 * r + c] = fma(-B.g[r], mc4[c], G[4 * r + c]);
      }
      if (S == 1 && B.n_contact) {
        // Eq. FRI contact points of this link: energy and dQ/dT = f [p; 1]^T
        const int c0 = B.c_off[l], c1 = B.c_off[l + 1];
        if (c1 > c0) {
          double Tk[12];
          load12(L.tk + 12 * l, Tk);
          for (int c = c0; c < c1; ++c) {
            const double pt[3] = {B.c_pt[3 * c], B.c_pt[3 * c + 1], B.c_pt[3 * c + 2]};
            double P[3], Pk[3], Q, f[3], H[9], Hk[9];
            body_point(T, pt, P);
            body_point(Tk, pt, Pk);
            if (ground_contact(P, Pk, B.c_z0, B.c_d1, B.c_d2, K.dt, &Q, f, H, Hk)) {
              Eown += Q;
#pragma unroll
              for (int r = 0; r < 3; ++r) {
#pragma unroll
                for (int k = 0; k < 3; ++k) G[4 * r + k] = fma(f[r], pt[k], G[4 * r + k]);
                G[4 * r + 3] += f[r];
              }
            }
          }
        }
      }
      store12(L.G + 12 * l, G);
      double w6[6];
      wrench(G, T, w6);
      for (int k = 0; k < 6; ++k) ws[L.acc + 6 * l + k] = w6[k];
#pragma unroll
      for (int k = 0; k < 12; ++k) Tp[k] = T[k];
    }
    // backward: subtree sums and joint contraction
    double rr = 0.0, tq = 0.0;
    double carry[6] = {0, 0, 0, 0, 0, 0};  // child subtree sum along a chain
    for (int l = N - 1; l >= 0; --l) {
      const int p = B.parent[l], d0 = B.dof[l], nd = ndof(l);
      double a[6];
      for (int k = 0; k < 6; ++k) a[k] = ws[L.acc + 6 * l + k] + carry[k];
      const double o[3] = {ws[L.T + 12 * l + 3], ws[L.T + 12 * l + 7], ws[L.T + 12 * l + 11]};
      double of[3];
      cross(o, a + 3, of);
      const double mo[3] = {a[0] - of[0], a[1] - of[1], a[2] - of[2]};
      // rotation: axis . moment about the joint; translation: axis . force
      const bool tr = B.jtype[l] == kTranslation;
      const double load[3] = {tr ? a[3] : mo[0], tr ? a[4] : mo[1], tr ? a[5] : mo[2]};
      for (int k = 0; k < nd; ++k) {
        const double w[3] = {ws[L.axes + 9 * l + 3 * k], ws[L.axes + 9 * l + 3 * k + 1],
                             ws[L.axes + 9 * l + 3 * k + 2]};
        const double tk = tau ? tau[gdof(d0 + k)] : 0.0;
        const double rk = dot3(w, load) - tk;
        ws[L.rt + d0 + k] = rk;
        rr = fma(rk, rk, rr);
        tq = fma(tk, ws[L.xt + d0 + k], tq);
      }
      if (chain) {
        for (int k = 0; k < 6; ++k) {
          carry[k] = a[k];
          ws[L.acc + 6 * l + k] = a[k];  // subtree sums are reused by the tangent pass
        }
      } else if (p >= 0) {
        for (int k = 0; k < 6; ++k) ws[L.acc + 6 * p + k] += a[k];
      }
    }
    return (S == 1) ? (Eown - tq) : rr;
  }

  // ------------------------------------------------ replica-split residual
  // One warp per instance (Newton) holds R = 32 / S replicas of the stage
  // group, and a binary64 FMA costs the sub-partition the same cycles
  // whatever the warp's active mask: the replicas evaluating the same point
  // redundantly cost R times the per-link work. primal_split gives each
  // replica the links rep, rep + R, ...: it computes their joint rotations,
  // joint axes, stage coupling, mass products, seeds and wrenches into its
  // own lanes' slots. The forward kinematics (a product along the tree) and
  // the subtree sums and joint contractions stay sequential on every lane,
  // in primal's order and with its arithmetic, so E, r, T and the subtree
  // sums come out bitwise equal to primal's. A lane then holds the axes,
  // seeds G and exponential-map coefficients of its own links only;
  // complete_split copies the others before a tangent pass reads them.
  // S >= 2 (the one-stage pass adds energy, drag and contact terms per link).
  // Called convergently by the whole warp; surplus lanes (rep == R) own no
  // link.
  __device__ __forceinline__ Lane owner_lane(int l, int R) const {
    Lane o;
    o.p = ws.p + ((l % R) * S + i - grp.lane);
    return o;
  }
  __device__ __noinline__ double primal_split(const double* tau, int rep, int R) const {
    const Ctx self(*this);
    return self.primal_split_body(tau, rep, R);
  }
  __device__ __forceinline__ double primal_split_body(const double* tau, int rep, int R) const {
    const bool chain = B.chain;
    const int slots = (N + R - 1) / R;
    // (1) joint rotations of the own links: R into the axes slots, Jr into
    //     the seed slots (both overwritten in (3)), the exponential-map
    //     coefficients into their own slots
    for (int s = 0; s < slots; ++s) {
      const int l = s * R + rep;
      if (rep >= R || l >= N) continue;
      const int nd = ndof(l), d0 = B.dof[l], jt = B.jtype[l];
      double q3[3], R9[9], Jr[9];
      ExpCoef ec;
#pragma unroll
      for (int k = 0; k < 3; ++k) q3[k] = k < nd ? ws[L.xt + d0 + k] : 0.0;
      const double u[3] = {B.axis[3 * l], B.axis[3 * l + 1], B.axis[3 * l + 2]};
      joint_rotation(jt, u, q3, R9, Jr, jt == kBall ? &ec : nullptr);
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        ws[L.axes + 9 * l + k] = R9[k];
        ws[L.G + 12 * l + k] = Jr[k];
      }
      if (jt == kBall) {
        ws[L.ec + 4 * l] = ec.c;
        ws[L.ec + 4 * l + 1] = ec.a;
        ws[L.ec + 4 * l + 2] = ec.b;
        ws[L.ec + 4 * l + 3] = ec.h;
      }
    }
    __syncwarp();
    // (2) forward kinematics, every lane, in link order
    double Tp[12];
    for (int l = 0; l < N; ++l) {
      const int p = B.parent[l], nd = ndof(l), d0 = B.dof[l];
      const Lane wo = owner_lane(l, R);
      double R9[9], q3[3], T[12];
#pragma unroll
      for (int k = 0; k < 9; ++k) R9[k] = wo[L.axes + 9 * l + k];
#pragma unroll
      for (int k = 0; k < 3; ++k) q3[k] = k < nd ? ws[L.xt + d0 + k] : 0.0;
      if (p >= 0 && !chain) load12(L.T + 12 * p, Tp);
      link_fk_rot(l, p >= 0 ? Tp : nullptr, q3, R9, T);
      store12(L.T + 12 * l, T);
#pragma unroll
      for (int k = 0; k < 12; ++k) Tp[k] = T[k];
    }
    __syncwarp();
    // (3) axes, stage coupling (Eq. HOC), mass product, seed and wrench of
    //     the own links; a replica without a link in a slot recomputes link
    //     N - 1 and stores nothing, so that every lane takes part in the
    //     stage shuffles
    for (int s = 0; s < slots; ++s) {
      const int lr = s * R + rep;
      const bool own = rep < R && lr < N;
      const int l = own ? lr : N - 1;
      double T[12], Jr[9], w[9];
      load12(L.T + 12 * l, T);
#pragma unroll
      for (int k = 0; k < 9; ++k) Jr[k] = ws[L.G + 12 * l + k];
      link_axes(l, T, Jr, w);
      double A[12];
      load12(L.C + 12 * l, A);
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const double wij = wu_row[j];
#pragma unroll
        for (int k = 0; k < 12; ++k) A[k] = fma(wij, grp.from_full(T[k], j), A[k]);
      }
      const MassMoment M = mass(l);
      double G[12];
      if (B.axial) mul_mass_axial(A, M, G);
      else mul_mass(A, M, G);
      double w6[6];
      wrench(G, T, w6);
      if (own) {
        const int nd = ndof(l);
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (k < 3 * nd) ws[L.axes + 9 * l + k] = w[k];
        store12(L.G + 12 * l, G);
#pragma unroll
        for (int k = 0; k < 6; ++k) ws[L.acc + 6 * l + k] = w6[k];
      }
    }
    __syncwarp();
    // (4) every lane: its own copy of each link's wrench, then primal's
    //     backward sweep (subtree sums and joint contraction)
    for (int l = 0; l < N; ++l) {
      const Lane wo = owner_lane(l, R);
      double w6[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) w6[k] = wo[L.acc + 6 * l + k];
      __syncwarp();
#pragma unroll
      for (int k = 0; k < 6; ++k) ws[L.acc + 6 * l + k] = w6[k];
    }
    __syncwarp();
    double rr = 0.0;
    double carry[6] = {0, 0, 0, 0, 0, 0};
    for (int l = N - 1; l >= 0; --l) {
      const int p = B.parent[l], d0 = B.dof[l], nd = ndof(l);
      const Lane wo = owner_lane(l, R);
      double a[6];
      for (int k = 0; k < 6; ++k) a[k] = ws[L.acc + 6 * l + k] + carry[k];
      const double o[3] = {ws[L.T + 12 * l + 3], ws[L.T + 12 * l + 7], ws[L.T + 12 * l + 11]};
      double of[3];
      cross(o, a + 3, of);
      const double mo[3] = {a[0] - of[0], a[1] - of[1], a[2] - of[2]};
      const bool tr = B.jtype[l] == kTranslation;
      const double load[3] = {tr ? a[3] : mo[0], tr ? a[4] : mo[1], tr ? a[5] : mo[2]};
      for (int k = 0; k < nd; ++k) {
        const double w[3] = {wo[L.axes + 9 * l + 3 * k], wo[L.axes + 9 * l + 3 * k + 1],
                             wo[L.axes + 9 * l + 3 * k + 2]};
        const double tk = tau ? tau[gdof(d0 + k)] : 0.0;
        const double rk = dot3(w, load) - tk;
        ws[L.rt + d0 + k] = rk;
        rr = fma(rk, rk, rr);
      }
      if (chain) {
        for (int k = 0; k < 6; ++k) {
          carry[k] = a[k];
          ws[L.acc + 6 * l + k] = a[k];
        }
      } else if (p >= 0) {
        for (int k = 0; k < 6; ++k) ws[L.acc + 6 * p + k] += a[k];
      }
    }
    return rr;
  }
  // Residual pass only at xt by primal_split: returns E (group total).
  __device__ double evaluate_primal_split(const double* tau, int rep, int R) const {
    const double e = primal_split(tau, rep, R);
    double E = 0.0;
#pragma unroll
    for (int j = 0; j < S; ++j) E += grp.from_full(e, j);
    return E;
  }
  // After primal_split: every lane copies the axes, seeds and exponential-map
  // coefficients of the links it does not own from their owners, so that its
  // slots hold what primal leaves.
  __device__ __noinline__ void complete_split(int R) const {
    __syncwarp();
    for (int l = 0; l < N; ++l) {
      const int o = (l % R) * S + i;
      const bool copy = o != grp.lane;
      const Lane wo = owner_lane(l, R);
      const int nd = ndof(l);
      double v[25];
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = wo[L.G + 12 * l + k];
#pragma unroll
      for (int k = 0; k < 9; ++k) v[12 + k] = k < 3 * nd ? wo[L.axes + 9 * l + k] : 0.0;
      const bool ball = B.jtype[l] == kBall;
#pragma unroll
      for (int k = 0; k < 4; ++k) v[21 + k] = ball ? wo[L.ec + 4 * l + k] : 0.0;
      __syncwarp();
      if (copy) {
#pragma unroll
        for (int k = 0; k < 12; ++k) ws[L.G + 12 * l + k] = v[k];
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (k < 3 * nd) ws[L.axes + 9 * l + k] = v[12 + k];
        if (ball)
#pragma unroll
          for (int k = 0; k < 4; ++k) ws[L.ec + 4 * l + k] = v[21 + k];
      }
    }
    __syncwarp();
  }

  // V += the twist of joint l's DOFs along the direction at offset dir (own
  // stage slice); o is the joint origin. Three DOFs are summed into one axis
  // rate first (one cross product instead of three).
  __device__ __forceinline__ void add_joint_twist(int l, int nd, int d0, const double* o, int dir,
                                                  double* V) const {
    if (nd == 1) {
      const double w[3] = {ws[L.axes + 9 * l], ws[L.axes + 9 * l + 1], ws[L.axes + 9 * l + 2]};
      add_twist(B.jtype[l], o, w, ws[dir + d0], V);
    } else {
      double wj[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double vk = ws[dir + d0 + k];
#pragma unroll
        for (int c = 0; c < 3; ++c) wj[c] = fma(vk, ws[L.axes + 9 * l + 3 * k + c], wj[c]);
      }
      add_twist(B.jtype[l], o, wj, 1.0, V);
    }
  }

  // ------------------------------------------------------- tangent passes
  // d/de of the residual pass of the own stage along a direction v (own
  // stage slice at workspace offset `dir`), with the seeds perturbed by
  //   kGrad: B_k,l = sum_i Wu[i][k] Tdot_i,l M_l  -> (Jr^T v)_k   (Eq. EQHOC gradient)
  //   kJvp:  B_i,l = sum_j Wu[i][j] Tdot_j,l M_l  -> (Jr v)_i     (Jacobian columns)
  //   kGn:   as kJvp but without the second-derivative terms of the
  //          kinematics: the Gauss-Newton product int dP/dq^T dP/dq v / dt^2
  //          of Eq. EQ (one stage).
  // The result, times `scale`, goes to offset `out`. Needs the primal pass's
  // T, G, axes and acc at the same point. Convergent across the warp.
  enum TangentMode { kGrad = 0, kJvp = 1, kGn = 2 };
  // [l_first, l_end) (warp-uniform): the links the direction can move. It
  // has no component on the DOFs outside that range, and every link it moves
  // lies in the subtree of one of its joints, numbered inside the range. So
  // the twists, seed tangents and wrench tangents are zero before l_first
  // (the forward sweep only stores those zeros) and past l_end, where the
  // residual tangents are zero too (no link there is an ancestor of a moved
  // one: ancestors come first); the backward sweep starts at l_end - 1.
  template <int MODE>
  __device__ __noinline__ void tangent_pass(int dir, int out, double scale, int l_first = 0,
                                            int l_end = -1) const {
    const Ctx self(*this);
    self.template tangent_body<MODE>(dir, out, scale, l_first, l_end < 0 ? N : l_end);
  }
  template <int MODE>
  __device__ __forceinline__ void tangent_body(int dir, int out, double scale, int l_first,
                                               int l_end) const {
    const bool chain = B.chain;
    double V[6] = {0, 0, 0, 0, 0, 0};  // parent twist (kept in registers along a chain)
    for (int l = 0; l < l_first; ++l)
      for (int k = 0; k < 6; ++k) {
        ws[L.V + 6 * l + k] = 0.0;
        ws[L.accd + 6 * l + k] = 0.0;
      }
    if (l_end < N)
      for (int d = B.dof[l_end]; d < n; ++d) ws[out + d] = 0.0;
    for (int l = l_first; l < l_end; ++l) {
      const int p = B.parent[l], d0 = B.dof[l], nd = ndof(l);
      if (!chain) {
        if (p >= 0) {
          for (int k = 0; k < 6; ++k) V[k] = ws[L.V + 6 * p + k];
        } else {
          for (int k = 0; k < 6; ++k) V[k] = 0.0;
        }
      }
      double T[12];
      load12(L.T + 12 * l, T);
      const double o[3] = {T[3], T[7], T[11]};
      add_joint_twist(l, nd, d0, o, dir, V);
      for (int k = 0; k < 6; ++k) ws[L.V + 6 * l + k] = V[k];
      // Tdot = [w]x T + v at the world origin
      double Td[12];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double col[3] = {T[c], T[4 + c], T[8 + c]};
        double wc[3];
        cross(V, col, wc);
        Td[c] = wc[0];
        Td[4 + c] = wc[1];
        Td[8 + c] = wc[2];
      }
      Td[3] += V[3];
      Td[7] += V[4];
      Td[11] += V[5];
      double Bs[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) Bs[k] = 0.0;
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const double wgt = (MODE == kGrad) ? wu_col[j] : wu_row[j];
#pragma unroll
        for (int k = 0; k < 12; ++k) Bs[k] = fma(wgt, grp.from_full(Td[k], j), Bs[k]);
      }
      const MassMoment M = mass(l);
      double Bm[12];
      if (B.axial) mul_mass_axial(Bs, M, Bm);
      else mul_mass(Bs, M, Bm);
      if (S == 1 && B.n_contact) {
        // contact points: d/de of f [p; 1]^T = (H Pdot) [p; 1]^T, Pdot = Tdot [p; 1]
        const int c0 = B.c_off[l], c1 = B.c_off[l + 1];
        if (c1 > c0) {
          double Tk[12];
          load12(L.tk + 12 * l, Tk);
          for (int c = c0; c < c1; ++c) {
            const double pt[3] = {B.c_pt[3 * c], B.c_pt[3 * c + 1], B.c_pt[3 * c + 2]};
            double P[3], Pk[3], Pd[3], Q, f[3], H[9], Hk[9];
            body_point(T, pt, P);
            body_point(Tk, pt, Pk);
            if (ground_contact(P, Pk, B.c_z0, B.c_d1, B.c_d2, K.dt, &Q, f, H, Hk)) {
              body_point(Td, pt, Pd);
#pragma unroll
              for (int r = 0; r < 3; ++r) {
                const double fd = fma(H[3 * r], Pd[0], fma(H[3 * r + 1], Pd[1], H[3 * r + 2] * Pd[2]));
#pragma unroll
                for (int k = 0; k < 3; ++k) Bm[4 * r + k] = fma(fd, pt[k], Bm[4 * r + k]);
                Bm[4 * r + 3] += fd;
              }
            }
          }
        }
      }
      double w6[6];
      if (MODE == kGn) {
        wrench(Bm, T, w6);
      } else {
        double G[12];
        load12(L.G + 12 * l, G);
        wrench_tangent(G, Bm, T, Td, w6);
      }
      for (int k = 0; k < 6; ++k) ws[L.accd + 6 * l + k] = w6[k];
    }
    double carry[6] = {0, 0, 0, 0, 0, 0};
    for (int l = l_end - 1; l >= 0; --l) {
      const int p = B.parent[l], d0 = B.dof[l], nd = ndof(l);
      double ad[6], T[12];
      for (int k = 0; k < 6; ++k) ad[k] = ws[L.accd + 6 * l + k] + carry[k];
      load12(L.T + 12 * l, T);
      const double o[3] = {T[3], T[7], T[11]};
      const int jt = B.jtype[l];
      if (MODE == kGn) {
        double t3[3];
        cross(o, ad + 3, t3);
        const double mdo[3] = {ad[0] - t3[0], ad[1] - t3[1], ad[2] - t3[2]};
        const bool tr = jt == kTranslation;
        const double load[3] = {tr ? ad[3] : mdo[0], tr ? ad[4] : mdo[1], tr ? ad[5] : mdo[2]};
        for (int k = 0; k < nd; ++k) {
          const double w[3] = {ws[L.axes + 9 * l + 3 * k], ws[L.axes + 9 * l + 3 * k + 1],
                               ws[L.axes + 9 * l + 3 * k + 2]};
          ws[out + d0 + k] = scale * dot3(w, load);
        }
      } else {
        double a[6], V[6];
        for (int k = 0; k < 6; ++k) {
          a[k] = ws[L.acc + 6 * l + k];
          V[k] = ws[L.V + 6 * l + k];
        }
        double od[3];
        cross(V, o, od);
        od[0] += V[3];
        od[1] += V[4];
        od[2] += V[5];
        double t1[3], t2[3], t3[3];
        cross(o, a + 3, t1);
        const double mo[3] = {a[0] - t1[0], a[1] - t1[1], a[2] - t1[2]};
        cross(od, a + 3, t2);
        cross(o, ad + 3, t3);
        const double mdo[3] = {ad[0] - t2[0] - t3[0], ad[1] - t2[1] - t3[1], ad[2] - t2[2] - t3[2]};
        // ball: d/de of w_k = R Jr e_k adds R dJr e_k, whose contraction
        // with mo is (dJr^T R^T mo)_k
        double zb[3] = {0.0, 0.0, 0.0};
        if (jt == kBall) {
          double th[3], v[3], cab[4], u[3];
          for (int k = 0; k < 3; ++k) {
            th[k] = ws[L.xt + d0 + k];
            v[k] = ws[dir + d0 + k];
          }
          for (int k = 0; k < 4; ++k) cab[k] = ws[L.ec + 4 * l + k];
#pragma unroll
          for (int c = 0; c < 3; ++c) u[c] = fma(T[c], mo[0], fma(T[4 + c], mo[1], T[8 + c] * mo[2]));
          jr_tangent_dot(th, v, cab, u, zb);
        }
        // rotation: d/de [w . (M - o x F)] = (V x w) . mo + w . mdo = w . (mo x V
        // + mdo); translation: d/de [w . F] = w . (F x V + Fd)
        // (jt is uniform across the warp: every lane is at link l)
        const bool tr = jt == kTranslation;
        double qv[3];
        cross(tr ? a + 3 : mo, V, qv);
#pragma unroll
        for (int r = 0; r < 3; ++r) qv[r] += tr ? ad[3 + r] : mdo[r];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if (k >= nd) break;
          const double w[3] = {ws[L.axes + 9 * l + 3 * k], ws[L.axes + 9 * l + 3 * k + 1],
                               ws[L.axes + 9 * l + 3 * k + 2]};
          ws[out + d0 + k] = scale * (dot3(w, qv) + zb[k]);
        }
      }
      if (chain) {
        for (int k = 0; k < 6; ++k) carry[k] = ad[k];
      } else if (p >= 0) {
        for (int k = 0; k < 6; ++k) ws[L.accd + 6 * p + k] += ad[k];
      }
    }
  }

  // gradient of Eq. EQHOC: 2 Jr^T r, into gt
  __device__ __forceinline__ void tangent() const { tangent_pass<kGrad>(L.rt, L.gt, 2.0, 0, N); }

  // Full evaluation at xt: returns E (group total, identical on the group's
  // lanes); rt = residual of the own stage; gt = dE/dq of the own stage.
  __device__ double evaluate(const double* tau) const {
    double e = primal(tau);
    double E = 0.0;
#pragma unroll
    for (int j = 0; j < S; ++j) E += grp.from_full(e, j);
    if (S == 1) {
      for (int d = 0; d < n; ++d) ws[L.gt + d] = ws[L.rt + d];
    } else {
      tangent();
    }
    return E;
  }

  // Residual pass only at xt: returns E (group total); rt = residual.
  __device__ double evaluate_primal(const double* tau) const {
    const double e = primal(tau);
    double E = 0.0;
#pragma unroll
    for (int j = 0; j < S; ++j) E += grp.from_full(e, j);
    return E;
  }

  // ----------------------------------------------------- Newton (LM), adjoint
  // Warp-cooperative dense algebra. One warp owns one instance: R = 32/S
  // replicas of the S-lane stage group evaluate the residual pass at the same
  // point and split the Jacobian columns; the Gram matrix, the factorisation
  // and the solves are shared by all 32 lanes through the instance's dense
  // region (D). All these functions are called convergently by the warp.

  // Column c = (stage k = c / n, dof e = c % n) of Jr at the primal point
  // (S >= 2: the stage residuals of Eq. HOC; S == 1 with exact = false: the
  // Gauss-Newton matrix of Eq. EQ, int dP/dq^T dP/dq / dt^2; exact = true:
  // the Hessian of Eq. EQ). Replica `rep` of R computes columns rep, rep+R,
  // ...; every lane writes its stage's rows. S n tangent passes in total.
  __device__ __noinline__ void build_jacobian_warp(double* D, const DenseLayout& DL, int rep, int R,
                                                   bool exact) const {
    const int Sn = S * n;
    const int rounds = (Sn + R - 1) / R;
    for (int t = 0; t < rounds; ++t) {
      // the round's columns run DOF-major (the stages of one DOF side by
      // side), so that one round covers few joints and their subtrees
      const int c = rep + t * R;
      const bool real = c < Sn && rep < R;
      const int cc = real ? c : Sn - 1;  // surplus replicas repeat the last column and discard it
      const int e = cc / S, k = cc - e * S;
      for (int d = 0; d < n; ++d) ws[L.u + d] = (i == k && d == e) ? 1.0 : 0.0;
      // the link that owns DOF e; the warp's passes cover the smallest such
      // link up to the end of the largest of their subtrees
      int le = N - 1;
      while (le > 0 && B.dof[le] > e) --le;
      const int lend = __reduce_max_sync(0xffffffffu, B.sub_end[le]);
      le = __reduce_min_sync(0xffffffffu, le);
      if (S == 1 && !exact) tangent_pass<kGn>(L.u, L.jc, 1.0, le, lend);
      else tangent_pass<kJvp>(L.u, L.jc, 1.0, le, lend);
      if (real)
        for (int d = 0; d < n; ++d) D[DL.J + (int64_t)(k * n + e) * Sn + i * n + d] = ws[L.jc + d];
    }
    __syncwarp();
  }

  // H = Jr^T Jr, gg = Jr^T r (S >= 2) or H = the Gauss-Newton matrix, gg = r
  // (S == 1). Needs r in D (written by replica 0 before). Returns max diag(H)
  // (same value on every lane).
  __device__ __noinline__ double gram_warp(double* D, const DenseLayout& DL) const {
    const int Sn = S * n;
    const int lane = threadIdx.x & 31;
    if (S == 1) {
      for (int a = lane; a < Sn; a += 32) {
        for (int c = 0; c < Sn; ++c) D[DL.H + (int64_t)a * Sn + c] = D[DL.J + (int64_t)c * Sn + a];
        D[DL.gg + a] = D[DL.r + a];
      }
    } else {
      // 4 x 4 blocks of the lower triangle, one block per lane at a time:
      // each entry is the same in-order dot product over the rows, with a
      // quarter of the loads of one entry per lane
      const int nb = (Sn + 3) / 4;
      const int nblocks = nb * (nb + 1) / 2;
      const double* J = D + DL.J;
      for (int q = lane; q < nblocks; q += 32) {
        // block (bi, bj), bi >= bj, row-major over the lower triangle
        int bi = (int)((sqrt(8.0 * q + 1.0) - 1.0) * 0.5);
        while ((bi + 1) * (bi + 2) / 2 <= q) ++bi;
        while (bi * (bi + 1) / 2 > q) --bi;
        const int bj = q - bi * (bi + 1) / 2;
        const int a0 = 4 * bi, c0 = 4 * bj;
        const double* ja[4];
        const double* jc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          ja[u] = J + (int64_t)min(a0 + u, Sn - 1) * Sn;  // rows past Sn repeat the last column
          jc[u] = J + (int64_t)min(c0 + u, Sn - 1) * Sn;
        }
        double h[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) h[u][v] = 0.0;
        for (int rr = 0; rr < Sn; ++rr) {
          double x[4], y[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            x[u] = ja[u][rr];
            y[u] = jc[u][rr];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) h[u][v] = fma(x[u], y[v], h[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int a = a0 + u, c = c0 + v;
            if (a < Sn && c <= a) {
              D[DL.H + (int64_t)a * Sn + c] = h[u][v];
              D[DL.H + (int64_t)c * Sn + a] = h[u][v];
            }
          }
      }
      for (int a = lane; a < Sn; a += 32) {
        const double* ja = D + DL.J + (int64_t)a * Sn;
        double g = 0.0;
        for (int rr = 0; rr < Sn; ++rr) g = fma(ja[rr], D[DL.r + rr], g);
        D[DL.gg + a] = g;
      }
    }
    __syncwarp();
    double hmax = 0.0;
    for (int a = lane; a < Sn; a += 32) hmax = fmax(hmax, D[DL.H + (int64_t)a * Sn + a]);
    for (int o = 16; o > 0; o >>= 1) hmax = fmax(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
    return hmax;
  }

  __device__ __forceinline__ static double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  }

  // Cholesky of H + lambda I into A (lower triangle stored column-major:
  // L[r][c] at A[c Sn + r], so that the lanes' rows of one column are
  // contiguous) and dl = -(H + lambda I)^-1 gg. Returns false (on every
  // lane) if a pivot is not positive.
  __device__ __noinline__ bool factor_solve_warp(double* D, const DenseLayout& DL, double lambda) const {
    const int Sn = S * n;
    const int lane = threadIdx.x & 31;
    double* A = D + DL.A;
    const double* H = D + DL.H;
    for (int j = 0; j < Sn; ++j) {
      double s = 0.0;
      for (int k = lane; k < j; k += 32) s = fma(A[(int64_t)k * Sn + j], A[(int64_t)k * Sn + j], s);
      s = warp_sum(s);
      const double dj = H[(int64_t)j * Sn + j] + lambda - s;
      if (!(dj > 0.0)) return false;
      const double ljj = sqrt(dj), inv = 1.0 / ljj;
      for (int r = j + 1 + lane; r < Sn; r += 32) {
        double t = H[(int64_t)j * Sn + r];  // = H[r][j] (symmetric), contiguous over the lanes
        for (int k = 0; k < j; ++k) t = fma(-A[(int64_t)k * Sn + r], A[(int64_t)k * Sn + j], t);
        A[(int64_t)j * Sn + r] = t * inv;
      }
      if (lane == 0) A[(int64_t)j * Sn + j] = ljj;
      __syncwarp();
    }
    double* y = D + DL.dl;
    for (int r = 0; r < Sn; ++r) {
      double s = 0.0;
      for (int k = lane; k < r; k += 32) s = fma(A[(int64_t)k * Sn + r], y[k], s);
      s = warp_sum(s);
      const double v = (-D[DL.gg + r] - s) / A[(int64_t)r * Sn + r];
      __syncwarp();
      if (lane == 0) y[r] = v;
      __syncwarp();
    }
    for (int r = Sn - 1; r >= 0; --r) {
      double s = 0.0;
      for (int k = r + 1 + lane; k < Sn; k += 32) s = fma(A[(int64_t)r * Sn + k], y[k], s);
      s = warp_sum(s);
      const double v = (y[r] - s) / A[(int64_t)r * Sn + r];
      __syncwarp();
      if (lane == 0) y[r] = v;
      __syncwarp();
    }
    return true;
  }

  // Solves Jr^T mu = gb by Gaussian elimination with partial pivoting on the
  // J region (column-major J read row-major is Jr^T), mu into dl. Returns
  // false on a zero pivot. Destroys J.
  __device__ __noinline__ bool lu_solve_transposed_warp(double* D, const DenseLayout& DL) const {
    const int Sn = S * n;
    const int lane = threadIdx.x & 31;
    double* M = D + DL.J;
    double* b = D + DL.gb;
    for (int c = 0; c < Sn; ++c) {
      double best = -1.0;
      int piv = Sn;
      for (int r = c + lane; r < Sn; r += 32) {
        const double v = fabs(M[(int64_t)r * Sn + c]);
        if (v > best) { best = v; piv = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, piv, o);
        if (ob > best || (ob == best && op < piv)) { best = ob; piv = op; }
      }
      if (!(best > 0.0)) return false;
      if (piv != c) {
        for (int k = lane; k < Sn; k += 32) {
          const double t = M[(int64_t)c * Sn + k];
          M[(int64_t)c * Sn + k] = M[(int64_t)piv * Sn + k];
          M[(int64_t)piv * Sn + k] = t;
        }
        if (lane == 0) {
          const double t = b[c];
          b[c] = b[piv];
          b[piv] = t;
        }
      }
      __syncwarp();
      const double inv = 1.0 / M[(int64_t)c * Sn + c];
      for (int r = c + 1 + lane; r < Sn; r += 32) {
        const double f = M[(int64_t)r * Sn + c] * inv;
        if (f != 0.0) {
          for (int k = c + 1; k < Sn; ++k) M[(int64_t)r * Sn + k] = fma(-f, M[(int64_t)c * Sn + k], M[(int64_t)r * Sn + k]);
          b[r] = fma(-f, b[c], b[r]);
        }
      }
      __syncwarp();
    }
    double* mu = D + DL.dl;
    for (int r = Sn - 1; r >= 0; --r) {
      double s = 0.0;
      for (int k = r + 1 + lane; k < Sn; k += 32) s = fma(M[(int64_t)r * Sn + k], mu[k], s);
      s = warp_sum(s);
      const double v = (b[r] - s) / M[(int64_t)r * Sn + r];
      __syncwarp();
      if (lane == 0) mu[r] = v;
      __syncwarp();
    }
    return true;
  }

  // Tangents Tdot_l of the own stage's transforms along the own slice of a
  // direction (offset `dir`), into the G region (12 per link). Needs the
  // primal pass's T and axes.
  __device__ __noinline__ void transform_tangents(int dir) const {
    for (int l = 0; l < N; ++l) {
      const int p = B.parent[l], d0 = B.dof[l], nd = ndof(l);
      double V[6];
      if (p >= 0) {
        for (int k = 0; k < 6; ++k) V[k] = ws[L.V + 6 * p + k];
      } else {
        for (int k = 0; k < 6; ++k) V[k] = 0.0;
      }
      double T[12];
      load12(L.T + 12 * l, T);
      const double o[3] = {T[3], T[7], T[11]};
      add_joint_twist(l, nd, d0, o, dir, V);
      for (int k = 0; k < 6; ++k) ws[L.V + 6 * l + k] = V[k];
      double Td[12];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double col[3] = {T[c], T[4 + c], T[8 + c]};
        double wc[3];
        cross(V, col, wc);
        Td[c] = wc[0];
        Td[4 + c] = wc[1];
        Td[8 + c] = wc[2];
      }
      Td[3] += V[3];
      Td[7] += V[4];
      Td[11] += V[5];
      store12(L.G + 12 * l, Td);
      if (S == 1 && B.n_contact) {
        // contact points: the load Hk^T Pdot at the point's position at q_k,
        // for the known-node product of q_cur (T holds the step end here)
        double Tk[12];
        load12(L.tk + 12 * l, Tk);
        for (int c = B.c_off[l]; c < B.c_off[l + 1]; ++c) {
          const double pt[3] = {B.c_pt[3 * c], B.c_pt[3 * c + 1], B.c_pt[3 * c + 2]};
          double P[3], Pk[3], Pd[3], Q, f[3], H[9], Hk[9];
          body_point(T, pt, P);
          body_point(Tk, pt, Pk);
          double g[3] = {0.0, 0.0, 0.0};
          if (ground_contact(P, Pk, B.c_z0, B.c_d1, B.c_d2, K.dt, &Q, f, H, Hk)) {
            body_point(Td, pt, Pd);
#pragma unroll
            for (int r = 0; r < 3; ++r) g[r] = fma(Hk[r], Pd[0], fma(Hk[3 + r], Pd[1], Hk[6 + r] * Pd[2]));
          }
#pragma unroll
          for (int r = 0; r < 3; ++r) ws[L.cg + 3 * c + r] = g[r];
        }
      }
    }
  }

  // Vector-Jacobian product of the residuals with the known node j (0 =
  // q_prev, 1 = q_cur) at configuration qj (offset): sum_i mu_i^T dr_i/dq_j
  // = contraction of the twists at q_j with the seeds
  //   B_l = (sum_i Wk[i][j] Tdot_i,l) M_l,
  // Tdot_i,l from transform_tangents along mu. Result into `out` (n).
  // Overwrites T, axes and acc. Convergent across the warp.
  __device__ __noinline__ void known_node_vjp(int j, int qj, int out) const {
    for (int l = 0; l < N; ++l) {
      const int p = B.parent[l], d0 = B.dof[l], nd = ndof(l);
      double Tp[12], T[12], Jr[9], q3[3], w[9];
      if (p >= 0) load12(L.T + 12 * p, Tp);
      for (int k = 0; k < nd; ++k) q3[k] = ws[qj + d0 + k];
      link_fk(l, p >= 0 ? Tp : nullptr, q3, T, Jr);
      store12(L.T + 12 * l, T);
      link_axes(l, T, Jr, w);
      for (int k = 0; k < 3 * nd; ++k) ws[L.axes + 9 * l + k] = w[k];
      double Bs[12], Td[12];
      load12(L.G + 12 * l, Td);
#pragma unroll
      for (int k = 0; k < 12; ++k) Bs[k] = 0.0;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const double wgt = fma(2.0 * B.drag, K.Vk[s][j], K.Wk[s][j]);  // seed weight incl. drag
#pragma unroll
        for (int k = 0; k < 12; ++k) Bs[k] = fma(wgt, grp.from_full(Td[k], s), Bs[k]);
      }
      const MassMoment M = mass(l);
      double Bm[12], w6[6];
      if (B.axial) mul_mass_axial(Bs, M, Bm);
      else mul_mass(Bs, M, Bm);
      if (S == 1 && j == 1 && B.n_contact) {
        // contact points: their loads (from transform_tangents) act at P(q_k)
        for (int c = B.c_off[l]; c < B.c_off[l + 1]; ++c) {
          const double pt[3] = {B.c_pt[3 * c], B.c_pt[3 * c + 1], B.c_pt[3 * c + 2]};
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            const double g = ws[L.cg + 3 * c + r];
#pragma unroll
            for (int k = 0; k < 3; ++k) Bm[4 * r + k] = fma(g, pt[k], Bm[4 * r + k]);
            Bm[4 * r + 3] += g;
          }
        }
      }
      wrench(Bm, T, w6);
      for (int k = 0; k < 6; ++k) ws[L.acc + 6 * l + k] = w6[k];
    }
    for (int l = N - 1; l >= 0; --l) {
      const int p = B.parent[l], d0 = B.dof[l], nd = ndof(l);
      double a[6];
      for (int k = 0; k < 6; ++k) a[k] = ws[L.acc + 6 * l + k];
      const double o[3] = {ws[L.T + 12 * l + 3], ws[L.T + 12 * l + 7], ws[L.T + 12 * l + 11]};
      double of[3];
      cross(o, a + 3, of);
      const double mo[3] = {a[0] - of[0], a[1] - of[1], a[2] - of[2]};
      const bool tr = B.jtype[l] == kTranslation;
      const double load[3] = {tr ? a[3] : mo[0], tr ? a[4] : mo[1], tr ? a[5] : mo[2]};
      for (int k = 0; k < nd; ++k) {
        const double w[3] = {ws[L.axes + 9 * l + 3 * k], ws[L.axes + 9 * l + 3 * k + 1],
                             ws[L.axes + 9 * l + 3 * k + 2]};
        ws[out + d0 + k] = dot3(w, load);
      }
      if (p >= 0)
        for (int k = 0; k < 6; ++k) ws[L.acc + 6 * p + k] += a[k];
    }
  }

  // ------------------------------------------------- L-BFGS vector algebra
  // (group-divergent code: group-mask shuffles only)
  // Vector sweeps over the own stage slice, kChunk DOFs at a time: a
  // chunk's loads are issued together before any of its arithmetic, so a
  // sweep waits for memory about n / kChunk times instead of n times. Sums
  // accumulate in plain sequential order.
  static constexpr int kChunk = 4;

  // group sum of v[a..] . v[b..]
  __device__ double gdot(int a, int b_) const {
    double s = 0.0;
    for (int d0 = 0; d0 < n; d0 += kChunk) {
      double u[kChunk], v[kChunk];
#pragma unroll
      for (int k = 0; k < kChunk; ++k)
        if (d0 + k < n) {
          u[k] = ws[a + d0 + k];
          v[k] = ws[b_ + d0 + k];
        }
#pragma unroll
      for (int k = 0; k < kChunk; ++k)
        if (d0 + k < n) s = fma(u[k], v[k], s);
    }
    return grp.sum(s);
  }

  // v[y..] <- ca v[a..] + v[b..] (b >= 0) or ca v[a..] (b < 0), chunked.
  __device__ void vlin(int y, double ca, int a, int b_) const {
    for (int d0 = 0; d0 < n; d0 += kChunk) {
      double av[kChunk], bv[kChunk];
#pragma unroll
      for (int k = 0; k < kChunk; ++k)
        if (d0 + k < n) {
          av[k] = ws[a + d0 + k];
          bv[k] = b_ >= 0 ? ws[b_ + d0 + k] : 0.0;
        }
#pragma unroll
      for (int k = 0; k < kChunk; ++k)
        if (d0 + k < n) ws[y + d0 + k] = b_ >= 0 ? fma(ca, av[k], bv[k]) : ca * av[k];
    }
  }

  // v[y..] <- v[y..] + cf v[x..] when `on`, then the group sum of v[z..] .
  // v[y..] (updated where on): one step of the two-loop recursion fused with
  // the next step's dot product. z < 0 skips the dot product (returns 0).
  __device__ double axpy_dot(int y, double cf, int x, int z, bool on) const {
    double s = 0.0;
    for (int d0 = 0; d0 < n; d0 += kChunk) {
      double yv[kChunk], xv[kChunk], zv[kChunk];
#pragma unroll
      for (int k = 0; k < kChunk; ++k)
        if (d0 + k < n) {
          yv[k] = ws[y + d0 + k];
          xv[k] = ws[x + d0 + k];
          zv[k] = z >= 0 ? ws[z + d0 + k] : 0.0;
        }
#pragma unroll
      for (int k = 0; k < kChunk; ++k)
        if (d0 + k < n) {
          if (on) {
            yv[k] = fma(cf, xv[k], yv[k]);
            ws[y + d0 + k] = yv[k];
          }
          s = fma(zv[k], yv[k], s);
        }
    }
    return z >= 0 ? grp.sum(s) : 0.0;
  }

  // ------------------------- binary32 search direction (PBAD_LBFGS_F32)
  // Binary32 vectors are packed two per workspace double: element d is the
  // low (even d) or high (odd d) word of slot d / 2. With n odd the high
  // word of the last slot is 0, which every update keeps at 0.
  __device__ static __forceinline__ float lo32(double v) { return __int_as_float(__double2loint(v)); }
  __device__ static __forceinline__ float hi32(double v) { return __int_as_float(__double2hiint(v)); }
  __device__ static __forceinline__ double pack32(float lo, float hi) {
    return __hiloint2double(__float_as_int(hi), __float_as_int(lo));
  }
  __device__ __forceinline__ int n2() const { return (n + 1) >> 1; }

  // v[y..] <- v[y..] + cf v[x..] (binary32, packed) when `on`, then the
  // binary32 group sum of v[z..] . v[y..] (z < 0: none, returns 0).
  __device__ float axpy_dot32(int y, float cf, int x, int z, bool on) const {
    const int h = n2();
    float s = 0.0f;
    for (int d0 = 0; d0 < h; d0 += kChunk) {
      double yv[kChunk], xv[kChunk], zv[kChunk];
#pragma unroll
      for (int k = 0; k < kChunk; ++k)
        if (d0 + k < h) {
          yv[k] = ws[y + d0 + k];
          xv[k] = ws[x + d0 + k];
          zv[k] = z >= 0 ? ws[z + d0 + k] : 0.0;
        }
#pragma unroll
      for (int k = 0; k < kChunk; ++k)
        if (d0 + k < h) {
          float y0 = lo32(yv[k]), y1 = hi32(yv[k]);
          if (on) {
            y0 = fmaf(cf, lo32(xv[k]), y0);
            y1 = fmaf(cf, hi32(xv[k]), y1);
            ws[y + d0 + k] = pack32(y0, y1);
          }
          s = fmaf(lo32(zv[k]), y0, s);
          s = fmaf(hi32(zv[k]), y1, s);
        }
    }
    return z >= 0 ? grp.sum(s) : 0.0f;
  }

  // Packed binary32 copy of ca v[a..] (binary64), rounded to nearest.
  __device__ void pack_scaled(int y, double ca, int a) const {
    const int h = n2();
    for (int d0 = 0; d0 < h; d0 += kChunk) {
      double v[2 * kChunk];
#pragma unroll
      for (int k = 0; k < 2 * kChunk; ++k) v[k] = 2 * d0 + k < n ? ws[a + 2 * d0 + k] : 0.0;
#pragma unroll
      for (int k = 0; k < kChunk; ++k)
        if (d0 + k < h)
          ws[y + d0 + k] = pack32(__double2float_rn(ca * v[2 * k]), __double2float_rn(ca * v[2 * k + 1]));
    }
  }

  // v[y..] <- the packed binary32 vector at a, widened, where `on`; returns
  // the binary64 group sum of v[g..] . (the widened vector), or 0 if g < 0.
  __device__ double unpack_dot(int y, int a, int g, bool on) const {
    const int h = n2();
    double s = 0.0;
    for (int d0 = 0; d0 < h; d0 += kChunk) {
      double pv[kChunk], gv[2 * kChunk];
#pragma unroll
      for (int k = 0; k < kChunk; ++k)
        if (d0 + k < h) pv[k] = ws[a + d0 + k];
#pragma unroll
      for (int k = 0; k < 2 * kChunk; ++k)
        if (2 * d0 + k < n) gv[k] = g >= 0 ? ws[g + 2 * d0 + k] : 0.0;
#pragma unroll
      for (int k = 0; k < 2 * kChunk; ++k) {
        const int d = 2 * d0 + k;
        if (d < n) {
          const double v = (double)((k & 1) ? hi32(pv[k >> 1]) : lo32(pv[k >> 1]));
          if (on) ws[y + d] = v;
          s = fma(gv[k], v, s);
        }
      }
    }
    return g >= 0 ? grp.sum(s) : 0.0;
  }

  // The two-loop recursion with every vector operation in binary32 on the
  // packed pairs (ring of m, newest at head - 1) and H0 = gamma P applied in
  // binary64 to the binary32 vector; for the groups with `start` the widened
  // direction goes to d. The packed working vector lives in the trial
  // gradient's region, dead at this point for every group. Returns g . d.
  __device__ __noinline__ double direction32(bool start, int nh, int head, double gamma,
                                             int m) const {
    const Ctx self(*this);
    return self.direction32_body(start, nh, head, gamma, m);
  }
  __device__ __forceinline__ double direction32_body(bool start, int nh, int head, double gamma,
                                                     int m) const {
    const int q = L.gt;
    const int nh_w = __reduce_max_sync(0xffffffffu, start ? nh : 0);
    if (start) pack_scaled(q, -1.0, L.g);
    auto slot = [&](int t) { return (head - 1 - t + 2 * m) % m; };
    float al[kMaxHistory];
    float a = 0.0f;
    if (nh_w > 0)
      a = (float)ws[L.rho + slot(0)] * axpy_dot32(q, 0.0f, q, L.sh + slot(0) * n, false);
    for (int t = 0; t < nh_w; ++t) {
      const int j = slot(t);
      al[t] = a;
      const bool more = t + 1 < nh_w;
      const int jn = more ? slot(t + 1) : 0;
      const float dot = axpy_dot32(q, -a, L.yh + j * n, more ? L.sh + jn * n : -1, start && t < nh);
      if (more) a = (float)ws[L.rho + jn] * dot;
    }
    unpack_dot(L.d, q, -1, start);
    precond(start ? L.d : L.gt);
    if (start) pack_scaled(q, gamma, L.d);
    if (nh_w > 0) {
      float bta = (float)ws[L.rho + slot(nh_w - 1)] *
                  axpy_dot32(q, 0.0f, q, L.yh + slot(nh_w - 1) * n, false);
      for (int t = nh_w - 1; t >= 0; --t) {
        const int j = slot(t);
        const int jn = t > 0 ? slot(t - 1) : 0;
        const float dot = axpy_dot32(q, al[t] - bta, L.sh + j * n, t > 0 ? L.yh + jn * n : -1,
                                     start && t < nh);
        if (t > 0) bta = (float)ws[L.rho + jn] * dot;
      }
    }
    return unpack_dot(L.d, q, L.g, start);
  }

  // v <- P v for the own slice of v at offset a (Kronecker: stage block Ps,
  // joint blocks Pb).
  __device__ __noinline__ void precond(int a) const {
    const Ctx self(*this);
    self.precond_body(a);
  }
  __device__ __forceinline__ void precond_body(int a) const {
    for (int l = 0; l < N; ++l) {
      const int d0 = B.dof[l], nd = ndof(l);
      double u[3] = {0.0, 0.0, 0.0}, t[3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (k < nd) u[k] = ws[a + d0 + k];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (r < nd && c < nd) s = fma(ws[L.Pb + 9 * l + nd * r + c], u[c], s);
        t[r] = s;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < S; ++j) s = fma(ps_row[j], grp.from(t[k], j), s);
        if (k < nd) ws[a + d0 + k] = s;
      }
    }
  }
};

}  // namespace pbad
