// Link-parallel mapping of the hot path for serial chains: one lane per
// (instance, collocation stage, link), S N lanes per instance (S N <= 32),
// floor(32 / (S N)) instances per warp.
//
// The stage-parallel mapping (pbad_kernels.cuh) walks the link tree
// sequentially in each stage lane and keeps its per-link arrays in a global
// workspace. Here every per-link quantity of the residual and tangent passes
// (transform, seed, joint axes, subtree wrench, exponential-map
// coefficients) is a register of its own lane, and the two sequential
// dependencies of Algorithm DERIV on a chain become warp-shuffle scans over
// the lanes of one stage:
//   - forward kinematics T_l = T_{l-1} X_l J(q_l): an inclusive product scan
//     of the joint-local transforms (Hillis-Steele, ceil(log2 N) compositions
//     per lane);
//   - the subtree (suffix) sums of the world wrenches and, in the tangent
//     pass, the prefix sums of the joint twists: additive scans.
// The coupling of the stages through the second-derivative weights of the
// collocation polynomial (Eq. HOC) reads the same link's lanes of the other
// stages by shuffles. The solver's vectors, the preconditioner blocks, the
// known-node combination and the L-BFGS history live in shared memory, one
// slot column per lane, so a loop trip touches global memory only for the
// model constants of its link, the torques and the outputs.
#pragma once
#include "pbad_df64.cuh"
#include "pbad_launch.cuh"

namespace pbad {

constexpr unsigned kFull = 0xffffffffu;

// Shared-memory slots of one lane (doubles): three DOF slots per vector
// (a hinge uses the first), then the known-node combination C (3x4), the
// preconditioner block Pb (3x3) and the L-BFGS ring (m pairs of 3 slots,
// rho per pair).
struct LpLayout {
  int x, g, d, r, xt, gt, rt, qp, qc, C, Pb, sh, yh, rho, total;
  __host__ __device__ void make(int m) {
    int o = 0;
    x = o; o += 3;
    g = o; o += 3;
    d = o; o += 3;
    r = o; o += 3;
    xt = o; o += 3;
    gt = o; o += 3;
    rt = o; o += 3;
    qp = o; o += 3;
    qc = o; o += 3;
    C = o; o += 12;
    Pb = o; o += 9;
    sh = o; o += 3 * m;
    yh = o; o += 3 * m;
    rho = o; o += (m > 0 ? m : 1);
    total = o;
  }
};

// Per-link values the residual pass leaves for the tangent pass (registers).
struct LpHot {
  double T[12];  // world transform of the own link at the own stage
  double G[12];  // seed dE/dT (Eq. HOC: sum_j W_ij T_j M - g [mc; m]^T)
  double w[9];   // world joint axes (hinge: w[0..2]; ball: columns of R Jr)
  double a[6];   // world wrench summed over the link and its descendants
  double cab[4]; // exponential-map coefficients (c, a, b, h) at the own q
};

template <int S>
struct LpCtx {
  Bucket B;
  const Colloc& K;
  LpLayout L;
  Lane sm;         // the lane's shared-memory slot column
  int lane, base;  // lane in the warp, first lane of its group
  int l, i;        // own link and stage
  int N, n, gs;    // links, DOFs, lanes per group (S N)
  bool real;       // the lane belongs to a full group
  int b;           // instance (always a valid index)
  int jt, nd, d0;  // own joint type, DOF count, first DOF
  double u[3];     // hinge axis
  double wk[2], wu_row[S], wu_col[S], ps_row[S];

  __device__ LpCtx(const Bucket& B_, const Colloc& K_, double* smem_warp, int m, int64_t warp,
                   bool* active)
      : B(B_), K(K_) {
    L.make(m);
    N = B.N;
    n = B.n;
    gs = S * N;
    lane = threadIdx.x & 31;
    const int G = 32 / gs;
    const int grp = lane / gs;
    real = grp < G;
    base = real ? grp * gs : lane;
    const int j = real ? lane - base : 0;
    l = j / S;
    i = j - l * S;
    const int64_t inst = warp * G + grp;
    *active = real && inst < B.count;
    b = *active ? (int)inst : 0;
    sm.p = smem_warp + lane;
    jt = B.jtype[l];
    nd = jt == kHinge ? 1 : 3;
    d0 = B.dof[l];
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = B.axis[3 * l + k];
    const double c2 = 2.0 * B.drag;
    wk[0] = fma(c2, K.Vk[i][0], K.Wk[i][0]);
    wk[1] = fma(c2, K.Vk[i][1], K.Wk[i][1]);
#pragma unroll
    for (int jj = 0; jj < S; ++jj) {
      wu_row[jj] = fma(c2, K.Vu[i][jj], K.Wu[i][jj]);
      wu_col[jj] = fma(c2, K.Vu[jj][i], K.Wu[jj][i]);
      ps_row[jj] = K.Ps[i][jj];
    }
  }

  // ------------------------------------------------------------ shuffles
  // (all convergent over the whole warp)
  // the same link's lane of stage j
  __device__ __forceinline__ double from_stage(double v, int j) const {
    return __shfl_sync(kFull, v, min(base + l * S + j, 31));
  }
  // the same stage's lane of link l - off (own value when l < off)
  __device__ __forceinline__ double from_down(double v, int off) const {
    return __shfl_sync(kFull, v, l >= off ? lane - S * off : lane);
  }
  // the same stage's lane of link l + off (own value past the tip)
  __device__ __forceinline__ double from_up(double v, int off) const {
    return __shfl_sync(kFull, v, l + off < N ? lane + S * off : lane);
  }
  // group sum, identical bits on every lane of the group: with one group
  // per warp an xor butterfly over the warp (lanes past the group add 0),
  // otherwise the group's lanes in order
  __device__ __forceinline__ double gsum(double v) const {
    if (gs > 16) {
      double t = real ? v : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
      return t;
    }
    double t = 0.0;
    for (int k = 0; k < gs; ++k) t += __shfl_sync(kFull, v, min(base + k, 31));
    return t;
  }
  __device__ __forceinline__ double gmax(double v) const {
    double t = real ? v : -1.0;
    if (gs > 16) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(kFull, t, o));
      return t;
    }
    double r = -1.0;
    for (int k = 0; k < gs; ++k) r = fmax(r, __shfl_sync(kFull, t, min(base + k, 31)));
    return r;
  }

  // ------------------------------------------------------ model constants
  __device__ __forceinline__ double rest(int k) const {
    return B.rest[((int64_t)l * 12 + k) * B.count + b];
  }
  __device__ __forceinline__ MassMoment mass() const {
    MassMoment M;
#pragma unroll
    for (int k = 0; k < 10; ++k) M.s[k] = B.mm[((int64_t)l * 10 + k) * B.count + b];
    return M;
  }
  __device__ __forceinline__ int64_t gdof(int k) const { return B.dof_off + (int64_t)b * n + d0 + k; }
  __device__ __forceinline__ int64_t gstage(int k) const {
    return (int64_t)S * B.dof_off + ((int64_t)b * S + i) * n + d0 + k;
  }
  __device__ __forceinline__ void load3(int off, double* q) const {
#pragma unroll
    for (int k = 0; k < 3; ++k) q[k] = k < nd ? sm[off + k] : 0.0;
  }

  // Joint-local transform X_l J(q_l) of the own link, its rotation R and
  // (balls, translations) Jr; cab receives the exponential-map coefficients.
  __device__ __forceinline__ void local_transform(const double* q, double* XJ, double* Jr,
                                                  double* cab) const {
    double R[9];
    ExpCoef ec;
    joint_rotation(jt, u, q, R, Jr, jt == kBall ? &ec : nullptr);
    if (cab && jt == kBall) {
      cab[0] = ec.c;
      cab[1] = ec.a;
      cab[2] = ec.b;
      cab[3] = ec.h;
    }
    if (B.rest_eye[l]) {
#pragma unroll
      for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int c = 0; c < 3; ++c) XJ[4 * r + c] = R[3 * r + c];
        XJ[4 * r + 3] = rest(4 * r + 3);
      }
      if (jt == kTranslation) {
#pragma unroll
        for (int r = 0; r < 3; ++r) XJ[4 * r + 3] += q[r];
      }
    } else {
      double X[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) X[k] = rest(k);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          XJ[4 * r + c] = fma(X[4 * r], R[c], fma(X[4 * r + 1], R[3 + c], X[4 * r + 2] * R[6 + c]));
        XJ[4 * r + 3] = jt == kTranslation
                            ? fma(X[4 * r], q[0], fma(X[4 * r + 1], q[1], fma(X[4 * r + 2], q[2], X[4 * r + 3])))
                            : X[4 * r + 3];
      }
    }
  }

  // Forward kinematics of the chain: inclusive product scan of the
  // joint-local transforms over the links of the own stage (T in: X_l J_l;
  // out: T_l = X_0 J_0 ... X_l J_l).
  __device__ __forceinline__ void fk_scan(double* T) const {
    for (int off = 1; off < N; off <<= 1) {
      double Tl[12], P[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) Tl[k] = from_down(T[k], off);
      compose(Tl, T, P);
      if (l >= off) {
#pragma unroll
        for (int k = 0; k < 12; ++k) T[k] = P[k];
      }
    }
  }
  // inclusive suffix sum over the links of the own stage (subtree sums of a
  // chain)
  template <int W>
  __device__ __forceinline__ void suffix_scan(double* a) const {
    for (int off = 1; off < N; off <<= 1) {
      double t[W];
#pragma unroll
      for (int k = 0; k < W; ++k) t[k] = from_up(a[k], off);
      if (l + off < N) {
#pragma unroll
        for (int k = 0; k < W; ++k) a[k] += t[k];
      }
    }
  }
  // inclusive prefix sum over the links of the own stage
  template <int W>
  __device__ __forceinline__ void prefix_scan(double* a) const {
    for (int off = 1; off < N; off <<= 1) {
      double t[W];
#pragma unroll
      for (int k = 0; k < W; ++k) t[k] = from_down(a[k], off);
      if (l >= off) {
#pragma unroll
        for (int k = 0; k < W; ++k) a[k] += t[k];
      }
    }
  }

  __device__ __forceinline__ void axes(const double* T, const double* Jr, double* w) const {
    if (jt == kHinge) {
#pragma unroll
      for (int r = 0; r < 3; ++r) w[r] = fma(T[4 * r], u[0], fma(T[4 * r + 1], u[1], T[4 * r + 2] * u[2]));
#pragma unroll
      for (int k = 3; k < 9; ++k) w[k] = 0.0;
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int r = 0; r < 3; ++r)
          w[3 * k + r] = fma(T[4 * r], Jr[k], fma(T[4 * r + 1], Jr[3 + k], T[4 * r + 2] * Jr[6 + k]));
    }
  }

  // Rounding floor of |r|_2 (the bound of Ctx::rnorm_floor), identical on
  // the lanes of a group.
  __device__ double rnorm_floor() const {
    double row = fabs(wk[0]) + fabs(wk[1]);
#pragma unroll
    for (int j = 0; j < S; ++j) row += fabs(wu_row[j]);
    const double What = gmax(row);
    const double x = rest(3), y = rest(7), z = rest(11);
    double R = sqrt(x * x + y * y + z * z);
    prefix_scan<1>(&R);
    const MassMoment M = mass();
    const double tr = M.s[0] + M.s[3] + M.s[5], m = M.s[9];
    const double a = sqrt(fmax(tr, 0.0)) + sqrt(fmax(m, 0.0)) * R;
    const double own_I = i == 0 ? a * a : 0.0;
    const double own_g = i == 0 ? sqrt(M.s[6] * M.s[6] + M.s[7] * M.s[7] + M.s[8] * M.s[8]) + m * R : 0.0;
    const double sI = gsum(own_I), sg = gsum(own_g);
    const double gn = sqrt(B.g[0] * B.g[0] + B.g[1] * B.g[1] + B.g[2] * B.g[2]);
    return 2.220446049250313e-16 * (What * sI + gn * sg);
  }

  // ----------------------------------------------------------- step setup
  // C = Wk[i][0] T(q_prev) + Wk[i][1] T(q_cur) of the own link and stage
  // (gravity folded in for S >= 2), the preconditioner block of the own
  // joint at q_cur (joint-space mass matrix block from the composite world
  // mass moments of the subtree) and the initial guess of the own stage.
  // With commit = false nothing is written (the pass still runs, so that the
  // warp runs it convergently).
  __device__ void setup(bool commit) const {
    double qa[3], qb[3], Tp[12], Tc[12], Jr[9], w[9];
    load3(L.qp, qa);
    load3(L.qc, qb);
    local_transform(qa, Tp, Jr, nullptr);
    local_transform(qb, Tc, Jr, nullptr);
    fk_scan(Tp);
    fk_scan(Tc);
    axes(Tc, Jr, w);
    if (commit) {
      double C[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) C[k] = fma(wk[0], Tp[k], wk[1] * Tc[k]);
      if (S > 1) {
#pragma unroll
        for (int r = 0; r < 3; ++r) C[4 * r + 3] -= B.g[r];
      }
#pragma unroll
      for (int k = 0; k < 12; ++k) sm[L.C + k] = C[k];
    }
    // composite world mass moment [Sigma_w (6) h (3) m] of the own link,
    // summed over the subtree
    const MassMoment M = mass();
    const double* s = M.s;
    double c10[10];
    {
      double RS[9];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        RS[3 * r + 0] = fma(Tc[4 * r], s[0], fma(Tc[4 * r + 1], s[1], Tc[4 * r + 2] * s[2]));
        RS[3 * r + 1] = fma(Tc[4 * r], s[1], fma(Tc[4 * r + 1], s[3], Tc[4 * r + 2] * s[4]));
        RS[3 * r + 2] = fma(Tc[4 * r], s[2], fma(Tc[4 * r + 1], s[4], Tc[4 * r + 2] * s[5]));
      }
      double Rm[3];
      const double t[3] = {Tc[3], Tc[7], Tc[11]};
#pragma unroll
      for (int r = 0; r < 3; ++r) Rm[r] = fma(Tc[4 * r], s[6], fma(Tc[4 * r + 1], s[7], Tc[4 * r + 2] * s[8]));
      const double m = s[9];
      const int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const int r = ij[e][0], c = ij[e][1];
        const double rsr = fma(RS[3 * r], Tc[4 * c], fma(RS[3 * r + 1], Tc[4 * c + 1], RS[3 * r + 2] * Tc[4 * c + 2]));
        c10[e] = rsr + Rm[r] * t[c] + t[r] * Rm[c] + m * t[r] * t[c];
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) c10[6 + r] = fma(m, t[r], Rm[r]);
      c10[9] = m;
    }
    suffix_scan<10>(c10);
    // joint block B = W Io W^T, Io = tr(Sig_o) I - Sig_o about the joint
    const double o[3] = {Tc[3], Tc[7], Tc[11]};
    const double h[3] = {c10[6], c10[7], c10[8]}, m = c10[9];
    const int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    double So[9];
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const int r = ij[e][0], q_ = ij[e][1];
      const double v = c10[e] - h[r] * o[q_] - o[r] * h[q_] + m * o[r] * o[q_];
      So[3 * r + q_] = v;
      So[3 * q_ + r] = v;
    }
    const double tr = So[0] + So[4] + So[8];
    double Io[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Io[k] = -So[k];
    Io[0] += tr;
    Io[4] += tr;
    Io[8] += tr;
    double Bj[9], IW[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int bb = 0; bb < 3; ++bb)
        IW[3 * r + bb] = fma(Io[3 * r], w[3 * bb], fma(Io[3 * r + 1], w[3 * bb + 1], Io[3 * r + 2] * w[3 * bb + 2]));
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) {
        const double sv = fma(w[3 * a], IW[bb], fma(w[3 * a + 1], IW[3 + bb], w[3 * a + 2] * IW[6 + bb]));
        Bj[3 * a + bb] = jt == kTranslation ? (a == bb ? c10[9] : 0.0) : sv;
      }
    {
      const double trb = nd == 1 ? Bj[0] : Bj[0] + Bj[4] + Bj[8];
      if (trb > 0.0) {
        const double lam = 1e-8 * trb / nd;
        Bj[0] += lam;
        Bj[4] += lam;
        Bj[8] += lam;
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) Bj[k] = (k % 4 == 0) ? 1.0 : 0.0;
      }
    }
    double Pj[9];
    if (nd == 1) {
      Pj[0] = 1.0 / Bj[0];
      if (S > 1) Pj[0] *= Pj[0];
#pragma unroll
      for (int k = 1; k < 9; ++k) Pj[k] = 0.0;
    } else {
      const double a = Bj[0], b_ = Bj[1], c_ = Bj[2], d = Bj[3], e = Bj[4], f = Bj[5], g = Bj[6],
                   hh = Bj[7], ii = Bj[8];
      const double det = a * (e * ii - f * hh) - b_ * (d * ii - f * g) + c_ * (d * hh - e * g);
      const double id = 1.0 / det;
      const double X[9] = {(e * ii - f * hh) * id, (c_ * hh - b_ * ii) * id, (b_ * f - c_ * e) * id,
                           (f * g - d * ii) * id,  (a * ii - c_ * g) * id,  (c_ * d - a * f) * id,
                           (d * hh - e * g) * id,  (b_ * g - a * hh) * id,  (a * e - b_ * d) * id};
      if (S > 1) {
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int q_ = 0; q_ < 3; ++q_)
            Pj[3 * r + q_] = X[3 * r] * X[q_] + X[3 * r + 1] * X[3 + q_] + X[3 * r + 2] * X[6 + q_];
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) Pj[k] = X[k];
      }
    }
    if (commit) {
#pragma unroll
      for (int k = 0; k < 9; ++k) sm[L.Pb + k] = Pj[k];
      const double sc = K.nodes[2 + i] / (0.0 - K.nodes[0]);
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (k < nd) sm[L.xt + k] = fma(sc, qb[k] - qa[k], qb[k]);
    }
  }

  // --------------------------------------------------- residual (primal)
  // At the own stage configuration xt: T, G, axes, subtree wrench; r of the
  // own DOFs into rt. Returns the lane's share of E (S = 1: its link's
  // energy terms minus its torque work; S >= 2: its |r|^2).
  __device__ double primal(const double* tau, LpHot& h) const {
    double q3[3], Jr[9];
    load3(L.xt, q3);
    local_transform(q3, h.T, Jr, h.cab);
    fk_scan(h.T);
    axes(h.T, Jr, h.w);
    double A[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) A[k] = sm[L.C + k];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const double wij = wu_row[j];
#pragma unroll
      for (int k = 0; k < 12; ++k) A[k] = fma(wij, from_stage(h.T[k], j), A[k]);
    }
    const MassMoment M = mass();
    if (B.axial) mul_mass_axial(A, M, h.G);
    else mul_mass(A, M, h.G);
    double Eown = 0.0;
    if (S == 1) {
      // Eq. EQ: tr(D M D^T)/(2 dt^2) with D = dt^2 A and -g.(T [mc; m])
      const double dt2 = K.dt * K.dt;
      double ek = 0.0, eg = 0.0;
#pragma unroll
      for (int k = 0; k < 12; ++k) ek = fma(A[k], h.G[k], ek);
#pragma unroll
      for (int r = 0; r < 3; ++r)
        eg = fma(B.g[r], fma(h.T[4 * r], M.s[6], fma(h.T[4 * r + 1], M.s[7], fma(h.T[4 * r + 2], M.s[8], h.T[4 * r + 3] * M.s[9]))), eg);
      Eown = 0.5 * dt2 * ek - eg;
      const double mc4[4] = {M.s[6], M.s[7], M.s[8], M.s[9]};
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) h.G[4 * r + c] = fma(-B.g[r], mc4[c], h.G[4 * r + c]);
    }
    wrench(h.G, h.T, h.a);
    suffix_scan<6>(h.a);
    const double o[3] = {h.T[3], h.T[7], h.T[11]};
    double of[3];
    cross(o, h.a + 3, of);
    const bool tr = jt == kTranslation;
    const double load[3] = {tr ? h.a[3] : h.a[0] - of[0], tr ? h.a[4] : h.a[1] - of[1],
                            tr ? h.a[5] : h.a[2] - of[2]};
    double rr = 0.0, tq = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (k < nd) {
        const double tk = tau ? tau[gdof(k)] : 0.0;
        const double rk = dot3(h.w + 3 * k, load) - tk;
        sm[L.rt + k] = rk;
        rr = fma(rk, rk, rr);
        tq = fma(tk, q3[k], tq);
      }
    }
    return (S == 1) ? (Eown - tq) : rr;
  }

  // The same residual pass with everything after the joint-local transform
  // (forward-kinematics scan, joint axes, stage coupling, mass product,
  // seeds, wrenches, subtree sums, contraction) in double-float arithmetic
  // on the binary32 pipes; the joint rotations stay binary64. Leaves the
  // tangent pass the same values, rounded to binary64.
  __device__ double primal_df64(const double* tau, LpHot& h) const {
    double q3[3], Jr[9], XJ[12];
    load3(L.xt, q3);
    local_transform(q3, XJ, Jr, h.cab);
    df64 T[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) T[k] = df_from(XJ[k]);
    for (int off = 1; off < N; off <<= 1) {
      df64 Tl[12], P[12];
      const int src = l >= off ? lane - S * off : lane;
#pragma unroll
      for (int k = 0; k < 12; ++k) Tl[k] = df_shfl(T[k], src);
      df_compose(Tl, T, P);
      if (l >= off) {
#pragma unroll
        for (int k = 0; k < 12; ++k) T[k] = P[k];
      }
    }
    df64 w[9];
    if (jt == kHinge) {
      const df64 ud[3] = {df_from(u[0]), df_from(u[1]), df_from(u[2])};
#pragma unroll
      for (int r = 0; r < 3; ++r) w[r] = df_fma(T[4 * r], ud[0], df_fma(T[4 * r + 1], ud[1], df_mul(T[4 * r + 2], ud[2])));
#pragma unroll
      for (int k = 3; k < 9; ++k) w[k] = df_zero();
    } else {
      df64 J[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) J[k] = df_from(Jr[k]);
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int r = 0; r < 3; ++r)
          w[3 * k + r] = df_fma(T[4 * r], J[k], df_fma(T[4 * r + 1], J[3 + k], df_mul(T[4 * r + 2], J[6 + k])));
    }
    df64 A[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) A[k] = df_from(sm[L.C + k]);
    const int sbase = min(base + l * S, 31);
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const df64 wij = df_from(wu_row[j]);
#pragma unroll
      for (int k = 0; k < 12; ++k) A[k] = df_fma(wij, df_shfl(T[k], min(sbase + j, 31)), A[k]);
    }
    const MassMoment M = mass();
    df64 s[10], G[12];
#pragma unroll
    for (int k = 0; k < 10; ++k) s[k] = df_from(M.s[k]);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const df64 a0 = A[4 * r], a1 = A[4 * r + 1], a2 = A[4 * r + 2], a3 = A[4 * r + 3];
      G[4 * r + 0] = df_fma(a0, s[0], df_fma(a1, s[1], df_fma(a2, s[2], df_mul(a3, s[6]))));
      G[4 * r + 1] = df_fma(a0, s[1], df_fma(a1, s[3], df_fma(a2, s[4], df_mul(a3, s[7]))));
      G[4 * r + 2] = df_fma(a0, s[2], df_fma(a1, s[4], df_fma(a2, s[5], df_mul(a3, s[8]))));
      G[4 * r + 3] = df_fma(a0, s[6], df_fma(a1, s[7], df_fma(a2, s[8], df_mul(a3, s[9]))));
    }
    double Eown = 0.0;
    if (S == 1) {
      df64 ek = df_zero(), eg = df_zero();
#pragma unroll
      for (int k = 0; k < 12; ++k) ek = df_fma(A[k], G[k], ek);
#pragma unroll
      for (int r = 0; r < 3; ++r)
        eg = df_fma(df_from(B.g[r]),
                    df_fma(T[4 * r], s[6], df_fma(T[4 * r + 1], s[7], df_fma(T[4 * r + 2], s[8], df_mul(T[4 * r + 3], s[9])))),
                    eg);
      Eown = 0.5 * K.dt * K.dt * df_to(ek) - df_to(eg);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const df64 gr = df_from(-B.g[r]);
#pragma unroll
        for (int c = 0; c < 4; ++c) G[4 * r + c] = df_fma(gr, s[6 + c], G[4 * r + c]);
      }
    }
    // world wrench of the seed: m = ax(G_R R^T) + t x f, f = G_t
    df64 a[6];
    {
      auto Y = [&](int r, int k) {
        return df_fma(G[4 * r], T[4 * k], df_fma(G[4 * r + 1], T[4 * k + 1], df_mul(G[4 * r + 2], T[4 * k + 2])));
      };
      const df64 f[3] = {G[3], G[7], G[11]};
      const df64 t[3] = {T[3], T[7], T[11]};
      df64 tf[3];
      df_cross(t, f, tf);
      a[0] = df_add(df_sub(Y(2, 1), Y(1, 2)), tf[0]);
      a[1] = df_add(df_sub(Y(0, 2), Y(2, 0)), tf[1]);
      a[2] = df_add(df_sub(Y(1, 0), Y(0, 1)), tf[2]);
      a[3] = f[0];
      a[4] = f[1];
      a[5] = f[2];
    }
    for (int off = 1; off < N; off <<= 1) {
      const int src = l + off < N ? lane + S * off : lane;
      df64 t[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) t[k] = df_shfl(a[k], src);
      if (l + off < N) {
#pragma unroll
        for (int k = 0; k < 6; ++k) a[k] = df_add(a[k], t[k]);
      }
    }
    const df64 o[3] = {T[3], T[7], T[11]};
    df64 of[3];
    df_cross(o, a + 3, of);
    const bool tr = jt == kTranslation;
    const df64 load[3] = {tr ? a[3] : df_sub(a[0], of[0]), tr ? a[4] : df_sub(a[1], of[1]),
                          tr ? a[5] : df_sub(a[2], of[2])};
    double rr = 0.0, tq = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (k < nd) {
        const double tk = tau ? tau[gdof(k)] : 0.0;
        const df64 wl = df_fma(w[3 * k], load[0], df_fma(w[3 * k + 1], load[1], df_mul(w[3 * k + 2], load[2])));
        const double rk = df_to(df_sub(wl, df_from(tk)));
        sm[L.rt + k] = rk;
        rr = fma(rk, rk, rr);
        tq = fma(tk, q3[k], tq);
      }
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      h.T[k] = df_to(T[k]);
      h.G[k] = df_to(G[k]);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) h.w[k] = df_to(w[k]);
#pragma unroll
    for (int k = 0; k < 6; ++k) h.a[k] = df_to(a[k]);
    return (S == 1) ? (Eown - tq) : rr;
  }

  // ------------------------------------------------------- tangent pass
  // d/de of the residual pass along the own stage slice of a direction v
  // (slots `dir`), with the seeds perturbed by B_k = sum_i Wu[i][k] Tdot_i M
  // (Eq. EQHOC gradient: (Jr^T v)_k), times `scale` into slots `out`.
  __device__ void tangent(const LpHot& h, int dir, int out, double scale) const {
    const double o[3] = {h.T[3], h.T[7], h.T[11]};
    double v[3];
    load3(dir, v);
    double V[6] = {0, 0, 0, 0, 0, 0};
    if (nd == 1) {
      add_twist(jt, o, h.w, v[0], V);
    } else {
      double wj[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) wj[c] = fma(v[0], h.w[c], fma(v[1], h.w[3 + c], v[2] * h.w[6 + c]));
      add_twist(jt, o, wj, 1.0, V);
    }
    prefix_scan<6>(V);
    double Td[12];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double col[3] = {h.T[c], h.T[4 + c], h.T[8 + c]};
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
      const double wgt = wu_col[j];
#pragma unroll
      for (int k = 0; k < 12; ++k) Bs[k] = fma(wgt, from_stage(Td[k], j), Bs[k]);
    }
    const MassMoment M = mass();
    double Bm[12];
    if (B.axial) mul_mass_axial(Bs, M, Bm);
    else mul_mass(Bs, M, Bm);
    double ad[6];
    wrench_tangent(h.G, Bm, h.T, Td, ad);
    suffix_scan<6>(ad);
    double od[3];
    cross(V, o, od);
    od[0] += V[3];
    od[1] += V[4];
    od[2] += V[5];
    double t1[3], t2[3], t3[3];
    cross(o, h.a + 3, t1);
    const double mo[3] = {h.a[0] - t1[0], h.a[1] - t1[1], h.a[2] - t1[2]};
    cross(od, h.a + 3, t2);
    cross(o, ad + 3, t3);
    const double mdo[3] = {ad[0] - t2[0] - t3[0], ad[1] - t2[1] - t3[1], ad[2] - t2[2] - t3[2]};
    double zb[3] = {0.0, 0.0, 0.0};
    if (jt == kBall) {
      double th[3], uu[3];
      load3(L.xt, th);
#pragma unroll
      for (int c = 0; c < 3; ++c) uu[c] = fma(h.T[c], mo[0], fma(h.T[4 + c], mo[1], h.T[8 + c] * mo[2]));
      jr_tangent_dot(th, v, h.cab, uu, zb);
    }
    const bool tr = jt == kTranslation;
    double qv[3];
    cross(tr ? h.a + 3 : mo, V, qv);
#pragma unroll
    for (int r = 0; r < 3; ++r) qv[r] += tr ? ad[3 + r] : mdo[r];
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k < nd) sm[out + k] = scale * (dot3(h.w + 3 * k, qv) + zb[k]);
  }

  // v <- P v on the own slots at `a`: joint block Pb, then the stage block
  // Ps across the same link's stage lanes.
  __device__ void precond(int a, bool on) const {
    double uu[3], t[3];
    load3(a, uu);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (r < nd && c < nd) s = fma(sm[L.Pb + nd * r + c], uu[c], s);
      t[r] = s;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < S; ++j) s = fma(ps_row[j], from_stage(t[k], j), s);
      if (on && k < nd) sm[a + k] = s;
    }
  }
  // group sum of own-slot dot products v[a] . v[b]
  __device__ __forceinline__ double gdot(int a, int b_) const {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k < nd) s = fma(sm[a + k], sm[b_ + k], s);
    return gsum(s);
  }
};

// ------------------------------------------------------------------------
// E, r and dE/dq at given stage configurations, link-parallel.
// ------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(128) k_eval_lp(const __grid_constant__ LaunchArgs A) {
  extern __shared__ double lp_smem[];
  const Bucket& B = A.bk[find_bucket(A)];
  LpLayout L;
  L.make(0);
  const int64_t warp = ((int64_t)(blockIdx.x - B.block_begin) * blockDim.x + threadIdx.x) >> 5;
  double* smw = lp_smem + (threadIdx.x >> 5) * (L.total * 32);
  bool active;
  LpCtx<S> c(B, A.K, smw, 0, warp, &active);
#pragma unroll
  for (int k = 0; k < 3; ++k)
    if (k < c.nd) {
      c.sm[L.qp + k] = A.q_prev0[c.gdof(k)];
      c.sm[L.qc + k] = A.q_cur0[c.gdof(k)];
    }
  c.setup(true);
#pragma unroll
  for (int k = 0; k < 3; ++k)
    if (k < c.nd) c.sm[L.xt + k] = A.q_star[c.gstage(k)];
  LpHot h;
  const double E = c.gsum(A.df64 ? c.primal_df64(A.tau, h) : c.primal(A.tau, h));
  if (S == 1) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k < c.nd) c.sm[L.gt + k] = c.sm[L.rt + k];
  } else {
    c.tangent(h, L.rt, L.gt, 2.0);
  }
  if (active) {
    if (c.l == 0 && c.i == 0) A.E_out[B.inst_off + c.b] = E;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k < c.nd) {
        A.grad_out[c.gstage(k)] = c.sm[L.gt + k];
        if (A.resid_out) A.resid_out[c.gstage(k)] = c.sm[L.rt + k];
      }
  }
}

// ------------------------------------------------------------------------
// Persistent L-BFGS rollout, link-parallel: the same algorithm, decisions
// and outputs as rollout_lbfgs (binary64 direction), one group of S N lanes
// per instance. Every loop trip is convergent over the warp: groups in
// different phases share each pass with per-group predicates.
// ------------------------------------------------------------------------
template <int S>
__device__ __forceinline__ void rollout_lp_body(const LaunchArgs& A, const Bucket& B) {
  extern __shared__ double lp_smem[];
  const int m = A.history;
  LpLayout L;
  L.make(m);
  const int64_t warp = ((int64_t)(blockIdx.x - B.block_begin) * blockDim.x + threadIdx.x) >> 5;
  double* smw = lp_smem + (threadIdx.x >> 5) * (L.total * 32);
  bool active;
  const LpCtx<S> c(B, A.K, smw, m, warp, &active);
  const Lane sm = c.sm;
  const int nd = c.nd;
  const int64_t D = A.D;
  const bool head_lane = c.l == 0 && c.i == 0;  // writes the per-instance outputs

#pragma unroll
  for (int k = 0; k < 3; ++k) {
    sm[L.qp + k] = k < nd ? A.q_prev0[c.gdof(k)] : 0.0;
    sm[L.qc + k] = k < nd ? A.q_cur0[c.gdof(k)] : 0.0;
  }
  int step = 0, phase = kFirst, k_it = 0, trials = 0, nh = 0, head = 0, step_evals = 0;
  int worst = kConverged, iters_total = 0, evals_total = 0, grads_total = 0;
  double E = 0.0, alpha = 1.0, gd = 0.0, gamma = 1.0, rn_x = 0.0;
  const double rstall = kStallFactor * c.rnorm_floor();
  const int max_evals = 4 * A.max_iter + kLsMax;
  c.setup(true);
  if (!active) phase = kDone;
  LpHot h;

  while (__any_sync(kFull, phase != kDone)) {
    const double* tau = A.tau ? A.tau + (int64_t)min(step, A.n_steps - 1) * D : nullptr;
    const double Et = c.gsum(c.primal(tau, h));
    const bool live = phase != kDone;
    if (live) {
      ++evals_total;
      ++step_evals;
    }
    const bool first = live && phase == kFirst;
    const bool trial = live && phase == kTrial;
    const bool need_g = first || (trial && isfinite(Et) &&
                                  (Et <= E + kLsEps * fabs(E) || Et <= E + kLsC1 * alpha * gd));
    if (need_g) ++grads_total;
    if (S == 1) {
      if (need_g) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if (k < nd) sm[L.gt + k] = sm[L.rt + k];
      }
    } else if (__any_sync(kFull, need_g)) {
      c.tangent(h, L.rt, L.gt, 2.0);
    }

    // (1) line-search test at xt = x + alpha d: Armijo or approximate Wolfe
    bool ok = false;
    if (__any_sync(kFull, trial)) {
      double gtd = 0.0, bad = 0.0;
      if (trial && need_g) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if (k < nd) {
            const double gv = sm[L.gt + k];
            if (!isfinite(gv)) bad = 1.0;
            gtd = fma(gv, sm[L.d + k], gtd);
          }
      }
      bad = c.gsum(bad);
      gtd = c.gsum(gtd);
      if (trial && bad == 0.0 && isfinite(Et)) {
        const bool armijo = Et <= E + kLsC1 * alpha * gd;
        const bool approx = (Et <= E + kLsEps * fabs(E)) && (gtd <= (1.0 - 2.0 * kLsDelta) * fabs(gd));
        ok = armijo || approx;
      }
    }
    int fin_st = -1;
    if (trial && !ok) {
      if (step_evals >= max_evals) fin_st = kMaxIter;
      else if (++trials >= kLsMax) fin_st = rn_x <= rstall ? kStalled : kLsFail;
      else alpha *= 0.5;
    }
    const bool back = trial && !ok && fin_st < 0;
    const bool acc = first || ok;

    // (2) accepted groups take (xt, gt, rt) and form the curvature pair s,
    // y (s into rt, y into gt and d); backtracking groups move xt.
    double sy = 0.0, ss = 0.0, yy = 0.0, rr = 0.0, badg = 0.0;
    if (__any_sync(kFull, acc || back)) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (k < nd) {
          if (acc) {
            const double xv = sm[L.xt + k], gv = sm[L.gt + k], rv = sm[L.rt + k];
            if (ok) {
              const double s_ = xv - sm[L.x + k], y_ = gv - sm[L.g + k];
              sy = fma(s_, y_, sy);
              ss = fma(s_, s_, ss);
              yy = fma(y_, y_, yy);
              sm[L.rt + k] = s_;
              sm[L.gt + k] = y_;
              sm[L.d + k] = y_;
            }
            sm[L.x + k] = xv;
            sm[L.g + k] = gv;
            sm[L.r + k] = rv;
            rr = fma(rv, rv, rr);
            if (!isfinite(gv)) badg = 1.0;
          } else if (back) {
            sm[L.xt + k] = fma(alpha, sm[L.d + k], sm[L.x + k]);
          }
        }
      }
      sy = c.gsum(sy);
      ss = c.gsum(ss);
      yy = c.gsum(yy);
      rr = c.gsum(rr);
      badg = c.gsum(badg);
    }

    // (3) curvature pair into the ring: rho = 1/s^T y, gamma = s^T y / y^T P y
    const bool pair = ok && m > 0 && sy > kCurvEps * sqrt(ss) * sqrt(yy);
    if (__any_sync(kFull, pair)) {
      c.precond(L.d, pair);
      double yPy = 0.0;
      if (pair) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if (k < nd) {
            const double yv = sm[L.gt + k];
            yPy = fma(yv, sm[L.d + k], yPy);
            sm[L.sh + 3 * head + k] = sm[L.rt + k];
            sm[L.yh + 3 * head + k] = yv;
          }
      }
      yPy = c.gsum(yPy);
      if (pair) {
        sm[L.rho + head] = 1.0 / sy;
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
        k_it = 0;
        nh = 0;
        head = 0;
        gamma = 1.0;
      } else {
        ++k_it;
        ++iters_total;
      }
      if (badg != 0.0 || !isfinite(E) || !isfinite(rr)) fin_st = kNonFinite;
      else if (sqrt(rr) < A.tol) fin_st = kConverged;
      else if (k_it >= A.max_iter || step_evals >= max_evals) fin_st = kMaxIter;
      else start = true;
    }

    // (5) steps that end: state shift, trajectory, logs; the next step's setup
    const bool fin = fin_st >= 0;
    if (__any_sync(kFull, fin)) {
      if (fin) {
        worst = status_worse(worst, fin_st);
        step_evals = 0;
        if (head_lane) {
          const int64_t o = (int64_t)step * A.n_inst + B.inst_off + c.b;
          if (A.step_status) A.step_status[o] = fin_st;
          if (A.step_rnorm) A.step_rnorm[o] = rn_x;
        }
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double xv = sm[L.x + k];
        const double xs = c.from_stage(xv, S - 1);
        const double xp = (S == 1) ? sm[L.qc + k] : c.from_stage(xv, S - 2);
        if (fin && k < nd) {
          sm[L.qp + k] = xp;
          sm[L.qc + k] = xs;
          if (c.i == 0) {
            if (A.traj_cur) A.traj_cur[(int64_t)step * D + c.gdof(k)] = xs;
            if (A.traj_prev) A.traj_prev[(int64_t)step * D + c.gdof(k)] = xp;
          }
          if (A.q_stages_out && step == A.n_steps - 1) A.q_stages_out[c.gstage(k)] = xv;
          if (A.stages_traj) A.stages_traj[(int64_t)step * S * D + c.gstage(k)] = xv;
        }
      }
      bool next = false;
      if (fin) {
        ++step;
        next = step < A.n_steps;
        phase = next ? kFirst : kDone;
      }
      if (__any_sync(kFull, next)) c.setup(next);
    }

    // (6) two-loop recursion with H0 = gamma P for the groups that start an
    // iteration; a non-descent direction falls back to -P g, then to -g.
    if (__any_sync(kFull, start)) {
      const int nh_w = __reduce_max_sync(kFull, start ? nh : 0);
      if (start) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if (k < nd) sm[L.d + k] = -sm[L.g + k];
      }
      auto slot = [&](int t) { return (head - 1 - t + 2 * m) % m; };
      double al[kMaxHistory];
      for (int t = 0; t < nh_w; ++t) {
        const int j = slot(t);
        const double a = sm[L.rho + j] * c.gdot(L.sh + 3 * j, L.d);
        al[t] = a;
        if (start && t < nh) {
#pragma unroll
          for (int k = 0; k < 3; ++k)
            if (k < nd) sm[L.d + k] = fma(-a, sm[L.yh + 3 * j + k], sm[L.d + k]);
        }
      }
      c.precond(L.d, start);
      if (start) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if (k < nd) sm[L.d + k] = gamma * sm[L.d + k];
      }
      for (int t = nh_w - 1; t >= 0; --t) {
        const int j = slot(t);
        const double bta = sm[L.rho + j] * c.gdot(L.yh + 3 * j, L.d);
        if (start && t < nh) {
#pragma unroll
          for (int k = 0; k < 3; ++k)
            if (k < nd) sm[L.d + k] = fma(al[t] - bta, sm[L.sh + 3 * j + k], sm[L.d + k]);
        }
      }
      const double gd0 = c.gdot(L.g, L.d);
      if (start) gd = gd0;
      const bool reset = start && !(gd < 0.0);
      if (__any_sync(kFull, reset)) {
        if (reset) {
          nh = 0;
          gamma = 1.0;
#pragma unroll
          for (int k = 0; k < 3; ++k)
            if (k < nd) sm[L.d + k] = -sm[L.g + k];
        }
        c.precond(L.d, reset);
        const double gd1 = c.gdot(L.g, L.d);
        if (reset) gd = gd1;
        const bool sd = reset && !(gd < 0.0);
        if (__any_sync(kFull, sd)) {
          if (sd) {
#pragma unroll
            for (int k = 0; k < 3; ++k)
              if (k < nd) sm[L.d + k] = -sm[L.g + k];
          }
          const double gd2 = c.gdot(L.g, L.d);
          if (sd) gd = gd2;
        }
      }
      if (start) {
        alpha = 1.0;
        trials = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if (k < nd) sm[L.xt + k] = sm[L.x + k] + sm[L.d + k];
        phase = kTrial;
      }
    }
  }
  if (active) {
    if (head_lane) {
      if (A.status) A.status[B.inst_off + c.b] = worst;
      if (A.iters) A.iters[B.inst_off + c.b] = iters_total;
      if (A.evals) A.evals[B.inst_off + c.b] = evals_total;
      if (A.grads) A.grads[B.inst_off + c.b] = grads_total;
    }
    if (c.i == 0) {
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (k < nd) {
          if (A.q_prev_out) A.q_prev_out[c.gdof(k)] = sm[L.qp + k];
          if (A.q_cur_out) A.q_cur_out[c.gdof(k)] = sm[L.qc + k];
        }
    }
  }
}

// A link-mapped bucket inside the mixed rollout kernel (a call keeps the
// other solvers' register allocation apart).
template <int S>
__device__ __noinline__ void rollout_lp(const LaunchArgs& A, const Bucket& B) {
  rollout_lp_body<S>(A, B);
}

// The rollout with every bucket in the link mapping (the body inlined).
template <int S>
__global__ void __launch_bounds__(128) k_rollout_lp(const __grid_constant__ LaunchArgs A) {
  rollout_lp_body<S>(A, A.bk[find_bucket(A)]);
}

}  // namespace pbad
