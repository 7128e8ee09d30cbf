// Device-side building blocks of the position-based articulated dynamics
// (PBAD) hot path: joint rotations, forward kinematics, the per-link seeds of
// Eq. EQ / Eq. HOC, world-frame wrench accumulation (Algorithm DERIV in world
// coordinates) and the tangent-over-adjoint sweep that gives the gradient of
// Eq. EQHOC in O(N).
//
// Execution model: a group of S lanes of one warp owns one instance; lane i
// of the group owns collocation stage i. Every lane walks the link tree
// sequentially; the stages meet only where Eq. HOC couples them (the second
// derivative of the collocation polynomial), through warp shuffles.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pbad {

constexpr int kMaxStages = 5;
constexpr int kMaxHistory = 16;

// Per-lane array in a warp-blocked workspace: element k of lane l of warp w
// lives at base[(w * per_lane + k) * 32 + l], so that the lanes of a warp
// touch consecutive words and each warp's working set is contiguous.
struct Lane {
  static constexpr int kStride = 32;  // lanes per warp block
  double* p;
  __device__ __forceinline__ double& operator[](int64_t k) const { return p[k * kStride]; }
};

// One bucket of instances that share a topology (a "model").
struct Bucket {
  int N, n, count;       // links, DOFs, instances
  const int* parent;     // [N]
  const int* jtype;      // [N] 0 hinge, 1 ball
  const int* dof;        // [N] first DOF of each joint
  const int* rest_eye;   // [N] 1 if every instance's rest rotation is the identity
  const int* sub_end;    // [N] link l's subtree is l .. sub_end[l] - 1 (N where not contiguous)
  const double* axis;    // [N][3] hinge axes (joint frame)
  const double* mm;      // [N][10][count] mass moments (SoA over instances)
  const double* rest;    // [N][12][count] rest transforms (SoA over instances)
  double g[3];           // gravity
  int64_t inst_off;      // first instance of the bucket in the batch
  int64_t dof_off;       // offset of the bucket's block in DOF-packed arrays
  double* ws;            // lane workspace
  int64_t ws_lane;       // doubles per lane in the workspace (its layout's total)
  int block_begin;       // first block of the launch that serves this bucket
  int solver;            // 0 L-BFGS, 1 Newton, 2 L-BFGS with the binary32 direction
  // instance queue (L-BFGS rollouts): the launch's groups start on instances
  // 0 .. first_dynamic - 1; a group that finishes its instance takes
  // first_dynamic + atomicAdd(queue, 1) while that is below count
  int* queue;            // device counter, zeroed before the launch (null = no queue)
  int first_dynamic;
  int chain;             // 1 if parent[l] == l - 1 for every link (serial chain)
  int cta;               // Newton: warps per instance (1, or kNewtonCtaWarps for large S n)
  int split;             // Newton, one warp per instance, S >= 2: residual passes at trial
                         // points spread over the warp's replicas (Ctx::primal_split)
  int lp;                // L-BFGS: 1 if the bucket runs the link mapping (one lane per stage and link)
  int axial;             // 1 if every mass moment has Sxy = Sxz = Syz = mcx = mcy = 0
  double* dense;         // per-instance dense Newton/adjoint storage (or null)
  int64_t dense_stride;  // doubles per instance in `dense`
  double drag;           // drag coefficient c of Q_drag (Section 6.2), 0 = none
  int tk;                // 1 if the lane workspace holds T(q_cur) (one-stage drag / contact)
  // penalty contact of Eq. FRI (one stage): points grouped by link,
  // c_off[l]..c_off[l+1] index c_pt[3k..3k+2] (link frame); ground z < c_z0
  int n_contact;
  const int* c_off;      // [N + 1]
  const double* c_pt;    // [n_contact][3]
  double c_z0, c_d1, c_d2;
};

// World position of a body point p (link frame) under the 3x4 transform T.
__device__ __forceinline__ void body_point(const double* T, const double* p, double* P) {
#pragma unroll
  for (int r = 0; r < 3; ++r) P[r] = fma(T[4 * r], p[0], fma(T[4 * r + 1], p[1], fma(T[4 * r + 2], p[2], T[4 * r + 3])));
}

// Penalty contact of one point (Eq. FRI against the ground z < z0): at world
// position P (unknown step end) and Pk (its position at q_k), Q, f = dQ/dP,
// H = d2Q/dP2 and Hk = d2Q/dP dPk (3x3 row-major, rows = components of f).
// Returns false (and touches nothing) when the point is not in the ground.
__device__ __forceinline__ bool ground_contact(const double* P, const double* Pk, double z0,
                                               double D1, double D2, double dt, double* Q,
                                               double* f, double* H, double* Hk) {
  const double d = z0 - P[2];
  if (!(d > 0.0)) return false;
  const double idt = 1.0 / dt;
  const double vx = (P[0] - Pk[0]) * idt, vy = (P[1] - Pk[1]) * idt;
  const double s = fma(vx, vx, vy * vy);
  const double d2 = d * d;
  *Q = d2 * fma(D2, s, D1);
  f[0] = 2.0 * D2 * d2 * vx * idt;
  f[1] = 2.0 * D2 * d2 * vy * idt;
  f[2] = -2.0 * d * fma(D2, s, D1);
  const double hxx = 2.0 * D2 * d2 * idt * idt;
  const double hxz = -4.0 * D2 * d * vx * idt, hyz = -4.0 * D2 * d * vy * idt;
  H[0] = hxx; H[1] = 0.0; H[2] = hxz;
  H[3] = 0.0; H[4] = hxx; H[5] = hyz;
  H[6] = hxz; H[7] = hyz; H[8] = 2.0 * fma(D2, s, D1);
  Hk[0] = -hxx; Hk[1] = 0.0; Hk[2] = 0.0;
  Hk[3] = 0.0; Hk[4] = -hxx; Hk[5] = 0.0;
  Hk[6] = -hxz; Hk[7] = -hyz; Hk[8] = 0.0;
  return true;
}

// Collocation constants of one launch (all in units of 1/dt^2 already).
struct Colloc {
  int S;
  double dt;
  double nodes[kMaxStages + 2];
  double Wk[kMaxStages][2];           // weights of the two known nodes
  double Wu[kMaxStages][kMaxStages];  // Wu[i][j]: residual stage i, unknown j
  double Ps[kMaxStages][kMaxStages];  // stage block of the L-BFGS H0
  // velocity weights of the drag force (V / dt^2 with V the first-derivative
  // weights; one stage: the backward difference [0, -1, 1])
  double Vk[kMaxStages][2];
  double Vu[kMaxStages][kMaxStages];
};

// ---------------------------------------------------------------- 3x4 math
struct M34 {
  double a[12];
};

__device__ __forceinline__ void compose(const double* A, const double* B, double* C) {
  // C = A * B for affine 3x4 matrices (implicit bottom row 0 0 0 1)
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const double a0 = A[4 * r], a1 = A[4 * r + 1], a2 = A[4 * r + 2], a3 = A[4 * r + 3];
#pragma unroll
    for (int c = 0; c < 3; ++c) C[4 * r + c] = fma(a0, B[c], fma(a1, B[4 + c], a2 * B[8 + c]));
    C[4 * r + 3] = fma(a0, B[3], fma(a1, B[7], fma(a2, B[11], a3)));
  }
}

__device__ __forceinline__ void cross(const double* a, const double* b, double* c) {
  c[0] = fma(a[1], b[2], -a[2] * b[1]);
  c[1] = fma(a[2], b[0], -a[0] * b[2]);
  c[2] = fma(a[0], b[1], -a[1] * b[0]);
}
__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
}

// Joint types: 0 hinge (1 DOF), 1 ball (3, exponential map), 2 translation
// (3 prismatic coordinates along the joint frame's axes; with a ball joint on
// a child at the same origin it forms a free 6-DOF root).
constexpr int kHinge = 0, kBall = 1, kTranslation = 2;

// World twist (angular; linear at the world origin) of a unit rate of a DOF
// with world axis w at origin o: rotation (w, o x w), translation (0, w).
__device__ __forceinline__ void add_twist(int jt, const double* o, const double* w, double vk,
                                          double* V) {
  if (jt == kTranslation) {
#pragma unroll
    for (int c = 0; c < 3; ++c) V[3 + c] = fma(vk, w[c], V[3 + c]);
  } else {
    double ow[3];
    cross(o, w, ow);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      V[c] = fma(vk, w[c], V[c]);
      V[3 + c] = fma(vk, ow[c], V[3 + c]);
    }
  }
}

// R = c0 I + c1 [v]x + c2 v v^T (Rodrigues form shared by hinges and the
// exponential map).
__device__ __forceinline__ void rodrigues(const double* v, double c0, double c1, double c2, double* R) {
  R[0] = fma(c2, v[0] * v[0], c0);
  R[1] = fma(c2, v[0] * v[1], -c1 * v[2]);
  R[2] = fma(c2, v[0] * v[2], c1 * v[1]);
  R[3] = fma(c2, v[1] * v[0], c1 * v[2]);
  R[4] = fma(c2, v[1] * v[1], c0);
  R[5] = fma(c2, v[1] * v[2], -c1 * v[0]);
  R[6] = fma(c2, v[2] * v[0], -c1 * v[1]);
  R[7] = fma(c2, v[2] * v[1], c1 * v[0]);
  R[8] = fma(c2, v[2] * v[2], c0);
}

// Scalar functions of x = |theta|^2 for the exponential map:
//   b(x) = (1 - cos phi)/x, h(x) = (phi - sin phi)/phi^3, cos phi and
//   a = sin(phi)/phi, and with DERIV the x-derivatives of b and h (the hot
//   passes take those from exp_coef_deriv instead, when a tangent pass needs
//   them). Power series below x = 1 (terms through x^8; the remainders are
//   below 1e-17), closed forms above.
struct ExpCoef {
  double c, a, b, h, db, dh;
};
template <bool DERIV = true>
__device__ __forceinline__ ExpCoef exp_coef(double x) {
  ExpCoef e;
  e.db = 0.0;
  e.dh = 0.0;
  if (x < 1.0) {
    // Horner in x; terms through x^8 (the tables run to x^9)
    // a = sum (-1)^k x^k/(2k+1)!, b = sum (-1)^k x^k/(2k+2)!, h = sum (-1)^k x^k/(2k+3)!
    const double ia[10] = {1.0, -1.0 / 6, 1.0 / 120, -1.0 / 5040, 1.0 / 362880, -1.0 / 39916800,
                           1.0 / 6227020800.0, -1.0 / 1307674368000.0, 1.0 / 355687428096000.0,
                           -1.0 / 121645100408832000.0};
    const double ib[10] = {1.0 / 2, -1.0 / 24, 1.0 / 720, -1.0 / 40320, 1.0 / 3628800,
                           -1.0 / 479001600, 1.0 / 87178291200.0, -1.0 / 20922789888000.0,
                           1.0 / 6402373705728000.0, -1.0 / 2432902008176640000.0};
    const double ih[10] = {1.0 / 6, -1.0 / 120, 1.0 / 5040, -1.0 / 362880, 1.0 / 39916800,
                           -1.0 / 6227020800.0, 1.0 / 1307674368000.0, -1.0 / 355687428096000.0,
                           1.0 / 121645100408832000.0, -1.0 / 51090942171709440000.0};
    double A = ia[8], B = ib[8], H = ih[8], dB = 8 * ib[8], dH = 8 * ih[8];
#pragma unroll
    for (int k = 7; k >= 0; --k) {
      A = fma(A, x, ia[k]);
      B = fma(B, x, ib[k]);
      H = fma(H, x, ih[k]);
    }
    if (DERIV) {
#pragma unroll
      for (int k = 7; k >= 1; --k) {
        dB = fma(dB, x, k * ib[k]);
        dH = fma(dH, x, k * ih[k]);
      }
      e.db = dB;
      e.dh = dH;
    }
    e.a = A;
    e.b = B;
    e.h = H;
    e.c = fma(-B, x, 1.0);  // cos phi = 1 - x b
  } else {
    const double phi = sqrt(x);
    double s, c;
    sincos(phi, &s, &c);
    const double ix = 1.0 / x;
    e.c = c;
    e.a = s / phi;
    e.b = (1.0 - c) * ix;
    e.h = (phi - s) * ix / phi;
    if (DERIV) {
      e.db = (phi * s - 2.0 * (1.0 - c)) * 0.5 * ix * ix;
      e.dh = (3.0 * s - phi * (2.0 + c)) * 0.5 * ix * ix / phi;
    }
  }
  return e;
}

// x-derivatives of b and h at x, from a = sin(phi)/phi and c = cos(phi) as
// exp_coef returns them: the same power series below x = 1, and above it
// db = (x a - 2 (1 - c)) / (2 x^2), dh = (3 a - 2 - c) / (2 x^2) (phi s = x a).
__device__ __forceinline__ void exp_coef_deriv(double x, double a, double c, double* db, double* dh) {
  if (x < 1.0) {
    const double ib[10] = {1.0 / 2, -1.0 / 24, 1.0 / 720, -1.0 / 40320, 1.0 / 3628800,
                           -1.0 / 479001600, 1.0 / 87178291200.0, -1.0 / 20922789888000.0,
                           1.0 / 6402373705728000.0, -1.0 / 2432902008176640000.0};
    const double ih[10] = {1.0 / 6, -1.0 / 120, 1.0 / 5040, -1.0 / 362880, 1.0 / 39916800,
                           -1.0 / 6227020800.0, 1.0 / 1307674368000.0, -1.0 / 355687428096000.0,
                           1.0 / 121645100408832000.0, -1.0 / 51090942171709440000.0};
    double dB = 8 * ib[8], dH = 8 * ih[8];  // terms through x^7 (remainder below 1e-17)
#pragma unroll
    for (int k = 7; k >= 1; --k) {
      dB = fma(dB, x, k * ib[k]);
      dH = fma(dH, x, k * ih[k]);
    }
    *db = dB;
    *dh = dH;
  } else {
    const double h2 = 0.5 / (x * x);
    *db = (x * a - 2.0 * (1.0 - c)) * h2;
    *dh = (3.0 * a - 2.0 - c) * h2;
  }
}

// Joint rotation (and, for balls, the right Jacobian Jr) of one joint.
//   hinge: R = Rot(u, q), world axis w = R_link u
//   ball:  R = exp([theta]x), world axes w_k = R_link Jr(theta) e_k
// ec (optional) receives the exponential-map coefficients (c, a, b, h), for
// the tangent passes at the same configuration.
__device__ __forceinline__ void joint_rotation(int jt, const double* u, const double* q, double* R,
                                               double* Jr, ExpCoef* ec = nullptr) {
  if (jt == 0) {
    double s, c;
    sincos(q[0], &s, &c);
    rodrigues(u, c, s, 1.0 - c, R);
  } else if (jt == 2) {
    // translation joint: no rotation; its three axes are the frame's own
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      R[k] = (k % 4 == 0) ? 1.0 : 0.0;
      if (Jr) Jr[k] = R[k];
    }
  } else {
    const double x = fma(q[0], q[0], fma(q[1], q[1], q[2] * q[2]));
    const ExpCoef e = exp_coef<false>(x);
    if (ec) *ec = e;
    rodrigues(q, e.c, e.a, e.b, R);
    // Jr = (1 - h x) I - b [theta]x + h theta theta^T (null: not wanted)
    if (Jr) rodrigues(q, fma(-e.h, x, 1.0), -e.b, e.h, Jr);
  }
}

// dJr^T u, the derivative of Jr along v contracted with u, without forming
// dJr = -2 (theta.v) b' K - b [v]x + 2 (theta.v) h' K^2 + h ([v]x K + K [v]x)
// (K = [theta]x, K^2 = theta theta^T - x I, [v]x K + K [v]x = v theta^T +
// theta v^T - 2 (v.theta) I): the transposes act on u as K^T u = u x theta,
// [v]x^T u = u x v, and the symmetric parts directly. cab = (c, a, b, h) of
// the exponential map at th, as cached by the residual pass.
__device__ __forceinline__ void jr_tangent_dot(const double* th, const double* v, const double* cab,
                                               const double* u, double* z) {
  const double x = fma(th[0], th[0], fma(th[1], th[1], th[2] * th[2]));
  double db, dh;
  exp_coef_deriv(x, cab[1], cab[0], &db, &dh);
  const double b = cab[2], h = cab[3];
  const double tv = dot3(th, v), tu = dot3(th, u), vu = dot3(v, u);
  const double cb = -2.0 * tv * db, ch = 2.0 * tv * dh;
  double ut[3], uv[3];
  cross(u, th, ut);
  cross(u, v, uv);
  // ch (theta tu - x u) + h (v tu + theta vu - 2 tv u)
  const double cu = -fma(ch, x, 2.0 * h * tv);
  const double ct = fma(ch, tu, h * vu);
  const double cv = h * tu;
#pragma unroll
  for (int r = 0; r < 3; ++r)
    z[r] = fma(cb, ut[r], fma(-b, uv[r], fma(ct, th[r], fma(cv, v[r], cu * u[r]))));
}

// Mass moment M (4x4 symmetric) of link l for instance b.
struct MassMoment {
  double s[10];  // Sxx Sxy Sxz Syy Syz Szz mcx mcy mcz m
  __device__ __forceinline__ double at(int r, int c) const {
    // index map of the symmetric 4x4
    const int idx[16] = {0, 1, 2, 6, 1, 3, 4, 7, 2, 4, 5, 8, 6, 7, 8, 9};
    return s[idx[4 * r + c]];
  }
};

// Y = A * M for a 3x4 A (the fourth column of M's row 3 is m).
__device__ __forceinline__ void mul_mass(const double* A, const MassMoment& M, double* Y) {
  const double* s = M.s;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const double a0 = A[4 * r], a1 = A[4 * r + 1], a2 = A[4 * r + 2], a3 = A[4 * r + 3];
    Y[4 * r + 0] = fma(a0, s[0], fma(a1, s[1], fma(a2, s[2], a3 * s[6])));
    Y[4 * r + 1] = fma(a0, s[1], fma(a1, s[3], fma(a2, s[4], a3 * s[7])));
    Y[4 * r + 2] = fma(a0, s[2], fma(a1, s[4], fma(a2, s[5], a3 * s[8])));
    Y[4 * r + 3] = fma(a0, s[6], fma(a1, s[7], fma(a2, s[8], a3 * s[9])));
  }
}

// The same product for a mass moment with Sxy = Sxz = Syz = mcx = mcy = 0
// (symmetric about the frame's z axis): the terms of mul_mass that remain, in
// its order, so the results are bitwise equal.
__device__ __forceinline__ void mul_mass_axial(const double* A, const MassMoment& M, double* Y) {
  const double* s = M.s;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const double a0 = A[4 * r], a1 = A[4 * r + 1], a2 = A[4 * r + 2], a3 = A[4 * r + 3];
    Y[4 * r + 0] = a0 * s[0];
    Y[4 * r + 1] = a1 * s[3];
    Y[4 * r + 2] = fma(a2, s[5], a3 * s[8]);
    Y[4 * r + 3] = fma(a2, s[8], a3 * s[9]);
  }
}

// World wrench (moment about the world origin, force) of a 3x4 seed G at
// transform T: m = ax(G_R R^T) + t x f, f = G_t, where ax(Y) = (Y21 - Y12,
// Y02 - Y20, Y10 - Y01). Derivation: G : (S T) = w.(m - o x f) for a unit
// twist S about an axis w through o.
__device__ __forceinline__ void wrench(const double* G, const double* T, double* w6) {
  // Y_rk = G_R[r] . R[k]
  auto Y = [&](int r, int k) {
    return fma(G[4 * r], T[4 * k], fma(G[4 * r + 1], T[4 * k + 1], G[4 * r + 2] * T[4 * k + 2]));
  };
  const double f[3] = {G[3], G[7], G[11]};
  const double t[3] = {T[3], T[7], T[11]};
  double tf[3];
  cross(t, f, tf);
  w6[0] = Y(2, 1) - Y(1, 2) + tf[0];
  w6[1] = Y(0, 2) - Y(2, 0) + tf[1];
  w6[2] = Y(1, 0) - Y(0, 1) + tf[2];
  w6[3] = f[0];
  w6[4] = f[1];
  w6[5] = f[2];
}

// Tangent of the wrench: d/de of wrench(G + e Gd, T + e Td).
__device__ __forceinline__ void wrench_tangent(const double* G, const double* Gd, const double* T,
                                               const double* Td, double* w6) {
  auto Y = [&](const double* A, const double* B, int r, int k) {
    return fma(A[4 * r], B[4 * k], fma(A[4 * r + 1], B[4 * k + 1], A[4 * r + 2] * B[4 * k + 2]));
  };
  auto Yd = [&](int r, int k) { return Y(Gd, T, r, k) + Y(G, Td, r, k); };
  const double f[3] = {G[3], G[7], G[11]}, fd[3] = {Gd[3], Gd[7], Gd[11]};
  const double t[3] = {T[3], T[7], T[11]}, td[3] = {Td[3], Td[7], Td[11]};
  double a1[3], a2[3];
  cross(td, f, a1);
  cross(t, fd, a2);
  w6[0] = Yd(2, 1) - Yd(1, 2) + a1[0] + a2[0];
  w6[1] = Yd(0, 2) - Yd(2, 0) + a1[1] + a2[1];
  w6[2] = Yd(1, 0) - Yd(0, 1) + a1[2] + a2[2];
  w6[3] = fd[0];
  w6[4] = fd[1];
  w6[5] = fd[2];
}

// ------------------------------------------------------- group primitives
template <int S>
struct Group {
  int lane, base, stage;
  unsigned mask;
  __device__ __forceinline__ Group() {
    lane = threadIdx.x & 31;
    stage = lane % S;
    base = lane - stage;
    mask = (S == 32) ? 0xffffffffu : (((1u << S) - 1u) << base);
  }
  // Source lane of stage j. The lanes past the last full group of a warp
  // (32 % S of them) form a short group; their sources are clamped to lane
  // 31 so that every shuffle reads a lane inside the caller's mask.
  __device__ __forceinline__ int src(int j) const { return min(base + j, 31); }
  // value of lane base+j (all lanes of the warp must call with full mask)
  __device__ __forceinline__ double from_full(double v, int j) const {
    return __shfl_sync(0xffffffffu, v, src(j));
  }
  __device__ __forceinline__ double from(double v, int j) const {
    return __shfl_sync(mask, v, src(j));
  }
  // group sum in a fixed order: identical bits on every lane of the group
  __device__ __forceinline__ double sum(double v) const {
    if (S == 1) return v;
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < S; ++j) s += __shfl_sync(mask, v, src(j));
    return s;
  }
  __device__ __forceinline__ float sum(float v) const {
    if (S == 1) return v;
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < S; ++j) s += __shfl_sync(mask, v, src(j));
    return s;
  }
};

}  // namespace pbad
