/*
 * CPU oracle for position-based articulated dynamics (PBAD), Pan & Manocha,
 * "Time Integrating Articulated Body Dynamics Using Position-Based Collocation
 * Methods" (arXiv 1709.04145).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, FP64 restatement of
 * the method that the CUDA path is checked against. Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it. It shares
 * no code, header, table or helper with the CUDA library.
 *
 * Conventions (the paper is silent on them; the same readings bind the CUDA
 * path):
 *   - links l = 0..N-1, parent[l] < l or -1 (world); link frame origin at its
 *     joint; T_l = T_parent(l) * X_l * Jm_l(q_l) with X_l the rest transform
 *     (3x4 row-major) and Jm_l the joint rotation (hinge: Rodrigues about a
 *     unit axis; ball: exponential map of a 3-vector; translation: Jm =
 *     [I | q], three prismatic coordinates along the frame axes - with a ball
 *     joint on a child at the same origin it gives the free 6-DOF root of
 *     Section 6.2's swimmer and spider).
 *   - mass moment M_l = int rho [p;1][p;1]^T dp over the link (4x4 symmetric),
 *     given by 10 numbers Sxx,Sxy,Sxz,Syy,Syz,Szz,mcx,mcy,mcz,m.
 *   - gravity potential Q = -rho g.P; generalised joint torques tau do work
 *     tau.q (Section 4: f in Eq. HOC; tau is added as a generalised force).
 *   - S = K-1 unknown stages per step, K the collocation order of Section 4.1.
 *
 * Nothing here is blocked, fused or reordered beyond the product rule written
 * out with cached partial products; every derivative is taken by the chain
 * rule along the root-to-link path (the brute-force counterpart of
 * Algorithm DERIV / HESS1 / HESS2).
 *
 * Parity is pinned (in the test suite) by central finite differences, closed
 * forms (rod mass moments, pendulum period, Legendre roots), quadrature of the
 * body integrals, rest invariance, a Newton-Euler reference integrator and
 * agreement between the two optimisers.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* model                                                               */
/* ------------------------------------------------------------------ */

typedef struct {
  int n_links, n_dof;
  int *parent, *jtype, *dof_off, *ndof;
  double *axis; /* [N][3] */
  double *mm;   /* [N][10] */
  double *rest; /* [N][12] */
  double g[3];
  double drag;   /* drag coefficient c of Q_drag (0 = none), see om_model_set_drag */
  /* penalty contact of Eq. FRI against the ground plane z = c_z0 */
  int n_contact;
  int *c_link;      /* [n_contact] */
  double *c_point;  /* [n_contact][3] in the link frame */
  double c_z0, c_d1, c_d2;
  int *path_len; /* number of joints from the root to l, inclusive */
  int *path;     /* [N][N]: path[l*N + k] = k-th joint on the root->l path */
  int fast;      /* 1: L-BFGS evaluates with om_eval_fast (O(N)), see there */
} om_model;

void om_model_free(void *p) {
  om_model *m = (om_model *)p;
  if (!m) return;
  free(m->parent); free(m->jtype); free(m->dof_off); free(m->ndof);
  free(m->c_link); free(m->c_point);
  free(m->axis); free(m->mm); free(m->rest); free(m->path_len); free(m->path);
  free(m);
}

/* Returns NULL on a malformed tree (parent[l] >= l) or unknown joint type. */
void *om_model_new(int n_links, const int *parent, const int *jtype,
                   const double *axis, const double *mm, const double *rest,
                   const double *g) {
  if (n_links <= 0 || n_links > 4096) return NULL;
  om_model *m = (om_model *)calloc(1, sizeof(om_model));
  int N = n_links;
  m->n_links = N;
  m->parent = (int *)malloc(sizeof(int) * N);
  m->jtype = (int *)malloc(sizeof(int) * N);
  m->dof_off = (int *)malloc(sizeof(int) * N);
  m->ndof = (int *)malloc(sizeof(int) * N);
  m->axis = (double *)malloc(sizeof(double) * 3 * N);
  m->mm = (double *)malloc(sizeof(double) * 10 * N);
  m->rest = (double *)malloc(sizeof(double) * 12 * N);
  m->path_len = (int *)malloc(sizeof(int) * N);
  m->path = (int *)malloc(sizeof(int) * N * N);
  int off = 0;
  for (int l = 0; l < N; ++l) {
    if (parent[l] >= l || parent[l] < -1 || jtype[l] < 0 || jtype[l] > 2) {
      om_model_free(m);
      return NULL;
    }
    m->parent[l] = parent[l];
    m->jtype[l] = jtype[l];
    m->ndof[l] = jtype[l] == 0 ? 1 : 3;
    m->dof_off[l] = off;
    off += m->ndof[l];
    for (int k = 0; k < 3; ++k) m->axis[3 * l + k] = axis[3 * l + k];
    for (int k = 0; k < 10; ++k) m->mm[10 * l + k] = mm[10 * l + k];
    for (int k = 0; k < 12; ++k) m->rest[12 * l + k] = rest[12 * l + k];
    /* root -> l path */
    int tmp[4096], len = 0;
    for (int a = l; a >= 0; a = parent[a]) tmp[len++] = a;
    m->path_len[l] = len;
    for (int k = 0; k < len; ++k) m->path[l * N + k] = tmp[len - 1 - k];
  }
  m->n_dof = off;
  for (int k = 0; k < 3; ++k) m->g[k] = g[k];
  return m;
}

int om_n_dof(void *p) { return ((om_model *)p)->n_dof; }

/* Drag potential of Section 6.2 (swimmer): Q_drag = D |(P(q_{k+1}) - P(q_k))/dt|^2
 * integrated over the body. With the mass-weighted moments M_l used here the
 * coefficient is per unit mass, c = D / rho:
 *   int Q_drag = c / dt^2 * tr((T_{k+1} - T_k) M (T_{k+1} - T_k)^T)
 * (Appendix A's I-expansion of Q_drag), whose gradient is the force density
 * -2 c rho v / dt with v = (P_{k+1} - P_k)/dt. For S >= 2 stages the same force
 * law enters every stage residual of Eq. HOC with v the velocity of the
 * collocation polynomial at the stage node (first-derivative weights of
 * om_colloc_vel). */
void om_model_set_drag(void *p, double c) { ((om_model *)p)->drag = c; }

/* Penalty frictional contact of Eq. FRI (Section 6.2, spider) against the
 * ground: obstacle = half-space z < z0, penetration depth d(P) = max(0, z0 -
 * P_z), tangential projection = the xy components. Over a set of body
 * points (the integral replaced by a sum over discrete contact points):
 *   Q_contact = sum_p D1 d(P_p)^2 + D2 d(P_p)^2 |Pi (P_p(q_{k+1}) - P_p(q_k))/dt|^2
 * with P_p = T_l(q) [p; 1]. Added to Eq. EQ (one stage); the oracle does not
 * define it for S >= 2. Returns -1 on a bad link index. */
int om_model_set_contact(void *p, int n, const int *link, const double *point, double z0,
                         double d1, double d2) {
  om_model *m = (om_model *)p;
  for (int k = 0; k < n; ++k)
    if (link[k] < 0 || link[k] >= m->n_links) return -1;
  free(m->c_link); free(m->c_point);
  m->c_link = NULL; m->c_point = NULL;
  m->n_contact = n;
  if (n > 0) {
    m->c_link = (int *)malloc(sizeof(int) * n);
    m->c_point = (double *)malloc(sizeof(double) * 3 * n);
    for (int k = 0; k < n; ++k) {
      m->c_link[k] = link[k];
      for (int c = 0; c < 3; ++c) m->c_point[3 * k + c] = point[3 * k + c];
    }
  }
  m->c_z0 = z0; m->c_d1 = d1; m->c_d2 = d2;
  return 0;
}

/* One contact point at world position P (from q_{k+1}) and Pk (from q_k):
 * Q, f = dQ/dP, H = d2Q/dP2 and Hk = d2Q/dP dPk (3x3 row-major, rows = the
 * components of f). Returns 0 when the point is outside the obstacle. */
static int contact_point(const om_model *m, double dt, const double *P, const double *Pk,
                         double *Q, double *f, double *H, double *Hk) {
  double d = m->c_z0 - P[2];
  if (!(d > 0.0)) return 0;
  double D1 = m->c_d1, D2 = m->c_d2;
  double vx = (P[0] - Pk[0]) / dt, vy = (P[1] - Pk[1]) / dt;
  double s = vx * vx + vy * vy;
  *Q = D1 * d * d + D2 * d * d * s;
  f[0] = 2 * D2 * d * d * vx / dt;
  f[1] = 2 * D2 * d * d * vy / dt;
  f[2] = -2 * d * (D1 + D2 * s);
  for (int k = 0; k < 9; ++k) { H[k] = 0; Hk[k] = 0; }
  H[0] = H[4] = 2 * D2 * d * d / (dt * dt);
  H[2] = H[6] = -4 * D2 * d * vx / dt;   /* d f_x/d P_z, d f_z/d P_x */
  H[5] = H[7] = -4 * D2 * d * vy / dt;
  H[8] = 2 * (D1 + D2 * s);
  Hk[0] = Hk[4] = -2 * D2 * d * d / (dt * dt);
  Hk[6] = 4 * D2 * d * vx / dt;          /* d f_z/d Pk_x */
  Hk[7] = 4 * D2 * d * vy / dt;
  return 1;
}

/* body point of link l: P = T_l [p; 1] (T row-major 4x4) */
static void point_world(const double *T, const double *pt, double *P) {
  for (int r = 0; r < 3; ++r)
    P[r] = T[4 * r] * pt[0] + T[4 * r + 1] * pt[1] + T[4 * r + 2] * pt[2] + T[4 * r + 3];
}

/* ------------------------------------------------------------------ */
/* small dense helpers (4x4 row-major homogeneous, 3x3 row-major)      */
/* ------------------------------------------------------------------ */

static void m4_mul(const double *A, const double *B, double *C) {
  double t[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0;
      for (int k = 0; k < 4; ++k) s += A[4 * i + k] * B[4 * k + j];
      t[4 * i + j] = s;
    }
  memcpy(C, t, sizeof(t));
}
static void m4_eye(double *A) {
  memset(A, 0, 16 * sizeof(double));
  A[0] = A[5] = A[10] = A[15] = 1.0;
}
static void m3_mul(const double *A, const double *B, double *C) {
  double t[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      t[3 * i + j] = s;
    }
  memcpy(C, t, sizeof(t));
}
static void skew3(const double *v, double *K) {
  K[0] = 0; K[1] = -v[2]; K[2] = v[1];
  K[3] = v[2]; K[4] = 0; K[5] = -v[0];
  K[6] = -v[1]; K[7] = v[0]; K[8] = 0;
}
/* 3x4 rest transform -> 4x4 */
static void rest4(const double *X12, double *X) {
  for (int k = 0; k < 12; ++k) X[k] = X12[k];
  X[12] = X[13] = X[14] = 0; X[15] = 1;
}
/* rotation (or its derivative) -> 4x4 with the given bottom-right entry */
static void rot4(const double *R, double corner, double *J) {
  memset(J, 0, 16 * sizeof(double));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) J[4 * i + j] = R[3 * i + j];
  J[15] = corner;
}
static void mm4(const double *mm, double *M) {
  M[0] = mm[0]; M[1] = mm[1]; M[2] = mm[2]; M[3] = mm[6];
  M[4] = mm[1]; M[5] = mm[3]; M[6] = mm[4]; M[7] = mm[7];
  M[8] = mm[2]; M[9] = mm[4]; M[10] = mm[5]; M[11] = mm[8];
  M[12] = mm[6]; M[13] = mm[7]; M[14] = mm[8]; M[15] = mm[9];
}
/* A : B over the top three rows (the bottom row of every derivative and of
 * every difference of homogeneous transforms is zero). */
static double contract34(const double *A, const double *B) {
  double s = 0;
  for (int k = 0; k < 12; ++k) s += A[k] * B[k];
  return s;
}

/* ------------------------------------------------------------------ */
/* joint rotations and their first/second derivatives                  */
/* ------------------------------------------------------------------ */

/* Coefficient functions of the exponential map R = I + a K + b K^2,
 * K = [theta]x, phi = |theta|, and c = a'/phi, d = b'/phi, e = c'/phi,
 * f = d'/phi. Series (all terms up to phi^24) below phi = 0.5, where the
 * closed forms cancel; closed forms above. */
static void expmap_coeffs(double phi, double *a, double *b, double *c,
                          double *d, double *e, double *f) {
  if (phi < 0.5) {
    double p2 = phi * phi;
    double fact[40];
    fact[0] = 1;
    for (int k = 1; k < 40; ++k) fact[k] = fact[k - 1] * k;
    double A = 0, B = 0, C = 0, D = 0, E = 0, F = 0, pw = 1; /* pw = p2^n */
    for (int n = 0; n <= 12; ++n) {
      double sg = (n % 2) ? -1.0 : 1.0;
      A += sg * pw / fact[2 * n + 1];
      B += sg * pw / fact[2 * n + 2];
      pw *= p2;
    }
    pw = 1; /* p2^(n-1) */
    for (int n = 1; n <= 13; ++n) {
      double sg = (n % 2) ? -1.0 : 1.0;
      C += sg * 2.0 * n * pw / fact[2 * n + 1];
      D += sg * 2.0 * n * pw / fact[2 * n + 2];
      pw *= p2;
    }
    pw = 1; /* p2^(n-2) */
    for (int n = 2; n <= 14; ++n) {
      double sg = (n % 2) ? -1.0 : 1.0;
      E += sg * 2.0 * n * (2.0 * n - 2.0) * pw / fact[2 * n + 1];
      F += sg * 2.0 * n * (2.0 * n - 2.0) * pw / fact[2 * n + 2];
      pw *= p2;
    }
    *a = A; *b = B; *c = C; *d = D; *e = E; *f = F;
  } else {
    double s = sin(phi), co = cos(phi);
    double p2 = phi * phi, p3 = p2 * phi, p4 = p2 * p2, p5 = p4 * phi,
           p6 = p3 * p3;
    *a = s / phi;
    *b = (1 - co) / p2;
    *c = (phi * co - s) / p3;
    *d = (phi * s - 2 * (1 - co)) / p4;
    *e = (3 * s - 3 * phi * co - p2 * s) / p5;
    *f = (p2 * co - 5 * phi * s + 8 * (1 - co)) / p6;
  }
}

/* R(q) of one joint. q points at the joint's own coordinates. */
void om_joint_rot(int type, const double *axis, const double *q, double *R) {
  double I[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, K[9], K2[9];
  if (type == 0) {
    skew3(axis, K);
    m3_mul(K, K, K2);
    double s = sin(q[0]), co = cos(q[0]);
    for (int k = 0; k < 9; ++k) R[k] = I[k] + s * K[k] + (1 - co) * K2[k];
  } else {
    double phi = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    double a, b, c, d, e, f;
    expmap_coeffs(phi, &a, &b, &c, &d, &e, &f);
    skew3(q, K);
    m3_mul(K, K, K2);
    for (int k = 0; k < 9; ++k) R[k] = I[k] + a * K[k] + b * K2[k];
  }
}

/* dR/dq_k (k = local coordinate index). */
void om_joint_drot(int type, const double *axis, const double *q, int k,
                   double *dR) {
  double K[9], K2[9];
  if (type == 0) {
    skew3(axis, K);
    m3_mul(K, K, K2);
    double s = sin(q[0]), co = cos(q[0]);
    for (int i = 0; i < 9; ++i) dR[i] = co * K[i] + s * K2[i];
  } else {
    double phi = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    double a, b, c, d, e, f;
    expmap_coeffs(phi, &a, &b, &c, &d, &e, &f);
    double ek[3] = {0, 0, 0}, Ek[9], EK[9], KE[9];
    ek[k] = 1;
    skew3(q, K);
    m3_mul(K, K, K2);
    skew3(ek, Ek);
    m3_mul(Ek, K, EK);
    m3_mul(K, Ek, KE);
    for (int i = 0; i < 9; ++i)
      dR[i] = c * q[k] * K[i] + a * Ek[i] + d * q[k] * K2[i] +
              b * (EK[i] + KE[i]);
  }
}

/* d2R/dq_k dq_m. */
void om_joint_ddrot(int type, const double *axis, const double *q, int k,
                    int m, double *ddR) {
  double K[9], K2[9];
  if (type == 0) {
    skew3(axis, K);
    m3_mul(K, K, K2);
    double s = sin(q[0]), co = cos(q[0]);
    for (int i = 0; i < 9; ++i) ddR[i] = -s * K[i] + co * K2[i];
  } else {
    double phi = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    double a, b, c, d, e, f;
    expmap_coeffs(phi, &a, &b, &c, &d, &e, &f);
    double ek[3] = {0, 0, 0}, em[3] = {0, 0, 0};
    ek[k] = 1;
    em[m] = 1;
    double Ek[9], Em[9], EkK[9], KEk[9], EmK[9], KEm[9], EkEm[9], EmEk[9];
    skew3(q, K);
    m3_mul(K, K, K2);
    skew3(ek, Ek);
    skew3(em, Em);
    m3_mul(Ek, K, EkK);
    m3_mul(K, Ek, KEk);
    m3_mul(Em, K, EmK);
    m3_mul(K, Em, KEm);
    m3_mul(Ek, Em, EkEm);
    m3_mul(Em, Ek, EmEk);
    double dkm = (k == m) ? 1.0 : 0.0;
    for (int i = 0; i < 9; ++i)
      ddR[i] = e * q[k] * q[m] * K[i] + c * dkm * K[i] + c * q[k] * Em[i] +
               c * q[m] * Ek[i] + f * q[k] * q[m] * K2[i] + d * dkm * K2[i] +
               d * q[k] * (EmK[i] + KEm[i]) + d * q[m] * (EkK[i] + KEk[i]) +
               b * (EkEm[i] + EmEk[i]);
  }
}

/* F_a(q) = X_a * Jm_a(q_a) as a 4x4 homogeneous matrix. */
static void joint_factor(const om_model *m, int a, const double *q, double *F) {
  double X[16], R[9], J[16];
  rest4(m->rest + 12 * a, X);
  if (m->jtype[a] == 2) {
    /* translation: Jm = [I | q] */
    const double *t = q + m->dof_off[a];
    m4_eye(J);
    J[3] = t[0]; J[7] = t[1]; J[11] = t[2];
  } else {
    om_joint_rot(m->jtype[a], m->axis + 3 * a, q + m->dof_off[a], R);
    rot4(R, 1.0, J);
  }
  m4_mul(X, J, F);
}
/* X_a * dJm_a/dq_k (bottom row zero). */
static void joint_factor_d(const om_model *m, int a, const double *q, int k,
                           double *F) {
  double X[16], R[9], J[16];
  rest4(m->rest + 12 * a, X);
  if (m->jtype[a] == 2) {
    /* dJm/dq_k = e_k in the translation column */
    for (int i = 0; i < 16; ++i) J[i] = 0.0;
    J[4 * k + 3] = 1.0;
  } else {
    om_joint_drot(m->jtype[a], m->axis + 3 * a, q + m->dof_off[a], k, R);
    rot4(R, 0.0, J);
  }
  m4_mul(X, J, F);
}
static void joint_factor_dd(const om_model *m, int a, const double *q, int k,
                            int kk, double *F) {
  double X[16], R[9], J[16];
  rest4(m->rest + 12 * a, X);
  if (m->jtype[a] == 2) {
    /* Jm is affine in q: no second derivative */
    for (int i = 0; i < 16; ++i) F[i] = 0.0;
    return;
  }
  om_joint_ddrot(m->jtype[a], m->axis + 3 * a, q + m->dof_off[a], k, kk, R);
  rot4(R, 0.0, J);
  m4_mul(X, J, F);
}

/* ------------------------------------------------------------------ */
/* forward kinematics and its derivatives (Section 5, T^i = T^{i-1}T)   */
/* ------------------------------------------------------------------ */

/* T_l for every link by the explicit product along the root->l path.
 * T: [N][16]. */
void om_fk(void *p, const double *q, double *T) {
  om_model *m = (om_model *)p;
  int N = m->n_links;
  for (int l = 0; l < N; ++l) {
    double P[16], F[16];
    m4_eye(P);
    for (int k = 0; k < m->path_len[l]; ++k) {
      joint_factor(m, m->path[l * N + k], q, F);
      m4_mul(P, F, P);
    }
    memcpy(T + 16 * l, P, sizeof(P));
  }
}

/* Per-link prefix/suffix products along the root->l path:
 * pre[k] = F_1...F_k (pre[0] = I), suf[k] = F_k...F_m (suf[m+1] = I),
 * 1-based over path positions. Arrays sized (m+2)*16. */
static void path_products(const om_model *m, int l, const double *q,
                          double *F, double *pre, double *suf) {
  int N = m->n_links, len = m->path_len[l];
  for (int k = 1; k <= len; ++k) joint_factor(m, m->path[l * N + k - 1], q, F + 16 * k);
  m4_eye(pre);
  for (int k = 1; k <= len; ++k) m4_mul(pre + 16 * (k - 1), F + 16 * k, pre + 16 * k);
  m4_eye(suf + 16 * (len + 1));
  for (int k = len; k >= 1; --k) m4_mul(F + 16 * k, suf + 16 * (k + 1), suf + 16 * k);
}

/* dT_l/dq_d for every DOF d (zero where d is not on the root->l path).
 * dT: [n][16]. */
void om_link_dT(void *p, const double *q, int l, double *dT) {
  om_model *m = (om_model *)p;
  int N = m->n_links, len = m->path_len[l], n = m->n_dof;
  double *F = (double *)malloc(sizeof(double) * 16 * (len + 2));
  double *pre = (double *)malloc(sizeof(double) * 16 * (len + 2));
  double *suf = (double *)malloc(sizeof(double) * 16 * (len + 2));
  path_products(m, l, q, F, pre, suf);
  memset(dT, 0, sizeof(double) * 16 * n);
  for (int s = 1; s <= len; ++s) {
    int a = m->path[l * N + s - 1];
    for (int k = 0; k < m->ndof[a]; ++k) {
      double Fd[16], t[16];
      joint_factor_d(m, a, q, k, Fd);
      m4_mul(pre + 16 * (s - 1), Fd, t);
      m4_mul(t, suf + 16 * (s + 1), dT + 16 * (m->dof_off[a] + k));
    }
  }
  free(F); free(pre); free(suf);
}

/* Algorithm DERIV in tree form (Section 5), the O(N) counterpart of the
 * path derivatives above: r_d = d/dq_d sum_l <G_l, T_l(q)> for fixed 3x4
 * seeds G_l (<A, B> = sum of entrywise products). From the leaves to the
 * root, Y_a = G_a + sum over the children c of a of Y_c F_c^T, with F_c =
 * X_c Jm_c(q_c) the child's local transform; for a DOF k of joint a,
 * r = <Y_a, T_parent(a) X_a dJm_a/dq_k>. The chain rule needs no product
 * along a root-to-link path. G: [N][12] row-major 3x4; r: [n]. */
void om_deriv(void *p, const double *q, const double *G, double *r) {
  om_model *m = (om_model *)p;
  int N = m->n_links;
  double *F = (double *)malloc(sizeof(double) * 16 * N);
  double *T = (double *)malloc(sizeof(double) * 16 * N);
  double *Y = (double *)malloc(sizeof(double) * 16 * N);
  for (int a = 0; a < N; ++a) { /* parent[a] < a */
    joint_factor(m, a, q, F + 16 * a);
    if (m->parent[a] < 0) memcpy(T + 16 * a, F + 16 * a, sizeof(double) * 16);
    else m4_mul(T + 16 * m->parent[a], F + 16 * a, T + 16 * a);
    for (int i = 0; i < 12; ++i) Y[16 * a + i] = G[12 * a + i];
    for (int i = 12; i < 16; ++i) Y[16 * a + i] = 0.0;
  }
  for (int a = N - 1; a >= 0; --a) { /* children before their parents */
    int pa = m->parent[a];
    for (int k = 0; k < m->ndof[a]; ++k) {
      double Fd[16], PD[16];
      joint_factor_d(m, a, q, k, Fd);
      if (pa >= 0) m4_mul(T + 16 * pa, Fd, PD);
      else memcpy(PD, Fd, sizeof(PD));
      double s = 0.0;
      for (int i = 0; i < 16; ++i) s += Y[16 * a + i] * PD[i];
      r[m->dof_off[a] + k] = s;
    }
    if (pa >= 0) {
      /* Y_parent += Y_a F_a^T */
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
          double s = 0.0;
          for (int t = 0; t < 4; ++t) s += Y[16 * a + 4 * i + t] * F[16 * a + 4 * j + t];
          Y[16 * pa + 4 * i + j] += s;
        }
    }
  }
  free(F); free(T); free(Y);
}

/* ------------------------------------------------------------------ */
/* O(N) evaluation: Algorithm DERIV and its tangent                     */
/* ------------------------------------------------------------------ */
/* Not the oracle's reference path (om_eval, brute force, checks the CUDA
 * kernels): the O(N) CPU evaluation the CPU baseline times, checked against
 * om_eval in the test suite. */
int om_colloc(int S, double *nodes, double *W);
int om_colloc_vel(int S, double *Vw);

/* Forward kinematics by the recursion T_a = T_parent(a) F_a and the
 * tangent Tdot_a = Tdot_parent F_a + T_parent Fdot_a along a direction v
 * (Fdot_a = sum_k v_ak X_a dJm_a/dq_k). T, Td: [N][16]; Td may be NULL. */
static void fk_tangent(const om_model *m, const double *q, const double *v, double *T,
                       double *Td) {
  for (int a = 0; a < m->n_links; ++a) {
    int pa = m->parent[a];
    double F[16], Fd[16], t1[16], t2[16];
    joint_factor(m, a, q, F);
    if (pa < 0) memcpy(T + 16 * a, F, sizeof(F));
    else m4_mul(T + 16 * pa, F, T + 16 * a);
    if (!Td) continue;
    for (int i = 0; i < 16; ++i) Fd[i] = 0.0;
    for (int k = 0; k < m->ndof[a]; ++k) {
      double D[16];
      joint_factor_d(m, a, q, k, D);
      for (int i = 0; i < 16; ++i) Fd[i] += v[m->dof_off[a] + k] * D[i];
    }
    if (pa < 0) {
      memcpy(Td + 16 * a, Fd, sizeof(Fd));
    } else {
      m4_mul(Td + 16 * pa, F, t1);
      m4_mul(T + 16 * pa, Fd, t2);
      for (int i = 0; i < 16; ++i) Td[16 * a + i] = t1[i] + t2[i];
    }
  }
}

/* d/de of om_deriv(q + e v, G) at e = 0 for fixed seeds G (the second
 * derivatives of sum_l <G_l, T_l(q)> along v): with Y_a = G_a + sum_c Y_c
 * F_c^T and r_ak = <Y_a, T_parent(a) X_a dJm_a/dq_k>,
 *   Ydot_a = sum_c (Ydot_c F_c^T + Y_c Fdot_c^T),
 *   rdot_ak = <Ydot_a, T_pa D_ak> + <Y_a, Tdot_pa D_ak>
 *             + <Y_a, T_pa sum_j v_aj X_a d2Jm_a/dq_k dq_j>. */
static void deriv_tangent(const om_model *m, const double *q, const double *v,
                          const double *G, double *rd) {
  int N = m->n_links;
  double *F = (double *)malloc(sizeof(double) * 16 * N);
  double *Fd = (double *)malloc(sizeof(double) * 16 * N);
  double *T = (double *)malloc(sizeof(double) * 16 * N);
  double *Td = (double *)malloc(sizeof(double) * 16 * N);
  double *Y = (double *)malloc(sizeof(double) * 16 * N);
  double *Yd = (double *)malloc(sizeof(double) * 16 * N);
  fk_tangent(m, q, v, T, Td);
  for (int a = 0; a < N; ++a) {
    joint_factor(m, a, q, F + 16 * a);
    for (int i = 0; i < 16; ++i) Fd[16 * a + i] = 0.0;
    for (int k = 0; k < m->ndof[a]; ++k) {
      double D[16];
      joint_factor_d(m, a, q, k, D);
      for (int i = 0; i < 16; ++i) Fd[16 * a + i] += v[m->dof_off[a] + k] * D[i];
    }
    for (int i = 0; i < 12; ++i) Y[16 * a + i] = G[12 * a + i];
    for (int i = 12; i < 16; ++i) Y[16 * a + i] = 0.0;
    for (int i = 0; i < 16; ++i) Yd[16 * a + i] = 0.0;
  }
  for (int a = N - 1; a >= 0; --a) {
    int pa = m->parent[a];
    for (int k = 0; k < m->ndof[a]; ++k) {
      double D[16], DD[16], PD[16], PdD[16], PDD[16];
      joint_factor_d(m, a, q, k, D);
      for (int i = 0; i < 16; ++i) DD[i] = 0.0;
      for (int j = 0; j < m->ndof[a]; ++j) {
        double H[16];
        joint_factor_dd(m, a, q, k, j, H);
        for (int i = 0; i < 16; ++i) DD[i] += v[m->dof_off[a] + j] * H[i];
      }
      if (pa >= 0) {
        m4_mul(T + 16 * pa, D, PD);
        m4_mul(Td + 16 * pa, D, PdD);
        m4_mul(T + 16 * pa, DD, PDD);
      } else {
        memcpy(PD, D, sizeof(PD));
        for (int i = 0; i < 16; ++i) PdD[i] = 0.0;
        memcpy(PDD, DD, sizeof(PDD));
      }
      double s = 0.0;
      for (int i = 0; i < 16; ++i)
        s += Yd[16 * a + i] * PD[i] + Y[16 * a + i] * (PdD[i] + PDD[i]);
      rd[m->dof_off[a] + k] = s;
    }
    if (pa >= 0) {
      /* Y_parent += Y_a F_a^T and its tangent */
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
          double s = 0.0, sd = 0.0;
          for (int t = 0; t < 4; ++t) {
            s += Y[16 * a + 4 * i + t] * F[16 * a + 4 * j + t];
            sd += Yd[16 * a + 4 * i + t] * F[16 * a + 4 * j + t] +
                  Y[16 * a + 4 * i + t] * Fd[16 * a + 4 * j + t];
          }
          Y[16 * pa + 4 * i + j] += s;
          Yd[16 * pa + 4 * i + j] += sd;
        }
    }
  }
  free(F); free(Fd); free(T); free(Td); free(Y); free(Yd);
}

/* E, r and dE/dq of one step in O(N) per stage (no contact points): the
 * residual of every stage by om_deriv with the seeds of Eq. HOC; for S >= 2
 * the gradient of Eq. EQHOC, 2 Jr^T r, by
 *   (Jr^T v)_k = d/de om_deriv(q_k + e v_k, G_k)   (own-stage curvature)
 *              + om_deriv(q_k, B_k),  B_k,l = (sum_i W_ik Tdot_i,l) M_l
 * (the seeds' dependence on stage k; Tdot_i,l = dT_l(q_i)/dq_i v_i, M_l
 * symmetric), with v = r. The same quantities as om_eval, in O(N). */
double om_eval_fast(void *p, int S, double dt, const double *qs, const double *q_prev,
                    const double *q_cur, const double *tau, double *r, double *grad) {
  om_model *m = (om_model *)p;
  int N = m->n_links, n = m->n_dof, P = S + 2, Sn = S * n;
  double nodes[16], W[8 * 16], Vw[8 * 16], Wt[8 * 16];
  om_colloc(S, nodes, W);
  om_colloc_vel(S, Vw);
  double idt2 = 1.0 / (dt * dt);
  for (int k = 0; k < S * P; ++k) Wt[k] = (W[k] + 2.0 * m->drag * Vw[k]) * idt2;
  double *T = (double *)malloc(sizeof(double) * 16 * N * P);
  double *G = (double *)malloc(sizeof(double) * 12 * N);
  double *rr = r ? r : (double *)malloc(sizeof(double) * Sn);
  const double *qnode[16];
  qnode[0] = q_prev;
  qnode[1] = q_cur;
  for (int i = 0; i < S; ++i) qnode[2 + i] = qs + i * n;
  for (int j = 0; j < P; ++j) fk_tangent(m, qnode[j], NULL, T + 16 * N * j, NULL);
  double E = 0.0;
  for (int i = 0; i < S; ++i) {
    for (int l = 0; l < N; ++l) {
      double A[16], M[16], GG[16];
      mm4(m->mm + 10 * l, M);
      for (int k = 0; k < 16; ++k) {
        double sum = 0;
        for (int j = 0; j < P; ++j) sum += Wt[i * P + j] * T[16 * N * j + 16 * l + k];
        A[k] = sum;
      }
      m4_mul(A, M, GG);
      for (int rw = 0; rw < 3; ++rw)
        for (int c = 0; c < 4; ++c) GG[4 * rw + c] -= m->g[rw] * m->mm[10 * l + 6 + c];
      memcpy(G + 12 * l, GG, sizeof(double) * 12);
    }
    om_deriv(m, qnode[2 + i], G, rr + i * n);
    for (int d = 0; d < n; ++d) rr[i * n + d] -= tau[d];
  }
  if (S == 1) {
    for (int l = 0; l < N; ++l) {
      double M[16], D[16], DM[16];
      mm4(m->mm + 10 * l, M);
      for (int k = 0; k < 16; ++k)
        D[k] = T[16 * N * 2 + 16 * l + k] - 2 * T[16 * N + 16 * l + k] + T[16 * l + k];
      m4_mul(D, M, DM);
      E += 0.5 * idt2 * contract34(DM, D);
      if (m->drag != 0.0) {
        double Dv[16], DvM[16];
        for (int k = 0; k < 16; ++k) Dv[k] = T[16 * N * 2 + 16 * l + k] - T[16 * N + 16 * l + k];
        m4_mul(Dv, M, DvM);
        E += m->drag * idt2 * contract34(DvM, Dv);
      }
      for (int rw = 0; rw < 3; ++rw)
        for (int c = 0; c < 4; ++c)
          E -= m->g[rw] * T[16 * N * 2 + 16 * l + 4 * rw + c] * m->mm[10 * l + 6 + c];
    }
    for (int d = 0; d < n; ++d) E -= tau[d] * qs[d];
    if (grad) memcpy(grad, rr, sizeof(double) * Sn);
  } else {
    for (int k = 0; k < Sn; ++k) E += rr[k] * rr[k];
    if (grad) {
      double *Td = (double *)malloc(sizeof(double) * 16 * N * S);
      double *Tt = (double *)malloc(sizeof(double) * 16 * N);
      double *rd = (double *)malloc(sizeof(double) * n);
      for (int i = 0; i < S; ++i) fk_tangent(m, qnode[2 + i], rr + i * n, Tt, Td + 16 * N * i);
      for (int k = 0; k < S; ++k) {
        /* own-stage curvature along v_k with the seeds G_k */
        for (int l = 0; l < N; ++l) {
          double A[16], M[16], GG[16];
          mm4(m->mm + 10 * l, M);
          for (int e = 0; e < 16; ++e) {
            double sum = 0;
            for (int j = 0; j < P; ++j) sum += Wt[k * P + j] * T[16 * N * j + 16 * l + e];
            A[e] = sum;
          }
          m4_mul(A, M, GG);
          for (int rw = 0; rw < 3; ++rw)
            for (int c = 0; c < 4; ++c) GG[4 * rw + c] -= m->g[rw] * m->mm[10 * l + 6 + c];
          memcpy(G + 12 * l, GG, sizeof(double) * 12);
        }
        deriv_tangent(m, qnode[2 + k], rr + k * n, G, grad + k * n);
        /* dependence of every stage's seeds on stage k */
        for (int l = 0; l < N; ++l) {
          double Bs[16], M[16], BM[16];
          mm4(m->mm + 10 * l, M);
          for (int e = 0; e < 16; ++e) {
            double sum = 0;
            for (int i = 0; i < S; ++i) sum += Wt[i * P + 2 + k] * Td[16 * N * i + 16 * l + e];
            Bs[e] = sum;
          }
          m4_mul(Bs, M, BM);
          memcpy(G + 12 * l, BM, sizeof(double) * 12);
        }
        om_deriv(m, qnode[2 + k], G, rd);
        for (int d = 0; d < n; ++d) grad[k * n + d] = 2.0 * (grad[k * n + d] + rd[d]);
      }
      free(Td); free(Tt); free(rd);
    }
  }
  free(T); free(G);
  if (!r) free(rr);
  return E;
}

/* Makes the model's L-BFGS evaluate with om_eval_fast (1) or om_eval (0). */
void om_model_set_fast(void *p, int fast) { ((om_model *)p)->fast = fast; }

/* Accumulates H[d][e] += sum over (d,e) on the root->l path of
 * (d2 T_l / dq_d dq_e) : G, with G a 3x4 (12 entries) matrix. H: [n][n]. */
static void link_ddT_contract(const om_model *m, int l, const double *q,
                              const double *G, double *H) {
  int N = m->n_links, len = m->path_len[l], n = m->n_dof;
  double *F = (double *)malloc(sizeof(double) * 16 * (len + 2));
  double *pre = (double *)malloc(sizeof(double) * 16 * (len + 2));
  double *suf = (double *)malloc(sizeof(double) * 16 * (len + 2));
  path_products(m, l, q, F, pre, suf);
  for (int s = 1; s <= len; ++s) {
    int a = m->path[l * N + s - 1];
    for (int k = 0; k < m->ndof[a]; ++k) {
      int d = m->dof_off[a] + k;
      /* same joint: X_a d2Jm/dq_k dq_kk */
      for (int kk = 0; kk < m->ndof[a]; ++kk) {
        double Fdd[16], t[16], u[16];
        joint_factor_dd(m, a, q, k, kk, Fdd);
        m4_mul(pre + 16 * (s - 1), Fdd, t);
        m4_mul(t, suf + 16 * (s + 1), u);
        H[d * n + m->dof_off[a] + kk] += contract34(u, G);
      }
      /* later joint on the path: pre * F'_s * F_{s+1}..F_{t-1} * F'_t * suf */
      double L[16], Fd[16];
      joint_factor_d(m, a, q, k, Fd);
      m4_mul(pre + 16 * (s - 1), Fd, L);
      for (int t = s + 1; t <= len; ++t) {
        int b = m->path[l * N + t - 1];
        for (int kk = 0; kk < m->ndof[b]; ++kk) {
          double Fe[16], u[16], v[16];
          joint_factor_d(m, b, q, kk, Fe);
          m4_mul(L, Fe, u);
          m4_mul(u, suf + 16 * (t + 1), v);
          double c = contract34(v, G);
          int e = m->dof_off[b] + kk;
          H[d * n + e] += c;
          H[e * n + d] += c;
        }
        m4_mul(L, F + 16 * t, L);
      }
    }
  }
  free(F); free(pre); free(suf);
}

/* d2T_l/dq_d dq_e as a 4x4 matrix, for tests: contracts against unit
 * matrices. */
void om_link_ddT(void *p, const double *q, int l, int d, int e, double *out) {
  om_model *m = (om_model *)p;
  int n = m->n_dof;
  double *H = (double *)malloc(sizeof(double) * n * n);
  for (int k = 0; k < 12; ++k) {
    double G[12] = {0};
    G[k] = 1;
    memset(H, 0, sizeof(double) * n * n);
    link_ddT_contract(m, l, q, G, H);
    out[k] = H[d * n + e];
  }
  out[12] = out[13] = out[14] = out[15] = 0;
  free(H);
}

/* ------------------------------------------------------------------ */
/* collocation (Section 4.1): Legendre nodes and second-derivative weights */
/* ------------------------------------------------------------------ */

/* Roots of the Legendre polynomial L_n on [-1,1], ascending, by Newton's
 * method on the three-term recurrence. */
int om_legendre_roots(int n, double *x) {
  if (n < 0 || n > 64) return -1;
  for (int i = 0; i < n; ++i) {
    double z = -cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = n == 0 ? 1 : p1, pm = n == 0 ? 0 : p0;
      if (n == 0) break;
      double dp = n * (z * pn - pm) / (z * z - 1);
      double dz = pn / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    x[i] = z;
  }
  return 0;
}

/* Nodes (units of dt, relative to t_k) in the order
 * [k-1+alpha_{S-1}, k, k+alpha_1, ..., k+alpha_S] with alpha_S = 1 and
 * alpha_1..alpha_{S-1} the roots of L_{S-1}(2 alpha - 1) (alpha_0 = 0).
 * W[i][j] = l_j''(alpha_i) of the Lagrange basis over all S+2 nodes
 * (units 1/dt^2), from the Vandermonde system. nodes: S+2, W: S x (S+2). */
int om_colloc(int S, double *nodes, double *W) {
  if (S < 1 || S > 8) return -1;
  int K = S + 1; /* polynomial degree */
  int P = S + 2; /* number of nodes */
  double alpha[16];
  double xr[16];
  om_legendre_roots(S - 1, xr);
  for (int i = 0; i < S - 1; ++i) alpha[i + 1] = 0.5 * (xr[i] + 1);
  alpha[0] = 0;
  alpha[S] = 1;
  nodes[0] = -1 + alpha[S - 1];
  nodes[1] = 0;
  for (int i = 1; i <= S; ++i) nodes[1 + i] = alpha[i];
  /* V c_j = e_j with V[r][k] = nodes[r]^k; solve for all j at once: C = V^-1 */
  double V[16 * 16], C[16 * 16];
  for (int r = 0; r < P; ++r)
    for (int k = 0; k < P; ++k) {
      V[r * P + k] = pow(nodes[r], k);
      C[r * P + k] = (r == k) ? 1.0 : 0.0;
    }
  /* Gauss-Jordan with partial pivoting on [V | I] -> [I | V^-1] */
  for (int col = 0; col < P; ++col) {
    int piv = col;
    for (int r = col + 1; r < P; ++r)
      if (fabs(V[r * P + col]) > fabs(V[piv * P + col])) piv = r;
    for (int k = 0; k < P; ++k) {
      double t = V[col * P + k]; V[col * P + k] = V[piv * P + k]; V[piv * P + k] = t;
      t = C[col * P + k]; C[col * P + k] = C[piv * P + k]; C[piv * P + k] = t;
    }
    double d = V[col * P + col];
    for (int k = 0; k < P; ++k) { V[col * P + k] /= d; C[col * P + k] /= d; }
    for (int r = 0; r < P; ++r) {
      if (r == col) continue;
      double fct = V[r * P + col];
      for (int k = 0; k < P; ++k) {
        V[r * P + k] -= fct * V[col * P + k];
        C[r * P + k] -= fct * C[col * P + k];
      }
    }
  }
  /* coefficient k of basis polynomial j is C[k][j] (column j of V^-1) */
  for (int i = 0; i < S; ++i) {
    double t = nodes[2 + i];
    for (int j = 0; j < P; ++j) {
      double s = 0;
      for (int k = 2; k <= K; ++k) s += k * (k - 1.0) * C[k * P + j] * pow(t, k - 2);
      W[i * P + j] = s;
    }
  }
  return 0;
}

/* First-derivative weights V (S x (S+2), row-major, units 1/dt): velocity of
 * the collocation polynomial at stage node i, v_i = sum_j V_ij q_j / dt. For
 * one stage, the backward difference of the drag potential (Section 6.2):
 * V = [0, -1, 1]. For S >= 2, V_ij = l_j'(alpha_i) of the Lagrange basis over
 * the S+2 nodes of om_colloc (its Vandermonde inverse, recomputed here). */
int om_colloc_vel(int S, double *Vw) {
  if (S < 1 || S > 8) return -1;
  int P = S + 2;
  if (S == 1) {
    Vw[0] = 0.0; Vw[1] = -1.0; Vw[2] = 1.0;
    return 0;
  }
  double nodes[16], Wtmp[8 * 16];
  om_colloc(S, nodes, Wtmp);
  double V[16 * 16], C[16 * 16];
  for (int r = 0; r < P; ++r)
    for (int k = 0; k < P; ++k) {
      V[r * P + k] = pow(nodes[r], k);
      C[r * P + k] = (r == k) ? 1.0 : 0.0;
    }
  for (int col = 0; col < P; ++col) {
    int piv = col;
    for (int r = col + 1; r < P; ++r)
      if (fabs(V[r * P + col]) > fabs(V[piv * P + col])) piv = r;
    for (int k = 0; k < P; ++k) {
      double t = V[col * P + k]; V[col * P + k] = V[piv * P + k]; V[piv * P + k] = t;
      t = C[col * P + k]; C[col * P + k] = C[piv * P + k]; C[piv * P + k] = t;
    }
    double d = V[col * P + col];
    for (int k = 0; k < P; ++k) { V[col * P + k] /= d; C[col * P + k] /= d; }
    for (int r = 0; r < P; ++r) {
      if (r == col) continue;
      double fct = V[r * P + col];
      for (int k = 0; k < P; ++k) {
        V[r * P + k] -= fct * V[col * P + k];
        C[r * P + k] -= fct * C[col * P + k];
      }
    }
  }
  for (int i = 0; i < S; ++i) {
    double t = nodes[2 + i];
    for (int j = 0; j < P; ++j) {
      double s = 0;
      for (int k = 1; k < P; ++k) s += k * C[k * P + j] * pow(t, k - 1);
      Vw[i * P + j] = s;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* mass moments (Eq. ATOM: int rho [p;1][p;1]^T dp)                     */
/* ------------------------------------------------------------------ */

/* Uniform thin rod of mass m from the joint (origin) to (0,0,-L). */
void om_mass_moment_rod(double m, double L, double *mm) {
  for (int k = 0; k < 10; ++k) mm[k] = 0;
  mm[5] = m * L * L / 3.0; /* Szz */
  mm[8] = -m * L / 2.0;    /* m cz */
  mm[9] = m;
}

/* Uniform solid capsule of total mass m: a cylinder of radius r whose axis
 * runs from the origin to (0,0,-L), capped by two hemispheres. Second moment
 * about the centroid c = (0,0,-L/2) from the textbook inertia tensor I_c:
 * Sigma_c = tr(I_c)/2 Id - I_c, then the parallel-axis shift m c c^T. */
void om_mass_moment_capsule(double m, double L, double r, double *mm) {
  double vc = M_PI * r * r * L, vh = 4.0 / 3.0 * M_PI * r * r * r;
  double rho = m / (vc + vh);
  double mc = rho * vc, mh = rho * vh;
  double Izz = mc * r * r / 2 + mh * 2.0 * r * r / 5;
  double Ixx = mc * (L * L / 12 + r * r / 4) +
               mh * (2.0 * r * r / 5 + L * L / 4 + 3.0 * L * r / 8);
  double tr = 2 * Ixx + Izz;
  double sxx = tr / 2 - Ixx, szz = tr / 2 - Izz;
  double cz = -L / 2;
  for (int k = 0; k < 10; ++k) mm[k] = 0;
  mm[0] = sxx;
  mm[3] = sxx;
  mm[5] = szz + m * cz * cz;
  mm[8] = m * cz;
  mm[9] = m;
}

/* ------------------------------------------------------------------ */
/* objective, residuals and their derivatives (Eq. EQ, HOC, EQHOC)      */
/* ------------------------------------------------------------------ */

/* Joint-space mass matrix int rho (dP/dq)^T (dP/dq) dp (the Gauss-Newton
 * Hessian of Eq. EQ times dt^2). H: [n][n]. */
void om_hmass(void *p, const double *q, double *H) {
  om_model *m = (om_model *)p;
  int N = m->n_links, n = m->n_dof;
  double *dT = (double *)malloc(sizeof(double) * 16 * n);
  memset(H, 0, sizeof(double) * n * n);
  for (int l = 0; l < N; ++l) {
    double M[16];
    mm4(m->mm + 10 * l, M);
    om_link_dT(p, q, l, dT);
    for (int d = 0; d < n; ++d) {
      double DM[16];
      m4_mul(dT + 16 * d, M, DM);
      for (int e = 0; e < n; ++e) H[d * n + e] += contract34(DM, dT + 16 * e);
    }
  }
  free(dT);
}

/* Evaluates stage residuals and the objective for one step.
 *   qs: S*n unknown stage configurations (stage-major), q_prev/q_cur the two
 *   known nodes, tau the generalised joint torques (piecewise constant).
 *   r (S*n): r_i = int dP(q_i)/dq_i^T [rho Pddot(t_i) - f] dp - tau   (Eq. HOC)
 *   returns E: S == 1 -> Eq. EQ energy; S >= 2 -> sum_i |r_i|^2 (Eq. EQHOC).
 *   Jr (S*n x S*n, optional): dr/dq_*. For S == 1 this is the exact Hessian
 *   of Eq. EQ.
 *   grad (S*n, optional): dE/dq_*; S == 1 -> r; S >= 2 -> 2 Jr^T r.
 * Any of r/grad/Jr may be NULL (grad for S >= 2 needs Jr internally). */
double om_eval(void *p, int S, double dt, const double *qs,
               const double *q_prev, const double *q_cur, const double *tau,
               double *r, double *grad, double *Jr) {
  om_model *m = (om_model *)p;
  int N = m->n_links, n = m->n_dof, P = S + 2, Sn = S * n;
  double nodes[16], W[8 * 16], Vw[8 * 16];
  om_colloc(S, nodes, W);
  om_colloc_vel(S, Vw);
  double idt2 = 1.0 / (dt * dt);
  const double cd = m->drag;
  /* seed weights: acceleration W/dt^2 plus the drag force 2 c V/dt^2 */
  double Wt[8 * 16];
  for (int k = 0; k < S * P; ++k) Wt[k] = (W[k] + 2.0 * cd * Vw[k]) * idt2;
  /* transforms at every node */
  double *T = (double *)malloc(sizeof(double) * 16 * N * P);
  om_fk(p, q_prev, T);
  om_fk(p, q_cur, T + 16 * N);
  for (int i = 0; i < S; ++i) om_fk(p, qs + i * n, T + 16 * N * (2 + i));
  const double *qnode[16];
  qnode[0] = q_prev;
  qnode[1] = q_cur;
  for (int i = 0; i < S; ++i) qnode[2 + i] = qs + i * n;

  int needJ = (Jr != NULL) || (grad != NULL && S >= 2);
  double *J = NULL;
  if (needJ) J = Jr ? Jr : (double *)malloc(sizeof(double) * Sn * Sn);
  if (needJ) memset(J, 0, sizeof(double) * Sn * Sn);
  double *rr = r ? r : (double *)malloc(sizeof(double) * Sn);
  for (int k = 0; k < Sn; ++k) rr[k] = -tau[k % n];

  double E = 0;
  double *dTi = (double *)malloc(sizeof(double) * 16 * n * S);
  for (int l = 0; l < N; ++l) {
    double M[16], mc4[4];
    mm4(m->mm + 10 * l, M);
    mc4[0] = m->mm[10 * l + 6]; mc4[1] = m->mm[10 * l + 7];
    mc4[2] = m->mm[10 * l + 8]; mc4[3] = m->mm[10 * l + 9];
    for (int i = 0; i < S; ++i) om_link_dT(p, qnode[2 + i], l, dTi + 16 * n * i);
    if (S == 1) {
      /* Eq. EQ: tr(D M D^T)/(2 dt^2) - g.(T [mc; m]) */
      double D[16], DM[16];
      for (int k = 0; k < 16; ++k)
        D[k] = T[16 * N * 2 + 16 * l + k] - 2 * T[16 * N + 16 * l + k] + T[16 * l + k];
      m4_mul(D, M, DM);
      E += 0.5 * idt2 * contract34(DM, D);
      if (cd != 0.0) {
        /* Q_drag: c / dt^2 tr(D' M D'^T), D' = T_{k+1} - T_k */
        double Dv[16], DvM[16];
        for (int k = 0; k < 16; ++k) Dv[k] = T[16 * N * 2 + 16 * l + k] - T[16 * N + 16 * l + k];
        m4_mul(Dv, M, DvM);
        E += cd * idt2 * contract34(DvM, Dv);
      }
      for (int rrow = 0; rrow < 3; ++rrow)
        for (int c = 0; c < 4; ++c)
          E -= m->g[rrow] * T[16 * N * 2 + 16 * l + 4 * rrow + c] * mc4[c];
    }
    for (int i = 0; i < S; ++i) {
      /* seed G_{i,l} = (sum_j (W_ij + 2c V_ij) T_l(q_j) / dt^2) M_l - g [mc; m]^T */
      double A[16], G[16];
      for (int k = 0; k < 16; ++k) {
        double s = 0;
        for (int j = 0; j < P; ++j) s += Wt[i * P + j] * T[16 * N * j + 16 * l + k];
        A[k] = s;
      }
      m4_mul(A, M, G);
      for (int rrow = 0; rrow < 3; ++rrow)
        for (int c = 0; c < 4; ++c) G[4 * rrow + c] -= m->g[rrow] * mc4[c];
      for (int d = 0; d < n; ++d) rr[i * n + d] += contract34(dTi + 16 * n * i + 16 * d, G);
      if (needJ) {
        /* own-stage second derivatives contracted with the seed */
        double *Hblk = (double *)calloc((size_t)n * n, sizeof(double));
        link_ddT_contract(m, l, qnode[2 + i], G, Hblk);
        for (int d = 0; d < n; ++d)
          for (int e = 0; e < n; ++e) J[(i * n + d) * Sn + i * n + e] += Hblk[d * n + e];
        free(Hblk);
        /* dependence of the seed on every unknown stage j through its weight */
        for (int j = 0; j < S; ++j) {
          double wij = Wt[i * P + 2 + j];
          for (int e = 0; e < n; ++e) {
            double DM[16];
            m4_mul(dTi + 16 * n * j + 16 * e, M, DM);
            for (int d = 0; d < n; ++d)
              J[(i * n + d) * Sn + j * n + e] += wij * contract34(dTi + 16 * n * i + 16 * d, DM);
          }
        }
      }
    }
  }
  if (S == 1 && m->n_contact > 0) {
    /* Eq. FRI contact points: energy, residual dP/dq . f and, for the
     * Jacobian, dP/dq^T H dP/dq + d2P/dq2 . f */
    double *dTl = (double *)malloc(sizeof(double) * 16 * n);
    double *dP = (double *)malloc(sizeof(double) * 3 * n);
    double *Hb = needJ ? (double *)calloc((size_t)n * n, sizeof(double)) : NULL;
    for (int c = 0; c < m->n_contact; ++c) {
      int l = m->c_link[c];
      const double *pt = m->c_point + 3 * c;
      double P[3], Pk[3], Q, f[3], H[9], Hk[9];
      point_world(T + 16 * N * 2 + 16 * l, pt, P);
      point_world(T + 16 * N + 16 * l, pt, Pk);
      if (!contact_point(m, dt, P, Pk, &Q, f, H, Hk)) continue;
      E += Q;
      om_link_dT(p, qs, l, dTl);
      for (int d = 0; d < n; ++d) {
        point_world(dTl + 16 * d, pt, dP + 3 * d);  /* dP/dq_d = dT_l/dq_d [p; 1] */
        rr[d] += dP[3 * d] * f[0] + dP[3 * d + 1] * f[1] + dP[3 * d + 2] * f[2];
      }
      if (needJ) {
        for (int d = 0; d < n; ++d)
          for (int e = 0; e < n; ++e) {
            double s = 0;
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b) s += dP[3 * d + a] * H[3 * a + b] * dP[3 * e + b];
            J[d * Sn + e] += s;
          }
        double Gc[16] = {0};
        for (int r = 0; r < 3; ++r) {
          Gc[4 * r] = f[r] * pt[0]; Gc[4 * r + 1] = f[r] * pt[1];
          Gc[4 * r + 2] = f[r] * pt[2]; Gc[4 * r + 3] = f[r];
        }
        memset(Hb, 0, sizeof(double) * n * n);
        link_ddT_contract(m, l, qs, Gc, Hb);
        for (int k = 0; k < n * n; ++k) J[k] += Hb[k];
      }
    }
    free(dTl);
    free(dP);
    free(Hb);
  }
  if (S == 1) {
    for (int d = 0; d < n; ++d) E -= tau[d] * qs[d];
  } else {
    for (int k = 0; k < Sn; ++k) E += rr[k] * rr[k];
  }
  if (grad) {
    if (S == 1) {
      for (int k = 0; k < Sn; ++k) grad[k] = rr[k];
    } else {
      for (int c = 0; c < Sn; ++c) {
        double s = 0;
        for (int k = 0; k < Sn; ++k) s += J[k * Sn + c] * rr[k];
        grad[c] = 2 * s;
      }
    }
  }
  free(dTi);
  free(T);
  if (!r) free(rr);
  if (needJ && !Jr) free(J);
  return E;
}

/* Partial derivatives of the residuals with respect to the two known nodes:
 * Jp = dr/dq_prev, Jc = dr/dq_cur (S*n x n each). dr/dtau = -I per stage. */
void om_resid_known_jac(void *p, int S, double dt, const double *qs,
                        const double *q_prev, const double *q_cur, double *Jp,
                        double *Jc) {
  om_model *m = (om_model *)p;
  int N = m->n_links, n = m->n_dof, P = S + 2, Sn = S * n;
  double nodes[16], W[8 * 16], Vw[8 * 16];
  om_colloc(S, nodes, W);
  om_colloc_vel(S, Vw);
  double idt2 = 1.0 / (dt * dt);
  const double cd = m->drag;
  memset(Jp, 0, sizeof(double) * Sn * n);
  memset(Jc, 0, sizeof(double) * Sn * n);
  double *dTi = (double *)malloc(sizeof(double) * 16 * n * S);
  double *dTp = (double *)malloc(sizeof(double) * 16 * n);
  double *dTc = (double *)malloc(sizeof(double) * 16 * n);
  for (int l = 0; l < N; ++l) {
    double M[16];
    mm4(m->mm + 10 * l, M);
    for (int i = 0; i < S; ++i) om_link_dT(p, qs + i * n, l, dTi + 16 * n * i);
    om_link_dT(p, q_prev, l, dTp);
    om_link_dT(p, q_cur, l, dTc);
    for (int i = 0; i < S; ++i) {
      double wp = (W[i * P + 0] + 2.0 * cd * Vw[i * P + 0]) * idt2;
      double wc = (W[i * P + 1] + 2.0 * cd * Vw[i * P + 1]) * idt2;
      for (int e = 0; e < n; ++e) {
        double DMp[16], DMc[16];
        m4_mul(dTp + 16 * e, M, DMp);
        m4_mul(dTc + 16 * e, M, DMc);
        for (int d = 0; d < n; ++d) {
          Jp[(i * n + d) * n + e] += wp * contract34(dTi + 16 * n * i + 16 * d, DMp);
          Jc[(i * n + d) * n + e] += wc * contract34(dTi + 16 * n * i + 16 * d, DMc);
        }
      }
    }
  }
  if (S == 1 && m->n_contact > 0) {
    /* Eq. FRI: the tangential velocity depends on q_k through P_p(q_k):
     * dr/dq_cur += dP/dq^T (d2Q/dP dPk) dPk/dq_cur */
    double *dP = (double *)malloc(sizeof(double) * 3 * n);
    double *dPk = (double *)malloc(sizeof(double) * 3 * n);
    double *Tn = (double *)malloc(sizeof(double) * 16 * N);
    double *Tc = (double *)malloc(sizeof(double) * 16 * N);
    om_fk(p, qs, Tn);
    om_fk(p, q_cur, Tc);
    for (int c = 0; c < m->n_contact; ++c) {
      int l = m->c_link[c];
      const double *pt = m->c_point + 3 * c;
      double P[3], Pk[3], Q, f[3], H[9], Hk[9];
      point_world(Tn + 16 * l, pt, P);
      point_world(Tc + 16 * l, pt, Pk);
      if (!contact_point(m, dt, P, Pk, &Q, f, H, Hk)) continue;
      om_link_dT(p, qs, l, dTi);
      om_link_dT(p, q_cur, l, dTc);
      for (int d = 0; d < n; ++d) {
        point_world(dTi + 16 * d, pt, dP + 3 * d);
        point_world(dTc + 16 * d, pt, dPk + 3 * d);
      }
      for (int d = 0; d < n; ++d)
        for (int e = 0; e < n; ++e) {
          double s = 0;
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) s += dP[3 * d + a] * Hk[3 * a + b] * dPk[3 * e + b];
          Jc[d * n + e] += s;
        }
    }
    free(dP); free(dPk); free(Tn); free(Tc);
  }
  free(dTi); free(dTp); free(dTc);
}

/* H += sum over the active contact points of dP/dq^T (d2Q/dP2) dP/dq at q
 * (one stage; q_cur gives the tangential velocity). H: n x n. */
static void contact_gn(om_model *m, double dt, const double *q, const double *q_cur, double *H) {
  if (m->n_contact == 0) return;
  int N = m->n_links, n = m->n_dof;
  double *Tn = (double *)malloc(sizeof(double) * 16 * N);
  double *Tc = (double *)malloc(sizeof(double) * 16 * N);
  double *dTl = (double *)malloc(sizeof(double) * 16 * n);
  double *dP = (double *)malloc(sizeof(double) * 3 * n);
  om_fk(m, q, Tn);
  om_fk(m, q_cur, Tc);
  for (int c = 0; c < m->n_contact; ++c) {
    int l = m->c_link[c];
    const double *pt = m->c_point + 3 * c;
    double P[3], Pk[3], Q, f[3], Hc[9], Hk[9];
    point_world(Tn + 16 * l, pt, P);
    point_world(Tc + 16 * l, pt, Pk);
    if (!contact_point(m, dt, P, Pk, &Q, f, Hc, Hk)) continue;
    om_link_dT(m, q, l, dTl);
    for (int d = 0; d < n; ++d) point_world(dTl + 16 * d, pt, dP + 3 * d);
    for (int d = 0; d < n; ++d)
      for (int e = 0; e < n; ++e) {
        double s = 0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) s += dP[3 * d + a] * Hc[3 * a + b] * dP[3 * e + b];
        H[d * n + e] += s;
      }
  }
  free(Tn); free(Tc); free(dTl); free(dP);
}

/* Test access: H (n x n, overwritten) = the contact term of the one-stage
 * Gauss-Newton matrix at q, as the Newton solve adds it. */
void om_contact_gn(void *p, double dt, const double *q, const double *q_cur, double *H) {
  om_model *m = (om_model *)p;
  memset(H, 0, sizeof(double) * m->n_dof * m->n_dof);
  contact_gn(m, dt, q, q_cur, H);
}

/* ------------------------------------------------------------------ */
/* dense linear algebra for the optimisers and the adjoint              */
/* ------------------------------------------------------------------ */

/* In-place Cholesky A = L L^T (lower triangle). Returns 0 on success. */
static int cholesky(double *A, int n) {
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
    if (!(s > 0)) return -1;
    double d = sqrt(s);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / d;
    }
  }
  return 0;
}
static void chol_solve(const double *L, int n, double *b) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i * n + k] * b[k];
    b[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * b[k];
    b[i] = s / L[i * n + i];
  }
}
/* Solves A x = b by Gaussian elimination with partial pivoting (A, b
 * overwritten; x returned in b). Returns 0 on success. */
static int lu_solve(double *A, int n, double *b) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0) return -1;
    if (piv != c) {
      for (int k = 0; k < n; ++k) {
        double t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t;
      }
      double t = b[c]; b[c] = b[piv]; b[piv] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
    b[r] = s / A[r * n + r];
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* optimisers (Section 5: LBFGS and LM)                                 */
/* ------------------------------------------------------------------ */

enum { OM_CONVERGED = 0, OM_MAX_ITER = 1, OM_LS_FAIL = 2, OM_CHOL_FAIL = 3,
       OM_NONFINITE = 4, OM_STALLED = 5 };

/* Severity order of the statuses for the worst over a rollout's steps:
 * CONVERGED < STALLED (solved to the rounding floor) < MAX_ITER < LS_FAIL <
 * CHOL_FAIL < NONFINITE. */
static int status_rank(int st) { return st == OM_STALLED ? 1 : (st == OM_CONVERGED ? 0 : st + 1); }
int om_status_worse(int a, int b) { return status_rank(b) > status_rank(a) ? b : a; }

/* Rounding floor of |r|_2 for one step (the paper is silent on it). A stage
 * residual of Eq. HOC (or the gradient of Eq. EQ) is a sum of terms of size
 * |W_ij| |T M| |lever| that cancel down to the answer, so binary64 cannot
 * resolve |r| below about eps times their size. The bound used:
 *   floor = eps (What sum_l I_l + |g| sum_l (|m c_l| + m_l R_l)),
 *   What = max_i sum_j |W_ij + 2 c V_ij| / dt^2 over all S+2 nodes (the
 *          acceleration and drag weights of the seeds),
 *   R_l  = sum of |t(X_a)| over the joints a on the root-to-l path (a bound
 *          on the distance of link l's frame from the root in rest geometry),
 *   I_l  = (sqrt(tr Sigma_l) + sqrt(m_l) R_l)^2 >= int rho |P|^2 over link l
 *          about the root.
 * Translation coordinates and contact points are not in the bound. A step
 * whose line search (or LM damping) cannot lower E while |r| <= 1e3 floor
 * ends STALLED instead of LS_FAIL: solved as far as binary64 resolves r. */
double om_floor(void *p, int S, double dt) {
  om_model *m = (om_model *)p;
  int N = m->n_links, P = S + 2;
  double nodes[16], W[8 * 16], Vw[8 * 16];
  om_colloc(S, nodes, W);
  om_colloc_vel(S, Vw);
  double What = 0;
  for (int i = 0; i < S; ++i) {
    double row = 0;
    for (int j = 0; j < P; ++j) row += fabs(W[i * P + j] + 2.0 * m->drag * Vw[i * P + j]);
    if (row > What) What = row;
  }
  What /= dt * dt;
  double sI = 0, sg = 0;
  for (int l = 0; l < N; ++l) {
    double R = 0;
    for (int a = l; a >= 0; a = m->parent[a]) {
      const double *X = m->rest + 12 * a;
      R += sqrt(X[3] * X[3] + X[7] * X[7] + X[11] * X[11]);
    }
    const double *mm = m->mm + 10 * l;
    double tr = mm[0] + mm[3] + mm[5];
    double mass = mm[9];
    double a = sqrt(tr > 0 ? tr : 0) + sqrt(mass > 0 ? mass : 0) * R;
    sI += a * a;
    sg += sqrt(mm[6] * mm[6] + mm[7] * mm[7] + mm[8] * mm[8]) + mass * R;
  }
  double gn = sqrt(m->g[0] * m->g[0] + m->g[1] * m->g[1] + m->g[2] * m->g[2]);
  return 2.220446049250313e-16 * (What * sI + gn * sg);
}
#define STALL_FACTOR 1e3

static double dot(const double *a, const double *b, int n) {
  double s = 0;
  for (int k = 0; k < n; ++k) s += a[k] * b[k];
  return s;
}
static int all_finite(const double *a, int n) {
  for (int k = 0; k < n; ++k)
    if (!isfinite(a[k])) return 0;
  return 1;
}

/* Initial guess: linear extrapolation through the two known nodes to every
 * stage node. */
static void initial_guess(int S, int n, const double *q_prev,
                          const double *q_cur, double *qs) {
  double nodes[16], W[8 * 16];
  om_colloc(S, nodes, W);
  double h = 0 - nodes[0];
  for (int i = 0; i < S; ++i)
    for (int d = 0; d < n; ++d)
      qs[i * n + d] = q_cur[d] + nodes[2 + i] * (q_cur[d] - q_prev[d]) / h;
}

/* Initial inverse Hessian of L-BFGS (H0 = gamma * P), from the joint-space
 * mass matrix Hmass at the current configuration q_cur, keeping only its
 * per-joint diagonal blocks B (1x1 for hinges, 3x3 for balls):
 *   S == 1 (Eq. EQ, Hessian ~ Hmass/dt^2):      P = dt^2 B^-1
 *   S >= 2 (Eq. EQHOC, Hessian ~ 2 Jr^T Jr with Jr ~ What (x) Hmass, What the
 *   unknown-stage columns of W/dt^2):           P = (What^T What)^-1 (x) B^-2 / 2
 * Stored as Pinv blocks: Pb[joint] (3x3, row-major, inverse of B or B^2) and
 * Ps (S x S, (What^T What)^-1 / 2 or dt^2). */
typedef struct {
  int S, n;
  double *Pb; /* [N][9] */
  double Ps[64];
} om_precond;

static int inv3(const double *A, double *X, int k) {
  if (k == 1) {
    if (!(A[0] > 0)) return -1;
    X[0] = 1.0 / A[0];
    return 0;
  }
  double a = A[0], b = A[1], c = A[2], d = A[3], e = A[4], f = A[5], g = A[6],
         h = A[7], i = A[8];
  double det = a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g);
  if (!(fabs(det) > 0)) return -1;
  X[0] = (e * i - f * h) / det; X[1] = (c * h - b * i) / det; X[2] = (b * f - c * e) / det;
  X[3] = (f * g - d * i) / det; X[4] = (a * i - c * g) / det; X[5] = (c * d - a * f) / det;
  X[6] = (d * h - e * g) / det; X[7] = (b * g - a * h) / det; X[8] = (a * e - b * d) / det;
  return 0;
}

static void lbfgs_precond(om_model *m, int S, double dt, const double *q_cur,
                          om_precond *pc) {
  int N = m->n_links, n = m->n_dof, P = S + 2;
  double nodes[16], W[8 * 16];
  om_colloc(S, nodes, W);
  pc->S = S;
  pc->n = n;
  double *H = (double *)malloc(sizeof(double) * n * n);
  om_hmass(m, q_cur, H);
  for (int j = 0; j < N; ++j) {
    int k = m->ndof[j], o = m->dof_off[j];
    double B[9] = {0}, B2[9] = {0};
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) B[a * k + b] = H[(o + a) * n + o + b];
    /* thin rods on ball joints have (near) singular blocks (no inertia about
     * the rod axis): add 1e-8 of the mean diagonal; a block with zero trace
     * (massless subtree) becomes the identity */
    double tr = 0;
    for (int a = 0; a < k; ++a) tr += B[a * k + a];
    if (tr > 0) {
      for (int a = 0; a < k; ++a) B[a * k + a] += 1e-8 * tr / k;
    } else {
      for (int a = 0; a < k * k; ++a) B[a] = (a % (k + 1) == 0) ? 1.0 : 0.0;
    }
    if (S >= 2) {
      for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) {
          double s = 0;
          for (int c = 0; c < k; ++c) s += B[a * k + c] * B[c * k + b];
          B2[a * k + b] = s;
        }
      memcpy(B, B2, sizeof(B));
    }
    inv3(B, pc->Pb + 9 * j, k);
  }
  free(H);
  if (S == 1) {
    pc->Ps[0] = dt * dt;
  } else {
    /* (What^T What)^-1 / 2 by Gauss-Jordan */
    double A[64], X[64];
    for (int a = 0; a < S; ++a)
      for (int b = 0; b < S; ++b) {
        double s = 0;
        for (int i = 0; i < S; ++i)
          s += W[i * P + 2 + a] * W[i * P + 2 + b] / (dt * dt * dt * dt);
        A[a * S + b] = s;
        X[a * S + b] = (a == b) ? 0.5 : 0.0;
      }
    for (int c = 0; c < S; ++c) {
      int piv = c;
      for (int r = c + 1; r < S; ++r)
        if (fabs(A[r * S + c]) > fabs(A[piv * S + c])) piv = r;
      for (int k = 0; k < S; ++k) {
        double t = A[c * S + k]; A[c * S + k] = A[piv * S + k]; A[piv * S + k] = t;
        t = X[c * S + k]; X[c * S + k] = X[piv * S + k]; X[piv * S + k] = t;
      }
      double d = A[c * S + c];
      for (int k = 0; k < S; ++k) { A[c * S + k] /= d; X[c * S + k] /= d; }
      for (int r = 0; r < S; ++r) {
        if (r == c) continue;
        double f = A[r * S + c];
        for (int k = 0; k < S; ++k) { A[r * S + k] -= f * A[c * S + k]; X[r * S + k] -= f * X[c * S + k]; }
      }
    }
    memcpy(pc->Ps, X, sizeof(double) * S * S);
  }
}

/* v <- P v (v: S*n, stage-major). */
static void precond_apply(const om_model *m, const om_precond *pc, double *v) {
  int S = pc->S, n = pc->n, N = m->n_links;
  double *t = (double *)malloc(sizeof(double) * S * n);
  /* stage mixing */
  for (int a = 0; a < S; ++a)
    for (int d = 0; d < n; ++d) {
      double s = 0;
      for (int b = 0; b < S; ++b) s += pc->Ps[a * S + b] * v[b * n + d];
      t[a * n + d] = s;
    }
  /* per-joint blocks */
  for (int a = 0; a < S; ++a)
    for (int j = 0; j < N; ++j) {
      int k = m->ndof[j], o = m->dof_off[j];
      for (int x = 0; x < k; ++x) {
        double s = 0;
        for (int y = 0; y < k; ++y) s += pc->Pb[9 * j + x * k + y] * t[a * n + o + y];
        v[a * n + o + x] = s;
      }
    }
  free(t);
}

/* Test access to the preconditioner: out = P v with P built at q_cur as the
 * L-BFGS solve builds it (v, out: S*n, stage-major). */
void om_precond_apply(void *p, int S, double dt, const double *q_cur, const double *v,
                      double *out) {
  om_model *m = (om_model *)p;
  om_precond pc;
  pc.Pb = (double *)malloc(sizeof(double) * 9 * m->n_links);
  lbfgs_precond(m, S, dt, q_cur, &pc);
  memcpy(out, v, sizeof(double) * S * m->n_dof);
  precond_apply(m, &pc, out);
  free(pc.Pb);
}

/* Line-search constants: Armijo c1, approximate-Wolfe delta and relative
 * energy slack (Hager & Zhang), backtracking factor and trial cap. */
#define LS_C1 1e-4
#define LS_DELTA 0.1
#define LS_EPS 1e-12
#define LS_SHRINK 0.5
#define LS_MAX 40
#define CURV_EPS 1e-14

typedef struct {
  double E;
  double *r, *g;
} om_point;

double om_eval_fast(void *p, int S, double dt, const double *qs, const double *q_prev,
                    const double *q_cur, const double *tau, double *r, double *grad);

static double eval_point(om_model *m, int S, double dt, const double *x,
                         const double *qp, const double *qc, const double *tau,
                         double *r, double *g) {
  if (m->fast && m->n_contact == 0) return om_eval_fast(m, S, dt, x, qp, qc, tau, r, g);
  return om_eval(m, S, dt, x, qp, qc, tau, r, g, NULL);
}

/* The L-BFGS search direction d = -H g by the two-loop recursion (Nocedal &
 * Wright, Algorithm 7.4) over the nh newest of the mh ring slots (newest at
 * head-1), with H0 = gamma P; P is applied in place by apply_P. sh, yh: ring
 * of pairs, [mh][Sn]; rho[j] = 1 / s_j^T y_j; alp: mh scratch.
 *
 * f32dir = 1 is the mixed-precision variant: every vector operation of the
 * recursion (the dot products, the updates, the sums) is done in binary32 on
 * binary32 copies of -g and of the pairs; H0 is applied in binary64 to the
 * binary32 vector and rounded back. rho and gamma enter rounded to binary32.
 * The result is widened to binary64. */
typedef void (*apply_fn)(void *ctx, double *v);

static float dot32(const float *a, const float *b, int n) {
  float s = 0.0f;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static void two_loop(int Sn, int nh, int mh, int head, const double *sh,
                     const double *yh, const double *rho, double gamma,
                     apply_fn apply_P, void *ctx, const double *g, int f32dir,
                     double *d, double *alp) {
  if (!f32dir) {
    for (int i = 0; i < Sn; ++i) d[i] = -g[i];
    for (int c = 0; c < nh; ++c) {
      int j = (head - 1 - c + 2 * mh) % mh;
      alp[j] = rho[j] * dot(sh + j * Sn, d, Sn);
      for (int i = 0; i < Sn; ++i) d[i] -= alp[j] * yh[j * Sn + i];
    }
    apply_P(ctx, d);
    for (int i = 0; i < Sn; ++i) d[i] *= gamma;
    for (int c = nh - 1; c >= 0; --c) {
      int j = (head - 1 - c + 2 * mh) % mh;
      double b = rho[j] * dot(yh + j * Sn, d, Sn);
      for (int i = 0; i < Sn; ++i) d[i] += (alp[j] - b) * sh[j * Sn + i];
    }
    return;
  }
  int nr = mh > 0 ? mh : 1;
  float *q = (float *)malloc(sizeof(float) * Sn);
  float *s32 = (float *)malloc(sizeof(float) * Sn * nr);
  float *y32 = (float *)malloc(sizeof(float) * Sn * nr);
  float *a32 = (float *)malloc(sizeof(float) * nr);
  for (int i = 0; i < Sn * mh; ++i) {
    s32[i] = (float)sh[i];
    y32[i] = (float)yh[i];
  }
  for (int i = 0; i < Sn; ++i) q[i] = (float)(-g[i]);
  for (int c = 0; c < nh; ++c) {
    int j = (head - 1 - c + 2 * mh) % mh;
    a32[j] = (float)rho[j] * dot32(s32 + j * Sn, q, Sn);
    for (int i = 0; i < Sn; ++i) q[i] -= a32[j] * y32[j * Sn + i];
  }
  for (int i = 0; i < Sn; ++i) d[i] = (double)q[i];
  apply_P(ctx, d);
  for (int i = 0; i < Sn; ++i) q[i] = (float)(gamma * d[i]);
  for (int c = nh - 1; c >= 0; --c) {
    int j = (head - 1 - c + 2 * mh) % mh;
    float b = (float)rho[j] * dot32(y32 + j * Sn, q, Sn);
    for (int i = 0; i < Sn; ++i) q[i] += (a32[j] - b) * s32[j * Sn + i];
  }
  for (int i = 0; i < Sn; ++i) d[i] = (double)q[i];
  for (int j = 0; j < mh; ++j) alp[j] = (double)a32[j];
  free(q); free(s32); free(y32); free(a32);
}

typedef struct {
  const om_model *m;
  const om_precond *pc;
} pc_ctx;

static void apply_pc(void *ctx, double *v) {
  pc_ctx *c = (pc_ctx *)ctx;
  precond_apply(c->m, c->pc, v);
}

typedef struct {
  int n;
  const double *P;
} dense_ctx;

static void apply_dense(void *ctx, double *v) {
  dense_ctx *c = (dense_ctx *)ctx;
  double *t = (double *)malloc(sizeof(double) * c->n);
  for (int a = 0; a < c->n; ++a) {
    double s = 0;
    for (int b = 0; b < c->n; ++b) s += c->P[a * c->n + b] * v[b];
    t[a] = s;
  }
  memcpy(v, t, sizeof(double) * c->n);
  free(t);
}

/* Test entry: two_loop with a dense H0 factor P (Sn x Sn, row-major). */
void om_lbfgs_direction(int Sn, int nh, int mh, int head, const double *sh,
                        const double *yh, const double *rho, double gamma,
                        const double *P, const double *g, int f32dir,
                        double *d) {
  dense_ctx c = {Sn, P};
  double *alp = (double *)malloc(sizeof(double) * (mh > 0 ? mh : 1));
  two_loop(Sn, nh, mh, head, sh, yh, rho, gamma, apply_dense, &c, g, f32dir, d, alp);
  free(alp);
}

/* One step of L-BFGS with history mh. x: in = initial guess, out = result.
 * Returns the status; *iters = accepted iterations, *evals = evaluations.
 * Besides max_iter accepted iterations, a step may use at most
 * 4 max_iter + LS_MAX objective evaluations (line-search trials included);
 * reaching either cap gives MAX_ITER. */
static int lbfgs_solve(om_model *m, int S, double dt, const double *qp,
                       const double *qc, const double *tau, int mh, double tol,
                       int max_iter, int use_precond, int f32dir, double *x,
                       int *iters, int *evals, double *rn_exit) {
  int n = m->n_dof, Sn = S * n;
  double *g = (double *)malloc(sizeof(double) * Sn);
  double *r = (double *)malloc(sizeof(double) * Sn);
  double *d = (double *)malloc(sizeof(double) * Sn);
  double *xt = (double *)malloc(sizeof(double) * Sn);
  double *gt = (double *)malloc(sizeof(double) * Sn);
  double *rt = (double *)malloc(sizeof(double) * Sn);
  double *Py = (double *)malloc(sizeof(double) * Sn);
  double *sh = (double *)malloc(sizeof(double) * Sn * (mh > 0 ? mh : 1));
  double *yh = (double *)malloc(sizeof(double) * Sn * (mh > 0 ? mh : 1));
  double *rho = (double *)malloc(sizeof(double) * (mh > 0 ? mh : 1));
  double *alp = (double *)malloc(sizeof(double) * (mh > 0 ? mh : 1));
  int nh = 0, head = 0; /* ring buffer: newest at (head-1) mod mh */
  double gamma = 1.0;
  int status = OM_MAX_ITER;
  int k = 0, ne = 0;

  om_precond pc;
  pc.Pb = (double *)malloc(sizeof(double) * 9 * m->n_links);
  if (use_precond) {
    lbfgs_precond(m, S, dt, qc, &pc);
  } else {
    pc.S = S; pc.n = n;
    memset(pc.Ps, 0, sizeof(pc.Ps));
    for (int a = 0; a < S; ++a) pc.Ps[a * S + a] = 1.0;
    for (int j = 0; j < m->n_links; ++j) {
      int k = m->ndof[j];
      for (int x = 0; x < 9; ++x) pc.Pb[9 * j + x] = 0;
      for (int x = 0; x < k; ++x) pc.Pb[9 * j + x * k + x] = 1.0;
    }
  }
  double E = eval_point(m, S, dt, x, qp, qc, tau, r, g);
  ne++;
  for (;;) {
    if (!isfinite(E) || !all_finite(g, Sn)) { status = OM_NONFINITE; break; }
    if (sqrt(dot(r, r, Sn)) < tol) { status = OM_CONVERGED; break; }
    if (k >= max_iter) { status = OM_MAX_ITER; break; }
    pc_ctx pctx = {m, &pc};
    two_loop(Sn, nh, mh, head, sh, yh, rho, gamma, apply_pc, &pctx, g, f32dir, d, alp);
    double gd = dot(g, d, Sn);
    if (!(gd < 0)) {
      /* not a descent direction: restart from the scaled gradient */
      nh = 0;
      gamma = 1.0;
      for (int i = 0; i < Sn; ++i) d[i] = -g[i];
      precond_apply(m, &pc, d);
      gd = dot(g, d, Sn);
      if (!(gd < 0)) {
        /* -P g is not a descent direction either (P not positive definite
         * in rounding): steepest descent */
        for (int i = 0; i < Sn; ++i) d[i] = -g[i];
        gd = dot(g, d, Sn);
      }
    }
    /* backtracking line search with Armijo or approximate-Wolfe acceptance */
    double a = 1.0;
    int accepted = 0, capped = 0;
    double Et = 0;
    for (int t = 0; t < LS_MAX; ++t) {
      if (ne >= 4 * max_iter + LS_MAX) { capped = 1; break; }
      for (int i = 0; i < Sn; ++i) xt[i] = x[i] + a * d[i];
      Et = eval_point(m, S, dt, xt, qp, qc, tau, rt, gt);
      ne++;
      if (isfinite(Et) && all_finite(gt, Sn)) {
        double gtd = dot(gt, d, Sn);
        int armijo = Et <= E + LS_C1 * a * gd;
        int approx = (Et <= E + LS_EPS * fabs(E)) &&
                     (gtd <= (1 - 2 * LS_DELTA) * fabs(gd));
        if (armijo || approx) { accepted = 1; break; }
      }
      a *= LS_SHRINK;
    }
    if (capped) { status = OM_MAX_ITER; break; }
    if (!accepted) {
      double rn = sqrt(dot(r, r, Sn));
      status = rn <= STALL_FACTOR * om_floor(m, S, dt) ? OM_STALLED : OM_LS_FAIL;
      break;
    }
    /* curvature pair */
    double sy = 0, ss = 0, yy = 0, yPy = 0;
    for (int i = 0; i < Sn; ++i) {
      double s_ = xt[i] - x[i], y_ = gt[i] - g[i];
      sy += s_ * y_; ss += s_ * s_; yy += y_ * y_;
      Py[i] = y_;
    }
    precond_apply(m, &pc, Py);
    for (int i = 0; i < Sn; ++i) yPy += (gt[i] - g[i]) * Py[i];
    if (mh > 0 && sy > CURV_EPS * sqrt(ss) * sqrt(yy)) {
      for (int i = 0; i < Sn; ++i) {
        sh[head * Sn + i] = xt[i] - x[i];
        yh[head * Sn + i] = gt[i] - g[i];
        if (f32dir) { /* the pairs are kept in binary32 */
          sh[head * Sn + i] = (double)(float)sh[head * Sn + i];
          yh[head * Sn + i] = (double)(float)yh[head * Sn + i];
        }
      }
      rho[head] = 1.0 / sy;
      head = (head + 1) % mh;
      if (nh < mh) nh++;
      gamma = sy / yPy;
    }
    memcpy(x, xt, sizeof(double) * Sn);
    memcpy(g, gt, sizeof(double) * Sn);
    memcpy(r, rt, sizeof(double) * Sn);
    E = Et;
    k++;
  }
  *iters = k;
  *evals = ne;
  if (rn_exit) *rn_exit = sqrt(dot(r, r, Sn));
  free(g); free(r); free(d); free(xt); free(gt); free(rt); free(Py); free(pc.Pb);
  free(sh); free(yh); free(rho); free(alp);
  return status;
}

/* One step of Levenberg-Marquardt (Section 5):
 *   q <- q - [H + lambda I]^-1 grad,
 * H = Jr^T Jr and grad = Jr^T r for S >= 2 (Eq. EQHOC, sum of squares);
 * H = Hmass/dt^2 (Gauss-Newton of the integral of squares) and grad = dE/dq
 * for S == 1. lambda starts at 1e-12 max diag(H). A damped step that does
 * not lower E is halved up to LM_HALVINGS times before lambda is multiplied
 * by 10 (a failed factorisation multiplies it at once); lambda is divided by
 * 10 (floor 1e-20 max diag(H)) after a full damped step is accepted and kept
 * after a halved one. The paper only asks that lambda keep E decreasing; the
 * small start and floor keep lambda below the smallest eigenvalues of
 * Jr^T Jr, whose condition number reaches 1e12-1e16 for thin links on ball
 * joints, and the halvings keep it there when the full Gauss-Newton step
 * overshoots along the stiff modes (raising lambda instead would damp the
 * soft modes by orders of magnitude and make the iteration crawl). */
#define LM_HALVINGS 3
static int lm_solve(om_model *m, int S, double dt, const double *qp,
                    const double *qc, const double *tau, double tol,
                    int max_iter, double *x, int *iters, int *evals,
                    double *rn_exit) {
  int n = m->n_dof, Sn = S * n;
  double *r = (double *)malloc(sizeof(double) * Sn);
  double *rt = (double *)malloc(sizeof(double) * Sn);
  double *J = (double *)malloc(sizeof(double) * Sn * Sn);
  double *H = (double *)malloc(sizeof(double) * Sn * Sn);
  double *A = (double *)malloc(sizeof(double) * Sn * Sn);
  double *gr = (double *)malloc(sizeof(double) * Sn);
  double *dx = (double *)malloc(sizeof(double) * Sn);
  double *xt = (double *)malloc(sizeof(double) * Sn);
  double *Hm = (double *)malloc(sizeof(double) * n * n);
  int status = OM_MAX_ITER, k = 0, ne = 0;
  double lambda = -1;
  double E = om_eval(m, S, dt, x, qp, qc, tau, r, NULL, J);
  ne++;
  for (;;) {
    if (!isfinite(E) || !all_finite(r, Sn)) { status = OM_NONFINITE; break; }
    double rn = sqrt(dot(r, r, Sn));
    if (rn < tol) { status = OM_CONVERGED; break; }
    if (k >= max_iter) { status = OM_MAX_ITER; break; }
    if (S == 1) {
      /* Gauss-Newton matrix of Eq. EQ (+ Q_drag): (1 + 2 c) H_mass / dt^2,
       * plus sum_p dP/dq^T (d2Q/dP2) dP/dq of the contact points (Eq. FRI) */
      om_hmass(m, x, Hm);
      for (int i = 0; i < Sn * Sn; ++i) H[i] = (1.0 + 2.0 * m->drag) * Hm[i] / (dt * dt);
      contact_gn(m, dt, x, qc, H);
      for (int i = 0; i < Sn; ++i) gr[i] = r[i];
    } else {
      for (int a = 0; a < Sn; ++a)
        for (int b = 0; b < Sn; ++b) {
          double s = 0;
          for (int c = 0; c < Sn; ++c) s += J[c * Sn + a] * J[c * Sn + b];
          H[a * Sn + b] = s;
        }
      for (int a = 0; a < Sn; ++a) {
        double s = 0;
        for (int c = 0; c < Sn; ++c) s += J[c * Sn + a] * r[c];
        gr[a] = s;
      }
    }
    double hmax = 0;
    for (int i = 0; i < Sn; ++i) hmax = fmax(hmax, H[i * Sn + i]);
    if (lambda < 0) lambda = 1e-12 * hmax;
    int accepted = 0, last_chol_fail = 0;
    double a = 1.0; /* fraction of the damped step that was accepted */
    for (int t = 0; t < 60; ++t) {
      memcpy(A, H, sizeof(double) * Sn * Sn);
      for (int i = 0; i < Sn; ++i) A[i * Sn + i] += lambda;
      last_chol_fail = 0;
      if (cholesky(A, Sn) != 0) { lambda *= 10; last_chol_fail = 1; continue; }
      for (int i = 0; i < Sn; ++i) dx[i] = -gr[i];
      chol_solve(A, Sn, dx);
      /* the damped step, then its halves down to 1/8, before a larger lambda */
      a = 1.0;
      for (int h = 0; h <= LM_HALVINGS; ++h) {
        for (int i = 0; i < Sn; ++i) xt[i] = x[i] + a * dx[i];
        double Et = om_eval(m, S, dt, xt, qp, qc, tau, rt, NULL, NULL);
        ne++;
        int ok = isfinite(Et) && all_finite(rt, Sn) &&
                 (Et < E || (S == 1 && Et <= E + LS_EPS * fabs(E) &&
                             dot(rt, rt, Sn) < rn * rn));
        if (ok) { accepted = 1; E = Et; break; }
        a *= 0.5;
      }
      if (accepted) break;
      lambda *= 10;
    }
    if (!accepted) {
      if (last_chol_fail) status = OM_CHOL_FAIL;
      else status = rn <= STALL_FACTOR * om_floor(m, S, dt) ? OM_STALLED : OM_LS_FAIL;
      break;
    }
    if (a == 1.0) lambda = fmax(lambda * 0.1, 1e-20 * hmax);
    memcpy(x, xt, sizeof(double) * Sn);
    E = om_eval(m, S, dt, x, qp, qc, tau, r, NULL, J);
    k++;
  }
  *iters = k;
  *evals = ne;
  if (rn_exit) *rn_exit = sqrt(dot(r, r, Sn));
  free(r); free(rt); free(J); free(H); free(A); free(gr); free(dx); free(xt); free(Hm);
  return status;
}

/* One time step: solve for the S stage configurations.
 *   solver 0 = LBFGS (history mh), 1 = LM, 2 = LBFGS with the binary32
 *   search direction (two_loop, f32dir). qs_out: S*n.
 * Returns the status code. */
int om_step(void *p, int S, double dt, const double *q_prev,
            const double *q_cur, const double *tau, int solver, int mh,
            double tol, int max_iter, int use_precond, double *qs_out,
            int *iters, int *evals, double *rn_exit) {
  om_model *m = (om_model *)p;
  initial_guess(S, m->n_dof, q_prev, q_cur, qs_out);
  if (solver == 0 || solver == 2)
    return lbfgs_solve(m, S, dt, q_prev, q_cur, tau, mh, tol, max_iter,
                       use_precond, solver == 2, qs_out, iters, evals, rn_exit);
  return lm_solve(m, S, dt, q_prev, q_cur, tau, tol, max_iter, qs_out, iters,
                  evals, rn_exit);
}

/* Rollout of n_steps steps. State after each step: q_prev' = stage S-1 (or
 * q_cur for S == 1, the node k-1+alpha_{S-1} of the next step), q_cur' =
 * stage S. tau_seq: [n_steps][n]. traj_prev/traj_cur (optional):
 * [n_steps][n] states after each step. Returns the worst status over the
 * steps (om_status_worse order); iters: total accepted iterations;
 * step_status / step_rnorm (optional, [n_steps]): each step's status and the
 * |r|_2 of the point it ended at. */
int om_rollout(void *p, int S, double dt, const double *q_prev0,
               const double *q_cur0, const double *tau_seq, int n_steps,
               int solver, int mh, double tol, int max_iter, int use_precond,
               double *traj_prev, double *traj_cur, double *q_prev_out,
               double *q_cur_out, int *iters_total, int *evals_total,
               int *step_status, double *step_rnorm) {
  om_model *m = (om_model *)p;
  int n = m->n_dof;
  double *qp = (double *)malloc(sizeof(double) * n);
  double *qc = (double *)malloc(sizeof(double) * n);
  double *qs = (double *)malloc(sizeof(double) * n * S);
  memcpy(qp, q_prev0, sizeof(double) * n);
  memcpy(qc, q_cur0, sizeof(double) * n);
  int worst = 0, it_tot = 0, ev_tot = 0;
  for (int s = 0; s < n_steps; ++s) {
    int it = 0, ev = 0;
    double rn = 0;
    int st = om_step(p, S, dt, qp, qc, tau_seq + (size_t)s * n, solver, mh, tol,
                     max_iter, use_precond, qs, &it, &ev, &rn);
    worst = om_status_worse(worst, st);
    if (step_status) step_status[s] = st;
    if (step_rnorm) step_rnorm[s] = rn;
    it_tot += it;
    ev_tot += ev;
    if (S == 1) memcpy(qp, qc, sizeof(double) * n);
    else memcpy(qp, qs + (S - 2) * n, sizeof(double) * n);
    memcpy(qc, qs + (S - 1) * n, sizeof(double) * n);
    if (traj_prev) memcpy(traj_prev + (size_t)s * n, qp, sizeof(double) * n);
    if (traj_cur) memcpy(traj_cur + (size_t)s * n, qc, sizeof(double) * n);
  }
  if (q_prev_out) memcpy(q_prev_out, qp, sizeof(double) * n);
  if (q_cur_out) memcpy(q_cur_out, qc, sizeof(double) * n);
  if (iters_total) *iters_total = it_tot;
  if (evals_total) *evals_total = ev_tot;
  free(qp); free(qc); free(qs);
  return worst;
}

/* ------------------------------------------------------------------ */
/* implicit-function-theorem adjoint of one converged step             */
/* ------------------------------------------------------------------ */

/* At a converged step r(q_*; q_prev, q_cur, tau) = 0, so
 * dq_* = -Jr^-1 (dr/dtheta) dtheta. Given gbar = dL/dq_* (S*n), returns
 * gq_prev = -(dr/dq_prev)^T mu, gq_cur = -(dr/dq_cur)^T mu and
 * gtau = sum_i mu_i, with Jr^T mu = gbar (dense LU). Returns 0 on success. */
int om_step_adjoint(void *p, int S, double dt, const double *q_prev,
                    const double *q_cur, const double *tau, const double *qs,
                    const double *gbar, double *gq_prev, double *gq_cur,
                    double *gtau) {
  om_model *m = (om_model *)p;
  int n = m->n_dof, Sn = S * n;
  double *J = (double *)malloc(sizeof(double) * Sn * Sn);
  double *JT = (double *)malloc(sizeof(double) * Sn * Sn);
  double *mu = (double *)malloc(sizeof(double) * Sn);
  double *Jp = (double *)malloc(sizeof(double) * Sn * n);
  double *Jc = (double *)malloc(sizeof(double) * Sn * n);
  om_eval(p, S, dt, qs, q_prev, q_cur, tau, NULL, NULL, J);
  for (int a = 0; a < Sn; ++a)
    for (int b = 0; b < Sn; ++b) JT[a * Sn + b] = J[b * Sn + a];
  memcpy(mu, gbar, sizeof(double) * Sn);
  int rc = lu_solve(JT, Sn, mu);
  om_resid_known_jac(p, S, dt, qs, q_prev, q_cur, Jp, Jc);
  for (int e = 0; e < n; ++e) {
    double sp = 0, sc = 0, st = 0;
    for (int k = 0; k < Sn; ++k) {
      sp += Jp[k * n + e] * mu[k];
      sc += Jc[k * n + e] * mu[k];
    }
    for (int i = 0; i < S; ++i) st += mu[i * n + e];
    gq_prev[e] = -sp;
    gq_cur[e] = -sc;
    gtau[e] = st;
  }
  free(J); free(JT); free(mu); free(Jp); free(Jc);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Newton-Euler reference (Eq. DYN_EXP) for hinge trees: RNEA + RK4     */
/* ------------------------------------------------------------------ */

static void cross3(const double *a, const double *b, double *c) {
  double t0 = a[1] * b[2] - a[2] * b[1];
  double t1 = a[2] * b[0] - a[0] * b[2];
  double t2 = a[0] * b[1] - a[1] * b[0];
  c[0] = t0; c[1] = t1; c[2] = t2;
}

/* Recursive Newton-Euler inverse dynamics for hinge-only trees, with spatial
 * vectors (angular; linear at the world origin) in world coordinates:
 * tau_out = M(q) qdd + C(q, qd) qd - Q_gravity(q). Returns -1 for ball
 * joints. */
int om_rnea(void *p, const double *q, const double *qd, const double *qdd,
            double *tau_out) {
  om_model *m = (om_model *)p;
  int N = m->n_links;
  for (int l = 0; l < N; ++l)
    if (m->jtype[l] != 0) return -1;
  double *T = (double *)malloc(sizeof(double) * 16 * N);
  double *v = (double *)malloc(sizeof(double) * 6 * N);
  double *a = (double *)malloc(sizeof(double) * 6 * N);
  double *f = (double *)malloc(sizeof(double) * 6 * N);
  double *s = (double *)malloc(sizeof(double) * 6 * N);
  om_fk(p, q, T);
  for (int l = 0; l < N; ++l) {
    /* world axis and a point on it (joint origin = link origin) */
    double *Tl = T + 16 * l;
    double u[3], o[3];
    const double *ax = m->axis + 3 * l;
    for (int i = 0; i < 3; ++i) {
      u[i] = Tl[4 * i + 0] * ax[0] + Tl[4 * i + 1] * ax[1] + Tl[4 * i + 2] * ax[2];
      o[i] = Tl[4 * i + 3];
    }
    double lin[3];
    cross3(o, u, lin); /* velocity at the world origin of a unit spin about (o,u) */
    s[6 * l + 0] = u[0]; s[6 * l + 1] = u[1]; s[6 * l + 2] = u[2];
    s[6 * l + 3] = lin[0]; s[6 * l + 4] = lin[1]; s[6 * l + 5] = lin[2];
    int pa = m->parent[l];
    double vp[6] = {0, 0, 0, 0, 0, 0};
    double ap[6] = {0, 0, 0, -m->g[0], -m->g[1], -m->g[2]}; /* base accel = -g */
    if (pa >= 0) {
      memcpy(vp, v + 6 * pa, sizeof(vp));
      memcpy(ap, a + 6 * pa, sizeof(ap));
    }
    int d = m->dof_off[l];
    for (int i = 0; i < 6; ++i) v[6 * l + i] = vp[i] + s[6 * l + i] * qd[d];
    /* a = a_p + s qdd + v x s qd (spatial motion cross product) */
    double *sl = s + 6 * l, *vl = v + 6 * l;
    double cw[3], cv1[3], cv2[3];
    cross3(vl, sl, cw);
    cross3(vl, sl + 3, cv1);
    cross3(vl + 3, sl, cv2);
    for (int i = 0; i < 3; ++i) {
      a[6 * l + i] = ap[i] + sl[i] * qdd[d] + cw[i] * qd[d];
      a[6 * l + 3 + i] = ap[3 + i] + sl[3 + i] * qdd[d] + (cv1[i] + cv2[i]) * qd[d];
    }
    /* spatial inertia at the world origin from the world mass moments:
     * first moment h = m c (world), rotational inertia about the origin
     * I_O = tr(Sigma_w) Id - Sigma_w, Sigma_w = R Sigma R^T + R mc t^T + t mc^T R^T + m t t^T */
    const double *mm = m->mm + 10 * l;
    double Sig[9] = {mm[0], mm[1], mm[2], mm[1], mm[3], mm[4], mm[2], mm[4], mm[5]};
    double mcl[3] = {mm[6], mm[7], mm[8]}, ms = mm[9];
    double R[9], t[3];
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) R[3 * i + j] = Tl[4 * i + j];
      t[i] = Tl[4 * i + 3];
    }
    double RS[9], RSRt[9], Rt[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Rt[3 * i + j] = R[3 * j + i];
    m3_mul(R, Sig, RS);
    m3_mul(RS, Rt, RSRt);
    double Rmc[3];
    for (int i = 0; i < 3; ++i) Rmc[i] = R[3 * i] * mcl[0] + R[3 * i + 1] * mcl[1] + R[3 * i + 2] * mcl[2];
    double h[3], Sw[9];
    for (int i = 0; i < 3; ++i) h[i] = Rmc[i] + ms * t[i];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        Sw[3 * i + j] = RSRt[3 * i + j] + Rmc[i] * t[j] + t[i] * Rmc[j] + ms * t[i] * t[j];
    double trS = Sw[0] + Sw[4] + Sw[8];
    double IO[9];
    for (int i = 0; i < 9; ++i) IO[i] = -Sw[i];
    IO[0] += trS; IO[4] += trS; IO[8] += trS;
    /* momentum-like products: I*x for x = (w, vO): n = IO w + h x vO, p = m vO - h x w */
    double *al = a + 6 * l;
    double n1[3], hx[3], p1[3], hw[3];
    for (int i = 0; i < 3; ++i) n1[i] = IO[3 * i] * al[0] + IO[3 * i + 1] * al[1] + IO[3 * i + 2] * al[2];
    cross3(h, al + 3, hx);
    cross3(h, al, hw);
    for (int i = 0; i < 3; ++i) { n1[i] += hx[i]; p1[i] = ms * al[3 + i] - hw[i]; }
    double n2[3], p2[3], hv[3], hw2[3];
    for (int i = 0; i < 3; ++i) n2[i] = IO[3 * i] * vl[0] + IO[3 * i + 1] * vl[1] + IO[3 * i + 2] * vl[2];
    cross3(h, vl + 3, hv);
    cross3(h, vl, hw2);
    for (int i = 0; i < 3; ++i) { n2[i] += hv[i]; p2[i] = ms * vl[3 + i] - hw2[i]; }
    /* v x* (I v): force cross product (w x n + vO x p, w x p) */
    double c1[3], c2[3], c3[3];
    cross3(vl, n2, c1);
    cross3(vl + 3, p2, c2);
    cross3(vl, p2, c3);
    for (int i = 0; i < 3; ++i) {
      f[6 * l + i] = n1[i] + c1[i] + c2[i];
      f[6 * l + 3 + i] = p1[i] + c3[i];
    }
  }
  for (int l = N - 1; l >= 0; --l) {
    tau_out[m->dof_off[l]] = dot(s + 6 * l, f + 6 * l, 6);
    int pa = m->parent[l];
    if (pa >= 0)
      for (int i = 0; i < 6; ++i) f[6 * pa + i] += f[6 * l + i];
  }
  free(T); free(v); free(a); free(f); free(s);
  return 0;
}

/* qdd = M^-1 (tau - bias) with M built column by column from RNEA. */
static int fd_accel(void *p, const double *q, const double *qd,
                    const double *tau, double *qdd) {
  om_model *m = (om_model *)p;
  int n = m->n_dof;
  double *Mm = (double *)malloc(sizeof(double) * n * n);
  double *z = (double *)calloc(n, sizeof(double));
  double *e = (double *)calloc(n, sizeof(double));
  double *col = (double *)malloc(sizeof(double) * n);
  double *bias = (double *)malloc(sizeof(double) * n);
  double *b0 = (double *)malloc(sizeof(double) * n);
  double g0[3] = {m->g[0], m->g[1], m->g[2]};
  int rc = om_rnea(p, q, qd, z, bias);
  if (rc == 0) {
    m->g[0] = m->g[1] = m->g[2] = 0;
    om_rnea(p, q, z, z, b0);
    for (int j = 0; j < n; ++j) {
      memset(e, 0, sizeof(double) * n);
      e[j] = 1;
      om_rnea(p, q, z, e, col);
      for (int i = 0; i < n; ++i) Mm[i * n + j] = col[i] - b0[i];
    }
    m->g[0] = g0[0]; m->g[1] = g0[1]; m->g[2] = g0[2];
    for (int i = 0; i < n; ++i) qdd[i] = tau[i] - bias[i];
    rc = lu_solve(Mm, n, qdd);
  }
  free(Mm); free(z); free(e); free(col); free(bias); free(b0);
  return rc;
}

/* Classical RK4 on (q, qd) with constant tau, n_steps of size h. */
int om_rk4(void *p, double *q, double *qd, const double *tau, double h,
           int n_steps) {
  om_model *m = (om_model *)p;
  int n = m->n_dof;
  double *k1q = (double *)malloc(sizeof(double) * n * 12);
  double *k1v = k1q + n, *k2q = k1q + 2 * n, *k2v = k1q + 3 * n;
  double *k3q = k1q + 4 * n, *k3v = k1q + 5 * n, *k4q = k1q + 6 * n;
  double *k4v = k1q + 7 * n, *tq = k1q + 8 * n, *tv = k1q + 9 * n;
  int rc = 0;
  for (int s = 0; s < n_steps && rc == 0; ++s) {
    memcpy(k1q, qd, sizeof(double) * n);
    rc |= fd_accel(p, q, qd, tau, k1v);
    for (int i = 0; i < n; ++i) { tq[i] = q[i] + 0.5 * h * k1q[i]; tv[i] = qd[i] + 0.5 * h * k1v[i]; }
    memcpy(k2q, tv, sizeof(double) * n);
    rc |= fd_accel(p, tq, tv, tau, k2v);
    for (int i = 0; i < n; ++i) { tq[i] = q[i] + 0.5 * h * k2q[i]; tv[i] = qd[i] + 0.5 * h * k2v[i]; }
    memcpy(k3q, tv, sizeof(double) * n);
    rc |= fd_accel(p, tq, tv, tau, k3v);
    for (int i = 0; i < n; ++i) { tq[i] = q[i] + h * k3q[i]; tv[i] = qd[i] + h * k3v[i]; }
    memcpy(k4q, tv, sizeof(double) * n);
    rc |= fd_accel(p, tq, tv, tau, k4v);
    for (int i = 0; i < n; ++i) {
      q[i] += h / 6 * (k1q[i] + 2 * k2q[i] + 2 * k3q[i] + k4q[i]);
      qd[i] += h / 6 * (k1v[i] + 2 * k2v[i] + 2 * k3v[i] + k4v[i]);
    }
  }
  free(k1q);
  return rc;
}
