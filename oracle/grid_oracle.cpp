// FP64 CPU oracle for GRiD's dynamics path (RNEA, M, M^-1, FD, dRNEA, dFD).
//
// TEST INFRASTRUCTURE ONLY. Only the tests, the package smoke check and the
// benchmark's CPU-baseline leg may load this library. It shares no code, header
// or table with the CUDA path; both sides read the same raw model arrays
// produced by grid_inputs.
//
// Everything is written as plainly as possible: dense 6x6 spatial matrices,
// textbook recursions, no blocking or fusion. Spatial vectors are ordered
// [angular; linear] as in Eq. (2). Every routine is templated on the scalar so
// that the same code also runs in std::complex<double> for complex-step
// differentiation (all operations used are analytic: +, -, *, /, sin, cos,
// sqrt away from its branch cut; no conjugation, no abs).
//
// Paper sections cited: Sec. III-B (Eq. (1) manipulator equation, frames with
// parent lambda_i < i, transforms iX_lambda from rotation and translation,
// spatial inertia I_i, motion subspace S_i, Eq. (2) cross operators);
// Sec. IV-B (the five algorithms: RNEA, M^-1, FD, dRNEA, dFD);
// Alg. 1 (dRNEA forward pass and its backward pass).
//
// Readings of the paper used here (listed with the others in the design notes):
//  * FD is qdd = +M^-1 (tau - RNEA(q, qd, 0)) (the printed leading minus sign in
//    Sec. IV-B is read as garbled; RNEA(q, qd, FD(q, qd, tau)) = tau pins it).
//  * In Alg. 1 the term "dv_lambda/du x S_i qd_i" is read as dv_i/du x S_i qd_i
//    (product rule on v_i x S_i qd_i).
//  * The case terms of Alg. 1 apply only in the column of joint i itself.
//  * The backward-pass term X^T (S_i x* f_i) uses the accumulated force f_i
//    (own plus children) and applies only for u = q_i.
//  * Gravity enters as a fictitious base acceleration a_0 = -g.
//  * iX_lambda = X_J(q_i) X_T,i. Joint types (Sec. IV-B lists revolute,
//    prismatic and fixed joints among the supported URDF joints): revolute X_J
//    is a coordinate rotation by q_i about the unit axis a_i, S_i = [a_i; 0];
//    prismatic X_J is a translation of the child origin by q_i a_i,
//    S_i = [0; a_i]; a fixed joint has X_J = 1 and no degree of freedom. Joint
//    arrays (q, qd, qdd, tau) hold the moving joints only, in body order.
#include <array>
#include <cmath>
#include <complex>
#include <cstring>
#include <thread>
#include <vector>

namespace {

template <class T> using V3 = std::array<T, 3>;
template <class T> using V6 = std::array<T, 6>;
template <class T> using M3 = std::array<std::array<T, 3>, 3>;
template <class T> using M6 = std::array<std::array<T, 6>, 6>;

template <class T> V6<T> zero6() { V6<T> r; for (auto& x : r) x = T(0); return r; }
template <class T> M6<T> zero66() { M6<T> r; for (auto& row : r) for (auto& x : row) x = T(0); return r; }

template <class T> V6<T> add(const V6<T>& a, const V6<T>& b) {
  V6<T> r; for (int k = 0; k < 6; ++k) r[k] = a[k] + b[k]; return r;
}
template <class T> V6<T> scale(const V6<T>& a, T s) {
  V6<T> r; for (int k = 0; k < 6; ++k) r[k] = a[k] * s; return r;
}
template <class T> T dot(const V6<T>& a, const V6<T>& b) {
  T s = T(0); for (int k = 0; k < 6; ++k) s += a[k] * b[k]; return s;
}
template <class T> V6<T> mul(const M6<T>& A, const V6<T>& x) {
  V6<T> r; for (int i = 0; i < 6; ++i) { T s = T(0); for (int k = 0; k < 6; ++k) s += A[i][k] * x[k]; r[i] = s; }
  return r;
}
template <class T> M6<T> mul(const M6<T>& A, const M6<T>& B) {
  M6<T> C; for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) {
    T s = T(0); for (int k = 0; k < 6; ++k) s += A[i][k] * B[k][j]; C[i][j] = s; }
  return C;
}
template <class T> M6<T> transpose(const M6<T>& A) {
  M6<T> B; for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) B[i][j] = A[j][i]; return B;
}
template <class T> M6<T> add(const M6<T>& A, const M6<T>& B) {
  M6<T> C; for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) C[i][j] = A[i][j] + B[i][j]; return C;
}
template <class T> V6<T> mulT(const M6<T>& A, const V6<T>& x) { return mul(transpose(A), x); }

// Eq. (2): the motion cross-product matrix v x, written entry by entry.
template <class T> M6<T> crm(const V6<T>& v) {
  M6<T> m = zero66<T>();
  m[0][1] = -v[2]; m[0][2] =  v[1];
  m[1][0] =  v[2]; m[1][2] = -v[0];
  m[2][0] = -v[1]; m[2][1] =  v[0];
  m[3][1] = -v[5]; m[3][2] =  v[4]; m[3][4] = -v[2]; m[3][5] =  v[1];
  m[4][0] =  v[5]; m[4][2] = -v[3]; m[4][3] =  v[2]; m[4][5] = -v[0];
  m[5][0] = -v[4]; m[5][1] =  v[3]; m[5][3] = -v[1]; m[5][4] =  v[0];
  return m;
}
// Eq. (2): the force cross-product matrix v x* = -(v x)^T.
template <class T> M6<T> crf(const V6<T>& v) {
  M6<T> m = transpose(crm(v));
  for (auto& row : m) for (auto& x : row) x = -x;
  return m;
}

template <class T> M3<T> skew(const V3<T>& p) {
  M3<T> s;
  s[0][0] = T(0);  s[0][1] = -p[2]; s[0][2] =  p[1];
  s[1][0] =  p[2]; s[1][1] = T(0);  s[1][2] = -p[0];
  s[2][0] = -p[1]; s[2][1] =  p[0]; s[2][2] = T(0);
  return s;
}
template <class T> M3<T> mul3(const M3<T>& A, const M3<T>& B) {
  M3<T> C; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) {
    T s = T(0); for (int k = 0; k < 3; ++k) s += A[i][k] * B[k][j]; C[i][j] = s; }
  return C;
}

// Plucker transform for motion vectors from frame A to frame B, where E maps
// A-coordinates to B-coordinates and r is B's origin expressed in A:
// X = [E 0; -E r~ E] (Featherstone, Rigid Body Dynamics Algorithms, eq. 2.24).
template <class T> M6<T> plucker(const M3<T>& E, const V3<T>& r) {
  M6<T> X = zero66<T>();
  M3<T> Erx = mul3(E, skew(r));
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) {
    X[i][j] = E[i][j];
    X[i + 3][j + 3] = E[i][j];
    X[i + 3][j] = -Erx[i][j];
  }
  return X;
}

// Coordinate rotation by angle q about unit axis a: E = R(a, q)^T where
// R(a, q) = cos q 1 + (1 - cos q) a a^T + sin q a~ (Rodrigues).
template <class T> M3<T> joint_E(const V3<double>& a, T q) {
  T c = std::cos(q), s = std::sin(q);
  M3<T> R;
  V3<T> at = {T(a[0]), T(a[1]), T(a[2])};
  M3<T> ax = skew(at);
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j)
    R[i][j] = (i == j ? c : T(0)) + (T(1) - c) * at[i] * at[j] + s * ax[i][j];
  M3<T> E; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) E[i][j] = R[j][i];
  return E;
}

// Spatial inertia about the link origin from mass m, COM c and rotational
// inertia Ic about the COM: [Ic + m c~ c~^T, m c~; m c~^T, m 1]
// (Featherstone eq. 2.63).
M6<double> spatial_inertia(const double* p) {
  double m = p[0];
  V3<double> c = {p[1], p[2], p[3]};
  M3<double> Ic = {{{p[4], p[7], p[8]}, {p[7], p[5], p[9]}, {p[8], p[9], p[6]}}};
  M3<double> C = skew(c);
  M6<double> I = zero66<double>();
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) {
    double cct = 0; for (int k = 0; k < 3; ++k) cct += C[i][k] * C[j][k];
    I[i][j] = Ic[i][j] + m * cct;
    I[i][j + 3] = m * C[i][j];
    I[i + 3][j] = m * C[j][i];
    I[i + 3][j + 3] = (i == j) ? m : 0.0;
  }
  return I;
}

enum { REVOLUTE = 0, PRISMATIC = 1, FIXED = 2 };

struct Model {
  int n = 0;                    // bodies
  int nd = 0;                   // degrees of freedom (moving joints)
  std::vector<int> parent;
  std::vector<int> jtype;       // REVOLUTE, PRISMATIC or FIXED
  std::vector<int> dof;         // body -> joint index, -1 for a fixed joint
  std::vector<V3<double>> axis;
  std::vector<M6<double>> XT;   // fixed transforms X_T,i
  std::vector<M6<double>> I;    // spatial inertias
  V6<double> a0;                // base acceleration -g
};

bool build_model(int n, const int* parent, const int* jtype, const double* axis, const double* xtree,
                 const double* inertia, const double* gravity, Model& m) {
  if (n <= 0) return false;
  m.n = n;
  m.parent.assign(parent, parent + n);
  m.jtype.assign(n, REVOLUTE);
  m.dof.assign(n, -1);
  m.nd = 0;
  m.axis.resize(n); m.XT.resize(n); m.I.resize(n);
  for (int i = 0; i < n; ++i) {
    if (parent[i] < -1 || parent[i] >= i) return false;   // Sec. III-B: lambda_i < i
    if (jtype) {
      if (jtype[i] < REVOLUTE || jtype[i] > FIXED) return false;
      m.jtype[i] = jtype[i];
    }
    if (m.jtype[i] != FIXED) m.dof[i] = m.nd++;
    m.axis[i] = {axis[3 * i], axis[3 * i + 1], axis[3 * i + 2]};
    M3<double> E; V3<double> r;
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) E[a][b] = xtree[12 * i + 3 * a + b];
    for (int a = 0; a < 3; ++a) r[a] = xtree[12 * i + 9 + a];
    m.XT[i] = plucker(E, r);
    m.I[i] = spatial_inertia(inertia + 10 * i);
  }
  m.a0 = {0, 0, 0, -gravity[0], -gravity[1], -gravity[2]};
  return m.nd > 0;
}

template <class T> M6<T> cast66(const M6<double>& A) {
  M6<T> B; for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) B[i][j] = T(A[i][j]); return B;
}
template <class T> V6<T> cast6(const V6<double>& a) {
  V6<T> b; for (int i = 0; i < 6; ++i) b[i] = T(a[i]); return b;
}
// S_i: [a; 0] for a revolute joint, [0; a] for a prismatic one (unused for a
// fixed joint, which has no degree of freedom).
template <class T> V6<T> motion_subspace(const Model& m, int i) {
  const T a0 = T(m.axis[i][0]), a1 = T(m.axis[i][1]), a2 = T(m.axis[i][2]);
  if (m.jtype[i] == PRISMATIC) return {T(0), T(0), T(0), a0, a1, a2};
  return {a0, a1, a2, T(0), T(0), T(0)};
}

// iX_lambda_i = X_J(q_i) X_T,i  (Sec. III-B).
template <class T> std::vector<M6<T>> transforms(const Model& m, const T* q) {
  std::vector<M6<T>> X(m.n);
  const M3<T> I3 = {{{T(1), T(0), T(0)}, {T(0), T(1), T(0)}, {T(0), T(0), T(1)}}};
  for (int i = 0; i < m.n; ++i) {
    M6<T> XJ;
    if (m.jtype[i] == REVOLUTE) {
      XJ = plucker(joint_E<T>(m.axis[i], q[m.dof[i]]), V3<T>{T(0), T(0), T(0)});
    } else if (m.jtype[i] == PRISMATIC) {
      const T d = q[m.dof[i]];
      XJ = plucker(I3, V3<T>{d * T(m.axis[i][0]), d * T(m.axis[i][1]), d * T(m.axis[i][2])});
    } else {
      XJ = plucker(I3, V3<T>{T(0), T(0), T(0)});
    }
    X[i] = mul(XJ, cast66<T>(m.XT[i]));
  }
  return X;
}

template <class T> struct RneaOut {
  std::vector<M6<T>> X;
  std::vector<V6<T>> v, a, f, F;   // f: own body force, F: accumulated over subtree
  std::vector<T> tau;
};

// Recursive Newton-Euler (Sec. IV-B, after Featherstone ch. 5):
// forward  v_i = X v_lambda + S qd_i,
//          a_i = X a_lambda + S qdd_i + v_i x S qd_i,  (a_base = -g, v_base = 0)
//          f_i = I a_i + v_i x* I v_i;
// backward tau_i = S^T F_i,  F_lambda += X^T F_i.
// (A fixed joint contributes no S terms and no tau entry.)
template <class T> RneaOut<T> rnea(const Model& m, const T* q, const T* qd, const T* qdd) {
  RneaOut<T> o;
  o.X = transforms<T>(m, q);
  o.v.resize(m.n); o.a.resize(m.n); o.f.resize(m.n); o.F.resize(m.n); o.tau.resize(m.nd);
  for (int i = 0; i < m.n; ++i) {
    int p = m.parent[i];
    V6<T> vp = p < 0 ? zero6<T>() : o.v[p];
    V6<T> ap = p < 0 ? cast6<T>(m.a0) : o.a[p];
    o.v[i] = mul(o.X[i], vp);
    o.a[i] = mul(o.X[i], ap);
    if (m.dof[i] >= 0) {
      V6<T> S = motion_subspace<T>(m, i);
      const int d = m.dof[i];
      o.v[i] = add(o.v[i], scale(S, qd[d]));
      o.a[i] = add(add(o.a[i], scale(S, qdd[d])), mul(crm(o.v[i]), scale(S, qd[d])));
    }
    M6<T> I = cast66<T>(m.I[i]);
    o.f[i] = add(mul(I, o.a[i]), mul(crf(o.v[i]), mul(I, o.v[i])));
    o.F[i] = o.f[i];
  }
  for (int i = m.n - 1; i >= 0; --i) {
    if (m.dof[i] >= 0) o.tau[m.dof[i]] = dot(motion_subspace<T>(m, i), o.F[i]);
    int p = m.parent[i];
    if (p >= 0) o.F[p] = add(o.F[p], mulT(o.X[i], o.F[i]));
  }
  return o;
}

// Joint-space mass matrix by the composite-rigid-body algorithm
// (Featherstone ch. 6): Ic_lambda += X^T Ic_i X, M_ii = S^T Ic_i S,
// off-diagonal entries by transporting F = Ic_i S_i towards the root.
template <class T> std::vector<T> crba(const Model& m, const T* q) {
  std::vector<M6<T>> X = transforms<T>(m, q);
  std::vector<M6<T>> Ic(m.n);
  for (int i = 0; i < m.n; ++i) Ic[i] = cast66<T>(m.I[i]);
  for (int i = m.n - 1; i >= 0; --i) {
    int p = m.parent[i];
    if (p >= 0) Ic[p] = add(Ic[p], mul(transpose(X[i]), mul(Ic[i], X[i])));
  }
  const int nd = m.nd;
  std::vector<T> M(nd * nd, T(0));
  for (int i = 0; i < m.n; ++i) {
    if (m.dof[i] < 0) continue;
    const int di = m.dof[i];
    V6<T> F = mul(Ic[i], motion_subspace<T>(m, i));
    M[di * nd + di] = dot(motion_subspace<T>(m, i), F);
    int j = i;
    while (m.parent[j] >= 0) {
      F = mulT(X[j], F);
      j = m.parent[j];
      if (m.dof[j] < 0) continue;
      const int dj = m.dof[j];
      T Mij = dot(motion_subspace<T>(m, j), F);
      M[di * nd + dj] = Mij;
      M[dj * nd + di] = Mij;
    }
  }
  return M;
}

template <class T> double re(const T& x) { return std::real(std::complex<double>(x)); }
template <> double re<double>(const double& x) { return x; }

// Cholesky M = L L^T (lower), non-conjugating so it stays analytic.
template <class T> bool cholesky(int n, const std::vector<T>& M, std::vector<T>& L) {
  L.assign(n * n, T(0));
  for (int j = 0; j < n; ++j) {
    T d = M[j * n + j];
    for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    if (!(re(d) > 0.0)) return false;
    T ljj = std::sqrt(d);
    L[j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      T s = M[i * n + j];
      for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = s / ljj;
    }
  }
  return true;
}

// Solve L L^T x = b in place.
template <class T> void chol_solve(int n, const std::vector<T>& L, T* x) {
  for (int i = 0; i < n; ++i) {
    T s = x[i];
    for (int k = 0; k < i; ++k) s -= L[i * n + k] * x[k];
    x[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    T s = x[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
    x[i] = s / L[i * n + i];
  }
}

// M^-1 = L^-T L^-1, computed column by column as the solution of M x = e_j.
template <class T> bool minv(const Model& m, const T* q, std::vector<T>& Mi) {
  const int nd = m.nd;
  std::vector<T> M = crba<T>(m, q), L;
  if (!cholesky<T>(nd, M, L)) return false;
  Mi.assign(nd * nd, T(0));
  std::vector<T> x(nd);
  for (int j = 0; j < nd; ++j) {
    for (int i = 0; i < nd; ++i) x[i] = T(i == j ? 1 : 0);
    chol_solve<T>(nd, L, x.data());
    for (int i = 0; i < nd; ++i) Mi[i * nd + j] = x[i];
  }
  return true;
}

// FD: qdd = M^-1 (tau - RNEA(q, qd, 0)) (Sec. IV-B), by a Cholesky solve.
template <class T> bool fd(const Model& m, const T* q, const T* qd, const T* tau, T* qdd) {
  std::vector<T> zero(m.nd, T(0));
  RneaOut<T> r = rnea<T>(m, q, qd, zero.data());
  std::vector<T> M = crba<T>(m, q), L;
  if (!cholesky<T>(m.nd, M, L)) return false;
  for (int i = 0; i < m.nd; ++i) qdd[i] = tau[i] - r.tau[i];
  chol_solve<T>(m.nd, L, qdd);
  return true;
}

// Analytical RNEA derivatives, one column per joint (Alg. 1 forward pass and
// its backward pass), at (q, qd, qdd). Outputs row-major nd x nd:
// dtau_dq[i*nd + j] = d tau_i / d q_j, likewise for qd. Column j belongs to the
// body bj whose joint is j; a fixed joint passes derivatives through its
// transform and has no case terms, row or column.
template <class T> void grad_rnea(const Model& m, const T* q, const T* qd, const T* qdd,
                                  T* dtau_dq, T* dtau_dqd) {
  const int n = m.n, nd = m.nd;
  RneaOut<T> r = rnea<T>(m, q, qd, qdd);
  std::vector<V6<T>> dv(n), da(n), df(n);
  for (int u = 0; u < 2; ++u) {                 // u = 0: d/dq, u = 1: d/dqd
    T* out = u == 0 ? dtau_dq : dtau_dqd;
    for (int bj = 0; bj < n; ++bj) {
      if (m.dof[bj] < 0) continue;
      const int j = m.dof[bj];
      // forward pass over frames i = 1..n
      for (int i = 0; i < n; ++i) {
        int p = m.parent[i];
        V6<T> dvp = p < 0 ? zero6<T>() : dv[p];
        V6<T> dap = p < 0 ? zero6<T>() : da[p];
        V6<T> vp = p < 0 ? zero6<T>() : r.v[p];
        V6<T> ap = p < 0 ? cast6<T>(m.a0) : r.a[p];
        dv[i] = mul(r.X[i], dvp);
        da[i] = mul(r.X[i], dap);
        if (m.dof[i] >= 0) {
          V6<T> S = motion_subspace<T>(m, i);
          if (i == bj) dv[i] = add(dv[i], u == 0 ? mul(crm(mul(r.X[i], vp)), S) : S);
          da[i] = add(da[i], mul(crm(dv[i]), scale(S, qd[m.dof[i]])));
          if (i == bj) da[i] = add(da[i], u == 0 ? mul(crm(mul(r.X[i], ap)), S) : mul(crm(r.v[i]), S));
        }
        M6<T> I = cast66<T>(m.I[i]);
        df[i] = add(add(mul(I, da[i]), mul(crf(dv[i]), mul(I, r.v[i]))),
                    mul(crf(r.v[i]), mul(I, dv[i])));
      }
      // backward pass over frames i = n..1
      for (int i = n - 1; i >= 0; --i) {
        if (m.dof[i] >= 0) out[m.dof[i] * nd + j] = dot(motion_subspace<T>(m, i), df[i]);
        int p = m.parent[i];
        if (p >= 0) {
          V6<T> up = mulT(r.X[i], df[i]);
          if (u == 0 && i == bj) up = add(up, mulT(r.X[i], mul(crf(motion_subspace<T>(m, i)), r.F[i])));
          df[p] = add(df[p], up);
        }
      }
    }
  }
}

// dFD: [dqdd/dq | dqdd/dqd] = -M^-1 [dID/dq | dID/dqd] at qdd = FD(q, qd, tau)
// (Sec. IV-B). J is row-major n x 2n.
template <class T> bool grad_fd(const Model& m, const T* q, const T* qd, const T* tau, T* J, T* qdd_out) {
  const int n = m.nd;
  std::vector<T> qdd(n);
  if (!fd<T>(m, q, qd, tau, qdd.data())) return false;
  std::vector<T> dq(n * n), dqd(n * n), Mi;
  grad_rnea<T>(m, q, qd, qdd.data(), dq.data(), dqd.data());
  if (!minv<T>(m, q, Mi)) return false;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      T s1 = T(0), s2 = T(0);
      for (int k = 0; k < n; ++k) { s1 += Mi[i * n + k] * dq[k * n + j]; s2 += Mi[i * n + k] * dqd[k * n + j]; }
      J[i * 2 * n + j] = -s1;
      J[i * 2 * n + n + j] = -s2;
    }
  if (qdd_out) for (int i = 0; i < n; ++i) qdd_out[i] = qdd[i];
  return true;
}

// Run f(k) for k in [0, N) on nthreads host threads; returns the first error.
template <class F> int parallel_for(int N, int nthreads, F f) {
  if (nthreads <= 1 || N <= 1) { for (int k = 0; k < N; ++k) { int e = f(k); if (e) return e; } return 0; }
  if (nthreads > N) nthreads = N;
  std::vector<int> err(nthreads, 0);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t] {
      for (int k = t; k < N; k += nthreads) { int e = f(k); if (e) { err[t] = e; return; } }
    });
  for (auto& x : th) x.join();
  for (int e : err) if (e) return e;
  return 0;
}

using C = std::complex<double>;

}  // namespace

// n is the number of bodies; jtype may be NULL (all revolute). Joint arrays
// have nd = (number of non-fixed joints) entries per knot point.
#define ORACLE_MODEL_ARGS int nb, const int* parent, const int* jtype, const double* axis, \
                          const double* xtree, const double* inertia, const double* gravity
#define ORACLE_BUILD Model m; if (!build_model(nb, parent, jtype, axis, xtree, inertia, gravity, m)) return 1; \
                     const int n = m.nd;

extern "C" {

// Status: 0 ok, 1 invalid model, 2 mass matrix not positive definite.

int oracle_rnea(ORACLE_MODEL_ARGS, int N, const double* q, const double* qd, const double* qdd,
                double* tau, int nthreads) {
  ORACLE_BUILD
  return parallel_for(N, nthreads, [&](int k) {
    RneaOut<double> r = rnea<double>(m, q + k * n, qd + k * n, qdd + k * n);
    for (int i = 0; i < n; ++i) tau[k * n + i] = r.tau[i];
    return 0;
  });
}

int oracle_mass_matrix(ORACLE_MODEL_ARGS, int N, const double* q, double* M, int nthreads) {
  ORACLE_BUILD
  return parallel_for(N, nthreads, [&](int k) {
    std::vector<double> Mk = crba<double>(m, q + k * n);
    std::memcpy(M + (size_t)k * n * n, Mk.data(), sizeof(double) * n * n);
    return 0;
  });
}

int oracle_minv(ORACLE_MODEL_ARGS, int N, const double* q, double* Minv, int nthreads) {
  ORACLE_BUILD
  return parallel_for(N, nthreads, [&](int k) {
    std::vector<double> Mi;
    if (!minv<double>(m, q + k * n, Mi)) return 2;
    std::memcpy(Minv + (size_t)k * n * n, Mi.data(), sizeof(double) * n * n);
    return 0;
  });
}

int oracle_fd(ORACLE_MODEL_ARGS, int N, const double* q, const double* qd, const double* tau,
              double* qdd, int nthreads) {
  ORACLE_BUILD
  return parallel_for(N, nthreads, [&](int k) {
    return fd<double>(m, q + k * n, qd + k * n, tau + k * n, qdd + k * n) ? 0 : 2;
  });
}

int oracle_grad_rnea(ORACLE_MODEL_ARGS, int N, const double* q, const double* qd, const double* qdd,
                     double* dtau_dq, double* dtau_dqd, int nthreads) {
  ORACLE_BUILD
  return parallel_for(N, nthreads, [&](int k) {
    grad_rnea<double>(m, q + k * n, qd + k * n, qdd + k * n,
                      dtau_dq + (size_t)k * n * n, dtau_dqd + (size_t)k * n * n);
    return 0;
  });
}

int oracle_grad_fd(ORACLE_MODEL_ARGS, int N, const double* q, const double* qd, const double* tau,
                   double* J, double* qdd, int nthreads) {
  ORACLE_BUILD
  return parallel_for(N, nthreads, [&](int k) {
    return grad_fd<double>(m, q + k * n, qd + k * n, tau + k * n, J + (size_t)k * 2 * n * n,
                           qdd ? qdd + k * n : nullptr) ? 0 : 2;
  });
}

// Complex-step derivatives of FD: J_cs[i][j] = Im(FD_i(q + i h e_j, qd, tau)) / h
// and J_cs[i][n + j] likewise for qd. Independent of the analytical route.
int oracle_fd_complex_step(ORACLE_MODEL_ARGS, int N, const double* q, const double* qd,
                           const double* tau, double h, double* J, int nthreads) {
  ORACLE_BUILD
  return parallel_for(N, nthreads, [&](int k) {
    std::vector<C> qc(n), qdc(n), tc(n), out(n);
    for (int u = 0; u < 2; ++u)
      for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) {
          qc[i] = C(q[k * n + i], 0); qdc[i] = C(qd[k * n + i], 0); tc[i] = C(tau[k * n + i], 0);
        }
        (u == 0 ? qc : qdc)[j] += C(0, h);
        if (!fd<C>(m, qc.data(), qdc.data(), tc.data(), out.data())) return 2;
        for (int i = 0; i < n; ++i) J[(size_t)k * 2 * n * n + i * 2 * n + u * n + j] = out[i].imag() / h;
      }
    return 0;
  });
}

// Complex-step derivatives of RNEA w.r.t. q and qd at fixed qdd.
int oracle_rnea_complex_step(ORACLE_MODEL_ARGS, int N, const double* q, const double* qd,
                             const double* qdd, double h, double* dtau_dq, double* dtau_dqd,
                             int nthreads) {
  ORACLE_BUILD
  return parallel_for(N, nthreads, [&](int k) {
    std::vector<C> qc(n), qdc(n), qddc(n);
    for (int u = 0; u < 2; ++u)
      for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) {
          qc[i] = C(q[k * n + i], 0); qdc[i] = C(qd[k * n + i], 0); qddc[i] = C(qdd[k * n + i], 0);
        }
        (u == 0 ? qc : qdc)[j] += C(0, h);
        RneaOut<C> r = rnea<C>(m, qc.data(), qdc.data(), qddc.data());
        double* out = (u == 0 ? dtau_dq : dtau_dqd) + (size_t)k * n * n;
        for (int i = 0; i < n; ++i) out[i * n + j] = r.tau[i].imag() / h;
      }
    return 0;
  });
}

}  // extern "C"
