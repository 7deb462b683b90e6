// Host-side model construction: validation, depth-first renumbering, device
// constants and the per-lane schedules of the derivative-column phase.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "grid_internal.h"

static thread_local char g_err[512] = "";

void grid_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

extern "C" const char* grid_last_error(void) { return g_err; }

namespace {

struct Unit {            // one root-to-leaf path of one derivative column
  std::vector<uint32_t> steps;
};

// ---- fixed-joint merging (host, FP64)
// Compact transform records Er = E (3x3 row-major) then r (3): X = [E 0; -E r~ E].
// X(A) X(B) = X(E_A E_B, r_B + E_B^T r_A) (B applied first).
void compose(const double* A, const double* B, double* out) {
  double o[12];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      o[3 * i + j] = s;
    }
  for (int i = 0; i < 3; ++i) {
    double s = B[9 + i];
    for (int k = 0; k < 3; ++k) s += B[3 * k + i] * A[9 + k];
    o[9 + i] = s;
  }
  std::memcpy(out, o, sizeof(o));
}

void plucker6(const double* Er, double X[6][6]) {
  const double* r = Er + 9;
  const double rx[3][3] = {{0, -r[2], r[1]}, {r[2], 0, -r[0]}, {-r[1], r[0], 0}};
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) X[i][j] = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      X[i][j] = X[i + 3][j + 3] = Er[3 * i + j];
      double s = 0;
      for (int k = 0; k < 3; ++k) s += Er[3 * i + k] * rx[k][j];
      X[i + 3][j] = -s;
    }
}

// (m, c, Ic) -> 6x6 spatial inertia about the body origin, and back.
void spatial_from_params(const double* p, double I[6][6]) {
  const double m = p[0], c[3] = {p[1], p[2], p[3]};
  const double Ic[3][3] = {{p[4], p[7], p[8]}, {p[7], p[5], p[9]}, {p[8], p[9], p[6]}};
  const double cx[3][3] = {{0, -c[2], c[1]}, {c[2], 0, -c[0]}, {-c[1], c[0], 0}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double cct = 0;
      for (int k = 0; k < 3; ++k) cct += cx[i][k] * cx[j][k];
      I[i][j] = Ic[i][j] + m * cct;
      I[i][j + 3] = m * cx[i][j];
      I[i + 3][j] = m * cx[j][i];
      I[i + 3][j + 3] = i == j ? m : 0.0;
    }
}

void params_from_spatial(const double I[6][6], double* p) {
  const double m = I[3][3];
  const double c[3] = {I[2][4] / m, I[0][5] / m, I[1][3] / m};   // m c~ is the upper-right block
  const double cx[3][3] = {{0, -c[2], c[1]}, {c[2], 0, -c[0]}, {-c[1], c[0], 0}};
  double Ic[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double cct = 0;
      for (int k = 0; k < 3; ++k) cct += cx[i][k] * cx[j][k];
      Ic[i][j] = I[i][j] - m * cct;
    }
  p[0] = m; p[1] = c[0]; p[2] = c[1]; p[3] = c[2];
  p[4] = Ic[0][0]; p[5] = Ic[1][1]; p[6] = Ic[2][2];
  p[7] = 0.5 * (Ic[0][1] + Ic[1][0]); p[8] = 0.5 * (Ic[0][2] + Ic[2][0]); p[9] = 0.5 * (Ic[1][2] + Ic[2][1]);
}

struct Reduced {
  int n = 0;
  std::vector<int> parent, jt;
  std::vector<double> axis, X_tree, inertia;
};

// Every fixed joint is merged into its nearest moving ancestor (or the base):
// the fixed body's spatial inertia, expressed in the ancestor's frame (X^T I X),
// is added to the ancestor's, and bodies hanging from it take the composed
// fixed transform. What remains has one degree of freedom per body; joint
// arrays index the moving joints in body order.
grid_status merge_fixed(int nb, const int* parent, const int* jtype, const double* axis,
                        const double* X_tree, const double* inertia, Reduced& R) {
  std::vector<int> anchor(nb, -1), newidx(nb, -1);
  std::vector<std::array<double, 12>> toanchor(nb);        // X from the anchor's frame to body f's
  std::vector<std::array<double, 36>> I6(nb);
  for (int i = 0; i < nb; ++i) {
    double I[6][6];
    spatial_from_params(inertia + 10 * i, I);
    std::memcpy(I6[i].data(), I, sizeof(I));
  }
  for (int i = 0; i < nb; ++i) {
    const int p = parent[i];
    const bool pfixed = p >= 0 && jtype && jtype[p] == GRID_JOINT_FIXED;
    const int host = pfixed ? anchor[p] : p;                // moving body (or -1) this one hangs from
    double Xt[12];
    std::memcpy(Xt, X_tree + 12 * i, sizeof(Xt));
    if (pfixed) compose(X_tree + 12 * i, toanchor[p].data(), Xt);
    if (jtype && jtype[i] == GRID_JOINT_FIXED) {
      anchor[i] = host;
      std::memcpy(toanchor[i].data(), Xt, sizeof(Xt));
      if (host >= 0) {                                      // I_host += X^T I_i X
        double X[6][6], I[6][6], T[6][6];
        plucker6(Xt, X);
        std::memcpy(I, I6[i].data(), sizeof(I));
        for (int a = 0; a < 6; ++a)
          for (int b = 0; b < 6; ++b) {
            double s = 0;
            for (int k = 0; k < 6; ++k) s += I[a][k] * X[k][b];
            T[a][b] = s;
          }
        for (int a = 0; a < 6; ++a)
          for (int b = 0; b < 6; ++b) {
            double s = 0;
            for (int k = 0; k < 6; ++k) s += X[k][a] * T[k][b];
            I6[host][6 * a + b] += s;
          }
      }
      continue;
    }
    newidx[i] = R.n++;
    R.parent.push_back(host < 0 ? -1 : newidx[host]);
    R.jt.push_back(jtype ? jtype[i] : GRID_JOINT_REVOLUTE);
    for (int a = 0; a < 3; ++a) R.axis.push_back(axis[3 * i + a]);
    for (int a = 0; a < 12; ++a) R.X_tree.push_back(Xt[a]);
  }
  R.inertia.resize(10 * R.n);
  for (int i = 0; i < nb; ++i)
    if (newidx[i] >= 0) {
      double I[6][6];
      std::memcpy(I, I6[i].data(), sizeof(I));
      params_from_spatial(I, R.inertia.data() + 10 * newidx[i]);
    }
  return GRID_OK;
}

}  // namespace

static grid_status build_moving(int n, const int* parent, const int* jt, const double* axis,
                                const double* X_tree, const double* inertia, const double* gravity,
                                ModelDev<float>* mf, ModelDev<double>* md);

grid_status grid_build_model(int nb, const int* parent, const int* jtype, const double* axis,
                             const double* X_tree, const double* inertia, const double* gravity,
                             ModelDev<float>* mf, ModelDev<double>* md) {
  if (nb < 1 || nb > GRID_MAX_BODIES) {
    grid_set_error("grid_create: %d bodies outside [1, %d]", nb, GRID_MAX_BODIES);
    return GRID_E_TOPOLOGY;
  }
  if (!parent || !axis || !X_tree || !inertia || !gravity) {
    grid_set_error("grid_create: null model array");
    return GRID_E_ARG;
  }
  for (int i = 0; i < nb; ++i) {
    if (parent[i] < -1 || parent[i] >= i) {
      grid_set_error("grid_create: parent[%d] = %d violates -1 <= parent[i] < i", i, parent[i]);
      return GRID_E_TOPOLOGY;
    }
    if (jtype && (jtype[i] < GRID_JOINT_REVOLUTE || jtype[i] > GRID_JOINT_FIXED)) {
      grid_set_error("grid_create: joint type %d of body %d is not 0, 1 or 2", jtype[i], i);
      return GRID_E_ARG;
    }
    if (jtype && jtype[i] == GRID_JOINT_FIXED && !(inertia[10 * i] >= 0.0)) {
      grid_set_error("grid_create: fixed body %d has mass %g (must be >= 0)", i, inertia[10 * i]);
      return GRID_E_NUMERIC;
    }
  }
  Reduced R;
  grid_status st = merge_fixed(nb, parent, jtype, axis, X_tree, inertia, R);
  if (st != GRID_OK) return st;
  if (R.n == 0) {
    grid_set_error("grid_create: every joint is fixed (no degree of freedom)");
    return GRID_E_TOPOLOGY;
  }
  return build_moving(R.n, R.parent.data(), R.jt.data(), R.axis.data(), R.X_tree.data(), R.inertia.data(),
                      gravity, mf, md);
}

static grid_status build_moving(int n, const int* parent, const int* jt, const double* axis,
                                const double* X_tree, const double* inertia, const double* gravity,
                                ModelDev<float>* mf, ModelDev<double>* md) {
  if (n < 1 || n > GRID_MAX_DOF) {
    grid_set_error("grid_create: %d degrees of freedom outside [1, %d]", n, GRID_MAX_DOF);
    return GRID_E_TOPOLOGY;
  }
  for (int i = 0; i < n; ++i) {
    if (parent[i] < -1 || parent[i] >= i) {
      grid_set_error("grid_create: parent[%d] = %d violates -1 <= parent[i] < i", i, parent[i]);
      return GRID_E_TOPOLOGY;
    }
    double an = std::sqrt(axis[3 * i] * axis[3 * i] + axis[3 * i + 1] * axis[3 * i + 1] +
                          axis[3 * i + 2] * axis[3 * i + 2]);
    if (!(std::fabs(an - 1.0) < 1e-6)) {
      grid_set_error("grid_create: axis %d has norm %g (must be unit)", i, an);
      return GRID_E_NUMERIC;
    }
    if (!(inertia[10 * i] > 0.0)) {
      grid_set_error("grid_create: body %d has mass %g (must be > 0)", i, inertia[10 * i]);
      return GRID_E_NUMERIC;
    }
  }
  // Depth-first preorder: children in caller order, roots in caller order.
  std::vector<std::vector<int>> kids(n);
  std::vector<int> roots;
  for (int i = 0; i < n; ++i) (parent[i] < 0 ? roots : kids[parent[i]]).push_back(i);
  std::vector<int> perm;          // internal -> caller
  std::vector<int> stack(roots.rbegin(), roots.rend());
  while (!stack.empty()) {
    int b = stack.back();
    stack.pop_back();
    perm.push_back(b);
    for (auto it = kids[b].rbegin(); it != kids[b].rend(); ++it) stack.push_back(*it);
  }
  std::vector<int> inv(n);
  for (int k = 0; k < n; ++k) inv[perm[k]] = k;

  ModelDev<double>& D = *md;
  std::memset(&D, 0, sizeof(D));
  D.n = n;
  std::vector<int> par(n), dep(n), send(n), clo(n), chi(n);
  for (int k = 0; k < n; ++k) {
    int p = parent[perm[k]];
    par[k] = p < 0 ? -1 : inv[p];
    dep[k] = par[k] < 0 ? 0 : dep[par[k]] + 1;
  }
  for (int k = n - 1; k >= 0; --k) {
    send[k] = k + 1;
    for (int m = k + 1; m < n && dep[m] > dep[k]; ++m) send[k] = m + 1;
  }
  int ncomp = 0;
  for (int k = 0; k < n; ++k) {
    if (par[k] < 0) { ++ncomp; clo[k] = k; chi[k] = send[k]; }
    else { clo[k] = clo[par[k]]; chi[k] = chi[par[k]]; }
  }
  int maxd = 0, nsk = 0, nbranch = 0;
  for (int k = 0; k < n; ++k) {
    maxd = std::max(maxd, dep[k] + 1);
    D.skoff[k] = nsk;
    nsk += dep[k] + 1;                      // ancestor subspaces (gravity rows live in the union)
    int nk = 0;
    for (int m = k + 1; m < n; ++m) nk += par[m] == k;
    D.branch[k] = nk >= 2 ? nbranch++ : -1;
  }
  D.maxd = maxd; D.nsk = nsk; D.ncomp = ncomp; D.nbranch = nbranch;
  if (nsk > 1023) {
    grid_set_error("grid_create: subspace table of %d rows exceeds the step descriptor", nsk);
    return GRID_E_TOPOLOGY;
  }
  D.ld = n;
  D.gmask = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
  for (int k = 0; k < n; ++k) {
    D.gslot[k] = k;
    D.gidx[k] = perm[k];
  }
  for (int k = 0; k < n; ++k) {
    int c = perm[k];
    D.parent[k] = par[k]; D.depth[k] = dep[k]; D.sub_end[k] = send[k];
    D.comp_lo[k] = clo[k]; D.comp_hi[k] = chi[k]; D.perm[k] = c;
    for (int a = 0; a < 3; ++a) D.axis[k][a] = axis[3 * c + a];
    bool ident = true;
    for (int a = 0; a < 9; ++a) {
      D.ET[k][a] = X_tree[12 * c + a];
      double e = (a % 4 == 0) ? 1.0 : 0.0;
      if (X_tree[12 * c + a] != e) ident = false;
    }
    D.et_ident[k] = ident ? 1 : 0;
    D.jt[k] = jt[c];
    if (jt[c] == GRID_JOINT_PRISMATIC) D.any_prism = 1;
    for (int a = 0; a < 3; ++a) D.rT[k][a] = X_tree[12 * c + 9 + a];
    // Spatial inertia about the body origin in compact form: mass m,
    // first moment h = m c, rotational inertia Ibar = Ic + m (c.c 1 - c c^T).
    const double* p = inertia + 10 * c;
    double m = p[0], cx = p[1], cy = p[2], cz = p[3];
    double cc = cx * cx + cy * cy + cz * cz;
    D.inert[k][0] = m;
    D.inert[k][1] = m * cx; D.inert[k][2] = m * cy; D.inert[k][3] = m * cz;
    D.inert[k][4] = p[4] + m * (cc - cx * cx);
    D.inert[k][5] = p[5] + m * (cc - cy * cy);
    D.inert[k][6] = p[6] + m * (cc - cz * cz);
    D.inert[k][7] = p[7] - m * cx * cy;
    D.inert[k][8] = p[8] - m * cx * cz;
    D.inert[k][9] = p[9] - m * cy * cz;
    // full 6x6 spatial inertia [Ibar h~; h~^T m1], stored by columns
    const double* in = D.inert[k];
    const double h[3] = {in[1], in[2], in[3]};
    const double Ib[3][3] = {{in[4], in[7], in[8]}, {in[7], in[5], in[9]}, {in[8], in[9], in[6]}};
    const double hx[3][3] = {{0, -h[2], h[1]}, {h[2], 0, -h[0]}, {-h[1], h[0], 0}};
    double I6[6][6];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        I6[a][b] = Ib[a][b];
        I6[a][b + 3] = hx[a][b];
        I6[a + 3][b] = hx[b][a];
        I6[a + 3][b + 3] = a == b ? m : 0.0;
      }
    for (int col = 0; col < 6; ++col)
      for (int row = 0; row < 6; ++row) D.Icol[k][col][row] = I6[row][col];
  }
  D.a0[0] = D.a0[1] = D.a0[2] = 0.0;
  D.a0[3] = -gravity[0]; D.a0[4] = -gravity[1]; D.a0[5] = -gravity[2];

  // Derivative-column work units: every root-to-leaf path of subtree(j), for
  // u in {q, qd} and every joint j. The first path through a body owns it.
  std::vector<Unit> units;
  for (int u = 0; u < 2; ++u)
    for (int j = 0; j < n; ++j) {
      std::vector<char> owned(n, 0);
      for (int leaf = j; leaf < send[j]; ++leaf) {
        bool is_leaf = (leaf + 1 >= send[j]) || dep[leaf + 1] <= dep[leaf];
        if (!is_leaf) continue;
        std::vector<int> path;
        for (int b = leaf; b != par[j]; b = par[b]) path.push_back(b);
        std::reverse(path.begin(), path.end());
        Unit un;
        for (size_t s = 0; s < path.size(); ++s) {
          int b = path[s];
          uint32_t d = (uint32_t)b | ((uint32_t)(u * n + j) << 5) | STEP_VALID |
                       ((uint32_t)dep[b] << 17) | ((uint32_t)D.skoff[b] << 22);
          if (s == 0) d |= STEP_RESET | STEP_ROOT;
          if (!owned[b]) { d |= STEP_OWNED; owned[b] = 1; }
          if (s + 1 == path.size()) d |= STEP_FLUSH;
          if (u == 0) d |= STEP_UQ;
          un.steps.push_back(d);
        }
        units.push_back(un);
      }
    }
  // Longest-processing-time assignment of paths to lanes, per lane count.
  std::vector<int> order(units.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return units[a].steps.size() > units[b].steps.size(); });
  int soff = 0;
  const int lanes_cfg[GRID_NUM_LANE_CFG] = {8, 16, 32};
  for (int c = 0; c < GRID_NUM_LANE_CFG; ++c) {
    int T = lanes_cfg[c];
    std::vector<std::vector<uint32_t>> lane(T);
    for (int ui : order) {
      int best = 0;
      for (int l = 1; l < T; ++l)
        if (lane[l].size() < lane[best].size()) best = l;
      lane[best].insert(lane[best].end(), units[ui].steps.begin(), units[ui].steps.end());
    }
    int S = 0;
    for (auto& v : lane) S = std::max(S, (int)v.size());
    if (soff + S * T > GRID_SCHED_MAX) {
      grid_set_error("grid_create: derivative schedule too large (%d steps)", soff + S * T);
      return GRID_E_TOPOLOGY;
    }
    D.steps[c] = S;
    D.sched_off[c] = soff;
    for (int s = 0; s < S; ++s)
      for (int l = 0; l < T; ++l)
        D.sched[soff + s * T + l] = s < (int)lane[l].size() ? lane[l][s] : 0u;
    soff += S * T;
  }
  D.L = make_layout(n, nsk, nbranch, 8, 0);
  D.LS = make_layout(n, nsk, nbranch, 8, 1);
  D.LV = make_layout(n, nsk, nbranch, 8, 2);

  // Float copy of everything; its own layout.
  ModelDev<float>& F = *mf;
  std::memset(&F, 0, sizeof(F));
  F.n = D.n; F.maxd = D.maxd; F.nsk = D.nsk; F.ncomp = D.ncomp; F.nbranch = D.nbranch;
  F.any_prism = D.any_prism;
  std::memcpy(F.jt, D.jt, sizeof(D.jt));
  std::memcpy(F.steps, D.steps, sizeof(D.steps));
  std::memcpy(F.sched_off, D.sched_off, sizeof(D.sched_off));
  std::memcpy(F.parent, D.parent, sizeof(D.parent));
  std::memcpy(F.depth, D.depth, sizeof(D.depth));
  std::memcpy(F.sub_end, D.sub_end, sizeof(D.sub_end));
  std::memcpy(F.comp_lo, D.comp_lo, sizeof(D.comp_lo));
  std::memcpy(F.comp_hi, D.comp_hi, sizeof(D.comp_hi));
  std::memcpy(F.perm, D.perm, sizeof(D.perm));
  std::memcpy(F.skoff, D.skoff, sizeof(D.skoff));
  std::memcpy(F.branch, D.branch, sizeof(D.branch));
  std::memcpy(F.et_ident, D.et_ident, sizeof(D.et_ident));
  F.ld = D.ld;
  F.gmask = D.gmask;
  std::memcpy(F.gslot, D.gslot, sizeof(D.gslot));
  std::memcpy(F.gidx, D.gidx, sizeof(D.gidx));
  std::memcpy(F.sched, D.sched, sizeof(D.sched));
  for (int k = 0; k < GRID_MAX_DOF; ++k) {
    for (int a = 0; a < 4; ++a) F.axis[k][a] = (float)D.axis[k][a];
    for (int a = 0; a < 3; ++a) F.rT[k][a] = (float)D.rT[k][a];
    for (int a = 0; a < 9; ++a) F.ET[k][a] = (float)D.ET[k][a];
    for (int a = 0; a < 12; ++a) F.inert[k][a] = (float)D.inert[k][a];
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 8; ++b) F.Icol[k][a][b] = (float)D.Icol[k][a][b];
  }
  for (int a = 0; a < 8; ++a) F.a0[a] = (float)D.a0[a];
  F.L = make_layout(n, nsk, nbranch, 4, 0);
  F.LS = make_layout(n, nsk, nbranch, 4, 1);
  F.LV = make_layout(n, nsk, nbranch, 4, 2);
  return GRID_OK;
}
