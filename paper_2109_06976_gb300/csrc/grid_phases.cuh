// Device phases of the dynamics kernels (included by grid_kernels.cu).
// Mapping and phase list: see grid_kernels.cu.
#pragma once

#include <type_traits>

#include "grid_internal.h"
#include "spatial.cuh"

enum { MODE_RNEA = 0, MODE_MINV = 1, MODE_FD = 2, MODE_GRAD = 3 };

template <class S>
struct Ctx {
  const ModelDev<S>& M;
  S* W;      // this knot point's workspace
  int l;     // lane within the group, 0..T-1
};

#ifndef GRID_SYNC
#define GRID_SYNC() __syncwarp()
#endif
#ifndef GRID_ATOMIC_ADD
#define GRID_ATOMIC_ADD(p, v) atomicAdd((p), (v))
#endif
#define SYNC() GRID_SYNC()

// ---------------------------------------------------------------- B1
template <class S, int T>
__device__ void ph_transforms(const Ctx<S>& c) {
  const ModelDev<S>& M = c.M;
  S* W = c.W;
  const KnotLayout& L = M.L;
  for (int k = c.l; k < M.n; k += T) {
    S qk = W[L.Q + M.perm[k]];
    S s, co;
    if constexpr (std::is_same<S, float>::value) sincosf(qk, &s, &co); else sincos(qk, &s, &co);
    const S* a = M.axis[k];
    // E_J = R(a, q)^T = cos q 1 + (1 - cos q) a a^T - sin q a~
    S EJ[9];
    const S omc = S(1) - co;
    EJ[0] = co + omc * a[0] * a[0];      EJ[1] = omc * a[0] * a[1] + s * a[2]; EJ[2] = omc * a[0] * a[2] - s * a[1];
    EJ[3] = omc * a[1] * a[0] - s * a[2]; EJ[4] = co + omc * a[1] * a[1];     EJ[5] = omc * a[1] * a[2] + s * a[0];
    EJ[6] = omc * a[2] * a[0] + s * a[1]; EJ[7] = omc * a[2] * a[1] - s * a[0]; EJ[8] = co + omc * a[2] * a[2];
    S* X = W + L.X + 12 * k;
    if (M.et_ident[k]) {
#pragma unroll
      for (int e = 0; e < 9; ++e) X[e] = EJ[e];
    } else {
      const S* ET = M.ET[k];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          X[3 * i + j] = EJ[3 * i] * ET[j] + EJ[3 * i + 1] * ET[3 + j] + EJ[3 * i + 2] * ET[6 + j];
    }
    X[9] = M.rT[k][0]; X[10] = M.rT[k][1]; X[11] = M.rT[k][2];
  }
  SYNC();
}

// ---------------------------------------------------------------- B2 / B5
// Forward sweep: v_i = X v_p + S qd_i, a_i = X a_p + S qdd_i + v_i x S qd_i,
// gamma_i = I v_i, f_i = I a_i + v_i x* gamma_i (a_base = -g).
// qdd_off < 0 means qdd = 0.
template <class S, int T>
__device__ void ph_rnea_fwd(const Ctx<S>& c, int qdd_off, bool qdd_caller_order) {
  const ModelDev<S>& M = c.M;
  S* W = c.W;
  const KnotLayout& L = M.L;
  const int l = c.l;
  const int U = L.UNION;
  for (int k = 0; k < M.n; ++k) {
    const int p = M.parent[k];
    const S* E = W + L.X + 12 * k;
    const S* r = E + 9;
    const S qdk = W[L.QD + M.perm[k]];
    S qddk = S(0);
    if (qdd_off >= 0) qddk = W[qdd_off + (qdd_caller_order ? M.perm[k] : k)];
    if (l < 6) {
      S vp[6], ap[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        vp[e] = p < 0 ? S(0) : W[L.V + 6 * p + e];
        ap[e] = p < 0 ? M.a0[e] : W[U + L.A + 6 * p + e];
      }
      S sc = l < 3 ? M.axis[k][l] : S(0);
      W[L.V + 6 * k + l] = x_mul_c(E, r, vp, l) + sc * qdk;
      W[U + L.A + 6 * k + l] = x_mul_c(E, r, ap, l) + sc * qddk;
    }
    SYNC();
    if (l < 6) {
      const S* v = W + L.V + 6 * k;
      const S* a = M.axis[k];
      // (v x S qd)_l: S qd = [a qd; 0]
      S sq[6] = {a[0] * qdk, a[1] * qdk, a[2] * qdk, S(0), S(0), S(0)};
      S vx[6];
      crm_mul(v, sq, vx);
      S add = vx[0];
#pragma unroll
      for (int e = 1; e < 6; ++e) add = (l == e) ? vx[e] : add;
      W[U + L.A + 6 * k + l] += add;
      W[L.GAM + 6 * k + l] = i_mul_c(M.inert[k], v, l);
    }
    SYNC();
    if (l < 6) {
      const S* v = W + L.V + 6 * k;
      S ia[6], vg[6];
      i_mul(M.inert[k], W + U + L.A + 6 * k, ia);
      crf_mul(v, W + L.GAM + 6 * k, vg);
      S x = ia[0] + vg[0];
#pragma unroll
      for (int e = 1; e < 6; ++e) x = (l == e) ? ia[e] + vg[e] : x;
      W[U + L.FO + 6 * k + l] = x;
      W[U + L.FA + 6 * k + l] = x;
    }
  }
  SYNC();
}

// Backward sweep: tau_i = S_i^T F_i, F_p += X_i^T F_i (F = accumulated forces).
template <class S, int T>
__device__ void ph_rnea_bwd(const Ctx<S>& c) {
  const ModelDev<S>& M = c.M;
  S* W = c.W;
  const KnotLayout& L = M.L;
  const int l = c.l;
  const int U = L.UNION;
  for (int k = M.n - 1; k >= 0; --k) {
    const int p = M.parent[k];
    const S* F = W + U + L.FA + 6 * k;
    if (l < 6 && p >= 0) {
      const S* E = W + L.X + 12 * k;
      W[U + L.FA + 6 * p + l] += xt_mul_c(E, E + 9, F, l);
    }
    if (l == 6) {
      const S* a = M.axis[k];
      W[L.CB + k] = a[0] * F[0] + a[1] * F[1] + a[2] * F[2];
    }
    SYNC();
  }
}

// ---------------------------------------------------------------- B3
// Direct M^-1 by the articulated-inertia recursion (Sec. IV-B, Carpentier 2018).
// Backward (leaves to root):
//   I^A_i = I_i + sum_children X_c^T (I^A_c - U_c D_c^-1 U_c^T) X_c
//   U_i = I^A_i S_i,  D_i = S_i^T U_i,  Minv[i][i] = D_i^-1
//   Minv[i][k] = -D_i^-1 S_i^T F[:, k]          for k in subtree(i), k != i
//   F[:, k] <- X_i^T (F[:, k] + U_i Minv[i][k])  for k in subtree(i)
// Forward (root to leaves), for k >= i in i's base-branch:
//   t = X_i P_p[:, k],  Minv[i][k] -= D_i^-1 U_i^T t,  P_i[:, k] = S_i Minv[i][k] + t
// F is one 6 x n buffer (columns are owned by one subtree at a time); the
// children's contributions to I^A and P_p are kept in depth-indexed stacks.
// With P = double (mixed precision) the pivots D_i, D_i^-1 and every update
// that divides by them are evaluated in FP64.
template <class S, class P, int T>
__device__ void ph_minv(const Ctx<S>& c) {
  const ModelDev<S>& M = c.M;
  S* W = c.W;
  const KnotLayout& L = M.L;
  const int l = c.l;
  const int n = M.n;
  const int U = L.UNION;
  S* MI = W + L.MINV;
  S* IAS = W + U + L.IAS;
  S* IAT = W + U + L.IAT;
  S* CT = W + U + L.CT;
  S* FB = W + U + L.FB;
  S* PST = W + U + L.PST;
  P* DINV = reinterpret_cast<P*>(W + L.DINV);
  for (int e = l; e < n * n; e += T) MI[e] = S(0);
  for (int e = l; e < 36 * M.maxd; e += T) IAS[e] = S(0);
  for (int e = l; e < 6 * n; e += T) FB[e] = S(0);
  SYNC();
  for (int k = n - 1; k >= 0; --k) {
    const int p = M.parent[k];
    const int d = M.depth[k];
    const S* E = W + L.X + 12 * k;
    const S* r = E + 9;
    const S* a = M.axis[k];
    for (int e = l; e < 36; e += T) {
      IAT[e] = i_entry(M.inert[k], e / 6, e % 6) + IAS[36 * d + e];
      IAS[36 * d + e] = S(0);
    }
    SYNC();
    S* Uk = W + L.UB + 6 * k;
    if (l < 6) Uk[l] = IAT[6 * l] * a[0] + IAT[6 * l + 1] * a[1] + IAT[6 * l + 2] * a[2];
    SYNC();
    const P Dk = P(a[0]) * P(Uk[0]) + P(a[1]) * P(Uk[1]) + P(a[2]) * P(Uk[2]);
    const P Dinv = P(1) / Dk;
    if (l == 0) DINV[k] = Dinv;
    for (int kk = k + l; kk < M.sub_end[k]; kk += T) {
      if (kk == k) MI[k * n + k] = S(Dinv);
      else MI[k * n + kk] = S(-Dinv * (P(a[0]) * P(FB[kk]) + P(a[1]) * P(FB[n + kk]) + P(a[2]) * P(FB[2 * n + kk])));
    }
    SYNC();
    if (p >= 0) {
      for (int kk = k + l; kk < M.sub_end[k]; kk += T) {
        S w[6], o[6];
        const S mik = MI[k * n + kk];
#pragma unroll
        for (int e = 0; e < 6; ++e) w[e] = FB[e * n + kk] + Uk[e] * mik;
        xt_mul(E, r, w, o);
#pragma unroll
        for (int e = 0; e < 6; ++e) FB[e * n + kk] = o[e];
      }
      for (int e = l; e < 36; e += T)
        IAT[e] = S(P(IAT[e]) - P(Uk[e / 6]) * P(Uk[e % 6]) * Dinv);
      SYNC();
      if (l < 6) {                       // CT[:, l] = X^T IAT[:, l]
        S col[6], o[6];
#pragma unroll
        for (int e = 0; e < 6; ++e) col[e] = IAT[6 * e + l];
        xt_mul(E, r, col, o);
#pragma unroll
        for (int e = 0; e < 6; ++e) CT[6 * e + l] = o[e];
      }
      SYNC();
      if (l < 6) {                       // column l of X^T IA X = X^T (row l of CT)
        S row[6], o[6];
#pragma unroll
        for (int e = 0; e < 6; ++e) row[e] = CT[6 * l + e];
        xt_mul(E, r, row, o);
        S* slot = IAS + 36 * (d - 1);
#pragma unroll
        for (int e = 0; e < 6; ++e) slot[6 * e + l] += o[e];
      }
      SYNC();
    }
  }
  // forward pass
  for (int k = 0; k < n; ++k) {
    const int p = M.parent[k];
    const int d = M.depth[k];
    const S* E = W + L.X + 12 * k;
    const S* r = E + 9;
    const S* a = M.axis[k];
    const S* Uk = W + L.UB + 6 * k;
    const P Dinv = DINV[k];
    for (int kk = k + l; kk < M.comp_hi[k]; kk += T) {
      S t[6] = {S(0), S(0), S(0), S(0), S(0), S(0)};
      S mk = MI[k * n + kk];
      if (p >= 0) {
        S pp[6];
#pragma unroll
        for (int e = 0; e < 6; ++e) pp[e] = PST[(6 * (d - 1) + e) * n + kk];
        x_mul(E, r, pp, t);
        P ut = P(Uk[0]) * P(t[0]);
#pragma unroll
        for (int e = 1; e < 6; ++e) ut += P(Uk[e]) * P(t[e]);
        mk = S(P(mk) - Dinv * ut);
        MI[k * n + kk] = mk;
      }
#pragma unroll
      for (int e = 0; e < 6; ++e) PST[(6 * d + e) * n + kk] = (e < 3 ? a[e] * mk : S(0)) + t[e];
    }
    SYNC();
  }
  for (int e = l; e < n * n; e += T) {
    const int i = e / n, j = e % n;
    if (j < i) MI[e] = MI[j * n + i];
  }
  SYNC();
}

// ---------------------------------------------------------------- B4
template <class S, int T>
__device__ void ph_fd(const Ctx<S>& c) {
  const ModelDev<S>& M = c.M;
  S* W = c.W;
  const KnotLayout& L = M.L;
  const int n = M.n;
  for (int i = c.l; i < n; i += T) {
    S acc = S(0);
    for (int j = M.comp_lo[i]; j < M.comp_hi[i]; ++j)
      acc += W[L.MINV + i * n + j] * (W[L.TAU + M.perm[j]] - W[L.CB + j]);
    W[L.QDD + i] = acc;
  }
  SYNC();
}

// ---------------------------------------------------------------- B5
// RNEA at the computed qdd: the accelerations change by da_i = X da_p + S qdd_i,
// own forces by I da_i; accumulated forces are then rebuilt.
template <class S, int T>
__device__ void ph_rnea_qdd_update(const Ctx<S>& c) {
  const ModelDev<S>& M = c.M;
  S* W = c.W;
  const KnotLayout& L = M.L;
  const int l = c.l;
  const int U = L.UNION;
  for (int k = 0; k < M.n; ++k) {
    const int p = M.parent[k];
    const S* E = W + L.X + 12 * k;
    if (l < 6) {
      S dp[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) dp[e] = p < 0 ? S(0) : W[U + L.DA + 6 * p + e];
      S sc = l < 3 ? M.axis[k][l] : S(0);
      W[U + L.DA + 6 * k + l] = x_mul_c(E, E + 9, dp, l) + sc * W[L.QDD + k];
    }
    SYNC();
    if (l < 6) {
      W[U + L.A + 6 * k + l] += W[U + L.DA + 6 * k + l];
      const S x = W[U + L.FO + 6 * k + l] + i_mul_c(M.inert[k], W + U + L.DA + 6 * k, l);
      W[U + L.FO + 6 * k + l] = x;
      W[U + L.FA + 6 * k + l] = x;
    }
  }
  SYNC();
}

// ---------------------------------------------------------------- B6
// Per-body terms of Alg. 2 that do not depend on the column:
//   beta_i = (X_i a_p) x S_i, phi_i = S_i x* F_i (the backward-pass term of
//   the q columns), and the subspaces s_i^(k) = kX_i S_i of every ancestor i of
//   k expressed in frame k (s_k^(k) = S_k, s_i^(k) = X_k s_i^(p)).
template <class S, int T>
__device__ void ph_aux(const Ctx<S>& c) {
  const ModelDev<S>& M = c.M;
  S* W = c.W;
  const KnotLayout& L = M.L;
  const int U = L.UNION;
  for (int k = c.l; k < M.n; k += T) {
    const int p = M.parent[k];
    const S* E = W + L.X + 12 * k;
    const S* a = M.axis[k];
    S ap[6], w[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) ap[e] = p < 0 ? M.a0[e] : W[U + L.A + 6 * p + e];
    x_mul(E, E + 9, ap, w);
    S* B = W + L.BET + 6 * k;
    cross3(w, a, B);             // (X a_p) x [a; 0] = [w_ang x a; w_lin x a]
    cross3(w + 3, a, B + 3);
    const S* F = W + U + L.FA + 6 * k;
    S* Ph = W + L.PHI + 6 * k;    // [a; 0] x* F = [a x F_ang; a x F_lin]
    cross3(a, F, Ph);
    cross3(a, F + 3, Ph + 3);
  }
  for (int k = 0; k < M.n; ++k) {
    const int dk = M.depth[k];
    const int p = M.parent[k];
    const S* E = W + L.X + 12 * k;
    for (int d = c.l; d <= dk; d += T) {
      S* row = W + L.SK + 8 * (M.skoff[k] + d);
      if (d == dk) {
        row[0] = M.axis[k][0]; row[1] = M.axis[k][1]; row[2] = M.axis[k][2];
        row[3] = row[4] = row[5] = S(0);
      } else {
        x_mul(E, E + 9, W + L.SK + 8 * (M.skoff[p] + d), row);
      }
    }
    SYNC();
  }
}

// ---------------------------------------------------------------- C
// Derivative columns. For column (u, j) and body k on a root-to-leaf path of
// subtree(j) (Alg. 1 / Alg. 2 forward pass, with the readings: the case terms
// act only at k = j, and the velocity-product term uses dv_k):
//   dv_k = X_k dv_p + [k=j] {v_k x S_k (u=q) ; S_k (u=qd)}
//   da_k = X_k da_p + dv_k x S_k qd_k + [k=j] {beta_k (u=q) ; v_k x S_k (u=qd)}
//   df_k = I_k da_k + dv_k x* gamma_k + v_k x* I_k dv_k
// ((X v_p) x S = v x S because S x S = 0.) The backward pass of Alg. 1 is
// applied in closed form: dc_i = sum over k in subtree(i) of s_i^(k) . df_k,
// plus s_i^(j) . phi_j for the strict ancestors i of j when u = q. Each lane
// accumulates these dot products per depth along its path in registers and
// adds them to dc at the path's end.
template <class S, int T, int MAXD>
__device__ void ph_columns(const Ctx<S>& c, const uint32_t* __restrict__ sched, int nsteps) {
  const ModelDev<S>& M = c.M;
  S* W = c.W;
  const KnotLayout& L = M.L;
  const int n = M.n;
  const int U = L.UNION;
  S* DC = W + U + L.DC;
  for (int e = c.l; e < 2 * n * n; e += T) DC[e] = S(0);
  SYNC();
  S dv[6], da[6], acc[MAXD];
#pragma unroll
  for (int e = 0; e < 6; ++e) { dv[e] = S(0); da[e] = S(0); }
#pragma unroll
  for (int d = 0; d < MAXD; ++d) acc[d] = S(0);
  for (int s = 0; s < nsteps; ++s) {
    const uint32_t st = sched[s * T + c.l];
    if (!(st & STEP_VALID)) continue;
    const int k = STEP_BODY(st);
    const int col = STEP_COL(st);
    const bool root = st & STEP_ROOT, uq = st & STEP_UQ;
    if (st & STEP_RESET) {
#pragma unroll
      for (int e = 0; e < 6; ++e) { dv[e] = S(0); da[e] = S(0); }
    }
    const S* E = W + L.X + 12 * k;
    const S* r = E + 9;
    const S* ax = M.axis[k];
    const S qdk = W[L.QD + M.perm[k]];
    S v[6], g[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) { v[e] = W[L.V + 6 * k + e]; g[e] = W[L.GAM + 6 * k + e]; }
    S ndv[6], nda[6], vxs[6];
    x_mul(E, r, dv, ndv);
    x_mul(E, r, da, nda);
    cross3(v, ax, vxs);          // v x [a; 0] = [w x a; v x a]
    cross3(v + 3, ax, vxs + 3);
    if (root) {
      if (uq) {
        const S* B = W + L.BET + 6 * k;
#pragma unroll
        for (int e = 0; e < 6; ++e) { ndv[e] += vxs[e]; nda[e] += B[e]; }
      } else {
        ndv[0] += ax[0]; ndv[1] += ax[1]; ndv[2] += ax[2];
#pragma unroll
        for (int e = 0; e < 6; ++e) nda[e] += vxs[e];
      }
    }
    {
      const S sq[3] = {ax[0] * qdk, ax[1] * qdk, ax[2] * qdk};
      S t[6];
      cross3(ndv, sq, t);        // dv x [a qd; 0]
      cross3(ndv + 3, sq, t + 3);
#pragma unroll
      for (int e = 0; e < 6; ++e) nda[e] += t[e];
    }
    S df[6], t1[6], t2[6], idv[6];
    i_mul(M.inert[k], nda, df);
    crf_mul(ndv, g, t1);
    i_mul(M.inert[k], ndv, idv);
    crf_mul(v, idv, t2);
#pragma unroll
    for (int e = 0; e < 6; ++e) df[e] += t1[e] + t2[e];
    if (root && uq) {
      const S* Ph = W + L.PHI + 6 * k;
#pragma unroll
      for (int e = 0; e < 6; ++e) df[e] += Ph[e];
    }
    const int dk = M.depth[k];
    if (st & STEP_OWNED) {
      const S* rows = W + L.SK + 8 * M.skoff[k];
#pragma unroll
      for (int d = 0; d < MAXD; ++d) {
        if (d <= dk) {
          const S* sr = rows + 8 * d;
          acc[d] += sr[0] * df[0] + sr[1] * df[1] + sr[2] * df[2] + sr[3] * df[3] + sr[4] * df[4] +
                    sr[5] * df[5];
        }
      }
    }
    if (st & STEP_FLUSH) {
      int b = k;
#pragma unroll
      for (int d = MAXD - 1; d >= 0; --d) {
        if (d <= dk) {
          GRID_ATOMIC_ADD(DC + b * 2 * n + col, acc[d]);
          acc[d] = S(0);
          b = M.parent[b];
        }
      }
    }
#pragma unroll
    for (int e = 0; e < 6; ++e) { dv[e] = ndv[e]; da[e] = nda[e]; }
  }
  SYNC();
}

// ---------------------------------------------------------------- D
// J = -M^-1 dc, restricted to base-branch blocks, written in caller order.
template <class S, int T>
__device__ void ph_product(const Ctx<S>& c) {
  const ModelDev<S>& M = c.M;
  S* W = c.W;
  const KnotLayout& L = M.L;
  const int n = M.n, n2 = 2 * n;
  const int U = L.UNION;
  const S* DC = W + U + L.DC;
  S* JS = W + U + L.JS;
  for (int e = c.l; e < 2 * n * n; e += T) {
    const int i = e / n2, col = e % n2;
    const int j = col < n ? col : col - n;
    S acc = S(0);
    if (M.comp_lo[j] <= i && i < M.comp_hi[j])
      for (int m = M.comp_lo[j]; m < M.comp_hi[j]; ++m) acc += W[L.MINV + i * n + m] * DC[m * n2 + col];
    const int ucol = (col < n ? 0 : n) + M.perm[j];
    JS[M.perm[i] * n2 + ucol] = -acc;
  }
  SYNC();
}

// One warp processes knot points k0 .. k0 + 32/T - 1 (those < N).
template <class S, int MODE, int T, int MAXD, bool MIXED>
__device__ void process_tile(const ModelDev<S>& M, const uint32_t* __restrict__ sched, int nsteps,
                             S* Wwarp, int lane32, int k0, int N, const S* __restrict__ q,
                             const S* __restrict__ qd, const S* __restrict__ x3, S* __restrict__ out,
                             S* __restrict__ out2) {
  using P = typename std::conditional<MIXED, double, S>::type;
  const KnotLayout& L = M.L;
  const int n = M.n;
  constexpr int G = 32 / T;
  const int g = lane32 / T;
  S* W = Wwarp + g * L.stride;
  const Ctx<S> c{M, W, lane32 % T};
  const int out_per = MODE == MODE_MINV ? n * n : (MODE == MODE_GRAD ? 2 * n * n : n);
  const int nvalid = min(G, N - k0);
  // stage inputs (coalesced across the warp)
  for (int e = lane32; e < G * n; e += 32) {
    const int kk = e / n, i = e % n;
    S* Wk = Wwarp + kk * L.stride;
    const bool ok = kk < nvalid;
    const size_t gi = (size_t)k0 * n + e;
    Wk[L.Q + i] = ok ? q[gi] : S(0);
    if (MODE != MODE_MINV) Wk[L.QD + i] = ok ? qd[gi] : S(0);
    if (MODE == MODE_RNEA) Wk[L.TAU + i] = (ok && x3) ? x3[gi] : S(0);
    if (MODE == MODE_FD || MODE == MODE_GRAD) Wk[L.TAU + i] = ok ? x3[gi] : S(0);
  }
  SYNC();
  ph_transforms<S, T>(c);
  if (MODE == MODE_RNEA) {
    ph_rnea_fwd<S, T>(c, L.TAU, true);
    ph_rnea_bwd<S, T>(c);
  } else if (MODE == MODE_MINV) {
    ph_minv<S, P, T>(c);
  } else {
    ph_rnea_fwd<S, T>(c, -1, false);
    ph_rnea_bwd<S, T>(c);                 // CB = RNEA(q, qd, 0)
    ph_minv<S, P, T>(c);
    ph_fd<S, T>(c);
    if (MODE == MODE_GRAD) {
      ph_rnea_qdd_update<S, T>(c);
      ph_rnea_bwd<S, T>(c);
      ph_aux<S, T>(c);
      ph_columns<S, T, MAXD>(c, sched, nsteps);
      ph_product<S, T>(c);
    }
  }
  // stage outputs in caller order
  S* OS = W + L.UNION + L.JS;
  if (MODE == MODE_RNEA) {
    for (int i = c.l; i < n; i += T) OS[M.perm[i]] = W[L.CB + i];
  } else if (MODE == MODE_FD) {
    for (int i = c.l; i < n; i += T) OS[M.perm[i]] = W[L.QDD + i];
  } else if (MODE == MODE_MINV) {
    for (int e = c.l; e < n * n; e += T) OS[M.perm[e / n] * n + M.perm[e % n]] = W[L.MINV + e];
  } else if (out2) {
    for (int i = c.l; i < n; i += T) W[L.CB + M.perm[i]] = W[L.QDD + i];
  }
  SYNC();
  for (int e = lane32; e < nvalid * out_per; e += 32) {
    const int kk = e / out_per, r = e % out_per;
    out[(size_t)k0 * out_per + e] = Wwarp[kk * L.stride + L.UNION + L.JS + r];
  }
  if (MODE == MODE_GRAD && out2) {
    for (int e = lane32; e < nvalid * n; e += 32) {
      const int kk = e / n, r = e % n;
      out2[(size_t)k0 * n + e] = Wwarp[kk * L.stride + L.CB + r];
    }
  }
  SYNC();
}

