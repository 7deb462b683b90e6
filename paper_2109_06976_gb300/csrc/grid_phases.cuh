// Device phases of the dynamics kernels (included by grid_kernels.cu).
//
// T lanes of a warp cooperate on one knot point (all groups of a warp run the
// same robot in lockstep; synchronisation is __syncwarp). Bodies use the
// internal depth-first numbering, so subtree(i) = [i, sub_end[i]) and the first
// child of i, if any, is i + 1. Phases, in order:
//  B1 joint transforms X_i(q_i)                                  lanes over bodies
//  B2 ancestor subspaces s_m^(k) = kX_m S_m and gravity rows      lanes over depths
//  B3 direct M^-1 (articulated-inertia recursion)                lanes own 6x6 columns / M^-1 columns
//  B4 RNEA(q, qd, 0) from the subspace table                     lanes over bodies
//  B5 bias c_i = sum_{k in subtree(i)} s_i^(k) . f_k             lanes over bodies
//  B6 qdd = M^-1 (tau - c)                                       lanes over rows
//  B7 RNEA at qdd, beta_i; accumulated forces F_i, phi_i         lanes over bodies / components
//  C  derivative columns (Alg. 1 / Alg. 2)                       host-balanced path schedules
//  D  J = -M^-1 dc                                               lanes over outputs
#pragma once

#include "grid_internal.h"
#include "spatial.cuh"

// ---------------------------------------------------------------- topology
// The robot's topology as the phases see it. RtTopo reads the staged model
// (any tree in depth-first numbering). ChainTopo is the serial chain
// parent(i) = i - 1 of N bodies: depths, subtree ranges, subspace-table
// offsets and the workspace layout follow from N at compile time, so loops
// over bodies unroll and their indices fold (per-body constants such as axes
// and inertias stay in the staged model).
// kPlace: whether the model may be a part placed in a robot's arrays
// (ModelDev::ld): 0 never, 1 always, 2 read from the model at run time.
template <class S, int MODE>
struct RtTopo {
  static constexpr int kPlace = 2;
  static constexpr int kUnroll = 1;
  static constexpr int kChainN = 0;       // not a compile-time chain
  static constexpr bool kConsecutivePaths = false;
  static constexpr int kBranches = 0;
  const ModelDev<S>& M;
  __device__ explicit RtTopo(const ModelDev<S>& m) : M(m) {}
  __device__ const KnotLayout& layout() const { return layout_of<MODE>(M); }
  __device__ int n() const { return M.n; }
  __device__ int maxd() const { return M.maxd; }
  __device__ int nbranch() const { return M.nbranch; }
  __device__ int parent(int i) const { return M.parent[i]; }
  __device__ int depth(int i) const { return M.depth[i]; }
  __device__ int sub_end(int i) const { return M.sub_end[i]; }
  __device__ int comp_lo(int i) const { return M.comp_lo[i]; }
  __device__ int comp_hi(int i) const { return M.comp_hi[i]; }
  __device__ int perm(int i) const { return M.perm[i]; }
  __device__ int skoff(int i) const { return M.skoff[i]; }
  __device__ int branch(int i) const { return M.branch[i]; }
  __device__ bool prism(int i) const { return M.jt[i] != 0; }
};

template <class S, int MODE, int N, bool PL = false>
struct ChainTopo {
  static constexpr int kPlace = PL ? 1 : 0;
  static constexpr int kUnroll = N;
  static constexpr int kChainN = N;
  static constexpr bool kConsecutivePaths = true;   // ancestor at depth d of k: k - depth(k) + d
  static constexpr int kBranches = 0;
  __device__ explicit ChainTopo(const ModelDev<S>&) {}
  GRID_HD static constexpr KnotLayout layout() {
    return make_layout(N, N * (N + 1) / 2, 0, (int)sizeof(S), layout_kind(MODE));
  }
  GRID_HD static constexpr int n() { return N; }
  GRID_HD static constexpr int maxd() { return N; }       // depth levels
  GRID_HD static constexpr int nbranch() { return 0; }
  GRID_HD static constexpr int parent(int i) { return i - 1; }
  GRID_HD static constexpr int depth(int i) { return i; }
  GRID_HD static constexpr int sub_end(int) { return N; }
  GRID_HD static constexpr int comp_lo(int) { return 0; }
  GRID_HD static constexpr int comp_hi(int) { return N; }
  GRID_HD static constexpr int perm(int i) { return i; }
  GRID_HD static constexpr int skoff(int i) { return i * (i + 1) / 2; }
  GRID_HD static constexpr int branch(int) { return -1; }
  GRID_HD static constexpr bool prism(int) { return false; }   // revolute chains only
};

// K serial chains of L bodies on the fixed base (a forest whose chains differ
// only in their parameters) run as K independent chains: the joints c L .. c L +
// L - 1 of knot point k are the joints of "virtual" knot point k K + c in the
// same memory (knot-major arrays), lane group g of a warp uses chain g mod K's
// model, and only J and M^-1 are placed differently: the chain's blocks on the
// diagonal of the K L-joint outputs, zeros elsewhere (the chains do not interact
// through a fixed base).
template <class S, int MODE, int L, int K>
struct BranchTopo : ChainTopo<S, MODE, L> {
  static constexpr int kBranches = K;
  __device__ explicit BranchTopo(const ModelDev<S>& m) : ChainTopo<S, MODE, L>(m) {}
};

// K identical serial chains of L bodies, each hanging from the fixed base, in
// depth-first numbering (a quadruped's legs: K = 4, L = 3). The phases take
// their general paths; only the topology folds.
template <class S, int MODE, int K, int L>
struct ForestTopo {
  static constexpr int kPlace = 0;
  static constexpr int kUnroll = K * L;
  static constexpr int kChainN = 0;
  static constexpr bool kConsecutivePaths = true;
  static constexpr int kBranches = 0;
  __device__ explicit ForestTopo(const ModelDev<S>&) {}
  GRID_HD static constexpr KnotLayout layout() {
    return make_layout(K * L, K * L * (L + 1) / 2, 0, (int)sizeof(S), layout_kind(MODE));
  }
  GRID_HD static constexpr int n() { return K * L; }
  GRID_HD static constexpr int maxd() { return L; }
  GRID_HD static constexpr int nbranch() { return 0; }
  GRID_HD static constexpr int parent(int i) { return i % L == 0 ? -1 : i - 1; }
  GRID_HD static constexpr int depth(int i) { return i % L; }
  GRID_HD static constexpr int sub_end(int i) { return (i / L + 1) * L; }
  GRID_HD static constexpr int comp_lo(int i) { return (i / L) * L; }
  GRID_HD static constexpr int comp_hi(int i) { return (i / L + 1) * L; }
  GRID_HD static constexpr int perm(int i) { return i; }
  GRID_HD static constexpr int skoff(int i) { return (i / L) * (L * (L + 1) / 2) + (i % L) * (i % L + 1) / 2; }
  GRID_HD static constexpr int branch(int) { return -1; }
  GRID_HD static constexpr bool prism(int) { return false; }
};

template <class S, class Tp>
struct Ctx {
  const ModelDev<S>& M;
  const ModelDev<S>* gM;  // the same model in device memory (tables not staged in shared memory)
  Tp tp;                  // topology
  S* W;                   // this knot point's workspace
  int l;                  // lane within the group, 0..T-1
  int lane32;             // lane within the warp
};

#ifndef GRID_SYNC
#define GRID_SYNC() __syncwarp()
#endif
#ifndef GRID_ATOMIC_ADD
#define GRID_ATOMIC_ADD(p, v) atomicAdd((p), (v))
#endif
#ifndef GRID_SHFL
#define GRID_SHFL(v, src) __shfl_sync(0xffffffffu, (v), (src))
#endif
#define SYNC() GRID_SYNC()

// Body of row d of body k's subspace rows (its ancestor at depth d): stored in
// the row's slot 7, or k - depth(k) + d where every root path is numbered
// consecutively (chains, forests of chains), which saves a conversion per row.
template <class Tp, class S>
__device__ __forceinline__ int row_body(int k, int dk, int d, S slot7) {
  if constexpr (Tp::kConsecutivePaths) return k - dk + d;
  else return (int)slot7;
}

// ---------------------------------------------------------------- B1
template <class S, int T, class Tp>
__device__ void ph_transforms(const Ctx<S, Tp>& c) {
  const ModelDev<S>& M = c.M;
  const Tp& tp = c.tp;
  S* W = c.W;
  const KnotLayout L = c.tp.layout();   // by value: offsets stay in registers
  for (int k = c.l; k < tp.n(); k += T) {
    S qk = W[L.Q + tp.perm(k)];
    const S* a = M.axis[k];
    S* X = W + L.X + 12 * k;
    if (tp.prism(k)) {
      // X_J = X(1, q a): X = X(E_T, r_T + E_T^T q a)
      const S* ET = M.ET[k];
      const S d[3] = {qk * a[0], qk * a[1], qk * a[2]};
#pragma unroll
      for (int e = 0; e < 9; ++e) X[e] = ET[e];
#pragma unroll
      for (int j = 0; j < 3; ++j) X[9 + j] = M.rT[k][j] + ET[j] * d[0] + ET[3 + j] * d[1] + ET[6 + j] * d[2];
      continue;
    }
    S s, co;
    if constexpr (grid_same<S, float>::value) sincosf(qk, &s, &co); else sincos(qk, &s, &co);
    // E_J = R(a, q)^T = cos q 1 + (1 - cos q) a a^T - sin q a~
    S EJ[9];
    const S omc = S(1) - co;
    EJ[0] = co + omc * a[0] * a[0];      EJ[1] = omc * a[0] * a[1] + s * a[2]; EJ[2] = omc * a[0] * a[2] - s * a[1];
    EJ[3] = omc * a[1] * a[0] - s * a[2]; EJ[4] = co + omc * a[1] * a[1];     EJ[5] = omc * a[1] * a[2] + s * a[0];
    EJ[6] = omc * a[2] * a[0] + s * a[1]; EJ[7] = omc * a[2] * a[1] - s * a[0]; EJ[8] = co + omc * a[2] * a[2];
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

// ---------------------------------------------------------------- B2
// Subspace rows of body k (8 scalars each, from SK + 8 * skoff[k]):
//   row d = 0..depth_k : s_m^(k) = kX_m S_m for the ancestor m of k at depth d
//                        (m = k at d = depth_k); slot 6 = qd_m, slot 7 = m
// and the gravity row g^(k) = kX_0 a_0 (the base acceleration -g in frame k),
// kept in the phase-local area GR.
// s_m^(k) = X_k s_m^(parent k). Row id rho (d, or maxd for gravity) belongs to
// lane rho mod T, which therefore only reads rows it wrote itself.
template <class S, int T, class Tp>
__device__ __forceinline__ void subspace_step(const Ctx<S, Tp>& c, int k, const S* E, S* carry) {
  const ModelDev<S>& M = c.M;
  const Tp& tp = c.tp;
  S* W = c.W;
  const KnotLayout L = c.tp.layout();   // by value: offsets stay in registers
  S* SK = W + L.SK;
  S* GR = W + L.UNION + L.GR;
  const int dk = tp.depth(k);
  const int p = tp.parent(k);
  const bool carry_ok = T > tp.maxd();        // one row id per lane: reuse the previous body's row
  for (int rho = c.l; rho <= tp.maxd(); rho += T) {
    if (rho == dk) {
      S row[8];
      joint_s(M.axis[k], tp.prism(k), row);
      row[6] = W[L.QD + tp.perm(k)];
      row[7] = S(k);
      S* dst = SK + 8 * (tp.skoff(k) + dk);
      st4(dst, row);
      st4(dst + 4, row + 4);
#pragma unroll
      for (int e = 0; e < 8; ++e) carry[e] = row[e];
    } else if (rho < dk || rho == tp.maxd()) {
      const bool grav = rho == tp.maxd();
      S src[8];
      if (p < 0) {
#pragma unroll
        for (int e = 0; e < 6; ++e) src[e] = M.a0[e];
        src[6] = src[7] = S(0);
      } else if (carry_ok && p == k - 1) {
#pragma unroll
        for (int e = 0; e < 8; ++e) src[e] = carry[e];
      } else {
        const S* sp = grav ? GR + 8 * p : SK + 8 * (tp.skoff(p) + rho);
        ld4(sp, src);
        ld4(sp + 4, src + 4);
      }
      S out[8];
      x_mul(E, E + 9, src, out);
      out[6] = src[6];
      out[7] = src[7];
      S* dst = grav ? GR + 8 * k : SK + 8 * (tp.skoff(k) + rho);
      st4(dst, out);
      st4(dst + 4, out + 4);
#pragma unroll
      for (int e = 0; e < 8; ++e) carry[e] = out[e];
    }
  }
}

template <class S, int T, class Tp>
__device__ void ph_subspaces(const Ctx<S, Tp>& c) {
  const KnotLayout L = c.tp.layout();   // by value: offsets stay in registers
  S carry[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) carry[e] = S(0);
#pragma unroll (Tp::kUnroll)
  for (int k = 0; k < c.tp.n(); ++k) {
    S E[12];
    ld12(c.W + L.X + 12 * k, E);
    subspace_step<S, T>(c, k, E, carry);
  }
  SYNC();
}

// ---------------------------------------------------------------- B3
// Direct M^-1 by the articulated-inertia recursion (Sec. IV-B; Carpentier 2018).
// Backward, bodies i = n-1 .. 0:
//   I^A_i = I_i + sum_children X_c^T (I^A_c - U_c D_c^-1 U_c^T) X_c
//   U_i = I^A_i S_i,  D_i = S_i^T U_i,  Minv[i][i] = D_i^-1
//   Minv[i][k] = -D_i^-1 S_i^T F[:, k]            k in subtree(i), k != i
//   F[:, k]   <- X_i^T (F[:, k] + U_i Minv[i][k])  k in subtree(i)
// Forward, bodies i = 0 .. n-1, columns k >= i of i's base branch:
//   t = X_i P_parent[:, k],  Minv[i][k] -= D_i^-1 U_i^T t,  P_i[:, k] = S_i Minv[i][k] + t
// Lanes 0..5 own column l of I^A_i in registers; the lane owning column k
// (k = l + c T) holds F[:, k] and P[:, k] in registers. A child's I^A
// contribution and P values pass through registers when the parent is the
// next body processed (the first child is i + 1), and through per-branch-body
// slots otherwise. With P = double (mixed precision) the pivots D_i, D_i^-1
// and every update divided by them are evaluated in FP64.
template <class S, class P, int T, int CPL, bool WITH_SK, class Tp>
__device__ void ph_minv(const Ctx<S, Tp>& c) {
  const ModelDev<S>& M = c.M;
  const Tp& tp = c.tp;
  S* W = c.W;
  const KnotLayout L = c.tp.layout();   // by value: offsets stay in registers
  const int l = c.l;
  const int n = tp.n();
  const int U = L.UNION;
  const int MS = L.MS;
  const int base = c.lane32 - l;
  S* MI = W + L.MINV;
  S* UB = W + U + L.UB;
  P* DINV = reinterpret_cast<P*>(W + U + L.DINV);
  S* BIA = W + U + L.BIA;
  S* BP = W + U + L.BP;
  if constexpr (Tp::kChainN > 0) {              // every entry is written; the padding is read as zero
    for (int e = l; e < n * (MS - n); e += T) MI[(e / (MS - n)) * MS + n + e % (MS - n)] = S(0);
  } else {
    for (int e = l; e < n * MS; e += T) MI[e] = S(0);
  }
  for (int e = l; e < 36 * tp.nbranch(); e += T) BIA[e] = S(0);
  SYNC();
  S carry[6], fb[CPL][6];
#pragma unroll
  for (int e = 0; e < 6; ++e) carry[e] = S(0);
#pragma unroll
  for (int cc = 0; cc < CPL; ++cc)
#pragma unroll
    for (int e = 0; e < 6; ++e) fb[cc][e] = S(0);
  // column l of the next body's inertia, fetched one body ahead (device memory)
  S icn[6] = {S(0), S(0), S(0), S(0), S(0), S(0)};
  if (l < 6) ldg6(c.gM->Icol[n - 1][l], icn);
#pragma unroll (Tp::kUnroll)
  for (int i = n - 1; i >= 0; --i) {
    const int p = tp.parent(i);
    const int br = tp.branch(i);
    S E[12];
    ld12(W + L.X + 12 * i, E);
    const S* r = E + 9;
    const S a[3] = {M.axis[i][0], M.axis[i][1], M.axis[i][2]};
    const bool pr = tp.prism(i);              // S_i = [0; a] instead of [a; 0]
    // Lanes 0..5 own column l of I^A_i; the other lanes carry zeros through the
    // same instructions (no divergent branches, so the compiler can interleave
    // the independent F-column and congruence work below).
    const bool own = l < 6;
    S ia[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) ia[e] = icn[e];
    if (i > 0) ldg6(c.gM->Icol[i - 1][own ? l : 0], icn);
    if (i > 0 && !own) {
#pragma unroll
      for (int e = 0; e < 6; ++e) icn[e] = S(0);
    }
    if (i + 1 < n && tp.parent(i + 1) == i) {
#pragma unroll
      for (int e = 0; e < 6; ++e) ia[e] += carry[e];
    }
    if (br >= 0) {
      const S* sl = BIA + 36 * br + 6 * (own ? l : 0);   // 6-scalar rows: scalar loads
#pragma unroll
      for (int e = 0; e < 6; ++e) ia[e] += own ? sl[e] : S(0);
    }
    const S ul = dot_s(a, pr, ia);            // U_l = (I^A S)_l (I^A symmetric)
    if (own) UB[8 * i + l] = ul;
    S u[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) u[e] = GRID_SHFL(ul, base + e);
    const S us0 = pr ? u[3] : u[0], us1 = pr ? u[4] : u[1], us2 = pr ? u[5] : u[2];   // S^T U
    const P Dk = P(a[0]) * P(us0) + P(a[1]) * P(us1) + P(a[2]) * P(us2);
    P Dinv;
    if constexpr (grid_same<P, float>::value) Dinv = rcp_pivot(Dk);
    else Dinv = __drcp_rn(Dk);
    if (l == 0) DINV[i] = Dinv;
#pragma unroll
    for (int cc = 0; cc < CPL; ++cc) {
      const int k = l + cc * T;
      const bool act = k >= i && k < tp.sub_end(i);
      const S f0 = pr ? fb[cc][3] : fb[cc][0], f1 = pr ? fb[cc][4] : fb[cc][1], f2 = pr ? fb[cc][5] : fb[cc][2];
      const S mik = (k == i) ? S(Dinv) : S(-Dinv * (P(a[0]) * P(f0) + P(a[1]) * P(f1) + P(a[2]) * P(f2)));
      if (act) MI[i * MS + k] = mik;
      if (p >= 0) {
        S w[6], fn[6];
#pragma unroll
        for (int e = 0; e < 6; ++e) w[e] = fb[cc][e] + u[e] * mik;
        xt_mul(E, r, w, fn);
#pragma unroll
        for (int e = 0; e < 6; ++e) fb[cc][e] = act ? fn[e] : fb[cc][e];
      }
    }
    S* CT = W + U + L.CT;                    // one buffer: a barrier before it is written again
    if (p >= 0) {
      S acol[6], cx[6];
      const P ulD = P(ul) * Dinv;
#pragma unroll
      for (int e = 0; e < 6; ++e) acol[e] = S(P(ia[e]) - P(u[e]) * ulD);
      xt_mul(E, r, acol, cx);                 // column l of C = X^T A
      if (own) st6(CT + 8 * l, cx);
    }
    SYNC();
    if (p >= 0 && l < 6) {
      // column l of X^T A X = X^T C^T e_l = X^T (row l of C); C symmetric-congruent
      S rowl[6], it[6];
#pragma unroll
      for (int m = 0; m < 6; ++m) rowl[m] = CT[8 * m + l];
      xt_mul(E, r, rowl, it);
      if (p == i - 1) {
#pragma unroll
        for (int e = 0; e < 6; ++e) carry[e] = it[e];
      } else {
        S* slot = BIA + 36 * tp.branch(p) + 6 * l;
#pragma unroll
        for (int e = 0; e < 6; ++e) slot[e] += it[e];
      }
    }
    SYNC();                                   // every lane has read CT before the next body writes it
  }
  SYNC();
  // forward pass (with the subspace-table step of the same body, for ILP)
  S pc[CPL][6], skc[8];
#pragma unroll
  for (int cc = 0; cc < CPL; ++cc)
#pragma unroll
    for (int e = 0; e < 6; ++e) pc[cc][e] = S(0);
#pragma unroll
  for (int e = 0; e < 8; ++e) skc[e] = S(0);
  if constexpr (Tp::kChainN > 0 && Tp::kChainN < T && CPL == 1 && WITH_SK) {
    // Serial chain with fewer bodies than lanes. At body i, lane l < i carries
    // subspace row l (s_l^(i) = X_i s_l^(i-1)), lanes i..N-1 their P column and
    // lane N the gravity row: one x_mul per lane, no divergent paths.
    constexpr int NB = Tp::kChainN;
    S* SK = W + L.SK;
    S* GR = W + U + L.GR;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      S E[12];
      ld12(W + L.X + 12 * i, E);
      const S* r = E + 9;
      const S* a = M.axis[i];
      S Ui[6];
      ld6(UB + 8 * i, Ui);
      const P Dinv = DINV[i];
      const bool row_lane = l < i || l == NB;
      S in[6], t[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) in[e] = (i == 0 && l == NB) ? M.a0[e] : (row_lane ? skc[e] : pc[0][e]);
      x_mul(E, r, in, t);
      if (l >= i && l < NB) {                  // P column l
        S mk = MI[i * MS + l];
        if (i > 0) {
          P ut;
          if constexpr (grid_same<P, S>::value) ut = dot6(Ui, t);
          else ut = (P(Ui[0]) * P(t[0]) + P(Ui[1]) * P(t[1])) + (P(Ui[2]) * P(t[2]) + P(Ui[3]) * P(t[3])) +
                    (P(Ui[4]) * P(t[4]) + P(Ui[5]) * P(t[5]));
          mk = S(P(mk) - Dinv * ut);
          MI[i * MS + l] = mk;
        }
        if (l > i) MI[l * MS + i] = mk;        // the mirrored entry
#pragma unroll
        for (int e = 0; e < 6; ++e) pc[0][e] = (e < 3 ? a[e] * mk : S(0)) + (i > 0 ? t[e] : S(0));
      }
      if (row_lane) {                          // transported ancestor row, or the gravity row
#pragma unroll
        for (int e = 0; e < 6; ++e) skc[e] = t[e];
        if (l == NB) skc[6] = skc[7] = S(0);
        S* dst = l == NB ? GR + 8 * i : SK + 8 * (tp.skoff(i) + l);
        st4(dst, skc);
        st4(dst + 4, skc + 4);
      } else if (l == i) {                     // own row s_i^(i) = S_i, with qd_i and i
        skc[0] = a[0]; skc[1] = a[1]; skc[2] = a[2];
        skc[3] = skc[4] = skc[5] = S(0);
        skc[6] = W[L.QD + i];
        skc[7] = S(i);
        S* dst = SK + 8 * (tp.skoff(i) + i);
        st4(dst, skc);
        st4(dst + 4, skc + 4);
      }
    }
  } else {
#pragma unroll (Tp::kUnroll)
  for (int i = 0; i < n; ++i) {
    const int p = tp.parent(i);
    const int br = tp.branch(i);
    S E[12];
    ld12(W + L.X + 12 * i, E);
    const S* r = E + 9;
    const S* a = M.axis[i];
    const bool pr = tp.prism(i);
    S Ui[6];
    ld6(UB + 8 * i, Ui);
    const P Dinv = DINV[i];
#pragma unroll
    for (int cc = 0; cc < CPL; ++cc) {
      const int k = l + cc * T;
      if (k >= i && k < tp.comp_hi(i)) {
        S t[6] = {S(0), S(0), S(0), S(0), S(0), S(0)};
        S mk = MI[i * MS + k];
        if (p >= 0) {
          S pp[6];
          if (p == i - 1) {
#pragma unroll
            for (int e = 0; e < 6; ++e) pp[e] = pc[cc][e];
          } else {
#pragma unroll
            for (int e = 0; e < 6; ++e) pp[e] = BP[(6 * tp.branch(p) + e) * n + k];
          }
          x_mul(E, r, pp, t);
          P ut;
          if constexpr (grid_same<P, S>::value) ut = dot6(Ui, t);
          else ut = (P(Ui[0]) * P(t[0]) + P(Ui[1]) * P(t[1])) + (P(Ui[2]) * P(t[2]) + P(Ui[3]) * P(t[3])) +
                    (P(Ui[4]) * P(t[4]) + P(Ui[5]) * P(t[5]));
          mk = S(P(mk) - Dinv * ut);
          MI[i * MS + k] = mk;
        }
#pragma unroll
        for (int e = 0; e < 6; ++e)
          pc[cc][e] = (pr ? (e >= 3 ? a[e - 3] * mk : S(0)) : (e < 3 ? a[e] * mk : S(0))) + t[e];
        if (br >= 0) {
#pragma unroll
          for (int e = 0; e < 6; ++e) BP[(6 * br + e) * n + k] = pc[cc][e];
        }
      }
    }
    if (WITH_SK) subspace_step<S, T>(c, i, E, skc);
  }
  }
  // mirror the columns this lane owns into the lower triangle (the chain's
  // forward pass has written them already)
  constexpr bool kMirrored = Tp::kChainN > 0 && Tp::kChainN < T && CPL == 1 && WITH_SK;
#pragma unroll
  for (int cc = 0; cc < (kMirrored ? 0 : CPL); ++cc) {
    const int k = l + cc * T;
    if (k < n)
      for (int i = tp.comp_lo(k); i < k; ++i) MI[k * MS + i] = MI[i * MS + k];
  }
  SYNC();
}

// ---------------------------------------------------------------- B4
// RNEA from the subspace table, for body k with root path m_0 .. m_d = k:
//   v_m^(k) = sum_{e <= m} s_e^(k) qd_e   (velocity of body m in frame k)
//   v_k = v_k^(k),  a_k = g^(k) + sum_m [ v_m^(k) x s_m^(k) qd_m + s_m^(k) qdd_m ]
//   gamma_k = I_k v_k,  f_k = I_k a_k + v_k x* gamma_k
// (the forward recursion v_i = X v_p + S qd_i, a_i = X a_p + S qdd_i + v_i x S qd_i
// unrolled over the path). qdd_off < 0 means qdd = 0.
template <class S, int T, class Tp>
__device__ void ph_rnea_bodies(const Ctx<S, Tp>& c, int qdd_off) {
  const ModelDev<S>& M = c.M;
  const Tp& tp = c.tp;
  S* W = c.W;
  const KnotLayout L = c.tp.layout();   // by value: offsets stay in registers
  const int U = L.UNION;
  for (int k = c.l; k < tp.n(); k += T) {
    const int dk = tp.depth(k);
    const S* rows = W + L.SK + 8 * tp.skoff(k);
    S v[6], a[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) v[e] = S(0);
    ld6(W + U + L.GR + 8 * k, a);
    for (int d = 0; d <= dk; ++d) {
      S s[8];
      ld4(rows + 8 * d, s);
      ld4(rows + 8 * d + 4, s + 4);
      const S qd = s[6];
      S sq[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) { sq[e] = s[e] * qd; v[e] += sq[e]; }
      crm_mul_acc(v, sq, a);
      S qdd = S(0);
      if (qdd_off >= 0) qdd = W[qdd_off + tp.perm(row_body<Tp>(k, dk, d, s[7]))];
#pragma unroll
      for (int e = 0; e < 6; ++e) a[e] += s[e] * qdd;
    }
    S g[6], ia[6];
    i_mul(M.inert[k], v, g);
    i_mul(M.inert[k], a, ia);
    crf_mul_acc(v, g, ia);
    st6(W + L.VG + 12 * k, v);
    st6u(W + L.VG + 12 * k + 6, g);
    st6(W + U + L.A + 8 * k, a);
    st6(W + U + L.F + 8 * k, ia);
  }
  SYNC();
}

// ---------------------------------------------------------------- B5
// Joint forces from body forces: c_i = S_i^T F_i = sum_{k in subtree(i)} s_i^(k) . f_k
// (the RNEA backward sweep F_p += X^T F_i, tau_i = S_i^T F_i, unrolled).
template <class S, int T, class Tp>
__device__ void ph_joint_forces(const Ctx<S, Tp>& c, int f_off, int out_off) {
  const ModelDev<S>& M = c.M;
  const Tp& tp = c.tp;
  S* W = c.W;
  const KnotLayout L = c.tp.layout();   // by value: offsets stay in registers
  if constexpr (Tp::kChainN > 0) {
    // Chain: the backward sweep F_k = f_k + X_{k+1}^T F_{k+1}, c_k = S_k^T F_k, in
    // every lane (broadcast reads of f and X; lane k stores c_k).
    S F[6] = {S(0), S(0), S(0), S(0), S(0), S(0)};
#pragma unroll
    for (int k = Tp::kChainN - 1; k >= 0; --k) {
      S f[6];
      ld6(W + f_off + 8 * k, f);
      if (k + 1 < Tp::kChainN) {
        S E[12], x[6];
        ld12(W + L.X + 12 * (k + 1), E);
        xt_mul(E, E + 9, F, x);
#pragma unroll
        for (int e = 0; e < 6; ++e) f[e] += x[e];
      }
#pragma unroll
      for (int e = 0; e < 6; ++e) F[e] = f[e];
      if (c.l == k) W[out_off + k] = dot_s(M.axis[k], false, F);
    }
    SYNC();
    return;
  }
  for (int i = c.l; i < tp.n(); i += T) {
    const int di = tp.depth(i);
    S acc = S(0);
    for (int k = i; k < tp.sub_end(i); ++k) {
      S s[6], f[6];
      ld6(W + L.SK + 8 * (tp.skoff(k) + di), s);
      ld6(W + f_off + 8 * k, f);
      acc += dot6(s, f);
    }
    W[out_off + i] = acc;
  }
  SYNC();
}

// ---------------------------------------------------------------- B6
template <class S, int T, class Tp>
__device__ void ph_fd(const Ctx<S, Tp>& c) {
  const ModelDev<S>& M = c.M;
  const Tp& tp = c.tp;
  S* W = c.W;
  const KnotLayout L = c.tp.layout();   // by value: offsets stay in registers
  const int n = tp.n();
  for (int i = c.l; i < n; i += T) {
    S acc = S(0);
#pragma unroll (Tp::kUnroll)
    for (int j = tp.comp_lo(i); j < tp.comp_hi(i); ++j)
      acc += W[L.MINV + i * L.MS + j] * (W[L.TAU + tp.perm(j)] - W[L.CB + j]);
    W[L.QDD + i] = acc;
  }
  SYNC();
}

// ---------------------------------------------------------------- B7
// RNEA at the computed qdd: a_k += sum_m s_m^(k) qdd_m, f_k += I_k (that);
// beta_k = (X_k a_p) x S_k with X_k a_p = a_k - (v_k x S_k) qd_k - S_k qdd_k
// (so beta_k = (a_k - qd_k v_k x S_k) x S_k, as S x S = 0). Then the
// accumulated forces F_i = f_i + sum_children X_c^T F_c (lanes over
// components) and phi_i = S_i x* F_i.
template <class S, int T, bool ADD_QDD, class Tp>
__device__ void ph_update_and_forces(const Ctx<S, Tp>& c) {
  const ModelDev<S>& M = c.M;
  const Tp& tp = c.tp;
  S* W = c.W;
  const KnotLayout L = c.tp.layout();   // by value: offsets stay in registers
  const int U = L.UNION;
  const int l = c.l;
  S* FA = W + U + L.F;                     // own forces, made accumulated in place
  S* FSL = W + U + L.FSL;
  for (int e = l; e < 8 * tp.nbranch(); e += T) FSL[e] = S(0);
  for (int k = l; k < tp.n(); k += T) {
    const int dk = tp.depth(k);
    const S* rows = W + L.SK + 8 * tp.skoff(k);
    S da[6] = {S(0), S(0), S(0), S(0), S(0), S(0)};
    if (ADD_QDD) {                          // accelerations so far exclude qdd
      for (int d = 0; d <= dk; ++d) {
        S s[8];
        ld4(rows + 8 * d, s);
        ld4(rows + 8 * d + 4, s + 4);
        const S qdd = W[L.QDD + row_body<Tp>(k, dk, d, s[7])];
#pragma unroll
        for (int e = 0; e < 6; ++e) da[e] += s[e] * qdd;
      }
    }
    const S* ax = M.axis[k];
    S v[6], a[6], fo[6];
    ld6(W + L.VG + 12 * k, v);
    ld6(W + U + L.A + 8 * k, a);
    ld6(FA + 8 * k, fo);
    const S qdk = W[L.QD + tp.perm(k)];
    const bool pr = tp.prism(k);
    S vxs[6], w[6];
    i_mul_acc(M.inert[k], da, fo);
    cross_s(v, ax, pr, vxs);
#pragma unroll
    for (int e = 0; e < 6; ++e) w[e] = a[e] + da[e] - qdk * vxs[e];
    st6(FA + 8 * k, fo);
    S B[6];
    cross_s(w, ax, pr, B);
    st6(W + L.BPH + 12 * k, B);
  }
  SYNC();
  if constexpr (Tp::kChainN > 0) {
    // Chain: every lane carries the whole accumulated force, F_k = f_k + X_{k+1}^T F_{k+1}
    // (no exchange between lanes; lane 0 stores it).
    S F[6] = {S(0), S(0), S(0), S(0), S(0), S(0)};
#pragma unroll
    for (int k = Tp::kChainN - 1; k >= 0; --k) {
      S f[6];
      ld6(FA + 8 * k, f);
      if (k + 1 < Tp::kChainN) {
        S E[12], x[6];
        ld12(W + L.X + 12 * (k + 1), E);
        xt_mul(E, E + 9, F, x);
#pragma unroll
        for (int e = 0; e < 6; ++e) f[e] += x[e];
      }
#pragma unroll
      for (int e = 0; e < 6; ++e) F[e] = f[e];
      SYNC();                                  // every lane has read f_k before it is overwritten
      if (l == 0) st6(FA + 8 * k, F);
    }
  } else {
    // Leaves to root: lane l < 6 holds component l of F_k; the full vector is
    // gathered by warp shuffles. A child's X^T F passes in a register to its
    // parent when the parent is the next body (k - 1), else through a slot.
    const int base = c.lane32 - l;
    S carry = S(0);
#pragma unroll (Tp::kUnroll)
    for (int k = tp.n() - 1; k >= 0; --k) {
      const int p = tp.parent(k);
      const int br = tp.branch(k);
      S fk = S(0);
      if (l < 6) {
        fk = FA[8 * k + l];
        if (k + 1 < tp.n() && tp.parent(k + 1) == k) fk += carry;
        if (br >= 0) fk += FSL[8 * br + l];
      }
      S F[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) F[e] = GRID_SHFL(fk, base + e);
      if (l < 6) {
        FA[8 * k + l] = fk;
        if (p >= 0) {
          const S cl = xt_mul_c(W + L.X + 12 * k, F, l);
          if (p == k - 1) carry = cl;
          else FSL[8 * tp.branch(p) + l] += cl;
        }
      }
    }
  }
  SYNC();
  for (int k = l; k < tp.n(); k += T) {
    S F[6];
    ld6(FA + 8 * k, F);
    const S* ax = M.axis[k];
    S Ph[6];                                   // S x* F
    crf_s(ax, tp.prism(k), F, Ph);
    st6u(W + L.BPH + 12 * k + 6, Ph);
  }
  SYNC();
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
template <class S, int T, int MAXD, class Tp>
__device__ void ph_columns(const Ctx<S, Tp>& c, const uint32_t* __restrict__ sched, int nsteps) {
  const ModelDev<S>& M = c.M;
  const Tp& tp = c.tp;
  S* W = c.W;
  const KnotLayout L = c.tp.layout();   // by value: offsets stay in registers
  const int n = tp.n();
  const int U = L.UNION;
  S* DC = W + U + L.DC;
  // In a chain every column has one path (j .. n-1), which writes its whole
  // column of dc at the end; elsewhere several paths add into it.
  if constexpr (Tp::kChainN == 0) {
    for (int e = c.l; e < 2 * n * n; e += T) DC[e] = S(0);
  }
  SYNC();
  S dv[6], da[6], acc[MAXD];
#pragma unroll
  for (int e = 0; e < 6; ++e) { dv[e] = S(0); da[e] = S(0); }
#pragma unroll
  for (int d = 0; d < MAXD; ++d) acc[d] = S(0);
  uint32_t st_next = nsteps > 0 ? sched[c.l] : 0u;   // descriptors are fetched one step ahead
  for (int s = 0; s < nsteps; ++s) {
    const uint32_t st = st_next;
    if (s + 1 < nsteps) st_next = sched[(s + 1) * T + c.l];
    if (!(st & STEP_VALID)) continue;
    const int k = STEP_BODY(st);
    const int col = STEP_COL(st);
    const bool root = st & STEP_ROOT, uq = st & STEP_UQ;
    const bool rs = st & STEP_RESET;           // first step of a path: no parent derivatives
#pragma unroll
    for (int e = 0; e < 6; ++e) { dv[e] = rs ? S(0) : dv[e]; da[e] = rs ? S(0) : da[e]; }
    const int dk = STEP_DEPTH(st);
    const S* rows = W + L.SK + 8 * STEP_SKOFF(st);
    S E[12];
    ld12(W + L.X + 12 * k, E);
    const S* r = E + 9;
    S ax[4], in[12];
    ld4(M.axis[k], ax);
    ld4(M.inert[k], in);
    ld4(M.inert[k] + 4, in + 4);
    ld4(M.inert[k] + 8, in + 8);
    const S qdk = rows[8 * dk + 6];            // qd_k is stored in body k's own subspace row
    S vg[12];
    ld12(W + L.VG + 12 * k, vg);
    const S* v = vg;
    const S* g = vg + 6;
    S ndv[6], nda[6], vxs[6];
    x_mul(E, r, dv, ndv);
    x_mul(E, r, da, nda);
    const bool pr = tp.prism(k);
    cross_s(v, ax, pr, vxs);     // v x S
    if (root) {                   // case terms at the column's own joint
      if (uq) {
        S B[6];
        ld6(W + L.BPH + 12 * k, B);
#pragma unroll
        for (int e = 0; e < 6; ++e) { ndv[e] += vxs[e]; nda[e] += B[e]; }
      } else {
        S s6[6];
        joint_s(ax, pr, s6);
#pragma unroll
        for (int e = 0; e < 6; ++e) { ndv[e] += s6[e]; nda[e] += vxs[e]; }
      }
    }
    {
      const S sq[3] = {ax[0] * qdk, ax[1] * qdk, ax[2] * qdk};
      cross_s_acc(ndv, sq, pr, nda);   // + dv x S qd
    }
    S df[6], idv[6];
    i_mul(in, nda, df);
    crf_mul_acc(ndv, g, df);
    i_mul(in, ndv, idv);
    crf_mul_acc(v, idv, df);
    if (root && uq) {                          // backward-pass term S x* F of Alg. 1
      S Ph[6];
      ld6u(W + L.BPH + 12 * k + 6, Ph);
#pragma unroll
      for (int e = 0; e < 6; ++e) df[e] += Ph[e];
    }
    if constexpr (Tp::kChainN > 0) {
      // chain: body d is the ancestor at depth d; every step owns its body.
      // Rows past depth dk are not needed: their loads read the rows of the
      // next bodies (inside the table: skoff(k) + N - 1 < N (N + 1) / 2) and
      // the result is discarded, which keeps the loop free of branches and
      // its addresses constant offsets.
      static_assert(Tp::kChainN <= MAXD, "accumulators");
#pragma unroll
      for (int d = 0; d < Tp::kChainN; ++d) {
        if (d <= dk) {                         // lanes past their depth load nothing
          S sr[6];
          ld6(rows + 8 * d, sr);
          acc[d] += dot6(sr, df);
        }
      }
      if (st & STEP_FLUSH) {                  // the path ends at body n - 1: all depths
#pragma unroll
        for (int d = 0; d < Tp::kChainN; ++d) {
          DC[d * 2 * n + col] = acc[d];
          acc[d] = S(0);
        }
      }
    } else {
      if (st & STEP_OWNED) {
#pragma unroll
        for (int d = 0; d < MAXD; ++d) {
          if (d <= dk) {
            S sr[6];
            ld6(rows + 8 * d, sr);
            acc[d] += dot6(sr, df);
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
            b = tp.parent(b);
          }
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
// With PL (a part placed in a robot's arrays) rows and columns go to the
// robot's joints gidx[i], in rows of rs = 2 ld with the d/dqd block at cqd = ld.
template <class S, int T, int CPL, class Tp, bool PL = false>
__device__ void ph_product(const Ctx<S, Tp>& c, S* __restrict__ J, int rs = 0, int cq = 0, int cqd = 0) {
  const ModelDev<S>& M = c.M;
  const Tp& tp = c.tp;
  S* W = c.W;
  const KnotLayout L = c.tp.layout();   // by value: offsets stay in registers
  const int n = tp.n(), n2 = 2 * n, MS = L.MS;
  const int U = L.UNION;
  const S* DC = W + U + L.DC;
  const S* MI = W + L.MINV;
  if (rs == 0) { rs = n2; cq = 0; cqd = n; }   // J rows of 2n; else rows of rs with the blocks at cq, cqd
  constexpr int NM = CPL * T;                  // >= n, a multiple of 4
  // Lane owns output columns col = l, l + T, ...: its dc column sits in
  // registers and every M^-1 row is read with 128-bit loads. J (this knot
  // point's [n][2n] block in caller order, or NULL for a padding knot point) is
  // written directly: the group's lanes cover consecutive columns of a row.
  for (int col = c.l; col < n2; col += T) {
    const int j = col < n ? col : col - n;
    const int lo = tp.comp_lo(j), hi = tp.comp_hi(j);
    S dcr[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) dcr[m] = (m >= lo && m < hi) ? DC[m * n2 + col] : S(0);
    const int ucol = (col < n ? cq : cqd) + (PL ? c.gM->gidx[j] : tp.perm(j));
    if (J) {
      for (int i = 0; i < lo; ++i) J[(PL ? c.gM->gidx[i] : tp.perm(i)) * rs + ucol] = S(0);   // other base branches
      for (int i = hi; i < n; ++i) J[(PL ? c.gM->gidx[i] : tp.perm(i)) * rs + ucol] = S(0);
    }
#pragma unroll (Tp::kUnroll)
    for (int i = lo; i < hi; ++i) {
      const S* mrow = MI + i * MS;
      S acc = S(0);
#pragma unroll
      for (int m = 0; m < NM; m += 4) {
        if (m < MS) {
          S mm[4];
          ld4(mrow + m, mm);
          acc += mm[0] * dcr[m] + mm[1] * dcr[m + 1] + mm[2] * dcr[m + 2] + mm[3] * dcr[m + 3];
        }
      }
      if (J) J[(PL ? c.gM->gidx[i] : tp.perm(i)) * rs + ucol] = -acc;
    }
  }
  SYNC();
}

// ---------------------------------------------------------------- V
// Vector-Jacobian product through FD. For gbar = dL/dqdd and lambda = M^-1 gbar:
//   dL/dtau = lambda,  dL/dq = -(dID/dq)^T lambda,  dL/dqd = -(dID/dqd)^T lambda,
// evaluated without forming dID by reverse-mode differentiation of RNEA. With
// psi_k = sum_{m on the root path of k} lambda_m s_m^(k) (lambda used as a
// joint velocity), lambda^T ID = sum_k psi_k . f_k, whose adjoint seeds are
//   abar_k = I_k psi_k,  vbar_k = -psi_k x* gamma_k - I_k (v_k x psi_k).
// One sweep from the leaves accumulates
//   Abar_k = abar_k + sum_children X_c^T Abar_c,
//   Vbar_k = vbar_k + (S_k qd_k) x* Abar_k + sum_children X_c^T Vbar_c,
// and for joint k
//   (dID/dqd)^T lambda |_k = S_k^T Vbar_k + Abar_k . (v_k x S_k)
//   (dID/dq)^T lambda  |_k = Vbar_k . (v_k x S_k) + Abar_k . beta_k + F_k . (psi_k x S_k).
template <class S, int T, class Tp>
__device__ void ph_vjp_seeds(const Ctx<S, Tp>& c) {
  const ModelDev<S>& M = c.M;
  const Tp& tp = c.tp;
  S* W = c.W;
  const KnotLayout L = c.tp.layout();   // by value: offsets stay in registers
  const int U = L.UNION;
  const int n = tp.n();
  for (int i = c.l; i < n; i += T) {
    S acc = S(0);
#pragma unroll (Tp::kUnroll)
    for (int j = tp.comp_lo(i); j < tp.comp_hi(i); ++j) acc += W[L.MINV + i * L.MS + j] * W[U + L.GB + tp.perm(j)];
    W[U + L.LAM + i] = acc;
  }
  SYNC();
  for (int k = c.l; k < n; k += T) {
    const int dk = tp.depth(k);
    const S* rows = W + L.SK + 8 * tp.skoff(k);
    S psi[6] = {S(0), S(0), S(0), S(0), S(0), S(0)};
    for (int d = 0; d <= dk; ++d) {
      S s[8];
      ld4(rows + 8 * d, s);
      ld4(rows + 8 * d + 4, s + 4);
      const S lam = W[U + L.LAM + row_body<Tp>(k, dk, d, s[7])];
#pragma unroll
      for (int e = 0; e < 6; ++e) psi[e] += s[e] * lam;
    }
    S vg[12], t1[6], vxp[6], t2[6];
    ld12(W + L.VG + 12 * k, vg);
    const S* v = vg;
    const S* g = vg + 6;
    i_mul(M.inert[k], psi, t1);
    st6(W + U + L.AB + 8 * k, t1);
    crf_mul(psi, g, t1);
    crm_mul(v, psi, vxp);
    i_mul(M.inert[k], vxp, t2);
#pragma unroll
    for (int e = 0; e < 6; ++e) t1[e] = -t1[e] - t2[e];
    st6(W + U + L.VB + 8 * k, t1);
    st6(W + U + L.PSI + 8 * k, psi);
  }
  for (int e = c.l; e < 8 * tp.nbranch(); e += T) { W[U + L.SA + e] = S(0); W[U + L.SV + e] = S(0); }
  SYNC();
}

template <class S, int T, class Tp>
__device__ void ph_vjp_sweep(const Ctx<S, Tp>& c) {
  const ModelDev<S>& M = c.M;
  const Tp& tp = c.tp;
  S* W = c.W;
  const KnotLayout L = c.tp.layout();   // by value: offsets stay in registers
  const int U = L.UNION;
  const int l = c.l;
  const int base = c.lane32 - l;
  S* SA = W + U + L.SA;
  S* SV = W + U + L.SV;
  S ca = S(0), cv = S(0);
#pragma unroll (Tp::kUnroll)
  for (int k = tp.n() - 1; k >= 0; --k) {
    const int p = tp.parent(k);
    const int br = tp.branch(k);
    const bool from_next = k + 1 < tp.n() && tp.parent(k + 1) == k;
    const S* ax = M.axis[k];
    const bool pr = tp.prism(k);
    const S qdk = W[L.QD + tp.perm(k)];
    S ab = S(0), vb = S(0);
    if (l < 6) {
      ab = W[U + L.AB + 8 * k + l] + (from_next ? ca : S(0)) + (br >= 0 ? SA[8 * br + l] : S(0));
      vb = W[U + L.VB + 8 * k + l] + (from_next ? cv : S(0)) + (br >= 0 ? SV[8 * br + l] : S(0));
    }
    S A[6], V[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) A[e] = GRID_SHFL(ab, base + e);
    {
      // (S qd) x* Abar
      const S sq[3] = {ax[0] * qdk, ax[1] * qdk, ax[2] * qdk};
      S t[6];
      crf_s(sq, pr, A, t);
      S add = t[0];
#pragma unroll
      for (int e = 1; e < 6; ++e) add = (l == e) ? t[e] : add;
      if (l < 6) vb += add;
    }
#pragma unroll
    for (int e = 0; e < 6; ++e) V[e] = GRID_SHFL(vb, base + e);
    if (l == 0) {
      S v[6], B[6], F[6], psi[6], vxs[6], pxs[6];
      ld6(W + L.VG + 12 * k, v);
      ld6(W + L.BPH + 12 * k, B);
      ld6(W + U + L.F + 8 * k, F);
      ld6(W + U + L.PSI + 8 * k, psi);
      cross_s(v, ax, pr, vxs);
      cross_s(psi, ax, pr, pxs);
      S gqd = dot_s(ax, pr, V);
      S gq = S(0);
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        gqd += A[e] * vxs[e];
        gq += V[e] * vxs[e] + A[e] * B[e] + F[e] * pxs[e];
      }
      W[U + L.DQ + k] = -gq;
      W[U + L.DQD + k] = -gqd;
    }
    if (p >= 0 && l < 6) {
      const S xa = xt_mul_c(W + L.X + 12 * k, A, l);
      const S xv = xt_mul_c(W + L.X + 12 * k, V, l);
      if (p == k - 1) { ca = xa; cv = xv; }
      else { SA[8 * tp.branch(p) + l] += xa; SV[8 * tp.branch(p) + l] += xv; }
    }
  }
  SYNC();
}

// One warp processes knot points k0 .. k0 + 32/T - 1 (those < N). M is the
// shared-memory copy of the model, gM the same model in device memory.
// CHAIN_N: 0 run-time topology, 0 < N < 100 a chain of N bodies, 100 + N a chain of
// N bodies that is a part placed in a robot's arrays, -(100 K + L) a forest of K
// chains of L
template <class S, int MODE, int CHAIN_N>
using topo_for = typename grid_cond<
    CHAIN_N == 0, RtTopo<S, MODE>,
    typename grid_cond<(CHAIN_N > 0),
                       ChainTopo<S, MODE, (CHAIN_N > 0 ? CHAIN_N % 100 : 1), (CHAIN_N > 100)>,
                       ForestTopo<S, MODE, (CHAIN_N < 0 ? -CHAIN_N / 100 : 1),
                                  (CHAIN_N < 0 ? -CHAIN_N % 100 : 1)>>::type>::type;

template <class S, int MODE, int T, int CPL, int MAXD, bool MIXED, class Tp>
__device__ void process_tile_t(const ModelDev<S>& M, const ModelDev<S>* gM, const uint32_t* __restrict__ sched,
                             int nsteps, S* Wwarp, int lane32, int k0, int N, const S* __restrict__ q,
                             const S* __restrict__ qd, const S* __restrict__ x3,
                             const S* __restrict__ x4, S* __restrict__ out, S* __restrict__ out2,
                             S* __restrict__ out3) {
  using P = typename grid_cond<MIXED, double, S>::type;
  const Tp tp(M);
  const auto& L = tp.layout();     // the staged layout (runtime topology) or a compile-time constant
  const int n = tp.n();
  constexpr int G = 32 / T;
  const int g = lane32 / T;
  S* W = Wwarp + g * L.stride;
  const Ctx<S, Tp> c{M, gM, tp, W, lane32 % T, lane32};
  const int nvalid = min(G, N - k0);
  // A part placed in a robot's arrays (MODE_GRAD only) reads and writes the
  // robot's joints of its own: knot point k's slot s is at k ld + gslot[s].
  const bool placed = MODE == MODE_GRAD && (Tp::kPlace == 2 ? M.ld != n : Tp::kPlace == 1);
  if (placed) {
    for (int e = lane32; e < G * n; e += 32) {
      const int kk = e / n, i = e % n;
      S* Wk = Wwarp + kk * L.stride;
      const bool ok = kk < nvalid;
      const size_t gi = (size_t)(k0 + kk) * M.ld + gM->gslot[i];
      Wk[L.Q + i] = ok ? q[gi] : S(0);
      Wk[L.QD + i] = ok ? qd[gi] : S(0);
      Wk[L.TAU + i] = ok ? x3[gi] : S(0);
    }
  } else {
    // stage inputs (coalesced across the warp)
    for (int e = lane32; e < G * n; e += 32) {
      const int kk = e / n, i = e % n;
      S* Wk = Wwarp + kk * L.stride;
      const bool ok = kk < nvalid;
      const size_t gi = (size_t)k0 * n + e;
      Wk[L.Q + i] = ok ? q[gi] : S(0);
      if (MODE != MODE_MINV) Wk[L.QD + i] = ok ? qd[gi] : S(0);
      if (MODE == MODE_RNEA || MODE == MODE_GRAD_ID) Wk[L.TAU + i] = (ok && x3) ? x3[gi] : S(0);
      if (MODE == MODE_FD || MODE == MODE_GRAD || MODE == MODE_VJP) Wk[L.TAU + i] = ok ? x3[gi] : S(0);
      if (MODE == MODE_VJP) Wk[L.UNION + L.GB + i] = ok ? x4[gi] : S(0);
    }
  }
  SYNC();
  ph_transforms<S, T>(c);
  if (MODE == MODE_MINV) {
    ph_minv<S, P, T, CPL, false>(c);
  } else if (MODE == MODE_RNEA || MODE == MODE_GRAD_ID) {
    ph_subspaces<S, T>(c);
    ph_rnea_bodies<S, T>(c, L.TAU);                 // qdd given (caller order)
    if (MODE == MODE_RNEA) ph_joint_forces<S, T>(c, L.UNION + L.F, L.CB);
    if (MODE == MODE_GRAD_ID) {
      ph_update_and_forces<S, T, false>(c);
      ph_columns<S, T, MAXD>(c, sched, nsteps);     // dc = [dID/dq | dID/dqd]
    }
  } else {
    ph_minv<S, P, T, CPL, true>(c);                 // also builds the subspace table
    ph_rnea_bodies<S, T>(c, -1);
    ph_joint_forces<S, T>(c, L.UNION + L.F, L.CB);  // CB = RNEA(q, qd, 0)
    ph_fd<S, T>(c);
    ph_update_and_forces<S, T, true>(c);
    if (MODE == MODE_GRAD) {
      ph_columns<S, T, MAXD>(c, sched, nsteps);
      if constexpr (Tp::kBranches > 0) {
        // rows b n .. b n + n - 1 of the K n-joint knot point: the chain's blocks at
        // columns b n and K n + b n, zeros in the rest of those rows
        constexpr int K = Tp::kBranches;
        const int nr = K * n, b = (k0 + g) % K;
        S* Jb = g < nvalid ? out + (size_t)((k0 + g) / K) * 2 * nr * nr + (size_t)b * n * 2 * nr : nullptr;
        ph_product<S, T, CPL>(c, Jb, 2 * nr, b * n, nr + b * n);
        if (Jb) {
          for (int e = c.l; e < n * 2 * nr; e += T) {
            const int col = e % (2 * nr), u = col < nr ? col - b * n : col - nr - b * n;
            if (u < 0 || u >= n) Jb[e] = S(0);
          }
        }
      } else if (placed) {
        // the part's rows of the robot's J: its blocks, zeros in the other columns
        const int ld = M.ld;
        S* Jk = g < nvalid ? out + (size_t)(k0 + g) * 2 * ld * ld : nullptr;
        ph_product<S, T, CPL, Tp, true>(c, Jk, 2 * ld, 0, ld);
        if (Jk) {
          for (int e = c.l; e < n * 2 * ld; e += T) {
            const int i = e / (2 * ld), cc = e % (2 * ld), jj = cc < ld ? cc : cc - ld;
            if (!((M.gmask >> jj) & 1u)) Jk[gM->gidx[i] * 2 * ld + cc] = S(0);
          }
        }
      } else {
        ph_product<S, T, CPL>(c, g < nvalid ? out + (size_t)(k0 + g) * 2 * n * n : nullptr);
      }
    }
    if (MODE == MODE_VJP) {
      ph_vjp_seeds<S, T>(c);
      ph_vjp_sweep<S, T>(c);
    }
  }
  if constexpr (MODE == MODE_GRAD) {
    if (out2) {                                     // qdd in caller order
      for (int i = c.l; i < n; i += T) W[L.CB + tp.perm(i)] = W[L.QDD + i];
      SYNC();
      if (placed) {
        for (int e = lane32; e < nvalid * n; e += 32) {
          const int kk = e / n, r = e % n;
          out2[(size_t)(k0 + kk) * M.ld + gM->gslot[r]] = Wwarp[kk * L.stride + L.CB + r];
        }
      } else {
        for (int e = lane32; e < nvalid * n; e += 32) {
          const int kk = e / n, r = e % n;
          out2[(size_t)k0 * n + e] = Wwarp[kk * L.stride + L.CB + r];
        }
      }
    }
    if (out3 && g < nvalid) {                       // M^-1 in caller order (full symmetric)
      if constexpr (Tp::kBranches > 0) {            // the chain's diagonal block, zeros beside it
        constexpr int K = Tp::kBranches;
        const int nr = K * n, b = (k0 + g) % K;
        S* Mo = out3 + (size_t)((k0 + g) / K) * nr * nr + (size_t)b * n * nr;
        for (int e = c.l; e < n * nr; e += T) {
          const int i = e / nr, u = e % nr - b * n;
          Mo[e] = (u >= 0 && u < n) ? W[L.MINV + i * L.MS + u] : S(0);
        }
      } else if (placed) {                          // the part's block of the robot's M^-1, zeros beside it
        const int ld = M.ld;
        S* Mo = out3 + (size_t)(k0 + g) * ld * ld;
        for (int e = c.l; e < n * n; e += T) {
          const int i = e / n, j = e % n;
          Mo[gM->gidx[i] * ld + gM->gidx[j]] = W[L.MINV + i * L.MS + j];
        }
        for (int e = c.l; e < n * ld; e += T) {
          const int i = e / ld, cc = e % ld;
          if (!((M.gmask >> cc) & 1u)) Mo[gM->gidx[i] * ld + cc] = S(0);
        }
      } else {
        S* Mo = out3 + (size_t)(k0 + g) * n * n;
        for (int e = c.l; e < n * n; e += T) {
          const int i = e / n, j = e % n;
          Mo[tp.perm(i) * n + tp.perm(j)] = W[L.MINV + i * L.MS + j];
        }
      }
    }
    SYNC();
  } else if constexpr (MODE == MODE_VJP) {
    S* OS = W + L.UNION + L.JS;
    for (int i = c.l; i < n; i += T) {
      OS[tp.perm(i)] = W[L.UNION + L.DQ + i];
      OS[n + tp.perm(i)] = W[L.UNION + L.DQD + i];
      OS[2 * n + tp.perm(i)] = W[L.UNION + L.LAM + i];
    }
    SYNC();
    for (int e = lane32; e < nvalid * n; e += 32) {
      const int kk = e / n, r = e % n;
      const S* os = Wwarp + kk * L.stride + L.UNION + L.JS;
      out[(size_t)k0 * n + e] = os[r];
      out2[(size_t)k0 * n + e] = os[n + r];
      out3[(size_t)k0 * n + e] = os[2 * n + r];
    }
    SYNC();
  } else {
    // stage outputs in caller order, then store them with coalesced writes
    const int out_per = MODE == MODE_MINV ? n * n : (MODE == MODE_GRAD_ID ? 2 * n * n : n);
    S* OS = W + L.UNION + L.JS;
    if (MODE == MODE_RNEA) {
      for (int i = c.l; i < n; i += T) OS[tp.perm(i)] = W[L.CB + i];
    } else if (MODE == MODE_FD) {
      for (int i = c.l; i < n; i += T) OS[tp.perm(i)] = W[L.QDD + i];
    } else if (MODE == MODE_MINV) {
      for (int e = c.l; e < n * n; e += T) OS[tp.perm(e / n) * n + tp.perm(e % n)] = W[L.MINV + (e / n) * L.MS + e % n];
    } else {
      const S* DC = W + L.UNION + L.DC;
      for (int e = c.l; e < 2 * n * n; e += T) {    // dc is [i][u n + j]
        const int i = e / (2 * n), col = e % (2 * n), j = col < n ? col : col - n;
        OS[tp.perm(i) * 2 * n + (col < n ? 0 : n) + tp.perm(j)] = DC[e];
      }
    }
    SYNC();
    for (int e = lane32; e < nvalid * out_per; e += 32) {
      const int kk = e / out_per, r = e % out_per;
      out[(size_t)k0 * out_per + e] = Wwarp[kk * L.stride + L.UNION + L.JS + r];
    }
    SYNC();
  }
}

template <class S, int MODE, int T, int CPL, int MAXD, bool MIXED, int CHAIN_N = 0>
__device__ __forceinline__ void process_tile(const ModelDev<S>& M, const ModelDev<S>* gM, const uint32_t* __restrict__ sched,
                             int nsteps, S* Wwarp, int lane32, int k0, int N, const S* __restrict__ q,
                             const S* __restrict__ qd, const S* __restrict__ x3,
                             const S* __restrict__ x4, S* __restrict__ out, S* __restrict__ out2,
                             S* __restrict__ out3) {
  process_tile_t<S, MODE, T, CPL, MAXD, MIXED, topo_for<S, MODE, CHAIN_N>>(M, gM, sched, nsteps, Wwarp, lane32, k0, N, q, qd, x3, x4, out, out2, out3);
}
