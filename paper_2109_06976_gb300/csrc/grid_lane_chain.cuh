// One lane per knot point for serial chains of revolute joints (device code and
// launcher; instantiated by grid_lane_chain.cu for the gradient of FD and by
// grid_lane_chain_fdv.cu for FD and the vector-Jacobian product through FD).
//
// Each lane evaluates the whole method for its own knot point, in the order of
// Sec. IV-B: joint transforms, the direct M^-1 (articulated-inertia recursion,
// backward then forward sweep), RNEA(q, qd, 0), qdd = M^-1 (tau - c), RNEA at
// qdd, then per derivative column (u, j) the forward pass of Alg. 1 over the
// bodies j .. n-1 and its backward pass down to the base (with the readings of
// the paper used by every kernel here: the case terms act only at the column's
// own joint, the velocity-product term uses dv_k, and the accumulated force F_j
// enters X_j^T (S_j x* F_j) for u = q), and J = -M^-1 dc column by column. FD
// stops after qdd; the vector-Jacobian product replaces the columns by one
// adjoint sweep.
//
// The lanes exchange no data while they compute (no shuffles, no warp barriers;
// only a chain placed in a larger robot hands its blocks of J and M^-1 to the
// warp at the end, for whole-row stores). What a lane
// keeps between phases (its transforms, velocities, the case-term vectors beta
// and phi, the M^-1 temporaries) sits in shared memory in a lane-major layout:
// slot s of lane t of a warp is element s * 32 + t of the warp's area, so a
// warp's 128-bit access moves 32 lanes' records in 4 wavefronts without bank
// conflicts, against one wavefront per knot point for the kernels whose lanes
// cooperate on one knot point. The robot's constants (axes, fixed transforms,
// inertias, gravity, placement) are kernel parameters, uniform across the warp.
// M^-1 and the per-column force derivatives live in registers.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "grid_internal.h"
#include "spatial.cuh"

namespace {

constexpr int kLcMaxB = 8;

// The robot's constants, passed by value.
struct LcParams {
  float axis[kLcMaxB][3];
  float rT[kLcMaxB][3];
  float ET[kLcMaxB][9];
  float inert[kLcMaxB][10];   // m, h = m c (3), Ibar about the body origin: xx yy zz xy xz yz
  float2 ip[kLcMaxB][9];      // the same, paired for lc_i_mul (see there)
  float a0[6];                // base acceleration -g
  unsigned et_ident;          // bit i: the fixed rotation of body i is the identity
  // Placement in the caller's arrays (a chain that is one component of a larger
  // robot): joints per knot point, the caller joint of body i, and a bit for
  // each caller joint of the chain. A whole robot has ld = n, slot[i] = i.
  int ld;
  int slot[kLcMaxB];
  unsigned mask;
};


// Lane-major workspace of one warp. Per body i, float4 slots 7 i + 0..6:
//   E0 = E[0..3], E1 = E[4..7], V0 = v[0..3], V1 = {v4, v5, E[8], qd_i},
//   B0 = beta[0..3], B1 = phi[0..3], B2 = {beta4, beta5, phi4, phi5}
// (while M^-1 is formed: V0, V1.xy hold U_i, B0 and B1 row i of M^-1 by column
// index, B2.x D_i^-1; between the RNEA passes B0, B2.xy hold X_i a_parent and
// B1, B2.zw the force f_i), then scalar slots 0 .. 7 (the bias forces c, then
// qdd). I v is recomputed where the columns need it, and M^-1 and dc sit in
// registers: 816 B per knot point of the 7-DoF chain, so that eight warps (two
// per scheduler) fit on an SM.
template <int NB, int PB = 7>
struct LcLayout {
  static constexpr int kMi = NB * (NB + 1) / 2;      // packed upper triangle of M^-1
  static constexpr int kPB = PB;
  static constexpr int kS4 = PB * NB;
  static constexpr int kS1 = 8;
  static constexpr int kWarpBytes = 32 * (16 * kS4 + 4 * kS1);
};

struct LcWs {
  float4* s4;   // this lane's element of float4 slot 0
  float* s1;
  __device__ float4& f4(int s) const { return s4[s * 32]; }
  __device__ float& f1(int s) const { return s1[s * 32]; }
};

// o = I_i m (o += I_i m for lc_i_mul_acc) in paired FP32: components k and 3 + k
// share three paired multiply-adds, with the coefficient pairs of ip[i]
//   (Ixx, m) (Ixy, h2) (Ixz, -h1) | (Iyy, m) (Ixy, -h2) (Iyz, h0) | (Izz, m) (Ixz, h1) (Iyz, -h0)
// against (m_k, m_3+k) and two broadcast operands; the two remaining terms of the
// angular component k (h x v) are scalar multiply-adds.
template <bool ACC>
__device__ __forceinline__ void lc_i_mul_t(const LcParams& P, int i, const float* m, float* o) {
  const float2* c = P.ip[i];
  const float h0 = P.inert[i][1], h1 = P.inert[i][2], h2 = P.inert[i][3];
  float2 a0, a1, a2;
  if constexpr (ACC) {
    a0 = __ffma2_rn(c[0], make_float2(m[0], m[3]), make_float2(o[0], o[3]));
    a1 = __ffma2_rn(c[3], make_float2(m[1], m[4]), make_float2(o[1], o[4]));
    a2 = __ffma2_rn(c[6], make_float2(m[2], m[5]), make_float2(o[2], o[5]));
  } else {
    a0 = __fmul2_rn(c[0], make_float2(m[0], m[3]));
    a1 = __fmul2_rn(c[3], make_float2(m[1], m[4]));
    a2 = __fmul2_rn(c[6], make_float2(m[2], m[5]));
  }
  a0 = __ffma2_rn(c[1], make_float2(m[1], m[1]), a0);
  a0 = __ffma2_rn(c[2], make_float2(m[2], m[2]), a0);
  a1 = __ffma2_rn(c[4], make_float2(m[0], m[0]), a1);
  a1 = __ffma2_rn(c[5], make_float2(m[2], m[2]), a1);
  a2 = __ffma2_rn(c[7], make_float2(m[0], m[0]), a2);
  a2 = __ffma2_rn(c[8], make_float2(m[1], m[1]), a2);
  o[0] = a0.x + h1 * m[5] - h2 * m[4];
  o[1] = a1.x + h2 * m[3] - h0 * m[5];
  o[2] = a2.x + h0 * m[4] - h1 * m[3];
  o[3] = a0.y;
  o[4] = a1.y;
  o[5] = a2.y;
}
__device__ __forceinline__ void lc_i_mul(const LcParams& P, int i, const float* m, float* o) {
  lc_i_mul_t<false>(P, i, m, o);
}
__device__ __forceinline__ void lc_i_mul_acc(const LcParams& P, int i, const float* m, float* o) {
  lc_i_mul_t<true>(P, i, m, o);
}

// E_i, and from the same slots v_i and qd_i
template <int PB>
__device__ __forceinline__ void lc_load_E(const LcWs& w, int i, float* E) {
  const float4 a = w.f4(PB * i), b = w.f4(PB * i + 1);
  E[0] = a.x; E[1] = a.y; E[2] = a.z; E[3] = a.w;
  E[4] = b.x; E[5] = b.y; E[6] = b.z; E[7] = b.w;
  E[8] = w.f4(PB * i + 3).z;
}

template <int PB>
__device__ __forceinline__ void lc_load_v(const LcWs& w, int i, float* v, float& qdi, float& e8) {
  const float4 a = w.f4(PB * i + 2), b = w.f4(PB * i + 3);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y;
  e8 = b.z;
  qdi = b.w;
}

// X_i = X_J(q_i) X_T,i with E_J = R(a, q)^T = cos q 1 + (1 - cos q) a a^T - sin q a~.
__device__ __forceinline__ void lc_transform(const LcParams& P, int i, float q, float* E) {
  const float* a = P.axis[i];
  float s, co;
  sincosf(q, &s, &co);
  const float omc = 1.0f - co;
  float EJ[9];
  EJ[0] = co + omc * a[0] * a[0];      EJ[1] = omc * a[0] * a[1] + s * a[2]; EJ[2] = omc * a[0] * a[2] - s * a[1];
  EJ[3] = omc * a[1] * a[0] - s * a[2]; EJ[4] = co + omc * a[1] * a[1];     EJ[5] = omc * a[1] * a[2] + s * a[0];
  EJ[6] = omc * a[2] * a[0] + s * a[1]; EJ[7] = omc * a[2] * a[1] - s * a[0]; EJ[8] = co + omc * a[2] * a[2];
  if ((P.et_ident >> i) & 1u) {
#pragma unroll
    for (int e = 0; e < 9; ++e) E[e] = EJ[e];
  } else {
    const float* ET = P.ET[i];
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
      for (int v = 0; v < 3; ++v)
        E[3 * u + v] = EJ[3 * u] * ET[v] + EJ[3 * u + 1] * ET[3 + v] + EJ[3 * u + 2] * ET[6 + v];
  }
}

// Structural zeros of the 6x6 spatial inertia [Ibar h~; h~^T m 1]: the diagonal
// of h~ and the off-diagonal entries of m 1.
__device__ __forceinline__ constexpr bool lc_izero(int u, int s) {
  return ((u < 3) != (s < 3) && u % 3 == s % 3) || (u >= 3 && s >= 3 && u != s);
}

// Packed upper triangle of the symmetric n x n M^-1: entry (r, c).
template <int NB>
__device__ __forceinline__ constexpr int lc_tri(int r, int c) {
  return r <= c ? r * NB - r * (r - 1) / 2 + (c - r) : c * NB - c * (c - 1) / 2 + (r - c);
}

// One derivative column (u, j), u = q when uq: the forward pass over bodies
// j .. n-1, the backward pass down to the base (dc_i for every body), then
// J[:, col] = -M^-1 dc. The loops run over the bodies at compile time (the
// bodies before j are skipped by a branch that is uniform across the warp), so
// body indices, shared-memory offsets and the robot's constants are immediate
// operands; one code path serves both kinds of column, which differ only in
// the case terms at the column's own joint.
// A body's record as the column passes read it.
struct LcBody {
  float E[9], v[6], qd;
};

template <int PB>
__device__ __forceinline__ void lc_load_body(const LcWs& w, int i, LcBody& b) {
  const float4 x0 = w.f4(PB * i), x1 = w.f4(PB * i + 1), a = w.f4(PB * i + 2), c = w.f4(PB * i + 3);
  b.E[0] = x0.x; b.E[1] = x0.y; b.E[2] = x0.z; b.E[3] = x0.w;
  b.E[4] = x1.x; b.E[5] = x1.y; b.E[6] = x1.z; b.E[7] = x1.w; b.E[8] = c.z;
  b.v[0] = a.x; b.v[1] = a.y; b.v[2] = a.z; b.v[3] = a.w; b.v[4] = c.x; b.v[5] = c.y;
  b.qd = c.w;
}

// One derivative column (u, j), u = q when uq: the forward pass over bodies
// j .. n-1, the backward pass down to the base (dc_i for every body), then
// J[:, col] = -M^-1 dc. The loops run over the bodies at compile time (the
// bodies before j are skipped by a branch that is uniform across the warp), so
// body indices, shared-memory offsets and the robot's constants are immediate
// operands; one code path serves both kinds of column, which differ only in
// the case terms at the column's own joint. The next body's record is loaded
// before the current body's arithmetic, so that the shared-memory latency
// overlaps it. With STG the column goes to the lane's staging block instead
// (entry (r, c) of the chain's n x 2n block at r * 2n + c), from which the warp
// writes whole rows of J together.
template <int NB, bool PL, bool DC = false, bool STG = false>
__device__ __forceinline__ void lc_column(const LcParams& P, const LcWs& w, int j, bool uq, const float* Mi,
                                          float* __restrict__ Jk) {
  constexpr int PB = 7;
  float df[NB][6];
  float dv[6], da[6];
  LcBody cur, nxt;
  lc_load_body<PB>(w, j, cur);
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    if (i >= j) {
      if (i + 1 < NB) lc_load_body<PB>(w, i + 1, nxt);
      const float* a = P.axis[i];
      const float* v = cur.v;
      float g[6], ndv[6], nda[6], vxs[6];
      lc_i_mul(P, i, v, g);                                 // gamma_i = I_i v_i
      cross_s(v, a, false, vxs);                       // v x S
      if (i == j) {
        // u = q: dv_j = v_j x S_j, da_j = beta_j;  u = qd: dv_j = S_j, da_j = v_j x S_j
        const float4 b0 = w.f4(PB * i + 4), b2 = w.f4(PB * i + 6);
        const float beta[6] = {b0.x, b0.y, b0.z, b0.w, b2.x, b2.y};
        const float s6[6] = {a[0], a[1], a[2], 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int e = 0; e < 6; ++e) {
          ndv[e] = uq ? vxs[e] : s6[e];
          nda[e] = uq ? beta[e] : vxs[e];
        }
      } else {
        x_mul(cur.E, P.rT[i], dv, ndv);
        x_mul(cur.E, P.rT[i], da, nda);
      }
      const float sq[3] = {a[0] * cur.qd, a[1] * cur.qd, a[2] * cur.qd};
      cross_s_acc(ndv, sq, false, nda);                // + dv x S qd
      float f[6], idv[6];
      lc_i_mul(P, i, nda, f);
      crf_mul_acc(ndv, g, f);
      lc_i_mul(P, i, ndv, idv);
      crf_mul_acc(v, idv, f);
      if (i == j && uq && j > 0) {                     // + S_j x* F_j (backward-pass term; it
                                                       // reaches the ancestors of j only)
        const float4 b1 = w.f4(PB * i + 5), b2 = w.f4(PB * i + 6);
        f[0] += b1.x; f[1] += b1.y; f[2] += b1.z; f[3] += b1.w; f[4] += b2.z; f[5] += b2.w;
      }
#pragma unroll
      for (int e = 0; e < 6; ++e) { df[i][e] = f[e]; dv[e] = ndv[e]; da[e] = nda[e]; }
      cur = nxt;
    }
  }
  // backward: dF_i = df_i + X_{i+1}^T dF_{i+1} (df_i = 0 above j's subtree),
  // dc_i = S_i^T dF_i
  float dF[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, dc[NB];
  float Ec[9], En[9];
  lc_load_E<PB>(w, NB - 1, Ec);
#pragma unroll
  for (int i = NB - 1; i >= 0; --i) {
    if (i > 1) lc_load_E<PB>(w, i - 1, En);
    if (i >= j) {
#pragma unroll
      for (int e = 0; e < 6; ++e) dF[e] += df[i][e];
    }
    dc[i] = dot_s(P.axis[i], false, dF);
    if (i > 0) {
      float t[6];
      xt_mul(Ec, P.rT[i], dF, t);
#pragma unroll
      for (int e = 0; e < 6; ++e) dF[e] = t[e];
#pragma unroll
      for (int e = 0; e < 9; ++e) Ec[e] = En[e];
    }
  }
  const int ld = PL ? P.ld : NB;
  const int col = (uq ? 0 : ld) + (PL ? P.slot[j] : j);
#pragma unroll
  for (int rr = 0; rr < NB; ++rr) {
    if constexpr (DC) {                                // the gradient of ID itself (no product)
      if constexpr (STG) Jk[rr * 2 * NB + (uq ? 0 : NB) + j] = dc[rr];
      else if (Jk) Jk[(PL ? P.slot[rr] : rr) * 2 * ld + col] = dc[rr];
    } else {
      float acc = 0.0f;
#pragma unroll
      for (int m = 0; m < NB; ++m) acc += Mi[lc_tri<NB>(rr, m)] * dc[m];
      if constexpr (STG) Jk[rr * 2 * NB + (uq ? 0 : NB) + j] = -acc;
      else if (Jk) Jk[(PL ? P.slot[rr] : rr) * 2 * ld + col] = -acc;
    }
  }
}

// Vector-Jacobian product through FD for one knot point (MODE_VJP), after the
// RNEA passes: with gbar = dL/dqdd and lambda = M^-1 gbar,
//   dL/dtau = lambda,  dL/dq = -(dID/dq)^T lambda,  dL/dqd = -(dID/dqd)^T lambda,
// by reverse-mode differentiation of RNEA, without forming dID: with
// psi_i = X_i psi_{i-1} + S_i lambda_i (lambda used as a joint velocity),
// lambda^T ID = sum_i psi_i . f_i; its adjoint seeds abar_i = I_i psi_i and
// vbar_i = -psi_i x* (I_i v_i) - I_i (v_i x psi_i); one sweep from the leaf
//   Abar_i = abar_i + X_{i+1}^T Abar_{i+1},
//   Vbar_i = vbar_i + (S_i qd_i) x* Abar_i + X_{i+1}^T Vbar_{i+1},
// and for joint i
//   (dID/dqd)^T lambda |_i = S_i^T Vbar_i + Abar_i . (v_i x S_i),
//   (dID/dq)^T lambda |_i = Vbar_i . (v_i x S_i) + Abar_i . beta_i + F_i . (psi_i x S_i).
// Slots: lambda in the scalar slots, psi_i in float4 slots 7 and 8 of body i.
template <int NB, bool PL, int PB>
__device__ __forceinline__ void lc_vjp(const LcParams& P, const LcWs& w, long k, int ld, const float* Mi,
                                       const float* __restrict__ gbar, float* __restrict__ dq,
                                       float* __restrict__ dqd, float* __restrict__ dtau) {
  static_assert(PB >= 9, "the VJP layout holds psi");
  {
    float g[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) g[i] = __ldg(gbar + k * ld + (PL ? P.slot[i] : i));
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      float acc = 0.0f;
#pragma unroll
      for (int kk = 0; kk < NB; ++kk) acc += Mi[lc_tri<NB>(i, kk)] * g[kk];
      w.f1(i) = acc;
    }
  }
  {
    float pp[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 1
    for (int i = 0; i < NB; ++i) {
      float E[9], ps[6];
      lc_load_E<PB>(w, i, E);
      x_mul(E, P.rT[i], pp, ps);                       // zero at the base
      const float lam = w.f1(i);
      const float* a = P.axis[i];
      ps[0] += a[0] * lam; ps[1] += a[1] * lam; ps[2] += a[2] * lam;
      w.f4(PB * i + 7) = make_float4(ps[0], ps[1], ps[2], ps[3]);
      w.f4(PB * i + 8) = make_float4(ps[4], ps[5], 0.0f, 0.0f);
#pragma unroll
      for (int e = 0; e < 6; ++e) pp[e] = ps[e];
    }
  }
  float CA[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, CV[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 1
  for (int i = NB - 1; i >= 0; --i) {
    const float* a = P.axis[i];
    const float4 v0 = w.f4(PB * i + 2), v1 = w.f4(PB * i + 3), b0 = w.f4(PB * i + 4), f0 = w.f4(PB * i + 5),
                 b2 = w.f4(PB * i + 6), p0 = w.f4(PB * i + 7), p1 = w.f4(PB * i + 8);
    const float v[6] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y};
    const float beta[6] = {b0.x, b0.y, b0.z, b0.w, b2.x, b2.y};
    const float F[6] = {f0.x, f0.y, f0.z, f0.w, b2.z, b2.w};
    const float psi[6] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y};
    const float qdi = v1.w;
    float g[6], A[6], Vb[6], t1[6], vxp[6], t2[6];
    lc_i_mul(P, i, v, g);                                   // I v
    lc_i_mul(P, i, psi, A);                                 // abar = I psi
    crf_mul(psi, g, t1);                               // psi x* (I v)
    crm_mul(v, psi, vxp);                              // v x psi
    lc_i_mul(P, i, vxp, t2);
#pragma unroll
    for (int e = 0; e < 6; ++e) { A[e] += CA[e]; Vb[e] = -t1[e] - t2[e] + CV[e]; }
    {
      const float sq[3] = {a[0] * qdi, a[1] * qdi, a[2] * qdi};
      float t[6];
      crf_s(sq, false, A, t);                          // (S qd) x* Abar
#pragma unroll
      for (int e = 0; e < 6; ++e) Vb[e] += t[e];
    }
    float vxs[6], pxs[6];
    cross_s(v, a, false, vxs);
    cross_s(psi, a, false, pxs);
    float gqd = dot_s(a, false, Vb), gq = 0.0f;
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      gqd += A[e] * vxs[e];
      gq += Vb[e] * vxs[e] + A[e] * beta[e] + F[e] * pxs[e];
    }
    const long gi = k * ld + (PL ? P.slot[i] : i);
    dq[gi] = -gq;
    dqd[gi] = -gqd;
    dtau[gi] = w.f1(i);
    if (i > 0) {
      float E[9];
      lc_load_E<PB>(w, i, E);
      xt_mul(E, P.rT[i], A, CA);
      xt_mul(E, P.rT[i], Vb, CV);
    }
  }
}

// Whether a chain placed in a larger robot stages its matrix blocks per warp
// (the gradient of FD, M^-1 and the gradient of ID; see lc_flush_rows).
__host__ __device__ constexpr bool lc_stages(bool PL, int MODE) {
  return PL && (MODE == MODE_GRAD || MODE == MODE_GRAD_ID || MODE == MODE_MINV);
}

// RNEA at a given qdd (NULL for zero) and, for MODE_GRAD_ID, the derivative
// columns of Alg. 1 at that qdd without the product with M^-1 (no M^-1 is
// formed): tau (MODE_RNEA) or D = [dID/dq | dID/dqd] (MODE_GRAD_ID) at the
// chain's caller joints. The records are those of the gradient of FD (E, v, qd,
// then X a_parent and f, then beta and phi).
template <int NB, bool PL, int MODE>
__device__ __forceinline__ void lc_id(const LcParams& P, const LcWs& w, long k, int ld, const float* __restrict__ q,
                                      const float* __restrict__ qd, const float* __restrict__ qdd,
                                      float* __restrict__ out, float* __restrict__ stg) {
  constexpr int PB = 7;
  {
    float vp[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, ap[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) ap[e] = P.a0[e];
#pragma unroll 1
    for (int i = 0; i < NB; ++i) {
      const long gi = k * ld + (PL ? P.slot[i] : i);
      float E[9];
      lc_transform(P, i, __ldg(q + gi), E);
      const float qdi = __ldg(qd + gi), qddi = qdd ? __ldg(qdd + gi) : 0.0f;
      const float* a = P.axis[i];
      const float* r = P.rT[i];
      const float sq[3] = {a[0] * qdi, a[1] * qdi, a[2] * qdi};   // S qd
      float v[6], Xa[6], acc[6], g[6], f[6];
      x_mul(E, r, vp, v);                              // v_parent = 0 at the base
      v[0] += sq[0]; v[1] += sq[1]; v[2] += sq[2];
      x_mul(E, r, ap, Xa);                             // a_parent = a_0 at the base
#pragma unroll
      for (int e = 0; e < 6; ++e) acc[e] = Xa[e];
      {
        const float vj[6] = {sq[0], sq[1], sq[2], 0.0f, 0.0f, 0.0f};
        crm_mul_acc(v, vj, acc);                       // a = X a_parent + v x S qd + S qdd
      }
      acc[0] += a[0] * qddi; acc[1] += a[1] * qddi; acc[2] += a[2] * qddi;
      lc_i_mul(P, i, v, g);
      lc_i_mul(P, i, acc, f);
      crf_mul_acc(v, g, f);
      w.f4(PB * i) = make_float4(E[0], E[1], E[2], E[3]);
      w.f4(PB * i + 1) = make_float4(E[4], E[5], E[6], E[7]);
      w.f4(PB * i + 2) = make_float4(v[0], v[1], v[2], v[3]);
      w.f4(PB * i + 3) = make_float4(v[4], v[5], E[8], qdi);
      w.f4(PB * i + 4) = make_float4(Xa[0], Xa[1], Xa[2], Xa[3]);
      w.f4(PB * i + 5) = make_float4(f[0], f[1], f[2], f[3]);
      w.f4(PB * i + 6) = make_float4(Xa[4], Xa[5], f[4], f[5]);
#pragma unroll
      for (int e = 0; e < 6; ++e) { vp[e] = v[e]; ap[e] = acc[e]; }
    }
  }
  // backward: F_i = f_i + X_{i+1}^T F_{i+1}; tau_i = S_i^T F_i, or beta_i =
  // (X_i a_parent) x S_i and phi_i = S_i x* F_i into the records
  float F[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 1
  for (int i = NB - 1; i >= 0; --i) {
    const float4 x0 = w.f4(PB * i + 4), f0 = w.f4(PB * i + 5), x2 = w.f4(PB * i + 6);
    float t[6];
    if (i + 1 < NB) {
      float E[9];
      lc_load_E<PB>(w, i + 1, E);
      xt_mul(E, P.rT[i + 1], F, t);
    } else {
#pragma unroll
      for (int e = 0; e < 6; ++e) t[e] = 0.0f;
    }
    F[0] = f0.x + t[0]; F[1] = f0.y + t[1]; F[2] = f0.z + t[2]; F[3] = f0.w + t[3];
    F[4] = x2.z + t[4]; F[5] = x2.w + t[5];
    const float* a = P.axis[i];
    if constexpr (MODE == MODE_RNEA) {
      out[k * ld + (PL ? P.slot[i] : i)] = dot_s(a, false, F);
    } else {
      const float Xa[6] = {x0.x, x0.y, x0.z, x0.w, x2.x, x2.y};
      float beta[6], ph[6];
      cross_s(Xa, a, false, beta);
      crf_s(a, false, F, ph);
      w.f4(PB * i + 4) = make_float4(beta[0], beta[1], beta[2], beta[3]);
      w.f4(PB * i + 5) = make_float4(ph[0], ph[1], ph[2], ph[3]);
      w.f4(PB * i + 6) = make_float4(beta[4], beta[5], ph[4], ph[5]);
    }
  }
  if constexpr (MODE == MODE_GRAD_ID) {
    constexpr bool kStg = lc_stages(PL, MODE);         // a placed chain stages its block of D
    float* Dk = kStg ? stg : out + k * 2 * ld * ld;
#pragma unroll 1
    for (int c = 0; c < 2 * NB; ++c) lc_column<NB, PL, true, kStg>(P, w, c >> 1, (c & 1) == 0, nullptr, Dk);
  }
}

// The gradient of FD of a chain placed in a larger robot stages its blocks of J
// and M^-1 in shared memory, and the warp writes whole rows of its 32 knot points
// (the blocks and the zeros beside them) with stores of consecutive words: a
// lane's own rows are short pieces of long rows, which as per-lane stores cost
// one L2 sector each and, into lines already evicted, a read of the rest.
// (M^-1 and the gradient of ID alone stage their one block the same way.)
// Staged floats per lane: J's (or D's) n x 2n block, then M^-1's n x n block at
// lc_stage_moff, made odd so that the lanes' blocks start in different banks.
template <int NB, int MODE>
__host__ __device__ constexpr int lc_stage_moff() { return MODE == MODE_MINV ? 0 : 2 * NB * NB; }
template <int NB, int MODE>
__host__ __device__ constexpr int lc_stage_floats() {
  return (lc_stage_moff<NB, MODE>() + (MODE == MODE_GRAD_ID ? 0 : NB * NB)) | 1;
}
template <int NB, bool PL, int MODE>
__host__ __device__ constexpr int lc_warp_bytes() {
  return LcLayout<NB, MODE == MODE_VJP ? 9 : 7>::kWarpBytes +
         (lc_stages(PL, MODE) ? 32 * 4 * lc_stage_floats<NB, MODE>() : 0);
}

// Whole rows of J (and of M^-1) of the warp's knot points kb .. kb + nk - 1 from
// the staged blocks: entry c of a row is the staged value where column c belongs
// to the chain, else zero. Lane l writes entries l and l + 32 of every row, so
// that each store of the warp covers consecutive words of one row; src0 / src1
// are the staged columns of entries l and l + 32 of a row of J and srcm that of
// entry l of a row of M^-1 (-1: a zero).
template <int NB, int MODE>
__device__ __forceinline__ void lc_flush_rows(const LcParams& P, const float* stg_warp, int lane, long kb, int nk,
                                              int src0, int src1, int srcm, float* __restrict__ J,
                                              float* __restrict__ Minv) {
  constexpr int SP = lc_stage_floats<NB, MODE>(), MO = lc_stage_moff<NB, MODE>();
  const int ld = P.ld, L = 2 * ld;
#pragma unroll 1
  for (int t = 0; t < nk; ++t) {
    const float* st = stg_warp + t * SP;
    if (J) {
      float* Jt = J + (kb + t) * (long)L * ld;
#pragma unroll
      for (int rr = 0; rr < NB; ++rr) {
        float* row = Jt + P.slot[rr] * L;
        if (lane < L) row[lane] = src0 >= 0 ? st[rr * 2 * NB + src0] : 0.0f;
        if (lane + 32 < L) row[lane + 32] = src1 >= 0 ? st[rr * 2 * NB + src1] : 0.0f;
      }
    }
    if (Minv && lane < ld) {
      float* Mt = Minv + (kb + t) * (long)ld * ld;
#pragma unroll
      for (int rr = 0; rr < NB; ++rr) Mt[P.slot[rr] * ld + lane] = srcm >= 0 ? st[MO + rr * NB + srcm] : 0.0f;
    }
  }
}

// The phases for one knot point. MODE_GRAD: x3 = tau, out = J, out2 = qdd (or
// NULL), out3 = M^-1 (or NULL). MODE_FD: x3 = tau, out = qdd. MODE_VJP: x3 = tau,
// x4 = gbar = dL/dqdd, out = dL/dq, out2 = dL/dqd, out3 = dL/dtau. MODE_MINV:
// out = M^-1. MODE_RNEA: x3 = qdd (or NULL), out = tau. MODE_GRAD_ID: x3 = qdd
// (or NULL), out = [dID/dq | dID/dqd]. For the gradient of FD of a placed chain
// (lc_stages) the chain's blocks of J and M^-1 go to the lane's staging block stg
// (J's n x 2n block, then M^-1's n x n block, row-major), which the warp then
// writes out as whole rows (lc_flush_rows).
template <int NB, bool PL, int MODE>
__device__ __forceinline__ void lc_knot(const LcParams& P, const LcWs& w, long k, const float* __restrict__ q,
                                        const float* __restrict__ qd, const float* __restrict__ x3,
                                        const float* __restrict__ x4, float* __restrict__ out,
                                        float* __restrict__ out2, float* __restrict__ out3, float* __restrict__ stg) {
  constexpr int PB = LcLayout<NB, MODE == MODE_VJP ? 9 : 7>::kPB;
  constexpr bool kStg = lc_stages(PL, MODE);
  const float* tau = x3;
  float* J = MODE == MODE_GRAD ? out : nullptr;
  float* qdd_out = MODE == MODE_GRAD ? out2 : (MODE == MODE_FD ? out : nullptr);
  float* minv_out = MODE == MODE_GRAD ? out3 : (MODE == MODE_MINV ? out : nullptr);
  // ---- a2 + a4: transforms and the backward sweep of the direct M^-1
  //   I^A_i = I_i + X_{i+1}^T (I^A_{i+1} - U_{i+1} D_{i+1}^-1 U_{i+1}^T) X_{i+1}
  //   U_i = I^A_i S_i, D_i = S_i^T U_i, Minv[i][i] = D_i^-1,
  //   Minv[i][k] = -D_i^-1 S_i^T F_k (k > i),  F_k <- X_i^T (F_k + U_i Minv[i][k]) (k >= i)
  // The sweeps are loops over bodies with the F and P columns indexed at
  // compile time, which keeps the code small. A placed chain (PL) reads and
  // writes the caller joints slot[i] of knot points of ld joints.
  const int ld = PL ? P.ld : NB;
  if constexpr (MODE == MODE_RNEA || MODE == MODE_GRAD_ID) {
    lc_id<NB, PL, MODE>(P, w, k, ld, q, qd, x3, out, stg);
    return;
  }
  {
    float Fc[NB][6], carry[6][6];
#pragma unroll
    for (int kk = 0; kk < NB; ++kk)
#pragma unroll
      for (int e = 0; e < 6; ++e) Fc[kk][e] = 0.0f;
#pragma unroll
    for (int u = 0; u < 6; ++u)
#pragma unroll
      for (int s = 0; s < 6; ++s) carry[u][s] = 0.0f;
    // a placed chain loads q_i and qd_i one body ahead, so that the latency of
    // its scattered rows overlaps a body (a whole chain's rows are contiguous, and
    // there the extra registers measured slower: 2.10 against 2.01 ms per step)
    float qn = 0.0f, qdn = 0.0f;
    if constexpr (PL) {
      qn = __ldg(q + k * ld + P.slot[NB - 1]);
      if constexpr (MODE != MODE_MINV) qdn = __ldg(qd + k * ld + P.slot[NB - 1]);
    }
#pragma unroll 1
    for (int i = NB - 1; i >= 0; --i) {
      float E[9];
      float qdi;
      if constexpr (PL) {
        const float qi = qn;
        qdi = qdn;
        if (i > 0) {
          const long gn = k * ld + P.slot[i - 1];
          qn = __ldg(q + gn);
          if constexpr (MODE != MODE_MINV) qdn = __ldg(qd + gn);
        }
        lc_transform(P, i, qi, E);
      } else {
        const long gi = k * ld + i;
        lc_transform(P, i, __ldg(q + gi), E);
        qdi = MODE == MODE_MINV ? 0.0f : __ldg(qd + gi);
      }
      w.f4(PB * i) = make_float4(E[0], E[1], E[2], E[3]);
      w.f4(PB * i + 1) = make_float4(E[4], E[5], E[6], E[7]);
      const float* a = P.axis[i];
      const float* r = P.rT[i];
      const float* in = P.inert[i];
      // I^A_i = I_i + the child's X^T A X (column s of it in carry[s]; zero for the
      // leaf); the structural zeros of I_i add nothing
      float IA[6][6];
#pragma unroll
      for (int u = 0; u < 6; ++u)
#pragma unroll
        for (int s = 0; s < 6; ++s) IA[u][s] = lc_izero(u, s) ? carry[s][u] : i_entry(in, u, s) + carry[s][u];
      float U[6];
#pragma unroll
      for (int u = 0; u < 6; ++u) U[u] = IA[u][0] * a[0] + IA[u][1] * a[1] + IA[u][2] * a[2];
      const float D = a[0] * U[0] + a[1] * U[1] + a[2] * U[2];
      const float Dinv = rcp_pivot(D);
      w.f4(PB * i + 2) = make_float4(U[0], U[1], U[2], U[3]);
      w.f4(PB * i + 3) = make_float4(U[4], U[5], E[8], qdi);
      float row[8];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        if (kk < NB) {
          const float st = a[0] * Fc[kk][0] + a[1] * Fc[kk][1] + a[2] * Fc[kk][2];
          row[kk] = kk == i ? Dinv : (kk > i ? -Dinv * st : 0.0f);
        } else {
          row[kk] = 0.0f;
        }
      }
      w.f4(PB * i + 4) = make_float4(row[0], row[1], row[2], row[3]);
      w.f4(PB * i + 5) = make_float4(row[4], row[5], row[6], row[7]);
      w.f4(PB * i + 6) = make_float4(Dinv, 0.0f, 0.0f, 0.0f);
#pragma unroll
      for (int kk = 0; kk < NB; ++kk) {
        if (kk == i) {
#pragma unroll
          for (int e = 0; e < 6; ++e) Fc[kk][e] = U[e] * Dinv;
        } else if (kk > i) {
#pragma unroll
          for (int e = 0; e < 6; ++e) Fc[kk][e] += U[e] * row[kk];
        }
      }
      if (i > 0) {
#pragma unroll
        for (int kk = 0; kk < NB; ++kk) {
          if (kk >= i) {
            float t[6];
            xt_mul(E, r, Fc[kk], t);
#pragma unroll
            for (int e = 0; e < 6; ++e) Fc[kk][e] = t[e];
          }
        }
        // X^T A X for A = I^A - U D^-1 U^T: B = X^T A column by column, then
        // column s of X^T A X = X^T (row s of B)   (A symmetric)
        float wv[6];
#pragma unroll
        for (int u = 0; u < 6; ++u) wv[u] = U[u] * Dinv;
        float A[6][6];                                  // upper triangle, mirrored
#pragma unroll
        for (int u = 0; u < 6; ++u)
#pragma unroll
          for (int s = u; s < 6; ++s) { A[u][s] = IA[u][s] - wv[u] * U[s]; A[s][u] = A[u][s]; }
        float B[6][6];                                  // B[s] = column s of X^T A
#pragma unroll
        for (int s = 0; s < 6; ++s) xt_mul(E, r, A[s], B[s]);   // (column s of A = row s)
#pragma unroll
        for (int s = 0; s < 6; ++s) {
          float rw[6];
#pragma unroll
          for (int u = 0; u < 6; ++u) rw[u] = B[u][s];
          xt_mul(E, r, rw, carry[s]);                   // column s of X^T A X (symmetric)
        }
      }
    }
  }
  // forward sweep: for k >= i, t = X_i P_{i-1}[k], Minv[i][k] -= D_i^-1 U_i^T t,
  // P_i[k] = S_i Minv[i][k] + t   (P_0[k] = S_0 Minv[0][k])
  {
    float Pc[NB][6];
    {
      const float* a = P.axis[0];
      const float4 m0 = w.f4(4), m1 = w.f4(5);
      const float row[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
      for (int kk = 0; kk < NB; ++kk) {
        Pc[kk][0] = a[0] * row[kk]; Pc[kk][1] = a[1] * row[kk]; Pc[kk][2] = a[2] * row[kk];
        Pc[kk][3] = Pc[kk][4] = Pc[kk][5] = 0.0f;
      }
    }
#pragma unroll 1
    for (int i = 1; i < NB; ++i) {
      const float* a = P.axis[i];
      float E[9];
      lc_load_E<PB>(w, i, E);
      const float4 u0 = w.f4(PB * i + 2), u1 = w.f4(PB * i + 3);
      const float U[6] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y};
      const float Dinv = w.f4(PB * i + 6).x;
      const float4 m0 = w.f4(PB * i + 4), m1 = w.f4(PB * i + 5);
      float row[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
      for (int kk = 0; kk < NB; ++kk) {
        if (kk >= i) {
          float t[6];
          x_mul(E, P.rT[i], Pc[kk], t);
          const float mk = row[kk] - Dinv * dot6(U, t);
          row[kk] = mk;
          Pc[kk][0] = a[0] * mk + t[0]; Pc[kk][1] = a[1] * mk + t[1]; Pc[kk][2] = a[2] * mk + t[2];
          Pc[kk][3] = t[3]; Pc[kk][4] = t[4]; Pc[kk][5] = t[5];
        }
      }
      w.f4(PB * i + 4) = make_float4(row[0], row[1], row[2], row[3]);
      w.f4(PB * i + 5) = make_float4(row[4], row[5], row[6], row[7]);
    }
  }
  // M^-1 (packed upper triangle) into registers, where it stays for FD and the
  // column products
  float Mi[LcLayout<NB>::kMi];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const float4 m0 = w.f4(PB * i + 4), m1 = w.f4(PB * i + 5);
    const float row[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
    for (int kk = i; kk < NB; ++kk) Mi[lc_tri<NB>(i, kk)] = row[kk];
  }
  if (kStg && minv_out) {
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
      for (int kk = 0; kk < NB; ++kk) stg[lc_stage_moff<NB, MODE>() + i * NB + kk] = Mi[lc_tri<NB>(i, kk)];
  } else if (minv_out) {
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      float* row = minv_out + (k * ld + (PL ? P.slot[i] : i)) * ld;
#pragma unroll
      for (int kk = 0; kk < NB; ++kk) row[PL ? P.slot[kk] : kk] = Mi[lc_tri<NB>(i, kk)];
    }
  }
  if constexpr (MODE == MODE_MINV) return;
  // ---- a3: RNEA(q, qd, 0); X_i a_parent in B0 / B2.xy and f_i in B1 / B2.zw
  {
    float vp[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, ap[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) ap[e] = P.a0[e];
#pragma unroll 1
    for (int i = 0; i < NB; ++i) {
      float E[9];
      lc_load_E<PB>(w, i, E);
      const float* a = P.axis[i];
      const float* r = P.rT[i];
      const float qdi = w.f4(PB * i + 3).w;
      const float sq[3] = {a[0] * qdi, a[1] * qdi, a[2] * qdi};   // S qd
      float v[6], Xa[6], acc[6], g[6], f[6];
      x_mul(E, r, vp, v);                              // v_parent = 0 at the base
      v[0] += sq[0]; v[1] += sq[1]; v[2] += sq[2];
      x_mul(E, r, ap, Xa);                             // a_parent = a_0 at the base
#pragma unroll
      for (int e = 0; e < 6; ++e) acc[e] = Xa[e];
      {
        const float vj[6] = {sq[0], sq[1], sq[2], 0.0f, 0.0f, 0.0f};
        crm_mul_acc(v, vj, acc);                       // a = X a_parent + v x S qd
      }
      lc_i_mul(P, i, v, g);
      lc_i_mul(P, i, acc, f);
      crf_mul_acc(v, g, f);
      w.f4(PB * i + 2) = make_float4(v[0], v[1], v[2], v[3]);
      w.f4(PB * i + 3) = make_float4(v[4], v[5], E[8], qdi);
      w.f4(PB * i + 4) = make_float4(Xa[0], Xa[1], Xa[2], Xa[3]);
      w.f4(PB * i + 5) = make_float4(f[0], f[1], f[2], f[3]);
      w.f4(PB * i + 6) = make_float4(Xa[4], Xa[5], f[4], f[5]);
#pragma unroll
      for (int e = 0; e < 6; ++e) { vp[e] = v[e]; ap[e] = acc[e]; }
    }
    // backward: F_i = f_i + X_{i+1}^T F_{i+1}, c_i = S_i^T F_i (scalar slot i)
    float F[6];
    {
      const float4 f0 = w.f4(PB * (NB - 1) + 5), f2 = w.f4(PB * (NB - 1) + 6);
      F[0] = f0.x; F[1] = f0.y; F[2] = f0.z; F[3] = f0.w; F[4] = f2.z; F[5] = f2.w;
      w.f1(NB - 1) = dot_s(P.axis[NB - 1], false, F);
    }
#pragma unroll 1
    for (int i = NB - 2; i >= 0; --i) {
      float E[9], t[6];
      lc_load_E<PB>(w, i + 1, E);
      xt_mul(E, P.rT[i + 1], F, t);
      const float4 f0 = w.f4(PB * i + 5), f2 = w.f4(PB * i + 6);
      F[0] = f0.x + t[0]; F[1] = f0.y + t[1]; F[2] = f0.z + t[2]; F[3] = f0.w + t[3];
      F[4] = f2.z + t[4]; F[5] = f2.w + t[5];
      w.f1(i) = dot_s(P.axis[i], false, F);
    }
  }
  // ---- a5: qdd = M^-1 (tau - c) (scalar slot i then holds qdd_i)
  {
    float rhs[NB], qdd[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) rhs[i] = __ldg(tau + k * ld + (PL ? P.slot[i] : i)) - w.f1(i);
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      float acc = 0.0f;
#pragma unroll
      for (int kk = 0; kk < NB; ++kk) acc += Mi[lc_tri<NB>(i, kk)] * rhs[kk];
      qdd[i] = acc;
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) w.f1(i) = qdd[i];
    if (qdd_out) {
#pragma unroll
      for (int i = 0; i < NB; ++i) qdd_out[k * ld + (PL ? P.slot[i] : i)] = qdd[i];
    }
  }
  if constexpr (MODE == MODE_FD) return;
  // ---- a6: RNEA at qdd: da_i = X_i da_{i-1} + S_i qdd_i, f_i += I_i da_i;
  // beta_i = (X_i a_parent) x S_i at qdd; accumulated forces F_i, phi_i = S_i x* F_i
  {
    float dap[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 1
    for (int i = 0; i < NB; ++i) {
      const float* a = P.axis[i];
      float E[9], da[6], Xa[6], f[6];
      lc_load_E<PB>(w, i, E);
      const float4 x0 = w.f4(PB * i + 4), f0 = w.f4(PB * i + 5), x2 = w.f4(PB * i + 6);
      Xa[0] = x0.x; Xa[1] = x0.y; Xa[2] = x0.z; Xa[3] = x0.w; Xa[4] = x2.x; Xa[5] = x2.y;
      f[0] = f0.x; f[1] = f0.y; f[2] = f0.z; f[3] = f0.w; f[4] = x2.z; f[5] = x2.w;
      x_mul(E, P.rT[i], dap, da);                      // zero at the base
#pragma unroll
      for (int e = 0; e < 6; ++e) Xa[e] += da[e];
      const float qddi = w.f1(i);
      da[0] += a[0] * qddi; da[1] += a[1] * qddi; da[2] += a[2] * qddi;
      lc_i_mul_acc(P, i, da, f);
      float beta[6];
      cross_s(Xa, a, false, beta);
      w.f4(PB * i + 4) = make_float4(beta[0], beta[1], beta[2], beta[3]);
      w.f4(PB * i + 5) = make_float4(f[0], f[1], f[2], f[3]);
      w.f4(PB * i + 6) = make_float4(beta[4], beta[5], f[4], f[5]);
#pragma unroll
      for (int e = 0; e < 6; ++e) dap[e] = da[e];
    }
    float F[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 1
    for (int i = NB - 1; i >= 0; --i) {
      const float4 f0 = w.f4(PB * i + 5), b2 = w.f4(PB * i + 6);
      float t[6];
      if (i + 1 < NB) {
        float E[9];
        lc_load_E<PB>(w, i + 1, E);
        xt_mul(E, P.rT[i + 1], F, t);
      } else {
#pragma unroll
        for (int e = 0; e < 6; ++e) t[e] = 0.0f;
      }
      F[0] = f0.x + t[0]; F[1] = f0.y + t[1]; F[2] = f0.z + t[2]; F[3] = f0.w + t[3];
      F[4] = b2.z + t[4]; F[5] = b2.w + t[5];
      if constexpr (MODE == MODE_VJP) {                // the VJP reads F_i itself
        w.f4(PB * i + 5) = make_float4(F[0], F[1], F[2], F[3]);
        w.f4(PB * i + 6) = make_float4(b2.x, b2.y, F[4], F[5]);
      } else {
        float ph[6];
        crf_s(P.axis[i], false, F, ph);
        w.f4(PB * i + 5) = make_float4(ph[0], ph[1], ph[2], ph[3]);
        w.f4(PB * i + 6) = make_float4(b2.x, b2.y, ph[4], ph[5]);
      }
    }
  }
  if constexpr (MODE == MODE_VJP) {
    lc_vjp<NB, PL, PB>(P, w, k, ld, Mi, x4, out, out2, out3);
    return;
  }
  // ---- a7 - a9: derivative columns and J = -M^-1 dc
  float* Jk = kStg ? stg : J + k * 2 * ld * ld;
#pragma unroll 1
  for (int c = 0; c < 2 * NB; ++c) lc_column<NB, PL, false, kStg>(P, w, c >> 1, (c & 1) == 0, Mi, Jk);
}

template <int NB, bool PL, int MODE>
__global__ void __launch_bounds__(256, 1) grid_lane_chain_kernel(const __grid_constant__ LcParams P, int N,
                                                                 const float* __restrict__ q,
                                                                 const float* __restrict__ qd,
                                                                 const float* __restrict__ x3,
                                                                 const float* __restrict__ x4, float* __restrict__ out,
                                                                 float* __restrict__ out2, float* __restrict__ out3) {
  extern __shared__ __align__(16) unsigned char lc_smem[];
  using Lay = LcLayout<NB, MODE == MODE_VJP ? 9 : 7>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* base = lc_smem + (size_t)warp * lc_warp_bytes<NB, PL, MODE>();
  LcWs w;
  w.s4 = reinterpret_cast<float4*>(base) + lane;
  w.s1 = reinterpret_cast<float*>(base + 32 * 16 * Lay::kS4) + lane;
  const long stride = (long)gridDim.x * blockDim.x;
  if constexpr (lc_stages(PL, MODE)) {
    // the warp's knot points kb .. kb + 31 together: each lane stages its blocks,
    // then the warp writes their rows (kb is the same for every lane of a warp)
    constexpr int SP = lc_stage_floats<NB, MODE>();
    float* stg_warp = reinterpret_cast<float*>(base + Lay::kWarpBytes);
    float* jrows = MODE == MODE_MINV ? nullptr : out;
    float* mrows = MODE == MODE_MINV ? out : (MODE == MODE_GRAD ? out3 : nullptr);
    const int ld = P.ld;
    int src0 = -1, src1 = -1, srcm = -1;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int sl = P.slot[i];
      if (lane == sl) { src0 = i; srcm = i; }        // q columns (and M^-1 columns) of the chain
      if (lane == ld + sl) src0 = NB + i;            // its qd columns, among entries 0 .. 31
      if (lane + 32 == ld + sl) src1 = NB + i;       // ... or among entries 32 .. 63
    }
    for (long kb = (long)blockIdx.x * blockDim.x + warp * 32; kb < N; kb += stride) {
      const long k = kb + lane;
      if (k < N) lc_knot<NB, PL, MODE>(P, w, k, q, qd, x3, x4, out, out2, out3, stg_warp + lane * SP);
      __syncwarp();
      lc_flush_rows<NB, MODE>(P, stg_warp, lane, kb, (int)(N - kb < 32 ? N - kb : 32), src0, src1, srcm, jrows,
                              mrows);
      __syncwarp();
    }
  } else {
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += stride)
      lc_knot<NB, PL, MODE>(P, w, k, q, qd, x3, x4, out, out2, out3, nullptr);
  }
}

struct LcDev {
  int nsm = 0, smem_optin = 0;
};

inline LcDev lc_dev(int dev) {
  static LcDev cache[64];
  static std::atomic<int> ready[64];
  if (dev < 0 || dev >= 64) return LcDev{};
  if (!ready[dev].load()) {
    LcDev d;
    cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cache[dev] = d;
    ready[dev].store(1);
  }
  return cache[dev];
}

template <int NB, bool PL, int MODE>
grid_status lc_launch(const grid_model* m, const LcParams& P, int N, const float* q, const float* qd,
                      const float* x3, const float* x4, float* out, float* out2, float* out3, cudaStream_t st) {
  auto kern = grid_lane_chain_kernel<NB, PL, MODE>;
  const int wb = lc_warp_bytes<NB, PL, MODE>();
  const LcDev di = lc_dev(m->device);
  static std::atomic<int> opted{0};
  if (!opted.load()) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, di.smem_optin);
    if (e != cudaSuccess) {
      grid_set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(e));
      return GRID_E_CUDA;
    }
    opted.store(1);
  }
  // warps per CTA: the count that keeps the most warps resident per SM
  static std::atomic<int> cached{0};
  int c0 = cached.load();
  int warps = c0 >> 8, per_sm = c0 & 0xff;
  if (!c0) {
    int best = 0;
    for (int wc = 8; wc >= 1; --wc) {
      if (wc * wb > di.smem_optin) continue;
      int b = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 32 * wc, (size_t)wc * wb);
      if (b * wc > best) { best = b * wc; warps = wc; per_sm = b; }
    }
    if (!warps) {
      grid_set_error("lane chain kernel: %d B of shared memory per warp do not fit", wb);
      return GRID_E_ARG;
    }
    cached.store((warps << 8) | per_sm);
  }
  if (m->ctas_opt > 0 && m->ctas_opt < per_sm) per_sm = m->ctas_opt;
  const int threads = 32 * warps;
  const long ctas = ((long)N + threads - 1) / threads;
  const int grid = (int)std::min<long>(ctas, (long)di.nsm * per_sm);
  kern<<<grid, threads, (size_t)warps * wb, st>>>(P, N, q, qd, x3, x4, out, out2, out3);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    grid_set_error("kernel launch: %s", cudaGetErrorString(e));
    return GRID_E_CUDA;
  }
  return GRID_OK;
}

template <bool PL, int MODE>
grid_status lc_dispatch(const grid_model* m, int n, const LcParams& P, int N, const float* q, const float* qd,
                        const float* x3, const float* x4, float* out, float* out2, float* out3, cudaStream_t st) {
  switch (n) {
    case 2: return lc_launch<2, PL, MODE>(m, P, N, q, qd, x3, x4, out, out2, out3, st);
    case 3: return lc_launch<3, PL, MODE>(m, P, N, q, qd, x3, x4, out, out2, out3, st);
    case 4: return lc_launch<4, PL, MODE>(m, P, N, q, qd, x3, x4, out, out2, out3, st);
    case 5: return lc_launch<5, PL, MODE>(m, P, N, q, qd, x3, x4, out, out2, out3, st);
    case 6: return lc_launch<6, PL, MODE>(m, P, N, q, qd, x3, x4, out, out2, out3, st);
    case 7: return lc_launch<7, PL, MODE>(m, P, N, q, qd, x3, x4, out, out2, out3, st);
    default: return lc_launch<8, PL, MODE>(m, P, N, q, qd, x3, x4, out, out2, out3, st);
  }
}

// The robot's constants and placement as kernel parameters, then the launch.
// With slot non-NULL the chain is one component of a robot of ld joints per knot
// point (ld <= 32) whose body i is caller joint slot[i]; the call writes only the
// chain's entries of the outputs: its joints' entries of the vectors and its whole
// rows of the matrices (its blocks and the zeros beside them).
template <int MODE>
grid_status lc_run(const grid_model* m, const ModelDev<float>* hm, int ld, const int* slot, int N, const float* q,
                   const float* qd, const float* x3, const float* x4, float* out, float* out2, float* out3,
                   cudaStream_t st) {
  const int n = hm->n;
  if (n < 2 || n > kLcMaxB || hm->any_prism || (slot && (ld < n || ld > 32)) || (!slot && ld != n)) {
    grid_set_error("lane chain kernel: %d bodies in knot points of %d joints", n, ld);
    return GRID_E_TOPOLOGY;
  }
  LcParams P{};
  P.ld = ld;
  for (int i = 0; i < n; ++i) {
    if (hm->parent[i] != i - 1 || hm->perm[i] != i) {
      grid_set_error("lane chain kernel: not a serial chain in caller order");
      return GRID_E_TOPOLOGY;
    }
    for (int e = 0; e < 3; ++e) { P.axis[i][e] = hm->axis[i][e]; P.rT[i][e] = hm->rT[i][e]; }
    for (int e = 0; e < 9; ++e) P.ET[i][e] = hm->ET[i][e];
    for (int e = 0; e < 10; ++e) P.inert[i][e] = hm->inert[i][e];
    {
      const float* in = P.inert[i];   // m, h0, h1, h2, Ixx, Iyy, Izz, Ixy, Ixz, Iyz
      const float2 ip[9] = {{in[4], in[0]}, {in[7], in[3]}, {in[8], -in[2]}, {in[5], in[0]}, {in[7], -in[3]},
                            {in[9], in[1]}, {in[6], in[0]}, {in[8], in[2]}, {in[9], -in[1]}};
      for (int e = 0; e < 9; ++e) P.ip[i][e] = ip[e];
    }
    if (hm->et_ident[i]) P.et_ident |= 1u << i;
    P.slot[i] = slot ? slot[i] : i;
    if (P.slot[i] < 0 || P.slot[i] >= ld || ((P.mask >> P.slot[i]) & 1u)) {
      grid_set_error("lane chain kernel: bad joint placement");
      return GRID_E_TOPOLOGY;
    }
    P.mask |= 1u << P.slot[i];
  }
  for (int e = 0; e < 6; ++e) P.a0[e] = hm->a0[e];
  return slot ? lc_dispatch<true, MODE>(m, n, P, N, q, qd, x3, x4, out, out2, out3, st)
              : lc_dispatch<false, MODE>(m, n, P, N, q, qd, x3, x4, out, out2, out3, st);
}

}  // namespace
