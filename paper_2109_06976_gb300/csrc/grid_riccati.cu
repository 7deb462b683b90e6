// iLQR backward pass (grid_riccati), compiled for each state size n <= 16 so
// that the small dense products unroll; used by grid_traj.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>

#include "grid_launch.cuh"

// Lane-strided loop over [0, COUNT); COUNT is a compile-time constant here, so
// the divisions and bounds in the body fold.
#define GRID_LANES(VAR, COUNT) for (int VAR = lane; VAR < (COUNT); VAR += 32)

namespace {

// ---------------------------------------------------------------- iLQR backward pass
// One warp per trajectory; m = 2n state components, n controls. Matrices live
// in the warp's shared-memory slice, row-major; lanes run over entries.
struct RicLayout {
  int Vxx, Vn, A, VA, Qxx, Bm, VB, Quu, Lc, Qux, Kk, QK, Vx, Qx, Qu, kk, Qk, lx, lu, stride;
};

GRID_HD constexpr RicLayout ric_layout(int n, int ssize) {
  RicLayout R{};
  const int m = 2 * n;
  int o = 0;
  R.Vxx = grid_take(o, m * m); R.Vn = grid_take(o, m * m); R.A = grid_take(o, m * m);
  R.VA = grid_take(o, m * m); R.Qxx = grid_take(o, m * m);
  R.Bm = grid_take(o, m * n); R.VB = grid_take(o, m * n); R.Quu = grid_take(o, n * n);
  R.Lc = grid_take(o, n * n); R.Qux = grid_take(o, n * m); R.Kk = grid_take(o, n * m);
  R.QK = grid_take(o, n * m);
  R.Vx = grid_take(o, m); R.Qx = grid_take(o, m); R.Qu = grid_take(o, n); R.kk = grid_take(o, n);
  R.Qk = grid_take(o, n); R.lx = grid_take(o, m); R.lu = grid_take(o, n);
  R.stride = o + (32 / ssize);
  return R;
}

template <class S, int NN>
__global__ void __launch_bounds__(128) riccati_kernel(
    int B, int H, S dt, const S* __restrict__ Q, const S* __restrict__ QD, const S* __restrict__ U,
    const S* __restrict__ J, const S* __restrict__ Minv, const S* __restrict__ Qr, const S* __restrict__ QDr,
    const S* __restrict__ wq, const S* __restrict__ wr, const S* __restrict__ wf, S mu, S* __restrict__ Ko,
    S* __restrict__ kffo, S* __restrict__ dV) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int n = NN, m = 2 * NN;
  constexpr RicLayout R = ric_layout(NN, (int)sizeof(S));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  S* Wb = reinterpret_cast<S*>(smem) + warp * R.stride;
  S* Vxx = Wb + R.Vxx; S* Vn = Wb + R.Vn; S* A = Wb + R.A; S* VA = Wb + R.VA; S* Qxx = Wb + R.Qxx;
  S* Bm = Wb + R.Bm; S* VB = Wb + R.VB; S* Quu = Wb + R.Quu; S* Lc = Wb + R.Lc; S* Qux = Wb + R.Qux;
  S* Kk = Wb + R.Kk; S* QK = Wb + R.QK; S* Vx = Wb + R.Vx; S* Qx = Wb + R.Qx; S* Qu = Wb + R.Qu;
  S* kk = Wb + R.kk; S* Qk = Wb + R.Qk; S* lx = Wb + R.lx; S* lu = Wb + R.lu;
  const size_t knots = (size_t)H + 1;
  for (int b = blockIdx.x * wpb + warp; b < B; b += gridDim.x * wpb) {
    const size_t kH = (size_t)b * knots + H;
    // terminal cost: V_x = W_f (x_H - r_H), V_xx = W_f
    GRID_LANES(e, m * m) Vxx[e] = (e / m == e % m) ? wf[e % m] : S(0);
    GRID_LANES(i, m) {
      const S x = i < n ? Q[kH * n + i] : QD[kH * n + i - n];
      const S r = i < n ? Qr[kH * n + i] : QDr[kH * n + i - n];
      Vx[i] = wf[i] * (x - r);
    }
    S dv0 = S(0), dv1 = S(0);
    bool pd = true;
    __syncwarp();
    for (int k = H - 1; k >= 0; --k) {
      const size_t kb = (size_t)b * knots + k;
      // step Jacobians: rows n..2n-1 (qd'), then rows 0..n-1 (q' = q + dt qd')
      const S* Jk = J + kb * n * m;
      const S* Mk = Minv + kb * n * n;
      GRID_LANES(e, n * m) {
        const int i = e / m, j = e % m;
        A[(n + i) * m + j] = dt * Jk[i * m + j] + ((j == n + i) ? S(1) : S(0));
      }
      GRID_LANES(e, n * n) {
        const int i = e / n, j = e % n;
        Bm[(n + i) * n + j] = dt * Mk[i * n + j];
      }
      GRID_LANES(i, m) {
        const S x = i < n ? Q[kb * n + i] : QD[kb * n + i - n];
        const S r = i < n ? Qr[kb * n + i] : QDr[kb * n + i - n];
        lx[i] = wq[i] * (x - r);
      }
      GRID_LANES(i, n) lu[i] = wr[i] * U[kb * n + i];
      __syncwarp();
      GRID_LANES(e, n * m) {
        const int i = e / m, j = e % m;
        A[i * m + j] = ((j == i) ? S(1) : S(0)) + dt * A[(n + i) * m + j];
      }
      GRID_LANES(e, n * n) Bm[e] = dt * Bm[n * n + e];
      __syncwarp();
      // V_xx A and V_xx B
      GRID_LANES(e, m * m) {
        const int r = e / m, cc = e % m;
        S s = S(0);
        _Pragma("unroll 4") for (int t = 0; t < m; ++t) s += Vxx[r * m + t] * A[t * m + cc];
        VA[e] = s;
      }
      GRID_LANES(e, m * n) {
        const int r = e / n, cc = e % n;
        S s = S(0);
        _Pragma("unroll 4") for (int t = 0; t < m; ++t) s += Vxx[r * m + t] * Bm[t * n + cc];
        VB[e] = s;
      }
      __syncwarp();
      // Q terms
      GRID_LANES(e, m * m) {
        const int r = e / m, cc = e % m;
        S s = (r == cc) ? wq[r] : S(0);
        _Pragma("unroll 4") for (int t = 0; t < m; ++t) s += A[t * m + r] * VA[t * m + cc];
        Qxx[e] = s;
      }
      GRID_LANES(e, n * n) {
        const int r = e / n, cc = e % n;
        S s = (r == cc) ? wr[r] + mu : S(0);
        _Pragma("unroll 4") for (int t = 0; t < m; ++t) s += Bm[t * n + r] * VB[t * n + cc];
        Quu[e] = s;
      }
      GRID_LANES(e, n * m) {
        const int r = e / m, cc = e % m;
        S s = S(0);
        _Pragma("unroll 4") for (int t = 0; t < m; ++t) s += Bm[t * n + r] * VA[t * m + cc];
        Qux[e] = s;
      }
      GRID_LANES(i, m) {
        S s = lx[i];
        _Pragma("unroll 4") for (int t = 0; t < m; ++t) s += A[t * m + i] * Vx[t];
        Qx[i] = s;
      }
      GRID_LANES(i, n) {
        S s = lu[i];
        _Pragma("unroll 4") for (int t = 0; t < m; ++t) s += Bm[t * n + i] * Vx[t];
        Qu[i] = s;
      }
      __syncwarp();
      // Cholesky Q_uu = L L^T (one lane; n <= 16)
      if (lane == 0) {
        for (int j = 0; j < n; ++j) {
          S d = Quu[j * n + j];
          for (int t = 0; t < j; ++t) d -= Lc[j * n + t] * Lc[j * n + t];
          if (!(d > S(0))) { pd = false; d = S(1); }
          const S ljj = sqrt(d);
          Lc[j * n + j] = ljj;
          for (int i = j + 1; i < n; ++i) {
            S s = Quu[i * n + j];
            for (int t = 0; t < j; ++t) s -= Lc[i * n + t] * Lc[j * n + t];
            Lc[i * n + j] = s / ljj;
          }
        }
      }
      __syncwarp();
      // K = -Q_uu^-1 Q_ux (columns 0..m-1), k = -Q_uu^-1 Q_u (column m): one lane per column
      GRID_LANES(cc, m + 1) {
        S y[NN];
        for (int i = 0; i < n; ++i) {
          S s = cc < m ? Qux[i * m + cc] : Qu[i];
          for (int t = 0; t < i; ++t) s -= Lc[i * n + t] * y[t];
          y[i] = s / Lc[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
          S s = y[i];
          for (int t = i + 1; t < n; ++t) s -= Lc[t * n + i] * y[t];
          y[i] = s / Lc[i * n + i];
        }
        for (int i = 0; i < n; ++i) {
          if (cc < m) Kk[i * m + cc] = -y[i];
          else kk[i] = -y[i];
        }
      }
      __syncwarp();
      // Q_uu K and Q_uu k
      GRID_LANES(e, n * m) {
        const int r = e / m, cc = e % m;
        S s = S(0);
        _Pragma("unroll 4") for (int t = 0; t < n; ++t) s += Quu[r * n + t] * Kk[t * m + cc];
        QK[e] = s;
      }
      GRID_LANES(i, n) {
        S s = S(0);
        _Pragma("unroll 4") for (int t = 0; t < n; ++t) s += Quu[i * n + t] * kk[t];
        Qk[i] = s;
      }
      __syncwarp();
      // V_x = Q_x + K^T Q_uu k + K^T Q_u + Q_ux^T k
      GRID_LANES(i, m) {
        S s = Qx[i];
        _Pragma("unroll 4") for (int t = 0; t < n; ++t) s += Kk[t * m + i] * Qk[t] + Kk[t * m + i] * Qu[t] + Qux[t * m + i] * kk[t];
        Vx[i] = s;
      }
      // V_xx = Q_xx + K^T Q_uu K + K^T Q_ux + Q_ux^T K
      GRID_LANES(e, m * m) {
        const int r = e / m, cc = e % m;
        S s = Qxx[e];
        _Pragma("unroll 4") for (int t = 0; t < n; ++t)
          s += Kk[t * m + r] * QK[t * m + cc] + Kk[t * m + r] * Qux[t * m + cc] + Qux[t * m + r] * Kk[t * m + cc];
        Vn[e] = s;
      }
      if (lane == 0) {
        S a = S(0), q2 = S(0);
        _Pragma("unroll 4") for (int t = 0; t < n; ++t) { a += kk[t] * Qu[t]; q2 += kk[t] * Qk[t]; }
        dv0 += a;
        dv1 += S(0.5) * q2;
      }
      GRID_LANES(e, n * m) Ko[kb * n * m + e] = Kk[e];
      GRID_LANES(i, n) kffo[kb * n + i] = kk[i];
      __syncwarp();
      GRID_LANES(e, m * m) {
        const int r = e / m, cc = e % m;
        Vxx[e] = S(0.5) * (Vn[r * m + cc] + Vn[cc * m + r]);
      }
      __syncwarp();
    }
    if (lane == 0) {
      const bool all_pd = pd;
      dV[2 * (size_t)b] = all_pd ? dv0 : S(NAN);
      dV[2 * (size_t)b + 1] = all_pd ? dv1 : S(NAN);
    }
    GRID_LANES(e, n * m) Ko[((size_t)b * knots + H) * n * m + e] = S(0);
    GRID_LANES(i, n) kffo[((size_t)b * knots + H) * n + i] = S(0);
    __syncwarp();
  }
}


// The same backward pass for n <= 8 with one matrix column per lane: lanes
// 0 .. m-1 own the state columns c (A[:, c], then V_xx A, Q_xx, Q_ux, K, Q_uu K and
// the new V_xx, all columns c), lanes m .. m+n-1 the control columns (B, V_xx B,
// Q_uu), lane m+n the feed-forward column (Q_u, k). A lane keeps its columns in
// registers and reads the other operand of each product by broadcast from the
// warp's shared memory (every lane reads the same entry), so a product is m
// independent accumulations per lane; every lane factors Q_uu = L L^T itself in
// registers. Same arithmetic, term for term, as riccati_kernel.
template <class S, int NN>
__global__ void __launch_bounds__(128) riccati_col_kernel(
    int B, int H, S dt, const S* __restrict__ Q, const S* __restrict__ QD, const S* __restrict__ U,
    const S* __restrict__ J, const S* __restrict__ Minv, const S* __restrict__ Qr, const S* __restrict__ QDr,
    const S* __restrict__ wq, const S* __restrict__ wr, const S* __restrict__ wf, S mu, S* __restrict__ Ko,
    S* __restrict__ kffo, S* __restrict__ dV) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int n = NN, m = 2 * NN;
  static_assert(m + n + 1 <= 32, "one column per lane");
  constexpr RicLayout R = ric_layout(NN, (int)sizeof(S));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  S* Wb = reinterpret_cast<S*>(smem) + warp * R.stride;
  S* Vxx = Wb + R.Vxx; S* Vn = Wb + R.Vn; S* A = Wb + R.A; S* Bm = Wb + R.Bm; S* Quu = Wb + R.Quu;
  S* Qux = Wb + R.Qux; S* Kk = Wb + R.Kk; S* Vx = Wb + R.Vx; S* Qu = Wb + R.Qu; S* kk = Wb + R.kk;
  S* Qk = Wb + R.Qk; S* lx = Wb + R.lx; S* lu = Wb + R.lu;
  const bool st_lane = lane < m, ct_lane = lane >= m && lane < m + n, ff_lane = lane == m + n;
  const int cb = lane - m;
  const size_t knots = (size_t)H + 1;
  for (int b = blockIdx.x * wpb + warp; b < B; b += gridDim.x * wpb) {
    const size_t kH = (size_t)b * knots + H;
    GRID_LANES(e, m * m) Vxx[e] = (e / m == e % m) ? wf[e % m] : S(0);
    GRID_LANES(i, m) {
      const S x = i < n ? Q[kH * n + i] : QD[kH * n + i - n];
      const S r = i < n ? Qr[kH * n + i] : QDr[kH * n + i - n];
      Vx[i] = wf[i] * (x - r);
    }
    S dv0 = S(0), dv1 = S(0);
    bool pd = true;
    // this lane's entries of the next step's J, M^-1, states and controls, loaded
    // one step ahead so that their latency overlaps the current step
    constexpr int PJ = (n * m + 31) / 32, PM = (n * n + 31) / 32;
    S pj[PJ], pm[PM], px = S(0), pr = S(0), pu = S(0);
    auto fetch = [&](int kf) {
      const size_t kb = (size_t)b * knots + kf;
#pragma unroll
      for (int u = 0; u < PJ; ++u) {
        const int e = lane + 32 * u;
        pj[u] = e < n * m ? J[kb * n * m + e] : S(0);
      }
#pragma unroll
      for (int u = 0; u < PM; ++u) {
        const int e = lane + 32 * u;
        pm[u] = e < n * n ? Minv[kb * n * n + e] : S(0);
      }
      if (lane < m) {
        px = lane < n ? Q[kb * n + lane] : QD[kb * n + lane - n];
        pr = lane < n ? Qr[kb * n + lane] : QDr[kb * n + lane - n];
      }
      if (lane < n) pu = U[kb * n + lane];
    };
    fetch(H - 1);
    __syncwarp();
    for (int k = H - 1; k >= 0; --k) {
      const size_t kb = (size_t)b * knots + k;
#pragma unroll
      for (int u = 0; u < PJ; ++u) {
        const int e = lane + 32 * u;
        if (e < n * m) {
          const int i = e / m, j = e % m;
          A[(n + i) * m + j] = dt * pj[u] + ((j == n + i) ? S(1) : S(0));
        }
      }
#pragma unroll
      for (int u = 0; u < PM; ++u) {
        const int e = lane + 32 * u;
        if (e < n * n) Bm[n * n + e] = dt * pm[u];
      }
      if (lane < m) lx[lane] = wq[lane] * (px - pr);
      if (lane < n) lu[lane] = wr[lane] * pu;
      if (k > 0) fetch(k - 1);
      __syncwarp();
      GRID_LANES(e, n * m) {
        const int i = e / m, j = e % m;
        A[i * m + j] = ((j == i) ? S(1) : S(0)) + dt * A[(n + i) * m + j];
      }
      GRID_LANES(e, n * n) Bm[e] = dt * Bm[n * n + e];
      __syncwarp();
      // this lane's column of A (state lanes) or B (control lanes), and of V_xx times it
      S a[m], col[m];
#pragma unroll
      for (int t = 0; t < m; ++t) a[t] = st_lane ? A[t * m + lane] : (ct_lane ? Bm[t * n + cb] : S(0));
#pragma unroll
      for (int r = 0; r < m; ++r) {
        S s = S(0);
#pragma unroll
        for (int t = 0; t < m; ++t) s += Vxx[r * m + t] * a[t];
        col[r] = s;
      }
      // Q columns: state lanes Q_xx[:, c] and Q_ux[:, c] (= B^T (V_xx A)[:, c]) and
      // Q_x[c]; control lanes Q_uu[:, cb] and Q_u[cb]
      S qcol[m], qux[n];
#pragma unroll
      for (int r = 0; r < m; ++r) {
        S s = (st_lane && r == lane) ? wq[r] : S(0);
#pragma unroll
        for (int t = 0; t < m; ++t) s += A[t * m + r] * col[t];
        qcol[r] = s;
      }
#pragma unroll
      for (int r = 0; r < n; ++r) {
        S s = (ct_lane && r == cb) ? wr[r] + mu : S(0);
#pragma unroll
        for (int t = 0; t < m; ++t) s += Bm[t * n + r] * col[t];
        qux[r] = s;                                     // Q_ux[r][c] (state) or Q_uu[r][cb] (control)
      }
      S qv = S(0);                                      // Q_x[c] (state) or Q_u[cb] (control)
      {
        S s = st_lane ? lx[lane] : (ct_lane ? lu[cb] : S(0));
#pragma unroll
        for (int t = 0; t < m; ++t) s += a[t] * Vx[t];
        qv = s;
      }
      if (st_lane) {
#pragma unroll
        for (int r = 0; r < n; ++r) Qux[r * m + lane] = qux[r];
      }
      if (ct_lane) {
#pragma unroll
        for (int r = 0; r < n; ++r) Quu[r * n + cb] = qux[r];
        Qu[cb] = qv;
      }
      __syncwarp();
      // Q_uu = L L^T in every lane (lower triangle of Q_uu as stored)
      S qu[n * n], L[n * n], linv[n];
#pragma unroll
      for (int e = 0; e < n * n; ++e) qu[e] = Quu[e];
      // (loops of fixed trip count with the triangle as a condition, so that they
      // unroll completely and L stays in registers)
#pragma unroll
      for (int j = 0; j < n; ++j) {
        S d = qu[j * n + j];
#pragma unroll
        for (int t = 0; t < n; ++t)
          if (t < j) d -= L[j * n + t] * L[j * n + t];
        if (!(d > S(0))) { pd = false; d = S(1); }
        const S li = rsqrtf(d);                         // 1 / L_jj (FP32 reciprocal square root)
        const S ljj = d * li;
        L[j * n + j] = ljj;
        linv[j] = li;
#pragma unroll
        for (int i = 0; i < n; ++i) {
          if (i > j) {
            S s = qu[i * n + j];
#pragma unroll
            for (int t = 0; t < n; ++t)
              if (t < j) s -= L[i * n + t] * L[j * n + t];
            L[i * n + j] = s * linv[j];
          }
        }
      }
      // K[:, c] = -Q_uu^-1 Q_ux[:, c] (state lanes), k = -Q_uu^-1 Q_u (feed-forward lane)
      S y[n];
#pragma unroll
      for (int i = 0; i < n; ++i) {
        S s = ff_lane ? Qu[i] : qux[i];
#pragma unroll
        for (int t = 0; t < n; ++t)
          if (t < i) s -= L[i * n + t] * y[t];
        y[i] = s * linv[i];
      }
#pragma unroll
      for (int ii = 0; ii < n; ++ii) {
        const int i = n - 1 - ii;
        S s = y[i];
#pragma unroll
        for (int t = 0; t < n; ++t)
          if (t > i) s -= L[t * n + i] * y[t];
        y[i] = s * linv[i];
      }
      S kc[n], qk[n];
#pragma unroll
      for (int i = 0; i < n; ++i) kc[i] = -y[i];
#pragma unroll
      for (int r = 0; r < n; ++r) {                     // Q_uu K[:, c] or Q_uu k
        S s = S(0);
#pragma unroll
        for (int t = 0; t < n; ++t) s += qu[r * n + t] * kc[t];
        qk[r] = s;
      }
      if (st_lane) {
#pragma unroll
        for (int i = 0; i < n; ++i) { Kk[i * m + lane] = kc[i]; Ko[kb * n * m + i * m + lane] = kc[i]; }
      }
      if (ff_lane) {
#pragma unroll
        for (int i = 0; i < n; ++i) { kk[i] = kc[i]; Qk[i] = qk[i]; kffo[kb * n + i] = kc[i]; }
      }
      __syncwarp();
      if (ff_lane) {
        S a0 = S(0), q2 = S(0);
#pragma unroll
        for (int t = 0; t < n; ++t) { a0 += kk[t] * Qu[t]; q2 += kk[t] * Qk[t]; }
        dv0 += a0;
        dv1 += S(0.5) * q2;
      }
      // V_x = Q_x + K^T Q_uu k + K^T Q_u + Q_ux^T k; V_xx columns before symmetrising
      S vxn = S(0);
      if (st_lane) {
        S s = qv;
#pragma unroll
        for (int t = 0; t < n; ++t) s += kc[t] * Qk[t] + kc[t] * Qu[t] + qux[t] * kk[t];
        vxn = s;
#pragma unroll
        for (int r = 0; r < m; ++r) {
          S v = qcol[r];
#pragma unroll
          for (int t = 0; t < n; ++t) v += Kk[t * m + r] * qk[t] + Kk[t * m + r] * qux[t] + Qux[t * m + r] * kc[t];
          Vn[r * m + lane] = v;
        }
      }
      __syncwarp();
      if (st_lane) {
        Vx[lane] = vxn;
#pragma unroll
        for (int r = 0; r < m; ++r) Vxx[r * m + lane] = S(0.5) * (Vn[r * m + lane] + Vn[lane * m + r]);
      }
      __syncwarp();
    }
    if (ff_lane) {                                      // dv0 and dv1 were summed in this lane
      dV[2 * (size_t)b] = pd ? dv0 : S(NAN);
      dV[2 * (size_t)b + 1] = pd ? dv1 : S(NAN);
    }
    GRID_LANES(e, n * m) Ko[((size_t)b * knots + H) * n * m + e] = S(0);
    GRID_LANES(i, n) kffo[((size_t)b * knots + H) * n + i] = S(0);
    __syncwarp();
  }
}

template <class S, int NN>
grid_status launch_riccati_n(const grid_model* m, int B, int H, S dt, const S* Q, const S* QD, const S* U,
                             const S* J, const S* Minv, const S* Qr, const S* QDr, const S* wq, const S* wr,
                             const S* wf, S mu, S* K, S* kff, S* dV, cudaStream_t st) {
  // FP32 and n <= 8: one matrix column per lane (riccati_col_kernel); otherwise
  // lanes over matrix entries
  auto kern = [] {
    if constexpr (std::is_same<S, float>::value && NN <= 8) return riccati_col_kernel<S, NN>;
    else return riccati_kernel<S, NN>;
  }();
  const DevInfo di = dev_info(m->device);
  static std::atomic<int> opted{0};
  if (!opted.load()) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, di.smem_optin) != cudaSuccess) {
      grid_set_error("cudaFuncSetAttribute failed");
      return GRID_E_CUDA;
    }
    opted.store(1);
  }
  constexpr size_t per_warp = (size_t)ric_layout(NN, (int)sizeof(S)).stride * sizeof(S);
  int warps = 0, per_sm = 0, best = 0;
  for (int w = 4; w >= 1; --w) {
    const size_t sm = w * per_warp;
    if (sm > (size_t)di.smem_optin) continue;
    int blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, 32 * w, sm);
    if (blocks * w > best) { best = blocks * w; warps = w; per_sm = blocks; }
  }
  if (!warps) {
    grid_set_error("Riccati workspace of %zu B exceeds shared memory", per_warp);
    return GRID_E_ARG;
  }
  const int grid = (int)std::min<long>(((long)B + warps - 1) / warps, (long)di.nsm * per_sm);
  kern<<<grid, 32 * warps, warps * per_warp, st>>>(B, H, dt, Q, QD, U, J, Minv, Qr, QDr, wq, wr, wf, mu, K, kff, dV);
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    grid_set_error("Riccati launch: %s", cudaGetErrorString(err));
    return GRID_E_CUDA;
  }
  return GRID_OK;
}

}  // namespace

template <class S>
grid_status launch_riccati(const grid_model* m, int B, int H, S dt, const S* Q, const S* QD, const S* U,
                           const S* J, const S* Minv, const S* Qr, const S* QDr, const S* wq, const S* wr,
                           const S* wf, S mu, S* K, S* kff, S* dV, cudaStream_t st) {
  switch (m->n) {
#define GRID_RIC(NB) \
    case NB: return launch_riccati_n<S, NB>(m, B, H, dt, Q, QD, U, J, Minv, Qr, QDr, wq, wr, wf, mu, K, kff, dV, st);
    GRID_RIC(1) GRID_RIC(2) GRID_RIC(3) GRID_RIC(4) GRID_RIC(5) GRID_RIC(6) GRID_RIC(7) GRID_RIC(8)
    GRID_RIC(9) GRID_RIC(10) GRID_RIC(11) GRID_RIC(12) GRID_RIC(13) GRID_RIC(14) GRID_RIC(15) GRID_RIC(16)
#undef GRID_RIC
    default: break;
  }
  grid_set_error("the Riccati pass supports n <= 16 (n = %d)", m->n);
  return GRID_E_ARG;
}

template grid_status launch_riccati<float>(const grid_model*, int, int, float, const float*, const float*,
                                           const float*, const float*, const float*, const float*, const float*,
                                           const float*, const float*, const float*, float, float*, float*, float*,
                                           cudaStream_t);
template grid_status launch_riccati<double>(const grid_model*, int, int, double, const double*, const double*,
                                            const double*, const double*, const double*, const double*,
                                            const double*, const double*, const double*, const double*, double,
                                            double*, double*, double*, cudaStream_t);
