// Compact spatial algebra for the kernels. Spatial vectors are [angular; linear]
// (the ordering of Eq. (2)). A transform iX_lambda is held as (E, r):
// X = [E 0; -E r~ E], so X m = [E w; E (v - r x w)] and
// X^T f = [E^T n + r x (E^T f); E^T f]. A spatial inertia is held as
// (m, h = m c, Ibar): I m = [Ibar w + h x v; m v - h x w].
//
// In FP32, compiled by nvcc for sm_100 and later, X m, X^T f and the 6-vector dot
// use the paired FP32 instructions (two independent multiply-adds per issue slot):
// X m pairs row i of E w with row i of E (v - r x w), X^T f pairs (E^T n)_i with
// (E^T f)_i, and the dot sums its even and odd products as two chains. Each scalar
// is still one correctly rounded FMA, but in a different order from the scalar
// form. The kernels spend most of their issue slots in these three, so this
// raises throughput. The FP64 forms and the run-time compiled kernels keep the
// scalar forms.
#pragma once

#ifndef GRID_PAIRED_F32
#if defined(__CUDACC__) && !defined(__CUDACC_RTC__)
#define GRID_PAIRED_F32 1
#else
#define GRID_PAIRED_F32 0
#endif
#endif

// 1 / x for an FP32 pivot D_i of the M^-1 recursion (a positive normal number): the
// hardware approximation rcp.approx.ftz.f32, within 1 ulp (PTX ISA). It sits on the serial
// path of the backward sweep, where the correctly rounded form measured 2.4 % slower.
__device__ __forceinline__ float rcp_pivot(float x) {
#if defined(__CUDA_ARCH__)
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
#else
  return 1.0f / x;
#endif
}

template <class S>
__device__ __forceinline__ void cross3(const S* a, const S* b, S* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// o = X m
template <class S>
__device__ __forceinline__ void x_mul(const S* E, const S* r, const S* m, S* o) {
  S t0 = m[3] - r[1] * m[2] + r[2] * m[1];   // v - r x w, two FMAs per row
  S t1 = m[4] - r[2] * m[0] + r[0] * m[2];
  S t2 = m[5] - r[0] * m[1] + r[1] * m[0];
#if GRID_PAIRED_F32
  if constexpr (sizeof(S) == 4) {   // angular and linear rows as pairs
    const float2 p0 = make_float2(m[0], t0), p1 = make_float2(m[1], t1), p2 = make_float2(m[2], t2);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float2 a = __fmul2_rn(make_float2(E[3 * i], E[3 * i]), p0);
      a = __ffma2_rn(make_float2(E[3 * i + 1], E[3 * i + 1]), p1, a);
      a = __ffma2_rn(make_float2(E[3 * i + 2], E[3 * i + 2]), p2, a);
      o[i] = a.x;
      o[3 + i] = a.y;
    }
    return;
  }
#endif
  o[0] = E[0] * m[0] + E[1] * m[1] + E[2] * m[2];
  o[1] = E[3] * m[0] + E[4] * m[1] + E[5] * m[2];
  o[2] = E[6] * m[0] + E[7] * m[1] + E[8] * m[2];
  o[3] = E[0] * t0 + E[1] * t1 + E[2] * t2;
  o[4] = E[3] * t0 + E[4] * t1 + E[5] * t2;
  o[5] = E[6] * t0 + E[7] * t1 + E[8] * t2;
}

// o = X^T f
template <class S>
__device__ __forceinline__ void xt_mul(const S* E, const S* r, const S* f, S* o) {
#if GRID_PAIRED_F32
  if constexpr (sizeof(S) == 4) {   // (E^T n)_i and (E^T f)_i as pairs
    const float2 p0 = make_float2(f[0], f[3]), p1 = make_float2(f[1], f[4]), p2 = make_float2(f[2], f[5]);
    float2 a[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      a[i] = __fmul2_rn(make_float2(E[i], E[i]), p0);
      a[i] = __ffma2_rn(make_float2(E[3 + i], E[3 + i]), p1, a[i]);
      a[i] = __ffma2_rn(make_float2(E[6 + i], E[6 + i]), p2, a[i]);
    }
    o[0] = a[0].x + r[1] * a[2].y - r[2] * a[1].y;
    o[1] = a[1].x + r[2] * a[0].y - r[0] * a[2].y;
    o[2] = a[2].x + r[0] * a[1].y - r[1] * a[0].y;
    o[3] = a[0].y; o[4] = a[1].y; o[5] = a[2].y;
    return;
  }
#endif
  S g0 = E[0] * f[3] + E[3] * f[4] + E[6] * f[5];
  S g1 = E[1] * f[3] + E[4] * f[4] + E[7] * f[5];
  S g2 = E[2] * f[3] + E[5] * f[4] + E[8] * f[5];
  S n0 = E[0] * f[0] + E[3] * f[1] + E[6] * f[2];
  S n1 = E[1] * f[0] + E[4] * f[1] + E[7] * f[2];
  S n2 = E[2] * f[0] + E[5] * f[1] + E[8] * f[2];
  o[0] = n0 + r[1] * g2 - r[2] * g1;
  o[1] = n1 + r[2] * g0 - r[0] * g2;
  o[2] = n2 + r[0] * g1 - r[1] * g0;
  o[3] = g0; o[4] = g1; o[5] = g2;
}

// o = I m with I = (m, h, Ibar); inert = {m, h0, h1, h2, Ixx, Iyy, Izz, Ixy, Ixz, Iyz}
template <class S>
__device__ __forceinline__ void i_mul(const S* in, const S* m, S* o) {
  const S mass = in[0], h0 = in[1], h1 = in[2], h2 = in[3];
  o[0] = in[4] * m[0] + in[7] * m[1] + in[8] * m[2] + h1 * m[5] - h2 * m[4];
  o[1] = in[7] * m[0] + in[5] * m[1] + in[9] * m[2] + h2 * m[3] - h0 * m[5];
  o[2] = in[8] * m[0] + in[9] * m[1] + in[6] * m[2] + h0 * m[4] - h1 * m[3];
  o[3] = mass * m[3] - h1 * m[2] + h2 * m[1];
  o[4] = mass * m[4] - h2 * m[0] + h0 * m[2];
  o[5] = mass * m[5] - h0 * m[1] + h1 * m[0];
}

// o = a x b (motion cross product, Eq. (2))
template <class S>
__device__ __forceinline__ void crm_mul(const S* a, const S* b, S* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
  o[3] = a[1] * b[5] - a[2] * b[4] + a[4] * b[2] - a[5] * b[1];
  o[4] = a[2] * b[3] - a[0] * b[5] + a[5] * b[0] - a[3] * b[2];
  o[5] = a[0] * b[4] - a[1] * b[3] + a[3] * b[1] - a[4] * b[0];
}

// o = a x* f = -(a x)^T f (force cross product, Eq. (2))
template <class S>
__device__ __forceinline__ void crf_mul(const S* a, const S* f, S* o) {
  o[0] = a[1] * f[2] - a[2] * f[1] + a[4] * f[5] - a[5] * f[4];
  o[1] = a[2] * f[0] - a[0] * f[2] + a[5] * f[3] - a[3] * f[5];
  o[2] = a[0] * f[1] - a[1] * f[0] + a[3] * f[4] - a[4] * f[3];
  o[3] = a[1] * f[5] - a[2] * f[4];
  o[4] = a[2] * f[3] - a[0] * f[5];
  o[5] = a[0] * f[4] - a[1] * f[3];
}

// Accumulating forms, o += ...: the first product of every component folds into an
// FMA with the accumulator instead of a separate add.
template <class S>
__device__ __forceinline__ void i_mul_acc(const S* in, const S* m, S* o) {
  const S mass = in[0], h0 = in[1], h1 = in[2], h2 = in[3];
  o[0] = o[0] + in[4] * m[0] + in[7] * m[1] + in[8] * m[2] + h1 * m[5] - h2 * m[4];
  o[1] = o[1] + in[7] * m[0] + in[5] * m[1] + in[9] * m[2] + h2 * m[3] - h0 * m[5];
  o[2] = o[2] + in[8] * m[0] + in[9] * m[1] + in[6] * m[2] + h0 * m[4] - h1 * m[3];
  o[3] = o[3] + mass * m[3] - h1 * m[2] + h2 * m[1];
  o[4] = o[4] + mass * m[4] - h2 * m[0] + h0 * m[2];
  o[5] = o[5] + mass * m[5] - h0 * m[1] + h1 * m[0];
}
template <class S>
__device__ __forceinline__ void crm_mul_acc(const S* a, const S* b, S* o) {
  o[0] = o[0] + a[1] * b[2] - a[2] * b[1];
  o[1] = o[1] + a[2] * b[0] - a[0] * b[2];
  o[2] = o[2] + a[0] * b[1] - a[1] * b[0];
  o[3] = o[3] + a[1] * b[5] - a[2] * b[4] + a[4] * b[2] - a[5] * b[1];
  o[4] = o[4] + a[2] * b[3] - a[0] * b[5] + a[5] * b[0] - a[3] * b[2];
  o[5] = o[5] + a[0] * b[4] - a[1] * b[3] + a[3] * b[1] - a[4] * b[0];
}
template <class S>
__device__ __forceinline__ void crf_mul_acc(const S* a, const S* f, S* o) {
  o[0] = o[0] + a[1] * f[2] - a[2] * f[1] + a[4] * f[5] - a[5] * f[4];
  o[1] = o[1] + a[2] * f[0] - a[0] * f[2] + a[5] * f[3] - a[3] * f[5];
  o[2] = o[2] + a[0] * f[1] - a[1] * f[0] + a[3] * f[4] - a[4] * f[3];
  o[3] = o[3] + a[1] * f[5] - a[2] * f[4];
  o[4] = o[4] + a[2] * f[3] - a[0] * f[5];
  o[5] = o[5] + a[0] * f[4] - a[1] * f[3];
}
template <class S>
__device__ __forceinline__ void cross3_acc(const S* a, const S* b, S* o) {
  o[0] = o[0] + a[1] * b[2] - a[2] * b[1];
  o[1] = o[1] + a[2] * b[0] - a[0] * b[2];
  o[2] = o[2] + a[0] * b[1] - a[1] * b[0];
}

// Component c (0..5) of X m, reading operands from memory.
template <class S>
__device__ __forceinline__ S x_mul_c(const S* E, const S* r, const S* m, int c) {
  if (c < 3) return E[3 * c] * m[0] + E[3 * c + 1] * m[1] + E[3 * c + 2] * m[2];
  const int k = c - 3;
  S t0 = m[3] - r[1] * m[2] + r[2] * m[1];   // v - r x w, two FMAs per row
  S t1 = m[4] - r[2] * m[0] + r[0] * m[2];
  S t2 = m[5] - r[0] * m[1] + r[1] * m[0];
  return E[3 * k] * t0 + E[3 * k + 1] * t1 + E[3 * k + 2] * t2;
}

// a . b for 6-vectors: a balanced sum (dependency depth 4 instead of 7), or in
// FP32 two paired chains of three multiply-adds (depth 4)
template <class S>
__device__ __forceinline__ S dot6(const S* a, const S* b) {
#if GRID_PAIRED_F32
  if constexpr (sizeof(S) == 4) {
    float2 p = __fmul2_rn(make_float2(a[0], a[1]), make_float2(b[0], b[1]));
    p = __ffma2_rn(make_float2(a[2], a[3]), make_float2(b[2], b[3]), p);
    p = __ffma2_rn(make_float2(a[4], a[5]), make_float2(b[4], b[5]), p);
    return p.x + p.y;
  }
#endif
  return (a[0] * b[0] + a[1] * b[1]) + (a[2] * b[2] + a[3] * b[3]) + (a[4] * b[4] + a[5] * b[5]);
}
// 6-vector stored in an 8-scalar record of read-only device memory (not shared)
template <class S>
__device__ __forceinline__ void ldg6(const S* p, S* o) {
#ifdef __CUDACC__
  if constexpr (sizeof(S) == 4) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    const float2 u = __ldg(reinterpret_cast<const float2*>(p + 4));
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w; o[4] = u.x; o[5] = u.y;
  } else {
    for (int e = 0; e < 6; e += 2) {
      const double2 t = __ldg(reinterpret_cast<const double2*>(p + e));
      o[e] = t.x; o[e + 1] = t.y;
    }
  }
#else
  for (int e = 0; e < 6; ++e) o[e] = p[e];
#endif
}

// ---- joint motion subspaces: S = [a; 0] (revolute) or [0; a] (prismatic, pr)
template <class S>
__device__ __forceinline__ void joint_s(const S* a, bool pr, S* s) {
  s[0] = pr ? S(0) : a[0]; s[1] = pr ? S(0) : a[1]; s[2] = pr ? S(0) : a[2];
  s[3] = pr ? a[0] : S(0); s[4] = pr ? a[1] : S(0); s[5] = pr ? a[2] : S(0);
}
// v x S = [w x a; v x a] (revolute) or [0; w x a] (prismatic)
template <class S>
__device__ __forceinline__ void cross_s(const S* v, const S* a, bool pr, S* out) {
  if (pr) {
    out[0] = out[1] = out[2] = S(0);
    cross3(v, a, out + 3);
  } else {
    cross3(v, a, out);
    cross3(v + 3, a, out + 3);
  }
}
// o += v x S
template <class S>
__device__ __forceinline__ void cross_s_acc(const S* v, const S* a, bool pr, S* o) {
  if (pr) {
    cross3_acc(v, a, o + 3);
  } else {
    cross3_acc(v, a, o);
    cross3_acc(v + 3, a, o + 3);
  }
}
// S x* f = [a x n; a x f] (revolute) or [a x f; 0] (prismatic), f = [n; f]
template <class S>
__device__ __forceinline__ void crf_s(const S* a, bool pr, const S* f, S* out) {
  if (pr) {
    cross3(a, f + 3, out);
    out[3] = out[4] = out[5] = S(0);
  } else {
    cross3(a, f, out);
    cross3(a, f + 3, out + 3);
  }
}
// S^T f
template <class S>
__device__ __forceinline__ S dot_s(const S* a, bool pr, const S* f) {
  const S f0 = pr ? f[3] : f[0], f1 = pr ? f[4] : f[1], f2 = pr ? f[5] : f[2];
  return a[0] * f0 + a[1] * f1 + a[2] * f2;
}

// Component c of X^T f = [E^T f_ang + r x E^T f_lin; E^T f_lin], with the
// transform record Er = E(9) r(3) read from memory: a lane-dependent c then
// indexes shared memory instead of forcing a local-memory copy of E.
template <class S>
__device__ __forceinline__ S xt_mul_c(const S* Er, const S* f, int c) {
  if (c >= 3) {
    const int k = c - 3;
    return Er[k] * f[3] + Er[3 + k] * f[4] + Er[6 + k] * f[5];
  }
  const int c1 = c == 2 ? 0 : c + 1, c2 = c == 0 ? 2 : c - 1;
  const S g1 = Er[c1] * f[3] + Er[3 + c1] * f[4] + Er[6 + c1] * f[5];
  const S g2 = Er[c2] * f[3] + Er[3 + c2] * f[4] + Er[6 + c2] * f[5];
  const S nc = Er[c] * f[0] + Er[3 + c] * f[1] + Er[6 + c] * f[2];
  return nc + Er[9 + c1] * g2 - Er[9 + c2] * g1;
}

// Component c of I m.
template <class S>
__device__ __forceinline__ S i_mul_c(const S* in, const S* m, int c) {
  S o[6];
  i_mul(in, m, o);
  S x = o[0];
#pragma unroll
  for (int k = 1; k < 6; ++k) x = (c == k) ? o[k] : x;
  return x;
}

// Entry (r, c) of the 6x6 spatial inertia matrix.
template <class S>
__device__ __forceinline__ S i_entry(const S* in, int r, int c) {
  const S h[3] = {in[1], in[2], in[3]};
  if (r < 3 && c < 3) {
    if (r == c) return in[4 + r];
    int a = r < c ? r : c, b = r < c ? c : r;          // (0,1)->7, (0,2)->8, (1,2)->9
    return in[a == 0 ? (b == 1 ? 7 : 8) : 9];
  }
  if (r >= 3 && c >= 3) return r == c ? in[0] : S(0);
  // upper-right block h~, lower-left block h~^T
  int i = r < 3 ? r : c, j = r < 3 ? c - 3 : r - 3;     // entry (i, j) of h~
  S v;
  if (i == j) v = S(0);
  else if (i == 0) v = (j == 1) ? -h[2] : h[1];
  else if (i == 1) v = (j == 0) ? h[2] : -h[0];
  else v = (j == 0) ? -h[1] : h[0];
  return v;
}

// Vector shared-memory access for records aligned to 16 bytes (p must be).
template <class S>
__device__ __forceinline__ void ld2(const S* p, S* o) {
#ifdef __CUDACC__
  if constexpr (sizeof(S) == 4) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    o[0] = t.x; o[1] = t.y;
  } else {
    const double2 t = *reinterpret_cast<const double2*>(p);
    o[0] = t.x; o[1] = t.y;
  }
#else
  o[0] = p[0]; o[1] = p[1];
#endif
}
template <class S>
__device__ __forceinline__ void ld4(const S* p, S* o) {
#ifdef __CUDACC__
  if constexpr (sizeof(S) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
  } else {
    ld2(p, o); ld2(p + 2, o + 2);
  }
#else
  for (int e = 0; e < 4; ++e) o[e] = p[e];
#endif
}
template <class S>
__device__ __forceinline__ void st2(S* p, S a, S b) {
#ifdef __CUDACC__
  if constexpr (sizeof(S) == 4) *reinterpret_cast<float2*>(p) = make_float2(a, b);
  else *reinterpret_cast<double2*>(p) = make_double2(a, b);
#else
  p[0] = a; p[1] = b;
#endif
}
template <class S>
__device__ __forceinline__ void st4(S* p, const S* v) {
#ifdef __CUDACC__
  if constexpr (sizeof(S) == 4) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  else { st2(p, v[0], v[1]); st2(p + 2, v[2], v[3]); }
#else
  for (int e = 0; e < 4; ++e) p[e] = v[e];
#endif
}
// 6-vector stored in an 8-scalar record
template <class S>
__device__ __forceinline__ void ld6(const S* p, S* o) { ld4(p, o); ld2(p + 4, o + 4); }
template <class S>
__device__ __forceinline__ void st6(S* p, const S* v) { st4(p, v); st2(p + 4, v[4], v[5]); }
// transform record E(9) r(3)
template <class S>
__device__ __forceinline__ void ld12(const S* p, S* o) { ld4(p, o); ld4(p + 4, o + 4); ld4(p + 8, o + 8); }
// 6-vector at an 8-byte (not 16-byte) aligned address
template <class S>
__device__ __forceinline__ void ld6u(const S* p, S* o) { ld2(p, o); ld2(p + 2, o + 2); ld2(p + 4, o + 4); }
template <class S>
__device__ __forceinline__ void st6u(S* p, const S* v) { st2(p, v[0], v[1]); st2(p + 2, v[2], v[3]); st2(p + 4, v[4], v[5]); }
