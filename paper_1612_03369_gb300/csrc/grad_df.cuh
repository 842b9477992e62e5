// grad_df.cuh -- the velocity gradient G = du_h/dx = (du_h/dx-hat) J^{-1} at a
// located point, in double-float arithmetic on the FP32 pipe (the FP64 pipe
// of GB300 issues ~1/75 of the FP32 rate).  Used by the property ODEs of
// Sec. 2.6 and by the adjoint sweep.
//
//   du/dx-hat   from the cell's monomial coefficients about its centre
//               (u_c = sum c_pqr s0^p s1^q s2^r, s = x-hat - 1/2, so
//               d/dx-hat = d/ds): Horner steps that carry each partial
//               sum's value and its derivatives along the axes already
//               passed
//   J           from the cell's monomial block (the map about vertex 0,
//               Phi = X_0 + sum_k a_k m_k(t)): J_ij = sum_k a_k,i dm_k/dt_j
//   J^{-1}      cofactors over the determinant, one double-float reciprocal
// Every product is a double-float product (two_prod), every sum a
// double-float sum, so G carries ~2^-44 relative error times the
// conditioning of J.
#pragma once

#include "df.cuh"
#include "fastpath.cuh"

namespace pic {

// 1 / a: FP32 reciprocal refined by one Newton step in double-float.
__device__ __forceinline__ df df_recip(df a) {
  const float r = __frcp_rn(a.hi);
  const df p = two_prod(a.hi, r);                  // a.hi r exactly
  const float e = __fsub_rn(__fsub_rn(1.0f, p.hi), __fmaf_rn(a.lo, r, p.lo));  // 1 - a r
  return fast_two_sum(r, __fmul_rn(r, e));
}

// One coefficient slice (the nine c_pq r of a fixed r, index 3 q + p, as
// q2_eval_df reads them) at s0, s1: its value g and its derivatives g0 along
// s0 and g1 along s1.  Along s0 each row q gives its value h and derivative
// h' = c_1 + 2 c_2 s0; along s1 the rows combine the same way.
__device__ __forceinline__ void grad_slice_df(const float4* __restrict__ sl, df s0, df s1, df& g, df& g0, df& g1) {
  float f[20];  // ten high parts, then ten low parts
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float4 v = __ldg(sl + k);
    f[4 * k] = v.x;
    f[4 * k + 1] = v.y;
    f[4 * k + 2] = v.z;
    f[4 * k + 3] = v.w;
  }
  df c[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) c[e] = df_make(f[e], f[10 + e]);
  df h[3], h0[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    h[q] = df_horner(df_horner(c[3 * q + 2], s0, c[3 * q + 1]), s0, c[3 * q]);
    h0[q] = df_horner(df_scale2(c[3 * q + 2], 2.0f), s0, c[3 * q + 1]);
  }
  g = df_horner(df_horner(h[2], s1, h[1]), s1, h[0]);
  g0 = df_horner(df_horner(h0[2], s1, h0[1]), s1, h0[0]);
  g1 = df_horner(df_scale2(h[2], 2.0f), s1, h[1]);
}

// Gu[c][j] = d u_c / d t_j in cell K at double-float reference coordinates
// t, from the cell's coefficient slices (u_c = sum_r slice_r(s0, s1) s2^r).
// Along s2 the slices combine as d0 = sum g0_r s2^r, d1 = sum g1_r s2^r,
// d2 = g_1 + 2 g_2 s2: 47 double-float Horner steps per component.
template <int D>
__device__ __forceinline__ void q2_grad_mono_df(const float4* __restrict__ Qc, uint32_t K, const df t[D],
                                                df Gu[D][D]) {
  constexpr int NS = (D == 3 ? 3 : 1);
  df s[D];
#pragma unroll
  for (int a = 0; a < D; ++a) s[a] = centred(t[a]);
  const float4* cell = Qc + (size_t)K * D * (5 * NS);
#pragma unroll 1
  for (int comp = 0; comp < D; ++comp) {
    const float4* cq = cell + comp * (5 * NS);
    df g[NS], g0[NS], g1[NS];
#pragma unroll
    for (int r = 0; r < NS; ++r) grad_slice_df(cq + 5 * r, s[0], s[1], g[r], g0[r], g1[r]);
    if constexpr (D == 3) {
      Gu[comp][0] = df_norm(df_horner(df_horner(g0[2], s[2], g0[1]), s[2], g0[0]));
      Gu[comp][1] = df_norm(df_horner(df_horner(g1[2], s[2], g1[1]), s[2], g1[0]));
      Gu[comp][2] = df_norm(df_horner(df_scale2(g[2], 2.0f), s[2], g[1]));
    } else {
      Gu[comp][0] = df_norm(g0[0]);
      Gu[comp][1] = df_norm(g1[0]);
    }
  }
}

// J_ij = dPhi_i/dt_j from the monomial block: in 3D the monomials are
// (t0, t1, t2, t0 t1, t0 t2, t1 t2, t0 t1 t2), in 2D (t0, t1, t0 t1).
template <int D>
__device__ __forceinline__ void map_jacobian_df(const CellBlock<D>& cb, const df t[D], df J[D][D]) {
  if constexpr (D == 3) {
    const df t01 = df_mul(t[0], t[1]), t02 = df_mul(t[0], t[2]), t12 = df_mul(t[1], t[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      df_acc j0 = acc_init(cb.a[0][i]), j1 = acc_init(cb.a[1][i]), j2 = acc_init(cb.a[2][i]);
      acc_mad(j0, cb.a[3][i], t[1]);
      acc_mad(j0, cb.a[4][i], t[2]);
      acc_mad(j0, cb.a[6][i], t12);
      acc_mad(j1, cb.a[3][i], t[0]);
      acc_mad(j1, cb.a[5][i], t[2]);
      acc_mad(j1, cb.a[6][i], t02);
      acc_mad(j2, cb.a[4][i], t[0]);
      acc_mad(j2, cb.a[5][i], t[1]);
      acc_mad(j2, cb.a[6][i], t01);
      J[i][0] = acc_result(j0);
      J[i][1] = acc_result(j1);
      J[i][2] = acc_result(j2);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      df_acc j0 = acc_init(cb.a[0][i]), j1 = acc_init(cb.a[1][i]);
      acc_mad(j0, cb.a[2][i], t[1]);
      acc_mad(j1, cb.a[2][i], t[0]);
      J[i][0] = acc_result(j0);
      J[i][1] = acc_result(j1);
    }
  }
}

// a b - c d
__device__ __forceinline__ df df_det2(df a, df b, df c, df d) {
  df_acc s = acc_zero();
  acc_mad(s, a, b);
  acc_mad(s, c, df_make(-d.hi, -d.lo));
  return acc_result(s);
}

template <int D>
__device__ __forceinline__ void invert_df(const df J[D][D], df Ji[D][D]) {
  if constexpr (D == 2) {
    const df inv = df_recip(df_det2(J[0][0], J[1][1], J[0][1], J[1][0]));
    Ji[0][0] = df_mul(J[1][1], inv);
    Ji[0][1] = df_mul(df_make(-J[0][1].hi, -J[0][1].lo), inv);
    Ji[1][0] = df_mul(df_make(-J[1][0].hi, -J[1][0].lo), inv);
    Ji[1][1] = df_mul(J[0][0], inv);
  } else {
    df c[3][3];
    c[0][0] = df_det2(J[1][1], J[2][2], J[1][2], J[2][1]);
    c[0][1] = df_det2(J[1][2], J[2][0], J[1][0], J[2][2]);
    c[0][2] = df_det2(J[1][0], J[2][1], J[1][1], J[2][0]);
    c[1][0] = df_det2(J[0][2], J[2][1], J[0][1], J[2][2]);
    c[1][1] = df_det2(J[0][0], J[2][2], J[0][2], J[2][0]);
    c[1][2] = df_det2(J[0][1], J[2][0], J[0][0], J[2][1]);
    c[2][0] = df_det2(J[0][1], J[1][2], J[0][2], J[1][1]);
    c[2][1] = df_det2(J[0][2], J[1][0], J[0][0], J[1][2]);
    c[2][2] = df_det2(J[0][0], J[1][1], J[0][1], J[1][0]);
    df_acc det = acc_zero();
    acc_mad(det, J[0][0], c[0][0]);
    acc_mad(det, J[0][1], c[0][1]);
    acc_mad(det, J[0][2], c[0][2]);
    const df inv = df_recip(acc_result(det));
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = 0; q < 3; ++q) Ji[r][q] = df_mul(c[q][r], inv);
  }
}

// G = du_h/dx at double-float reference coordinates t of cell K.
template <int D>
__device__ __forceinline__ void velocity_gradient_df(const MeshView& m, uint32_t K, const df t[D], df G[D][D]) {
  df Gu[D][D], J[D][D], Ji[D][D];
  q2_grad_mono_df<D>(m.Qc, K, t, Gu);
  CellBlock<D> cb;
  load_block<D>(m, K, cb);
  map_jacobian_df<D>(cb, t, J);
  invert_df<D>(J, Ji);
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int q = 0; q < D; ++q) {
      df_acc s = acc_zero();
#pragma unroll
      for (int j = 0; j < D; ++j) acc_mad(s, Gu[c][j], Ji[j][q]);
      G[c][q] = acc_result(s);
    }
}

// sqrt(a), a >= 0: FP32 root refined by one Newton step in double-float.
__device__ __forceinline__ df df_sqrt(df a) {
  if (!(a.hi > 0.f)) return df_make(0.f, 0.f);
  const float r = __fsqrt_rn(a.hi);
  const df r2 = two_prod(r, r);
  const float e = __fdiv_rn(__fadd_rn(__fsub_rn(a.hi, r2.hi), __fsub_rn(a.lo, r2.lo)), __fmul_rn(2.0f, r));
  return fast_two_sum(r, e);
}

}  // namespace pic
