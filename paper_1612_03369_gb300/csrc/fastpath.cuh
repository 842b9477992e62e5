// fastpath.cuh -- the advection hot path in double-float arithmetic on the
// FP32 pipe (Sec. 2.3 velocity evaluation, Sec. 2.4 location).
//
// Layouts (built once per mesh / velocity field):
//   cell block   per cell, the (bi/tri)linear map in monomial form about
//                vertex 0: Phi_K(t) = X_0 + sum_k a_k m_k(t) with
//                m = (t0, t1, t2, t0 t1, t0 t2, t1 t2, t0 t1 t2) in 3D and
//                (t0, t1, t0 t1) in 2D; X_0 and every a_k as double-floats
//                (192 B per hex, 64 B per quad, 16-byte aligned)
//   U2           Q2 nodal values as double-floats, node-major [node][dim]
//                (the source of the coefficient slices below)
//
// Qc, the Q2 field's per-cell monomial coefficients about the cell centre
// (double-float, 720 B per hex), and Qf, their high parts alone for the
// FP32-basis form (336 B per hex), are built with the field (mesh.cu).
//
// Where a cell's blocks are read from is a template parameter: GlobalCells
// reads the mesh arrays; StagedCells a shared-memory copy of the cells a
// warp's particles start in (advect.cu), and the mesh arrays for any other
// cell.  The arithmetic is the same either way, so every kernel that inlines
// it computes the same bits.
//
// Inverse map (Newton, Sec. 2.2 / Remark 2.1): FP32 iterations on the local
// offset y - X_0 until the update falls below 1e-5, then one Newton step
// whose residual (y - X_0) - sum_k a_k m_k(t) is evaluated in double-float
// (absolute accuracy ~2^-47 h), with the FP32 Jacobian at the current
// iterate.  That leaves |t - t*| ~ 1e-14.  If the FP32 phase does not settle
// the cell is handed to the FP64 Newton of pic_internal.cuh (rare).
#pragma once

#include "df.cuh"
#include "locate.cuh"
#include "pic_internal.cuh"

namespace pic {

// FP32 phase ends when max|update| <= kSettle32: the iterate is then within
// ~C*kSettle32^2 + 1e-7 of the root (C ~ 1 for cells jittered by 10%), and
// the double-float step takes that to ~C*(2e-7)^2 + 3e-7*2e-7 ~ 1e-13 (the
// FP32 Jacobian and the approximate reciprocal of solve32 scale the update).
constexpr float kSettle32 = 2e-4f;
constexpr int kMaxIt32 = 8;

template <int D>
struct CellBlock {
  df x0[D];
  df a[(1 << D) - 1][D];
};

// The high parts alone (what the FP32 Newton iterations read).
template <int D>
struct CellBlock32 {
  float x0[D];
  float a[(1 << D) - 1][D];
};

template <int D>
__host__ __device__ constexpr int block_float4s() {
  return (2 * D + 2 * D * ((1 << D) - 1)) / 4;  // 12 (3D) or 4 (2D)
}
// float4 per cell of Qc: per component NS slices of 5 float4 (ten high
// parts, then ten low parts; the tenth of each is zero).
template <int D>
__host__ __device__ constexpr int qc_float4s() {
  return D * 5 * (D == 3 ? 3 : 1);  // 45 (3D) or 10 (2D)
}
// Qf: per component the 3^D high parts in the order r*9 + q*3 + p (the
// coefficient of s2^r s1^q s0^p), padded to 28 (3D) or 12 (2D) floats.
template <int D>
__host__ __device__ constexpr int qf_floats_per_comp() {
  return D == 3 ? 28 : 12;
}
template <int D>
__host__ __device__ constexpr int qf_float4s() {
  return D * qf_floats_per_comp<D>() / 4;  // 21 (3D) or 6 (2D)
}

// ------------------------------------------------------ cell data source --

template <int D, bool F32B>
struct GlobalCells {
  static constexpr int NB = block_float4s<D>();
  static constexpr int NQ = F32B ? qf_float4s<D>() : qc_float4s<D>();
  const MeshView& m;
  __device__ __forceinline__ const float4* block(uint32_t K) const { return m.blk + (size_t)K * NB; }
  __device__ __forceinline__ const float4* coef(uint32_t K) const { return (F32B ? m.Qf : m.Qc) + (size_t)K * NQ; }
  __device__ __forceinline__ float4 ld(const float4* p) const { return __ldg(p); }
};

// Cells [K0, K0 + n) from shared memory (sbase: their map blocks in order,
// then from sbase + kStage * NB their coefficient blocks), every other cell
// from the mesh arrays.  Loads are generic, so one instruction serves both.
template <int D, bool F32B, int kStage>
struct StagedCells {
  static constexpr int NB = block_float4s<D>();
  static constexpr int NQ = F32B ? qf_float4s<D>() : qc_float4s<D>();
  const MeshView& m;
  const float4* sbase;
  uint32_t K0, n;
  __device__ __forceinline__ const float4* block(uint32_t K) const {
    const uint32_t o = K - K0;
    return o < n ? sbase + o * NB : m.blk + (size_t)K * NB;
  }
  __device__ __forceinline__ const float4* coef(uint32_t K) const {
    const uint32_t o = K - K0;
    return o < n ? sbase + kStage * NB + o * NQ : (F32B ? m.Qf : m.Qc) + (size_t)K * NQ;
  }
  __device__ __forceinline__ float4 ld(const float4* p) const { return *p; }
};

// Block layout per cell: NF = D + (2^D - 1) D high parts (X_0, then a_k,c in
// (k, c) order), then the NF low parts in the same order.  B points at the
// cell's block, read through the source's loader.
template <int D, class Cells>
__device__ __forceinline__ void load_block_half(const Cells& cs, const float4* B, int half, float f[]) {
  constexpr int NH = block_float4s<D>() / 2;
  const float4* p = B + half * NH;
#pragma unroll
  for (int q = 0; q < NH; ++q) {
    const float4 v = cs.ld(p + q);
    f[4 * q] = v.x;
    f[4 * q + 1] = v.y;
    f[4 * q + 2] = v.z;
    f[4 * q + 3] = v.w;
  }
}

template <int D, class Cells>
__device__ __forceinline__ void load_block32(const Cells& cs, const float4* B, CellBlock32<D>& cb) {
  float f[2 * block_float4s<D>()];
  load_block_half<D>(cs, B, 0, f);
#pragma unroll
  for (int a = 0; a < D; ++a) cb.x0[a] = f[a];
#pragma unroll
  for (int k = 0; k < (1 << D) - 1; ++k)
#pragma unroll
    for (int a = 0; a < D; ++a) cb.a[k][a] = f[D + k * D + a];
}

template <int D>
__device__ __forceinline__ void load_block(const MeshView& m, uint32_t K, CellBlock<D>& cb) {
  constexpr int NF = 2 * block_float4s<D>();  // floats per half
  const GlobalCells<D, false> cs{m};
  const float4* B = cs.block(K);
  float hi[NF], lo[NF];
  load_block_half<D>(cs, B, 0, hi);
  load_block_half<D>(cs, B, 1, lo);
#pragma unroll
  for (int a = 0; a < D; ++a) cb.x0[a] = df_make(hi[a], lo[a]);
#pragma unroll
  for (int k = 0; k < (1 << D) - 1; ++k)
#pragma unroll
    for (int a = 0; a < D; ++a) cb.a[k][a] = df_make(hi[D + k * D + a], lo[D + k * D + a]);
}

// FP32 map offset phi(t) = sum_k a_k m_k(t) and Jacobian, from the high parts.
template <int D>
__device__ __forceinline__ void map32(const CellBlock32<D>& cb, const float t[D], float phi[D], float J[D][D]) {
  if constexpr (D == 2) {
    const float t01 = __fmul_rn(t[0], t[1]);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float a1 = cb.a[0][c], a2 = cb.a[1][c], a3 = cb.a[2][c];
      phi[c] = fmaf(a3, t01, fmaf(a2, t[1], __fmul_rn(a1, t[0])));
      J[c][0] = fmaf(a3, t[1], a1);
      J[c][1] = fmaf(a3, t[0], a2);
    }
  } else {
    const float t01 = __fmul_rn(t[0], t[1]), t02 = __fmul_rn(t[0], t[2]), t12 = __fmul_rn(t[1], t[2]);
    const float t012 = __fmul_rn(t01, t[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float a1 = cb.a[0][c], a2 = cb.a[1][c], a3 = cb.a[2][c], a4 = cb.a[3][c];
      const float a5 = cb.a[4][c], a6 = cb.a[5][c], a7 = cb.a[6][c];
      phi[c] = fmaf(a7, t012, fmaf(a6, t12, fmaf(a5, t02, fmaf(a4, t01, fmaf(a3, t[2], fmaf(a2, t[1], __fmul_rn(a1, t[0])))))));
      J[c][0] = fmaf(a7, t12, fmaf(a5, t[2], fmaf(a4, t[1], a1)));
      J[c][1] = fmaf(a7, t02, fmaf(a6, t[2], fmaf(a4, t[0], a2)));
      J[c][2] = fmaf(a7, t01, fmaf(a6, t[1], fmaf(a5, t[0], a3)));
    }
  }
}

template <int D>
__device__ __forceinline__ bool solve32(const float J[D][D], const float r[D], float d[D]) {
  // Every operation is an explicit rounded intrinsic, in a fixed order, so
  // that every kernel inlining this (the advect kernel's template instances,
  // the stage-recording kernel, the adjoint's stage kernel) computes the same
  // iterates bit for bit, whatever the compiler would contract on its own.
  // The determinant's reciprocal is the hardware approximation (one
  // instruction, within 2 ulp; the IEEE division took a dozen): it scales a
  // Newton update whose last, double-float-residual step is ~1e-7, so it
  // moves the root by ~3e-14, the size of the FP32 Jacobian's own error.  A
  // zero or non-finite determinant fails here; one so small that its
  // reciprocal overflows gives an update the caller rejects (|d| > 1e3).
  auto det2 = [](float a, float b, float c, float e) { return __fmaf_rn(a, b, -__fmul_rn(c, e)); };  // a b - c e
  if constexpr (D == 2) {
    const float det = det2(J[0][0], J[1][1], J[0][1], J[1][0]);
    if (!(fabsf(det) > 0.f) || !isfinite(det)) return false;
    const float inv = __fdividef(1.0f, det);
    d[0] = __fmul_rn(det2(J[1][1], r[0], J[0][1], r[1]), inv);
    d[1] = __fmul_rn(det2(J[0][0], r[1], J[1][0], r[0]), inv);
    return true;
  } else {
    const float c00 = det2(J[1][1], J[2][2], J[1][2], J[2][1]);
    const float c01 = det2(J[1][2], J[2][0], J[1][0], J[2][2]);
    const float c02 = det2(J[1][0], J[2][1], J[1][1], J[2][0]);
    const float det = __fmaf_rn(J[0][2], c02, __fmaf_rn(J[0][1], c01, __fmul_rn(J[0][0], c00)));
    if (!(fabsf(det) > 0.f) || !isfinite(det)) return false;
    const float inv = __fdividef(1.0f, det);
    const float c10 = det2(J[0][2], J[2][1], J[0][1], J[2][2]);
    const float c11 = det2(J[0][0], J[2][2], J[0][2], J[2][0]);
    const float c12 = det2(J[0][1], J[2][0], J[0][0], J[2][1]);
    const float c20 = det2(J[0][1], J[1][2], J[0][2], J[1][1]);
    const float c21 = det2(J[0][2], J[1][0], J[0][0], J[1][2]);
    const float c22 = det2(J[0][0], J[1][1], J[0][1], J[1][0]);
    d[0] = __fmul_rn(__fmaf_rn(c20, r[2], __fmaf_rn(c10, r[1], __fmul_rn(c00, r[0]))), inv);
    d[1] = __fmul_rn(__fmaf_rn(c21, r[2], __fmaf_rn(c11, r[1], __fmul_rn(c01, r[0]))), inv);
    d[2] = __fmul_rn(__fmaf_rn(c22, r[2], __fmaf_rn(c12, r[1], __fmul_rn(c02, r[0]))), inv);
    return true;
  }
}

// Double-float residual r = dloc - sum_k a_k m_k(t) at a single-float point t
// (the monomials of t are formed exactly with two_prod).
template <int D>
__device__ __forceinline__ void residual_df(const CellBlock32<D>& cb, const float lo[], const df dloc[D], const float t[D],
                                            float r[D]) {
  auto A = [&](int k, int c) { return df_make(-cb.a[k][c], -lo[D + k * D + c]); };
  const df m01 = two_prod(t[0], t[1]);
  if constexpr (D == 2) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      df_acc acc = acc_init(dloc[c]);
      acc_mad_f(acc, A(0, c), t[0]);
      acc_mad_f(acc, A(1, c), t[1]);
      acc_mad(acc, A(2, c), m01);
      r[c] = __fadd_rn(acc.s, acc.e);
    }
  } else {
    const df m02 = two_prod(t[0], t[2]);
    const df m12 = two_prod(t[1], t[2]);
    const df m012 = df_mul_f(m01, t[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      df_acc acc = acc_init(dloc[c]);
      acc_mad_f(acc, A(0, c), t[0]);
      acc_mad_f(acc, A(1, c), t[1]);
      acc_mad_f(acc, A(2, c), t[2]);
      acc_mad(acc, A(3, c), m01);
      acc_mad(acc, A(4, c), m02);
      acc_mad(acc, A(5, c), m12);
      acc_mad(acc, A(6, c), m012);
      r[c] = __fadd_rn(acc.s, acc.e);
    }
  }
}

// Outcome of the inverse map in one cell (kCellDefer: the fast path alone
// cannot decide, see kDefer).
enum : int { kCellOut = 0, kCellIn = 1, kCellFail = -1, kCellDefer = -2 };

// Returned instead of a cell by the fast-path-only locate (kFast == true)
// where the full locate would enter a rare path (the FP64 Newton, the
// lowest-index test of the cells across a nearby facet, the FP64 walk): the
// caller hands the particle to a second kernel that runs the full step.  A
// kernel without those out-of-line calls needs no spill code around them.
constexpr uint32_t kDefer = 0xFFFFFFFEu;

// Points and results passed by value to and from the out-of-line rare paths,
// so that no variable of the hot loop has its address taken (an address-
// taken variable lives in local memory for its whole life).
template <int D>
struct DfPt {
  df v[D];
};
template <int D>
struct RarePath {
  DfPt<D> t;       // reference coordinates found
  uint32_t K;      // cell found (PIC_LOST: none)
  int r;           // kCellIn / kCellOut / kCellFail (single-cell tests)
  int iters;       // Newton iterations spent
  unsigned flags;  // flags raised
};
template <int D>
__device__ __forceinline__ DfPt<D> pack(const df a[D]) {
  DfPt<D> p;
#pragma unroll
  for (int i = 0; i < D; ++i) p.v[i] = a[i];
  return p;
}

// Inverse map of y in cell K (fast path).  t32 holds the FP32 start on entry;
// on return t holds the double-float reference coordinates.
// With accurate == false (stage points of the FP32-basis form) the FP32
// phase runs to kSettle32Tight and the double-float step is skipped: x-hat is
// then good to ~1e-7, which is what an FP32 basis evaluation can use.
constexpr float kSettle32Tight = 1e-5f;

template <int D, class Cells>
__device__ __forceinline__ int solve_cell_df(const Cells& cs, uint32_t K, const df y[D], float t32[D], df t[D],
                                             int& iters, bool accurate = true) {
  const float4* B = cs.block(K);
  CellBlock32<D> cb;
  load_block32<D>(cs, B, cb);
  df dloc[D];
  float d32[D];
  {
    // X_0's low parts lead the block's second half
    const float4 x0lo = cs.ld(B + block_float4s<D>() / 2);
    const float l[3] = {x0lo.x, x0lo.y, x0lo.z};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      dloc[a] = df_sub(y[a], df_make(cb.x0[a], l[a]));
      d32[a] = dloc[a].hi;
    }
  }
  float phi[D], J[D][D], r[D], dt[D];
  bool settled = false;
#pragma unroll 1
  for (int it = 0; it < kMaxIt32; ++it) {
    ++iters;
    map32<D>(cb, t32, phi, J);
#pragma unroll
    for (int a = 0; a < D; ++a) r[a] = d32[a] - phi[a];
    if (!solve32<D>(J, r, dt)) return kCellFail;
    float mx = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      t32[a] += dt[a];
      mx = fmaxf(mx, fabsf(dt[a]));
    }
    if (!(mx <= 1e3f)) return kCellFail;  // diverging or NaN
    // Clearly outside: the iterate lies outside [0,1] by much more than the
    // last update (Newton is in its quadratic regime once the update is
    // small), so the root is outside too.  Stop here; t32 tells the walk
    // where to go.  A wrong call only costs time: the walk then falls back
    // to the FP64 search, and ownership is still the lowest-index rule.
    if (mx < 0.05f) {
      float out = 0.f;
#pragma unroll
      for (int a = 0; a < D; ++a) out = fmaxf(out, fmaxf(-t32[a], t32[a] - 1.0f));
      if (out > 4.f * mx + 1e-3f) return kCellOut;
    }
    if (mx <= (accurate ? kSettle32 : kSettle32Tight)) {
      settled = true;
      break;
    }
  }
  if (!settled) return kCellFail;
  if (!accurate) {
    bool in = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      t[a] = df_make(t32[a], 0.f);
      in = in && (t32[a] >= -(float)kInsideEps) && (t32[a] <= 1.0f + (float)kInsideEps);
    }
    return in ? kCellIn : kCellOut;
  }
  // one Newton step with the double-float residual
  ++iters;
  map32<D>(cb, t32, phi, J);
  {
    float lo[2 * block_float4s<D>()];
    load_block_half<D>(cs, B, 1, lo);
    residual_df<D>(cb, lo, dloc, t32, r);
  }
  if (!solve32<D>(J, r, dt)) return kCellFail;
  float mx = 0.f;
#pragma unroll
  for (int a = 0; a < D; ++a) mx = fmaxf(mx, fabsf(dt[a]));
  if (!(mx <= 1e-5f)) return kCellFail;
  bool in = true;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    t[a] = two_sum(t32[a], dt[a]);
    // t >= -eps  <=>  t32 >= -eps - dt ;  t <= 1 + eps  <=>  t32 - 1 <= eps - dt
    in = in && (t32[a] >= -(float)kInsideEps - dt[a]) && (t32[a] - 1.0f <= (float)kInsideEps - dt[a]);
  }
  return in ? kCellIn : kCellOut;
}

// FP64 Newton for a cell the fast path could not settle (rare; out of line
// so that the hot loop stays small in the instruction cache); s32 holds the
// FP32 start in its high parts.
template <int D>
__device__ __noinline__ RarePath<D> test_cell_fp64(const MeshView& m, uint32_t K, DfPt<D> y, DfPt<D> s32) {
  RarePath<D> o;
  o.iters = 0;
  o.flags = 0;
  o.K = K;
  double yd[D], tt[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    yd[a] = df_to_double(y.v[a]);
    const float st = s32.v[a].hi;
    tt[a] = isfinite(st) && fabsf(st) < 4.f ? (double)st : 0.5;
  }
  bool conv = false;
  const bool in = try_cell<D>(m, K, yd, tt, o.iters, o.flags, &conv);
#pragma unroll
  for (int a = 0; a < D; ++a) o.t.v[a] = df_from_double(tt[a]);
  o.r = !conv ? kCellFail : (in ? kCellIn : kCellOut);
  return o;
}

// Fast path, then the FP64 Newton when the fast path does not settle.
// y inside cell K's padded bounding box (padding 1e-6 of the cell's extent,
// far wider than the kInsideEps band in reference coordinates): a point
// outside it is not in K.  The FP32 copy of the box is widened outward, so
// the test on y's high parts is conservative, with no FP64 instruction.
template <int D>
__device__ __forceinline__ bool in_cell_box(const MeshView& m, uint32_t K, const df y[D]) {
  const float4 lo = __ldg(m.bbox32 + 2 * (size_t)K), hi = __ldg(m.bbox32 + 2 * (size_t)K + 1);
  const float l[3] = {lo.x, lo.y, lo.z}, h[3] = {hi.x, hi.y, hi.z};
  bool in = true;
#pragma unroll
  for (int a = 0; a < D; ++a) in = in && y[a].hi >= l[a] && y[a].hi <= h[a];
  return in;
}

template <int D, bool kFast = false, class Cells>
__device__ __forceinline__ int test_cell(const Cells& cs, const MeshView& m, uint32_t K, const df y[D], float t32[D],
                                         df t[D], int& iters, unsigned& flags, bool accurate = true) {
  DfPt<D> s;
#pragma unroll
  for (int a = 0; a < D; ++a) s.v[a] = df_make(t32[a], 0.f);
  const int r = solve_cell_df<D>(cs, K, y, t32, t, iters, accurate);
  if (r != kCellFail) return r;
  if constexpr (kFast) return kCellDefer;
  const RarePath<D> o = test_cell_fp64<D>(m, K, pack<D>(y), s);
  iters += o.iters;
  flags |= o.flags | kFlagFallback64;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    t[a] = o.t.v[a];
    t32[a] = t[a].hi;
  }
  return o.r;
}

// Lowest-index rule (see lowest_owner in locate.cuh) on the fast path.  The
// band test is inline; the neighbour tests (rare) are out of line and read
// the cells from the mesh arrays.
template <int D>
__device__ __noinline__ RarePath<D> lowest_owner_df_slow(const MeshView& m, DfPt<D> y, uint32_t found, DfPt<D> t) {
  RarePath<D> o;
  o.iters = 0;
  o.flags = 0;
  o.r = kCellIn;
  int c[3];
  cell_ijk<D>(m, found, c);
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    lo[a] = (t.v[a].hi < (float)kTieBand && c[a] > 0) ? -1 : 0;
    hi[a] = (t.v[a].hi > 1.0f - (float)kTieBand && c[a] < m.n[a] - 1) ? 1 : 0;
  }
  uint32_t best = found;
  DfPt<D> tb = t;
  for (int o2 = (D == 3 ? lo[2] : 0); o2 <= (D == 3 ? hi[2] : 0); ++o2)
    for (int o1 = lo[1]; o1 <= hi[1]; ++o1)
      for (int o0 = lo[0]; o0 <= hi[0]; ++o0) {
        if (o0 == 0 && o1 == 0 && o2 == 0) continue;
        const uint32_t K = cell_index<D>(m, c[0] + o0, c[1] + o1, c[2] + o2);
        if (K >= best) continue;
        const int off[3] = {o0, o1, o2};
        float s[D];
        df tt[D];
#pragma unroll
        for (int a = 0; a < D; ++a) s[a] = t.v[a].hi - (float)off[a];
        if (test_cell<D>(GlobalCells<D, false>{m}, m, K, y.v, s, tt, o.iters, o.flags) == kCellIn) {
          best = K;
          tb = pack<D>(tt);
        }
      }
  o.K = best;
  o.t = tb;
  return o;
}

template <int D, bool kFast = false>
__device__ __forceinline__ uint32_t lowest_owner_df(const MeshView& m, const df y[D], uint32_t found, df t[D],
                                                    int& iters, unsigned& flags) {
  // band test first (cheap); the cell's (i,j,k), which needs integer
  // divisions, only when some coordinate is near a facet
  bool near = false;
#pragma unroll
  for (int a = 0; a < D; ++a) near = near || t[a].hi < (float)kTieBand || t[a].hi > 1.0f - (float)kTieBand;
  if (!near) return found;
  int c[3];
  cell_ijk<D>(m, found, c);
  bool any = false;
#pragma unroll
  for (int a = 0; a < D; ++a)
    any = any || (t[a].hi < (float)kTieBand && c[a] > 0) || (t[a].hi > 1.0f - (float)kTieBand && c[a] < m.n[a] - 1);
  if (!any) return found;
  if constexpr (kFast) return kDefer;
  const RarePath<D> o = lowest_owner_df_slow<D>(m, pack<D>(y), found, pack<D>(t));
  iters += o.iters;
  flags |= o.flags;
#pragma unroll
  for (int a = 0; a < D; ++a) t[a] = o.t.v[a];
  return o.K;
}

// Past the hint cell and its predicted neighbour: the walk over the hint's
// other vertex neighbours in the paper's order (Sec. 2.4: v the vertex of the
// hint closest to y, descending (y - v).(c_K' - v) over the neighbours' centres
// c_K'), each cell tested with the double-float inverse map (FP64 Newton only
// where that does not settle), then the all-cells search.  The order only
// affects the cost: the first cell found is settled by the lowest-index
// rule, so the ordering heuristic is computed in FP32.  Each candidate's
// Newton starts from the cell centre.
template <int D>
__device__ __noinline__ RarePath<D> locate_df_slow(const MeshView& m, DfPt<D> y, uint32_t hintK) {
  RarePath<D> o;
  o.iters = 0;
  o.flags = 0;
  o.r = kCellIn;
  double yd[D];
#pragma unroll
  for (int a = 0; a < D; ++a) yd[a] = df_to_double(y.v[a]);
  bool inside_box = true;
#pragma unroll
  for (int a = 0; a < D; ++a) inside_box = inside_box && yd[a] >= m.dlo[a] && yd[a] <= m.dhi[a];
  if (!inside_box) {
    // outside the padded domain box: in no cell (see locate in locate.cuh)
    o.K = PIC_LOST;
#pragma unroll
    for (int a = 0; a < D; ++a) o.t.v[a] = df_make(0.f, 0.f);
    return o;
  }
  if (hintK < m.C) {
    o.flags |= kFlagWalk;
    int c[3];
    cell_ijk<D>(m, hintK, c);
    // corner positions of cell (i,j,k) from the vertex array, in FP32
    auto vertex = [&](int i, int j, int k, float p[D]) {
      const int64_t v = (int64_t)i + (int64_t)m.nv[0] * ((int64_t)j + (D == 3 ? (int64_t)m.nv[1] * k : 0));
#pragma unroll
      for (int a = 0; a < D; ++a) p[a] = (float)__ldg(m.X + a * m.nverts + v);
    };
    float yf[D], v[D], best = 3.4e38f;
#pragma unroll
    for (int a = 0; a < D; ++a) yf[a] = y.v[a].hi;
    for (int q = 0; q < (1 << D); ++q) {
      float p[D], d2 = 0.f;
      vertex(c[0] + (q & 1), c[1] + ((q >> 1) & 1), D == 3 ? c[2] + ((q >> 2) & 1) : 0, p);
#pragma unroll
      for (int a = 0; a < D; ++a) d2 += (yf[a] - p[a]) * (yf[a] - p[a]);
      if (d2 < best) {
        best = d2;
#pragma unroll
        for (int a = 0; a < D; ++a) v[a] = p[a];
      }
    }
    constexpr int NN = (D == 3 ? 27 : 9);
    float score[NN];
    uint32_t cand = 0;  // bit mask of the neighbours still to test
    for (int q = 0; q < NN; ++q) {
      const int o0 = q % 3 - 1, o1 = (q / 3) % 3 - 1, o2 = (D == 3 ? q / 9 - 1 : 0);
      score[q] = 0.f;
      if (o0 == 0 && o1 == 0 && o2 == 0) continue;
      const int i = c[0] + o0, j = c[1] + o1, k = c[2] + o2;
      if (i < 0 || j < 0 || i >= m.n[0] || j >= m.n[1]) continue;
      if (D == 3 && (k < 0 || k >= m.n[2])) continue;
      float ctr[D] = {};
      for (int w = 0; w < (1 << D); ++w) {
        float p[D];
        vertex(i + (w & 1), j + ((w >> 1) & 1), D == 3 ? k + ((w >> 2) & 1) : 0, p);
#pragma unroll
        for (int a = 0; a < D; ++a) ctr[a] += p[a] * (1.f / (1 << D));
      }
      float sc = 0.f;
#pragma unroll
      for (int a = 0; a < D; ++a) sc += (yf[a] - v[a]) * (ctr[a] - v[a]);
      score[q] = sc;
      cand |= 1u << q;
    }
    const GlobalCells<D, false> cs{m};
    while (cand) {
      int qb = __ffs(cand) - 1;  // a valid candidate even if every score is NaN
      float sb = score[qb];
      for (int q = qb + 1; q < NN; ++q)
        if (((cand >> q) & 1u) && score[q] > sb) {
          sb = score[q];
          qb = q;
        }
      cand &= ~(1u << qb);
      const int off[3] = {qb % 3 - 1, (qb / 3) % 3 - 1, D == 3 ? qb / 9 - 1 : 0};
      const uint32_t K = cell_index<D>(m, c[0] + off[0], c[1] + off[1], c[2] + off[2]);
      if (!in_cell_box<D>(m, K, y.v)) continue;  // cannot hold y: no Newton there
      float s32[D];
      df tt[D];
#pragma unroll
      for (int a = 0; a < D; ++a) s32[a] = 0.5f;  // from the cell centre (R2)
      if (test_cell<D>(cs, m, K, y.v, s32, tt, o.iters, o.flags) == kCellIn) {
        o.K = lowest_owner_df<D>(m, y.v, K, tt, o.iters, o.flags);
        o.t = pack<D>(tt);
        return o;
      }
    }
  }
  double to[D];
  o.K = global_search<D>(m, yd, to, o.iters, o.flags);
#pragma unroll
  for (int a = 0; a < D; ++a) o.t.v[a] = df_from_double(to[a]);
  return o;
}

template <int D>
__device__ __forceinline__ uint32_t locate_slow(const MeshView& m, const df y[D], uint32_t hintK, df t[D], int& iters,
                                                unsigned& flags) {
  const RarePath<D> o = locate_df_slow<D>(m, pack<D>(y), hintK);
  iters += o.iters;
  flags |= o.flags;
#pragma unroll
  for (int a = 0; a < D; ++a) t[a] = o.t.v[a];
  return o.K;
}

// Owner of y (lowest index) and its double-float reference coordinates.
// Search order: the hint cell, then up to two hops to the neighbour that the
// current cell's Newton iterate points to (across every facet it violates),
// then (out of line) the FP64 walk over the hint's vertex neighbours in the
// paper's a.b order and the all-cells search.  The owner does not depend on
// the order: the first cell found to hold y is settled by the lowest-index
// rule.
constexpr int kPredictedHops = 2;

template <int D, bool kFast = false, class Cells>
__device__ __forceinline__ uint32_t locate_df(const Cells& cs, const MeshView& m, const df y[D], uint32_t hintK,
                                              const float hint_t[D], df t[D], int& iters, unsigned& flags,
                                              bool accurate = true) {
  if (hintK >= m.C) {
    if constexpr (kFast) return kDefer;
    flags |= kFlagBounds;
    return locate_slow<D>(m, y, hintK, t, iters, flags);
  }
  float t32[D];
#pragma unroll
  for (int a = 0; a < D; ++a) t32[a] = hint_t[a];
  uint32_t K = hintK;
#pragma unroll 1
  for (int pass = 0; pass <= kPredictedHops; ++pass) {
    const int r = test_cell<D, kFast>(cs, m, K, y, t32, t, iters, flags, accurate);
    if constexpr (kFast)
      if (r == kCellDefer) return kDefer;
    if (r == kCellIn) return lowest_owner_df<D, kFast>(m, y, K, t, iters, flags);
    if (pass == kPredictedHops || r != kCellOut) break;
    flags |= kFlagWalk;
    int c[3], pred[3] = {0, 0, 0};
    cell_ijk<D>(m, K, c);
    bool have_pred = false;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      pred[a] = t32[a] < 0.f ? -1 : (t32[a] >= 1.f ? 1 : 0);
      if (c[a] + pred[a] < 0 || c[a] + pred[a] >= m.n[a]) pred[a] = 0;
      have_pred = have_pred || pred[a] != 0;
      t32[a] -= (float)pred[a];
    }
    if (!have_pred) break;
    K = cell_index<D>(m, c[0] + pred[0], c[1] + pred[1], c[2] + pred[2]);
  }
  if constexpr (kFast) return kDefer;
  flags |= kFlagWalk | kFlagWalk64;
  return locate_slow<D>(m, y, hintK, t, iters, flags);
}

// The same reading every block from the mesh arrays.
template <int D>
__device__ __forceinline__ uint32_t locate_df(const MeshView& m, const df y[D], uint32_t hintK, const float hint_t[D],
                                              df t[D], int& iters, unsigned& flags, bool accurate = true) {
  return locate_df<D>(GlobalCells<D, false>{m}, m, y, hintK, hint_t, t, iters, flags, accurate);
}

// ---------------------------------------------------------- Q2 velocity --
// u_h = sum_{a,b,c} U[node(K; a,b,c)] l_a(t0) l_b(t1) l_c(t2) with the 1D
// quadratic Lagrange basis on {0, 1/2, 1}:
//   l0 = (1-t)(1-2t) = -w v,  l1 = 4 t w,  l2 = t v,  w = 1-t, v = 2t-1.
// lagrange2_df gives the basis in double-float (used by the gradient).

__device__ __forceinline__ void lagrange2_df(df t, df l[3]) {
  const df ws = two_sum(1.0f, -t.hi);
  const df w = fast_two_sum(ws.hi, __fsub_rn(ws.lo, t.lo));
  const df vs = two_sum(__fmul_rn(2.0f, t.hi), -1.0f);
  const df v = fast_two_sum(vs.hi, __fmaf_rn(2.0f, t.lo, vs.lo));
  const df wv = df_mul(w, v);
  l[0] = df_make(-wv.hi, -wv.lo);
  l[1] = df_scale2(df_mul(t, w), 4.0f);
  l[2] = df_mul(t, v);
}

// The evaluation itself uses the per-cell monomial form about the cell
// centre (built from the nodal values when the field is set):
//   u_c(s) = sum_{p,q,r} C_pqr s0^p s1^q s2^r,   s = t - 1/2,
// evaluated by nested Horner steps, 26 per component in 3D (8 in 2D),
// each a double-float multiply-add.  For smooth fields |C_pqr| falls
// with p + q + r (C_000 is the centre node's value), so the evaluation is
// well conditioned.

// c + a s in double-float, the result left unnormalised (its low part may
// exceed half an ulp of the high part slightly; the next step multiplies it
// exactly through two_prod and an FMA).
__device__ __forceinline__ df df_horner(df a, df s, df c) {
  const df p = two_prod(a.hi, s.hi);
  float e = __fmaf_rn(a.hi, s.lo, p.lo);
  e = __fmaf_rn(a.lo, s.hi, e);
  const df q = two_sum(p.hi, c.hi);
  return df_make(q.hi, __fadd_rn(q.lo, __fadd_rn(e, c.lo)));
}

// s = t - 1/2 in double-float.
__device__ __forceinline__ df centred(df t) {
  const df d = two_sum(t.hi, -0.5f);
  return fast_two_sum(d.hi, __fadd_rn(d.lo, t.lo));
}

// From the cell's Qc block `cell`, read through ld.ld().
template <int D, class Ld>
__device__ __forceinline__ void q2_eval_df(const Ld& ld, const float4* cell, const df t[D], df u[D]) {
  constexpr int NS = (D == 3 ? 3 : 1);
  df s[D];
#pragma unroll
  for (int a = 0; a < D; ++a) s[a] = centred(t[a]);
#pragma unroll 1
  for (int comp = 0; comp < D; ++comp) {
    const float4* cq = cell + comp * (5 * NS);
    df g[NS];
#pragma unroll
    for (int r = 0; r < NS; ++r) {
      float f[20];  // ten high parts, then ten low parts
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const float4 v = ld.ld(cq + 5 * r + k);
        f[4 * k] = v.x;
        f[4 * k + 1] = v.y;
        f[4 * k + 2] = v.z;
        f[4 * k + 3] = v.w;
      }
      df c[10];
#pragma unroll
      for (int e = 0; e < 10; ++e) c[e] = df_make(f[e], f[10 + e]);
      df h[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) h[q] = df_horner(df_horner(c[3 * q + 2], s[0], c[3 * q + 1]), s[0], c[3 * q]);
      g[r] = df_horner(df_horner(h[2], s[1], h[1]), s[1], h[0]);
    }
    df rr;
    if constexpr (D == 3)
      rr = df_norm(df_horner(df_horner(g[2], s[2], g[1]), s[2], g[0]));
    else
      rr = df_norm(g[0]);
    // constant indices keep u in registers under the rolled loop
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (a == comp) u[a] = rr;
  }
}

// FP32 basis and contraction (precision form) from the cell's Qf block: the
// same monomial form on the high parts, FP32 Horner steps.
template <int D, class Ld>
__device__ __forceinline__ void q2_eval_f32(const Ld& ld, const float4* cell, const df t[D], df u[D]) {
  constexpr int NS = (D == 3 ? 3 : 1);
  constexpr int NF4 = qf_floats_per_comp<D>() / 4;  // float4 per component
  float s[D];
#pragma unroll
  for (int a = 0; a < D; ++a) s[a] = t[a].hi - 0.5f;
#pragma unroll
  for (int comp = 0; comp < D; ++comp) {
    float c[4 * NF4];
#pragma unroll
    for (int k = 0; k < NF4; ++k) {
      const float4 v = ld.ld(cell + comp * NF4 + k);
      c[4 * k] = v.x;
      c[4 * k + 1] = v.y;
      c[4 * k + 2] = v.z;
      c[4 * k + 3] = v.w;
    }
    float g[NS];
#pragma unroll
    for (int r = 0; r < NS; ++r) {
      float h[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) h[q] = fmaf(fmaf(c[9 * r + 3 * q + 2], s[0], c[9 * r + 3 * q + 1]), s[0], c[9 * r + 3 * q]);
      g[r] = fmaf(fmaf(h[2], s[1], h[1]), s[1], h[0]);
    }
    const df rr = df_make((D == 3) ? fmaf(fmaf(g[2], s[2], g[1]), s[2], g[0]) : g[0], 0.f);
    // constant indices keep u in registers under a rolled loop
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (a == comp) u[a] = rr;
  }
}

}  // namespace pic
