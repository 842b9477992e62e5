// advect.cuh -- one particle's time step with located stages (Sec. 2.3 and
// 2.4 of Gassmoeller et al., arXiv 1612.03369), shared by the single-mesh
// advect kernel and the ensemble kernels.
#pragma once

#include "fastpath.cuh"
#include "locate.cuh"
#include "pic_internal.cuh"

namespace pic {

// Warp-aggregated counter updates (one atomic per warp).
__device__ __forceinline__ void flush_counters(DevCounters* ctr, unsigned steps, int iters, unsigned lost,
                                               unsigned walks, unsigned globals, unsigned flags) {
  const unsigned mask = __activemask();
  const unsigned s = __reduce_add_sync(mask, steps);
  const unsigned it = __reduce_add_sync(mask, (unsigned)iters);
  const unsigned l = __reduce_add_sync(mask, lost);
  const unsigned w = __reduce_add_sync(mask, walks);
  const unsigned g = __reduce_add_sync(mask, globals);
  const unsigned f = __reduce_or_sync(mask, flags);
  const unsigned fb = __reduce_add_sync(mask, (flags & kFlagFallback64) ? 1u : 0u);
  const unsigned w64 = __reduce_add_sync(mask, (flags & kFlagWalk64) ? 1u : 0u);
  const int leader = __ffs(mask) - 1;
  if ((int)(threadIdx.x & 31) == leader) {
    if (s) atomicAdd(&ctr->particle_steps, (unsigned long long)s);
    if (it) atomicAdd(&ctr->newton_iterations, (unsigned long long)it);
    if (l) atomicAdd(&ctr->lost_total, (unsigned long long)l);
    if (w) atomicAdd(&ctr->walks, (unsigned long long)w);
    if (g) atomicAdd(&ctr->global_searches, (unsigned long long)g);
    if (fb) atomicAdd(&ctr->fallback64, (unsigned long long)fb);
    if (w64) atomicAdd(&ctr->walk64, (unsigned long long)w64);
    unsigned st = 0;
    if (f & kFlagNonConv) st |= PIC_STATUS_NEWTON_NONCONV;
    if (f & kFlagGlobal) st |= PIC_STATUS_GLOBAL_SEARCH;
    if (f & kFlagBounds) st |= PIC_STATUS_BOUNDS;
    if (st) atomicOr(&ctr->status, st);
  }
}

// u-tilde_h at double-float reference coordinates t of cell K and stage time
// t^n + theta dt, theta = 0, 1/2, 1 for tcode = 0, 1, 2: the steady field,
// or with a second field set, (1 - theta) u_h^n + theta u_h^{n+1} (reading
// of the time interpolation of Sec. 2.3; theta = 1/2 is the exact average).
// The Q2 evaluation (per-cell monomial form, Horner) is in double-float, or
// FP32 for the precision form; it sits in a rolled loop over the (one or two)
// fields so the kernel holds one copy of it.
template <int D, bool F32B, bool TWO, class Cells>
__device__ __forceinline__ void velocity(const Cells& cs, const MeshView& m, uint32_t K, const df t[D], int tcode,
                                         df u[D]) {
  if constexpr (!TWO) {
    if constexpr (F32B)
      q2_eval_f32<D>(cs, cs.coef(K), t, u);
    else
      q2_eval_df<D>(cs, cs.coef(K), t, u);
    return;
  } else {
    // the first field's blocks through the source, the second field's from
    // the mesh arrays
    constexpr int NQ = F32B ? qf_float4s<D>() : qc_float4s<D>();
    const GlobalCells<D, F32B> g{m};
    const float4* second = (F32B ? m.Qfn : m.Qcn) + (size_t)K * NQ;
    const bool two = m.has_next && tcode == 1;
    const bool only_next = m.has_next && tcode == 2;
#pragma unroll 1
    for (int f = 0; f < (two ? 2 : 1); ++f) {
      df v[D];
      if (f == 1 || only_next) {
        if constexpr (F32B)
          q2_eval_f32<D>(g, second, t, v);
        else
          q2_eval_df<D>(g, second, t, v);
      } else {
        if constexpr (F32B)
          q2_eval_f32<D>(cs, cs.coef(K), t, v);
        else
          q2_eval_df<D>(cs, cs.coef(K), t, v);
      }
#pragma unroll
      for (int a = 0; a < D; ++a) u[a] = (f == 0) ? v[a] : df_scale2(df_add(u[a], v[a]), 0.5f);
    }
  }
}

// One time step for every particle of the store (in place), recording the
// new owner cell in cell_new (PIC_LOST if a stage point or the new position
// lies in no cell) and counting particles per new cell.
//   Euler: x' = x + k1
//   RK2:   x' = x + dt u(x + k1/2)                            (midpoint)
//   RK4:   x' = x + (k1 + 2 k2 + 2 k3 + k4) / 6
// with k1 = dt u(x) taken at the stored (cell, x-hat), and every later stage
// point located before u_h is evaluated there (Sec. 2.4: every sub-step is
// followed by a determination of the containing cell).
//
// The stages run as one loop over evaluation points p = 0..S (S = number of
// stages): point 0 is the stored position, points 1..S-1 the stage points,
// point S the new position.  Each point p > 0 is located, each p < S gets a
// velocity evaluation, so the kernel holds one copy of the locate and of
// the Q2 contraction (instruction-cache footprint).
//
// Arithmetic: the stored position x is FP64; it is split once into a
// double-float, and the stages, the increments k_s and the stage points are
// double-floats on the FP32 pipe.  The new position is x + D in FP64, where
// D is the double-float increment; the new position is located from the
// double-float x + D (the two differ by ~1e-16).
template <int RK>
struct Tableau;
template <>
struct Tableau<1> {  // forward Euler
  static constexpr int S = 1;
  __device__ static int tcode(int) { return 0; }  // stage time: 0 -> t^n, 1 -> t^n + dt/2, 2 -> t^{n+1}
  __device__ static float c(int) { return 0.f; }
  __device__ static float w(int) { return 1.f; }
  __device__ static bool divide6() { return false; }
};
template <>
struct Tableau<2> {  // midpoint rule
  static constexpr int S = 2;
  __device__ static int tcode(int p) { return p == 0 ? 0 : 1; }
  __device__ static float c(int p) { return 0.5f; }  // y_1 = x + k_0 / 2
  __device__ static float w(int p) { return p == 0 ? 0.f : 1.f; }
  __device__ static bool divide6() { return false; }
};
template <>
struct Tableau<4> {  // classical RK4: y_1 = x + k0/2, y_2 = x + k1/2, y_3 = x + k2
  static constexpr int S = 4;
  __device__ static int tcode(int p) { return p == 0 ? 0 : (p == 3 ? 2 : 1); }
  __device__ static float c(int p) { return p == 3 ? 1.f : 0.5f; }
  __device__ static float w(int p) { return (p == 0 || p == 3) ? 1.f : 2.f; }  // then / 6
  __device__ static bool divide6() { return true; }
};

// Resident blocks per SM requested from the register allocator by the
// stage-recording and replay kernels, which inline the particle step (tuning
// knob, swept at build time with -DPIC_ADVECT_MIN_BLOCKS=n).  The step kernel
// and the ensemble kernels have their own knobs (advect.cu, ensemble.cu).
#ifndef PIC_ADVECT_MIN_BLOCKS
#define PIC_ADVECT_MIN_BLOCKS 6
#endif

// Per-stage work riding on the position integration: hook.stage(p, K, t) is
// called at every evaluation point p < S with its located cell and double-
// float reference coordinates.  The plain advection passes NoHook, which
// compiles to nothing.
struct NoHook {
  template <int D>
  __device__ __forceinline__ void stage(int, uint32_t, const df*) {}
};

// Writes stage p's cell and x-hat of the particle in slot i to the stage
// records (the StageRec layout).
struct RecordHook {
  StageRec r;
  uint32_t i;
  template <int D>
  __device__ __forceinline__ void stage(int p, uint32_t K, const df* t) {
    r.cell[(size_t)p * r.cap + i] = K;
#pragma unroll
    for (int a = 0; a < D; ++a) r.t[((size_t)a * 4 + p) * r.cap + i] = make_float2(t[a].hi, t[a].lo);
  }
};

// One time step of particle i of store s in mesh m, starting in cell K.
// TWO: the mesh carries a second field (time interpolation).
// Writes the new x and x-hat in place when the particle survives and returns
// its new cell, or PIC_LOST.
// advect_particle_cells reads particle i of store s and writes its new x and
// x-hat to slot j of store d (the same slot of the same store for the
// in-place step; another buffer when the step also applies the previous
// step's reordering), reading the cells' blocks from the source cs.
// kFast: the fast path only; returns kDefer (and writes nothing) where a
// rare path would be needed.
template <int D, int RK, bool F32B, bool TWO = false, class Hook = NoHook, bool kFast = false, class Cells>
__device__ __forceinline__ uint32_t advect_particle_cells(const Cells& cs, const MeshView& m, const StoreView& s,
                                                          uint32_t i, const StoreView& d, uint32_t j, uint32_t K,
                                                          df dt, int& iters, unsigned& flags, Hook&& hook = Hook()) {
  using TB = Tableau<RK>;
  const df sixth = df_make(0.16666667163372039795f, -4.967053879312289e-09f);  // 1/6 = hi + lo
  if (K >= m.C) {
    if constexpr (kFast) return kDefer;
    flags |= kFlagBounds;
    return PIC_LOST;
  }
  uint32_t Ks = K;
  double x[D];
  df xd[D], ts[D], k[D], acc[D], y[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    x[a] = s.x[a * s.cap + i];
    const float2 v = s.xhat[a * s.cap + i];
    ts[a] = df_make(v.x, v.y);
    xd[a] = df_from_double(x[a]);
    acc[a] = df_make(0.f, 0.f);
  }
#pragma unroll 1
  for (int p = 0; p <= TB::S; ++p) {
    if (p > 0) {
      float hint[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        hint[a] = ts[a].hi;
        y[a] = df_add(xd[a], p < TB::S ? df_scale2(k[a], TB::c(p)) : acc[a]);
      }
      // the FP32-basis form needs double-float x-hat only where it is stored
      // (unless the stage points are asked for it too)
      Ks = locate_df<D, kFast>(cs, m, y, Ks, hint, ts, iters, flags, !F32B || p == TB::S || m.stage_df);
      if (Ks == PIC_LOST) return PIC_LOST;
      if constexpr (kFast)
        if (Ks == kDefer) return kDefer;
      if (p == TB::S) break;
    }
    hook.template stage<D>(p, Ks, ts);
    df u[D];
    velocity<D, F32B, TWO>(cs, m, Ks, ts, TB::tcode(p), u);
    const float w = TB::w(p);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      k[a] = df_mul(dt, u[a]);
      if (w != 0.f) acc[a] = df_add(acc[a], df_scale2(k[a], w));
    }
    if (p == TB::S - 1 && TB::divide6()) {
#pragma unroll
      for (int a = 0; a < D; ++a) acc[a] = df_mul(acc[a], sixth);
    }
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    d.x[a * d.cap + j] = (x[a] + (double)acc[a].hi) + (double)acc[a].lo;
    d.xhat[a * d.cap + j] = make_float2(ts[a].hi, ts[a].lo);
  }
  return Ks;
}

// The same reading every block from the mesh arrays.
template <int D, int RK, bool F32B, bool TWO = false, class Hook = NoHook>
__device__ __forceinline__ uint32_t advect_particle_to(const MeshView& m, const StoreView& s, uint32_t i,
                                                       const StoreView& d, uint32_t j, uint32_t K, df dt, int& iters,
                                                       unsigned& flags, Hook&& hook = Hook()) {
  return advect_particle_cells<D, RK, F32B, TWO>(GlobalCells<D, F32B>{m}, m, s, i, d, j, K, dt, iters, flags,
                                                 static_cast<Hook&&>(hook));
}

template <int D, int RK, bool F32B, bool TWO = false, class Hook = NoHook>
__device__ __forceinline__ uint32_t advect_particle(const MeshView& m, const StoreView& s, uint32_t i, uint32_t K,
                                                    df dt, int& iters, unsigned& flags, Hook&& hook = Hook()) {
  return advect_particle_to<D, RK, F32B, TWO>(m, s, i, s, i, K, dt, iters, flags, static_cast<Hook&&>(hook));
}

// The full step of one particle (every rare path of the locate available),
// out of line: the fallback of a fast-path step that returned kDefer.  It
// re-reads the particle from s, so nothing of the abandoned fast step is
// kept.
struct FullStep {
  uint32_t K;
  int iters;
  unsigned flags;
};
template <int D, int RK, bool F32B, bool TWO>
__device__ __noinline__ FullStep advect_particle_full(const MeshView& m, const StoreView& s, uint32_t i,
                                                      const StoreView& d, uint32_t j, uint32_t K, df dt) {
  FullStep o;
  o.iters = 0;
  o.flags = 0;
  o.K = advect_particle_to<D, RK, F32B, TWO>(m, s, i, d, j, K, dt, o.iters, o.flags);
  return o;
}

}  // namespace pic
