// advect.cu -- particle advection with located stages (Sec. 2.3 and 2.4 of
// Gassmoeller et al., arXiv 1612.03369), stand-alone relocation and
// stateless point location.
//
// One thread per particle, grid-stride over the store, which is sorted by
// (cell, id): neighbouring threads share a cell, so the vertex and Q2 node
// loads of a warp hit the same lines in L1.
#include <cmath>

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

// Velocity at double-float reference coordinates t of cell K: the Q2
// contraction in double-float, or in FP32 for the precision form.
template <int D, bool F32B>
__device__ __forceinline__ void velocity(const MeshView& m, uint32_t K, const df t[D], df u[D]) {
  if constexpr (F32B)
    q2_eval_f32<D>(m, K, t, u);
  else
    q2_eval_df<D>(m, K, t, u);
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
  __device__ static float c(int) { return 0.f; }
  __device__ static float w(int) { return 1.f; }
  __device__ static bool divide6() { return false; }
};
template <>
struct Tableau<2> {  // midpoint rule
  static constexpr int S = 2;
  __device__ static float c(int p) { return 0.5f; }  // y_1 = x + k_0 / 2
  __device__ static float w(int p) { return p == 0 ? 0.f : 1.f; }
  __device__ static bool divide6() { return false; }
};
template <>
struct Tableau<4> {  // classical RK4: y_1 = x + k0/2, y_2 = x + k1/2, y_3 = x + k2
  static constexpr int S = 4;
  __device__ static float c(int p) { return p == 3 ? 1.f : 0.5f; }
  __device__ static float w(int p) { return (p == 0 || p == 3) ? 1.f : 2.f; }  // then / 6
  __device__ static bool divide6() { return true; }
};

// Resident blocks per SM requested from the register allocator (tuning knob,
// swept at build time with -DPIC_ADVECT_MIN_BLOCKS=n).
#ifndef PIC_ADVECT_MIN_BLOCKS
#define PIC_ADVECT_MIN_BLOCKS 5
#endif

template <int D, int RK, bool F32B>
__global__ void __launch_bounds__(128, PIC_ADVECT_MIN_BLOCKS) advect_kernel(MeshView m, StoreView s, df dt, uint32_t* __restrict__ cell_new,
                                                     uint32_t* __restrict__ counts, DevCounters* __restrict__ ctr) {
  using TB = Tableau<RK>;
  const uint32_t n = ctr->n_alive;
  const uint32_t stride = gridDim.x * blockDim.x;
  const df sixth = df_make(0.16666667163372039795f, -4.967053879312289e-09f);  // 1/6 = hi + lo
  for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += stride) {
    const uint32_t i = base + threadIdx.x;
    int iters = 0;
    unsigned flags = 0, lost = 0, steps = 0;
    if (i < n) {
      steps = 1;
      uint32_t Ks = s.cell[i];
      uint32_t Kn = PIC_LOST;
      if (Ks >= m.C) {
        flags |= kFlagBounds;
      } else {
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
        bool ok = true;
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
            Ks = locate_df<D>(m, y, Ks, hint, ts, iters, flags, !F32B || p == TB::S);
            if (Ks == PIC_LOST) {
              ok = false;
              break;
            }
            if (p == TB::S) break;
          }
          df u[D];
          velocity<D, F32B>(m, Ks, ts, u);
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
        if (ok) {
          Kn = Ks;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            s.x[a * s.cap + i] = (x[a] + (double)acc[a].hi) + (double)acc[a].lo;
            s.xhat[a * s.cap + i] = make_float2(ts[a].hi, ts[a].lo);
          }
        }
      }
      cell_new[i] = Kn;
      if (Kn != PIC_LOST)
        atomicAdd(counts + Kn, 1u);
      else
        lost = 1;
    }
    flush_counters(ctr, steps, iters, lost, (flags & kFlagWalk) ? 1u : 0u, (flags & kFlagGlobal) ? 1u : 0u, flags);
  }
}

// Relocate every particle at its current x (hint: its current cell).
template <int D>
__global__ void __launch_bounds__(128) relocate_kernel(MeshView m, StoreView s, uint32_t* __restrict__ cell_new,
                                                       uint32_t* __restrict__ counts, DevCounters* __restrict__ ctr) {
  const uint32_t n = ctr->n_alive;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += stride) {
    const uint32_t i = base + threadIdx.x;
    int iters = 0;
    unsigned flags = 0, lost = 0;
    if (i < n) {
      df y[D], tn[D];
      float hint[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        y[a] = df_from_double(s.x[a * s.cap + i]);
        hint[a] = s.xhat[a * s.cap + i].x;
      }
      const uint32_t Kn = locate_df<D>(m, y, s.cell[i], hint, tn, iters, flags);
      if (Kn != PIC_LOST) {
#pragma unroll
        for (int a = 0; a < D; ++a) s.xhat[a * s.cap + i] = make_float2(tn[a].hi, tn[a].lo);
        atomicAdd(counts + Kn, 1u);
      } else {
        lost = 1;
      }
      cell_new[i] = Kn;
    }
    flush_counters(ctr, 0, iters, lost, (flags & kFlagWalk) ? 1 : 0, (flags & kFlagGlobal) ? 1 : 0, flags);
  }
}

// Stateless location of n points.  Without hints, the start cell is the
// point's cell in a uniform background grid over the mesh's bounding box.
template <int D>
__global__ void __launch_bounds__(128) locate_points_kernel(MeshView m, size_t n, const double* __restrict__ x,
                                                            const uint32_t* __restrict__ hint, uint32_t* __restrict__ cell_out,
                                                            double* __restrict__ xhat_out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double y[D], t0[D], t[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      y[a] = x[a * n + i];
      t0[a] = 0.5;
    }
    uint32_t h;
    if (hint) {
      h = hint[i];
    } else {
      int g[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) {
        double f = (y[a] - m.dlo[a]) / (m.dhi[a] - m.dlo[a]) * (double)m.n[a];
        f = isfinite(f) ? f : 0.0;
        int gi = (int)fmin(fmax(floor(f), 0.0), (double)(m.n[a] - 1));
        g[a] = gi;
      }
      h = cell_index<D>(m, g[0], g[1], g[2]);
    }
    int iters = 0;
    unsigned flags = 0;
    const uint32_t K = locate<D>(m, y, h, t0, t, iters, flags);
    cell_out[i] = K;
#pragma unroll
    for (int a = 0; a < D; ++a) xhat_out[a * n + i] = (K == PIC_LOST) ? 0.0 : t[a];
  }
}

static int grid_for(size_t n, int block) {
  const size_t want = (n + block - 1) / block;
  const size_t cap = (size_t)num_sms() * 16;
  size_t g = want < cap ? want : cap;
  return (int)(g > 0 ? g : 1);
}

template <int D, int RK, bool F32B>
static void launch_advect(pic_particles_s* p, const MeshView& m, double dt, cudaStream_t st) {
  const float hi = (float)dt;
  const df dtd = {hi, (float)(dt - (double)hi)};
  advect_kernel<D, RK, F32B><<<grid_for(p->capacity, 128), 128, 0, st>>>(m, store_view(p, p->cur), dtd, p->cell_new,
                                                                         p->counts, p->ctr);
  count_launches(1);
}

// Three events per timed step (before advect, after advect, after rebin),
// created on first use and kept with the handle.
static cudaEvent_t* timing_slot(pic_particles_s* p) {
  if (p->n_ev == p->ev_cap) {
    const int cap = p->ev_cap ? 2 * p->ev_cap : 64;
    cudaEvent_t* ev = (cudaEvent_t*)realloc(p->ev, sizeof(cudaEvent_t) * 3 * cap);
    if (!ev) return nullptr;
    for (int k = 3 * p->ev_cap; k < 3 * cap; ++k)
      if (cudaEventCreate(&ev[k]) != cudaSuccess) return nullptr;
    p->ev = ev;
    p->ev_cap = cap;
  }
  return p->ev + 3 * (p->n_ev++);
}

template <int D, bool F32B>
static void launch_advect_rk(pic_particles_s* p, const MeshView& m, double dt, int rk, cudaStream_t st) {
  if (rk == 1)
    launch_advect<D, 1, F32B>(p, m, dt, st);
  else if (rk == 2)
    launch_advect<D, 2, F32B>(p, m, dt, st);
  else
    launch_advect<D, 4, F32B>(p, m, dt, st);
}

}  // namespace pic

using namespace pic;

extern "C" pic_status pic_advect(pic_particles parts, pic_mesh mesh, double dt, pic_integrator integrator,
                                 pic_precision precision, int n_steps, void* stream) {
  if (!parts || !mesh) return (set_error("pic_advect: null handle"), PIC_ERR_ARG);
  if (parts->mesh != mesh || parts->dim != mesh->dim) return (set_error("pic_advect: mesh mismatch"), PIC_ERR_ARG);
  if (!std::isfinite(dt)) return (set_error("pic_advect: dt not finite"), PIC_ERR_ARG);
  if (n_steps < 0) return (set_error("pic_advect: n_steps < 0"), PIC_ERR_ARG);
  if (integrator != PIC_EULER && integrator != PIC_RK2 && integrator != PIC_RK4)
    return (set_error("pic_advect: unknown integrator %d", (int)integrator), PIC_ERR_ARG);
  if (precision != PIC_FP64 && precision != PIC_FP32_BASIS)
    return (set_error("pic_advect: unknown precision %d", (int)precision), PIC_ERR_ARG);
  if (!mesh->has_velocity) return (set_error("pic_advect: velocity not set"), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  const MeshView m = mesh_view(mesh);
  for (int step = 0; step < n_steps; ++step) {
    PIC_CUDA(cudaMemsetAsync(parts->counts, 0, sizeof(uint32_t) * parts->C, st));
    cudaEvent_t* ev = parts->timing ? timing_slot(parts) : nullptr;
    if (ev) PIC_CUDA(cudaEventRecord(ev[0], st));
    const bool f32 = precision == PIC_FP32_BASIS;
    if (mesh->dim == 2) {
      if (f32)
        launch_advect_rk<2, true>(parts, m, dt, (int)integrator, st);
      else
        launch_advect_rk<2, false>(parts, m, dt, (int)integrator, st);
    } else {
      if (f32)
        launch_advect_rk<3, true>(parts, m, dt, (int)integrator, st);
      else
        launch_advect_rk<3, false>(parts, m, dt, (int)integrator, st);
    }
    PIC_CUDA(cudaGetLastError());
    if (ev) PIC_CUDA(cudaEventRecord(ev[1], st));
    pic_status r = rebin_from_counts(parts, st);
    if (r != PIC_OK) return r;
    if (ev) PIC_CUDA(cudaEventRecord(ev[2], st));
  }
  return PIC_OK;
}

extern "C" pic_status pic_locate(pic_particles parts, pic_mesh mesh, void* stream) {
  if (!parts || !mesh) return (set_error("pic_locate: null handle"), PIC_ERR_ARG);
  if (parts->mesh != mesh) return (set_error("pic_locate: mesh mismatch"), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  const MeshView m = mesh_view(mesh);
  PIC_CUDA(cudaMemsetAsync(parts->counts, 0, sizeof(uint32_t) * parts->C, st));
  if (mesh->dim == 2)
    relocate_kernel<2><<<grid_for(parts->capacity, 128), 128, 0, st>>>(m, store_view(parts, parts->cur),
                                                                       parts->cell_new, parts->counts, parts->ctr);
  else
    relocate_kernel<3><<<grid_for(parts->capacity, 128), 128, 0, st>>>(m, store_view(parts, parts->cur),
                                                                       parts->cell_new, parts->counts, parts->ctr);
  count_launches(1);
  PIC_CUDA(cudaGetLastError());
  return rebin_from_counts(parts, st);
}

extern "C" pic_status pic_locate_points(pic_mesh mesh, size_t n, const double* x, const uint32_t* hint,
                                        uint32_t* cell_out, double* xhat_out, void* stream) {
  if (!mesh) return (set_error("pic_locate_points: null mesh"), PIC_ERR_ARG);
  if (n == 0) return PIC_OK;
  if (!x || !cell_out || !xhat_out) return (set_error("pic_locate_points: null array"), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  const MeshView m = mesh_view(mesh);
  if (mesh->dim == 2)
    locate_points_kernel<2><<<grid_for(n, 128), 128, 0, st>>>(m, n, x, hint, cell_out, xhat_out);
  else
    locate_points_kernel<3><<<grid_for(n, 128), 128, 0, st>>>(m, n, x, hint, cell_out, xhat_out);
  count_launches(1);
  PIC_CUDA(cudaGetLastError());
  return PIC_OK;
}
