// advect.cu -- particle advection with located stages (Sec. 2.3 and 2.4 of
// Gassmoeller et al., arXiv 1612.03369), stand-alone relocation and
// stateless point location.
//
// One thread per particle, grid-stride over the store, which is sorted by
// (cell, id): neighbouring threads share a cell, so the vertex and Q2 node
// loads of a warp hit the same lines in L1.
#include <cmath>

#include "advect.cuh"

namespace pic {

template <int D, int RK, bool F32B, bool TWO>
__global__ void __launch_bounds__(128, PIC_ADVECT_MIN_BLOCKS) advect_kernel(MeshView m, StoreView s, df dt,
                                                                          uint32_t* __restrict__ cell_new,
                                                                          uint32_t* __restrict__ counts,
                                                                          DevCounters* __restrict__ ctr) {
  const uint32_t n = ctr->n_alive;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += stride) {
    const uint32_t i = base + threadIdx.x;
    int iters = 0;
    unsigned flags = 0, lost = 0, steps = 0;
    if (i < n) {
      steps = 1;
      const uint32_t Kn = advect_particle<D, RK, F32B, TWO>(m, s, i, s.cell[i], dt, iters, flags);
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
  if (m.has_next)
    advect_kernel<D, RK, F32B, true><<<grid_for(p->capacity, 128), 128, 0, st>>>(m, store_view(p, p->cur), dtd,
                                                                                 p->cell_new, p->counts, p->ctr);
  else
    advect_kernel<D, RK, F32B, false><<<grid_for(p->capacity, 128), 128, 0, st>>>(m, store_view(p, p->cur), dtd,
                                                                                  p->cell_new, p->counts, p->ctr);
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
