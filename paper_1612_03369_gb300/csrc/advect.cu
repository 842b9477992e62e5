// advect.cu -- particle advection with located stages (Sec. 2.3 and 2.4 of
// Gassmoeller et al., arXiv 1612.03369), stand-alone relocation and
// stateless point location.
//
// One thread per particle, grid-stride over the store, which is sorted by
// (cell, id): neighbouring threads share a cell, so the vertex and Q2 node
// loads of a warp hit the same lines in L1.
#include <cmath>

#include "advect.cuh"
#include "rebin.cuh"

namespace pic {

template <int D, int RK, bool F32B, bool TWO>
__global__ void __launch_bounds__(128, PIC_ADVECT_MIN_BLOCKS) advect_kernel(MeshView m, StoreView s, StoreView d,
                                                                          const uint32_t* __restrict__ perm, df dt,
                                                                          uint32_t* __restrict__ cell_new,
                                                                          uint32_t* __restrict__ counts,
                                                                          DevCounters* __restrict__ ctr) {
  // perm == nullptr: particle j of s advances in place (d is s).  Otherwise
  // the previous step's reordering is applied on the way: slot j of d takes
  // particle perm[j] of s (its cell is already in d.cell[j], written by the
  // previous rebin), with its id and properties.
  const uint32_t n = ctr->n_alive;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += stride) {
    const uint32_t j = base + threadIdx.x;
    int iters = 0;
    unsigned flags = 0, lost = 0, steps = 0;
    uint32_t Kc = PIC_LOST;  // the new cell to count
    if (j < n) {
      steps = 1;
      uint32_t i = j, K;
      if (perm) {
        i = perm[j];
        K = d.cell[j];
        if (i >= s.cap) {
          flags |= kFlagBounds;
          K = PIC_LOST;
          i = 0;
        } else {
          d.id[j] = s.id[i];
          for (int q = 0; q < s.n_props; ++q) d.props[(size_t)q * d.cap + j] = s.props[(size_t)q * s.cap + i];
        }
      } else {
        K = s.cell[j];
      }
      const uint32_t Kn = advect_particle_to<D, RK, F32B, TWO>(m, s, i, d, j, K, dt, iters, flags);
      cell_new[j] = Kn;
      Kc = Kn;
      lost = Kn == PIC_LOST ? 1u : 0u;
    }
    (void)aggregated_increment(counts, Kc, Kc != PIC_LOST);
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

// One advect launch.  With `fused` the previous step's reordering (perm,
// sorted cells in the other buffer) is applied on the way: the step reads
// buffer cur and writes buffer 1 - cur, which becomes cur.
template <int D, int RK, bool F32B>
static void launch_advect(pic_particles_s* p, const MeshView& m, double dt, bool fused, cudaStream_t st) {
  const float hi = (float)dt;
  const df dtd = {hi, (float)(dt - (double)hi)};
  const StoreView s = store_view(p, p->cur), d = fused ? store_view(p, 1 - p->cur) : s;
  const uint32_t* perm = fused ? p->perm : nullptr;
  if (m.has_next)
    advect_kernel<D, RK, F32B, true><<<grid_for(p->capacity, 128), 128, 0, st>>>(m, s, d, perm, dtd, p->cell_new,
                                                                                 p->counts, p->ctr);
  else
    advect_kernel<D, RK, F32B, false><<<grid_for(p->capacity, 128), 128, 0, st>>>(m, s, d, perm, dtd, p->cell_new,
                                                                                  p->counts, p->ctr);
  count_launches(1);
  if (fused) p->cur = 1 - p->cur;
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
static void launch_advect_rk(pic_particles_s* p, const MeshView& m, double dt, int rk, bool fused, cudaStream_t st) {
  if (rk == 1)
    launch_advect<D, 1, F32B>(p, m, dt, fused, st);
  else if (rk == 2)
    launch_advect<D, 2, F32B>(p, m, dt, fused, st);
  else
    launch_advect<D, 4, F32B>(p, m, dt, fused, st);
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
  // Each step's rebin computes the new order (perm, sorted cells); the
  // particles themselves move with the next step's advect, which reads them
  // through perm, and after the last step with one gather.  Every step thus
  // reads and writes the particle state once instead of twice.
  bool pending = false;
  for (int step = 0; step < n_steps; ++step) {
    PIC_CUDA(cudaMemsetAsync(parts->counts, 0, sizeof(uint32_t) * parts->C, st));
    cudaEvent_t* ev = parts->timing ? timing_slot(parts) : nullptr;
    if (ev) PIC_CUDA(cudaEventRecord(ev[0], st));
    const bool f32 = precision == PIC_FP32_BASIS;
    if (mesh->dim == 2) {
      if (f32)
        launch_advect_rk<2, true>(parts, m, dt, (int)integrator, pending, st);
      else
        launch_advect_rk<2, false>(parts, m, dt, (int)integrator, pending, st);
    } else {
      if (f32)
        launch_advect_rk<3, true>(parts, m, dt, (int)integrator, pending, st);
      else
        launch_advect_rk<3, false>(parts, m, dt, (int)integrator, pending, st);
    }
    PIC_CUDA(cudaGetLastError());
    if (ev) PIC_CUDA(cudaEventRecord(ev[1], st));
    pic_status r = rebin_order_from_counts(parts, st);
    if (r != PIC_OK) return r;
    pending = true;
    if (step + 1 == n_steps) {
      r = rebin_apply_order(parts, st);
      if (r != PIC_OK) return r;
      pending = false;
    }
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
