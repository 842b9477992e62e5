// props.cu -- property ODEs integrated along the particle paths (Sec. 2.6 of
// Gassmoeller et al., arXiv 1612.03369):
//   damage              d' = alpha |eps-dot(u)| - beta d,  eps-dot = (G + G^T)/2
//   deformation gradient F' = G F,                         G = grad u_h
// with |.| the Frobenius norm.  The properties and the position form one
// system z = (x, d, F) stepped by the same RK tableau over the same located
// stage points.  Each time step runs in three kernels:
//   1. the particle step of pic_advect (the same advect_particle, so
//      positions, cells and order are those of pic_advect bit for bit),
//      recording every stage's (cell, x-hat);
//   2. G = grad u_h at every recorded stage point, thread per (stage,
//      particle), in double-float on the FP32 pipe;
//   3. the ODEs over the stages with those G, in double-float.
// Kept apart, each kernel fits the instruction cache (one kernel doing 2
// and 3 stalled on instruction fetch) and 2 runs without the ODE state live.
// Then the rebin carries the properties with the particles.  The stage
// records and gradients take 4 (4 + 8 dim + 8 dim^2) bytes per particle of
// scratch, allocated with the store on first use.
#include <cmath>

#include "advect.cuh"
#include "grad_df.cuh"
#include "rebin.cuh"

namespace pic {

struct OdeArgs {
  int damage;   // property slot of d, or -1
  int defgrad;  // first of D*D slots of F (row-major), or -1
  df alpha, beta;
};

// Phase 1: the particle step of pic_advect (the same advect_particle, so
// positions, cells and order are bit for bit those of pic_advect), leaving
// each stage's (cell, x-hat) behind.
template <int D, int RK>
__global__ void __launch_bounds__(128, PIC_ADVECT_MIN_BLOCKS) advect_record_kernel(const __grid_constant__ MeshView m, const __grid_constant__ StoreView s, df dt,
                                                                                  const __grid_constant__ StageRec rec,
                                                                                  uint32_t* __restrict__ cell_new,
                                                                                  uint32_t* __restrict__ counts,
                                                                                  DevCounters* __restrict__ ctr) {
  const uint32_t n = ctr->n_alive;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += stride) {
    const uint32_t i = base + threadIdx.x;
    int iters = 0;
    unsigned flags = 0, lost = 0, steps = 0;
    uint32_t Kc = PIC_LOST;  // the new cell to count
    if (i < n) {
      steps = 1;
      RecordHook hook{rec, i};
      const uint32_t Kn = advect_particle<D, RK, false, false>(m, s, i, s.cell[i], dt, iters, flags, hook);
      cell_new[i] = Kn;
      Kc = Kn;
      lost = Kn == PIC_LOST ? 1u : 0u;
    }
    (void)aggregated_increment(counts, Kc, Kc != PIC_LOST);
    flush_counters(ctr, steps, iters, lost, (flags & kFlagWalk) ? 1u : 0u, (flags & kFlagGlobal) ? 1u : 0u, flags);
  }
}

// Phase 2, thread per (stage, surviving particle): G_p = grad u_h at the
// recorded stage point, in double-float, stored as G[(p D^2 + e) cap + i].
// A kernel of its own, so that neither it nor the ODE kernel outgrows the
// instruction cache.
template <int D>
__global__ void __launch_bounds__(128, 4) props_grad_kernel(const __grid_constant__ MeshView m, const __grid_constant__ StageRec rec, int S,
                                                           const uint32_t* __restrict__ cell_new,
                                                           const DevCounters* __restrict__ ctr,
                                                           float2* __restrict__ Gs) {
  const uint32_t n = ctr->n_alive;
  const size_t items = (size_t)S * n;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < items; k += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(k / n);
    const uint32_t i = (uint32_t)(k - (size_t)p * n);
    if (cell_new[i] == PIC_LOST) continue;
    const uint32_t K = rec.cell[(size_t)p * rec.cap + i];
    if (K >= m.C) continue;  // cannot happen for a survivor
    df t[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const float2 v = rec.t[((size_t)a * 4 + p) * rec.cap + i];
      t[a] = df_make(v.x, v.y);
    }
    df G[D][D];
    velocity_gradient_df<D>(m, K, t, G);
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int q = 0; q < D; ++q) Gs[((size_t)p * D * D + r * D + q) * rec.cap + i] = make_float2(G[r][q].hi, G[r][q].lo);
  }
}

// Phase 3, thread per surviving particle: the property ODEs over the recorded
// stages, in double-float.  For stage p: z_p = z + c_p k_{p-1},
// k_p = dt f(G_p, z_p), and z' = z + sum_p w_p k_p (/ 6 for RK4), with
//   f_d = alpha |(G + G^T)/2|_F - beta d,   f_F = G F.
// Resident blocks per SM requested from the register allocator (swept at
// build time with -DPIC_PROPS_MIN_BLOCKS=n).
#ifndef PIC_PROPS_MIN_BLOCKS
#define PIC_PROPS_MIN_BLOCKS 4
#endif

template <int D, int RK>
__global__ void __launch_bounds__(128, PIC_PROPS_MIN_BLOCKS) props_ode_kernel(const __grid_constant__ StoreView s, df dt, OdeArgs o,
                                                                              const float2* __restrict__ Gs,
                                                                              const uint32_t* __restrict__ cell_new,
                                                                              const DevCounters* __restrict__ ctr) {
  using TB = Tableau<RK>;
  constexpr int NZ = 1 + D * D;  // z = (d, F_00, F_01, ...)
  const df sixth = df_make(0.16666667163372039795f, -4.967053879312289e-09f);
  const uint32_t n = ctr->n_alive;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (cell_new[i] == PIC_LOST) continue;
    df z[NZ], k[NZ], acc[NZ];
    z[0] = o.damage >= 0 ? df_from_double(s.props[(size_t)o.damage * s.cap + i]) : df_make(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < D * D; ++q)
      z[1 + q] = o.defgrad >= 0 ? df_from_double(s.props[(size_t)(o.defgrad + q) * s.cap + i]) : df_make(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < NZ; ++q) k[q] = acc[q] = df_make(0.f, 0.f);
#pragma unroll 1
    for (int p = 0; p < TB::S; ++p) {
      df G[D][D];
#pragma unroll
      for (int r = 0; r < D; ++r)
#pragma unroll
        for (int q = 0; q < D; ++q) {
          const float2 v = Gs[((size_t)p * D * D + r * D + q) * s.cap + i];
          G[r][q] = df_make(v.x, v.y);
        }
      const float c = p == 0 ? 0.f : TB::c(p);
      df zs[NZ];
#pragma unroll
      for (int q = 0; q < NZ; ++q) zs[q] = p == 0 ? z[q] : df_add(z[q], df_scale2(k[q], c));
      df f[NZ];
      f[0] = df_make(0.f, 0.f);
      if (o.damage >= 0) {
        df_acc e2 = acc_zero();
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int q = 0; q < D; ++q) {
            const df e = df_scale2(df_add(G[r][q], G[q][r]), 0.5f);
            acc_mad(e2, e, e);
          }
        df_acc fd = acc_zero();
        acc_mad(fd, o.alpha, df_sqrt(acc_result(e2)));
        acc_mad(fd, df_make(-o.beta.hi, -o.beta.lo), zs[0]);
        f[0] = acc_result(fd);
      }
#pragma unroll
      for (int r = 0; r < D; ++r)
#pragma unroll
        for (int q = 0; q < D; ++q) {
          df_acc a = acc_zero();
          if (o.defgrad >= 0) {
#pragma unroll
            for (int j = 0; j < D; ++j) acc_mad(a, G[r][j], zs[1 + j * D + q]);
          }
          f[1 + r * D + q] = acc_result(a);
        }
      const float w = TB::w(p);
#pragma unroll
      for (int q = 0; q < NZ; ++q) {
        k[q] = df_mul(dt, f[q]);
        if (w != 0.f) acc[q] = df_add(acc[q], df_scale2(k[q], w));
      }
    }
#pragma unroll
    for (int q = 0; q < NZ; ++q) {
      const df zn = df_add(z[q], TB::divide6() ? df_mul(acc[q], sixth) : acc[q]);
      if (q == 0) {
        if (o.damage >= 0) s.props[(size_t)o.damage * s.cap + i] = df_to_double(zn);
      } else if (o.defgrad >= 0) {
        s.props[(size_t)(o.defgrad + q - 1) * s.cap + i] = df_to_double(zn);
      }
    }
  }
}

// The stage gradients follow the stage records in the store's scratch.
static float2* stage_gradients(pic_particles_s* p) {
  return (float2*)((char*)p->stage_rec + (size_t)4 * p->capacity * (sizeof(uint32_t) + sizeof(float2) * p->dim));
}

static int props_grid(size_t n) {
  const size_t want = (n + 127) / 128;
  const size_t cap = (size_t)num_sms() * 16;
  const size_t g = want < cap ? want : cap;
  return (int)(g > 0 ? g : 1);
}

template <int D, int RK>
static void launch_props_rk(pic_particles_s* p, const MeshView& m, df dt, const OdeArgs& o, StageRec rec,
                            cudaStream_t st) {
  const StoreView s = store_view(p, p->cur);
  const int g = props_grid(p->capacity);
  float2* Gs = stage_gradients(p);
  advect_record_kernel<D, RK><<<g, 128, 0, st>>>(m, s, dt, rec, p->cell_new, p->counts, p->ctr);
  props_grad_kernel<D><<<props_grid((size_t)Tableau<RK>::S * p->capacity), 128, 0, st>>>(m, rec, Tableau<RK>::S,
                                                                                        p->cell_new, p->ctr, Gs);
  props_ode_kernel<D, RK><<<g, 128, 0, st>>>(s, dt, o, Gs, p->cell_new, p->ctr);
  count_launches(3);
}

template <int D>
static void launch_props(pic_particles_s* p, const MeshView& m, double dt, int rk, const OdeArgs& o, StageRec rec,
                         cudaStream_t st) {
  const float hi = (float)dt;
  const df dtd = {hi, (float)(dt - (double)hi)};
  if (rk == 1)
    launch_props_rk<D, 1>(p, m, dtd, o, rec, st);
  else if (rk == 2)
    launch_props_rk<D, 2>(p, m, dtd, o, rec, st);
  else
    launch_props_rk<D, 4>(p, m, dtd, o, rec, st);
}

template <int D>
static void launch_record_d(pic_particles_s* p, const MeshView& m, df dt, int rk, const StageRec& rec,
                            cudaStream_t st) {
  const StoreView s = store_view(p, p->cur);
  const int g = props_grid(p->capacity);
  if (rk == 1)
    advect_record_kernel<D, 1><<<g, 128, 0, st>>>(m, s, dt, rec, p->cell_new, p->counts, p->ctr);
  else if (rk == 2)
    advect_record_kernel<D, 2><<<g, 128, 0, st>>>(m, s, dt, rec, p->cell_new, p->counts, p->ctr);
  else
    advect_record_kernel<D, 4><<<g, 128, 0, st>>>(m, s, dt, rec, p->cell_new, p->counts, p->ctr);
  count_launches(1);
}

void launch_advect_record(pic_particles_s* p, const MeshView& m, double dt, int rk, const StageRec& rec,
                          cudaStream_t st) {
  const float hi = (float)dt;
  const df dtd = {hi, (float)(dt - (double)hi)};
  if (p->dim == 2)
    launch_record_d<2>(p, m, dtd, rk, rec, st);
  else
    launch_record_d<3>(p, m, dtd, rk, rec, st);
}

}  // namespace pic

using namespace pic;

extern "C" pic_status pic_advect_properties(pic_particles parts, pic_mesh mesh, double dt, pic_integrator integrator,
                                            int n_steps, const pic_property_odes* odes, void* stream) {
  if (!parts || !mesh || !odes) return (set_error("pic_advect_properties: null argument"), PIC_ERR_ARG);
  if (parts->mesh != mesh || parts->dim != mesh->dim)
    return (set_error("pic_advect_properties: mesh mismatch"), PIC_ERR_ARG);
  if (!std::isfinite(dt)) return (set_error("pic_advect_properties: dt not finite"), PIC_ERR_ARG);
  if (n_steps < 0) return (set_error("pic_advect_properties: n_steps < 0"), PIC_ERR_ARG);
  if (integrator != PIC_EULER && integrator != PIC_RK2 && integrator != PIC_RK4)
    return (set_error("pic_advect_properties: unknown integrator %d", (int)integrator), PIC_ERR_ARG);
  if (!mesh->has_velocity) return (set_error("pic_advect_properties: velocity not set"), PIC_ERR_ARG);
  if (mesh->has_next)
    return (set_error("pic_advect_properties: a second velocity field is set; the property ODEs take the steady "
                      "field"),
            PIC_ERR_STATE);
  const int d = parts->dim, P = parts->n_props;
  if (odes->damage < -1 || odes->damage >= P)
    return (set_error("pic_advect_properties: damage slot %d outside [-1, %d)", odes->damage, P), PIC_ERR_ARG);
  if (odes->deformation < -1 || (odes->deformation >= 0 && odes->deformation + d * d > P))
    return (set_error("pic_advect_properties: deformation slots %d..%d outside the %d properties",
                      odes->deformation, odes->deformation + d * d - 1, P),
            PIC_ERR_ARG);
  if (odes->damage >= 0 && odes->deformation >= 0 && odes->damage >= odes->deformation &&
      odes->damage < odes->deformation + d * d)
    return (set_error("pic_advect_properties: damage slot overlaps the deformation slots"), PIC_ERR_ARG);
  if (odes->damage >= 0 && !(std::isfinite(odes->alpha) && std::isfinite(odes->beta)))
    return (set_error("pic_advect_properties: alpha, beta not finite"), PIC_ERR_ARG);
  auto split = [](double v) {
    const float hi = (float)v;
    return df{hi, (float)(v - (double)hi)};
  };
  const OdeArgs o = {odes->damage, odes->deformation, split(odes->alpha), split(odes->beta)};
  cudaStream_t st = (cudaStream_t)stream;
  {
    const pic_status r0 = settle_order(parts, st);
    if (r0 != PIC_OK) return r0;
  }
  const MeshView m = mesh_view(mesh);
  if (!parts->stage_rec) {
    const size_t bytes = (size_t)4 * parts->capacity * (sizeof(uint32_t) + sizeof(float2) * d + sizeof(float2) * d * d);
    if (cudaMalloc(&parts->stage_rec, bytes) != cudaSuccess) {
      cudaGetLastError();
      parts->stage_rec = nullptr;
      return (set_error("pic_advect_properties: cannot allocate %zu bytes of stage records and gradients", bytes),
              PIC_ERR_OOM);
    }
  }
  const StageRec rec = {(uint32_t*)parts->stage_rec,
                        (float2*)((char*)parts->stage_rec + (size_t)4 * parts->capacity * sizeof(uint32_t)),
                        parts->capacity};
  for (int step = 0; step < n_steps; ++step) {
    PIC_CUDA(cudaMemsetAsync(parts->counts, 0, sizeof(uint32_t) * parts->C, st));
    if (d == 2)
      launch_props<2>(parts, m, dt, (int)integrator, o, rec, st);
    else
      launch_props<3>(parts, m, dt, (int)integrator, o, rec, st);
    PIC_CUDA(cudaGetLastError());
    pic_status r = rebin_from_counts(parts, st);
    if (r != PIC_OK) return r;
  }
  return PIC_OK;
}
