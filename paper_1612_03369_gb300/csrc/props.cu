// props.cu -- property ODEs integrated along the particle paths (Sec. 2.6 of
// Gassmoeller et al., arXiv 1612.03369):
//   damage              d' = alpha |eps-dot(u)| - beta d,  eps-dot = (G + G^T)/2
//   deformation gradient F' = G F,                         G = grad u_h
// with |.| the Frobenius norm.  The properties and the position form one
// system z = (x, d, F) stepped by the same RK tableau over the same located
// stage points: the position part runs through advect_particle unchanged
// (double-float stages, the same locate), so positions and cells are those
// of pic_advect bit for bit, and at every stage an OdeHook evaluates G (in
// double-float on the FP32 pipe, handed back in FP64) at the stage's
// (cell, x-hat) and advances its own stage values in FP64.
#include <cmath>

#include "advect.cuh"
#include "grad_df.cuh"

namespace pic {

struct OdeArgs {
  int damage;   // property slot of d, or -1
  int defgrad;  // first of D*D slots of F (row-major), or -1
  double alpha, beta;
};

template <int D, int RK>
struct OdeHook {
  static constexpr int NZ = 1 + D * D;  // z = (d, F_00, F_01, ...)
  const MeshView& m;
  const double dt;
  const OdeArgs& o;
  double z[NZ], k[NZ], acc[NZ];

  __device__ __forceinline__ OdeHook(const MeshView& m_, const StoreView& s, uint32_t i, double dt_,
                                     const OdeArgs& o_)
      : m(m_), dt(dt_), o(o_) {
    z[0] = o.damage >= 0 ? s.props[(size_t)o.damage * s.cap + i] : 0.0;
#pragma unroll
    for (int q = 0; q < D * D; ++q) z[1 + q] = o.defgrad >= 0 ? s.props[(size_t)(o.defgrad + q) * s.cap + i] : 0.0;
#pragma unroll
    for (int q = 0; q < NZ; ++q) k[q] = acc[q] = 0.0;
  }

  // Evaluation point p: stage value z_p = z + c_p k_{p-1}, increment
  // k_p = dt f(z_p) with f from G at the located stage point.
  template <int DD>
  __device__ __forceinline__ void stage(int p, uint32_t K, const df* t) {
    using TB = Tableau<RK>;
    const double c = p == 0 ? 0.0 : (double)TB::c(p);
    double zs[NZ];
#pragma unroll
    for (int q = 0; q < NZ; ++q) zs[q] = p == 0 ? z[q] : z[q] + c * k[q];
    double G[D][D];
    velocity_gradient_df<D>(m, K, t, G);
    double f[NZ];
    f[0] = 0.0;
    if (o.damage >= 0) {
      double s = 0.0;
#pragma unroll
      for (int r = 0; r < D; ++r)
#pragma unroll
        for (int q = 0; q < D; ++q) {
          const double e = 0.5 * (G[r][q] + G[q][r]);
          s += e * e;
        }
      f[0] = o.alpha * sqrt(s) - o.beta * zs[0];
    }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int q = 0; q < D; ++q) {
        double a = 0.0;
        if (o.defgrad >= 0) {
#pragma unroll
          for (int j = 0; j < D; ++j) a += G[r][j] * zs[1 + j * D + q];
        }
        f[1 + r * D + q] = a;
      }
    const double w = (double)TB::w(p);
#pragma unroll
    for (int q = 0; q < NZ; ++q) {
      k[q] = dt * f[q];
      if (w != 0.0) acc[q] += w * k[q];
    }
  }

  // z_{n+1} = z + sum_s b_s k_s, written to the enabled slots.
  __device__ __forceinline__ void finish(const StoreView& s, uint32_t i) const {
    using TB = Tableau<RK>;
    double zn[NZ];
#pragma unroll
    for (int q = 0; q < NZ; ++q) zn[q] = TB::divide6() ? z[q] + acc[q] / 6.0 : z[q] + acc[q];
    if (o.damage >= 0) s.props[(size_t)o.damage * s.cap + i] = zn[0];
    if (o.defgrad >= 0) {
#pragma unroll
      for (int q = 0; q < D * D; ++q) s.props[(size_t)(o.defgrad + q) * s.cap + i] = zn[1 + q];
    }
  }
};

// Resident blocks per SM requested from the register allocator (swept at
// build time with -DPIC_PROPS_MIN_BLOCKS=n).
#ifndef PIC_PROPS_MIN_BLOCKS
#define PIC_PROPS_MIN_BLOCKS 6
#endif

template <int D, int RK>
__global__ void __launch_bounds__(128, PIC_PROPS_MIN_BLOCKS) advect_props_kernel(MeshView m, StoreView s, df dt, double dt64, OdeArgs o,
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
      OdeHook<D, RK> hook(m, s, i, dt64, o);
      const uint32_t Kn = advect_particle<D, RK, false, false>(m, s, i, s.cell[i], dt, iters, flags, hook);
      cell_new[i] = Kn;
      if (Kn != PIC_LOST) {
        hook.finish(s, i);
        atomicAdd(counts + Kn, 1u);
      } else {
        lost = 1;
      }
    }
    flush_counters(ctr, steps, iters, lost, (flags & kFlagWalk) ? 1u : 0u, (flags & kFlagGlobal) ? 1u : 0u, flags);
  }
}

static int props_grid(size_t n) {
  const size_t want = (n + 127) / 128;
  const size_t cap = (size_t)num_sms() * 16;
  const size_t g = want < cap ? want : cap;
  return (int)(g > 0 ? g : 1);
}

template <int D>
static void launch_props(pic_particles_s* p, const MeshView& m, double dt, int rk, const OdeArgs& o,
                         cudaStream_t st) {
  const float hi = (float)dt;
  const df dtd = {hi, (float)(dt - (double)hi)};
  const StoreView s = store_view(p, p->cur);
  const int g = props_grid(p->capacity);
  if (rk == 1)
    advect_props_kernel<D, 1><<<g, 128, 0, st>>>(m, s, dtd, dt, o, p->cell_new, p->counts, p->ctr);
  else if (rk == 2)
    advect_props_kernel<D, 2><<<g, 128, 0, st>>>(m, s, dtd, dt, o, p->cell_new, p->counts, p->ctr);
  else
    advect_props_kernel<D, 4><<<g, 128, 0, st>>>(m, s, dtd, dt, o, p->cell_new, p->counts, p->ctr);
  count_launches(1);
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
  const OdeArgs o = {odes->damage, odes->deformation, odes->alpha, odes->beta};
  cudaStream_t st = (cudaStream_t)stream;
  const MeshView m = mesh_view(mesh);
  for (int step = 0; step < n_steps; ++step) {
    PIC_CUDA(cudaMemsetAsync(parts->counts, 0, sizeof(uint32_t) * parts->C, st));
    if (d == 2)
      launch_props<2>(parts, m, dt, (int)integrator, o, st);
    else
      launch_props<3>(parts, m, dt, (int)integrator, o, st);
    PIC_CUDA(cudaGetLastError());
    pic_status r = rebin_from_counts(parts, st);
    if (r != PIC_OK) return r;
  }
  return PIC_OK;
}
