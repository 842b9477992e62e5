// advect.cu -- particle advection with located stages (Sec. 2.3 and 2.4 of
// Gassmoeller et al., arXiv 1612.03369), stand-alone relocation and
// stateless point location.
//
// One thread per particle, grid-stride over the store, which is sorted by
// (cell, id): neighbouring threads share a cell, so the vertex and Q2 node
// loads of a warp hit the same lines in L1.
#include <cmath>

#include "advect.cuh"
#include "bulk.cuh"
#include "rebin.cuh"

namespace pic {

// ------------------------------------------------------ the step kernel --
// A persistent grid walks the (cell, id)-sorted store in warp tiles of 32
// particles, one particle per lane.  Warps take tiles from a work counter
// (one atomic per tile), two tiles ahead, so that warps that finish early
// take more and the grid ends together (a static split ran 13% slower).
//
// The kernel runs the fast path, which has no out-of-line calls, so the
// register allocation of the hot code carries no spill code around them: a
// particle whose fast path would enter a rare path (FP64 Newton, the
// lowest-index test across a nearby facet, the neighbour walk) is redone by
// advect_particle_full, called from the tile loop where few values are live.
// Both run the same arithmetic, so a particle's result does not depend on
// which ran it.  (With the rare paths called from inside the fast path the
// kernel spent 1.2x (FP64 form) to 1.5x (FP32-basis form) the time.)
//
// STAGE: each warp copies the map and coefficient blocks of the cells its
// tile starts in (at most kWarpStageCells) into its own slice of shared
// memory with one bulk copy per table (TMA, cp.async.bulk) counted on its own
// mbarrier, double-buffered (the copy for the warp's next tile is issued
// before the current tile is computed), and reads them from there; stage
// points that leave those cells read the mesh arrays.  Every wait on a copy
// is bounded (kStageWaitNs); if one runs out, the warp latches
// PIC_STATUS_TIMEOUT and reads the mesh arrays from then on.  Without STAGE
// the blocks are read through the read-only cache, where the ~20 particles of
// a cell find them; that is the faster of the two (the staged loads are
// generic, and the kernel is bound by instruction issue, not by the cell
// data's latency).
constexpr int kAdvectThreads = 128;
constexpr int kAdvectWarps = kAdvectThreads / 32;
constexpr int kWarpStageCells = 3;
constexpr unsigned long long kStageWaitNs = 2000000000ull;

template <int D, bool F32B>
struct StageLayout {
  static constexpr int NB = block_float4s<D>();
  static constexpr int NQ = F32B ? qf_float4s<D>() : qc_float4s<D>();
  static constexpr int BUF = kWarpStageCells * (NB + NQ);  // float4 per buffer: the map blocks, then the coefficients
  static constexpr size_t bytes() { return (size_t)kAdvectWarps * 2 * BUF * sizeof(float4); }
};

// One particle of a tile: slot j of d, from particle perm[j] of s when perm
// is given (the previous step's order applied on the way: its cell is in
// d.cell[j], its id and properties are carried over), else slot j of s in
// place.  Returns the new cell (PIC_LOST if none); *full is set when the full
// path redid it.
template <int D, int RK, bool F32B, bool TWO, class Cells>
__device__ __forceinline__ uint32_t tile_particle(const Cells& cs, const MeshView& m, const StoreView& s,
                                                  const StoreView& d, const uint32_t* __restrict__ perm, df dt,
                                                  uint32_t j, int& iters, unsigned& flags, uint32_t& full) {
  uint32_t i = j, K;
  if (perm) {
    i = perm[j];
    K = d.cell[j];
    if (i >= s.cap) {
      flags |= kFlagBounds;
      return PIC_LOST;
    }
    d.id[j] = s.id[i];
    for (int q = 0; q < s.n_props; ++q) d.props[(size_t)q * d.cap + j] = s.props[(size_t)q * s.cap + i];
  } else {
    K = s.cell[j];
  }
  uint32_t Kn = advect_particle_cells<D, RK, F32B, TWO, NoHook, true>(cs, m, s, i, d, j, K, dt, iters, flags);
  if (Kn == kDefer) {
    const FullStep f = advect_particle_full<D, RK, F32B, TWO>(m, s, i, d, j, K, dt);
    Kn = f.K;
    iters = f.iters;
    flags = f.flags;
    full = 1;
  }
  return Kn;
}

// Resident blocks per SM of the step kernel, swept on the 128^3 x 20 step
// (CUDA events, the same GB300 nodes back to back):
// - FP64 form: 7 blocks (72 registers) 14.47 ms, 6 blocks (80) 14.76 ms,
//   5 blocks 16.29 ms;
// - FP32-basis form: 8 blocks (64 registers) 6.81 ms on most nodes but
//   9.27 ms on others, 7 blocks 6.82 or 8.18 ms from one run to the next on
//   one node, 6 blocks (80 registers, fewest spills) 7.01-7.02 ms on every
//   node and run, so it takes 6.
#ifndef PIC_ADVECT_MIN_BLOCKS_F64
#define PIC_ADVECT_MIN_BLOCKS_F64 7
#endif
#ifndef PIC_ADVECT_MIN_BLOCKS_F32
#define PIC_ADVECT_MIN_BLOCKS_F32 6
#endif
template <int D, int RK, bool F32B, bool TWO, bool STAGE>
__global__ void __launch_bounds__(kAdvectThreads, F32B ? PIC_ADVECT_MIN_BLOCKS_F32 : PIC_ADVECT_MIN_BLOCKS_F64)
    advect_kernel(const __grid_constant__ MeshView m, const __grid_constant__ StoreView s,
                  const __grid_constant__ StoreView d, const uint32_t* __restrict__ perm, df dt,
                  uint32_t* __restrict__ cell_new, uint32_t* __restrict__ counts, DevCounters* __restrict__ ctr) {
  using L = StageLayout<D, F32B>;
  extern __shared__ float4 stage_smem[];  // STAGE: [warp][2 buffers][BUF]
  __shared__ __align__(8) uint64_t bars[kAdvectWarps][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4* const wbuf = stage_smem + (size_t)warp * 2 * L::BUF;
  uint64_t* const bar = bars[warp];

  const uint32_t n = ctr->n_alive;
  const uint32_t ntiles = (n + 31) / 32;
  const uint32_t* __restrict__ start_cell = perm ? d.cell : s.cell;
  auto grab = [&]() -> uint32_t {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(&ctr->tile_next, 1u);
    return __shfl_sync(0xffffffffu, t, 0);
  };
  auto start_of = [&](uint32_t t) -> uint32_t {
    const uint32_t j = t * 32 + lane;
    return (t < ntiles && j < n) ? start_cell[j] : PIC_LOST;
  };
  // the warp: copy the blocks of the cells its tile starts in (kc: each
  // lane's start cell) into buffer b; k0, cnt receive the first staged cell
  // and the number staged (the same in every lane)
  auto issue = [&](uint32_t kc, int b, uint32_t& k0, uint32_t& cnt) {
    const bool ok = kc < m.C;
    const uint32_t lo = __reduce_min_sync(0xffffffffu, ok ? kc : 0xffffffffu);
    const uint32_t hi = __reduce_max_sync(0xffffffffu, ok ? kc : 0u);
    k0 = lo;
    cnt = lo <= hi ? (hi - lo + 1 < (uint32_t)kWarpStageCells ? hi - lo + 1 : (uint32_t)kWarpStageCells) : 0u;
    if (lane == 0) {
      fence_proxy_async_shared();
      mbar_arrive_expect_tx(&bar[b], cnt * (L::NB + L::NQ) * (uint32_t)sizeof(float4));
      if (cnt) {
        float4* dst = wbuf + b * L::BUF;
        bulk_copy_g2s(dst, m.blk + (size_t)k0 * L::NB, cnt * L::NB * (uint32_t)sizeof(float4), &bar[b]);
        bulk_copy_g2s(dst + kWarpStageCells * L::NB, (F32B ? m.Qf : m.Qc) + (size_t)k0 * L::NQ,
                      cnt * L::NQ * (uint32_t)sizeof(float4), &bar[b]);
      }
    }
  };

  if constexpr (STAGE) {
    if (lane == 0) {
      mbar_init(&bar[0], 1);
      mbar_init(&bar[1], 1);
      mbar_init_fence();
    }
    __syncwarp();
  }
  bool staging = STAGE;
  uint32_t t = grab(), tn = grab();
  bool need = staging && t < ntiles;  // a copy into the current buffer is in flight
  uint32_t k0_cur = 0, n_cur = 0, k0_nxt = 0, n_nxt = 0;
  if (need) issue(start_of(t), 0, k0_cur, n_cur);
  uint32_t kc_n = staging ? start_of(tn) : PIC_LOST;  // start cells of the next tile
  uint32_t it = 0;
  uint32_t stuck = 0, stuck_parity = 0;  // per buffer (bit b): a wait that ran out, and its phase
  while (t < ntiles) {
    const int b = (int)(it & 1u);
    const bool need_next = staging && tn < ntiles;
    if (need_next) issue(kc_n, b ^ 1, k0_nxt, n_nxt);
    // the tile after next (and its start cells): their latency hides behind
    // this tile
    const uint32_t tnn = tn < ntiles ? grab() : tn;
    if (staging) kc_n = start_of(tnn);
    bool ok = true;
    if (need) {
      ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[b], (it >> 1) & 1u, kStageWaitNs));
      if (!ok) {
        staging = false;
        if (lane == 0) latch_status(ctr, PIC_STATUS_TIMEOUT);
        stuck |= 1u << b;
        stuck_parity = (stuck_parity & ~(1u << b)) | (((it >> 1) & 1u) << b);
      }
    }

    const uint32_t j = t * 32 + lane;
    int iters = 0;
    unsigned flags = 0, lost = 0, steps = 0;
    uint32_t Kc = PIC_LOST, full = 0;  // the new cell to count
    if (j < n) {
      steps = 1;
      uint32_t Kn;
      if constexpr (STAGE) {
        const StagedCells<D, F32B, kWarpStageCells> cs{m, wbuf + b * L::BUF, k0_cur, (need && ok) ? n_cur : 0u};
        Kn = tile_particle<D, RK, F32B, TWO>(cs, m, s, d, perm, dt, j, iters, flags, full);
      } else {
        Kn = tile_particle<D, RK, F32B, TWO>(GlobalCells<D, F32B>{m}, m, s, d, perm, dt, j, iters, flags, full);
      }
      cell_new[j] = Kn;
      Kc = Kn;
      lost = Kn == PIC_LOST ? 1u : 0u;
    }
    {
      const unsigned dc = __reduce_add_sync(0xffffffffu, full);
      if (dc && lane == 0) atomicAdd(&ctr->deferred, (unsigned long long)dc);
    }
    (void)aggregated_increment(counts, Kc, Kc != PIC_LOST);
    flush_counters(ctr, steps, iters, lost, (flags & kFlagWalk) ? 1u : 0u, (flags & kFlagGlobal) ? 1u : 0u, flags);
    if constexpr (STAGE) __syncwarp();  // this buffer is free for the copy issued one tile on
    need = need_next;
    k0_cur = k0_nxt;
    n_cur = n_nxt;
    t = tn;
    tn = tnn;
    ++it;
  }
  // a copy whose wait ran out may still be in flight: give it one more
  // bounded wait before the block's shared memory is released
  if (STAGE && lane == 0)
    for (int b = 0; b < 2; ++b)
      if ((stuck >> b) & 1u) (void)mbar_wait_bounded(&bar[b], (stuck_parity >> b) & 1u, kStageWaitNs);
}

// Relocate every particle at its current x (hint: its current cell).
template <int D>
__global__ void __launch_bounds__(128) relocate_kernel(const __grid_constant__ MeshView m, const __grid_constant__ StoreView s, uint32_t* __restrict__ cell_new,
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
__global__ void __launch_bounds__(128) locate_points_kernel(const __grid_constant__ MeshView m, size_t n, const double* __restrict__ x,
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
// Persistent grid: PIC_ADVECT_MIN_BLOCKS_F64 / _F32 blocks per SM (the register
// budget's residency), fewer when the store has fewer warp tiles.
static int advect_grid(size_t n, bool f32b) {
  const size_t blocks = (n + kAdvectThreads - 1) / kAdvectThreads;
  const size_t cap = (size_t)num_sms() * (f32b ? PIC_ADVECT_MIN_BLOCKS_F32 : PIC_ADVECT_MIN_BLOCKS_F64);
  const size_t g = blocks < cap ? blocks : cap;
  return (int)(g > 0 ? g : 1);
}

template <int D, int RK, bool F32B>
static void launch_advect(pic_particles_s* p, const MeshView& m, double dt, bool fused, cudaStream_t st) {
  const float hi = (float)dt;
  const df dtd = {hi, (float)(dt - (double)hi)};
  const StoreView s = store_view(p, p->cur), d = fused ? store_view(p, 1 - p->cur) : s;
  const uint32_t* perm = fused ? p->perm : nullptr;
  const int grid = advect_grid(p->capacity, F32B);
  if (m.has_next) {
    advect_kernel<D, RK, F32B, true, false><<<grid, kAdvectThreads, 0, st>>>(m, s, d, perm, dtd, p->cell_new,
                                                                             p->counts, p->ctr);
  } else if (D == 3 && p->stage_cells) {
    advect_kernel<D, RK, F32B, false, D == 3><<<grid, kAdvectThreads, StageLayout<D, F32B>::bytes(), st>>>(
        m, s, d, perm, dtd, p->cell_new, p->counts, p->ctr);
  } else {
    advect_kernel<D, RK, F32B, false, false><<<grid, kAdvectThreads, 0, st>>>(m, s, d, perm, dtd, p->cell_new,
                                                                              p->counts, p->ctr);
  }
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
  if (precision != PIC_FP64 && precision != PIC_FP32_BASIS && precision != PIC_FP32_BASIS_STAGE_DF)
    return (set_error("pic_advect: unknown precision %d", (int)precision), PIC_ERR_ARG);
  if (!mesh->has_velocity) return (set_error("pic_advect: velocity not set"), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  if (precision != PIC_FP64) {
    const pic_status r = ensure_fp32_coefficients(mesh, st);
    if (r != PIC_OK) return r;
  }
  MeshView m = mesh_view(mesh);
  m.stage_df = precision == PIC_FP32_BASIS_STAGE_DF ? 1 : 0;
  // Each step's rebin computes the new order (perm, sorted cells); the
  // particles themselves move with the next step's advect, which reads them
  // through perm.  Every step thus reads and writes the particle state once
  // instead of twice.  The last step's order stays pending for the next
  // call (see settle_order).
  bool pending = parts->pending_order != 0;
  for (int step = 0; step < n_steps; ++step) {
    PIC_CUDA(cudaMemsetAsync(parts->counts, 0, sizeof(uint32_t) * parts->C, st));
    PIC_CUDA(cudaMemsetAsync(&parts->ctr->tile_next, 0, sizeof(unsigned int), st));
    cudaEvent_t* ev = parts->timing ? timing_slot(parts) : nullptr;
    if (ev) PIC_CUDA(cudaEventRecord(ev[0], st));
    const bool f32 = precision != PIC_FP64;
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
    parts->pending_order = 0;  // consumed by this step's advect
    pic_status r = rebin_order_from_counts(parts, st);
    if (r != PIC_OK) return r;
    pending = true;
    parts->pending_order = 1;
    if (ev) PIC_CUDA(cudaEventRecord(ev[2], st));
  }
  return PIC_OK;
}

extern "C" pic_status pic_locate(pic_particles parts, pic_mesh mesh, void* stream) {
  if (!parts || !mesh) return (set_error("pic_locate: null handle"), PIC_ERR_ARG);
  if (parts->mesh != mesh) return (set_error("pic_locate: mesh mismatch"), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  {
    const pic_status r0 = settle_order(parts, st);
    if (r0 != PIC_OK) return r0;
  }
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
