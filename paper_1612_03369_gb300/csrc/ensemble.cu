// ensemble.cu -- many independent problems (meshes, fields and particle sets
// of uneven size) advanced together.
//
// All problems share one particle store: problem p's cells are the store
// cells base[p] .. base[p+1]-1, so one rebin over the concatenated cells
// keeps every problem sorted by (cell, id), and the work of a step is spread
// over the particles of all problems regardless of how uneven the problems
// are.  Each particle finds its problem by a binary search of base[] and
// advances with exactly the per-particle code of pic_advect (advect.cuh), so
// a problem run in the ensemble matches the same problem run alone bit for
// bit.
//
// Two ways to run n steps, both captured once into a CUDA graph and replayed:
//   mode 0  per step: the ensemble advect kernel + the rebin kernels
//   mode 1  one persistent cooperative kernel for all n steps; its phases
//           (advect over dynamically claimed tiles, scan, scatter, rank,
//           gather) are separated by a grid barrier whose waits are bounded
//           by a time limit: a wait that runs out sets an error flag, every
//           block leaves, and the call reports PIC_ERR_TIMEOUT.
// The persistent kernel's blocks per SM and tile size come from a small
// autotuner that times one step per candidate on a snapshot of the store.
#include <cstdlib>
#include <cstring>
#include <vector>

#include "advect.cuh"
#include "rebin.cuh"
#include "seed.cuh"

namespace pic {

constexpr int kMaxEnsemble = 128;
constexpr int kEnsBlock = 128;
constexpr int kMaxBlocksPerSm = 32;  // the hardware's limit of resident blocks

// Resident blocks per SM the ensemble kernels are compiled for (72
// registers).  On the 64-problem 2D ensemble, 7 against 6: per-step mode
// 8.48 against 8.65 ms per step, persistent kernel 8.89 against 8.95 ms; 8
// (64 registers) made the persistent kernel slower (9.19 ms).
#ifndef PIC_ENSEMBLE_MIN_BLOCKS
#define PIC_ENSEMBLE_MIN_BLOCKS 7
#endif

struct GridBarrier {
  unsigned int count;
  unsigned int gen;
  unsigned int err;
  unsigned int pad;
};

// Grid-wide barrier for co-resident blocks (sense by generation count).  The
// wait of each block is bounded by timeout_ns; on expiry (or when another
// block has flagged an error) it sets b->err and returns false, and callers
// leave the kernel.
__device__ __forceinline__ bool grid_sync(GridBarrier* b, unsigned int nblocks, unsigned long long timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* vgen = &b->gen;
    volatile unsigned int* verr = &b->err;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&b->count, 1u) + 1u;
    if (arrived == nblocks) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*vgen == g) {
        if (*verr) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > timeout_ns) {
          atomicOr(&b->err, 1u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok && (*verr == 0u);
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ int problem_of(const uint32_t* sbase, int P, uint32_t gcell) {
  int lo = 0, hi = P;  // base[lo] <= gcell < base[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (sbase[mid] <= gcell)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

struct EnsShared {
  MeshView views[kMaxEnsemble];
  uint32_t base[kMaxEnsemble + 1];
  df dt[kMaxEnsemble];
};

__device__ __forceinline__ void load_ensemble(EnsShared& sh, const MeshView* views, const uint32_t* base,
                                              const df* dts, int P) {
  for (int q = threadIdx.x; q <= P; q += blockDim.x) {
    sh.base[q] = base[q];
    if (q < P) {
      sh.views[q] = views[q];
      sh.dt[q] = dts[q];
    }
  }
  __syncthreads();
}

// One particle of the ensemble: its problem from the global cell, then the
// single-mesh step (the fast path, and the full step where the fast path
// defers, as in pic_advect), then back to a global cell.  With perm ==
// nullptr slot j of s advances in place (d is s); otherwise slot j of d takes
// particle perm[j] of s, whose global cell the previous rebin left in
// d.cell[j], with its id and properties (the previous step's order applied on
// the way).  Returns the new global cell (PIC_LOST if none); *full is set
// when the full step ran.
template <int D, int RK>
__device__ __forceinline__ uint32_t ensemble_particle(const EnsShared& sh, int P, const StoreView& s,
                                                      const StoreView& d, const uint32_t* __restrict__ perm, uint32_t j,
                                                      int& iters, unsigned& flags, uint32_t& full) {
  uint32_t i = j, g;
  if (perm) {
    i = perm[j];
    g = d.cell[j];
    if (i >= s.cap) {
      flags |= kFlagBounds;
      return PIC_LOST;
    }
    d.id[j] = s.id[i];
    for (int q = 0; q < s.n_props; ++q) d.props[(size_t)q * d.cap + j] = s.props[(size_t)q * s.cap + i];
  } else {
    g = s.cell[j];
  }
  if (g >= sh.base[P]) {
    flags |= kFlagBounds;
    return PIC_LOST;
  }
  const int p = problem_of(sh.base, P, g);
  const MeshView& m = sh.views[p];
  const uint32_t K = g - sh.base[p];
  uint32_t Kn = advect_particle_cells<D, RK, false, false, NoHook, true>(GlobalCells<D, false>{m}, m, s, i, d, j, K,
                                                                         sh.dt[p], iters, flags);
  if (Kn == kDefer) {
    const FullStep f = advect_particle_full<D, RK, false, false>(m, s, i, d, j, K, sh.dt[p]);
    Kn = f.K;
    iters = f.iters;
    flags = f.flags;
    full = 1;
  }
  return Kn == PIC_LOST ? PIC_LOST : sh.base[p] + Kn;
}

// One step's advect: every warp takes tiles of `tile` particles (a multiple
// of 32) from *tile_ctr, the next one while it works on the current one,
// and advances them 32 at a time, one particle per lane; each new cell is
// counted (warp-aggregated) and written to cell_new.  Warps that finish
// early take more tiles, so the grid ends together.
template <int D, int RK>
__device__ __forceinline__ void ensemble_advect_tiles(const EnsShared& sh, int P, const StoreView& s,
                                                      const StoreView& d, const uint32_t* __restrict__ perm,
                                                      uint32_t n, uint32_t tile, uint32_t* tile_ctr,
                                                      uint32_t* __restrict__ cell_new, uint32_t* __restrict__ counts,
                                                      DevCounters* __restrict__ ctr) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t ntiles = (n + tile - 1) / tile;
  auto grab = [&]() -> uint32_t {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(tile_ctr, 1u);
    return __shfl_sync(0xffffffffu, t, 0);
  };
  uint32_t t = grab();
  while (t < ntiles) {
    const uint32_t tn = grab();
    const uint32_t end = (t + 1) * tile < n ? (t + 1) * tile : n;
    for (uint32_t j0 = t * tile; j0 < end; j0 += 32u) {
      const uint32_t j = j0 + lane;
      int iters = 0;
      unsigned flags = 0, lost = 0, steps = 0;
      uint32_t Kc = PIC_LOST, full = 0;
      if (j < end) {
        steps = 1;
        Kc = ensemble_particle<D, RK>(sh, P, s, d, perm, j, iters, flags, full);
        cell_new[j] = Kc;
        lost = Kc == PIC_LOST ? 1u : 0u;
      }
      const unsigned dc = __reduce_add_sync(0xffffffffu, full);
      if (dc && lane == 0) atomicAdd(&ctr->deferred, (unsigned long long)dc);
      (void)aggregated_increment(counts, Kc, Kc != PIC_LOST);
      flush_counters(ctr, steps, iters, lost, (flags & kFlagWalk) ? 1u : 0u, (flags & kFlagGlobal) ? 1u : 0u,
                     flags);
    }
    t = tn;
  }
}

// Per-step mode: one step's advect over the whole ensemble (tiles from the
// store's work counter, cleared before the launch).
template <int D, int RK>
__global__ void __launch_bounds__(kEnsBlock, PIC_ENSEMBLE_MIN_BLOCKS) ensemble_advect_kernel(
    const MeshView* __restrict__ views, const uint32_t* __restrict__ base, const df* __restrict__ dts, int P,
    const __grid_constant__ StoreView s, const __grid_constant__ StoreView d, const uint32_t* __restrict__ perm,
    uint32_t tile, uint32_t* __restrict__ cell_new, uint32_t* __restrict__ counts, DevCounters* __restrict__ ctr) {
  __shared__ EnsShared sh;
  load_ensemble(sh, views, base, dts, P);
  ensemble_advect_tiles<D, RK>(sh, P, s, d, perm, ctr->n_alive, tile, &ctr->tile_next, cell_new, counts, ctr);
}

struct PersistArgs {
  const MeshView* views;
  const uint32_t* base;
  const df* dts;
  int P;
  StoreView sv[2];
  int start;  // buffer holding the store at the first step
  uint32_t *cell_new, *counts, *cursor, *cell_off, *chunk_sums, *key_src, *perm, *tile_ctr;
  uint64_t* key_id;
  DevCounters* ctr;
  GridBarrier* bar;
  uint32_t C;
  size_t cap;
  int dim, n_steps, tile;
  unsigned long long timeout_ns;
};

// All n_steps of the ensemble in one launch (see the file comment).  A step
// is five phases, each ended by a grid barrier: advect (warp tiles); the sums
// of the blocks' chunks of the per-cell counts; each chunk's offsets; the
// scatter, which also clears the counts for the next step (the offsets are
// built, nothing reads them again); the rank.  counts and the tile counters
// are cleared before the launch.
template <int D, int RK>
__global__ void __launch_bounds__(kEnsBlock, PIC_ENSEMBLE_MIN_BLOCKS) ensemble_persistent_kernel(PersistArgs A) {
  __shared__ EnsShared sh;
  load_ensemble(sh, A.views, A.base, A.dts, A.P);
  const uint32_t nb = gridDim.x, bid = blockIdx.x;
  const uint32_t gtid = bid * blockDim.x + threadIdx.x, gthreads = nb * blockDim.x;
  // The particles of buffer curb stand in the order of the previous rebin
  // (pending) or in the store's order; each step's advect applies the
  // pending order on the way (reading curb, writing the other buffer), and
  // one gather after the last step applies the last order.
  int curb = A.start;
  bool pending = false;
  uint32_t n = *(volatile uint32_t*)&A.ctr->n_alive;
  for (int step = 0; step < A.n_steps; ++step) {
    ensemble_advect_tiles<D, RK>(sh, A.P, A.sv[curb], A.sv[pending ? 1 - curb : curb], pending ? A.perm : nullptr, n,
                                 (uint32_t)A.tile, A.tile_ctr + step, A.cell_new, A.counts, A.ctr);
    if (pending) curb = 1 - curb;
    const StoreView& cur = A.sv[curb];
    const StoreView& nxt = A.sv[1 - curb];
    if (!grid_sync(A.bar, nb, A.timeout_ns)) return;
    scan_phase_chunk_sums(A.counts, A.C, A.chunk_sums, bid, nb);
    if (!grid_sync(A.bar, nb, A.timeout_ns)) return;
    scan_phase_chunk_apply(A.counts, A.C, A.chunk_sums, A.cell_off, A.cursor, &A.ctr->n_next, bid, nb);
    if (!grid_sync(A.bar, nb, A.timeout_ns)) return;
    const uint32_t nn = *(volatile uint32_t*)&A.ctr->n_next;
    for (uint32_t c = gtid; c < A.C; c += gthreads) A.counts[c] = 0u;
    if (gtid == 0) A.ctr->n_alive = nn;
    scatter_phase(A.cell_new, cur.id, A.cursor, A.key_id, A.key_src, A.C, A.cap, n, &A.ctr->status, gtid, gthreads);
    if (!grid_sync(A.bar, nb, A.timeout_ns)) return;
    rank_phase(A.cell_off, A.key_id, A.key_src, A.perm, nxt.cell, A.C, A.cap, &A.ctr->status, gtid >> 5,
               gthreads >> 5);
    if (!grid_sync(A.bar, nb, A.timeout_ns)) return;
    n = nn;
    pending = true;
  }
  if (pending) gather_phase(A.sv[curb], A.sv[1 - curb], A.perm, A.dim, n, &A.ctr->status, gtid, gthreads);
}

// Barrier self-test: the barrier expects one block more than the launch has,
// so every wait must run out (nothing else ever arrives).
__global__ void barrier_selftest_kernel(GridBarrier* b, unsigned long long timeout_ns) {
  (void)grid_sync(b, gridDim.x + 1, timeout_ns);
}

__global__ void xhat_pairs_kernel(const float2* __restrict__ src, double* __restrict__ dst, size_t n, size_t cap,
                                  size_t beg, int dim) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n * dim; q += (size_t)gridDim.x * blockDim.x) {
    const size_t a = q / n, j = q % n;
    const float2 v = src[a * cap + beg + j];
    dst[q] = (double)v.x + (double)v.y;
  }
}

__global__ void local_cells_kernel(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, uint32_t n,
                                   uint32_t base) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i] - base;
}

}  // namespace pic

using namespace pic;

struct pic_ensemble_s {
  int P, dim, n_props;
  std::vector<pic_mesh> meshes;
  std::vector<uint32_t> base_host;
  MeshView* views_dev;
  uint32_t* base_dev;
  df* dt_dev;
  int has_dt;
  pic_particles_s* store;
  GridBarrier* bar;
  uint32_t* chunk_sums;  // one per block of the persistent grid
  uint32_t* tile_ctr;
  int tile_ctr_cap;
  int blocks_per_sm, tile;
  double timeout_s;
  struct Cached {
    cudaGraphExec_t exec;
    int n_steps, mode, integrator, start;
  } cache[4];
  int n_cache;
  cudaStream_t cap_stream;  // private stream used only to capture graphs
};

static void drop_graphs(pic_ensemble_s* e) {
  for (int k = 0; k < e->n_cache; ++k) cudaGraphExecDestroy(e->cache[k].exec);
  e->n_cache = 0;
}

extern "C" pic_status pic_ensemble_destroy(pic_ensemble e) {
  if (!e) return PIC_OK;
  drop_graphs(e);
  if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
  cudaFree(e->views_dev);
  cudaFree(e->base_dev);
  cudaFree(e->dt_dev);
  cudaFree(e->bar);
  cudaFree(e->chunk_sums);
  cudaFree(e->tile_ctr);
  pic_destroy_particles(e->store);
  delete e;
  return PIC_OK;
}

extern "C" pic_status pic_ensemble_create(int n_problems, const pic_mesh* meshes, const uint32_t* const* per_cell,
                                          const uint32_t* uniform_counts, const uint64_t* seeds, int n_props,
                                          void* stream, pic_ensemble* out) {
  if (!out) return (set_error("pic_ensemble_create: out is NULL"), PIC_ERR_ARG);
  *out = nullptr;
  if (n_problems < 1 || n_problems > kMaxEnsemble)
    return (set_error("pic_ensemble_create: 1 <= n_problems <= %d", kMaxEnsemble), PIC_ERR_ARG);
  if (!meshes || !seeds || (!per_cell && !uniform_counts))
    return (set_error("pic_ensemble_create: null array"), PIC_ERR_ARG);
  if (n_props < 0 || n_props > kMaxProps) return (set_error("pic_ensemble_create: bad n_props"), PIC_ERR_ARG);
  const int dim = meshes[0] ? meshes[0]->dim : 0;
  for (int p = 0; p < n_problems; ++p) {
    if (!meshes[p] || meshes[p]->dim != dim)
      return (set_error("pic_ensemble_create: mesh %d missing or of another dimension", p), PIC_ERR_ARG);
    if (!meshes[p]->has_velocity) return (set_error("pic_ensemble_create: mesh %d has no velocity", p), PIC_ERR_ARG);
    if (meshes[p]->has_next)
      return (set_error("pic_ensemble_create: mesh %d has a second field; the ensemble runs steady fields", p),
              PIC_ERR_ARG);
  }
  cudaStream_t st = (cudaStream_t)stream;
  pic_ensemble_s* e = new pic_ensemble_s();
  e->P = n_problems;
  e->dim = dim;
  e->n_props = n_props;
  e->meshes.assign(meshes, meshes + n_problems);
  e->base_host.resize(n_problems + 1);
  e->timeout_s = 4.0;
  e->blocks_per_sm = 0;
  e->tile = 32;
  uint64_t Ct = 0;
  for (int p = 0; p < n_problems; ++p) {
    e->base_host[p] = (uint32_t)Ct;
    Ct += meshes[p]->C;
  }
  if (Ct >= (1ull << 31)) {
    delete e;
    return (set_error("pic_ensemble_create: too many cells in total"), PIC_ERR_ARG);
  }
  e->base_host[n_problems] = (uint32_t)Ct;
  const uint32_t C = (uint32_t)Ct;
  std::vector<MeshView> views(n_problems);
  for (int p = 0; p < n_problems; ++p) views[p] = mesh_view(meshes[p]);
  auto fail = [&](pic_status s) {
    pic_ensemble_destroy(e);
    return s;
  };
  uint32_t *counts = nullptr, *off = nullptr, *sums = nullptr, *total = nullptr;
  if (cudaMalloc(&e->views_dev, sizeof(MeshView) * n_problems) != cudaSuccess ||
      cudaMalloc(&e->base_dev, sizeof(uint32_t) * (n_problems + 1)) != cudaSuccess ||
      cudaMalloc(&e->dt_dev, sizeof(df) * n_problems) != cudaSuccess ||
      cudaMalloc(&e->bar, sizeof(GridBarrier)) != cudaSuccess ||
      cudaMalloc(&counts, sizeof(uint32_t) * C) != cudaSuccess ||
      cudaMalloc(&off, sizeof(uint32_t) * ((size_t)C + 1)) != cudaSuccess ||
      cudaMalloc(&sums, scan_scratch_bytes(C)) != cudaSuccess ||
      cudaMalloc(&total, sizeof(uint32_t) * 2) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(counts);
    cudaFree(off);
    cudaFree(sums);
    cudaFree(total);
    set_error("pic_ensemble_create: device allocation failed");
    return fail(PIC_ERR_OOM);
  }
  PIC_CUDA(cudaMemcpyAsync(e->views_dev, views.data(), sizeof(MeshView) * n_problems, cudaMemcpyHostToDevice, st));
  PIC_CUDA(cudaMemcpyAsync(e->base_dev, e->base_host.data(), sizeof(uint32_t) * (n_problems + 1),
                           cudaMemcpyHostToDevice, st));
  PIC_CUDA(cudaMemsetAsync(e->bar, 0, sizeof(GridBarrier), st));
  // per-problem counts into the concatenated cells, one scan for all
  uint64_t N = 0;
  for (int p = 0; p < n_problems; ++p) {
    const uint32_t Cp = meshes[p]->C;
    const uint32_t* pc = per_cell ? per_cell[p] : nullptr;
    const uint32_t u = uniform_counts ? uniform_counts[p] : 0u;
    fill_counts_kernel<<<(Cp + 255) / 256 < 4096 ? (Cp + 255) / 256 : 4096, 256, 0, st>>>(pc, u, counts + e->base_host[p],
                                                                                         Cp);
  }
  pic_status r = scan_u32(counts, off, C, sums, total, nullptr, st);
  uint32_t hN = 0;
  cudaError_t ce = cudaMemcpyAsync(&hN, total, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  cudaFree(counts);
  cudaFree(sums);
  cudaFree(total);
  if (r != PIC_OK || ce != cudaSuccess) {
    cudaFree(off);
    if (ce != cudaSuccess) cuda_fail(ce, "pic_ensemble_create: counting");
    return fail(r != PIC_OK ? r : PIC_ERR_CUDA);
  }
  N = hN;
  e->store = store_alloc(dim, n_props, C, N, off);
  if (!e->store) return fail(PIC_ERR_OOM);
  e->store->stream = st;
  DevCounters h{};
  h.n_alive = (uint32_t)N;
  h.n_next = (uint32_t)N;
  PIC_CUDA(cudaMemcpyAsync(e->store->ctr, &h, sizeof(h), cudaMemcpyHostToDevice, st));
  for (int p = 0; p < n_problems; ++p) {
    const uint32_t Cp = meshes[p]->C;
    const int grid = (int)((Cp + 127) / 128 < 8192 ? (Cp + 127) / 128 : 8192);
    if (dim == 2)
      seed_kernel<2><<<grid, 128, 0, st>>>(views[p], store_view(e->store, 0), off, seeds[p], 0, e->base_host[p]);
    else
      seed_kernel<3><<<grid, 128, 0, st>>>(views[p], store_view(e->store, 0), off, seeds[p], 0, e->base_host[p]);
  }
  PIC_CUDA(cudaGetLastError());
  PIC_CUDA(cudaStreamSynchronize(st));
  *out = e;
  return PIC_OK;
}

extern "C" pic_status pic_ensemble_set_dt(pic_ensemble e, const double* dts, void* stream) {
  if (!e || !dts) return (set_error("pic_ensemble_set_dt: null argument"), PIC_ERR_ARG);
  std::vector<df> v(e->P);
  for (int p = 0; p < e->P; ++p) {
    if (!(dts[p] == dts[p]) || dts[p] - dts[p] != 0.0) return (set_error("pic_ensemble_set_dt: dt %d not finite", p), PIC_ERR_ARG);
    const float hi = (float)dts[p];
    v[p].hi = hi;
    v[p].lo = (float)(dts[p] - (double)hi);
  }
  PIC_CUDA(cudaMemcpyAsync(e->dt_dev, v.data(), sizeof(df) * e->P, cudaMemcpyHostToDevice, (cudaStream_t)stream));
  PIC_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  e->has_dt = 1;
  return PIC_OK;
}

namespace pic {

static int ensemble_max_blocks_per_sm(int dim, int rk) {
  int b = 0;
  cudaError_t r;
  if (dim == 2)
    r = rk == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ensemble_persistent_kernel<2, 1>, kEnsBlock, 0)
        : rk == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ensemble_persistent_kernel<2, 2>, kEnsBlock, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ensemble_persistent_kernel<2, 4>, kEnsBlock, 0);
  else
    r = rk == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ensemble_persistent_kernel<3, 1>, kEnsBlock, 0)
        : rk == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ensemble_persistent_kernel<3, 2>, kEnsBlock, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ensemble_persistent_kernel<3, 4>, kEnsBlock, 0);
  if (r != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return b > 0 ? b : 1;
}

// Resident blocks per SM of the per-step advect kernel (its grid: one
// resident wave; the warps take tiles from the work counter).
static int ensemble_advect_blocks_per_sm(int dim, int rk) {
  static int cache[2][5] = {};
  int& b = cache[dim == 3][rk];
  if (b > 0) return b;
  cudaError_t r;
  if (dim == 2)
    r = rk == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ensemble_advect_kernel<2, 1>, kEnsBlock, 0)
        : rk == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ensemble_advect_kernel<2, 2>, kEnsBlock, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ensemble_advect_kernel<2, 4>, kEnsBlock, 0);
  else
    r = rk == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ensemble_advect_kernel<3, 1>, kEnsBlock, 0)
        : rk == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ensemble_advect_kernel<3, 2>, kEnsBlock, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ensemble_advect_kernel<3, 4>, kEnsBlock, 0);
  if (r != cudaSuccess || b < 1) {
    cudaGetLastError();
    b = 1;
  }
  return b;
}

template <int D, int RK>
static cudaError_t launch_persistent(const PersistArgs& A, int grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kEnsBlock);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, ensemble_persistent_kernel<D, RK>, A);
}

// Enqueue n_steps (no capture, no synchronisation).
static pic_status enqueue_run(pic_ensemble_s* e, int integrator, int n_steps, int mode, cudaStream_t st) {
  pic_particles_s* s = e->store;
  const int rk = integrator;
  if (mode == 0) {
    const int grid = ensemble_advect_blocks_per_sm(e->dim, rk) * num_sms();
    const uint32_t tile = (uint32_t)e->tile;
    for (int step = 0; step < n_steps; ++step) {
      PIC_CUDA(cudaMemsetAsync(s->counts, 0, sizeof(uint32_t) * s->C, st));
      PIC_CUDA(cudaMemsetAsync(&s->ctr->tile_next, 0, sizeof(uint32_t), st));
      // as in pic_advect: each step applies the previous step's order on the
      // way, and the last step's order is applied by one gather
      const bool fused = step > 0;
      const StoreView sv = store_view(s, s->cur), dv = fused ? store_view(s, 1 - s->cur) : sv;
      const uint32_t* pm = fused ? s->perm : nullptr;
      if (e->dim == 2) {
        if (rk == 1) ensemble_advect_kernel<2, 1><<<grid, kEnsBlock, 0, st>>>(e->views_dev, e->base_dev, e->dt_dev, e->P, sv, dv, pm, tile, s->cell_new, s->counts, s->ctr);
        else if (rk == 2) ensemble_advect_kernel<2, 2><<<grid, kEnsBlock, 0, st>>>(e->views_dev, e->base_dev, e->dt_dev, e->P, sv, dv, pm, tile, s->cell_new, s->counts, s->ctr);
        else ensemble_advect_kernel<2, 4><<<grid, kEnsBlock, 0, st>>>(e->views_dev, e->base_dev, e->dt_dev, e->P, sv, dv, pm, tile, s->cell_new, s->counts, s->ctr);
      } else {
        if (rk == 1) ensemble_advect_kernel<3, 1><<<grid, kEnsBlock, 0, st>>>(e->views_dev, e->base_dev, e->dt_dev, e->P, sv, dv, pm, tile, s->cell_new, s->counts, s->ctr);
        else if (rk == 2) ensemble_advect_kernel<3, 2><<<grid, kEnsBlock, 0, st>>>(e->views_dev, e->base_dev, e->dt_dev, e->P, sv, dv, pm, tile, s->cell_new, s->counts, s->ctr);
        else ensemble_advect_kernel<3, 4><<<grid, kEnsBlock, 0, st>>>(e->views_dev, e->base_dev, e->dt_dev, e->P, sv, dv, pm, tile, s->cell_new, s->counts, s->ctr);
      }
      count_launches(1);
      PIC_CUDA(cudaGetLastError());
      if (fused) s->cur = 1 - s->cur;
      pic_status r = rebin_order_from_counts(s, st);
      if (r != PIC_OK) return r;
      if (step + 1 == n_steps) {
        r = rebin_apply_order(s, st);
        if (r != PIC_OK) return r;
      }
    }
    return PIC_OK;
  }
  // persistent (scratch allocated beforehand by prepare_persistent)
  const int bps = e->blocks_per_sm > 0 ? e->blocks_per_sm : ensemble_max_blocks_per_sm(e->dim, rk);
  const int grid = bps * num_sms();
  if (!e->chunk_sums || e->tile_ctr_cap < n_steps || grid > num_sms() * kMaxBlocksPerSm)
    return (set_error("pic_ensemble_run: persistent scratch missing"), PIC_ERR_STATE);
  PIC_CUDA(cudaMemsetAsync(e->tile_ctr, 0, sizeof(uint32_t) * n_steps, st));
  PIC_CUDA(cudaMemsetAsync(s->counts, 0, sizeof(uint32_t) * s->C, st));
  PIC_CUDA(cudaMemsetAsync(e->bar, 0, sizeof(GridBarrier), st));
  PersistArgs A;
  A.views = e->views_dev;
  A.base = e->base_dev;
  A.dts = e->dt_dev;
  A.P = e->P;
  A.sv[0] = store_view(s, 0);
  A.sv[1] = store_view(s, 1);
  A.start = s->cur;
  A.cell_new = s->cell_new;
  A.counts = s->counts;
  A.cursor = s->cursor;
  A.cell_off = s->cell_off;
  A.chunk_sums = e->chunk_sums;
  A.key_src = s->key_src;
  A.perm = s->perm;
  A.tile_ctr = e->tile_ctr;
  A.key_id = s->key_id;
  A.ctr = s->ctr;
  A.bar = e->bar;
  A.C = s->C;
  A.cap = s->capacity;
  A.dim = e->dim;
  A.n_steps = n_steps;
  A.tile = e->tile;
  A.timeout_ns = (unsigned long long)(e->timeout_s * 1e9);
  cudaError_t ce;
  if (e->dim == 2)
    ce = rk == 1 ? launch_persistent<2, 1>(A, grid, st) : rk == 2 ? launch_persistent<2, 2>(A, grid, st) : launch_persistent<2, 4>(A, grid, st);
  else
    ce = rk == 1 ? launch_persistent<3, 1>(A, grid, st) : rk == 2 ? launch_persistent<3, 2>(A, grid, st) : launch_persistent<3, 4>(A, grid, st);
  if (ce != cudaSuccess) return cuda_fail(ce, "pic_ensemble_run: persistent launch");
  count_launches(1);
  if (n_steps & 1) s->cur = 1 - s->cur;
  return PIC_OK;
}

// Scratch of the persistent kernel (the scan's chunk sums, one per block;
// per-step tile counters); allocated outside any stream capture.
static pic_status prepare_persistent(pic_ensemble_s* e, int n_steps) {
  if (!e->chunk_sums) PIC_CUDA(cudaMalloc(&e->chunk_sums, sizeof(uint32_t) * num_sms() * kMaxBlocksPerSm));
  if (e->tile_ctr_cap < n_steps) {
    cudaFree(e->tile_ctr);
    e->tile_ctr = nullptr;
    PIC_CUDA(cudaMalloc(&e->tile_ctr, sizeof(uint32_t) * n_steps));
    e->tile_ctr_cap = n_steps;
  }
  return PIC_OK;
}

static pic_status barrier_status(pic_ensemble_s* e) {
  GridBarrier h;
  PIC_CUDA(cudaMemcpy(&h, e->bar, sizeof(h), cudaMemcpyDeviceToHost));
  if (h.err) return (set_error("pic_ensemble_run: a grid barrier wait ran out"), PIC_ERR_TIMEOUT);
  return PIC_OK;
}

}  // namespace pic

extern "C" pic_status pic_ensemble_run(pic_ensemble e, pic_integrator integrator, int n_steps, int mode,
                                       int use_graph, void* stream) {
  if (!e) return (set_error("pic_ensemble_run: null handle"), PIC_ERR_ARG);
  if (!e->has_dt) return (set_error("pic_ensemble_run: time steps not set (pic_ensemble_set_dt)"), PIC_ERR_ARG);
  if (n_steps < 0 || (mode != 0 && mode != 1)) return (set_error("pic_ensemble_run: bad n_steps or mode"), PIC_ERR_ARG);
  if (integrator != PIC_EULER && integrator != PIC_RK2 && integrator != PIC_RK4)
    return (set_error("pic_ensemble_run: unknown integrator"), PIC_ERR_ARG);
  if (n_steps == 0) return PIC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  pic_status r;
  if (mode == 1 && (r = prepare_persistent(e, n_steps)) != PIC_OK) return r;
  if (!use_graph) {
    r = enqueue_run(e, (int)integrator, n_steps, mode, st);
  } else {
    const int start = e->store->cur;
    int hit = -1;
    for (int k = 0; k < e->n_cache; ++k) {
      const auto& c = e->cache[k];
      if (c.n_steps == n_steps && c.mode == mode && c.integrator == (int)integrator && c.start == start) hit = k;
    }
    if (hit < 0) {
      // Capture on a private stream: the caller's stream may be the legacy
      // default stream, which cannot be captured.  Capturing executes nothing.
      if (e->n_cache == 4) drop_graphs(e);
      if (!e->cap_stream) PIC_CUDA(cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking));
      cudaGraph_t g;
      PIC_CUDA(cudaStreamBeginCapture(e->cap_stream, cudaStreamCaptureModeThreadLocal));
      r = enqueue_run(e, (int)integrator, n_steps, mode, e->cap_stream);
      cudaError_t ce = cudaStreamEndCapture(e->cap_stream, &g);
      if (r != PIC_OK) {
        if (ce == cudaSuccess) cudaGraphDestroy(g);
        e->store->cur = start;
        return r;
      }
      if (ce != cudaSuccess) {
        e->store->cur = start;
        return cuda_fail(ce, "pic_ensemble_run: stream capture");
      }
      cudaGraphExec_t ex;
      ce = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (ce != cudaSuccess) {
        e->store->cur = start;
        return cuda_fail(ce, "pic_ensemble_run: graph instantiation");
      }
      e->cache[e->n_cache++] = {ex, n_steps, mode, (int)integrator, start};
      hit = e->n_cache - 1;
      e->store->cur = start;  // the capture flipped it; the launch below does it again
    }
    PIC_CUDA(cudaGraphLaunch(e->cache[hit].exec, st));
    if (n_steps & 1) e->store->cur = 1 - e->store->cur;
    r = PIC_OK;
  }
  if (r != PIC_OK) return r;
  if (mode == 1) {
    PIC_CUDA(cudaStreamSynchronize(st));
    return barrier_status(e);
  }
  return PIC_OK;
}

// Autotuner: for each candidate (blocks per SM, tile size) of the persistent
// kernel, restore a snapshot of the store, time one step, keep the fastest;
// the store is restored at the end.
extern "C" pic_status pic_ensemble_tune(pic_ensemble e, pic_integrator integrator, int* blocks_per_sm, int* tile,
                                        double* best_ms, void* stream) {
  if (!e || !e->has_dt) return (set_error("pic_ensemble_tune: null handle or no time steps"), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  pic_particles_s* s = e->store;
  const size_t cap = s->capacity, d = (size_t)e->dim;
  const int c0 = s->cur;
  // snapshot of the current buffer and counters
  double *x = nullptr, *pr = nullptr;
  float2* xh = nullptr;
  uint64_t* id = nullptr;
  uint32_t *cell = nullptr, *off = nullptr;
  DevCounters ctr;
  bool ok = cudaMalloc(&x, sizeof(double) * d * cap) == cudaSuccess &&
            cudaMalloc(&xh, sizeof(float2) * d * cap) == cudaSuccess &&
            cudaMalloc(&id, sizeof(uint64_t) * cap) == cudaSuccess &&
            cudaMalloc(&cell, sizeof(uint32_t) * cap) == cudaSuccess &&
            cudaMalloc(&off, sizeof(uint32_t) * ((size_t)s->C + 1)) == cudaSuccess &&
            cudaMalloc(&pr, sizeof(double) * (e->n_props > 0 ? e->n_props : 1) * cap) == cudaSuccess;
  auto release = [&]() {
    cudaFree(x);
    cudaFree(xh);
    cudaFree(id);
    cudaFree(cell);
    cudaFree(off);
    cudaFree(pr);
  };
  if (!ok) {
    cudaGetLastError();
    release();
    return (set_error("pic_ensemble_tune: snapshot allocation failed"), PIC_ERR_OOM);
  }
  auto copy_state = [&](bool save) -> cudaError_t {
    cudaError_t r = cudaSuccess;
    const int c = s->cur;
    auto cp = [&](void* dst, const void* src, size_t bytes) {
      if (r == cudaSuccess) r = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
    };
    if (save) {
      cp(x, s->x[c], sizeof(double) * d * cap);
      cp(xh, s->xhat[c], sizeof(float2) * d * cap);
      cp(id, s->id[c], sizeof(uint64_t) * cap);
      cp(cell, s->cell[c], sizeof(uint32_t) * cap);
      cp(off, s->cell_off, sizeof(uint32_t) * ((size_t)s->C + 1));
      cp(pr, s->props[c], sizeof(double) * (e->n_props > 0 ? e->n_props : 1) * cap);
      if (r == cudaSuccess) r = cudaMemcpyAsync(&ctr, s->ctr, sizeof(ctr), cudaMemcpyDeviceToHost, st);
      if (r == cudaSuccess) r = cudaStreamSynchronize(st);
    } else {
      cp(s->x[c], x, sizeof(double) * d * cap);
      cp(s->xhat[c], xh, sizeof(float2) * d * cap);
      cp(s->id[c], id, sizeof(uint64_t) * cap);
      cp(s->cell[c], cell, sizeof(uint32_t) * cap);
      cp(s->cell_off, off, sizeof(uint32_t) * ((size_t)s->C + 1));
      cp(s->props[c], pr, sizeof(double) * (e->n_props > 0 ? e->n_props : 1) * cap);
      if (r == cudaSuccess) r = cudaMemcpyAsync(s->ctr, &ctr, sizeof(ctr), cudaMemcpyHostToDevice, st);
      if (r == cudaSuccess) r = cudaStreamSynchronize(st);
    }
    return r;
  };
  cudaError_t ce = copy_state(true);
  if (ce != cudaSuccess) {
    release();
    return cuda_fail(ce, "pic_ensemble_tune: snapshot");
  }
  const int maxb = ensemble_max_blocks_per_sm(e->dim, (int)integrator);
  {
    pic_status pr = prepare_persistent(e, 1);
    if (pr != PIC_OK) {
      release();
      return pr;
    }
  }
  const int tiles[3] = {32, 128, 512};
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  double best = 1e300;
  int bb = maxb, bt = 32;
  const int save_b = e->blocks_per_sm, save_t = e->tile;
  pic_status result = PIC_OK;
  for (int b = 1; b <= maxb && result == PIC_OK; ++b)
    for (int q = 0; q < 3 && result == PIC_OK; ++q) {
      s->cur = c0;
      if ((ce = copy_state(false)) != cudaSuccess) {
        result = cuda_fail(ce, "pic_ensemble_tune: restore");
        break;
      }
      e->blocks_per_sm = b;
      e->tile = tiles[q];
      cudaEventRecord(ev0, st);
      pic_status r = enqueue_run(e, (int)integrator, 1, 1, st);
      cudaEventRecord(ev1, st);
      if (r == PIC_OK) {
        cudaEventSynchronize(ev1);
        r = barrier_status(e);
      }
      if (r != PIC_OK) {
        result = r;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev0, ev1);
      if (ms < best) {
        best = ms;
        bb = b;
        bt = tiles[q];
      }
    }
  s->cur = c0;
  ce = copy_state(false);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  release();
  if (result != PIC_OK) {
    e->blocks_per_sm = save_b;
    e->tile = save_t;
    return result;
  }
  if (ce != cudaSuccess) return cuda_fail(ce, "pic_ensemble_tune: final restore");
  e->blocks_per_sm = bb;
  e->tile = bt;
  drop_graphs(e);
  if (blocks_per_sm) *blocks_per_sm = bb;
  if (tile) *tile = bt;
  if (best_ms) *best_ms = best;
  return PIC_OK;
}

extern "C" pic_status pic_ensemble_state(pic_ensemble e, size_t* n_alive, size_t* n_lost, uint32_t* status) {
  if (!e) return (set_error("pic_ensemble_state: null handle"), PIC_ERR_ARG);
  return pic_get_state(e->store, n_alive, n_lost, status);
}

extern "C" pic_status pic_ensemble_export(pic_ensemble e, int problem, double* x, double* xhat, uint64_t* id,
                                          uint32_t* cell, size_t* n_out, void* stream) {
  if (!e || problem < 0 || problem >= e->P) return (set_error("pic_ensemble_export: bad argument"), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  pic_particles_s* s = e->store;
  PIC_CUDA(cudaDeviceSynchronize());
  uint32_t r[2];
  PIC_CUDA(cudaMemcpy(&r[0], s->cell_off + e->base_host[problem], sizeof(uint32_t), cudaMemcpyDeviceToHost));
  PIC_CUDA(cudaMemcpy(&r[1], s->cell_off + e->base_host[problem + 1], sizeof(uint32_t), cudaMemcpyDeviceToHost));
  const size_t beg = r[0], n = r[1] - r[0], cap = s->capacity;
  if (n_out) *n_out = n;
  if (n == 0) return PIC_OK;
  const int c = s->cur;
  for (int a = 0; a < e->dim; ++a) {
    if (x) PIC_CUDA(cudaMemcpyAsync(x + a * n, s->x[c] + a * cap + beg, sizeof(double) * n, cudaMemcpyDefault, st));
  }
  if (xhat) {
    xhat_pairs_kernel<<<1024, 256, 0, st>>>(s->xhat[c], xhat, n, cap, beg, e->dim);
    PIC_CUDA(cudaGetLastError());
  }
  if (id) PIC_CUDA(cudaMemcpyAsync(id, s->id[c] + beg, sizeof(uint64_t) * n, cudaMemcpyDefault, st));
  if (cell) {
    local_cells_kernel<<<(int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, st>>>(s->cell[c] + beg, cell,
                                                                                                (uint32_t)n,
                                                                                                e->base_host[problem]);
    PIC_CUDA(cudaGetLastError());
  }
  return PIC_OK;
}

extern "C" pic_status pic_barrier_selftest(double timeout_s, void* stream) {
  if (!(timeout_s > 0.0) || timeout_s > 10.0) return (set_error("pic_barrier_selftest: timeout in (0, 10] s"), PIC_ERR_ARG);
  GridBarrier* b = nullptr;
  PIC_CUDA(cudaMalloc(&b, sizeof(GridBarrier)));
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(b, 0, sizeof(GridBarrier), st);
  if (e == cudaSuccess) {
    barrier_selftest_kernel<<<2, 32, 0, st>>>(b, (unsigned long long)(timeout_s * 1e9));
    e = cudaGetLastError();
  }
  GridBarrier h{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, b, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(b);
  if (e != cudaSuccess) return cuda_fail(e, "pic_barrier_selftest");
  if (h.err) return (set_error("pic_barrier_selftest: the barrier wait ran out (expected)"), PIC_ERR_TIMEOUT);
  return PIC_OK;
}
