// particles.cu -- the particle store (Sec. 2.1): generation from local
// coordinates (Sec. 2.2), properties (Sec. 2.6), state queries and export.
#include <cstdlib>
#include <cstring>

#include "pic_internal.cuh"
#include "seed.cuh"

namespace pic {

// double-float reference coordinates -> FP64 (export)
__global__ void xhat_to_double_kernel(const float2* __restrict__ src, double* __restrict__ dst, size_t cap, size_t n,
                                      int dim) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n * dim; i += (size_t)gridDim.x * blockDim.x) {
    const size_t a = i / n, j = i % n;
    const float2 v = src[a * cap + j];
    dst[a * n + j] = (double)v.x + (double)v.y;
  }
}

__global__ void set_prop_kernel(double* __restrict__ dst, const double* __restrict__ src, const DevCounters* ctr) {
  const uint32_t n = ctr->n_alive;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

}  // namespace pic

using namespace pic;

extern "C" pic_status pic_destroy_particles(pic_particles p) {
  if (!p) return PIC_OK;
  for (int b = 0; b < 2; ++b) {
    cudaFree(p->x[b]);
    cudaFree(p->xhat[b]);
    cudaFree(p->id[b]);
    cudaFree(p->cell[b]);
    cudaFree(p->props[b]);
  }
  cudaFree(p->cell_off);
  cudaFree(p->cell_new);
  cudaFree(p->counts);
  cudaFree(p->cursor);
  cudaFree(p->block_sums);
  cudaFree(p->key_id);
  cudaFree(p->key_src);
  cudaFree(p->perm);
  cudaFree(p->ctr);
  cudaFree(p->xfer);
  cudaFree(p->stage_rec);
  for (int k = 0; k < 3 * p->ev_cap; ++k) cudaEventDestroy(p->ev[k]);
  free(p->ev);
  free(p);
  return PIC_OK;
}

namespace pic {

// A store of `capacity` particles over C cells (both rebin buffers and the
// rebin scratch).  Takes ownership of cell_off.  NULL (error message set,
// cell_off freed) if an allocation fails.
pic_particles_s* store_alloc(int dim, int n_props, uint32_t C, size_t capacity, uint32_t* cell_off) {
  pic_particles_s* p = (pic_particles_s*)calloc(1, sizeof(pic_particles_s));
  if (!p) {
    cudaFree(cell_off);
    set_error("store_alloc: host allocation failed");
    return nullptr;
  }
  p->dim = dim;
  p->n_props = n_props;
  p->C = C;
  p->capacity = capacity > 0 ? capacity : 1;
  p->cell_off = cell_off;
  const size_t cap = p->capacity, d = (size_t)dim;
  bool ok = true;
  for (int b = 0; b < 2 && ok; ++b) {
    ok = ok && cudaMalloc(&p->x[b], sizeof(double) * d * cap) == cudaSuccess;
    ok = ok && cudaMalloc(&p->xhat[b], sizeof(float2) * d * cap) == cudaSuccess;
    ok = ok && cudaMalloc(&p->id[b], sizeof(uint64_t) * cap) == cudaSuccess;
    ok = ok && cudaMalloc(&p->cell[b], sizeof(uint32_t) * cap) == cudaSuccess;
    ok = ok && cudaMalloc(&p->props[b], sizeof(double) * (n_props > 0 ? n_props : 1) * cap) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&p->cell_new, sizeof(uint32_t) * cap) == cudaSuccess;
  ok = ok && cudaMalloc(&p->counts, sizeof(uint32_t) * C) == cudaSuccess;
  ok = ok && cudaMalloc(&p->cursor, sizeof(uint32_t) * C) == cudaSuccess;
  ok = ok && cudaMalloc(&p->block_sums, scan_scratch_bytes(C)) == cudaSuccess;
  ok = ok && cudaMalloc(&p->key_id, sizeof(uint64_t) * cap) == cudaSuccess;
  ok = ok && cudaMalloc(&p->key_src, sizeof(uint32_t) * cap) == cudaSuccess;
  ok = ok && cudaMalloc(&p->perm, sizeof(uint32_t) * cap) == cudaSuccess;
  ok = ok && cudaMalloc(&p->ctr, sizeof(DevCounters)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    pic_destroy_particles(p);
    set_error("store_alloc: device allocation failed (capacity %zu)", cap);
    return nullptr;
  }
  return p;
}

}  // namespace pic

namespace pic {

// The part of seeding shared by every generator: per-cell numbers (device
// array, or `uniform_count` everywhere) -> cell offsets -> an allocated store
// of `capacity` (0 = exactly the number created) whose counters say N
// particles.  The generator's kernel then fills slots cell_off[K] ..
// cell_off[K+1]-1 of buffer 0.
pic_status seed_prepare(pic_mesh mesh, const uint32_t* per_cell, uint32_t uniform_count, int n_props, size_t capacity,
                        cudaStream_t st, const char* who, pic_particles_s** out, size_t* n_out) {
  *out = nullptr;
  if (n_props < 0 || n_props > kMaxProps) return (set_error("%s: n_props must be in [0, %d]", who, kMaxProps), PIC_ERR_ARG);
  const uint32_t C = mesh->C;
  uint32_t *counts = nullptr, *off = nullptr, *sums = nullptr, *total = nullptr;
  if (cudaMalloc(&counts, sizeof(uint32_t) * C) != cudaSuccess || cudaMalloc(&off, sizeof(uint32_t) * (C + 1)) != cudaSuccess ||
      cudaMalloc(&sums, scan_scratch_bytes(C)) != cudaSuccess || cudaMalloc(&total, sizeof(uint32_t) * 2) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(counts);
    cudaFree(off);
    cudaFree(sums);
    cudaFree(total);
    return (set_error("%s: device allocation failed", who), PIC_ERR_OOM);
  }
  auto cleanup_tmp = [&]() {
    cudaFree(counts);
    cudaFree(sums);
    cudaFree(total);
  };
  fill_counts_kernel<<<(C + 255) / 256 < 4096 ? (C + 255) / 256 : 4096, 256, 0, st>>>(per_cell, uniform_count, counts, C);
  // 64-bit total check: the scan is 32-bit, so guard against overflow first
  uint64_t total64 = 0;
  if (per_cell) {
    uint32_t* h = (uint32_t*)malloc(sizeof(uint32_t) * C);
    cudaError_t e = h ? cudaMemcpyAsync(h, per_cell, sizeof(uint32_t) * C, cudaMemcpyDefault, st) : cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      free(h);
      cleanup_tmp();
      cudaFree(off);
      return cuda_fail(e, who);
    }
    for (uint32_t K = 0; K < C; ++K) total64 += h[K];
    free(h);
  } else {
    total64 = (uint64_t)uniform_count * C;
  }
  if (total64 >= 0xFFFFFFF0ull) {
    cleanup_tmp();
    cudaFree(off);
    return (set_error("%s: %llu particles exceed the 32-bit store", who, (unsigned long long)total64), PIC_ERR_CAPACITY);
  }
  const size_t N = (size_t)total64;
  if (capacity == 0) capacity = N;
  if (capacity < N) {
    cleanup_tmp();
    cudaFree(off);
    return (set_error("%s: capacity %zu < %zu particles", who, capacity, N), PIC_ERR_CAPACITY);
  }
  if (capacity >= 0xFFFFFFF0ull) {
    cleanup_tmp();
    cudaFree(off);
    return (set_error("%s: capacity exceeds the 32-bit store", who), PIC_ERR_CAPACITY);
  }
  pic_status r = scan_u32(counts, off, C, sums, total, nullptr, st);
  cleanup_tmp();
  if (r != PIC_OK) {
    cudaFree(off);
    return r;
  }
  pic_particles_s* p = store_alloc(mesh->dim, n_props, C, capacity, off);
  if (!p) return PIC_ERR_OOM;
  p->mesh = mesh;
  p->stream = st;
  DevCounters h{};
  h.n_alive = (uint32_t)N;
  h.n_next = (uint32_t)N;
  cudaError_t e = cudaMemcpyAsync(p->ctr, &h, sizeof(h), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    pic_destroy_particles(p);
    return cuda_fail(e, who);
  }
  p->cur = 0;
  *out = p;
  *n_out = N;
  return PIC_OK;
}

}  // namespace pic

extern "C" pic_status pic_seed_particles(pic_mesh mesh, const uint32_t* per_cell, uint32_t uniform_count, uint64_t seed,
                                         uint64_t first_id, int n_props, size_t capacity, void* stream,
                                         pic_particles* out) {
  if (!out) return (set_error("pic_seed_particles: out is NULL"), PIC_ERR_ARG);
  *out = nullptr;
  if (!mesh) return (set_error("pic_seed_particles: null mesh"), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  pic_particles_s* p = nullptr;
  size_t N = 0;
  pic_status r = seed_prepare(mesh, per_cell, uniform_count, n_props, capacity, st, "pic_seed_particles", &p, &N);
  if (r != PIC_OK) return r;
  const uint32_t C = mesh->C;
  const MeshView m = mesh_view(mesh);
  const int grid = (int)((C + 127) / 128 < 8192 ? (C + 127) / 128 : 8192);
  if (mesh->dim == 2)
    seed_kernel<2><<<grid, 128, 0, st>>>(m, store_view(p, 0), p->cell_off, seed, first_id, 0u);
  else
    seed_kernel<3><<<grid, 128, 0, st>>>(m, store_view(p, 0), p->cell_off, seed, first_id, 0u);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    pic_destroy_particles(p);
    return cuda_fail(e, "pic_seed_particles: seed kernel");
  }
  *out = p;
  return PIC_OK;
}

extern "C" pic_status pic_set_properties(pic_particles p, int prop, const double* values, void* stream) {
  if (!p || !values) return (set_error("pic_set_properties: null argument"), PIC_ERR_ARG);
  if (prop < 0 || prop >= p->n_props) return (set_error("pic_set_properties: property %d out of range", prop), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  {
    const pic_status r0 = settle_order(p, st);
    if (r0 != PIC_OK) return r0;
  }
  set_prop_kernel<<<1024, 256, 0, st>>>(p->props[p->cur] + (size_t)prop * p->capacity, values, p->ctr);
  count_launches(1);
  PIC_CUDA(cudaGetLastError());
  return PIC_OK;
}

static pic_status read_counters(pic_particles p, DevCounters* h) {
  PIC_CUDA(cudaDeviceSynchronize());
  PIC_CUDA(cudaMemcpy(h, p->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost));
  return PIC_OK;
}

extern "C" pic_status pic_get_state(pic_particles p, size_t* n_alive, size_t* n_lost, uint32_t* status_word) {
  if (!p) return (set_error("pic_get_state: null handle"), PIC_ERR_ARG);
  DevCounters h;
  pic_status r = read_counters(p, &h);
  if (r != PIC_OK) return r;
  if (n_alive) *n_alive = h.n_alive;
  if (n_lost) *n_lost = (size_t)h.lost_total;
  if (status_word) *status_word = h.status;
  return PIC_OK;
}

extern "C" pic_status pic_get_stats(pic_particles p, uint64_t* particle_steps, uint64_t* walks, uint64_t* global_searches,
                                    uint64_t* newton_iterations) {
  if (!p) return (set_error("pic_get_stats: null handle"), PIC_ERR_ARG);
  DevCounters h;
  pic_status r = read_counters(p, &h);
  if (r != PIC_OK) return r;
  if (particle_steps) *particle_steps = h.particle_steps;
  if (walks) *walks = h.walks;
  if (global_searches) *global_searches = h.global_searches;
  if (newton_iterations) *newton_iterations = h.newton_iterations;
  return PIC_OK;
}

extern "C" pic_status pic_get_counters(pic_particles p, uint64_t* values, int n_values) {
  if (!p || (!values && n_values > 0) || n_values < 0) return (set_error("pic_get_counters: bad argument"), PIC_ERR_ARG);
  DevCounters h;
  pic_status r = read_counters(p, &h);
  if (r != PIC_OK) return r;
  const uint64_t v[PIC_N_COUNTERS] = {h.particle_steps, h.walks, h.global_searches, h.newton_iterations,
                                      h.lost_total, h.fallback64, h.walk64, h.deferred};
  for (int k = 0; k < n_values && k < PIC_N_COUNTERS; ++k) values[k] = v[k];
  return PIC_OK;
}

extern "C" pic_status pic_export(pic_particles p, double* x, double* xhat, uint64_t* id, uint32_t* cell, double* props,
                                 void* stream) {
  if (!p) return (set_error("pic_export: null handle"), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  {
    const pic_status r0 = settle_order(p, st);
    if (r0 != PIC_OK) return r0;
  }
  DevCounters h;
  pic_status r = read_counters(p, &h);
  if (r != PIC_OK) return r;
  const size_t N = h.n_alive, cap = p->capacity;
  const int c = p->cur;
  if (N == 0) return PIC_OK;
  for (int a = 0; a < p->dim; ++a) {
    if (x) PIC_CUDA(cudaMemcpyAsync(x + a * N, p->x[c] + a * cap, sizeof(double) * N, cudaMemcpyDefault, st));
  }
  if (xhat) {
    cudaPointerAttributes at;
    const bool dev = cudaPointerGetAttributes(&at, xhat) == cudaSuccess && at.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    double* tmp = xhat;
    if (!dev) PIC_CUDA(cudaMallocAsync((void**)&tmp, sizeof(double) * p->dim * N, st));
    xhat_to_double_kernel<<<1024, 256, 0, st>>>(p->xhat[c], tmp, cap, N, p->dim);
    PIC_CUDA(cudaGetLastError());
    if (!dev) {
      PIC_CUDA(cudaMemcpyAsync(xhat, tmp, sizeof(double) * p->dim * N, cudaMemcpyDefault, st));
      PIC_CUDA(cudaFreeAsync(tmp, st));
    }
  }
  if (id) PIC_CUDA(cudaMemcpyAsync(id, p->id[c], sizeof(uint64_t) * N, cudaMemcpyDefault, st));
  if (cell) PIC_CUDA(cudaMemcpyAsync(cell, p->cell[c], sizeof(uint32_t) * N, cudaMemcpyDefault, st));
  for (int q = 0; q < p->n_props && props; ++q)
    PIC_CUDA(cudaMemcpyAsync(props + q * N, p->props[c] + q * cap, sizeof(double) * N, cudaMemcpyDefault, st));
  return PIC_OK;
}

extern "C" pic_status pic_cell_offsets(pic_particles p, uint32_t* off, void* stream) {
  if (!p || !off) return (set_error("pic_cell_offsets: null argument"), PIC_ERR_ARG);
  PIC_CUDA(cudaMemcpyAsync(off, p->cell_off, sizeof(uint32_t) * ((size_t)p->C + 1), cudaMemcpyDefault,
                           (cudaStream_t)stream));
  return PIC_OK;
}
