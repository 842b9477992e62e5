// generate.cu -- particle generation with a density and from prescribed
// locations (Sec. 2.2 of Gassmoeller et al., arXiv 1612.03369).
//
//   pic_cell_weights       w_K = int_K rho_h dx, rho_h the (bi/tri)linear
//                          interpolant of vertex values; tensor 2-point Gauss
//                          (exact: the integrand has degree <= 3 per axis)
//   pic_draw_cell_counts   N draws over the accumulated weights (the listing's
//                          second and third loops, on one GPU)
//   pic_seed_particles_mh  in-cell Metropolis-Hastings with target
//                          rho-hat = rho_h(Phi_K(x-hat)) |det grad-hat Phi_K|
//                          and uniform proposals, thinned by J
//   pic_import_particles   owner search for every prescribed point, ids in
//                          input order among the points found
//
// The decisions that turn floating point into integers (which cell a draw
// falls in, whether a proposal is accepted) must not depend on the device:
// the accumulated weights are one left fold, and rho-hat is evaluated as a
// fixed sequence of correctly rounded IEEE operations (the _rn intrinsics
// keep the compiler from contracting or reordering them):
//   rho_h   = sum over local vertices v = 0..2^D-1 of rho_v * w_v(t),
//             w_v = product over axes a = 0..D-1 of (bit a of v ? t_a : 1 - t_a)
//   J_ij    = sum over v of X_{v,i} * dw_v/dt_j (the same product with the
//             factor of axis j replaced by +1 or -1)
//   det J   = J00 J11 - J01 J10 (2D);
//             J00 (J11 J22 - J12 J21) + J01 (J12 J20 - J10 J22)
//             + J02 (J10 J21 - J11 J20), summed left to right (3D)
//   rho-hat = rho_h * |det J|
#include <cmath>
#include <cstdlib>

#include "pic_internal.cuh"
#include "seed.cuh"

namespace pic {

template <int D>
__device__ __forceinline__ int64_t local_vertex(const MeshView& m, const int c[3], int v) {
  return (int64_t)(c[0] + (v & 1)) +
         (int64_t)m.nv[0] * ((int64_t)(c[1] + ((v >> 1) & 1)) + (D == 3 ? (int64_t)m.nv[1] * (c[2] + ((v >> 2) & 1)) : 0));
}

template <int D>
__device__ __forceinline__ double vweight_rn(int v, const double t[D], int skip = -1) {
  double w = 1.0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const bool hi = (v >> a) & 1;
    const double f = (a == skip) ? (hi ? 1.0 : -1.0) : (hi ? t[a] : __dsub_rn(1.0, t[a]));
    w = __dmul_rn(w, f);
  }
  return w;
}

template <int D>
__device__ double rho_hat_rn(const MeshView& m, uint32_t K, const double* __restrict__ rho, const double t[D]) {
  int c[3];
  cell_ijk<D>(m, K, c);
  double r = 0.0;
#pragma unroll
  for (int v = 0; v < (1 << D); ++v) r = __dadd_rn(r, __dmul_rn(__ldg(rho + local_vertex<D>(m, c, v)), vweight_rn<D>(v, t)));
  double J[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double s = 0.0;
#pragma unroll
      for (int v = 0; v < (1 << D); ++v)
        s = __dadd_rn(s, __dmul_rn(__ldg(m.X + i * m.nverts + local_vertex<D>(m, c, v)), vweight_rn<D>(v, t, j)));
      J[i][j] = s;
    }
  double det;
  if constexpr (D == 2) {
    det = __dsub_rn(__dmul_rn(J[0][0], J[1][1]), __dmul_rn(J[0][1], J[1][0]));
  } else {
    const double c0 = __dsub_rn(__dmul_rn(J[1][1], J[2][2]), __dmul_rn(J[1][2], J[2][1]));
    const double c1 = __dsub_rn(__dmul_rn(J[1][2], J[2][0]), __dmul_rn(J[1][0], J[2][2]));
    const double c2 = __dsub_rn(__dmul_rn(J[1][0], J[2][1]), __dmul_rn(J[1][1], J[2][0]));
    det = __dadd_rn(__dadd_rn(__dmul_rn(J[0][0], c0), __dmul_rn(J[0][1], c1)), __dmul_rn(J[0][2], c2));
  }
  return __dmul_rn(r, fabs(det));
}

// x = Phi_K(t) = sum_v X_v w_v(t), in the same rounded sequence.
template <int D>
__device__ __forceinline__ void phi_rn(const MeshView& m, uint32_t K, const double t[D], double x[D]) {
  int c[3];
  cell_ijk<D>(m, K, c);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double s = 0.0;
#pragma unroll
    for (int v = 0; v < (1 << D); ++v)
      s = __dadd_rn(s, __dmul_rn(__ldg(m.X + i * m.nverts + local_vertex<D>(m, c, v)), vweight_rn<D>(v, t)));
    x[i] = s;
  }
}

__device__ __forceinline__ double unit53(uint64_t r) { return (double)(r >> 11) * 0x1.0p-53; }

// ------------------------------------------------------------ cell weights

template <int D>
__global__ void __launch_bounds__(128) cell_weights_kernel(const __grid_constant__ MeshView m, const double* __restrict__ rho,
                                                           double* __restrict__ w) {
  const double g0 = __dsub_rn(0.5, __ddiv_rn(0.5, __dsqrt_rn(3.0)));
  const double g1 = __dadd_rn(0.5, __ddiv_rn(0.5, __dsqrt_rn(3.0)));
  for (uint32_t K = blockIdx.x * blockDim.x + threadIdx.x; K < m.C; K += gridDim.x * blockDim.x) {
    double s = 0.0;
#pragma unroll 1
    for (int q = 0; q < (1 << D); ++q) {
      double t[D];
#pragma unroll
      for (int a = 0; a < D; ++a) t[a] = ((q >> a) & 1) ? g1 : g0;
      double wq = 1.0;
#pragma unroll
      for (int a = 0; a < D; ++a) wq = __dmul_rn(wq, 0.5);
      s = __dadd_rn(s, __dmul_rn(wq, rho_hat_rn<D>(m, K, rho, t)));
    }
    w[K] = s;
  }
}

// ------------------------------------------------------------ cell counts

struct DrawInfo {
  double W;          // total weight
  long long last;    // last cell of positive weight, -1 if none
  unsigned bad;      // a weight was negative or not finite
};

// The accumulated weights as one left fold, by one warp: every lane runs the
// same sequential sum over a 32-value chunk read with one coalesced load
// (values broadcast by shuffles), lane q keeps the q-th partial sum and the
// chunk is stored coalesced.  The next chunk is loaded before the fold.
__global__ void __launch_bounds__(32) accumulate_weights_kernel(const double* __restrict__ w, uint32_t C,
                                                                double* __restrict__ acc, DrawInfo* __restrict__ info) {
  const int lane = threadIdx.x;
  double s = 0.0;
  long long last = -1;
  unsigned bad = 0;
  double next = lane < (int)C ? w[lane] : 0.0;
  for (uint32_t base = 0; base < C; base += 32) {
    const double v = next;
    const uint32_t nb = base + 32 + lane;
    next = nb < C ? w[nb] : 0.0;
    const uint32_t k = base + lane;
    if (k < C) {
      if (!(v >= 0.0) || !isfinite(v)) bad = 1;
      if (v > 0.0) last = k;
    }
    double mine = 0.0;
    const int lim = (C - base) < 32u ? (int)(C - base) : 32;
    for (int q = 0; q < lim; ++q) {
      s = __dadd_rn(s, __shfl_sync(0xffffffffu, v, q));
      if (lane == q) mine = s;
    }
    if (k < C) acc[k] = mine;
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  long long lmax = last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long other = __shfl_xor_sync(0xffffffffu, lmax, o);
    lmax = other > lmax ? other : lmax;
  }
  if (lane == 0) {
    info->W = s;
    info->last = lmax;
    info->bad = bad;
  }
}

// Draw i: u = top 53 bits of SplitMix64 output i times 2^-53, r = W u, the
// first cell with acc > r (or the last cell of positive weight if W u
// rounded up to W).
__global__ void __launch_bounds__(256) draw_cells_kernel(const double* __restrict__ acc, uint32_t C,
                                                         const DrawInfo* __restrict__ info, uint64_t n,
                                                         uint64_t seed, uint32_t* __restrict__ counts) {
  const double W = info->W;
  const long long last = info->last;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const double r = __dmul_rn(W, unit53(splitmix64_at(seed, i)));
    uint32_t lo = 0, hi = C;
    while (lo < hi) {
      const uint32_t mid = lo + (hi - lo) / 2;
      if (acc[mid] > r)
        hi = mid;
      else
        lo = mid + 1;
    }
    const long long K = lo < C ? (long long)lo : last;
    if (K >= 0) atomicAdd(counts + K, 1u);
  }
}

// ------------------------------------------------------ Metropolis-Hastings

// Thread per cell: the cell's chain, started at the centre; step st of the
// chain is global step g = J * cell_off[K] + st and uses SplitMix64 outputs
// g (D+1) + a (proposal coordinate a) and g (D+1) + D (acceptance uniform).
// States J, 2J, ... become the cell's particles, in order.
template <int D>
__global__ void __launch_bounds__(128) mh_seed_kernel(const __grid_constant__ MeshView m, const __grid_constant__ StoreView s, const uint32_t* __restrict__ cell_off,
                                                      const double* __restrict__ rho, uint32_t J, uint64_t seed,
                                                      uint64_t first_id) {
  for (uint32_t K = blockIdx.x * blockDim.x + threadIdx.x; K < m.C; K += gridDim.x * blockDim.x) {
    const uint32_t beg = cell_off[K], end = cell_off[K + 1];
    if (end > s.cap || beg >= end) continue;
    double cur[D];
#pragma unroll
    for (int a = 0; a < D; ++a) cur[a] = 0.5;
    double rc = rho_hat_rn<D>(m, K, rho, cur);
    const uint64_t g0 = (uint64_t)J * beg, len = (uint64_t)J * (end - beg);
    uint32_t q = beg;
    uint32_t phase = 0;
    for (uint64_t st = 0; st < len; ++st) {
      const uint64_t g = g0 + st;
      double y[D];
#pragma unroll
      for (int a = 0; a < D; ++a) y[a] = unit53(splitmix64_at(seed, g * (D + 1) + a));
      const double u = unit53(splitmix64_at(seed, g * (D + 1) + D));
      const double ry = rho_hat_rn<D>(m, K, rho, y);
      if (__dmul_rn(u, rc) < ry) {
#pragma unroll
        for (int a = 0; a < D; ++a) cur[a] = y[a];
        rc = ry;
      }
      if (++phase == J) {
        phase = 0;
        double x[D];
        phi_rn<D>(m, K, cur, x);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          s.x[a * s.cap + q] = x[a];
          const float hi = __double2float_rn(cur[a]);
          s.xhat[a * s.cap + q] = make_float2(hi, __double2float_rn(cur[a] - (double)hi));
        }
        s.id[q] = first_id + q;
        s.cell[q] = K;
        for (int p = 0; p < s.n_props; ++p) s.props[(size_t)p * s.cap + q] = 0.0;
        ++q;
      }
    }
  }
}

// ------------------------------------------------------- prescribed points

__global__ void found_flags_kernel(const uint32_t* __restrict__ cell, size_t n, uint32_t C, uint32_t* __restrict__ f) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    f[i] = cell[i] < C ? 1u : 0u;
}

__global__ void import_ids_kernel(const uint32_t* __restrict__ rank, size_t n, uint64_t first_id,
                                  uint64_t* __restrict__ id) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    id[i] = first_id + rank[i];
}

template <int D>
__global__ void import_gather_kernel(const __grid_constant__ StoreView s, const uint32_t* __restrict__ perm, const uint32_t* __restrict__ kept_p,
                                     size_t n, const double* __restrict__ x, const double* __restrict__ xh,
                                     const uint32_t* __restrict__ cell, const uint64_t* __restrict__ id) {
  const uint32_t kept = *kept_p;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < kept; j += gridDim.x * blockDim.x) {
    const uint32_t i = perm[j];
    if (i >= n || j >= s.cap) continue;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      s.x[a * s.cap + j] = x[a * n + i];
      const double t = xh[a * n + i];
      const float hi = __double2float_rn(t);
      s.xhat[a * s.cap + j] = make_float2(hi, __double2float_rn(t - (double)hi));
    }
    s.id[j] = id[i];
    s.cell[j] = cell[i];
    for (int p = 0; p < s.n_props; ++p) s.props[(size_t)p * s.cap + j] = 0.0;
  }
}

static int gen_grid(size_t n, int block) {
  size_t g = (n + block - 1) / block;
  const size_t cap = (size_t)num_sms() * 16;
  if (g > cap) g = cap;
  return (int)(g ? g : 1);
}

}  // namespace pic

using namespace pic;

extern "C" pic_status pic_cell_weights(pic_mesh mesh, const double* rho, double* w, void* stream) {
  if (!mesh || !rho || !w) return (set_error("pic_cell_weights: null argument"), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  const MeshView m = mesh_view(mesh);
  if (mesh->dim == 2)
    cell_weights_kernel<2><<<gen_grid(m.C, 128), 128, 0, st>>>(m, rho, w);
  else
    cell_weights_kernel<3><<<gen_grid(m.C, 128), 128, 0, st>>>(m, rho, w);
  count_launches(1);
  PIC_CUDA(cudaGetLastError());
  return PIC_OK;
}

extern "C" pic_status pic_draw_cell_counts(uint32_t n_cells, const double* w, uint64_t n_particles, uint64_t seed,
                                           uint32_t* counts, void* stream) {
  if (!w || !counts || n_cells == 0) return (set_error("pic_draw_cell_counts: null argument or no cells"), PIC_ERR_ARG);
  if (n_particles >= 0xFFFFFFF0ull)
    return (set_error("pic_draw_cell_counts: %llu particles exceed the 32-bit store",
                      (unsigned long long)n_particles),
            PIC_ERR_CAPACITY);
  cudaStream_t st = (cudaStream_t)stream;
  double* acc = nullptr;
  DrawInfo* info = nullptr;
  if (cudaMalloc(&acc, sizeof(double) * n_cells) != cudaSuccess || cudaMalloc(&info, sizeof(DrawInfo)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(acc);
    cudaFree(info);
    return (set_error("pic_draw_cell_counts: device allocation failed"), PIC_ERR_OOM);
  }
  accumulate_weights_kernel<<<1, 32, 0, st>>>(w, n_cells, acc, info);
  DrawInfo h{};
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, info, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(acc);
    cudaFree(info);
    return cuda_fail(e, "pic_draw_cell_counts: accumulate");
  }
  if (h.bad || !(h.W > 0.0) || !std::isfinite(h.W)) {
    cudaFree(acc);
    cudaFree(info);
    return (set_error("pic_draw_cell_counts: weights must be finite and >= 0 with a positive sum"), PIC_ERR_ARG);
  }
  e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * n_cells, st);
  if (e == cudaSuccess && n_particles > 0) {
    draw_cells_kernel<<<gen_grid((size_t)n_particles, 256), 256, 0, st>>>(acc, n_cells, info, n_particles, seed,
                                                                          counts);
    e = cudaGetLastError();
  }
  count_launches(n_particles > 0 ? 2 : 1);
  cudaFreeAsync(acc, st);
  cudaFreeAsync(info, st);
  if (e != cudaSuccess) return cuda_fail(e, "pic_draw_cell_counts: draws");
  return PIC_OK;
}

extern "C" pic_status pic_seed_particles_mh(pic_mesh mesh, const uint32_t* per_cell, const double* rho,
                                            uint32_t thinning, uint64_t seed, uint64_t first_id, int n_props,
                                            size_t capacity, void* stream, pic_particles* out) {
  if (!out) return (set_error("pic_seed_particles_mh: out is NULL"), PIC_ERR_ARG);
  *out = nullptr;
  if (!mesh || !per_cell || !rho) return (set_error("pic_seed_particles_mh: null argument"), PIC_ERR_ARG);
  if (thinning < 1) return (set_error("pic_seed_particles_mh: thinning must be >= 1"), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  pic_particles_s* p = nullptr;
  size_t N = 0;
  pic_status r = seed_prepare(mesh, per_cell, 0, n_props, capacity, st, "pic_seed_particles_mh", &p, &N);
  if (r != PIC_OK) return r;
  const MeshView m = mesh_view(mesh);
  if (mesh->dim == 2)
    mh_seed_kernel<2><<<gen_grid(m.C, 128), 128, 0, st>>>(m, store_view(p, 0), p->cell_off, rho, thinning, seed,
                                                          first_id);
  else
    mh_seed_kernel<3><<<gen_grid(m.C, 128), 128, 0, st>>>(m, store_view(p, 0), p->cell_off, rho, thinning, seed,
                                                          first_id);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    pic_destroy_particles(p);
    return cuda_fail(e, "pic_seed_particles_mh: kernel");
  }
  *out = p;
  return PIC_OK;
}

extern "C" pic_status pic_import_particles(pic_mesh mesh, size_t n, const double* x, uint64_t first_id, int n_props,
                                           size_t capacity, void* stream, pic_particles* out, size_t* n_outside) {
  if (!out) return (set_error("pic_import_particles: out is NULL"), PIC_ERR_ARG);
  *out = nullptr;
  if (!mesh || (n > 0 && !x)) return (set_error("pic_import_particles: null argument"), PIC_ERR_ARG);
  if (n >= 0xFFFFFFF0ull) return (set_error("pic_import_particles: n exceeds the 32-bit store"), PIC_ERR_CAPACITY);
  if (n_props < 0 || n_props > kMaxProps)
    return (set_error("pic_import_particles: n_props must be in [0, %d]", kMaxProps), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t C = mesh->C;
  const int d = mesh->dim;
  const size_t nn = n > 0 ? n : 1;
  uint32_t *cell = nullptr, *flag = nullptr, *rank = nullptr, *sums = nullptr, *total = nullptr, *perm = nullptr,
           *off = nullptr;
  double* xh = nullptr;
  uint64_t* id = nullptr;
  bool ok = cudaMalloc(&cell, sizeof(uint32_t) * nn) == cudaSuccess &&
            cudaMalloc(&flag, sizeof(uint32_t) * nn) == cudaSuccess &&
            cudaMalloc(&rank, sizeof(uint32_t) * (nn + 1)) == cudaSuccess &&
            cudaMalloc(&sums, scan_scratch_bytes((uint32_t)nn)) == cudaSuccess &&
            cudaMalloc(&total, sizeof(uint32_t) * 2) == cudaSuccess &&
            cudaMalloc(&perm, sizeof(uint32_t) * nn) == cudaSuccess &&
            cudaMalloc(&off, sizeof(uint32_t) * (C + 1)) == cudaSuccess &&
            cudaMalloc(&xh, sizeof(double) * d * nn) == cudaSuccess &&
            cudaMalloc(&id, sizeof(uint64_t) * nn) == cudaSuccess;
  auto release = [&](bool keep_off) {
    cudaFree(cell);
    cudaFree(flag);
    cudaFree(rank);
    cudaFree(sums);
    cudaFree(total);
    cudaFree(perm);
    if (!keep_off) cudaFree(off);
    cudaFree(xh);
    cudaFree(id);
  };
  if (!ok) {
    cudaGetLastError();
    release(false);
    return (set_error("pic_import_particles: device allocation failed"), PIC_ERR_OOM);
  }
  pic_status r = PIC_OK;
  uint32_t kept = 0;
  if (n > 0) {
    r = pic_locate_points(mesh, n, x, nullptr, cell, xh, stream);
    if (r == PIC_OK) {
      found_flags_kernel<<<gen_grid(n, 256), 256, 0, st>>>(cell, n, C, flag);
      r = scan_u32(flag, rank, (uint32_t)n, sums, total, nullptr, st);
    }
    if (r == PIC_OK) {
      import_ids_kernel<<<gen_grid(n, 256), 256, 0, st>>>(rank, n, first_id, id);
      count_launches(2);
      r = pic_sort_by_cell(n, cell, id, C, perm, off, stream);
    }
    if (r == PIC_OK) {
      cudaError_t e = cudaMemcpyAsync(&kept, off + C, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) r = cuda_fail(e, "pic_import_particles: count");
    }
  } else {
    cudaError_t e = cudaMemsetAsync(off, 0, sizeof(uint32_t) * (C + 1), st);
    if (e != cudaSuccess) r = cuda_fail(e, "pic_import_particles: offsets");
  }
  if (r == PIC_OK && capacity == 0) capacity = kept;
  if (r == PIC_OK && capacity < kept)
    r = (set_error("pic_import_particles: capacity %zu < %u particles", capacity, kept), PIC_ERR_CAPACITY);
  if (r != PIC_OK) {
    release(false);
    return r;
  }
  pic_particles_s* p = store_alloc(d, n_props, C, capacity, off);  // takes `off`
  if (!p) {
    release(true);
    return PIC_ERR_OOM;
  }
  p->mesh = mesh;
  p->stream = st;
  DevCounters h{};
  h.n_alive = kept;
  h.n_next = kept;
  cudaError_t e = cudaMemcpyAsync(p->ctr, &h, sizeof(h), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && kept > 0) {
    if (d == 2)
      import_gather_kernel<2><<<gen_grid(kept, 128), 128, 0, st>>>(store_view(p, 0), perm, off + C, n, x, xh, cell, id);
    else
      import_gather_kernel<3><<<gen_grid(kept, 128), 128, 0, st>>>(store_view(p, 0), perm, off + C, n, x, xh, cell, id);
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  release(true);
  if (e != cudaSuccess) {
    pic_destroy_particles(p);
    return cuda_fail(e, "pic_import_particles: gather");
  }
  p->cur = 0;
  if (n_outside) *n_outside = n - kept;
  *out = p;
  return PIC_OK;
}
