// transfer.cu -- particle -> field transfers of Sec. 2.7 beyond cell
// averages, both linear in the number of particles because the store is
// sorted by cell:
//   (iv) shape-function-weighted averages at the mesh vertices,
//        p_v = sum_i phi_v(x_i) p_i / sum_i phi_v(x_i) over the particles of
//        the cells around v, phi_v the (bi/tri)linear nodal basis function
//   (v)  per-cell linear least squares in reference coordinates,
//        f(x-hat) = c_0 + sum_j c_{j+1} (x-hat_j - 1/2)
// Both fold the particles in store order; no atomics, so the results are
// reproducible run to run.  The vertex sums are formed per cell first and
// the cells' partial sums then added in increasing cell index, which rounds
// differently from one left fold over the support (the definition) by a few
// ulps of the sum.
#include "pic_internal.cuh"

namespace pic {

__device__ __forceinline__ double xhat64(const float2* __restrict__ xh, size_t idx) {
  const float2 v = xh[idx];
  return (double)v.x + (double)v.y;
}

// Two phases, both deterministic.
// Phase 1, thread per cell: each particle of the cell is read once and its
// 2^D corner weights (the tensor product of (1 - t_a, t_a), multiplied in
// axis order) are folded, in store order, into the cell's partial sums
//   num[c][K] = sum w_c(x-hat_i) p_i,   den[c][K] = sum w_c(x-hat_i)
// stored corner-major ([c][C]) so that the phase-2 reads of a warp coalesce.
template <int D>
__global__ void __launch_bounds__(128) vertex_partial_kernel(const uint32_t* __restrict__ cell_off,
                                                             const float2* __restrict__ xh, const double* __restrict__ prop,
                                                             uint32_t C, size_t cap, double* __restrict__ part,
                                                             DevCounters* __restrict__ ctr) {
  constexpr int NC = 1 << D;
  for (uint32_t K = blockIdx.x * blockDim.x + threadIdx.x; K < C; K += gridDim.x * blockDim.x) {
    const uint32_t beg = cell_off[K], end = cell_off[K + 1];
    double num[NC], den[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) num[c] = den[c] = 0.0;
    if (end > cap || beg > end) {
      latch_status(ctr, PIC_STATUS_BOUNDS);
    } else {
      for (uint32_t i = beg; i < end; ++i) {
        double t[D];
#pragma unroll
        for (int a = 0; a < D; ++a) t[a] = xhat64(xh, a * cap + i);
        const double p = prop[i];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          double w = 1.0;
#pragma unroll
          for (int a = 0; a < D; ++a) w *= ((c >> a) & 1) ? t[a] : 1.0 - t[a];
          num[c] += w * p;
          den[c] += w;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      part[(size_t)c * C + K] = num[c];
      part[(size_t)(NC + c) * C + K] = den[c];
    }
  }
}

// Phase 2, thread per vertex: the partial sums of the cells around the
// vertex, added in increasing cell index.
template <int D>
__global__ void __launch_bounds__(256) vertex_gather_kernel(const __grid_constant__ MeshView m, const double* __restrict__ part,
                                                            double empty_fill, double* __restrict__ avg,
                                                            double* __restrict__ weight) {
  constexpr int NC = 1 << D;
  const uint32_t nv = (uint32_t)m.nverts, C = m.C;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    int vc[3];
    vc[0] = (int)(v % (uint32_t)m.nv[0]);
    const uint32_t r = v / (uint32_t)m.nv[0];
    vc[1] = D == 3 ? (int)(r % (uint32_t)m.nv[1]) : (int)r;
    vc[2] = D == 3 ? (int)(r / (uint32_t)m.nv[1]) : 0;
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int o = 0; o < NC; ++o) {
      // bit a of o is the offset along axis a (x fastest, the last axis
      // slowest), so the cells come in increasing index
      int c[3] = {0, 0, 0}, corner = 0;
      bool ok = true;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        c[a] = vc[a] - 1 + ((o >> a) & 1);
        ok = ok && c[a] >= 0 && c[a] < m.n[a];
        corner |= (vc[a] - c[a]) << a;
      }
      if (!ok) continue;
      const uint32_t K = cell_index<D>(m, c[0], c[1], c[2]);
      num += part[(size_t)corner * C + K];
      den += part[(size_t)(NC + corner) * C + K];
    }
    avg[v] = den > 0.0 ? num / den : empty_fill;
    if (weight) weight[v] = den;
  }
}

// Thread per cell: normal equations (A^T A) c = A^T p of the cell's design
// matrix, rows (1, x-hat_i - 1/2), folded in store order; Gaussian
// elimination with partial pivoting; the mean where the cell has at most D
// particles or a pivot is <= 1e-12 of the largest diagonal entry.
template <int D>
__global__ void __launch_bounds__(128) lsq_linear_kernel(const uint32_t* __restrict__ cell_off,
                                                         const float2* __restrict__ xh, const double* __restrict__ prop,
                                                         uint32_t C, size_t cap, double empty_fill,
                                                         double* __restrict__ coef, uint32_t* __restrict__ count,
                                                         DevCounters* __restrict__ ctr) {
  constexpr int NB = D + 1;
  for (uint32_t K = blockIdx.x * blockDim.x + threadIdx.x; K < C; K += gridDim.x * blockDim.x) {
    const uint32_t beg = cell_off[K], end = cell_off[K + 1];
    if (end > cap || beg > end) {
      latch_status(ctr, PIC_STATUS_BOUNDS);
      continue;
    }
    double M[NB][NB + 1], sum = 0.0;
#pragma unroll
    for (int r = 0; r < NB; ++r)
#pragma unroll
      for (int q = 0; q <= NB; ++q) M[r][q] = 0.0;
    for (uint32_t i = beg; i < end; ++i) {
      double a[NB];
      a[0] = 1.0;
#pragma unroll
      for (int j = 0; j < D; ++j) a[j + 1] = xhat64(xh, j * cap + i) - 0.5;
      const double p = prop[i];
#pragma unroll
      for (int r = 0; r < NB; ++r) {
#pragma unroll
        for (int q = r; q < NB; ++q) M[r][q] += a[r] * a[q];  // upper triangle; a[r] a[q] = a[q] a[r]
        M[r][NB] += a[r] * p;
      }
      sum += p;
    }
#pragma unroll
    for (int r = 1; r < NB; ++r)
#pragma unroll
      for (int q = 0; q < r; ++q) M[r][q] = M[q][r];
    const uint32_t n = end - beg;
    double c[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) c[r] = 0.0;
    if (n == 0) {
      c[0] = empty_fill;
    } else {
      bool ok = n > (uint32_t)D;
      double dmax = 0.0;
#pragma unroll
      for (int r = 0; r < NB; ++r) dmax = M[r][r] > dmax ? M[r][r] : dmax;
#pragma unroll
      for (int col = 0; col < NB; ++col) {
        if (!ok) break;
        int piv = col;
#pragma unroll
        for (int r = col + 1; r < NB; ++r)
          if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
        if (!(fabs(M[piv][col]) > 1e-12 * dmax)) {
          ok = false;
          break;
        }
        if (piv != col) {
#pragma unroll
          for (int q = 0; q <= NB; ++q) {
            const double t = M[col][q];
            M[col][q] = M[piv][q];
            M[piv][q] = t;
          }
        }
#pragma unroll
        for (int r = col + 1; r < NB; ++r) {
          const double f = M[r][col] / M[col][col];
#pragma unroll
          for (int q = col; q <= NB; ++q) M[r][q] -= f * M[col][q];
        }
      }
      if (ok) {
#pragma unroll
        for (int r = NB - 1; r >= 0; --r) {
          double s = M[r][NB];
#pragma unroll
          for (int q = r + 1; q < NB; ++q) s -= M[r][q] * c[q];
          c[r] = s / M[r][r];
        }
      } else {
        c[0] = sum / (double)n;
      }
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) coef[(size_t)r * C + K] = c[r];
    if (count) count[K] = n;
  }
}

static int transfer_grid(size_t n, int block) {
  size_t g = (n + block - 1) / block;
  const size_t cap = (size_t)num_sms() * 16;
  if (g > cap) g = cap;
  return (int)(g ? g : 1);
}

}  // namespace pic

using namespace pic;

extern "C" pic_status pic_interpolate_to_vertices(pic_particles p, pic_mesh mesh, int prop, double* avg,
                                                  double* weight, double empty_fill, void* stream) {
  if (!p || !mesh || !avg) return (set_error("pic_interpolate_to_vertices: null argument"), PIC_ERR_ARG);
  if (p->mesh != mesh) return (set_error("pic_interpolate_to_vertices: mesh mismatch"), PIC_ERR_ARG);
  if (prop < 0 || prop >= p->n_props)
    return (set_error("pic_interpolate_to_vertices: property %d out of range", prop), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  {
    const pic_status r0 = settle_order(p, st);
    if (r0 != PIC_OK) return r0;
  }
  const MeshView m = mesh_view(mesh);
  if (!p->xfer) {
    const size_t bytes = sizeof(double) * 2 * ((size_t)1 << mesh->dim) * (size_t)p->C;
    if (cudaMalloc(&p->xfer, bytes) != cudaSuccess) {
      cudaGetLastError();
      p->xfer = nullptr;
      return (set_error("pic_interpolate_to_vertices: cannot allocate %zu bytes", bytes), PIC_ERR_OOM);
    }
  }
  const double* pv = p->props[p->cur] + (size_t)prop * p->capacity;
  const int g1 = transfer_grid(p->C, 128), g2 = transfer_grid((size_t)m.nverts, 256);
  if (mesh->dim == 2) {
    vertex_partial_kernel<2><<<g1, 128, 0, st>>>(p->cell_off, p->xhat[p->cur], pv, p->C, p->capacity, p->xfer,
                                                 p->ctr);
    vertex_gather_kernel<2><<<g2, 256, 0, st>>>(m, p->xfer, empty_fill, avg, weight);
  } else {
    vertex_partial_kernel<3><<<g1, 128, 0, st>>>(p->cell_off, p->xhat[p->cur], pv, p->C, p->capacity, p->xfer,
                                                 p->ctr);
    vertex_gather_kernel<3><<<g2, 256, 0, st>>>(m, p->xfer, empty_fill, avg, weight);
  }
  count_launches(2);
  PIC_CUDA(cudaGetLastError());
  return PIC_OK;
}

extern "C" pic_status pic_project_linear(pic_particles p, pic_mesh mesh, int prop, double* coef, uint32_t* count,
                                         double empty_fill, void* stream) {
  if (!p || !mesh || !coef) return (set_error("pic_project_linear: null argument"), PIC_ERR_ARG);
  if (p->mesh != mesh) return (set_error("pic_project_linear: mesh mismatch"), PIC_ERR_ARG);
  if (prop < 0 || prop >= p->n_props)
    return (set_error("pic_project_linear: property %d out of range", prop), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  {
    const pic_status r0 = settle_order(p, st);
    if (r0 != PIC_OK) return r0;
  }
  const double* pv = p->props[p->cur] + (size_t)prop * p->capacity;
  const int g = transfer_grid(p->C, 128);
  if (mesh->dim == 2)
    lsq_linear_kernel<2><<<g, 128, 0, st>>>(p->cell_off, p->xhat[p->cur], pv, p->C, p->capacity, empty_fill, coef,
                                            count, p->ctr);
  else
    lsq_linear_kernel<3><<<g, 128, 0, st>>>(p->cell_off, p->xhat[p->cur], pv, p->C, p->capacity, empty_fill, coef,
                                            count, p->ctr);
  count_launches(1);
  PIC_CUDA(cudaGetLastError());
  return PIC_OK;
}
