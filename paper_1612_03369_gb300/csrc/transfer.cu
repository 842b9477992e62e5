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
#include "df.cuh"
#include "pic_internal.cuh"

namespace pic {

// The arithmetic per particle is double-float on the FP32 pipe (the stored
// x-hat already is a double-float pair; the property is split once): GB300's
// FP64 pipe runs about 1/80 of the FP32 rate, and the FP64 form of these
// kernels was bound by it.  Every product keeps ~2^-47 of its value and the
// sums are compensated (acc_mad, acc_add), so the per-cell sums carry a
// relative error of a few 2^-47 against the FP64 definition.
__device__ __forceinline__ df one_minus(df t) {  // 1 - t
  const df d = two_sum(1.0f, -t.hi);
  return fast_two_sum(d.hi, __fsub_rn(d.lo, t.lo));
}
__device__ __forceinline__ df minus_half(df t) {  // t - 1/2
  const df d = two_sum(t.hi, -0.5f);
  return fast_two_sum(d.hi, __fadd_rn(d.lo, t.lo));
}
__device__ __forceinline__ double df_to_f64(df a) { return (double)a.hi + (double)a.lo; }

// Two phases, both deterministic.
// Phase 1, thread per cell: each particle of the cell is read once and its
// 2^D corner weights (the tensor product of (1 - t_a, t_a), multiplied in
// axis order) are folded, in store order, into the cell's partial sums
//   num[c][K] = sum w_c(x-hat_i) p_i,   den[c][K] = sum w_c(x-hat_i)
// stored as double-float pairs, corner-major ([c][C]) so that the phase-2
// reads of a warp coalesce.
template <int D>
__global__ void __launch_bounds__(128) vertex_partial_kernel(const uint32_t* __restrict__ cell_off,
                                                             const float2* __restrict__ xh, const double* __restrict__ prop,
                                                             uint32_t C, size_t cap, float2* __restrict__ part,
                                                             DevCounters* __restrict__ ctr) {
  constexpr int NC = 1 << D;
  for (uint32_t K = blockIdx.x * blockDim.x + threadIdx.x; K < C; K += gridDim.x * blockDim.x) {
    const uint32_t beg = cell_off[K], end = cell_off[K + 1];
    df_acc num[NC], den[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) num[c] = den[c] = acc_zero();
    if (end > cap || beg > end) {
      latch_status(ctr, PIC_STATUS_BOUNDS);
    } else {
      for (uint32_t i = beg; i < end; ++i) {
        df f[D][2];  // f[a][0] = 1 - t_a, f[a][1] = t_a
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const float2 v = xh[a * cap + i];
          f[a][1] = df_make(v.x, v.y);
          f[a][0] = one_minus(f[a][1]);
        }
        const df p = df_from_double(prop[i]);
        df w01[4];  // the first two axes' products, corner bits 0 and 1
#pragma unroll
        for (int c = 0; c < 4; ++c) w01[c] = df_mul(f[0][c & 1], f[1][(c >> 1) & 1]);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const df w = D == 3 ? df_mul(w01[c & 3], f[D - 1][(c >> 2) & 1]) : w01[c];
          acc_mad(num[c], w, p);
          acc_add(den[c], w);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const df a = acc_result(num[c]), b = acc_result(den[c]);
      part[(size_t)c * C + K] = make_float2(a.hi, a.lo);
      part[(size_t)(NC + c) * C + K] = make_float2(b.hi, b.lo);
    }
  }
}

// Phase 2, thread per vertex: the partial sums of the cells around the
// vertex, added in increasing cell index (double-float), then one FP64
// division.
template <int D>
__global__ void __launch_bounds__(256) vertex_gather_kernel(const __grid_constant__ MeshView m, const float2* __restrict__ part,
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
    df_acc num = acc_zero(), den = acc_zero();
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
      const float2 a = part[(size_t)corner * C + K], b = part[(size_t)(NC + corner) * C + K];
      acc_add(num, df_make(a.x, a.y));
      acc_add(den, df_make(b.x, b.y));
    }
    const double dn = df_to_f64(acc_result(den));
    avg[v] = dn > 0.0 ? df_to_f64(acc_result(num)) / dn : empty_fill;
    if (weight) weight[v] = dn;
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
    // the upper triangle of A^T A, A^T p and sum p, accumulated in
    // double-float (row a = (1, x-hat - 1/2)), then converted once
    df_acc Ma[NB][NB + 1], sa = acc_zero();
#pragma unroll
    for (int r = 0; r < NB; ++r)
#pragma unroll
      for (int q = 0; q <= NB; ++q) Ma[r][q] = acc_zero();
    for (uint32_t i = beg; i < end; ++i) {
      df a[NB];
      a[0] = df_make(1.0f, 0.f);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const float2 v = xh[j * cap + i];
        a[j + 1] = minus_half(df_make(v.x, v.y));
      }
      const df p = df_from_double(prop[i]);
#pragma unroll
      for (int r = 0; r < NB; ++r) {
#pragma unroll
        for (int q = r; q < NB; ++q) {
          if (r == 0)
            acc_add(Ma[r][q], a[q]);  // a[0] = 1
          else
            acc_mad(Ma[r][q], a[r], a[q]);
        }
        if (r == 0)
          acc_add(Ma[r][NB], p);
        else
          acc_mad(Ma[r][NB], a[r], p);
      }
      acc_add(sa, p);
    }
    double M[NB][NB + 1];
#pragma unroll
    for (int r = 0; r < NB; ++r)
#pragma unroll
      for (int q = r; q <= NB; ++q) M[r][q] = df_to_f64(acc_result(Ma[r][q]));
    const double sum = df_to_f64(acc_result(sa));
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
      double dmax = 0.0, invd[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) dmax = M[r][r] > dmax ? M[r][r] : dmax;
#pragma unroll
      for (int col = 0; col < NB; ++col) {
        if (!ok) break;
        int piv = col;
        double best = fabs(M[col][col]);
#pragma unroll
        for (int r = col + 1; r < NB; ++r)
          if (fabs(M[r][col]) > best) {
            best = fabs(M[r][col]);
            piv = r;
          }
        if (!(best > 1e-12 * dmax)) {
          ok = false;
          break;
        }
        // the swap with compile-time row indices keeps M in registers
#pragma unroll
        for (int r = col + 1; r < NB; ++r)
          if (r == piv) {
#pragma unroll
            for (int q = 0; q <= NB; ++q) {
              const double t = M[col][q];
              M[col][q] = M[r][q];
              M[r][q] = t;
            }
          }
        // one reciprocal per pivot (FP64 divisions are sequences on the FP64
        // pipe; the solve's rounding is covered by the kappa-scaled bound)
        const double inv = 1.0 / M[col][col];
        invd[col] = inv;
#pragma unroll
        for (int r = col + 1; r < NB; ++r) {
          const double f = M[r][col] * inv;
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
          c[r] = s * invd[r];
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
  float2* part = reinterpret_cast<float2*>(p->xfer);  // [2 * 2^dim][C] double-float pairs
  if (mesh->dim == 2) {
    vertex_partial_kernel<2><<<g1, 128, 0, st>>>(p->cell_off, p->xhat[p->cur], pv, p->C, p->capacity, part, p->ctr);
    vertex_gather_kernel<2><<<g2, 256, 0, st>>>(m, part, empty_fill, avg, weight);
  } else {
    vertex_partial_kernel<3><<<g1, 128, 0, st>>>(p->cell_off, p->xhat[p->cur], pv, p->C, p->capacity, part, p->ctr);
    vertex_gather_kernel<3><<<g2, 256, 0, st>>>(m, part, empty_fill, avg, weight);
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
