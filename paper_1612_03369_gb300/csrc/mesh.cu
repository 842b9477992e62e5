// mesh.cu -- mesh and velocity handles: vertex upload, per-cell bounding
// boxes for the all-cells search, and the Q2 nodal velocity (Sec. 2.3).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "df.cuh"
#include "fastpath.cuh"
#include "pic_internal.cuh"

namespace pic {

// Padded bounding box of every cell (lo xyz, hi xyz): the all-cells search
// of Sec. 2.4 only runs the inverse map in cells whose box holds the point.
// The FP32 copy is rounded outward and widened by four ulps, so that a test
// of a double-float point's high part against it never rejects a point of
// the FP64 box.
__device__ __forceinline__ float widen_down(double v) {
  float f = __double2float_rd(v);
  for (int k = 0; k < 4; ++k) f = nextafterf(f, -INFINITY);
  return f;
}
__device__ __forceinline__ float widen_up(double v) {
  float f = __double2float_ru(v);
  for (int k = 0; k < 4; ++k) f = nextafterf(f, INFINITY);
  return f;
}

template <int D>
__global__ void cell_bbox_kernel(const __grid_constant__ MeshView m, double* __restrict__ bbox,
                                 float4* __restrict__ bbox32) {
  for (uint32_t K = blockIdx.x * blockDim.x + threadIdx.x; K < m.C; K += gridDim.x * blockDim.x) {
    CellGeom<D> g;
    load_cell<D>(m, K, g);
    float lo32[3], hi32[3];
    for (int a = 0; a < 3; ++a) {
      double lo = 0.0, hi = 0.0;
      if (a < D) {
        lo = hi = g.x0[a];
        for (int v = 1; v < (1 << D); ++v) {
          lo = fmin(lo, g.x0[a] + g.e[v][a]);
          hi = fmax(hi, g.x0[a] + g.e[v][a]);
        }
        const double pad = 1e-6 * (hi - lo);
        lo -= pad;
        hi += pad;
      }
      bbox[6 * (size_t)K + a] = lo;
      bbox[6 * (size_t)K + 3 + a] = hi;
      lo32[a] = widen_down(lo);
      hi32[a] = widen_up(hi);
    }
    bbox32[2 * (size_t)K] = make_float4(lo32[0], lo32[1], lo32[2], 0.f);
    bbox32[2 * (size_t)K + 1] = make_float4(hi32[0], hi32[1], hi32[2], 0.f);
  }
}

__device__ __forceinline__ float2 split_df(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}

// Per-cell map block: X_0 and the monomial coefficients of Phi_K - X_0
// (3D: t0, t1, t2, t0t1, t0t2, t1t2, t0t1t2; 2D: t0, t1, t0t1), each as a
// double-float.  With e_v = X_v - X_0 (v = bit pattern of the vertex):
//   a_t0 = e1, a_t1 = e2, a_t2 = e4, a_t0t1 = e3 - e1 - e2,
//   a_t0t2 = e5 - e1 - e4, a_t1t2 = e6 - e2 - e4,
//   a_t0t1t2 = e7 - e3 - e5 - e6 + e1 + e2 + e4.
// Stored as the NF high parts (X_0, then a_k,c in (k, c) order) followed by
// the NF low parts in the same order, so that the FP32 Newton iterations
// read only the first half.
template <int D>
__global__ void cell_block_kernel(const __grid_constant__ MeshView m, float* __restrict__ blk) {
  constexpr int NK = (1 << D) - 1;
  constexpr int NF = D + NK * D;
  for (uint32_t K = blockIdx.x * blockDim.x + threadIdx.x; K < m.C; K += gridDim.x * blockDim.x) {
    CellGeom<D> g;
    load_cell<D>(m, K, g);
    float* out = blk + (size_t)K * 2 * NF;
    auto put = [&](int idx, double v) {
      const float2 p = split_df(v);
      out[idx] = p.x;
      out[NF + idx] = p.y;
    };
    for (int a = 0; a < D; ++a) put(a, g.x0[a]);
    for (int a = 0; a < D; ++a) {
      double coef[NK];
      if constexpr (D == 2) {
        coef[0] = g.e[1][a];
        coef[1] = g.e[2][a];
        coef[2] = g.e[3][a] - g.e[1][a] - g.e[2][a];
      } else {
        coef[0] = g.e[1][a];
        coef[1] = g.e[2][a];
        coef[2] = g.e[4][a];
        coef[3] = g.e[3][a] - g.e[1][a] - g.e[2][a];
        coef[4] = g.e[5][a] - g.e[1][a] - g.e[4][a];
        coef[5] = g.e[6][a] - g.e[2][a] - g.e[4][a];
        coef[6] = g.e[7][a] - g.e[3][a] - g.e[5][a] - g.e[6][a] + g.e[1][a] + g.e[2][a] + g.e[4][a];
      }
      for (int k = 0; k < NK; ++k) put(D + k * D + a, coef[k]);
    }
  }
}

// Index of node (2i, 2j, 2k), the first Q2 node of cell (i, j, k).
template <int D>
__global__ void cell_qbase_kernel(const __grid_constant__ MeshView m, uint32_t* __restrict__ qbase) {
  for (uint32_t K = blockIdx.x * blockDim.x + threadIdx.x; K < m.C; K += gridDim.x * blockDim.x) {
    int c[3];
    cell_ijk<D>(m, K, c);
    qbase[K] = (uint32_t)(2 * (int64_t)c[0] + (int64_t)m.nq[0] * (2 * c[1] + (D == 3 ? (int64_t)m.nq[1] * 2 * c[2] : 0)));
  }
}

// U [comp][node] FP64 -> U2 [node][comp] double-float.
__global__ void to_df_nodes_kernel(const double* __restrict__ U, float2* __restrict__ U2, int dim, size_t nnodes) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nnodes * dim; i += (size_t)gridDim.x * blockDim.x) {
    const size_t node = i / dim, comp = i % dim;
    U2[i] = split_df(U[comp * nnodes + node]);
  }
}

// Per-cell monomial coefficients of the Q2 field about the cell centre:
// with s = t - 1/2 the 1D Lagrange basis on {0, 1/2, 1} is
//   l_0 = -s + 2 s^2,   l_1 = 1 - 4 s^2,   l_2 = s + 2 s^2,
// i.e. l_a(s) = sum_p T[p][a] s^p with T = [[0, 1, 0], [-1, 0, 1], [2, -4, 2]],
// so u_c(s) = sum_{p,q,r} C_pqr s0^p s1^q s2^r with C = (T x T x T) U_cell.
// Each slice of 5 float4 holds the high parts of C[r][q][p] at q*3 + p
// (the tenth is zero) and then the ten low parts, so that the FP32 form
// reads only the first three float4.
// Computed in double-float on the FP32 pipe from the nodal double-float copy
// U2 (each node converted once), one axis at a time (scalings by 2 and 4 are
// exact; sums and differences carry ~2^-47 of their operands, the order of
// the storage rounding itself), stored as double-float pairs:
// per cell and component, slice r (3 in 3D, 1 in 2D) holds C[r][q][p] at
// pair q*3 + p of 5 float4 (the tenth pair is zero).
__device__ __forceinline__ void t_axis(df v0, df v1, df v2, df& c0, df& c1, df& c2) {
  c0 = v1;
  c1 = df_sub(v2, v0);
  c2 = df_sub(df_scale2(df_add(v0, v2), 2.0f), df_scale2(v1, 4.0f));
}

// With Qf given, the block also writes the coefficients' high parts, per
// cell and component in the order r*9 + q*3 + p, padded to 28 (3D) or 12
// (2D) floats: the FP32-basis form's table.
template <int D>
__global__ void __launch_bounds__(32 * D) q2_coeff_kernel(const __grid_constant__ MeshView m, const float2* __restrict__ U2,
                                                          float4* __restrict__ Qc, float4* __restrict__ Qf) {
  // A block builds the coefficients of a group of 32 consecutive cells:
  // thread (comp, lane) does cell K0 + lane, component comp (neighbouring
  // lanes read neighbouring nodes of one component), leaves its 5 NS float4
  // in shared memory, and the block then writes the group's output region,
  // which is contiguous ([K][comp][5 NS]), with coalesced float4 stores.
  constexpr int NS = (D == 3 ? 3 : 1);
  constexpr int PER = 5 * NS;  // float4 per (cell, component)
  constexpr int PERF = qf_floats_per_comp<D>();  // floats per (cell, component) of Qf
  __shared__ float4 sh[32 * D * PER];
  __shared__ __align__(16) float shf[32 * D * PERF];
  const int lane = threadIdx.x & 31, comp = threadIdx.x >> 5;
  const int64_t sy = m.nq[0], sz = (int64_t)m.nq[0] * m.nq[1];
  for (uint32_t K0 = blockIdx.x * 32u; K0 < m.C; K0 += gridDim.x * 32u) {
    const uint32_t K = K0 + lane;
    if (K < m.C) {
      int c[3];
      cell_ijk<D>(m, K, c);
      const int64_t base = 2 * (int64_t)c[0] + sy * 2 * c[1] + (D == 3 ? sz * 2 * c[2] : 0);
      const float2* Uc = U2 + base * D + comp;  // node-major [node][comp]
      df V[3][3][3];  // [r (z)][q (y)][p (x)]
#pragma unroll
      for (int r = 0; r < NS; ++r)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const float2* row = Uc + (q * sy + (D == 3 ? r * sz : 0)) * D;
          const float2 a = row[0], b = row[D], e = row[2 * D];
          t_axis(df_make(a.x, a.y), df_make(b.x, b.y), df_make(e.x, e.y), V[r][q][0], V[r][q][1], V[r][q][2]);
        }
#pragma unroll
      for (int r = 0; r < NS; ++r)
#pragma unroll
        for (int p = 0; p < 3; ++p) t_axis(V[r][0][p], V[r][1][p], V[r][2][p], V[r][0][p], V[r][1][p], V[r][2][p]);
      if constexpr (D == 3) {
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
          for (int p = 0; p < 3; ++p) t_axis(V[0][q][p], V[1][q][p], V[2][q][p], V[0][q][p], V[1][q][p], V[2][q][p]);
      }
      float4* out = sh + (lane * D + comp) * PER;
#pragma unroll
      for (int r = 0; r < NS; ++r) {
        df pr[10];
#pragma unroll
        for (int e = 0; e < 9; ++e) pr[e] = V[r][e / 3][e % 3];
        pr[9] = df_make(0.f, 0.f);
        float f[20];  // the ten high parts, then the ten low parts
#pragma unroll
        for (int e = 0; e < 10; ++e) {
          f[e] = pr[e].hi;
          f[10 + e] = pr[e].lo;
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) out[5 * r + k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
      }
      float* outf = shf + (lane * D + comp) * PERF;
#pragma unroll
      for (int r = 0; r < NS; ++r)
#pragma unroll
        for (int e = 0; e < 9; ++e) outf[9 * r + e] = V[r][e / 3][e % 3].hi;
#pragma unroll
      for (int e = 9 * NS; e < PERF; ++e) outf[e] = 0.f;
    }
    __syncthreads();
    const uint32_t ncell = (m.C - K0) < 32u ? (m.C - K0) : 32u;
    const uint32_t nf4 = ncell * D * PER;
    float4* dst = Qc + (size_t)K0 * D * PER;
    for (uint32_t q = threadIdx.x; q < nf4; q += blockDim.x) dst[q] = sh[q];
    if (Qf) {
      const uint32_t nff = ncell * D * (PERF / 4);
      float4* dstf = Qf + (size_t)K0 * D * (PERF / 4);
      const float4* shf4 = reinterpret_cast<const float4*>(shf);
      for (uint32_t q = threadIdx.x; q < nff; q += blockDim.x) dstf[q] = shf4[q];
    }
    __syncthreads();
  }
}

// Coefficients of one field into Qc: the FP64 values U are first split into
// the node-major double-float copy U2 (one conversion per nodal value).
static void build_coefficients(const pic_mesh_s* m, const double* U, float2* U2, float4* Qc, float4* Qf,
                               cudaStream_t st) {
  const size_t n = (size_t)m->dim * (size_t)m->nnodes;
  const int gn = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  to_df_nodes_kernel<<<gn, 256, 0, st>>>(U, U2, m->dim, (size_t)m->nnodes);
  MeshView v = mesh_view(m);
  const size_t groups = ((size_t)m->C + 31) / 32;
  const size_t cap = (size_t)num_sms() * 16;
  const int g = (int)(groups < cap ? groups : cap);
  if (m->dim == 2)
    q2_coeff_kernel<2><<<g, 64, 0, st>>>(v, U2, Qc, Qf);
  else
    q2_coeff_kernel<3><<<g, 96, 0, st>>>(v, U2, Qc, Qf);
  count_launches(2);
}

static size_t coeff_float4s(const pic_mesh_s* m) { return (size_t)m->C * m->dim * (m->dim == 3 ? 15 : 5); }
static size_t coeff32_float4s(const pic_mesh_s* m) {
  return (size_t)m->C * (m->dim == 3 ? qf_float4s<3>() : qf_float4s<2>());
}

pic_status ensure_fp32_coefficients(pic_mesh_s* m, cudaStream_t st) {
  if (!m->has_velocity) return PIC_OK;
  if (!m->Qf) {
    if (cudaMalloc(&m->Qf, sizeof(float4) * coeff32_float4s(m)) != cudaSuccess) {
      cudaGetLastError();
      m->Qf = nullptr;
      return (set_error("FP32 coefficient table: device allocation failed"), PIC_ERR_OOM);
    }
    build_coefficients(m, m->U, m->U2, m->Qc, m->Qf, st);
  }
  if (m->has_next && !m->Qfn) {
    if (cudaMalloc(&m->Qfn, sizeof(float4) * coeff32_float4s(m)) != cudaSuccess) {
      cudaGetLastError();
      m->Qfn = nullptr;
      return (set_error("FP32 coefficient table: device allocation failed"), PIC_ERR_OOM);
    }
    build_coefficients(m, m->Un, m->U2n, m->Qcn, m->Qfn, st);
  }
  PIC_CUDA(cudaGetLastError());
  return PIC_OK;
}


}  // namespace pic

using namespace pic;

extern "C" pic_status pic_create_mesh(int dim, const int* n_cells, const double* vertices, int vertices_on_device,
                                      void* stream, pic_mesh* out) {
  if (!out) return (set_error("pic_create_mesh: out is NULL"), PIC_ERR_ARG);
  *out = nullptr;
  if (dim != 2 && dim != 3) return (set_error("pic_create_mesh: dim must be 2 or 3 (got %d)", dim), PIC_ERR_ARG);
  if (!n_cells || !vertices) return (set_error("pic_create_mesh: null array"), PIC_ERR_ARG);
  uint64_t C = 1, nv = 1, nq = 1;
  for (int a = 0; a < dim; ++a) {
    if (n_cells[a] < 1) return (set_error("pic_create_mesh: n_cells[%d] = %d < 1", a, n_cells[a]), PIC_ERR_ARG);
    C *= (uint64_t)n_cells[a];
    nv *= (uint64_t)n_cells[a] + 1;
    nq *= 2 * (uint64_t)n_cells[a] + 1;
  }
  if (C >= (1ull << 31) || nq >= (1ull << 32))
    return (set_error("pic_create_mesh: mesh too large (%llu cells)", (unsigned long long)C), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  pic_mesh_s* m = (pic_mesh_s*)calloc(1, sizeof(pic_mesh_s));
  if (!m) return (set_error("pic_create_mesh: host allocation failed"), PIC_ERR_OOM);
  m->dim = dim;
  for (int a = 0; a < 3; ++a) {
    m->n[a] = a < dim ? n_cells[a] : 1;
    m->nv[a] = a < dim ? n_cells[a] + 1 : 1;
    m->nq[a] = a < dim ? 2 * n_cells[a] + 1 : 1;
  }
  m->C = (uint32_t)C;
  m->nverts = (int64_t)nv;
  m->nnodes = (int64_t)nq;
  auto fail = [&](pic_status s) {
    pic_destroy_mesh(m);
    return s;
  };
  const size_t blk_f4 = dim == 3 ? 12 : 4;
  if (cudaMalloc(&m->X, sizeof(double) * dim * nv) != cudaSuccess ||
      cudaMalloc(&m->bbox, sizeof(double) * 6 * C) != cudaSuccess ||
      cudaMalloc(&m->bbox32, sizeof(float4) * 2 * C) != cudaSuccess ||
      cudaMalloc(&m->blk, sizeof(float4) * blk_f4 * C) != cudaSuccess ||
      cudaMalloc(&m->qbase, sizeof(uint32_t) * C) != cudaSuccess) {
    cudaGetLastError();
    set_error("pic_create_mesh: device allocation failed");
    return fail(PIC_ERR_OOM);
  }
  // Host copy of the vertices for the padded domain box.
  std::vector<double> hX((size_t)dim * nv);
  cudaError_t e = cudaMemcpyAsync(hX.data(), vertices, sizeof(double) * dim * nv,
                                  vertices_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->X, hX.data(), sizeof(double) * dim * nv, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(cuda_fail(e, "pic_create_mesh: vertex upload"));
  for (int a = 0; a < 3; ++a) {
    double lo = 0.0, hi = 0.0;
    if (a < dim) {
      lo = INFINITY;
      hi = -INFINITY;
      for (uint64_t v = 0; v < nv; ++v) {
        const double c = hX[(size_t)a * nv + v];
        if (!std::isfinite(c)) {
          set_error("pic_create_mesh: vertex %llu has a non-finite coordinate", (unsigned long long)v);
          return fail(PIC_ERR_ARG);
        }
        lo = c < lo ? c : lo;
        hi = c > hi ? c : hi;
      }
      const double pad = 1e-9 * (hi - lo);
      lo -= pad;
      hi += pad;
    }
    m->dlo[a] = lo;
    m->dhi[a] = hi;
  }
  const MeshView mv = mesh_view(m);
  const int grid = (int)((C + 255) / 256 < 4096 ? (C + 255) / 256 : 4096);
  if (dim == 2) {
    cell_bbox_kernel<2><<<grid, 256, 0, st>>>(mv, m->bbox, m->bbox32);
    cell_block_kernel<2><<<grid, 256, 0, st>>>(mv, (float*)m->blk);
    cell_qbase_kernel<2><<<grid, 256, 0, st>>>(mv, m->qbase);
  } else {
    cell_bbox_kernel<3><<<grid, 256, 0, st>>>(mv, m->bbox, m->bbox32);
    cell_block_kernel<3><<<grid, 256, 0, st>>>(mv, (float*)m->blk);
    cell_qbase_kernel<3><<<grid, 256, 0, st>>>(mv, m->qbase);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(cuda_fail(e, "pic_create_mesh: set-up kernels"));
  *out = m;
  return PIC_OK;
}

extern "C" pic_status pic_destroy_mesh(pic_mesh m) {
  if (!m) return PIC_OK;
  cudaFree(m->Ustage);
  if (m->ev_staged) cudaEventDestroy(m->ev_staged);
  if (m->ev_free) cudaEventDestroy(m->ev_free);
  cudaFree(m->X);
  cudaFree(m->U);
  cudaFree(m->bbox);
  cudaFree(m->bbox32);
  cudaFree(m->blk);
  cudaFree(m->qbase);
  cudaFree(m->U2);
  cudaFree(m->Un);
  cudaFree(m->U2n);
  cudaFree(m->Qc);
  cudaFree(m->Qcn);
  cudaFree(m->Qf);
  cudaFree(m->Qfn);
  free(m);
  return PIC_OK;
}

extern "C" pic_status pic_set_velocity_dofs(pic_mesh m, const double* U, const double* U_next, void* stream) {
  if (!m || !U) return (set_error("pic_set_velocity_dofs: null argument"), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)m->dim * (size_t)m->nnodes;
  if (!m->U) {
    if (cudaMalloc(&m->U, sizeof(double) * n) != cudaSuccess || cudaMalloc(&m->U2, sizeof(float2) * n) != cudaSuccess ||
        cudaMalloc(&m->Qc, sizeof(float4) * coeff_float4s(m)) != cudaSuccess) {
      cudaGetLastError();
      return (set_error("pic_set_velocity_dofs: device allocation failed"), PIC_ERR_OOM);
    }
  }
  if (U_next && !m->Un) {
    if (cudaMalloc(&m->Un, sizeof(double) * n) != cudaSuccess || cudaMalloc(&m->U2n, sizeof(float2) * n) != cudaSuccess ||
        cudaMalloc(&m->Qcn, sizeof(float4) * coeff_float4s(m)) != cudaSuccess) {
      cudaGetLastError();
      return (set_error("pic_set_velocity_dofs: device allocation failed"), PIC_ERR_OOM);
    }
  }
  if (U_next && m->Qf && !m->Qfn) {
    if (cudaMalloc(&m->Qfn, sizeof(float4) * coeff32_float4s(m)) != cudaSuccess) {
      cudaGetLastError();
      m->Qfn = nullptr;
      return (set_error("pic_set_velocity_dofs: device allocation failed"), PIC_ERR_OOM);
    }
  }
  PIC_CUDA(cudaMemcpyAsync(m->U, U, sizeof(double) * n, cudaMemcpyDefault, st));
  build_coefficients(m, m->U, m->U2, m->Qc, m->Qf, st);
  if (U_next) {
    PIC_CUDA(cudaMemcpyAsync(m->Un, U_next, sizeof(double) * n, cudaMemcpyDefault, st));
    build_coefficients(m, m->Un, m->U2n, m->Qcn, m->Qfn, st);
  }
  PIC_CUDA(cudaGetLastError());
  m->has_velocity = 1;
  m->has_next = U_next ? 1 : 0;
  return PIC_OK;
}

// Staged upload (overlap of the next field's copy with the current step).
// The copy goes to a staging buffer on `copy_stream`; it first waits for the
// buffer to be free (the conversions of the commit that last released it).
extern "C" pic_status pic_stage_velocity_dofs(pic_mesh m, const double* U, void* copy_stream) {
  if (!m || !U) return (set_error("pic_stage_velocity_dofs: null argument"), PIC_ERR_ARG);
  if (!m->has_velocity) return (set_error("pic_stage_velocity_dofs: set a first field with pic_set_velocity_dofs"), PIC_ERR_STATE);
  if (m->staged) return (set_error("pic_stage_velocity_dofs: a staged field is not committed yet"), PIC_ERR_STATE);
  cudaStream_t cs = (cudaStream_t)copy_stream;
  const size_t n = (size_t)m->dim * (size_t)m->nnodes;
  if (!m->Ustage) {
    if (cudaMalloc(&m->Ustage, sizeof(double) * n) != cudaSuccess) {
      cudaGetLastError();
      m->Ustage = nullptr;
      return (set_error("pic_stage_velocity_dofs: device allocation failed"), PIC_ERR_OOM);
    }
  }
  if (!m->ev_staged) PIC_CUDA(cudaEventCreateWithFlags(&m->ev_staged, cudaEventDisableTiming));
  if (!m->ev_free) PIC_CUDA(cudaEventCreateWithFlags(&m->ev_free, cudaEventDisableTiming));
  if (m->free_recorded) PIC_CUDA(cudaStreamWaitEvent(cs, m->ev_free, 0));
  PIC_CUDA(cudaMemcpyAsync(m->Ustage, U, sizeof(double) * n, cudaMemcpyDefault, cs));
  PIC_CUDA(cudaEventRecord(m->ev_staged, cs));
  m->staged = 1;
  return PIC_OK;
}

// Make the staged field the field u_h^n on `stream`: wait for the copy, swap
// the FP64 buffers, rebuild the FP32 and double-float copies, and mark the
// released buffer free once those conversions have run.
extern "C" pic_status pic_commit_velocity_dofs(pic_mesh m, void* stream) {
  if (!m) return (set_error("pic_commit_velocity_dofs: null mesh"), PIC_ERR_ARG);
  if (!m->staged) return (set_error("pic_commit_velocity_dofs: nothing staged"), PIC_ERR_STATE);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)m->dim * (size_t)m->nnodes;
  PIC_CUDA(cudaStreamWaitEvent(st, m->ev_staged, 0));
  double* t = m->U;
  m->U = m->Ustage;
  m->Ustage = t;
  build_coefficients(m, m->U, m->U2, m->Qc, m->Qf, st);
  PIC_CUDA(cudaGetLastError());
  PIC_CUDA(cudaEventRecord(m->ev_free, st));
  m->free_recorded = 1;
  m->staged = 0;
  return PIC_OK;
}
