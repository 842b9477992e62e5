// adjoint.cu -- gradients of a function of the final particle positions with
// respect to the Q2 nodal velocities (the adjoint of the Sec. 2.3 integrators
// over located stages), for inverse flow reconstruction from tracer
// endpoints.
//
// pic_advect_record advances the store like pic_advect and keeps, for every
// step, each particle's stage records (the located cell and double-float
// x-hat of every stage point, exactly as the step used them) and the rebin's
// permutation (new slot -> old slot).  A checkpoint tape keeps instead the
// store at the start of each step and replays the step in the sweep with the
// same particle step, which rewrites the same records (half the memory, one
// more advect per step).  pic_tape_adjoint then sweeps the steps backwards.  For one step, with y_s = x + a_s k_{s-1}, k_s = dt u(y_s),
// x' = x + sum_s b_s k_s and G_s = du/dx at y_s (cell held fixed):
//   lambda_k_s = b_s lambda' + a_{s+1} lambda_y_{s+1}
//   lambda_y_s = dt G_s^T lambda_k_s,       lambda = lambda' + sum_s lambda_y_s
//   dL/dU_i   += dt phi-hat_i(x-hat_s) lambda_k_s
// G and lambda in double-float.  Each stage's contribution (stage cell,
// x-hat_s, dt lambda_k_s) is a record keyed by (stage, slot); the records are
// sorted by (cell, key), summed per cell in that order, and the cells' sums
// are added into the nodes in increasing cell order.  No floating-point
// atomics, so the gradient is bit-for-bit reproducible.
#include <cmath>
#include <cstdlib>

#include "advect.cuh"
#include "fastpath.cuh"
#include "grad_df.cuh"
#include "locate.cuh"
#include "pic_internal.cuh"

struct pic_tape_s {
  pic_particles_s* parts;
  const pic_mesh_s* mesh;
  int dim, n_steps, integrator;
  double dt;
  size_t cap;
  uint32_t C;
  int kind;          // pic_tape_kind
  int n_rec;         // stage-record sets: n_steps (stage tapes) or 1 (the replay's, checkpoint tapes)
  uint32_t** rcell;  // [n_rec] of [4][cap]: stage cells (StageRec layout, slots of the start of the step)
  float2** rt;       // [n_rec] of [dim][4][cap]: stage x-hat, double-float
  double** x;        // checkpoint tapes: [n_steps] of [dim][cap], the store at the start of the step
  float2** xhat;     //   [n_steps] of [dim][cap]
  uint32_t** cell;   //   [n_steps] of [cap]
  double* sink_x;    //   [dim][cap] the replayed step's new positions (discarded)
  float2* sink_xhat; //   [dim][cap]
  uint32_t** perm;   // [n_steps] of [cap] (new slot -> old slot)
  uint32_t* n_dev;   // [n_steps + 1] particles at the start of each step (and at the end)
  // reverse-sweep work
  float2* lam[2];      // [dim][cap] double-float
  uint32_t* rec_cell;  // [4 cap] stage cells of the step's survivors, PIC_LOST elsewhere (the sort's keys)
  uint64_t* rec_key;   // [4 cap]
  float2* rec_w;       // [dim][4 cap] double-float dt lambda_k
  uint32_t* rec_perm;  // [4 cap]
  uint32_t* rec_off;   // [C + 1]
  void* sort_scratch;
  double* partial;     // [C][3^dim][dim]
};

namespace pic {

constexpr int kRecPerParticle = 4;

// The tableaux with a_s (a power of two or zero) as float and b_s as a
// double-float (1/6 and 1/3 to ~2^-48).
template <int RK>
struct AdjTableau;
template <>
struct AdjTableau<1> {
  static constexpr int S = 1;
  __device__ static float a(int) { return 0.f; }
  __device__ static df b(int) { return df_make(1.f, 0.f); }
};
template <>
struct AdjTableau<2> {
  static constexpr int S = 2;
  __device__ static float a(int s) { return s == 1 ? 0.5f : 0.f; }
  __device__ static df b(int s) { return df_make(s == 1 ? 1.f : 0.f, 0.f); }
};
template <>
struct AdjTableau<4> {
  static constexpr int S = 4;
  __device__ static float a(int s) { return s == 3 ? 1.f : (s == 0 ? 0.f : 0.5f); }
  __device__ static df b(int s) {
    return (s == 0 || s == 3) ? df_make(0.1666666716337204f, -4.967053879312289e-09f)
                              : df_make(0.3333333432674408f, -9.934107758624577e-09f);
  }
};

struct TapeStep {
  const uint32_t* rcell;
  const float2* rt;
  const uint32_t* perm;
  const uint32_t* n_next;  // particles after the step
};

// Resident blocks per SM requested from the register allocator for the
// lambda sweep (swept at build time with -DPIC_REVERSE_MIN_BLOCKS=n).
#ifndef PIC_REVERSE_MIN_BLOCKS
#define PIC_REVERSE_MIN_BLOCKS 4
#endif

// One reverse step, thread per particle alive after the step (new slot j,
// old slot i = perm[j]): the stages backwards with G_s = du/dx at the
// recorded stage points, all in double-float on the FP32 pipe:
//   lambda_k_s = b_s lambda' + a_{s+1} lambda_y_{s+1}
//   lambda_y_s = dt G_s^T lambda_k_s,   lambda = lambda' + sum_s lambda_y_s
// and record r = s cap + i gets its cell, key and weight dt lambda_k_s.  The
// records of particles that did not survive the step stay PIC_LOST.
template <int D, int RK>
__global__ void __launch_bounds__(128, PIC_REVERSE_MIN_BLOCKS) reverse_lambda_kernel(
    const __grid_constant__ MeshView m, const __grid_constant__ TapeStep tp, size_t cap, df dt, const float2* __restrict__ lam_in, float2* __restrict__ lam_out,
    uint32_t* __restrict__ rec_cell, uint64_t* __restrict__ rec_key, float2* __restrict__ rec_w,
    DevCounters* __restrict__ ctr) {
  using TB = AdjTableau<RK>;
  constexpr int S = TB::S;
  const uint32_t n = *tp.n_next;
  const size_t rcap = kRecPerParticle * cap;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const uint32_t i = tp.perm[j];
    if (i >= cap) {
      latch_status(ctr, PIC_STATUS_BOUNDS);
      continue;
    }
    uint32_t Ks[S];
    bool ok = true;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      Ks[s] = tp.rcell[(size_t)s * cap + i];
      ok = ok && Ks[s] < m.C;
    }
    if (!ok) {  // cannot happen for a particle that survived the step
      latch_status(ctr, PIC_STATUS_BOUNDS);
      continue;
    }
    df lam[D], lam_x[D], lam_ynext[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const float2 v = lam_in[a * cap + j];
      lam[a] = df_make(v.x, v.y);
      lam_x[a] = lam[a];
      lam_ynext[a] = df_make(0.f, 0.f);
    }
#pragma unroll 1
    for (int s = S - 1; s >= 0; --s) {
      const size_t r = (size_t)s * cap + i;
      df t[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const float2 v = tp.rt[a * rcap + r];
        t[a] = df_make(v.x, v.y);
      }
      uint32_t K = Ks[0];
#pragma unroll
      for (int q = 1; q < S; ++q) K = (s == q) ? Ks[q] : K;
      df G[D][D];
      velocity_gradient_df<D>(m, K, t, G);
      const df bs = TB::b(s);
      const float an = s + 1 < S ? TB::a(s + 1) : 0.f;
      df lk[D];
#pragma unroll
      for (int a = 0; a < D; ++a) lk[a] = df_add(df_mul(bs, lam[a]), df_scale2(lam_ynext[a], an));
      rec_cell[r] = K;
      rec_key[r] = r;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const df w = df_mul(dt, lk[a]);
        rec_w[a * rcap + r] = make_float2(w.hi, w.lo);
      }
#pragma unroll
      for (int q = 0; q < D; ++q) {
        df_acc acc = acc_zero();
#pragma unroll
        for (int c = 0; c < D; ++c) acc_mad(acc, G[c][q], lk[c]);
        lam_ynext[q] = df_mul(dt, acc_result(acc));
        lam_x[q] = df_add(lam_x[q], lam_ynext[q]);
      }
    }
#pragma unroll
    for (int a = 0; a < D; ++a) lam_out[a * cap + i] = make_float2(lam_x[a].hi, lam_x[a].lo);
  }
}

// Checkpoint tapes: the step replayed from the store as it was at the start
// of the step, for every particle then alive, by the forward's own
// advect_particle (so the stage records are the forward's bit for bit); the
// new positions go to a sink.
template <int D, int RK>
__global__ void __launch_bounds__(128, PIC_ADVECT_MIN_BLOCKS) replay_step_kernel(const __grid_constant__ MeshView m, const __grid_constant__ StoreView s, const __grid_constant__ StoreView sink,
                                                                                const uint32_t* __restrict__ n_start,
                                                                                df dt, const __grid_constant__ StageRec rec) {
  const uint32_t n = *n_start;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int iters = 0;
    unsigned flags = 0;
    RecordHook hook{rec, i};
    advect_particle_to<D, RK, false, false>(m, s, i, sink, i, s.cell[i], dt, iters, flags, hook);
  }
}

// Warp per cell: the records of the cell, in (cell, key) order, summed into
// the cell's 3^D x D block of nodal gradient entries (lane e owns entries e,
// e+32, ...), in double-float on the FP32 pipe; every cell is written (FP64),
// empty ones with zeros.  The entry (node (a, b, c), comp) of a record is
// (w_comp l_a(t0)) (l_b(t1) l_c(t2)): records are taken 32 at a time, lane i
// forms record i's D x 3 left factors and 3^(D-1) right factors once and
// leaves them in shared memory, then every lane adds its entries' products
// over those records in record order.
template <int D>
__global__ void __launch_bounds__(256) cell_partial_kernel(uint32_t C, const uint32_t* __restrict__ rec_off,
                                                           const uint32_t* __restrict__ rec_perm,
                                                           const float2* __restrict__ rec_t,
                                                           const float2* __restrict__ rec_w, size_t rcap,
                                                           double* __restrict__ partial) {
  constexpr int NN = (D == 3 ? 27 : 9);
  constexpr int NE = NN * D;
  constexpr int PER = (NE + 31) / 32;
  constexpr int NA = 3 * D;             // w_comp l_a(t0), index comp * 3 + a
  constexpr int NB = (D == 3 ? 9 : 3);  // l_b(t1) l_c(t2), index c * 3 + b (2D: l_b(t1))
  __shared__ float2 fac[256 / 32][32][NA + NB];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  int ia[PER], ib[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int ent = lane + 32 * q;
    const int node = ent / D, comp = ent % D;
    ia[q] = comp * 3 + node % 3;
    ib[q] = NA + (D == 3 ? (node / 9) * 3 + (node / 3) % 3 : (node / 3) % 3);
  }
  for (uint32_t K = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; K < C; K += warps) {
    df_acc acc[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) acc[q] = acc_zero();
    const uint32_t beg = rec_off[K], end = rec_off[K + 1];
    for (uint32_t e0 = beg; e0 < end; e0 += 32) {
      const uint32_t e = e0 + lane;
      if (e < end) {
        const uint32_t r = rec_perm[e];
        df l[D][3], w[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const float2 tv = rec_t[a * rcap + r], wv = rec_w[a * rcap + r];
          lagrange2_df(df_make(tv.x, tv.y), l[a]);
          w[a] = df_make(wv.x, wv.y);
        }
#pragma unroll
        for (int comp = 0; comp < D; ++comp)
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const df v = df_mul(w[comp], l[0][a]);
            fac[wib][lane][comp * 3 + a] = make_float2(v.hi, v.lo);
          }
#pragma unroll
        for (int c = 0; c < (D == 3 ? 3 : 1); ++c)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const df v = (D == 3) ? df_mul(l[1][b], l[2 % D][c]) : l[1][b];
            fac[wib][lane][NA + c * 3 + b] = make_float2(v.hi, v.lo);
          }
      }
      __syncwarp();
      const int cnt = (end - e0) < 32u ? (int)(end - e0) : 32;
      for (int j = 0; j < cnt; ++j) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
          if (lane + 32 * q < NE) {
            const float2 A = fac[wib][j][ia[q]], B = fac[wib][j][ib[q]];
            acc_mad(acc[q], df_make(A.x, A.y), df_make(B.x, B.y));
          }
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int ent = lane + 32 * q;
      if (ent < NE) {
        const df v = acc_result(acc[q]);
        partial[(size_t)K * NE + ent] = df_to_double(v);
      }
    }
  }
}

// Thread per (node, component): add the blocks of the cells that share the
// node, in increasing cell order.
template <int D>
__global__ void node_reduce_kernel(const __grid_constant__ MeshView m, const double* __restrict__ partial, double* __restrict__ grad) {
  constexpr int NN = (D == 3 ? 27 : 9);
  const size_t total = (size_t)m.nnodes * D;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const size_t comp = q / m.nnodes, node = q % m.nnodes;
    int I[3] = {(int)(node % m.nq[0]), (int)((node / m.nq[0]) % m.nq[1]), (int)(node / ((size_t)m.nq[0] * m.nq[1]))};
    // cells touching the node along each axis: node index I = 2i + a, a in {0,1,2}
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= D) continue;
      if (I[a] % 2 == 1) {
        lo[a] = hi[a] = I[a] / 2;
      } else {
        lo[a] = I[a] / 2 - 1;
        hi[a] = I[a] / 2;
        if (lo[a] < 0) lo[a] = 0;
        if (hi[a] > m.n[a] - 1) hi[a] = m.n[a] - 1;
      }
    }
    double s = 0.0;
    for (int ck = lo[2]; ck <= hi[2]; ++ck)
      for (int cj = lo[1]; cj <= hi[1]; ++cj)
        for (int ci = lo[0]; ci <= hi[0]; ++ci) {
          const uint32_t K = cell_index<D>(m, ci, cj, ck);
          const int a = I[0] - 2 * ci, b = I[1] - 2 * cj, c = (D == 3 ? I[2] - 2 * ck : 0);
          const int local = a + 3 * b + 9 * c;
          s += partial[((size_t)K * NN + local) * D + comp];
        }
    grad[comp * m.nnodes + node] += s;
  }
}

// lam[a*cap + j] = src[a*n + j] for j < n (dense caller layout -> strided,
// FP64 -> double-float).
__global__ void copy_in_kernel(const double* __restrict__ src, float2* __restrict__ dst, const uint32_t* n_dev, int dim,
                               size_t cap) {
  const uint32_t n = *n_dev;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < (size_t)n * dim; q += (size_t)gridDim.x * blockDim.x) {
    const df v = df_from_double(src[q]);
    dst[(q / n) * cap + q % n] = make_float2(v.hi, v.lo);
  }
}

__global__ void copy_out_kernel(const float2* __restrict__ src, double* __restrict__ dst, const uint32_t* n_dev, int dim,
                                size_t cap) {
  const uint32_t n = *n_dev;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < (size_t)n * dim; q += (size_t)gridDim.x * blockDim.x) {
    const float2 v = src[(q / n) * cap + q % n];
    dst[q] = df_to_double(df_make(v.x, v.y));
  }
}

static int grid_of(size_t n, int block) {
  size_t g = (n + block - 1) / block;
  const size_t cap = (size_t)num_sms() * 16;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

template <int D, int RK>
static void launch_reverse(pic_tape_s* tp, const MeshView& m, int step, const TapeStep& ts, const float2* lin,
                           float2* lout, cudaStream_t st) {
  const float hi = (float)tp->dt;
  const df dtd = {hi, (float)(tp->dt - (double)hi)};
  if (tp->kind == PIC_TAPE_CHECKPOINTS) {
    StoreView s{}, sink{};
    s.x = tp->x[step];
    s.xhat = tp->xhat[step];
    s.cell = tp->cell[step];
    s.cap = tp->cap;
    sink.x = tp->sink_x;
    sink.xhat = tp->sink_xhat;
    sink.cap = tp->cap;
    replay_step_kernel<D, RK><<<grid_of(tp->cap, 128), 128, 0, st>>>(m, s, sink, tp->n_dev + step, dtd,
                                                                     StageRec{tp->rcell[0], tp->rt[0], tp->cap});
    count_launches(1);
  }
  reverse_lambda_kernel<D, RK><<<grid_of(tp->cap, 128), 128, 0, st>>>(m, ts, tp->cap, dtd, lin, lout, tp->rec_cell,
                                                                       tp->rec_key, tp->rec_w, tp->parts->ctr);
}

}  // namespace pic

using namespace pic;

extern "C" pic_status pic_destroy_tape(pic_tape tp) {
  if (!tp) return PIC_OK;
  for (int s = 0; s < tp->n_rec; ++s) {
    if (tp->rcell) cudaFree(tp->rcell[s]);
    if (tp->rt) cudaFree(tp->rt[s]);
  }
  for (int s = 0; s < tp->n_steps; ++s) {
    if (tp->perm) cudaFree(tp->perm[s]);
    if (tp->x) cudaFree(tp->x[s]);
    if (tp->xhat) cudaFree(tp->xhat[s]);
    if (tp->cell) cudaFree(tp->cell[s]);
  }
  free(tp->rcell);
  free(tp->rt);
  free(tp->perm);
  free(tp->x);
  free(tp->xhat);
  free(tp->cell);
  cudaFree(tp->sink_x);
  cudaFree(tp->sink_xhat);
  cudaFree(tp->n_dev);
  cudaFree(tp->lam[0]);
  cudaFree(tp->lam[1]);
  cudaFree(tp->rec_cell);
  cudaFree(tp->rec_key);
  cudaFree(tp->rec_w);
  cudaFree(tp->rec_perm);
  cudaFree(tp->rec_off);
  cudaFree(tp->sort_scratch);
  cudaFree(tp->partial);
  free(tp);
  return PIC_OK;
}

extern "C" pic_status pic_advect_record_tape(pic_particles parts, pic_mesh mesh, double dt, pic_integrator integrator,
                                             int n_steps, pic_tape_kind kind, void* stream, pic_tape* out) {
  if (!out) return (set_error("pic_advect_record: out is NULL"), PIC_ERR_ARG);
  *out = nullptr;
  if (kind != PIC_TAPE_STAGES && kind != PIC_TAPE_CHECKPOINTS)
    return (set_error("pic_advect_record: unknown tape kind %d", (int)kind), PIC_ERR_ARG);
  if (!parts || !mesh || parts->mesh != mesh || parts->dim != mesh->dim)
    return (set_error("pic_advect_record: bad handles"), PIC_ERR_ARG);
  if (!std::isfinite(dt)) return (set_error("pic_advect_record: dt not finite"), PIC_ERR_ARG);
  if (n_steps < 1) return (set_error("pic_advect_record: n_steps must be >= 1"), PIC_ERR_ARG);
  if (integrator != PIC_EULER && integrator != PIC_RK2 && integrator != PIC_RK4)
    return (set_error("pic_advect_record: unknown integrator"), PIC_ERR_ARG);
  if (!mesh->has_velocity) return (set_error("pic_advect_record: velocity not set"), PIC_ERR_ARG);
  if (mesh->has_next)
    return (set_error("pic_advect_record: the adjoint supports a steady field only (no U_next)"), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  {
    const pic_status r0 = settle_order(parts, st);
    if (r0 != PIC_OK) return r0;
  }
  pic_tape_s* tp = (pic_tape_s*)calloc(1, sizeof(pic_tape_s));
  tp->parts = parts;
  tp->mesh = mesh;
  tp->dim = mesh->dim;
  tp->n_steps = n_steps;
  tp->integrator = (int)integrator;
  tp->dt = dt;
  tp->cap = parts->capacity;
  tp->C = mesh->C;
  tp->kind = (int)kind;
  const bool ckpt = kind == PIC_TAPE_CHECKPOINTS;
  tp->n_rec = ckpt ? 1 : n_steps;
  const size_t cap = tp->cap, d = (size_t)tp->dim, rcap = kRecPerParticle * cap;
  const int NE = (tp->dim == 3 ? 27 : 9) * tp->dim;
  tp->rcell = (uint32_t**)calloc(tp->n_rec, sizeof(uint32_t*));
  tp->rt = (float2**)calloc(tp->n_rec, sizeof(float2*));
  tp->perm = (uint32_t**)calloc(n_steps, sizeof(uint32_t*));
  bool ok = tp->rcell && tp->rt && tp->perm;
  if (ckpt) {
    tp->x = (double**)calloc(n_steps, sizeof(double*));
    tp->xhat = (float2**)calloc(n_steps, sizeof(float2*));
    tp->cell = (uint32_t**)calloc(n_steps, sizeof(uint32_t*));
    ok = ok && tp->x && tp->xhat && tp->cell;
    ok = ok && cudaMalloc(&tp->sink_x, sizeof(double) * d * cap) == cudaSuccess;
    ok = ok && cudaMalloc(&tp->sink_xhat, sizeof(float2) * d * cap) == cudaSuccess;
  }
  for (int s = 0; s < tp->n_rec && ok; ++s) {
    ok = ok && cudaMalloc(&tp->rcell[s], sizeof(uint32_t) * rcap) == cudaSuccess;
    ok = ok && cudaMalloc(&tp->rt[s], sizeof(float2) * d * rcap) == cudaSuccess;
  }
  for (int s = 0; s < n_steps && ok; ++s) {
    ok = ok && cudaMalloc(&tp->perm[s], sizeof(uint32_t) * cap) == cudaSuccess;
    if (ckpt) {
      ok = ok && cudaMalloc(&tp->x[s], sizeof(double) * d * cap) == cudaSuccess;
      ok = ok && cudaMalloc(&tp->xhat[s], sizeof(float2) * d * cap) == cudaSuccess;
      ok = ok && cudaMalloc(&tp->cell[s], sizeof(uint32_t) * cap) == cudaSuccess;
    }
  }
  ok = ok && cudaMalloc(&tp->n_dev, sizeof(uint32_t) * (n_steps + 1)) == cudaSuccess;
  ok = ok && cudaMalloc(&tp->lam[0], sizeof(float2) * d * cap) == cudaSuccess;
  ok = ok && cudaMalloc(&tp->lam[1], sizeof(float2) * d * cap) == cudaSuccess;
  ok = ok && cudaMalloc(&tp->rec_cell, sizeof(uint32_t) * rcap) == cudaSuccess;
  ok = ok && cudaMalloc(&tp->rec_key, sizeof(uint64_t) * rcap) == cudaSuccess;
  ok = ok && cudaMalloc(&tp->rec_w, sizeof(float2) * d * rcap) == cudaSuccess;
  ok = ok && cudaMalloc(&tp->rec_perm, sizeof(uint32_t) * rcap) == cudaSuccess;
  ok = ok && cudaMalloc(&tp->rec_off, sizeof(uint32_t) * ((size_t)tp->C + 1)) == cudaSuccess;
  ok = ok && cudaMalloc(&tp->sort_scratch, sort_scratch_bytes(rcap, tp->C)) == cudaSuccess;
  ok = ok && cudaMalloc(&tp->partial, sizeof(double) * NE * (size_t)tp->C) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    pic_destroy_tape(tp);
    return (set_error("pic_advect_record: device allocation failed"), PIC_ERR_OOM);
  }
  const MeshView m = mesh_view(mesh);
  for (int s = 0; s < n_steps; ++s) {
    cudaError_t e = cudaMemcpyAsync(tp->n_dev + s, &parts->ctr->n_alive, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(parts->counts, 0, sizeof(uint32_t) * parts->C, st);
    if (ckpt) {
      const int c = parts->cur;
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(tp->x[s], parts->x[c], sizeof(double) * d * cap, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(tp->xhat[s], parts->xhat[c], sizeof(float2) * d * cap, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(tp->cell[s], parts->cell[c], sizeof(uint32_t) * cap, cudaMemcpyDeviceToDevice, st);
    }
    if (e != cudaSuccess) {
      pic_destroy_tape(tp);
      return cuda_fail(e, "pic_advect_record: checkpoint");
    }
    // a checkpoint tape keeps one record set, which the sweep's replay rewrites
    launch_advect_record(parts, m, dt, (int)integrator, StageRec{tp->rcell[ckpt ? 0 : s], tp->rt[ckpt ? 0 : s], cap},
                         st);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      pic_destroy_tape(tp);
      return cuda_fail(e, "pic_advect_record: step");
    }
    pic_status r = rebin_from_counts(parts, st);
    if (r != PIC_OK) {
      pic_destroy_tape(tp);
      return r;
    }
    e = cudaMemcpyAsync(tp->perm[s], parts->perm, sizeof(uint32_t) * cap, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
      pic_destroy_tape(tp);
      return cuda_fail(e, "pic_advect_record: permutation");
    }
  }
  cudaError_t e = cudaMemcpyAsync(tp->n_dev + n_steps, &parts->ctr->n_alive, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) {
    pic_destroy_tape(tp);
    return cuda_fail(e, "pic_advect_record: count");
  }
  *out = tp;
  return PIC_OK;
}

extern "C" pic_status pic_advect_record(pic_particles parts, pic_mesh mesh, double dt, pic_integrator integrator,
                                        int n_steps, void* stream, pic_tape* out) {
  return pic_advect_record_tape(parts, mesh, dt, integrator, n_steps, PIC_TAPE_STAGES, stream, out);
}

extern "C" pic_status pic_tape_adjoint(pic_tape tp, const double* dL_dxfinal, double* dL_dU, double* dL_dx0,
                                       void* stream) {
  if (!tp || !dL_dxfinal || !dL_dU) return (set_error("pic_tape_adjoint: null argument"), PIC_ERR_ARG);
  const pic_mesh_s* mesh = tp->mesh;
  cudaStream_t st = (cudaStream_t)stream;
  const MeshView m = mesh_view(mesh);
  const size_t cap = tp->cap, d = (size_t)tp->dim, rcap = kRecPerParticle * cap;
  PIC_CUDA(cudaMemsetAsync(dL_dU, 0, sizeof(double) * d * (size_t)mesh->nnodes, st));
  PIC_CUDA(cudaMemsetAsync(tp->lam[0], 0, sizeof(float2) * d * cap, st));
  copy_in_kernel<<<grid_of(d * cap, 256), 256, 0, st>>>(dL_dxfinal, tp->lam[0], tp->n_dev + tp->n_steps, tp->dim, cap);
  count_launches(1);
  int cur = 0;
  const SortScratch sc = sort_scratch_layout(tp->sort_scratch, rcap, tp->C);
  for (int s = tp->n_steps - 1; s >= 0; --s) {
    TapeStep ts;
    ts.rcell = tp->rcell[tp->kind == PIC_TAPE_CHECKPOINTS ? 0 : s];
    ts.rt = tp->rt[tp->kind == PIC_TAPE_CHECKPOINTS ? 0 : s];
    ts.perm = tp->perm[s];
    ts.n_next = tp->n_dev + s + 1;
    PIC_CUDA(cudaMemsetAsync(tp->lam[1 - cur], 0, sizeof(float2) * d * cap, st));
    PIC_CUDA(cudaMemsetAsync(tp->rec_cell, 0xFF, sizeof(uint32_t) * rcap, st));
    const float2* lin = tp->lam[cur];
    float2* lout = tp->lam[1 - cur];
    if (tp->dim == 2) {
      if (tp->integrator == 1) launch_reverse<2, 1>(tp, m, s, ts, lin, lout, st);
      else if (tp->integrator == 2) launch_reverse<2, 2>(tp, m, s, ts, lin, lout, st);
      else launch_reverse<2, 4>(tp, m, s, ts, lin, lout, st);
    } else {
      if (tp->integrator == 1) launch_reverse<3, 1>(tp, m, s, ts, lin, lout, st);
      else if (tp->integrator == 2) launch_reverse<3, 2>(tp, m, s, ts, lin, lout, st);
      else launch_reverse<3, 4>(tp, m, s, ts, lin, lout, st);
    }
    count_launches(1);
    PIC_CUDA(cudaGetLastError());
    pic_status r = sort_by_cell_run(rcap, tp->rec_cell, tp->rec_key, tp->C, tp->rec_perm, tp->rec_off, sc, st);
    if (r != PIC_OK) return r;
    const int gp = grid_of((size_t)tp->C * 32, 256);
    const int gn = grid_of(d * (size_t)mesh->nnodes, 256);
    if (tp->dim == 2) {
      cell_partial_kernel<2><<<gp, 256, 0, st>>>(tp->C, tp->rec_off, tp->rec_perm, ts.rt, tp->rec_w, rcap, tp->partial);
      node_reduce_kernel<2><<<gn, 256, 0, st>>>(m, tp->partial, dL_dU);
    } else {
      cell_partial_kernel<3><<<gp, 256, 0, st>>>(tp->C, tp->rec_off, tp->rec_perm, ts.rt, tp->rec_w, rcap, tp->partial);
      node_reduce_kernel<3><<<gn, 256, 0, st>>>(m, tp->partial, dL_dU);
    }
    count_launches(2);
    PIC_CUDA(cudaGetLastError());
    cur = 1 - cur;
  }
  if (dL_dx0) {
    copy_out_kernel<<<grid_of(d * cap, 256), 256, 0, st>>>(tp->lam[cur], dL_dx0, tp->n_dev, tp->dim, cap);
    count_launches(1);
    PIC_CUDA(cudaGetLastError());
  }
  return PIC_OK;
}
