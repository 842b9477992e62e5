// pic_internal.cuh -- handle layouts, device views and device-side building
// blocks shared by the translation units of libpic.so.
//
// The method is the particle hot path of Gassmoeller, Heien, Puckett &
// Bangerth, arXiv 1612.03369: Q2 velocity evaluated at stored reference
// coordinates (Sec. 2.3, Remark 2.1), RK integration (Sec. 2.3), point
// location by inverse mapping plus a vertex-neighbour walk (Sec. 2.4), and a
// particle store kept sorted by cell (Sec. 2.1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pic.h"

#define PIC_LOST 0xFFFFFFFFu

namespace pic {

// ------------------------------------------------------------ constants --
// Inverse-map Newton: stop when max|delta| <= 1e-14 (reference coordinates
// are dimensionless), give up after 30 iterations (then "not in this cell").
constexpr double kNewtonTol = 1e-14;
constexpr int kNewtonMaxIt = 30;
// A point is inside K when its reference coordinates lie in [-eps, 1+eps]^d;
// the band keeps points on shared faces inside both neighbours, and the
// lowest cell index then owns them.
constexpr double kInsideEps = 1e-10;
// Reference-coordinate distance to a facet under which the cells across that
// facet are also tested for the lowest-index rule.  Any other cell that holds
// the point (within kInsideEps) must lie across a facet closer than this.
constexpr double kTieBand = 1e-6;
constexpr int kMaxProps = 16;

// ------------------------------------------------------------ handles --

struct DevCounters {
  unsigned long long particle_steps;
  unsigned long long walks;
  unsigned long long global_searches;
  unsigned long long newton_iterations;
  unsigned long long lost_total;
  unsigned long long fallback64;  // particle-steps where a cell went to the FP64 Newton
  unsigned long long walk64;      // particle-steps where the walk went past the predicted neighbour
  unsigned long long deferred;    // particle-steps the advect kernel redid on the full path (a rare path was needed)
  unsigned int status;
  unsigned int n_alive;  // particles in the store
  unsigned int n_next;   // particles after the pending rebin
  unsigned int fail_count;
  unsigned int tile_next;  // work counter of the advect kernel's dynamic tiles (cleared before each launch)
  unsigned int pad_;
};

}  // namespace pic

struct pic_mesh_s {
  int dim;
  int n[3];      // cells per axis (1 on unused axes)
  int nv[3];     // vertices per axis
  int nq[3];     // Q2 nodes per axis
  uint32_t C;    // cells
  int64_t nverts, nnodes;
  double* X;     // [dim][nverts]
  double* U;     // [dim][nnodes]
  double* bbox;  // [C][6] padded cell bounding boxes: lo xyz, hi xyz
  float4* bbox32;  // [C][2] the same in FP32, rounded outward and widened by a few ulps: lo xyz_, hi xyz_
  float4* blk;   // [C][12 (3D) or 4 (2D)] per-cell map blocks (double-float, see fastpath.cuh)
  uint32_t* qbase;  // [C] index of the cell's first Q2 node (2i, 2j, 2k)
  float2* U2;    // [nnodes][dim] Q2 nodal values as double-floats (hi, lo): the coefficients' source
  double* Un;    // the field at the end of the step (time interpolation), when set
  float2* U2n;   // its double-float nodal copy (the source of Qcn)
  float4* Qc;    // [C][dim][slices][5] per-cell monomial coefficients (double-float pairs, see fastpath.cuh)
  float4* Qcn;   // the same for the field at the end of the step
  float4* Qf;    // [C][dim][28 or 12 floats] their high parts (FP32-basis form), allocated on first use
  float4* Qfn;   // the same for the field at the end of the step
  int has_next;
  double dlo[3], dhi[3];  // padded domain bounding box
  int has_velocity;
  // staged upload of the next field (pic_stage_velocity_dofs): FP64 buffer,
  // "copy done" and "buffer free" events, created on first use
  double* Ustage;
  cudaEvent_t ev_staged, ev_free;
  int staged, free_recorded;
};

struct pic_particles_s {
  int dim;
  int n_props;
  uint32_t C;             // cells of the mesh it was seeded on
  const pic_mesh_s* mesh;
  size_t capacity;
  // double-buffered store, component-major with stride `capacity`;
  // reference coordinates are kept as double-floats (hi, lo)
  double* x[2];
  float2* xhat[2];
  uint64_t* id[2];
  uint32_t* cell[2];
  double* props[2];
  int cur;                // which buffer holds the sorted store
  int pending_order;      // pic_advect left the last rebin's order unapplied (perm; sorted cells in the other buffer)
  int stage_cells;        // pic_advect stages the cells' blocks in shared memory (pic_set_advect_staging)
  uint32_t* cell_off;     // [C+1]
  // scratch for the rebin
  uint32_t* cell_new;     // [capacity]
  uint32_t* counts;       // [C]
  uint32_t* cursor;       // [C]
  uint32_t* block_sums;   // scan scratch (scan_scratch_bytes(C))
  uint64_t* key_id;       // [capacity]
  uint32_t* key_src;      // [capacity]
  uint32_t* perm;         // [capacity]
  pic::DevCounters* ctr;  // device counters and status word
  double* xfer;           // [2 * 2^dim][C] per-cell partial sums of the vertex averages, allocated on first use
  void* stage_rec;        // property ODEs, on first use: StageRec cell [4][cap] u32, x-hat [dim][4][cap] float2, then G [4][dim^2][cap] float2
  cudaStream_t stream;
  // optional event timing of pic_advect (instrumentation)
  int timing;
  int n_ev;                // event pairs recorded since the last read
  int ev_cap;
  cudaEvent_t* ev;         // 3 events per step: before advect, after advect, after rebin
};

namespace pic {

// ---------------------------------------------------- host error helpers --
void set_error(const char* fmt, ...);
pic_status cuda_fail(cudaError_t e, const char* what);
#define PIC_CUDA(call)                                 \
  do {                                                 \
    cudaError_t _e = (call);                           \
    if (_e != cudaSuccess) return pic::cuda_fail(_e, #call); \
  } while (0)

// ------------------------------------------------------- device views --

struct MeshView {
  int n[3], nv[3], nq[3];
  uint32_t C;
  int64_t nverts, nnodes;
  const double* X;
  const double* U;
  const double* bbox;
  const float4* bbox32;
  const float4* blk;
  const uint32_t* qbase;
  const float4* Qc;   // per-cell monomial coefficients of the field (and of the second field)
  const float4* Qcn;
  const float4* Qf;   // their high parts (FP32-basis form; null until that form is first used)
  const float4* Qfn;
  int has_next;
  int stage_df;  // FP32-basis form: stage points too take the double-float Newton step (set per pic_advect call)
  double dlo[3], dhi[3];
};

inline MeshView mesh_view(const pic_mesh_s* m) {
  MeshView v;
  for (int a = 0; a < 3; ++a) {
    v.n[a] = m->n[a];
    v.nv[a] = m->nv[a];
    v.nq[a] = m->nq[a];
    v.dlo[a] = m->dlo[a];
    v.dhi[a] = m->dhi[a];
  }
  v.C = m->C;
  v.nverts = m->nverts;
  v.nnodes = m->nnodes;
  v.X = m->X;
  v.U = m->U;
  v.bbox = m->bbox;
  v.bbox32 = m->bbox32;
  v.blk = m->blk;
  v.qbase = m->qbase;
  v.Qc = m->Qc;
  v.Qcn = m->Qcn;
  v.Qf = m->Qf;
  v.Qfn = m->Qfn;
  v.has_next = m->has_next;
  v.stage_df = 0;
  return v;
}

struct StoreView {
  double* x;      // [dim][cap]
  float2* xhat;   // [dim][cap] double-float reference coordinates
  uint64_t* id;
  uint32_t* cell;
  double* props;  // [P][cap]
  size_t cap;
  int n_props;
};

inline StoreView store_view(pic_particles_s* p, int buf) {
  StoreView s;
  s.x = p->x[buf];
  s.xhat = p->xhat[buf];
  s.id = p->id[buf];
  s.cell = p->cell[buf];
  s.props = p->props[buf];
  s.cap = p->capacity;
  s.n_props = p->n_props;
  return s;
}

// Nanoseconds of the GPU's global timer (bounds every device-side wait).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void latch_status(DevCounters* c, unsigned int bit) {
  if ((c->status & bit) == 0) atomicOr(&c->status, bit);
}

// Cell (i,j,k) from its index.
template <int D>
__device__ __forceinline__ void cell_ijk(const MeshView& m, uint32_t K, int ijk[3]) {
  ijk[0] = (int)(K % (uint32_t)m.n[0]);
  if (D == 3) {
    uint32_t r = K / (uint32_t)m.n[0];
    ijk[1] = (int)(r % (uint32_t)m.n[1]);
    ijk[2] = (int)(r / (uint32_t)m.n[1]);
  } else {
    ijk[1] = (int)(K / (uint32_t)m.n[0]);
    ijk[2] = 0;
  }
}

template <int D>
__device__ __forceinline__ uint32_t cell_index(const MeshView& m, int i, int j, int k) {
  return (uint32_t)i + (uint32_t)m.n[0] * ((uint32_t)j + (D == 3 ? (uint32_t)m.n[1] * (uint32_t)k : 0u));
}

// --------------------------------------------------- cell geometry (FP64) --
// The (bi/tri)linear map Phi_K(t) = sum_v X_v w_v(t), w_v = prod_j (v_j ? t_j
// : 1-t_j), is held as offsets from vertex 0 so that the Newton residual
// (y - X_0) - sum_v (X_v - X_0) w_v(t) carries no cancellation of O(1)
// coordinates.

template <int D>
struct CellGeom {
  double x0[D];                 // vertex 0
  double e[(1 << D)][D];        // X_v - X_0 (e[0] = 0)
};

template <int D>
__device__ __forceinline__ void load_cell(const MeshView& m, uint32_t K, CellGeom<D>& g) {
  int c[3];
  cell_ijk<D>(m, K, c);
  int64_t v0 = (int64_t)c[0] + (int64_t)m.nv[0] * ((int64_t)c[1] + (D == 3 ? (int64_t)m.nv[1] * c[2] : 0));
#pragma unroll
  for (int a = 0; a < D; ++a) g.x0[a] = __ldg(m.X + a * m.nverts + v0);
#pragma unroll
  for (int v = 0; v < (1 << D); ++v) {
    int64_t off = (int64_t)(v & 1) + (int64_t)m.nv[0] * ((int64_t)((v >> 1) & 1) +
                                                        (D == 3 ? (int64_t)m.nv[1] * ((v >> 2) & 1) : 0));
#pragma unroll
    for (int a = 0; a < D; ++a) g.e[v][a] = (v == 0) ? 0.0 : __ldg(m.X + a * m.nverts + v0 + off) - g.x0[a];
  }
}

// phi = Phi_K(t) - X_0 and J = dPhi/dt.
template <int D>
__device__ __forceinline__ void map_and_jacobian(const CellGeom<D>& g, const double t[D], double phi[D],
                                                 double J[D][D]) {
#pragma unroll
  for (int a = 0; a < D; ++a) {
    phi[a] = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j) J[a][j] = 0.0;
  }
#pragma unroll
  for (int v = 1; v < (1 << D); ++v) {
    double w = 1.0, dw[D];
#pragma unroll
    for (int j = 0; j < D; ++j) dw[j] = 1.0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const bool hi = (v >> j) & 1;
      const double f = hi ? t[j] : 1.0 - t[j];
      const double df = hi ? 1.0 : -1.0;
      w *= f;
#pragma unroll
      for (int q = 0; q < D; ++q) dw[q] *= (q == j) ? df : f;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      phi[a] += g.e[v][a] * w;
#pragma unroll
      for (int j = 0; j < D; ++j) J[a][j] += g.e[v][a] * dw[j];
    }
  }
}

template <int D>
__device__ __forceinline__ void map_point(const CellGeom<D>& g, const double t[D], double x[D]) {
  double phi[D], J[D][D];
  map_and_jacobian<D>(g, t, phi, J);
#pragma unroll
  for (int a = 0; a < D; ++a) x[a] = g.x0[a] + phi[a];
}

// Solve J d = r with the adjugate; false if J is singular.
template <int D>
__device__ __forceinline__ bool solve(const double J[D][D], const double r[D], double d[D]) {
  if (D == 2) {
    double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    if (!(fabs(det) > 0.0) || !isfinite(det)) return false;
    double inv = 1.0 / det;
    d[0] = (J[1][1] * r[0] - J[0][1] * r[1]) * inv;
    d[1] = (J[0][0] * r[1] - J[1][0] * r[0]) * inv;
    return true;
  } else {
    double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    if (!(fabs(det) > 0.0) || !isfinite(det)) return false;
    double inv = 1.0 / det;
    double c10 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    double c11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    double c12 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    double c20 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    double c21 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    double c22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    // inverse = adj / det, adj[i][j] = cofactor[j][i]
    d[0] = (c00 * r[0] + c10 * r[1] + c20 * r[2]) * inv;
    d[1] = (c01 * r[0] + c11 * r[1] + c21 * r[2]) * inv;
    d[2] = (c02 * r[0] + c12 * r[1] + c22 * r[2]) * inv;
    return true;
  }
}

// Newton for t = Phi_K^{-1}(y); `t` holds the start on entry.  Returns true
// on convergence; adds the iterations to `iters`.
template <int D>
__device__ __forceinline__ bool newton(const CellGeom<D>& g, const double y[D], double t[D], int& iters) {
  double y0[D];
#pragma unroll
  for (int a = 0; a < D; ++a) y0[a] = y[a] - g.x0[a];
  for (int it = 0; it < kNewtonMaxIt; ++it) {
    ++iters;
    double phi[D], J[D][D], r[D], d[D];
    map_and_jacobian<D>(g, t, phi, J);
#pragma unroll
    for (int a = 0; a < D; ++a) r[a] = y0[a] - phi[a];
    if (!solve<D>(J, r, d)) return false;
    double dm = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      t[a] += d[a];
      dm = fmax(dm, fabs(d[a]));
    }
    if (!isfinite(dm)) return false;
    if (dm <= kNewtonTol) return true;
  }
  return false;
}

template <int D>
__device__ __forceinline__ bool in_ref_cell(const double t[D]) {
  bool in = true;
#pragma unroll
  for (int a = 0; a < D; ++a) in = in && (t[a] >= -kInsideEps) && (t[a] <= 1.0 + kInsideEps);
  return in;
}

}  // namespace pic

namespace pic {
// ---------------------------------------------- host-side internal calls --
// Rebuild the sorted store from the cells found by the last locate
// (cell_new, counts already filled).  Defined in rebin.cu.
pic_status rebin_from_counts(pic_particles_s* p, cudaStream_t s);
// The two halves of rebin_from_counts: the new order (perm, offsets, sorted
// cells in the other buffer), then the gather that applies it.
pic_status rebin_order_from_counts(pic_particles_s* p, cudaStream_t s);
// Stage records of one step (props.cu): for evaluation point p < 4 of the
// particle in slot i (store order at the start of the step), the located
// cell at cell[p cap + i] and component a of its double-float x-hat at
// t[(4 a + p) cap + i], so that record r = p cap + i has its components at
// t[a 4 cap + r].
struct StageRec {
  uint32_t* cell;
  float2* t;
  size_t cap;
};
// One particle step of pic_advect (FP64 form, in place, counts and cell_new
// for the rebin) that also writes the stage records.
void launch_advect_record(pic_particles_s* p, const MeshView& m, double dt, int rk, const StageRec& rec,
                          cudaStream_t st);
pic_status rebin_apply_order(pic_particles_s* p, cudaStream_t s);
// pic_advect leaves its last rebin's order pending (the next pic_advect
// applies it inside its advect, pic_interpolate_to_cells reads through it);
// every other call that reads or writes the particle arrays in slot order
// applies it first with this (a gather on stream s; nothing when none is
// pending).  Defined in rebin.cu.
pic_status settle_order(pic_particles_s* p, cudaStream_t s);
// Counting, cell offsets and store allocation shared by the generators
// (particles.cu); the store's buffer 0 is then filled by the caller.
pic_status seed_prepare(pic_mesh mesh, const uint32_t* per_cell, uint32_t uniform_count, int n_props, size_t capacity,
                        cudaStream_t st, const char* who, pic_particles_s** out, size_t* n_out);
// Exclusive scan of n u32 values into out[0..n] (out[n] = total); total also
// written to *total_dev when non-null; cursor_init, when non-null, receives
// out[0..n) too.  scratch: scan_scratch_bytes(n) bytes (cleared by the
// call).  Defined in rebin.cu.
pic_status scan_u32(const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* scratch, uint32_t* total_dev,
                    uint32_t* cursor_init, cudaStream_t s, unsigned int* status = nullptr);
int num_sms();
// Allocate a store (particles.cu); takes ownership of cell_off.
pic_particles_s* store_alloc(int dim, int n_props, uint32_t C, size_t capacity, uint32_t* cell_off);
// Stateless sort of items by (cell, id), used by pic_sort_by_cell.  Defined
// in rebin.cu.
struct SortScratch {
  uint32_t* misc;  // [0] item count, [1] status bits, [2] items kept
  uint32_t* counts;
  uint32_t* cursor;
  uint32_t* block_sums;
  uint64_t* key_id;
  uint32_t* key_src;
};
// Items per tile of the single-pass scan (scan_u32), and the bytes of its
// scratch: one 64-bit state word per tile and the tile counter.
constexpr uint32_t kScanTileCells = 4096;
__host__ __device__ constexpr uint32_t scan_tiles(uint32_t n) { return (n + kScanTileCells - 1) / kScanTileCells; }
constexpr size_t scan_scratch_bytes(uint32_t n) { return sizeof(uint64_t) * ((size_t)scan_tiles(n) + 1); }
// Bytes of the stateless sort's scratch for n items and C cells, in the order
// sort_scratch_layout carves them (each piece rounded up to 256 B): status
// words, counts[C], cursor[C], scan scratch, key_id[n] u64, key_src[n] u32.
constexpr size_t sort_scratch_up(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t sort_scratch_bytes(size_t n, uint32_t C) {
  return sort_scratch_up(sizeof(uint32_t) * 4) + 2 * sort_scratch_up(sizeof(uint32_t) * (size_t)C) +
         sort_scratch_up(scan_scratch_bytes(C)) + sort_scratch_up(sizeof(uint64_t) * (n ? n : 1)) +
         sort_scratch_up(sizeof(uint32_t) * (n ? n : 1));
}
SortScratch sort_scratch_layout(void* base, size_t n, uint32_t C);
pic_status sort_by_cell_check(size_t n, const uint32_t* cell, const uint64_t* id, uint32_t C, const uint32_t* perm,
                              const uint32_t* cell_off, const char* who);
pic_status sort_by_cell_run(size_t n, const uint32_t* cell, const uint64_t* id, uint32_t C, uint32_t* perm,
                            uint32_t* cell_off, const SortScratch& sc, cudaStream_t s);
// Host-side count of kernel launches (instrumentation).
void count_launches(int n);
// Allocate and fill the FP32 coefficient tables (Qf, and Qfn with a second
// field) of the mesh's current fields, if not there yet; later field
// updates keep them current.  Defined in mesh.cu.
pic_status ensure_fp32_coefficients(pic_mesh_s* m, cudaStream_t st);
}  // namespace pic
