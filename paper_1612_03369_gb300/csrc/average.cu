// average.cu -- particle -> cell transfer, scheme (ii) of Sec. 2.7
// (arithmetic average of the particles of each cell; linear in the particle
// count because the store is sorted by cell).
#include "pic_internal.cuh"

namespace pic {

// Thread per cell: the particles of a cell are folded in store order (the
// order of the definition), then combined with their number.  The threads of
// a warp read neighbouring segments, so every sector fetched from HBM is used
// by the following iterations through L1.  Kinds (Sec. 2.7 (ii)):
//   0 arithmetic  sum v / n
//   1 geometric   exp(sum log v / n)   (NaN if the cell holds a v <= 0)
//   2 harmonic    n / sum (1 / v)      (NaN if the cell holds a v <= 0)
// PERM (an order left pending by pic_advect): slot i's value is
// prop[perm[i]], the same values in the same order as after the gather.
template <int KIND, bool PERM>
__global__ void __launch_bounds__(256) cell_average_kernel(const uint32_t* __restrict__ cell_off,
                                                           const double* __restrict__ prop,
                                                           const uint32_t* __restrict__ perm, uint32_t C, size_t cap,
                                                           double empty_fill, double* __restrict__ avg,
                                                           uint32_t* __restrict__ count, DevCounters* __restrict__ ctr) {
  for (uint32_t K = blockIdx.x * blockDim.x + threadIdx.x; K < C; K += gridDim.x * blockDim.x) {
    const uint32_t beg = cell_off[K], end = cell_off[K + 1];
    if (end > cap || beg > end) {
      latch_status(ctr, PIC_STATUS_BOUNDS);
      continue;
    }
    double s = 0.0;
    bool bad = false;
    for (uint32_t i = beg; i < end; ++i) {
      uint32_t src = i;
      if constexpr (PERM) {
        src = perm[i];
        if (src >= cap) {
          bad = true;
          latch_status(ctr, PIC_STATUS_BOUNDS);
          continue;
        }
      }
      const double v = prop[src];
      if constexpr (KIND == 0) {
        s += v;
      } else {
        bad = bad || !(v > 0.0);
        s += (KIND == 1) ? log(v) : 1.0 / v;
      }
    }
    const uint32_t n = end - beg;
    double r = empty_fill;
    if (n) {
      if constexpr (KIND == 0)
        r = s / (double)n;
      else if (bad)
        r = __longlong_as_double(0x7ff8000000000000ll);
      else
        r = (KIND == 1) ? exp(s / (double)n) : (double)n / s;
    }
    avg[K] = r;
    if (count) count[K] = n;
  }
}

}  // namespace pic

using namespace pic;

extern "C" pic_status pic_interpolate_to_cells(pic_particles p, pic_mesh mesh, int prop, pic_average kind, double* avg,
                                               uint32_t* count, double empty_fill, void* stream) {
  if (!p || !mesh || !avg) return (set_error("pic_interpolate_to_cells: null argument"), PIC_ERR_ARG);
  if (p->mesh != mesh) return (set_error("pic_interpolate_to_cells: mesh mismatch"), PIC_ERR_ARG);
  if (prop < 0 || prop >= p->n_props)
    return (set_error("pic_interpolate_to_cells: property %d out of range", prop), PIC_ERR_ARG);
  if (kind != PIC_AVG_ARITHMETIC && kind != PIC_AVG_GEOMETRIC && kind != PIC_AVG_HARMONIC)
    return (set_error("pic_interpolate_to_cells: unknown average %d", (int)kind), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  size_t grid = ((size_t)p->C + 255) / 256;
  const size_t cap = (size_t)num_sms() * 16;
  if (grid > cap) grid = cap;
  const int g = (int)(grid ? grid : 1);
  const double* pv = p->props[p->cur] + (size_t)prop * p->capacity;
  // read through a pending order, do not apply it
  const uint32_t* pm = p->perm;
  const uint32_t C = p->C;
  const size_t cp = p->capacity;
  if (p->pending_order) {
    if (kind == PIC_AVG_ARITHMETIC)
      cell_average_kernel<0, true><<<g, 256, 0, st>>>(p->cell_off, pv, pm, C, cp, empty_fill, avg, count, p->ctr);
    else if (kind == PIC_AVG_GEOMETRIC)
      cell_average_kernel<1, true><<<g, 256, 0, st>>>(p->cell_off, pv, pm, C, cp, empty_fill, avg, count, p->ctr);
    else
      cell_average_kernel<2, true><<<g, 256, 0, st>>>(p->cell_off, pv, pm, C, cp, empty_fill, avg, count, p->ctr);
  } else {
    if (kind == PIC_AVG_ARITHMETIC)
      cell_average_kernel<0, false><<<g, 256, 0, st>>>(p->cell_off, pv, pm, C, cp, empty_fill, avg, count, p->ctr);
    else if (kind == PIC_AVG_GEOMETRIC)
      cell_average_kernel<1, false><<<g, 256, 0, st>>>(p->cell_off, pv, pm, C, cp, empty_fill, avg, count, p->ctr);
    else
      cell_average_kernel<2, false><<<g, 256, 0, st>>>(p->cell_off, pv, pm, C, cp, empty_fill, avg, count, p->ctr);
  }
  count_launches(1);
  PIC_CUDA(cudaGetLastError());
  return PIC_OK;
}
