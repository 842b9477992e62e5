// exchange.cu -- moving particles between stores: a contiguous range of the
// sorted store out, and particles with known cells in (Sec. 2.4: particles
// that leave a process's part of the mesh are sent to the owner of their new
// cell together with that cell, so that the receiver does not search for it).
//
// With the mesh split into slabs of whole cell layers along the last axis,
// a store's sorted order puts the particles that moved into the layers
// below its own at the start and those that moved above at the end: each
// is one contiguous range (pic_export_range).  The receiver keeps its own
// cells' particles, adds the received ones at their cells and re-sorts
// (pic_merge_particles).
#include "df.cuh"
#include "pic_internal.cuh"
#include "rebin.cuh"

namespace pic {

__global__ void range_xhat_kernel(const float2* __restrict__ src, double* __restrict__ dst, size_t cap, size_t first,
                                  size_t count, int dim) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < count * dim; q += (size_t)gridDim.x * blockDim.x) {
    const size_t a = q / count, i = q % count;
    const float2 v = src[a * cap + first + i];
    dst[a * count + i] = (double)v.x + (double)v.y;  // exact: the pair holds at most 48 significant bits
  }
}

// Slots [0, n_old) keep their particle if its cell lies in [keep_lo,
// keep_hi); slots [n_old, n_old + n_in) receive the incoming particles at
// their cells (cell_in + shift).  Every kept or received particle is counted
// in its cell; the others get no cell and are dropped by the rebin.
__global__ void merge_classify_kernel(StoreView s, uint32_t n_old, uint32_t n_in, const double* __restrict__ x_in,
                                      const double* __restrict__ xhat_in, const uint64_t* __restrict__ id_in,
                                      const uint32_t* __restrict__ cell_in, long long shift,
                                      const double* __restrict__ props_in, int dim, uint32_t keep_lo, uint32_t keep_hi,
                                      uint32_t C, uint32_t* __restrict__ cell_new, uint32_t* __restrict__ counts,
                                      DevCounters* __restrict__ ctr) {
  const uint32_t total = n_old + n_in;
  const uint32_t lane = threadIdx.x & 31u;
  for (uint32_t base = blockIdx.x * blockDim.x + threadIdx.x - lane; base < total; base += gridDim.x * blockDim.x) {
    const uint32_t j = base + lane;
    uint32_t K = PIC_LOST;
    if (j < n_old) {
      const uint32_t c = s.cell[j];
      K = (c >= keep_lo && c < keep_hi && c < C) ? c : PIC_LOST;
    } else if (j < total) {
      const uint32_t i = j - n_old;
      const long long c = (long long)cell_in[i] + shift;
      if (c >= 0 && c < (long long)C) {
        K = (uint32_t)c;
      } else {
        latch_status(ctr, PIC_STATUS_BOUNDS);
      }
      for (int a = 0; a < dim; ++a) {
        s.x[a * s.cap + j] = x_in[(size_t)a * n_in + i];
        const double t = xhat_in[(size_t)a * n_in + i];
        const float hi = __double2float_rn(t);
        s.xhat[a * s.cap + j] = make_float2(hi, __double2float_rn(t - (double)hi));
      }
      s.id[j] = id_in[i];
      for (int q = 0; q < s.n_props; ++q) s.props[(size_t)q * s.cap + j] = props_in ? props_in[(size_t)q * n_in + i] : 0.0;
      s.cell[j] = K;
    }
    if (j < total) cell_new[j] = K;
    (void)aggregated_increment(counts, K, K != PIC_LOST);
  }
}

__global__ void set_alive_kernel(DevCounters* __restrict__ ctr, uint32_t n) { ctr->n_alive = n; }

}  // namespace pic

using namespace pic;

__global__ void range_cell_kernel(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, size_t first,
                                  size_t count, long long shift) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (uint32_t)((long long)src[first + i] + shift);
}

extern "C" pic_status pic_export_range(pic_particles p, size_t first, size_t count, long long cell_shift, double* x,
                                       double* xhat, uint64_t* id, uint32_t* cell, double* props, void* stream) {
  if (!p) return (set_error("pic_export_range: null handle"), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  {
    const pic_status r0 = settle_order(p, st);
    if (r0 != PIC_OK) return r0;
  }
  unsigned int n_alive = 0;
  PIC_CUDA(cudaMemcpyAsync(&n_alive, &p->ctr->n_alive, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  PIC_CUDA(cudaStreamSynchronize(st));
  if (first > n_alive || count > n_alive - first)
    return (set_error("pic_export_range: [%zu, %zu) past the %u particles of the store", first, first + count, n_alive),
            PIC_ERR_ARG);
  if (count == 0) return PIC_OK;
  const size_t cap = p->capacity;
  const int c = p->cur;
  for (int a = 0; a < p->dim && x; ++a)
    PIC_CUDA(cudaMemcpyAsync(x + a * count, p->x[c] + a * cap + first, sizeof(double) * count, cudaMemcpyDefault, st));
  if (xhat) {
    cudaPointerAttributes at;
    const bool dev = cudaPointerGetAttributes(&at, xhat) == cudaSuccess && at.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    if (!dev) return (set_error("pic_export_range: xhat must be device memory"), PIC_ERR_ARG);
    range_xhat_kernel<<<1024, 256, 0, st>>>(p->xhat[c], xhat, cap, first, count, p->dim);
    count_launches(1);
    PIC_CUDA(cudaGetLastError());
  }
  if (id) PIC_CUDA(cudaMemcpyAsync(id, p->id[c] + first, sizeof(uint64_t) * count, cudaMemcpyDefault, st));
  if (cell) {
    if (cell_shift == 0) {
      PIC_CUDA(cudaMemcpyAsync(cell, p->cell[c] + first, sizeof(uint32_t) * count, cudaMemcpyDefault, st));
    } else {
      cudaPointerAttributes at;
      const bool dev = cudaPointerGetAttributes(&at, cell) == cudaSuccess && at.type == cudaMemoryTypeDevice;
      cudaGetLastError();
      if (!dev) return (set_error("pic_export_range: shifted cells need a device array"), PIC_ERR_ARG);
      range_cell_kernel<<<256, 256, 0, st>>>(p->cell[c], cell, first, count, cell_shift);
      count_launches(1);
      PIC_CUDA(cudaGetLastError());
    }
  }
  for (int q = 0; q < p->n_props && props; ++q)
    PIC_CUDA(cudaMemcpyAsync(props + q * count, p->props[c] + q * cap + first, sizeof(double) * count,
                             cudaMemcpyDefault, st));
  return PIC_OK;
}

extern "C" pic_status pic_merge_particles(pic_particles p, uint32_t keep_lo, uint32_t keep_hi, size_t n_in,
                                          const double* x_in, const double* xhat_in, const uint64_t* id_in,
                                          const uint32_t* cell_in, long long cell_shift, const double* props_in,
                                          void* stream) {
  if (!p) return (set_error("pic_merge_particles: null handle"), PIC_ERR_ARG);
  if (n_in && (!x_in || !xhat_in || !id_in || !cell_in))
    return (set_error("pic_merge_particles: null input array"), PIC_ERR_ARG);
  if (keep_lo > keep_hi || keep_hi > p->C)
    return (set_error("pic_merge_particles: kept cells [%u, %u) outside [0, %u)", keep_lo, keep_hi, p->C), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  {
    const pic_status r0 = settle_order(p, st);
    if (r0 != PIC_OK) return r0;
  }
  unsigned int n_old = 0;
  PIC_CUDA(cudaMemcpyAsync(&n_old, &p->ctr->n_alive, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  PIC_CUDA(cudaStreamSynchronize(st));
  if ((size_t)n_old + n_in > p->capacity)
    return (set_error("pic_merge_particles: %u + %zu particles exceed the capacity %zu", n_old, n_in, p->capacity),
            PIC_ERR_CAPACITY);
  const uint32_t total = n_old + (uint32_t)n_in;
  PIC_CUDA(cudaMemsetAsync(p->counts, 0, sizeof(uint32_t) * p->C, st));
  if (total) {
    const size_t want = ((size_t)total + 255) / 256, cap = (size_t)num_sms() * 16;
    const int g = (int)(want < cap ? want : cap);
    merge_classify_kernel<<<g, 256, 0, st>>>(store_view(p, p->cur), n_old, (uint32_t)n_in, x_in, xhat_in, id_in,
                                             cell_in, cell_shift, props_in, p->dim, keep_lo, keep_hi, p->C,
                                             p->cell_new, p->counts, p->ctr);
    set_alive_kernel<<<1, 1, 0, st>>>(p->ctr, total);
    count_launches(2);
    PIC_CUDA(cudaGetLastError());
  }
  return rebin_from_counts(p, st);
}
