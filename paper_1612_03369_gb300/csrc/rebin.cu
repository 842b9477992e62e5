// rebin.cu -- rebuilding the particle store sorted by (cell, id) after the
// particles have been located (Sec. 2.1: the store keeps particles sorted
// by containing cell; Sec. 2.4: movers are collected and re-inserted in one
// batch, and particles in no cell are discarded).
//
// A counting sort by new cell followed by a rank sort by id inside each
// cell's segment:
//   counts[K]   particles whose new cell is K (filled by the locate kernel)
//   scan        cell_off = exclusive prefix sum of counts; cursor = cell_off
//   scatter     (id, old slot) of each particle to a free slot of its cell
//   rank        slot of each particle = segment start + its rank by id
//   gather      every field copied from the old slot to the new slot
// The result is a function of the particle set alone (no dependence on the
// order the atomics of the scatter were served in).
#include "pic_internal.cuh"
#include "rebin.cuh"

namespace pic {

constexpr int kScanThreads = 1024;
constexpr uint32_t kScanTile = kScanThreads * kScanItems;
static_assert(kScanTile == kScanTileCells, "scan tile size and the scratch layout disagree");

// Single-pass exclusive scan (decoupled look-back, after Merrill & Garland,
// "Single-pass parallel prefix scan with decoupled look-back", NVIDIA 2016).
// A block takes its tile in arrival order from a counter, so every tile it
// waits on belongs to a block that has already started.  It sums its tile
// (warp shuffles, then one warp over the warp sums), publishes the sum
// (flag A), then its first warp walks back over the predecessors 32 at a
// time: the nearest inclusive prefix (flag P) in the window ends the walk
// with the sums (flag A) after it added, a window of sums only is added and
// the walk goes on.  The block then publishes its own inclusive prefix (flag P)
// and writes its tile.  Each state word holds the flag in its top two bits
// and the value below.  The wait for a predecessor that has not published is
// bounded by the global timer; if it runs out the block latches
// PIC_STATUS_TIMEOUT (its offsets are then wrong, which the rebin's bounds
// checks catch and flag).
constexpr uint64_t kScanFlagA = 1ull << 62, kScanFlagP = 2ull << 62, kScanValue = (1ull << 62) - 1;
constexpr unsigned long long kScanWaitNs = 1000000000ull;

__global__ void __launch_bounds__(kScanThreads) scan_single_pass_kernel(const uint32_t* __restrict__ in, uint32_t n,
                                                                        uint64_t* __restrict__ state,
                                                                        uint32_t* __restrict__ out,
                                                                        uint32_t* __restrict__ cursor,
                                                                        uint32_t* __restrict__ total_dev,
                                                                        unsigned int* __restrict__ status) {
  __shared__ uint32_t s_tile, s_prefix, s_total;
  const uint32_t ntiles = scan_tiles(n);
  if (threadIdx.x == 0) s_tile = atomicAdd(reinterpret_cast<unsigned int*>(state + ntiles), 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  if (t >= ntiles) return;  // block-uniform
  const uint32_t base = t * kScanTileCells + threadIdx.x * kScanItems;
  uint32_t v[kScanItems], sum = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    v[q] = (base + q < n) ? in[base + q] : 0u;
    sum += v[q];
  }
  const uint32_t ex = block_excl_scan(sum, &s_total);  // ends with a block barrier
  if (threadIdx.x < 32) {
    const uint32_t lane = threadIdx.x;
    const uint32_t total = s_total;
    uint64_t prefix = 0;
    if (t == 0) {
      if (lane == 0) {
        __threadfence();
        atomicExch(reinterpret_cast<unsigned long long*>(state), (unsigned long long)(kScanFlagP | total));
      }
    } else {
      if (lane == 0) {
        __threadfence();
        atomicExch(reinterpret_cast<unsigned long long*>(state + t), (unsigned long long)(kScanFlagA | total));
      }
      // warp 0 reads the 32 predecessors [p_end - 31, p_end] at once (lane
      // 31 the nearest; before tile 0 an inclusive prefix of 0): once all
      // have published, the nearest inclusive prefix and the sums after it
      // end the walk, else their 32 sums are added and the window moves on
      volatile uint64_t* vs = state;
      int64_t p_end = (int64_t)t - 1;
      const unsigned long long t0 = global_ns();
      for (;;) {
        const int64_t p = p_end - (31 - (int64_t)lane);
        uint64_t w = kScanFlagP;
        if (p >= 0) w = vs[p];
        const uint64_t flag = w & ~kScanValue;
        if (__any_sync(0xffffffffu, flag == 0)) {
          if (__any_sync(0xffffffffu, global_ns() - t0 > kScanWaitNs)) {
            if (lane == 0) atomicOr(status, PIC_STATUS_TIMEOUT);
            break;
          }
          continue;
        }
        const unsigned pm = __ballot_sync(0xffffffffu, flag == kScanFlagP);
        const int hp = pm ? 31 - __clz((int)pm) : -1;
        prefix += __reduce_add_sync(0xffffffffu, (int)lane >= hp ? (uint32_t)(w & kScanValue) : 0u);
        if (pm) break;
        p_end -= 32;
      }
      if (lane == 0) {
        __threadfence();
        atomicExch(reinterpret_cast<unsigned long long*>(state + t),
                   (unsigned long long)(kScanFlagP | (prefix + total)));
      }
    }
    if (lane == 0) s_prefix = (uint32_t)prefix;
  }
  __syncthreads();
  uint32_t run = s_prefix + ex;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    const uint32_t i = base + q;
    if (i < n) {
      out[i] = run;
      if (cursor) cursor[i] = run;
    }
    run += v[q];
    if (i + 1 == n) {
      out[n] = run;
      if (total_dev) *total_dev = run;
    }
  }
}

// The scan's status word: the store's counters where there is one, else a
// word of the scratch past the tile states (cleared with them).
pic_status scan_u32(const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* scratch, uint32_t* total_dev,
                    uint32_t* cursor_init, cudaStream_t s, unsigned int* status) {
  if (n == 0) return PIC_OK;
  const uint32_t nt = scan_tiles(n);
  uint64_t* state = reinterpret_cast<uint64_t*>(scratch);
  PIC_CUDA(cudaMemsetAsync(state, 0, sizeof(uint64_t) * (nt + 1), s));
  unsigned int* st = status ? status : reinterpret_cast<unsigned int*>(state + nt) + 1;
  scan_single_pass_kernel<<<nt, kScanThreads, 0, s>>>(in, n, state, out, cursor_init, total_dev, st);
  count_launches(1);
  PIC_CUDA(cudaGetLastError());
  return PIC_OK;
}

// (id, old slot) of every located particle into a free slot of its new cell.
// The item count is *n_dev; anything else found wrong is latched in *status.
__global__ void __launch_bounds__(256) scatter_keys_kernel(const uint32_t* __restrict__ cell_new,
                                                           const uint64_t* __restrict__ id, uint32_t* __restrict__ cursor,
                                                           uint64_t* __restrict__ key_id, uint32_t* __restrict__ key_src,
                                                           uint32_t C, size_t cap, const uint32_t* __restrict__ n_dev,
                                                           unsigned int* __restrict__ status) {
  scatter_phase(cell_new, id, cursor, key_id, key_src, C, cap, *n_dev, status, blockIdx.x * blockDim.x + threadIdx.x,
                gridDim.x * blockDim.x);
}

// Rank by id within each cell.  cell_out may be NULL.  When publish_dst is
// given, block 0 copies *publish_src there (the new particle count).
__global__ void __launch_bounds__(256) rank_by_id_kernel(const uint32_t* __restrict__ cell_off, const uint64_t* __restrict__ key_id,
                                                         const uint32_t* __restrict__ key_src, uint32_t* __restrict__ perm,
                                                         uint32_t* __restrict__ cell_out, uint32_t C, size_t cap,
                                                         unsigned int* __restrict__ status, uint32_t* publish_dst,
                                                         const uint32_t* publish_src) {
  if (publish_dst && blockIdx.x == 0 && threadIdx.x == 0) *publish_dst = *publish_src;
  rank_phase(cell_off, key_id, key_src, perm, cell_out, C, cap, status, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
             (gridDim.x * blockDim.x) >> 5);
}

// Copy every field from the old slot perm[j] to the new slot j.
__global__ void __launch_bounds__(256) gather_kernel(const __grid_constant__ StoreView src, const __grid_constant__ StoreView dst, const uint32_t* __restrict__ perm, int dim,
                                                     DevCounters* __restrict__ ctr) {
  gather_phase(src, dst, perm, dim, ctr->n_alive, &ctr->status, blockIdx.x * blockDim.x + threadIdx.x,
               gridDim.x * blockDim.x);
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
  }
  return sms;
}

static int grid_cap(size_t n, int block, int per_sm) {
  size_t want = (n + block - 1) / block;
  size_t cap = (size_t)num_sms() * per_sm;
  size_t g = want < cap ? want : cap;
  return (int)(g ? g : 1);
}

// The new order of the store after a step: cell offsets, perm (new slot ->
// old slot) and the sorted cells written into the other buffer; n_alive
// becomes the survivors' count.  The particles have not moved yet.
pic_status rebin_order_from_counts(pic_particles_s* p, cudaStream_t s) {
  pic_status r = scan_u32(p->counts, p->cell_off, p->C, p->block_sums, &p->ctr->n_next, p->cursor, s, &p->ctr->status);
  if (r != PIC_OK) return r;
  const StoreView a = store_view(p, p->cur), b = store_view(p, 1 - p->cur);
  scatter_keys_kernel<<<grid_cap(p->capacity, 256, 16), 256, 0, s>>>(p->cell_new, a.id, p->cursor, p->key_id, p->key_src,
                                                                     p->C, p->capacity, &p->ctr->n_alive, &p->ctr->status);
  rank_by_id_kernel<<<grid_cap((size_t)p->C * 32, 256, 16), 256, 0, s>>>(p->cell_off, p->key_id, p->key_src, p->perm,
                                                                        b.cell, p->C, p->capacity, &p->ctr->status,
                                                                        &p->ctr->n_alive, &p->ctr->n_next);
  count_launches(2);
  PIC_CUDA(cudaGetLastError());
  return PIC_OK;
}

// Move the particles into the order rebin_order_from_counts computed.
pic_status rebin_apply_order(pic_particles_s* p, cudaStream_t s) {
  const StoreView a = store_view(p, p->cur), b = store_view(p, 1 - p->cur);
  gather_kernel<<<grid_cap(p->capacity, 256, 16), 256, 0, s>>>(a, b, p->perm, p->dim, p->ctr);
  count_launches(1);
  PIC_CUDA(cudaGetLastError());
  p->cur = 1 - p->cur;
  return PIC_OK;
}

pic_status settle_order(pic_particles_s* p, cudaStream_t s) {
  if (!p->pending_order) return PIC_OK;
  p->pending_order = 0;
  return rebin_apply_order(p, s);
}

pic_status rebin_from_counts(pic_particles_s* p, cudaStream_t s) {
  pic_status r = rebin_order_from_counts(p, s);
  if (r != PIC_OK) return r;
  return rebin_apply_order(p, s);
}

// cell_new = cell, counts = histogram of cell (the identity relocation).
__global__ void identity_cells_kernel(const uint32_t* __restrict__ cell, uint32_t* __restrict__ cell_new,
                                      uint32_t* __restrict__ counts, uint32_t C, DevCounters* __restrict__ ctr) {
  const uint32_t n = ctr->n_alive;
  const uint32_t lane = threadIdx.x & 31u;
  for (uint32_t base = blockIdx.x * blockDim.x + threadIdx.x - lane; base < n; base += gridDim.x * blockDim.x) {
    const uint32_t i = base + lane;
    uint32_t K = PIC_LOST;
    if (i < n) {
      K = cell[i];
      if (K >= C) {
        latch_status(ctr, PIC_STATUS_BOUNDS);
        K = PIC_LOST;
      }
      cell_new[i] = K;
    }
    (void)aggregated_increment(counts, K, K != PIC_LOST);
  }
}

// Histogram of the cells of n items (entries >= C, lost or not, are skipped;
// entries other than PIC_LOST that are >= C are flagged).
__global__ void count_cells_kernel(const uint32_t* __restrict__ cell, uint32_t n, uint32_t C,
                                   uint32_t* __restrict__ counts, unsigned int* __restrict__ status) {
  const uint32_t lane = threadIdx.x & 31u;
  for (uint32_t base = blockIdx.x * blockDim.x + threadIdx.x - lane; base < n; base += gridDim.x * blockDim.x) {
    const uint32_t i = base + lane;
    const uint32_t K = i < n ? cell[i] : PIC_LOST;
    if (K != PIC_LOST && K >= C) atomicOr(status, PIC_STATUS_BOUNDS);
    (void)aggregated_increment(counts, K, K < C);
  }
}

SortScratch sort_scratch_layout(void* base, size_t n, uint32_t C) {
  // the pieces and their order are those counted by sort_scratch_bytes
  auto up = sort_scratch_up;
  char* p = (char*)base;
  SortScratch sc;
  sc.misc = (uint32_t*)p;  // [0] n, [1] status, [2] kept
  p += up(sizeof(uint32_t) * 4);
  sc.counts = (uint32_t*)p;
  p += up(sizeof(uint32_t) * (size_t)C);
  sc.cursor = (uint32_t*)p;
  p += up(sizeof(uint32_t) * (size_t)C);
  sc.block_sums = (uint32_t*)p;
  p += up(scan_scratch_bytes(C));
  sc.key_id = (uint64_t*)p;
  p += up(sizeof(uint64_t) * (n ? n : 1));
  sc.key_src = (uint32_t*)p;
  return sc;
}

__global__ void sort_init_kernel(uint32_t* misc, uint32_t n) {
  misc[0] = n;
  misc[1] = 0;
  misc[2] = 0;
}

// Order of n items by (cell, id): counting sort by cell, then rank by id
// within each cell (the rebin of the store, on caller-owned arrays).
pic_status sort_by_cell_run(size_t n, const uint32_t* cell, const uint64_t* id, uint32_t C, uint32_t* perm,
                            uint32_t* cell_off, const SortScratch& sc, cudaStream_t s) {
  PIC_CUDA(cudaMemsetAsync(sc.counts, 0, sizeof(uint32_t) * C, s));
  sort_init_kernel<<<1, 1, 0, s>>>(sc.misc, (uint32_t)n);
  if (n) count_cells_kernel<<<grid_cap(n, 256, 16), 256, 0, s>>>(cell, (uint32_t)n, C, sc.counts, sc.misc + 1);
  pic_status r = scan_u32(sc.counts, cell_off, C, sc.block_sums, sc.misc + 2, sc.cursor, s, sc.misc + 1);
  if (r != PIC_OK) return r;
  if (n) {
    scatter_keys_kernel<<<grid_cap(n, 256, 16), 256, 0, s>>>(cell, id, sc.cursor, sc.key_id, sc.key_src, C, n, sc.misc,
                                                             sc.misc + 1);
    rank_by_id_kernel<<<grid_cap((size_t)C * 32, 256, 16), 256, 0, s>>>(cell_off, sc.key_id, sc.key_src, perm, nullptr, C,
                                                                        n, sc.misc + 1, nullptr, nullptr);
  }
  count_launches(n ? 4 : 1);
  PIC_CUDA(cudaGetLastError());
  return PIC_OK;
}

pic_status sort_by_cell_check(size_t n, const uint32_t* cell, const uint64_t* id, uint32_t C, const uint32_t* perm,
                              const uint32_t* cell_off, const char* who) {
  if (C == 0) return (set_error("%s: n_cells must be >= 1", who), PIC_ERR_ARG);
  if (n >= 0xFFFFFFF0ull) return (set_error("%s: %zu items exceed the 32-bit index range", who, n), PIC_ERR_ARG);
  if (!cell_off || (n && (!cell || !id || !perm))) return (set_error("%s: null array", who), PIC_ERR_ARG);
  return PIC_OK;
}

}  // namespace pic

using namespace pic;

extern "C" pic_status pic_sort_by_cell(size_t n, const uint32_t* cell, const uint64_t* id, uint32_t n_cells,
                                       uint32_t* perm, uint32_t* cell_off, void* stream) {
  pic_status r = sort_by_cell_check(n, cell, id, n_cells, perm, cell_off, "pic_sort_by_cell");
  if (r != PIC_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  void* scratch = nullptr;
  PIC_CUDA(cudaMallocAsync(&scratch, sort_scratch_bytes(n, n_cells), st));
  r = sort_by_cell_run(n, cell, id, n_cells, perm, cell_off, sort_scratch_layout(scratch, n, n_cells), st);
  cudaError_t e = cudaFreeAsync(scratch, st);
  if (r != PIC_OK) return r;
  if (e != cudaSuccess) return cuda_fail(e, "pic_sort_by_cell: cudaFreeAsync");
  return PIC_OK;
}

extern "C" pic_status pic_rebin(pic_particles parts, void* stream) {
  if (!parts) return (set_error("pic_rebin: null handle"), PIC_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  {
    const pic_status r0 = settle_order(parts, st);
    if (r0 != PIC_OK) return r0;
  }
  PIC_CUDA(cudaMemsetAsync(parts->counts, 0, sizeof(uint32_t) * parts->C, st));
  identity_cells_kernel<<<grid_cap(parts->capacity, 256, 16), 256, 0, st>>>(parts->cell[parts->cur], parts->cell_new,
                                                                          parts->counts, parts->C, parts->ctr);
  count_launches(1);
  PIC_CUDA(cudaGetLastError());
  return rebin_from_counts(parts, st);
}
