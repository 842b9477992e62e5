// rebin.cuh -- the phases of the rebin (Sec. 2.1 store sorted by cell,
// Sec. 2.4 batched re-insertion) as device functions over a "virtual grid"
// (block index bid of nb blocks), so that the stand-alone kernels of
// rebin.cu and the persistent ensemble kernel run the same code.
//
//   scan   exclusive prefix sum of per-cell counts in tiles of
//          blockDim.x * kScanItems cells: tile sums, one block scans them,
//          then every tile applies its offset
//   scatter (id, old slot) of each particle to a free slot of its new cell
//   rank   new slot = segment start + rank of the id among the cell's ids
//   gather every field copied from its old slot to its new slot
#pragma once

#include "pic_internal.cuh"

namespace pic {

constexpr int kScanItems = 4;
constexpr int kMaxBlockThreads = 1024;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive
// prefix and writes the block total to *total (shared memory).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sums[kMaxBlockThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t inc = warp_incl_scan(v);
  if (lane == 31) warp_sums[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0u;
    uint32_t si = warp_incl_scan(s);
    if (lane < (int)(blockDim.x >> 5)) warp_sums[lane] = si - s;
    if (lane == 31) *total = si;
  }
  __syncthreads();
  const uint32_t r = warp_sums[w] + inc - v;
  __syncthreads();
  return r;
}

__device__ __forceinline__ uint32_t scan_tile_size() { return blockDim.x * kScanItems; }

// Tile sums of in[0..n) for tiles bid, bid + nb, ...
__device__ __forceinline__ void scan_phase_reduce(const uint32_t* __restrict__ in, uint32_t n,
                                                  uint32_t* __restrict__ tile_sums, uint32_t bid, uint32_t nb) {
  __shared__ uint32_t tot;
  const uint32_t T = scan_tile_size(), ntiles = (n + T - 1) / T;
  for (uint32_t t = bid; t < ntiles; t += nb) {
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
      const uint32_t i = t * T + q * blockDim.x + threadIdx.x;
      if (i < n) s += in[i];
    }
    (void)block_excl_scan(s, &tot);
    if (threadIdx.x == 0) tile_sums[t] = tot;
    __syncthreads();
  }
}

// One block: exclusive scan of the tile sums in place.
__device__ __forceinline__ void scan_phase_sums(uint32_t* __restrict__ sums, uint32_t ntiles) {
  __shared__ uint32_t carry_s, tot;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (uint32_t base = 0; base < ntiles; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < ntiles ? sums[i] : 0u;
    const uint32_t ex = block_excl_scan(v, &tot);
    const uint32_t carry = carry_s;
    if (i < ntiles) sums[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry_s = carry + tot;
    __syncthreads();
  }
}

// out[i] = exclusive prefix of in (and cursor[i] when given); out[n] and
// *total_dev get the total.
__device__ __forceinline__ void scan_phase_apply(const uint32_t* __restrict__ in, uint32_t n,
                                                 const uint32_t* __restrict__ tile_sums, uint32_t* __restrict__ out,
                                                 uint32_t* __restrict__ cursor, uint32_t* __restrict__ total_dev,
                                                 uint32_t bid, uint32_t nb) {
  __shared__ uint32_t tot;
  const uint32_t T = scan_tile_size(), ntiles = (n + T - 1) / T;
  for (uint32_t t = bid; t < ntiles; t += nb) {
    const uint32_t base = t * T + threadIdx.x * kScanItems;
    uint32_t v[kScanItems], s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
      v[q] = (base + q < n) ? in[base + q] : 0u;
      s += v[q];
    }
    uint32_t ex = block_excl_scan(s, &tot) + tile_sums[t];
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
      const uint32_t i = base + q;
      if (i < n) {
        out[i] = ex;
        if (cursor) cursor[i] = ex;
      }
      ex += v[q];
      if (i + 1 == n) {
        out[n] = ex;
        if (total_dev) *total_dev = ex;
      }
    }
  }
}

// Warp-aggregated increment of ctr[K]: the lanes of a warp holding the same K
// (all 32 lanes call this; lanes with take == false only vote) share one
// atomic, issued by the lowest of them.  Returns the counter's old value plus
// the lane's rank among its peers.  The particles arrive sorted by their old
// cell and most stay in it, so a warp usually holds two or three distinct
// cells: a few atomics per warp instead of 32 on the same addresses.
__device__ __forceinline__ uint32_t aggregated_increment(uint32_t* __restrict__ ctr, uint32_t K, bool take) {
  const unsigned peers = __match_any_sync(0xffffffffu, take ? K : 0xFFFFFFFFu);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (take && lane == leader) base = atomicAdd(ctr + K, (uint32_t)__popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  return base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

// (id, old slot) of every located particle i < n into a free slot of its new
// cell.  first - lane and stride must be multiples of 32 (whole warps), so
// that every lane of a warp takes part in the aggregated increments.
__device__ __forceinline__ void scatter_phase(const uint32_t* __restrict__ cell_new, const uint64_t* __restrict__ id,
                                              uint32_t* __restrict__ cursor, uint64_t* __restrict__ key_id,
                                              uint32_t* __restrict__ key_src, uint32_t C, size_t cap, uint32_t n,
                                              unsigned int* __restrict__ status, uint32_t first, uint32_t stride) {
  // four particles per thread and pass, their cells loaded before the first
  // increment (memory-level parallelism when the grid is small, as in a
  // persistent kernel)
  constexpr int U = 4;
  const uint32_t lane = threadIdx.x & 31u;
  for (size_t base = (size_t)first - lane; base < n; base += (size_t)U * stride) {
    uint32_t K[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const size_t i = base + (size_t)u * stride + lane;
      K[u] = i < n ? cell_new[i] : PIC_LOST;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t i = (uint32_t)(base + (size_t)u * stride + lane);
      if (K[u] != PIC_LOST && K[u] >= C) atomicOr(status, PIC_STATUS_BOUNDS);
      const bool take = K[u] < C;
      const uint32_t slot = aggregated_increment(cursor, K[u], take);
      if (!take) continue;
      if (slot >= cap) {
        atomicOr(status, PIC_STATUS_BOUNDS);
        continue;
      }
      key_id[slot] = id[i];
      key_src[slot] = i;
    }
  }
}

// New slot = segment start + number of smaller ids in the segment (ids are
// unique within a cell).  Warp w of nw takes G consecutive cells at a time
// (G a power of two <= 32, the largest with C / G >= nw, so that small meshes
// still spread over all warps): lane q < G holds the segment start of cell
// K0 + q, and the particles of the G segments are ranked 32 at a time, each
// lane finding its slot's cell among the G starts (a shuffle binary search)
// and counting the smaller ids of that segment.  All lanes work whatever the
// cells' sizes, where one warp per cell left most lanes idle at ~10-20
// particles per cell.
__device__ __forceinline__ void rank_phase(const uint32_t* __restrict__ cell_off, const uint64_t* __restrict__ key_id,
                                           const uint32_t* __restrict__ key_src, uint32_t* __restrict__ perm,
                                           uint32_t* __restrict__ cell_out, uint32_t C, size_t cap,
                                           unsigned int* __restrict__ status, uint32_t w, uint32_t nw) {
  const int lane = threadIdx.x & 31;
  const uint32_t per_warp = C / (nw ? nw : 1u);
  uint32_t G = 1;
  while (G < 32u && 2u * G <= per_warp) G *= 2u;
  for (uint32_t K0 = w * G; K0 < C; K0 += nw * G) {
    const int nc = (C - K0) < G ? (int)(C - K0) : (int)G;  // cells in this group
    const uint32_t start = cell_off[K0 + (uint32_t)(lane < nc ? lane : nc)];  // lanes >= nc: the group's end
    const uint32_t end_all = cell_off[K0 + (uint32_t)nc];
    const uint32_t beg_all = __shfl_sync(0xffffffffu, start, 0);
    // segment starts must be non-decreasing and inside the store
    const uint32_t prev = __shfl_up_sync(0xffffffffu, start, 1);
    const bool bad = end_all > cap || (lane > 0 && lane < nc && start < prev) || (lane == nc - 1 && end_all < start);
    if (__any_sync(0xffffffffu, bad)) {
      if (lane == 0) atomicOr(status, PIC_STATUS_BOUNDS);
      continue;
    }
    for (uint32_t j0 = beg_all; j0 < end_all; j0 += 32u) {
      const uint32_t j = j0 + lane;
      // c = the last of the nc cells whose segment starts at or before j
      int c = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const uint32_t sc = __shfl_sync(0xffffffffu, start, (c + step) & 31);
        if (c + step < nc && sc <= j) c += step;
      }
      const uint32_t beg = __shfl_sync(0xffffffffu, start, c);
      const uint32_t nxt = __shfl_sync(0xffffffffu, start, (c + 1) & 31);
      const uint32_t end = c + 1 < nc ? nxt : end_all;
      if (j < end_all) {
        const uint64_t my = key_id[j];
        uint32_t rank = 0;
#pragma unroll 4
        for (uint32_t f = beg; f < end; ++f) rank += (key_id[f] < my) ? 1u : 0u;
        perm[beg + rank] = key_src[j];
        if (cell_out) cell_out[beg + rank] = K0 + (uint32_t)c;
      }
    }
  }
}

// Copy every field from old slot perm[j] to new slot j, j < n.  Each thread
// takes four slots per pass and issues their loads before their stores
// (memory-level parallelism when the grid is small, as in a persistent
// kernel).
__device__ __forceinline__ void gather_phase(const StoreView& src, const StoreView& dst,
                                             const uint32_t* __restrict__ perm, int dim, uint32_t n,
                                             unsigned int* __restrict__ status, uint32_t first, uint32_t stride) {
  constexpr int U = 4;
  for (uint32_t j0 = first; j0 < n; j0 += U * stride) {
    uint32_t sidx[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t j = j0 + u * stride;
      sidx[u] = j < n ? perm[j] : 0u;
      ok[u] = j < n && sidx[u] < src.cap;
      if (j < n && !ok[u]) atomicOr(status, PIC_STATUS_BOUNDS);
    }
    for (int a = 0; a < dim; ++a) {
      double xv[U];
      float2 tv[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (ok[u]) {
          xv[u] = src.x[a * src.cap + sidx[u]];
          tv[u] = src.xhat[a * src.cap + sidx[u]];
        }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (ok[u]) {
          dst.x[a * dst.cap + j0 + u * stride] = xv[u];
          dst.xhat[a * dst.cap + j0 + u * stride] = tv[u];
        }
    }
    {
      uint64_t iv[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (ok[u]) iv[u] = src.id[sidx[u]];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (ok[u]) dst.id[j0 + u * stride] = iv[u];
    }
    for (int q = 0; q < src.n_props; ++q) {
      double pv[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (ok[u]) pv[u] = src.props[q * src.cap + sidx[u]];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (ok[u]) dst.props[q * dst.cap + j0 + u * stride] = pv[u];
    }
  }
}

}  // namespace pic
