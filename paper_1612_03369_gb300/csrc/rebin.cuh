// rebin.cuh -- the phases of the rebin (Sec. 2.1 store sorted by cell,
// Sec. 2.4 batched re-insertion) as device functions over a "virtual grid"
// (block index bid of nb blocks), so that the stand-alone kernels of
// rebin.cu and the persistent ensemble kernel run the same code.
//
//   scan   exclusive prefix sum of per-cell counts: each block of the grid
//          sums a contiguous chunk, then offsets its chunk by the sums of
//          the chunks before it (the stand-alone rebin uses the single-pass
//          kernel of rebin.cu instead)
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

// The exclusive scan of a co-resident grid (the persistent ensemble kernel),
// in two phases with a grid barrier between them.  Block bid of nb owns the
// contiguous chunk [bid n / nb, (bid + 1) n / nb) of the n values.
__device__ __forceinline__ void scan_chunk(uint32_t n, uint32_t bid, uint32_t nb, uint32_t& lo, uint32_t& hi) {
  lo = (uint32_t)((uint64_t)bid * n / nb);
  hi = (uint32_t)((uint64_t)(bid + 1) * n / nb);
}

// Phase 1: sums[bid] = the sum of block bid's chunk.
__device__ __forceinline__ void scan_phase_chunk_sums(const uint32_t* __restrict__ in, uint32_t n,
                                                      uint32_t* __restrict__ sums, uint32_t bid, uint32_t nb) {
  __shared__ uint32_t tot;
  uint32_t lo, hi, s = 0;
  scan_chunk(n, bid, nb, lo, hi);
  for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += in[i];
  (void)block_excl_scan(s, &tot);
  if (threadIdx.x == 0) sums[bid] = tot;
  __syncthreads();
}

// Phase 2: block bid adds up sums[0..bid) and writes the exclusive prefix of
// its chunk to out (and cursor when given), kScanItems consecutive values
// per thread and pass; the last block writes the total to out[n] and
// *total_dev.
__device__ __forceinline__ void scan_phase_chunk_apply(const uint32_t* __restrict__ in, uint32_t n,
                                                       const uint32_t* __restrict__ sums, uint32_t* __restrict__ out,
                                                       uint32_t* __restrict__ cursor, uint32_t* __restrict__ total_dev,
                                                       uint32_t bid, uint32_t nb) {
  __shared__ uint32_t tot;
  uint32_t lo, hi, before = 0;
  scan_chunk(n, bid, nb, lo, hi);
  for (uint32_t k = threadIdx.x; k < bid; k += blockDim.x) before += sums[k];
  (void)block_excl_scan(before, &tot);
  uint32_t carry = tot;
  const uint32_t T = blockDim.x * kScanItems;
  for (uint32_t base0 = lo; base0 < hi; base0 += T) {
    const uint32_t base = base0 + threadIdx.x * kScanItems;
    uint32_t v[kScanItems], s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
      v[q] = (base + q < hi) ? in[base + q] : 0u;
      s += v[q];
    }
    uint32_t ex = carry + block_excl_scan(s, &tot);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
      if (base + q < hi) {
        out[base + q] = ex;
        if (cursor) cursor[base + q] = ex;
      }
      ex += v[q];
    }
    carry += tot;
    __syncthreads();  // tot is rewritten by the next pass
  }
  if (bid + 1 == nb && threadIdx.x == 0) {
    out[n] = carry;
    if (total_dev) *total_dev = carry;
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
// that every lane of a warp takes part in the aggregated increments.  Each
// thread takes U particles per pass and issues their loads, then the U
// warp-aggregated atomics, before it waits on any of them (memory-level
// parallelism when the grid is small, as in a persistent kernel).
__device__ __forceinline__ void scatter_phase(const uint32_t* __restrict__ cell_new, const uint64_t* __restrict__ id,
                                              uint32_t* __restrict__ cursor, uint64_t* __restrict__ key_id,
                                              uint32_t* __restrict__ key_src, uint32_t C, size_t cap, uint32_t n,
                                              unsigned int* __restrict__ status, uint32_t first, uint32_t stride) {
  constexpr int U = 4;
  const uint32_t lane = threadIdx.x & 31u;
  const unsigned below = (1u << lane) - 1u;
  for (size_t base = (size_t)first - lane; base < n; base += (size_t)U * stride) {
    uint32_t K[U];
    uint64_t iv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const size_t i = base + (size_t)u * stride + lane;
      K[u] = i < n ? cell_new[i] : PIC_LOST;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const size_t i = base + (size_t)u * stride + lane;
      iv[u] = K[u] < C ? id[i] : 0ull;
    }
    unsigned peers[U];
    uint32_t old[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (K[u] != PIC_LOST && K[u] >= C) atomicOr(status, PIC_STATUS_BOUNDS);
      const bool take = K[u] < C;
      peers[u] = __match_any_sync(0xffffffffu, take ? K[u] : 0xFFFFFFFFu);
      old[u] = 0;
      if (take && (int)lane == __ffs(peers[u]) - 1) old[u] = atomicAdd(cursor + K[u], (uint32_t)__popc(peers[u]));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t slot = __shfl_sync(0xffffffffu, old[u], __ffs(peers[u]) - 1) + (uint32_t)__popc(peers[u] & below);
      if (K[u] >= C) continue;
      if (slot >= cap) {
        atomicOr(status, PIC_STATUS_BOUNDS);
        continue;
      }
      key_id[slot] = iv[u];
      key_src[slot] = (uint32_t)(base + (size_t)u * stride + lane);
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
  // the segment starts of group K0 (lanes >= nc: the group's end); the next
  // group's are loaded while this one is ranked
  auto starts = [&](uint32_t K0, int& nc, uint32_t& st, uint32_t& end_all) {
    nc = K0 < C ? ((C - K0) < G ? (int)(C - K0) : (int)G) : 0;
    st = K0 < C ? cell_off[K0 + (uint32_t)(lane < nc ? lane : nc)] : 0u;
    end_all = K0 < C ? cell_off[K0 + (uint32_t)nc] : 0u;
  };
  int nc_n;
  uint32_t st_n, end_n;
  starts(w * G, nc_n, st_n, end_n);
  for (uint32_t K0 = w * G; K0 < C; K0 += nw * G) {
    const int nc = nc_n;  // cells in this group
    const uint32_t start = st_n, end_all = end_n;
    starts(K0 + nw * G, nc_n, st_n, end_n);
    const uint32_t beg_all = __shfl_sync(0xffffffffu, start, 0);
    // segment starts must be non-decreasing and inside the store
    const uint32_t prev = __shfl_up_sync(0xffffffffu, start, 1);
    const bool bad = end_all > cap || (lane > 0 && lane < nc && start < prev) || (lane == nc - 1 && end_all < start);
    if (__any_sync(0xffffffffu, bad)) {
      if (lane == 0) atomicOr(status, PIC_STATUS_BOUNDS);
      continue;
    }
    // each chunk's key and source are loaded one chunk ahead
    uint64_t my_n = 0;
    uint32_t src_n = 0;
    if (beg_all + lane < end_all) {
      my_n = key_id[beg_all + lane];
      src_n = key_src[beg_all + lane];
    }
    for (uint32_t j0 = beg_all; j0 < end_all; j0 += 32u) {
      const uint32_t j = j0 + lane;
      const uint64_t my = my_n;
      const uint32_t src = src_n;
      if (j + 32u < end_all) {
        my_n = key_id[j + 32u];
        src_n = key_src[j + 32u];
      }
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
        uint32_t rank = 0;
#pragma unroll 4
        for (uint32_t f = beg; f < end; ++f) rank += (key_id[f] < my) ? 1u : 0u;
        perm[beg + rank] = src;
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
