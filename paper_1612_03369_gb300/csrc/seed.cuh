// seed.cuh -- particle generation from local coordinates (Sec. 2.2, Remark
// on local generation), shared by the single-mesh store and the ensemble.
#pragma once

#include "pic_internal.cuh"

namespace pic {

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used as a counter-based
// generator: output n of the stream seeded with `seed` is the finaliser
// applied to seed + (n + 1) * 0x9E3779B97F4A7C15.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static __global__ void fill_counts_kernel(const uint32_t* __restrict__ per_cell, uint32_t uniform, uint32_t* __restrict__ counts,
                                   uint32_t C) {
  for (uint32_t K = blockIdx.x * blockDim.x + threadIdx.x; K < C; K += gridDim.x * blockDim.x)
    counts[K] = per_cell ? per_cell[K] : uniform;
}

// The remark on generating in local coordinates (Sec. 2.2): loop over cells
// in order and over local coordinates inside each; only the forward map
// Phi_K is needed.
//
// The mesh's cells occupy store cells cell_base .. cell_base + C - 1 (an
// ensemble packs several meshes into one store); ordinals, ids and random
// numbers count from the mesh's first particle.
template <int D>
__global__ void seed_kernel(MeshView m, StoreView s, const uint32_t* __restrict__ cell_off, uint64_t seed,
                            uint64_t first_id, uint32_t cell_base) {
  const uint32_t q0 = cell_off[cell_base];
  for (uint32_t K = blockIdx.x * blockDim.x + threadIdx.x; K < m.C; K += gridDim.x * blockDim.x) {
    const uint32_t beg = cell_off[cell_base + K], end = cell_off[cell_base + K + 1];
    if (end > s.cap) continue;
    CellGeom<D> g;
    load_cell<D>(m, K, g);
    for (uint32_t q = beg; q < end; ++q) {
      double t[D], x[D];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const uint64_t r = splitmix64_at(seed, (uint64_t)(q - q0) * D + j);
        t[j] = (double)(r >> 11) * 0x1.0p-53;
      }
      map_point<D>(g, t, x);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        s.x[j * s.cap + q] = x[j];
        const float hi = __double2float_rn(t[j]);
        s.xhat[j * s.cap + q] = make_float2(hi, __double2float_rn(t[j] - (double)hi));
      }
      s.id[q] = first_id + (q - q0);
      s.cell[q] = cell_base + K;
      for (int p = 0; p < s.n_props; ++p) s.props[p * s.cap + q] = 0.0;
    }
  }
}

}  // namespace pic
