// locate.cuh -- point location on the device (Sec. 2.4 of Gassmoeller et
// al., arXiv 1612.03369): the inverse map in the hint cell, then the cells
// that share a vertex with it ("vertex neighbours"), then a search over all
// cells.  Ownership of points on shared faces, edges and vertices goes to
// the lowest cell index.
#pragma once

#include "pic_internal.cuh"

namespace pic {

enum : unsigned {
  kFlagWalk = 1u,
  kFlagGlobal = 2u,
  kFlagNonConv = 4u,
  kFlagBounds = 8u,
  kFlagFallback64 = 16u,  // the FP32/double-float inverse map handed a cell to the FP64 Newton
  kFlagWalk64 = 32u       // the walk went past the predicted neighbour (FP64 walk)
};

// Newton in cell K from the start held in t; true if y is inside K.
template <int D>
__device__ __forceinline__ bool try_cell(const MeshView& m, uint32_t K, const double y[D], double t[D], int& iters,
                                         unsigned& flags, bool* converged = nullptr) {
  CellGeom<D> g;
  load_cell<D>(m, K, g);
  const bool conv = newton<D>(g, y, t, iters);
  if (converged) *converged = conv;
  if (!conv) {
    flags |= kFlagNonConv;
    return false;
  }
  return in_ref_cell<D>(t);
}

// Lowest-index rule: a point inside `found` whose reference coordinates lie
// within kTieBand of some facets may also lie (within kInsideEps) in the
// cells across those facets, edges or vertices; test those with a lower
// index and keep the lowest that holds the point.
template <int D>
__device__ __forceinline__ uint32_t lowest_owner(const MeshView& m, const double y[D], uint32_t found, double t[D],
                                                 int& iters, unsigned& flags) {
  int c[3];
  cell_ijk<D>(m, found, c);
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  bool any = false;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    lo[a] = (t[a] < kTieBand && c[a] > 0) ? -1 : 0;
    hi[a] = (t[a] > 1.0 - kTieBand && c[a] < m.n[a] - 1) ? 1 : 0;
    any = any || lo[a] != 0 || hi[a] != 0;
  }
  if (!any) return found;
  uint32_t best = found;
  double tb[D];
#pragma unroll
  for (int a = 0; a < D; ++a) tb[a] = t[a];
  for (int o2 = (D == 3 ? lo[2] : 0); o2 <= (D == 3 ? hi[2] : 0); ++o2)
    for (int o1 = lo[1]; o1 <= hi[1]; ++o1)
      for (int o0 = lo[0]; o0 <= hi[0]; ++o0) {
        if (o0 == 0 && o1 == 0 && o2 == 0) continue;
        const uint32_t K = cell_index<D>(m, c[0] + o0, c[1] + o1, c[2] + o2);
        if (K >= best) continue;
        double tt[D];
        const int o[3] = {o0, o1, o2};
#pragma unroll
        for (int a = 0; a < D; ++a) tt[a] = t[a] - (double)o[a];
        if (try_cell<D>(m, K, y, tt, iters, flags)) {
          best = K;
#pragma unroll
          for (int a = 0; a < D; ++a) tb[a] = tt[a];
        }
      }
#pragma unroll
  for (int a = 0; a < D; ++a) t[a] = tb[a];
  return best;
}

// All-cells search (the last resort of Sec. 2.4, every cell tried), entered
// only when no vertex neighbour holds the point.  The cells around the point's
// position in a uniform background grid are tried first; a hit there is then
// settled by the lowest-index rule, which covers every other cell that can
// hold the point.  Otherwise every cell is visited in index order and the
// first that holds the point is the lowest owner.
template <int D>
__device__ uint32_t global_search(const MeshView& m, const double y[D], double t[D], int& iters, unsigned& flags) {
  flags |= kFlagGlobal;
#pragma unroll
  for (int a = 0; a < D; ++a)
    if (!(y[a] >= m.dlo[a] && y[a] <= m.dhi[a])) return PIC_LOST;
  int g[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    double f = (y[a] - m.dlo[a]) / (m.dhi[a] - m.dlo[a]) * (double)m.n[a];
    int gi = (int)floor(f);
    g[a] = gi < 0 ? 0 : (gi > m.n[a] - 1 ? m.n[a] - 1 : gi);
  }
  for (int o2 = (D == 3 ? -1 : 0); o2 <= (D == 3 ? 1 : 0); ++o2)
    for (int o1 = -1; o1 <= 1; ++o1)
      for (int o0 = -1; o0 <= 1; ++o0) {
        const int i = g[0] + o0, j = g[1] + o1, k = g[2] + o2;
        if (i < 0 || j < 0 || i >= m.n[0] || j >= m.n[1]) continue;
        if (D == 3 && (k < 0 || k >= m.n[2])) continue;
        const uint32_t K = cell_index<D>(m, i, j, k);
        double tt[D];
#pragma unroll
        for (int a = 0; a < D; ++a) tt[a] = 0.5;
        if (try_cell<D>(m, K, y, tt, iters, flags)) {
#pragma unroll
          for (int a = 0; a < D; ++a) t[a] = tt[a];
          return lowest_owner<D>(m, y, K, t, iters, flags);
        }
      }
  for (uint32_t K = 0; K < m.C; ++K) {
    const double* bb = m.bbox + 6 * (size_t)K;
    bool in = true;
#pragma unroll
    for (int a = 0; a < D; ++a) in = in && y[a] >= __ldg(bb + a) && y[a] <= __ldg(bb + 3 + a);
    if (!in) continue;
    double tt[D];
#pragma unroll
    for (int a = 0; a < D; ++a) tt[a] = 0.5;
    if (try_cell<D>(m, K, y, tt, iters, flags)) {
#pragma unroll
      for (int a = 0; a < D; ++a) t[a] = tt[a];
      return K;
    }
  }
  return PIC_LOST;
}

// Owner of y (lowest index) and its reference coordinates t.  hint_t is the
// Newton start in the hint cell.  Returns PIC_LOST if no cell holds y.
template <int D>
__device__ uint32_t locate(const MeshView& m, const double y[D], uint32_t hintK, const double hint_t[D], double t[D],
                           int& iters, unsigned& flags) {
#pragma unroll
  for (int a = 0; a < D; ++a) t[a] = hint_t[a];
  if (hintK >= m.C) {
    flags |= kFlagBounds;
    return global_search<D>(m, y, t, iters, flags);
  }
  // A point outside the padded bounding box of the whole mesh (padding 1e-9
  // of its extent) is in no cell: a cell accepts only points within about
  // 1e-10 of its own size of it.  Testing the box first spares such points
  // the walk over every neighbour of the hint (the paper's remark on testing
  // the subdomain's bounding box before its cells, Sec. 2.2).
#pragma unroll
  for (int a = 0; a < D; ++a)
    if (!(y[a] >= m.dlo[a] && y[a] <= m.dhi[a])) return PIC_LOST;
  bool conv = false;
  if (try_cell<D>(m, hintK, y, t, iters, flags, &conv)) return lowest_owner<D>(m, y, hintK, t, iters, flags);

  // Vertex-neighbour walk.  The Newton iterate in the hint cell, when it
  // converged, already points at the neighbour across the violated facets;
  // that cell is tried first.  The remaining vertex neighbours K' follow in
  // the order of the paper's heuristic: v = vertex of K closest to y,
  // a = y - v, b = c_K' - v, descending a.b.
  flags |= kFlagWalk;
  int c[3];
  cell_ijk<D>(m, hintK, c);
  int pred[3] = {0, 0, 0};
  bool have_pred = false;
  if (conv) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      pred[a] = t[a] < 0.0 ? -1 : (t[a] > 1.0 ? 1 : 0);
      if (c[a] + pred[a] < 0 || c[a] + pred[a] >= m.n[a]) pred[a] = 0;
      have_pred = have_pred || pred[a] != 0;
    }
  }
  double tconv[D];
#pragma unroll
  for (int a = 0; a < D; ++a) tconv[a] = t[a];
  if (have_pred) {
    const uint32_t K = cell_index<D>(m, c[0] + pred[0], c[1] + pred[1], c[2] + pred[2]);
    double tt[D];
#pragma unroll
    for (int a = 0; a < D; ++a) tt[a] = tconv[a] - (double)pred[a];
    if (try_cell<D>(m, K, y, tt, iters, flags)) {
#pragma unroll
      for (int a = 0; a < D; ++a) t[a] = tt[a];
      return lowest_owner<D>(m, y, K, t, iters, flags);
    }
  }
  // remaining neighbours in descending a.b
  CellGeom<D> g;
  load_cell<D>(m, hintK, g);
  double v[D], best_d2 = 1e300;
  for (int q = 0; q < (1 << D); ++q) {
    double d2 = 0.0, p[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      p[a] = g.x0[a] + g.e[q][a];
      d2 += (y[a] - p[a]) * (y[a] - p[a]);
    }
    if (d2 < best_d2) {
      best_d2 = d2;
#pragma unroll
      for (int a = 0; a < D; ++a) v[a] = p[a];
    }
  }
  constexpr int NN = (D == 3 ? 27 : 9);
  double score[NN];
  int nbr_ok = 0;  // bit mask of candidates still to test
  for (int q = 0; q < NN; ++q) {
    const int o0 = q % 3 - 1, o1 = (q / 3) % 3 - 1, o2 = (D == 3 ? q / 9 - 1 : 0);
    score[q] = 0.0;
    if (o0 == 0 && o1 == 0 && o2 == 0) continue;
    if (o0 == pred[0] && o1 == pred[1] && o2 == pred[2] && have_pred) continue;
    const int i = c[0] + o0, j = c[1] + o1, k = c[2] + o2;
    if (i < 0 || j < 0 || i >= m.n[0] || j >= m.n[1]) continue;
    if (D == 3 && (k < 0 || k >= m.n[2])) continue;
    const uint32_t K = cell_index<D>(m, i, j, k);
    CellGeom<D> gk;
    load_cell<D>(m, K, gk);
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double ctr = gk.x0[a];
      for (int w = 0; w < (1 << D); ++w) ctr += gk.e[w][a] / (double)(1 << D);
      s += (y[a] - v[a]) * (ctr - v[a]);
    }
    score[q] = s;
    nbr_ok |= 1 << q;
  }
  while (nbr_ok) {
    int qb = __ffs(nbr_ok) - 1;  // a valid candidate even if every score is NaN
    double sb = score[qb];
    for (int q = qb + 1; q < NN; ++q)
      if (((nbr_ok >> q) & 1) && score[q] > sb) {
        sb = score[q];
        qb = q;
      }
    nbr_ok &= ~(1 << qb);
    const int o0 = qb % 3 - 1, o1 = (qb / 3) % 3 - 1, o2 = (D == 3 ? qb / 9 - 1 : 0);
    const uint32_t K = cell_index<D>(m, c[0] + o0, c[1] + o1, c[2] + o2);
    double tt[D];
    const int o[3] = {o0, o1, o2};
#pragma unroll
    for (int a = 0; a < D; ++a) tt[a] = conv ? tconv[a] - (double)o[a] : 0.5;
    if (try_cell<D>(m, K, y, tt, iters, flags)) {
#pragma unroll
      for (int a = 0; a < D; ++a) t[a] = tt[a];
      return lowest_owner<D>(m, y, K, t, iters, flags);
    }
  }
  return global_search<D>(m, y, t, iters, flags);
}

}  // namespace pic
