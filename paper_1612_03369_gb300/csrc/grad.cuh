// grad.cuh -- the velocity gradient du_h/dx at a located point in FP64
// (chain rule through the inverse map, the cell held fixed): used by the
// adjoint sweep and by the particle property ODEs of Sec. 2.6.
#pragma once

#include "pic_internal.cuh"

namespace pic {

// u and du/dt at reference coordinates t of cell K (FP64, sum factorisation):
// Gu[c][j] = d u_c / d t_j.
template <int D>
__device__ __forceinline__ void q2_value_grad(const MeshView& m, uint32_t K, const double t[D], double u[D],
                                              double Gu[D][D]) {
  int c[3];
  cell_ijk<D>(m, K, c);
  const int64_t sy = m.nq[0], sz = (int64_t)m.nq[0] * m.nq[1];
  const int64_t base = 2 * (int64_t)c[0] + sy * 2 * c[1] + (D == 3 ? sz * 2 * c[2] : 0);
  double l[D][3], dl[D][3];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    lagrange2<double>(t[a], l[a]);
    dl[a][0] = 4.0 * t[a] - 3.0;
    dl[a][1] = 4.0 - 8.0 * t[a];
    dl[a][2] = 4.0 * t[a] - 1.0;
  }
#pragma unroll
  for (int comp = 0; comp < D; ++comp) {
    const double* Uc = m.U + comp * m.nnodes + base;
    double v = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
#pragma unroll
    for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz) {
      double sv = 0.0, s0 = 0.0, s1 = 0.0;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const double* row = Uc + b * sy + (D == 3 ? cz * sz : 0);
        const double r0 = __ldg(row), r1 = __ldg(row + 1), r2 = __ldg(row + 2);
        const double rv = l[0][0] * r0 + l[0][1] * r1 + l[0][2] * r2;
        const double rd = dl[0][0] * r0 + dl[0][1] * r1 + dl[0][2] * r2;
        sv += l[1][b] * rv;
        s0 += l[1][b] * rd;
        s1 += dl[1][b] * rv;
      }
      if constexpr (D == 3) {
        v += l[2][cz] * sv;
        g0 += l[2][cz] * s0;
        g1 += l[2][cz] * s1;
        g2 += dl[2][cz] * sv;
      } else {
        v = sv;
        g0 = s0;
        g1 = s1;
      }
    }
    u[comp] = v;
    Gu[comp][0] = g0;
    Gu[comp][1] = g1;
    if constexpr (D == 3) Gu[comp][2] = g2;
  }
}

template <int D>
__device__ __forceinline__ void invert(const double J[D][D], double Ji[D][D]) {
  if constexpr (D == 2) {
    const double inv = 1.0 / (J[0][0] * J[1][1] - J[0][1] * J[1][0]);
    Ji[0][0] = J[1][1] * inv;
    Ji[0][1] = -J[0][1] * inv;
    Ji[1][0] = -J[1][0] * inv;
    Ji[1][1] = J[0][0] * inv;
  } else {
    double c[3][3];
    c[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    c[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    c[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    c[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    c[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    c[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    c[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    c[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    c[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double inv = 1.0 / (J[0][0] * c[0][0] + J[0][1] * c[0][1] + J[0][2] * c[0][2]);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = 0; q < 3; ++q) Ji[r][q] = c[q][r] * inv;
  }
}

// G = du_h/dx = (du/dt) J^{-1} at reference coordinates t of cell K.
template <int D>
__device__ __forceinline__ void velocity_gradient(const MeshView& m, uint32_t K, const double t[D], double G[D][D]) {
  double u[D], Gu[D][D], phi[D], J[D][D], Ji[D][D];
  q2_value_grad<D>(m, K, t, u, Gu);
  CellGeom<D> g;
  load_cell<D>(m, K, g);
  map_and_jacobian<D>(g, t, phi, J);
  invert<D>(J, Ji);
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int q = 0; q < D; ++q) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < D; ++j) acc += Gu[c][j] * Ji[j][q];
      G[c][q] = acc;
    }
}

}  // namespace pic
