/*
 * pic_oracle.c -- plain, slow, obviously-correct CPU oracle for the particle
 * hot path of Gassmoeller, Heien, Puckett & Bangerth, "Flexible and scalable
 * particle-in-cell methods for massively parallel computations" (arXiv
 * 1612.03369).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or helper with the
 * CUDA library; the two meet only through the seeded input generators.
 *
 * Everything is IEEE binary64, compiled with -ffp-contract=off, with no
 * blocking, fusion or reordering: each function follows the paper's
 * statement of the step it computes, and its comment names the section or
 * equation.  Where the paper is silent or its printed formulas are garbled,
 * the reading taken is named R1..R16 (the list of readings is kept with the
 * design notes of the repository).
 *
 * Layouts (chosen for the oracle alone):
 *   vertices X[dim][nverts], vertex (i,j,k) at i + (nx+1)*(j + (ny+1)*k)
 *   Q2 nodal values U[dim][nnodes], node (I,J,K) at I + (2nx+1)*(J + (2ny+1)*K)
 *   cell (i,j,k) at i + nx*(j + ny*k)
 *   particles: array of structs, one struct per particle (Sec. 2.1 listing)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NEWTON_TOL 1e-14   /* R2: stop when max|delta| <= 1e-14          */
#define ORC_NEWTON_MAXIT 30    /* R2: or after 30 iterations (= not inside)  */
#define ORC_INSIDE_EPS 1e-10   /* R3: x-hat in [-eps, 1+eps]^d means inside  */

typedef struct {
  int dim;
  int64_t n[3];   /* cells per axis; n[2] = 1 in 2D */
  int64_t nv[3];  /* vertices per axis */
  int64_t nq[3];  /* Q2 nodes per axis */
  int64_t ncells, nverts, nnodes;
  double *X; /* [dim][nverts] */
  double *U; /* [dim][nnodes], NULL until set */
  double *Unext; /* [dim][nnodes] velocity at the end of the step, or NULL (steady) */
  /* exact bounding-box filter for the owner search: a cell can only contain
   * x if its (padded) bounding box contains x, so testing only those cells is
   * the brute-force search of Sec. 2.2 (prescribed positions) with a filter
   * that cannot drop a true owner. */
  double *bb_lo, *bb_hi; /* [ncells][3] */
  double org[3], bs[3];
  int64_t nb[3];
  int64_t *bin_start; /* [nbins+1] */
  int64_t *bin_cells;
} orc_mesh;

typedef struct {
  uint64_t id;
  int64_t cell; /* owner cell, -1 = lost */
  double x[3];
  double xhat[3];
  double *props;
} orc_particle;

/* ---------------------------------------------------------------- mesh --- */

static int64_t cell_index(const orc_mesh *m, int64_t i, int64_t j, int64_t k) {
  return i + m->n[0] * (j + m->n[1] * k);
}

static void cell_ijk(const orc_mesh *m, int64_t c, int64_t *i, int64_t *j, int64_t *k) {
  *i = c % m->n[0];
  *j = (c / m->n[0]) % m->n[1];
  *k = c / (m->n[0] * m->n[1]);
}

/* Vertex v (v = a + 2b + 4c, lexicographic) of cell K, coordinate comp. */
static double cell_vertex(const orc_mesh *m, int64_t K, int v, int comp) {
  int64_t i, j, k;
  cell_ijk(m, K, &i, &j, &k);
  int64_t a = v & 1, b = (v >> 1) & 1, c = (v >> 2) & 1;
  int64_t gv = (i + a) + m->nv[0] * ((j + b) + m->nv[1] * (k + c));
  return m->X[(int64_t)comp * m->nverts + gv];
}

static void build_bins(orc_mesh *m);

orc_mesh *orc_mesh_create(int dim, const int64_t *n, const double *X) {
  orc_mesh *m = (orc_mesh *)calloc(1, sizeof(orc_mesh));
  m->dim = dim;
  for (int a = 0; a < 3; ++a) {
    m->n[a] = a < dim ? n[a] : 1;
    m->nv[a] = a < dim ? n[a] + 1 : 1;
    m->nq[a] = a < dim ? 2 * n[a] + 1 : 1;
  }
  m->ncells = m->n[0] * m->n[1] * m->n[2];
  m->nverts = m->nv[0] * m->nv[1] * m->nv[2];
  m->nnodes = m->nq[0] * m->nq[1] * m->nq[2];
  m->X = (double *)malloc(sizeof(double) * dim * m->nverts);
  memcpy(m->X, X, sizeof(double) * dim * m->nverts);
  build_bins(m);
  return m;
}

void orc_mesh_set_velocity(orc_mesh *m, const double *U) {
  if (!m->U) m->U = (double *)malloc(sizeof(double) * m->dim * m->nnodes);
  memcpy(m->U, U, sizeof(double) * m->dim * m->nnodes);
}

/* Velocity at the end of every time step (Sec. 2.3, eq. position-ode-approx:
 * u-tilde_h interpolates u_h^n and u_h^{n+1} in time); NULL = steady field. */
void orc_mesh_set_velocity_next(orc_mesh *m, const double *Un) {
  free(m->Unext);
  m->Unext = NULL;
  if (!Un) return;
  m->Unext = (double *)malloc(sizeof(double) * m->dim * m->nnodes);
  memcpy(m->Unext, Un, sizeof(double) * m->dim * m->nnodes);
}

void orc_mesh_destroy(orc_mesh *m) {
  if (!m) return;
  free(m->X);
  free(m->U);
  free(m->Unext);
  free(m->bb_lo);
  free(m->bb_hi);
  free(m->bin_start);
  free(m->bin_cells);
  free(m);
}

int64_t orc_mesh_ncells(const orc_mesh *m) { return m->ncells; }

static int64_t clampi(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

static void build_bins(orc_mesh *m) {
  int d = m->dim, nvc = 1 << d;
  m->bb_lo = (double *)malloc(sizeof(double) * 3 * m->ncells);
  m->bb_hi = (double *)malloc(sizeof(double) * 3 * m->ncells);
  double glo[3] = {0, 0, 0}, ghi[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) {
    glo[a] = INFINITY;
    ghi[a] = -INFINITY;
  }
  for (int64_t K = 0; K < m->ncells; ++K) {
    for (int a = 0; a < d; ++a) {
      double lo = INFINITY, hi = -INFINITY;
      for (int v = 0; v < nvc; ++v) {
        double xv = cell_vertex(m, K, v, a);
        if (xv < lo) lo = xv;
        if (xv > hi) hi = xv;
      }
      /* pad by 1e-6 of the cell's extent: far wider than the eps band of R3 */
      double pad = 1e-6 * (hi - lo);
      m->bb_lo[3 * K + a] = lo - pad;
      m->bb_hi[3 * K + a] = hi + pad;
      if (lo - pad < glo[a]) glo[a] = lo - pad;
      if (hi + pad > ghi[a]) ghi[a] = hi + pad;
    }
  }
  int64_t nbins = 1;
  for (int a = 0; a < 3; ++a) {
    if (a < d) {
      m->nb[a] = m->n[a];
      m->org[a] = glo[a];
      m->bs[a] = (ghi[a] - glo[a]) / (double)m->nb[a];
    } else {
      m->nb[a] = 1;
      m->org[a] = 0;
      m->bs[a] = 1;
    }
    nbins *= m->nb[a];
  }
  /* two passes: count, then fill (CSR) */
  m->bin_start = (int64_t *)calloc(nbins + 1, sizeof(int64_t));
  for (int pass = 0; pass < 2; ++pass) {
    int64_t *fill = NULL;
    if (pass == 1) {
      for (int64_t b = 0; b < nbins; ++b) m->bin_start[b + 1] += m->bin_start[b];
      m->bin_cells = (int64_t *)malloc(sizeof(int64_t) * (m->bin_start[nbins] + 1));
      fill = (int64_t *)calloc(nbins, sizeof(int64_t));
    }
    for (int64_t K = 0; K < m->ncells; ++K) {
      int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) {
        lo[a] = clampi((int64_t)floor((m->bb_lo[3 * K + a] - m->org[a]) / m->bs[a]), 0, m->nb[a] - 1);
        hi[a] = clampi((int64_t)floor((m->bb_hi[3 * K + a] - m->org[a]) / m->bs[a]), 0, m->nb[a] - 1);
      }
      for (int64_t bk = lo[2]; bk <= hi[2]; ++bk)
        for (int64_t bj = lo[1]; bj <= hi[1]; ++bj)
          for (int64_t bi = lo[0]; bi <= hi[0]; ++bi) {
            int64_t b = bi + m->nb[0] * (bj + m->nb[1] * bk);
            if (pass == 0)
              m->bin_start[b + 1]++;
            else
              m->bin_cells[m->bin_start[b] + fill[b]++] = K;
          }
    }
    free(fill);
  }
}

/* ------------------------------------------- mapping Phi_K (Remark 2.1) --- */

/* Multilinear weight of local vertex v at x-hat: prod_j (bit_j ? t_j : 1-t_j) */
static double vertex_weight(int dim, int v, const double *t) {
  double w = 1.0;
  for (int j = 0; j < dim; ++j) w = w * (((v >> j) & 1) ? t[j] : 1.0 - t[j]);
  return w;
}

/* d w_v / d t_jd */
static double vertex_weight_deriv(int dim, int v, const double *t, int jd) {
  double w = 1.0;
  for (int j = 0; j < dim; ++j) {
    if (j == jd)
      w = w * (((v >> j) & 1) ? 1.0 : -1.0);
    else
      w = w * (((v >> j) & 1) ? t[j] : 1.0 - t[j]);
  }
  return w;
}

/* x = Phi_K(x-hat) = sum_v X_{K,v} w_v(x-hat), the (bi/tri)linear map. */
void orc_phi(const orc_mesh *m, int64_t K, const double *xhat, double *x) {
  int d = m->dim;
  for (int i = 0; i < d; ++i) {
    double s = 0.0;
    for (int v = 0; v < (1 << d); ++v) s = s + cell_vertex(m, K, v, i) * vertex_weight(d, v, xhat);
    x[i] = s;
  }
}

/* Phi_K(x-hat) - X_{K,0} written with vertex offsets (same map; keeps the
 * Newton residual free of the cancellation of two O(1) coordinates). */
static void phi_local(const orc_mesh *m, int64_t K, const double *xhat, double *y) {
  int d = m->dim;
  for (int i = 0; i < d; ++i) {
    double x0 = cell_vertex(m, K, 0, i), s = 0.0;
    for (int v = 1; v < (1 << d); ++v) s = s + (cell_vertex(m, K, v, i) - x0) * vertex_weight(d, v, xhat);
    y[i] = s;
  }
}

/* J_ij = d Phi_i / d xhat_j */
static void phi_jacobian(const orc_mesh *m, int64_t K, const double *xhat, double J[3][3]) {
  int d = m->dim;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int v = 0; v < (1 << d); ++v) s = s + cell_vertex(m, K, v, i) * vertex_weight_deriv(d, v, xhat, j);
      J[i][j] = s;
    }
}

/* Solve J delta = r by Cramer's rule. Returns 0 if J is singular. */
static int solve_cramer(int d, double J[3][3], const double *r, double *delta) {
  if (d == 2) {
    double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    if (det == 0.0 || !isfinite(det)) return 0;
    delta[0] = (r[0] * J[1][1] - J[0][1] * r[1]) / det;
    delta[1] = (J[0][0] * r[1] - r[0] * J[1][0]) / det;
    return 1;
  }
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  if (det == 0.0 || !isfinite(det)) return 0;
  for (int c = 0; c < 3; ++c) {
    double A[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) A[i][j] = (j == c) ? r[i] : J[i][j];
    double dc = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    delta[c] = dc / det;
  }
  return 1;
}

/* x-hat = Phi_K^{-1}(x) by Newton's method (the iterative inversion that
 * Sec. 2.2 and Remark 2.1 call for; reading R2 for start, tolerance and
 * iteration cap).
 * Returns 1 if converged; *iters receives the iteration count. */
int orc_newton(const orc_mesh *m, int64_t K, const double *x, const double *start, double *xhat, int *iters) {
  int d = m->dim;
  double t[3] = {0, 0, 0}, rhs[3] = {0, 0, 0};
  for (int j = 0; j < d; ++j) {
    t[j] = start[j];
    rhs[j] = x[j] - cell_vertex(m, K, 0, j);
  }
  int conv = 0, it = 0;
  for (it = 1; it <= ORC_NEWTON_MAXIT; ++it) {
    double y[3], r[3], J[3][3], delta[3];
    phi_local(m, K, t, y);
    for (int j = 0; j < d; ++j) r[j] = rhs[j] - y[j];
    phi_jacobian(m, K, t, J);
    if (!solve_cramer(d, J, r, delta)) break;
    double dmax = 0.0;
    for (int j = 0; j < d; ++j) {
      t[j] = t[j] + delta[j];
      if (fabs(delta[j]) > dmax) dmax = fabs(delta[j]);
    }
    if (!isfinite(dmax)) break;
    if (dmax <= ORC_NEWTON_TOL) {
      conv = 1;
      break;
    }
  }
  for (int j = 0; j < d; ++j) xhat[j] = t[j];
  if (iters) *iters = it > ORC_NEWTON_MAXIT ? ORC_NEWTON_MAXIT : it;
  return conv;
}

/* inside(K, x): Newton from the cell centre converges and x-hat lies in the
 * closed reference cell widened by eps (R2, R3; Sec. 2.4 "testing whether
 * x-hat is in K-hat"). */
int orc_inside(const orc_mesh *m, int64_t K, const double *x, double *xhat) {
  double start[3] = {0.5, 0.5, 0.5}, t[3] = {0, 0, 0};
  int conv = orc_newton(m, K, x, start, t, NULL);
  if (xhat)
    for (int j = 0; j < m->dim; ++j) xhat[j] = t[j];
  if (!conv) return 0;
  for (int j = 0; j < m->dim; ++j)
    if (!(t[j] >= -ORC_INSIDE_EPS && t[j] <= 1.0 + ORC_INSIDE_EPS)) return 0;
  return 1;
}

/* owner(x) = min { K : inside(K, x) } over ALL cells, no filter at all
 * (Sec. 2.2, generation at prescribed positions: search all cells; R4 fixes
 * the lowest index on shared faces).  -1 if no cell contains x (lost). */
int64_t orc_owner_brute(const orc_mesh *m, const double *x, double *xhat) {
  for (int64_t K = 0; K < m->ncells; ++K) {
    double t[3];
    if (orc_inside(m, K, x, t)) {
      if (xhat)
        for (int j = 0; j < m->dim; ++j) xhat[j] = t[j];
      return K;
    }
  }
  return -1;
}

/* The same minimum, visiting only cells whose padded bounding box holds x
 * (a necessary condition for inside, so the minimum is unchanged). */
int64_t orc_owner(const orc_mesh *m, const double *x, double *xhat) {
  int d = m->dim;
  int64_t bi[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) {
    if (!isfinite(x[a])) return -1;
    double f = floor((x[a] - m->org[a]) / m->bs[a]);
    if (f < 0 || f >= (double)m->nb[a]) {
      /* the padded global box can still hold x on its upper face */
      if (!(x[a] >= m->org[a] && x[a] <= m->org[a] + m->bs[a] * (double)m->nb[a])) return -1;
    }
    bi[a] = clampi((int64_t)f, 0, m->nb[a] - 1);
  }
  int64_t b = bi[0] + m->nb[0] * (bi[1] + m->nb[1] * bi[2]);
  int64_t best = -1;
  double tb[3] = {0, 0, 0};
  for (int64_t q = m->bin_start[b]; q < m->bin_start[b + 1]; ++q) {
    int64_t K = m->bin_cells[q];
    if (best >= 0 && K > best) continue;
    int inbox = 1;
    for (int a = 0; a < d; ++a)
      if (!(x[a] >= m->bb_lo[3 * K + a] && x[a] <= m->bb_hi[3 * K + a])) inbox = 0;
    if (!inbox) continue;
    double t[3];
    if (orc_inside(m, K, x, t)) {
      best = K;
      for (int j = 0; j < d; ++j) tb[j] = t[j];
    }
  }
  if (best >= 0 && xhat)
    for (int j = 0; j < d; ++j) xhat[j] = tb[j];
  return best;
}

/* --------------------------------------------- Q2 velocity (Sec. 2.3) --- */

/* 1D quadratic Lagrange basis on nodes 0, 1/2, 1. */
static double lagrange2(int a, double t) {
  if (a == 0) return (1.0 - t) * (1.0 - 2.0 * t);
  if (a == 1) return 4.0 * t * (1.0 - t);
  return t * (2.0 * t - 1.0);
}

/* The Q2 field with nodal values F ([dim][nnodes]) at x-hat in cell K. */
static void q2_eval_field(const orc_mesh *m, const double *F, int64_t K, const double *xhat, double *u) {
  int d = m->dim;
  int64_t i, j, k;
  cell_ijk(m, K, &i, &j, &k);
  int cmax = d == 3 ? 3 : 1;
  for (int comp = 0; comp < d; ++comp) {
    double s = 0.0;
    for (int c = 0; c < cmax; ++c)
      for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
          int64_t node = (2 * i + a) + m->nq[0] * ((2 * j + b) + m->nq[1] * (2 * k + c));
          double w = lagrange2(a, xhat[0]) * lagrange2(b, xhat[1]);
          if (d == 3) w = w * lagrange2(c, xhat[2]);
          s = s + F[(int64_t)comp * m->nnodes + node] * w;
        }
    u[comp] = s;
  }
}

/* u_h(x) = sum_i U_i phi-hat_i(x-hat) over the 3^d Q2 nodes of cell K: the
 * finite-element field evaluated at the stored reference coordinates
 * (the velocity evaluation of Sec. 2.3, and Remark 2.1). */
void orc_q2_eval(const orc_mesh *m, int64_t K, const double *xhat, double *u) { q2_eval_field(m, m->U, K, xhat, u); }

/* ------------------------------------------------ seeding (Sec. 2.2) --- */

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output n (n >= 0) of the
 * generator seeded with `seed` is mix(seed + (n+1) * golden gamma). */
uint64_t orc_splitmix64(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* R11: local-coordinate generation (the remark of Sec. 2.2): walk the
 * cells in order, draw x-hat uniform in [0,1)^d, x = Phi_K(x-hat), ids in
 * creation order.  per_cell may be NULL (then uniform_count in every cell).
 * Outputs particle-major: x[N][dim], xhat[N][dim], cell[N], id[N].
 * Returns N. */
int64_t orc_seed(const orc_mesh *m, const uint32_t *per_cell, uint32_t uniform_count, uint64_t seed,
                 uint64_t first_id, double *x, double *xhat, int64_t *cell, uint64_t *id) {
  int d = m->dim;
  int64_t g = 0;
  for (int64_t K = 0; K < m->ncells; ++K) {
    uint32_t nk = per_cell ? per_cell[K] : uniform_count;
    for (uint32_t q = 0; q < nk; ++q, ++g) {
      double t[3] = {0, 0, 0}, p[3] = {0, 0, 0};
      for (int j = 0; j < d; ++j) {
        uint64_t r = orc_splitmix64(seed, (uint64_t)g * (uint64_t)d + (uint64_t)j);
        t[j] = (double)(r >> 11) * 0x1.0p-53;
      }
      orc_phi(m, K, t, p);
      for (int j = 0; j < d; ++j) {
        x[g * d + j] = p[j];
        xhat[g * d + j] = t[j];
      }
      cell[g] = K;
      id[g] = first_id + (uint64_t)g;
    }
  }
  return g;
}

/* -------------------------------------------- advection (Sec. 2.3/2.4) --- */

/* u-tilde_h at stage time t^n + theta dt in cell K (R6): linear in time
 * between the two nodal fields, (1 - theta) u_h^n + theta u_h^{n+1}; the
 * steady field when no second field is set. */
static void velocity_at(const orc_mesh *m, int64_t K, const double *xhat, double theta, double *u) {
  orc_q2_eval(m, K, xhat, u);
  if (!m->Unext) return;
  double un[3] = {0, 0, 0};
  orc_mesh *mm = (orc_mesh *)m;
  double *keep = mm->U;
  mm->U = mm->Unext;
  orc_q2_eval(mm, K, xhat, un);
  mm->U = keep;
  for (int j = 0; j < m->dim; ++j) u[j] = (1.0 - theta) * u[j] + theta * un[j];
}

/* Velocity at a stage point: locate it (R7: every sub-step is followed by a
 * determination of the containing cell, Sec. 2.4), then evaluate u-tilde_h
 * there.  Returns 0 if the point has no owner (the particle is lost). */
static int stage_velocity(const orc_mesh *m, const double *y, double theta, double *u) {
  double t[3];
  int64_t K = orc_owner(m, y, t);
  if (K < 0) return 0;
  velocity_at(m, K, t, theta, u);
  return 1;
}

/* One time step of one particle (Sec. 2.3 with reading R5):
 *   Euler: x' = x + dt u(x)
 *   RK2  : k1 = dt u(x);             x' = x + dt u(x + k1/2)      (midpoint)
 *   RK4  : k1 = dt u(x), k2 = dt u(x + k1/2), k3 = dt u(x + k2/2),
 *          k4 = dt u(x + k3);        x' = x + (k1 + 2k2 + 2k3 + k4)/6
 * The first stage uses the stored (cell, x-hat) (Remark 2.1).  Stage s is
 * evaluated at time t^n + c_s dt with c = (0, 1/2, 1/2, 1) (RK4), (0, 1/2)
 * (RK2), (0) (Euler) when two fields are set (R6).  Then x' is located
 * (Sec. 2.4); no owner -> lost (option 3, R7). */
static void step_particle(const orc_mesh *m, orc_particle *p, double dt, int integrator) {
  int d = m->dim;
  double u[3] = {0, 0, 0}, k1[3] = {0, 0, 0}, k2[3] = {0, 0, 0}, k3[3] = {0, 0, 0}, k4[3] = {0, 0, 0};
  double y[3] = {0, 0, 0}, xn[3] = {0, 0, 0};
  velocity_at(m, p->cell, p->xhat, 0.0, u);
  for (int j = 0; j < d; ++j) k1[j] = dt * u[j];
  if (integrator == 1) {
    for (int j = 0; j < d; ++j) xn[j] = p->x[j] + k1[j];
  } else if (integrator == 2) {
    for (int j = 0; j < d; ++j) y[j] = p->x[j] + 0.5 * k1[j];
    if (!stage_velocity(m, y, 0.5, u)) goto lost;
    for (int j = 0; j < d; ++j) k2[j] = dt * u[j];
    for (int j = 0; j < d; ++j) xn[j] = p->x[j] + k2[j];
  } else {
    for (int j = 0; j < d; ++j) y[j] = p->x[j] + 0.5 * k1[j];
    if (!stage_velocity(m, y, 0.5, u)) goto lost;
    for (int j = 0; j < d; ++j) k2[j] = dt * u[j];
    for (int j = 0; j < d; ++j) y[j] = p->x[j] + 0.5 * k2[j];
    if (!stage_velocity(m, y, 0.5, u)) goto lost;
    for (int j = 0; j < d; ++j) k3[j] = dt * u[j];
    for (int j = 0; j < d; ++j) y[j] = p->x[j] + k3[j];
    if (!stage_velocity(m, y, 1.0, u)) goto lost;
    for (int j = 0; j < d; ++j) k4[j] = dt * u[j];
    for (int j = 0; j < d; ++j) xn[j] = p->x[j] + (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]) / 6.0;
  }
  {
    double t[3] = {0, 0, 0};
    int64_t K = orc_owner(m, xn, t);
    if (K < 0) goto lost;
    for (int j = 0; j < d; ++j) {
      p->x[j] = xn[j];
      p->xhat[j] = t[j];
    }
    p->cell = K;
  }
  return;
lost:
  p->cell = -1;
}

static int cmp_cell_id(const void *a, const void *b) {
  const orc_particle *p = (const orc_particle *)a, *q = (const orc_particle *)b;
  if (p->cell != q->cell) return p->cell < q->cell ? -1 : 1;
  if (p->id != q->id) return p->id < q->id ? -1 : 1;
  return 0;
}

/* n_steps x (advance every particle, then update the particle-cell map):
 * lost particles are removed (option 3 of the Sec. 2.4 listing), the rest
 * are ordered by (cell, id) (R9: the multimap's order, made canonical).
 * Arrays are particle-major and updated in place; props is [N][n_props].
 * Returns the number of particles still alive; *n_lost_out gets the rest. */
int64_t orc_advect(const orc_mesh *m, int64_t N, double *x, double *xhat, int64_t *cell, uint64_t *id, double *props,
                   int n_props, double dt, int integrator, int n_steps, int64_t *n_lost_out) {
  int d = m->dim;
  orc_particle *P = (orc_particle *)calloc(N > 0 ? N : 1, sizeof(orc_particle));
  double *pool = (double *)malloc(sizeof(double) * (N * n_props + 1));
  for (int64_t i = 0; i < N; ++i) {
    P[i].id = id[i];
    P[i].cell = cell[i];
    for (int j = 0; j < d; ++j) {
      P[i].x[j] = x[i * d + j];
      P[i].xhat[j] = xhat[i * d + j];
    }
    P[i].props = pool + i * n_props;
    for (int q = 0; q < n_props; ++q) P[i].props[q] = props[i * n_props + q];
  }
  int64_t n = N, lost = 0;
  for (int s = 0; s < n_steps; ++s) {
    for (int64_t i = 0; i < n; ++i) step_particle(m, &P[i], dt, integrator);
    int64_t w = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (P[i].cell < 0) {
        ++lost;
        continue;
      }
      P[w++] = P[i];
    }
    n = w;
    qsort(P, (size_t)n, sizeof(orc_particle), cmp_cell_id);
  }
  for (int64_t i = 0; i < n; ++i) {
    id[i] = P[i].id;
    cell[i] = P[i].cell;
    for (int j = 0; j < d; ++j) {
      x[i * d + j] = P[i].x[j];
      xhat[i * d + j] = P[i].xhat[j];
    }
    for (int q = 0; q < n_props; ++q) props[i * n_props + q] = P[i].props[q];
  }
  free(pool);
  free(P);
  if (n_lost_out) *n_lost_out = lost;
  return n;
}

/* Relocate arbitrary points: owner cell and x-hat of each (Sec. 2.4). */
void orc_locate_points(const orc_mesh *m, int64_t n, const double *x, int64_t *cell, double *xhat, int brute) {
  int d = m->dim;
  for (int64_t i = 0; i < n; ++i) {
    double t[3] = {0, 0, 0};
    int64_t K = brute ? orc_owner_brute(m, x + i * d, t) : orc_owner(m, x + i * d, t);
    cell[i] = K;
    for (int j = 0; j < d; ++j) xhat[i * d + j] = K >= 0 ? t[j] : 0.0;
  }
}

/* --------------------------- particle -> cell transfer (Sec. 2.7 (ii)) --- */

/* Arithmetic average of one property over the particles of each cell, left
 * fold in store order, divided by the count; empty cells get empty_fill and
 * count 0 (R10). */
void orc_cell_average(int64_t ncells, int64_t N, const int64_t *cell, const double *value, double empty_fill,
                      double *avg, int64_t *count) {
  double *sum = (double *)calloc(ncells > 0 ? ncells : 1, sizeof(double));
  for (int64_t K = 0; K < ncells; ++K) count[K] = 0;
  for (int64_t i = 0; i < N; ++i) {
    sum[cell[i]] = sum[cell[i]] + value[i];
    count[cell[i]] += 1;
  }
  for (int64_t K = 0; K < ncells; ++K) avg[K] = count[K] > 0 ? sum[K] / (double)count[K] : empty_fill;
  free(sum);
}

/* ------------------------------------ adjoint of the advection (form 3) --- */

/* d l_a / dt for the quadratic Lagrange basis on {0, 1/2, 1}. */
static double lagrange2_deriv(int a, double t) {
  if (a == 0) return 4.0 * t - 3.0;
  if (a == 1) return 4.0 - 8.0 * t;
  return 4.0 * t - 1.0;
}

/* Gu[c][j] = d u_c / d xhat_j = sum_i U_i,c d phi-hat_i / d xhat_j in cell K. */
static void q2_grad_ref(const orc_mesh *m, int64_t K, const double *xhat, double Gu[3][3]) {
  int d = m->dim;
  int64_t i, j, k;
  cell_ijk(m, K, &i, &j, &k);
  int cmax = d == 3 ? 3 : 1;
  for (int comp = 0; comp < d; ++comp)
    for (int jd = 0; jd < d; ++jd) {
      double s = 0.0;
      for (int c = 0; c < cmax; ++c)
        for (int b = 0; b < 3; ++b)
          for (int a = 0; a < 3; ++a) {
            int64_t node = (2 * i + a) + m->nq[0] * ((2 * j + b) + m->nq[1] * (2 * k + c));
            int idx[3] = {a, b, c};
            double w = 1.0;
            for (int q = 0; q < d; ++q) w = w * (q == jd ? lagrange2_deriv(idx[q], xhat[q]) : lagrange2(idx[q], xhat[q]));
            s = s + m->U[(int64_t)comp * m->nnodes + node] * w;
          }
      Gu[comp][jd] = s;
    }
}

/* Inverse of a 2x2 or 3x3 matrix by the adjugate. */
static void inverse_small(int d, double A[3][3], double B[3][3]) {
  if (d == 2) {
    double det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    B[0][0] = A[1][1] / det;
    B[0][1] = -A[0][1] / det;
    B[1][0] = -A[1][0] / det;
    B[1][1] = A[0][0] / det;
    return;
  }
  double c[3][3];
  c[0][0] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
  c[0][1] = A[1][2] * A[2][0] - A[1][0] * A[2][2];
  c[0][2] = A[1][0] * A[2][1] - A[1][1] * A[2][0];
  c[1][0] = A[0][2] * A[2][1] - A[0][1] * A[2][2];
  c[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
  c[1][2] = A[0][1] * A[2][0] - A[0][0] * A[2][1];
  c[2][0] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
  c[2][1] = A[0][2] * A[1][0] - A[0][0] * A[1][2];
  c[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
  double det = A[0][0] * c[0][0] + A[0][1] * c[0][1] + A[0][2] * c[0][2];
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) B[r][q] = c[q][r] / det;
}

/* du/dx at a located point: Gu J^{-1}, J = dPhi_K/dxhat (chain rule through
 * the inverse map; the cell is held fixed, reading R12). */
static void velocity_jacobian(const orc_mesh *m, int64_t K, const double *xhat, double G[3][3]) {
  int d = m->dim;
  double Gu[3][3] = {{0}}, J[3][3] = {{0}}, Ji[3][3] = {{0}};
  q2_grad_ref(m, K, xhat, Gu);
  phi_jacobian(m, K, xhat, J);
  inverse_small(d, J, Ji);
  for (int c = 0; c < d; ++c)
    for (int q = 0; q < d; ++q) {
      double s = 0.0;
      for (int j = 0; j < d; ++j) s = s + Gu[c][j] * Ji[j][q];
      G[c][q] = s;
    }
}

/* grad[comp][node] += w[comp] * phi-hat_node(xhat) over the Q2 nodes of K. */
static void scatter_basis(const orc_mesh *m, int64_t K, const double *xhat, const double *w, double *grad) {
  int d = m->dim;
  int64_t i, j, k;
  cell_ijk(m, K, &i, &j, &k);
  int cmax = d == 3 ? 3 : 1;
  for (int c = 0; c < cmax; ++c)
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a) {
        int64_t node = (2 * i + a) + m->nq[0] * ((2 * j + b) + m->nq[1] * (2 * k + c));
        double phi = lagrange2(a, xhat[0]) * lagrange2(b, xhat[1]);
        if (d == 3) phi = phi * lagrange2(c, xhat[2]);
        for (int comp = 0; comp < d; ++comp) grad[(int64_t)comp * m->nnodes + node] += w[comp] * phi;
      }
}

/* Loss L = sum over particles alive after n_steps of |x_final - target|^2 and
 * its gradient with respect to every nodal velocity value, by a reverse sweep
 * of the Sec. 2.3 integrators (reading R5) recomputed from per-step position
 * checkpoints.  Particles are independent, so each is swept on its own:
 *   forward  x_{n+1} = x_n + sum_s b_s k_s,  k_s = dt u(y_s),  y_s = x_n + a_s k_{s-1}
 *   reverse  lambda_k_s = b_s lambda + a_{s+1} lambda_y_{s+1},
 *            lambda_y_s = dt G_s^T lambda_k_s  (G_s = du/dx at y_s),
 *            dL/dU += dt phi-hat(xhat_s) lambda_k_s,
 *            lambda  <- lambda + sum_s lambda_y_s
 * Lost particles contribute nothing.  Inputs are particle-major; targets is
 * [N][dim] in input order; grad is [dim][nnodes] (overwritten).  Returns L. */
double orc_advect_adjoint(const orc_mesh *m, int64_t N, const double *x, const double *xhat, const int64_t *cell,
                          double dt, int integrator, int n_steps, const double *targets, double *grad) {
  int d = m->dim;
  int S = integrator == 1 ? 1 : (integrator == 2 ? 2 : 4);
  double a_[4] = {0.0, 0.5, 0.5, 1.0}, b_[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  if (S == 1) b_[0] = 1.0;
  if (S == 2) {
    b_[0] = 0.0;
    b_[1] = 1.0;
  }
  for (int64_t q = 0; q < (int64_t)d * m->nnodes; ++q) grad[q] = 0.0;
  double loss = 0.0;
  double *xs = (double *)malloc(sizeof(double) * (size_t)(n_steps + 1) * 3);
  double *ts = (double *)malloc(sizeof(double) * (size_t)(n_steps + 1) * 3);
  int64_t *ks = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_steps + 1));
  for (int64_t p = 0; p < N; ++p) {
    /* forward with checkpoints */
    orc_particle P;
    double props_dummy = 0.0;
    P.id = 0;
    P.cell = cell[p];
    P.props = &props_dummy;
    for (int j = 0; j < d; ++j) {
      P.x[j] = x[p * d + j];
      P.xhat[j] = xhat[p * d + j];
    }
    int alive = 1;
    for (int n = 0; n < n_steps; ++n) {
      for (int j = 0; j < d; ++j) {
        xs[n * 3 + j] = P.x[j];
        ts[n * 3 + j] = P.xhat[j];
      }
      ks[n] = P.cell;
      step_particle(m, &P, dt, integrator);
      if (P.cell < 0) {
        alive = 0;
        break;
      }
    }
    if (!alive) continue;
    double lam[3] = {0, 0, 0};
    for (int j = 0; j < d; ++j) {
      double r = P.x[j] - targets[p * d + j];
      loss = loss + r * r;
      lam[j] = 2.0 * r;
    }
    /* reverse sweep */
    for (int n = n_steps - 1; n >= 0; --n) {
      double xn[3], y[4][3], k[4][3], th[4][3], u[3];
      int64_t K[4];
      for (int j = 0; j < d; ++j) xn[j] = xs[n * 3 + j];
      K[0] = ks[n];
      for (int j = 0; j < d; ++j) {
        y[0][j] = xn[j];
        th[0][j] = ts[n * 3 + j];
      }
      for (int s = 0; s < S; ++s) {
        if (s > 0) {
          for (int j = 0; j < d; ++j) y[s][j] = xn[j] + a_[s] * k[s - 1][j];
          K[s] = orc_owner(m, y[s], th[s]);
        }
        orc_q2_eval(m, K[s], th[s], u);
        for (int j = 0; j < d; ++j) k[s][j] = dt * u[j];
      }
      double lam_x[3], lam_k[4][3], lam_y_next[3] = {0, 0, 0};
      for (int j = 0; j < d; ++j) lam_x[j] = lam[j];
      for (int s = S - 1; s >= 0; --s) {
        double G[3][3] = {{0}}, w[3];
        for (int j = 0; j < d; ++j) lam_k[s][j] = b_[s] * lam[j] + (s + 1 < S ? a_[s + 1] * lam_y_next[j] : 0.0);
        velocity_jacobian(m, K[s], th[s], G);
        double lam_y[3];
        for (int q = 0; q < d; ++q) {
          double acc = 0.0;
          for (int c = 0; c < d; ++c) acc = acc + G[c][q] * lam_k[s][c];
          lam_y[q] = dt * acc;
        }
        for (int j = 0; j < d; ++j) {
          w[j] = dt * lam_k[s][j];
          lam_x[j] = lam_x[j] + lam_y[j];
          lam_y_next[j] = lam_y[j];
        }
        scatter_basis(m, K[s], th[s], w, grad);
      }
      for (int j = 0; j < d; ++j) lam[j] = lam_x[j];
    }
  }
  free(xs);
  free(ts);
  free(ks);
  return loss;
}

/* Forward (tangent-linear) mode of the same map: the derivative of each
 * surviving particle's final position in the direction V of the nodal
 * velocities ([dim][nnodes]).  Per step, with the stage points re-formed from
 * the step's start as in the reverse sweep and v_h the Q2 field of V,
 *   delta-y_s = delta-x + a_s delta-k_{s-1},
 *   delta-k_s = dt (G_s delta-y_s + v_h(y_s)),
 *   delta-x'  = delta-x + sum_s b_s delta-k_s
 * (cells held fixed, R12); the trajectory itself is stepped by step_particle.
 * Written apart from the reverse sweep, it checks that sweep through
 * <J V, W> = <V, J^T W>.  Inputs particle-major; dx [N][dim] (0 for lost
 * particles) and alive [N] are written. */
void orc_advect_tangent(const orc_mesh *m, int64_t N, const double *x, const double *xhat, const int64_t *cell,
                        double dt, int integrator, int n_steps, const double *V, double *dx, int32_t *alive) {
  int d = m->dim;
  int S = integrator == 1 ? 1 : (integrator == 2 ? 2 : 4);
  double a_[4] = {0.0, 0.5, 0.5, 1.0}, b_[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  if (S == 1) b_[0] = 1.0;
  if (S == 2) {
    b_[0] = 0.0;
    b_[1] = 1.0;
  }
  for (int64_t p = 0; p < N; ++p) {
    orc_particle P;
    double props_dummy = 0.0;
    P.id = 0;
    P.cell = cell[p];
    P.props = &props_dummy;
    double dxp[3] = {0, 0, 0};
    for (int j = 0; j < d; ++j) {
      P.x[j] = x[p * d + j];
      P.xhat[j] = xhat[p * d + j];
    }
    int ok = 1;
    for (int n = 0; n < n_steps && ok; ++n) {
      double k[4][3] = {{0}}, dk[4][3] = {{0}}, dnew[3];
      for (int j = 0; j < d; ++j) dnew[j] = dxp[j];
      for (int s = 0; s < S && ok; ++s) {
        double y[3] = {0, 0, 0}, dy[3] = {0, 0, 0}, th[3] = {0, 0, 0}, u[3] = {0, 0, 0}, v[3] = {0, 0, 0};
        double G[3][3] = {{0}};
        int64_t K;
        for (int j = 0; j < d; ++j) {
          y[j] = s == 0 ? P.x[j] : P.x[j] + a_[s] * k[s - 1][j];
          dy[j] = s == 0 ? dxp[j] : dxp[j] + a_[s] * dk[s - 1][j];
        }
        if (s == 0) {
          K = P.cell;
          for (int j = 0; j < d; ++j) th[j] = P.xhat[j];
        } else {
          K = orc_owner(m, y, th);
          if (K < 0) {
            ok = 0;
            break;
          }
        }
        orc_q2_eval(m, K, th, u);
        q2_eval_field(m, V, K, th, v);
        velocity_jacobian(m, K, th, G);
        for (int c = 0; c < d; ++c) {
          double gd = 0.0;
          for (int q = 0; q < d; ++q) gd = gd + G[c][q] * dy[q];
          k[s][c] = dt * u[c];
          dk[s][c] = dt * (gd + v[c]);
          dnew[c] = dnew[c] + b_[s] * dk[s][c];
        }
      }
      if (!ok) break;
      step_particle(m, &P, dt, integrator);
      if (P.cell < 0) ok = 0;
      for (int j = 0; j < d; ++j) dxp[j] = dnew[j];
    }
    alive[p] = ok;
    for (int j = 0; j < d; ++j) dx[p * d + j] = ok ? dxp[j] : 0.0;
  }
}

/* The loss alone (the forward of the adjoint), for finite differences. */
double orc_advect_loss(const orc_mesh *m, int64_t N, const double *x, const double *xhat, const int64_t *cell,
                       double dt, int integrator, int n_steps, const double *targets) {
  int d = m->dim;
  double loss = 0.0;
  for (int64_t p = 0; p < N; ++p) {
    orc_particle P;
    double props_dummy = 0.0;
    P.id = 0;
    P.cell = cell[p];
    P.props = &props_dummy;
    for (int j = 0; j < d; ++j) {
      P.x[j] = x[p * d + j];
      P.xhat[j] = xhat[p * d + j];
    }
    int alive = 1;
    for (int n = 0; n < n_steps && alive; ++n) {
      step_particle(m, &P, dt, integrator);
      if (P.cell < 0) alive = 0;
    }
    if (!alive) continue;
    for (int j = 0; j < d; ++j) {
      double r = P.x[j] - targets[p * d + j];
      loss = loss + r * r;
    }
  }
  return loss;
}

/* Sec. 2.7 (ii) also names the geometric and harmonic averages of the
 * particles of a cell:
 *   geometric  exp( (1/n_K) sum log v )      (defined for v > 0)
 *   harmonic   n_K / sum (1 / v)             (defined for v > 0)
 * A cell holding a value <= 0 gets NaN (reading R14: the paper is silent);
 * empty cells get empty_fill (R10).  kind: 0 arithmetic, 1 geometric,
 * 2 harmonic.  Left folds in store order. */
void orc_cell_average_kind(int64_t ncells, int64_t N, const int64_t *cell, const double *value, int kind,
                           double empty_fill, double *avg, int64_t *count) {
  if (kind == 0) {
    orc_cell_average(ncells, N, cell, value, empty_fill, avg, count);
    return;
  }
  double *sum = (double *)calloc(ncells > 0 ? ncells : 1, sizeof(double));
  int *bad = (int *)calloc(ncells > 0 ? ncells : 1, sizeof(int));
  for (int64_t K = 0; K < ncells; ++K) count[K] = 0;
  for (int64_t i = 0; i < N; ++i) {
    int64_t K = cell[i];
    double v = value[i];
    if (!(v > 0.0)) bad[K] = 1;
    sum[K] = sum[K] + (kind == 1 ? log(v) : 1.0 / v);
    count[K] += 1;
  }
  for (int64_t K = 0; K < ncells; ++K) {
    if (count[K] == 0)
      avg[K] = empty_fill;
    else if (bad[K])
      avg[K] = NAN;
    else if (kind == 1)
      avg[K] = exp(sum[K] / (double)count[K]);
    else
      avg[K] = (double)count[K] / sum[K];
  }
  free(sum);
  free(bad);
}

/* ------------------------------- property ODEs on particles (Sec. 2.6) --- */

/* Right-hand side of the particle system z = (x, d, F) at a located point
 * (cell K, reference coordinates xhat), Sec. 2.6:
 *   x' = u_h
 *   d' = alpha |eps-dot| - beta d,   eps-dot = (G + G^T) / 2,
 *        |.| the Frobenius norm (reading R15)
 *   F' = G F                          (F(0) = I, the total deformation)
 * with G = grad u_h at the point (cell held fixed, as for the adjoint).
 * z is laid out [x_0..x_{dim-1}, d, F_00, F_01, .., F_{dim-1,dim-1}]. */
static void props_rhs(const orc_mesh *m, int64_t K, const double *xhat, const double *z, int use_damage,
                      double alpha, double beta, int use_defgrad, double *f) {
  int d = m->dim;
  double u[3] = {0, 0, 0}, G[3][3] = {{0}};
  orc_q2_eval(m, K, xhat, u);
  for (int j = 0; j < d; ++j) f[j] = u[j];
  f[d] = 0.0;
  for (int q = 0; q < d * d; ++q) f[d + 1 + q] = 0.0;
  if (!use_damage && !use_defgrad) return;
  velocity_jacobian(m, K, xhat, G);
  if (use_damage) {
    double s = 0.0;
    for (int r = 0; r < d; ++r)
      for (int c = 0; c < d; ++c) {
        double e = 0.5 * (G[r][c] + G[c][r]);
        s = s + e * e;
      }
    f[d] = alpha * sqrt(s) - beta * z[d];
  }
  if (use_defgrad) {
    const double *F = z + d + 1;
    for (int r = 0; r < d; ++r)
      for (int c = 0; c < d; ++c) {
        double acc = 0.0;
        for (int q = 0; q < d; ++q) acc = acc + G[r][q] * F[q * d + c];
        f[d + 1 + r * d + c] = acc;
      }
  }
}

/* One step of the coupled system with the integrators of step_particle
 * (reading R5), every stage point located before the right-hand side is
 * evaluated there (R7).  The position part is the same arithmetic as
 * step_particle.  Returns 0 if the particle is lost. */
static int step_particle_props(const orc_mesh *m, orc_particle *p, double *z_in, double dt, int integrator,
                               int use_damage, double alpha, double beta, int use_defgrad) {
  int d = m->dim, nz = d + 1 + d * d;
  double z[13], y[13], f[13], k1[13], k2[13], k3[13], k4[13], zn[13], t[3] = {0, 0, 0};
  for (int q = 0; q < nz; ++q) z[q] = z_in[q];
  for (int j = 0; j < d; ++j) z[j] = p->x[j];
  props_rhs(m, p->cell, p->xhat, z, use_damage, alpha, beta, use_defgrad, f);
  for (int q = 0; q < nz; ++q) k1[q] = dt * f[q];
  if (integrator == 1) {
    for (int q = 0; q < nz; ++q) zn[q] = z[q] + k1[q];
  } else if (integrator == 2) {
    int64_t K;
    for (int q = 0; q < nz; ++q) y[q] = z[q] + 0.5 * k1[q];
    if ((K = orc_owner(m, y, t)) < 0) return 0;
    props_rhs(m, K, t, y, use_damage, alpha, beta, use_defgrad, f);
    for (int q = 0; q < nz; ++q) k2[q] = dt * f[q];
    for (int q = 0; q < nz; ++q) zn[q] = z[q] + k2[q];
  } else {
    int64_t K;
    for (int q = 0; q < nz; ++q) y[q] = z[q] + 0.5 * k1[q];
    if ((K = orc_owner(m, y, t)) < 0) return 0;
    props_rhs(m, K, t, y, use_damage, alpha, beta, use_defgrad, f);
    for (int q = 0; q < nz; ++q) k2[q] = dt * f[q];
    for (int q = 0; q < nz; ++q) y[q] = z[q] + 0.5 * k2[q];
    if ((K = orc_owner(m, y, t)) < 0) return 0;
    props_rhs(m, K, t, y, use_damage, alpha, beta, use_defgrad, f);
    for (int q = 0; q < nz; ++q) k3[q] = dt * f[q];
    for (int q = 0; q < nz; ++q) y[q] = z[q] + k3[q];
    if ((K = orc_owner(m, y, t)) < 0) return 0;
    props_rhs(m, K, t, y, use_damage, alpha, beta, use_defgrad, f);
    for (int q = 0; q < nz; ++q) k4[q] = dt * f[q];
    for (int q = 0; q < nz; ++q) zn[q] = z[q] + (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]) / 6.0;
  }
  int64_t K = orc_owner(m, zn, t);
  if (K < 0) return 0;
  for (int j = 0; j < d; ++j) {
    p->x[j] = zn[j];
    p->xhat[j] = t[j];
  }
  p->cell = K;
  for (int q = d; q < nz; ++q) z_in[q] = zn[q];
  return 1;
}

/* orc_advect with the Sec. 2.6 property ODEs integrated along the particle
 * paths: property slot `damage` holds d (or -1 = none), slots
 * defgrad .. defgrad + dim^2 - 1 hold F row-major (or defgrad = -1).  Other
 * properties ride along unchanged.  The steady field only (a second field
 * set returns -1).  Returns the number alive; *n_lost_out gets the rest. */
int64_t orc_advect_properties(const orc_mesh *m, int64_t N, double *x, double *xhat, int64_t *cell, uint64_t *id,
                              double *props, int n_props, double dt, int integrator, int n_steps, int damage,
                              double alpha, double beta, int defgrad, int64_t *n_lost_out) {
  if (m->Unext) return -1;
  int d = m->dim;
  int use_damage = damage >= 0, use_defgrad = defgrad >= 0;
  orc_particle *P = (orc_particle *)calloc(N > 0 ? N : 1, sizeof(orc_particle));
  double *pool = (double *)malloc(sizeof(double) * (N * n_props + 1));
  for (int64_t i = 0; i < N; ++i) {
    P[i].id = id[i];
    P[i].cell = cell[i];
    for (int j = 0; j < d; ++j) {
      P[i].x[j] = x[i * d + j];
      P[i].xhat[j] = xhat[i * d + j];
    }
    P[i].props = pool + i * n_props;
    for (int q = 0; q < n_props; ++q) P[i].props[q] = props[i * n_props + q];
  }
  int64_t n = N, lost = 0;
  for (int s = 0; s < n_steps; ++s) {
    for (int64_t i = 0; i < n; ++i) {
      double z[13] = {0};
      if (use_damage) z[d] = P[i].props[damage];
      if (use_defgrad)
        for (int q = 0; q < d * d; ++q) z[d + 1 + q] = P[i].props[defgrad + q];
      if (!step_particle_props(m, &P[i], z, dt, integrator, use_damage, alpha, beta, use_defgrad)) {
        P[i].cell = -1;
        continue;
      }
      if (use_damage) P[i].props[damage] = z[d];
      if (use_defgrad)
        for (int q = 0; q < d * d; ++q) P[i].props[defgrad + q] = z[d + 1 + q];
    }
    int64_t w = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (P[i].cell < 0) {
        ++lost;
        continue;
      }
      P[w++] = P[i];
    }
    n = w;
    qsort(P, (size_t)n, sizeof(orc_particle), cmp_cell_id);
  }
  for (int64_t i = 0; i < n; ++i) {
    id[i] = P[i].id;
    cell[i] = P[i].cell;
    for (int j = 0; j < d; ++j) {
      x[i * d + j] = P[i].x[j];
      xhat[i * d + j] = P[i].xhat[j];
    }
    for (int q = 0; q < n_props; ++q) props[i * n_props + q] = P[i].props[q];
  }
  free(pool);
  free(P);
  if (n_lost_out) *n_lost_out = lost;
  return n;
}

/* ------------------ particle -> field transfer, Sec. 2.7 (iv) and (v) --- */

/* (iv) Shape-function-weighted averaging (reading R17): the value at mesh
 * vertex v is
 *     p_v = sum_i phi_v(x_i) p_i / sum_i phi_v(x_i)
 * over the particles i in the support of phi_v, the (bi/tri)linear nodal
 * basis function of v.  In the particle's cell K, phi_v(x_i) is the map's
 * weight of v's local vertex at the particle's reference coordinates.  Both
 * sums are left folds over the particles in store order (cell, then id).
 * A vertex whose weights sum to 0 gets empty_fill; weight[v] is that sum. */
void orc_vertex_average(const orc_mesh *m, int64_t N, const int64_t *cell, const double *xhat, const double *value,
                        double empty_fill, double *avg, double *weight) {
  int d = m->dim;
  double *num = (double *)calloc(m->nverts > 0 ? m->nverts : 1, sizeof(double));
  for (int64_t v = 0; v < m->nverts; ++v) weight[v] = 0.0;
  for (int64_t p = 0; p < N; ++p) {
    int64_t i, j, k;
    cell_ijk(m, cell[p], &i, &j, &k);
    for (int lv = 0; lv < (1 << d); ++lv) {
      int64_t vi = i + (lv & 1), vj = j + ((lv >> 1) & 1), vk = k + (d == 3 ? ((lv >> 2) & 1) : 0);
      int64_t v = vi + m->nv[0] * (vj + m->nv[1] * vk);
      double w = vertex_weight(d, lv, xhat + p * d);
      num[v] = num[v] + w * value[p];
      weight[v] = weight[v] + w;
    }
  }
  for (int64_t v = 0; v < m->nverts; ++v) avg[v] = weight[v] > 0.0 ? num[v] / weight[v] : empty_fill;
  free(num);
}

/* (v) Linear least-squares projection (reading R18): in every cell, the
 * function f(xhat) = c_0 + sum_j c_{j+1} (xhat_j - 1/2), linear in the
 * reference coordinates, that minimises sum_{i in K} (f(xhat_i) - p_i)^2.
 * The minimiser solves the normal equations (A^T A) c = A^T p, A the cell's
 * design matrix with rows (1, xhat_i - 1/2); A^T A and A^T p are left folds
 * in store order, and the system is solved by Gaussian elimination with
 * partial pivoting.  A cell with at most dim particles, or whose elimination
 * meets a pivot <= 1e-12 times the largest diagonal entry of A^T A, gets the
 * arithmetic mean (c_0 = mean, slopes 0); an empty cell gets c_0 =
 * empty_fill.  coef is [ncells][dim+1]; count[K] is the cell's particles. */
void orc_cell_lsq_linear(const orc_mesh *m, int64_t N, const int64_t *cell, const double *xhat, const double *value,
                         double empty_fill, double *coef, int64_t *count) {
  int d = m->dim, nb = d + 1;
  int64_t C = m->ncells;
  double *M = (double *)calloc((size_t)(C > 0 ? C : 1) * 16, sizeof(double));
  double *b = (double *)calloc((size_t)(C > 0 ? C : 1) * 4, sizeof(double));
  double *sum = (double *)calloc((size_t)(C > 0 ? C : 1), sizeof(double));
  for (int64_t K = 0; K < C; ++K) count[K] = 0;
  for (int64_t p = 0; p < N; ++p) {
    int64_t K = cell[p];
    double a[4];
    a[0] = 1.0;
    for (int j = 0; j < d; ++j) a[j + 1] = xhat[p * d + j] - 0.5;
    for (int r = 0; r < nb; ++r) {
      for (int c = 0; c < nb; ++c) M[K * 16 + r * 4 + c] = M[K * 16 + r * 4 + c] + a[r] * a[c];
      b[K * 4 + r] = b[K * 4 + r] + a[r] * value[p];
    }
    sum[K] = sum[K] + value[p];
    count[K] += 1;
  }
  for (int64_t K = 0; K < C; ++K) {
    double *c = coef + K * nb;
    for (int r = 0; r < nb; ++r) c[r] = 0.0;
    if (count[K] == 0) {
      c[0] = empty_fill;
      continue;
    }
    int ok = count[K] > d;
    double A[4][5];
    double dmax = 0.0;
    for (int r = 0; r < nb; ++r) {
      for (int q = 0; q < nb; ++q) A[r][q] = M[K * 16 + r * 4 + q];
      A[r][nb] = b[K * 4 + r];
      if (A[r][r] > dmax) dmax = A[r][r];
    }
    for (int col = 0; col < nb && ok; ++col) {
      int piv = col;
      for (int r = col + 1; r < nb; ++r)
        if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
      if (!(fabs(A[piv][col]) > 1e-12 * dmax)) {
        ok = 0;
        break;
      }
      if (piv != col)
        for (int q = 0; q <= nb; ++q) {
          double t = A[col][q];
          A[col][q] = A[piv][q];
          A[piv][q] = t;
        }
      for (int r = col + 1; r < nb; ++r) {
        double f = A[r][col] / A[col][col];
        for (int q = col; q <= nb; ++q) A[r][q] = A[r][q] - f * A[col][q];
      }
    }
    if (!ok) {
      c[0] = sum[K] / (double)count[K];
      continue;
    }
    for (int r = nb - 1; r >= 0; --r) {
      double s = A[r][nb];
      for (int q = r + 1; q < nb; ++q) s = s - A[r][q] * c[q];
      c[r] = s / A[r][r];
    }
  }
  free(M);
  free(b);
  free(sum);
}

/* ----------------------- generation with a density rho(x), Sec. 2.2 --- */

/* Global index of local vertex v of cell K. */
static int64_t cell_vertex_index(const orc_mesh *m, int64_t K, int v) {
  int64_t i, j, k;
  cell_ijk(m, K, &i, &j, &k);
  return (i + (v & 1)) + m->nv[0] * ((j + ((v >> 1) & 1)) + m->nv[1] * (k + ((v >> 2) & 1)));
}

/* det J by cofactors of the first row, summed left to right:
 *   2D  J00 J11 - J01 J10
 *   3D  J00 (J11 J22 - J12 J21) + J01 (J12 J20 - J10 J22) + J02 (J10 J21 - J11 J20) */
static double det_small(int d, double J[3][3]) {
  if (d == 2) return J[0][0] * J[1][1] - J[0][1] * J[1][0];
  double c0 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  double c1 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  double c2 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  return J[0][0] * c0 + J[0][1] * c1 + J[0][2] * c2;
}

/* The density pulled back to the reference cell (Sec. 2.2, MH paragraph):
 *   rho-hat(xhat) = rho_h(Phi_K(xhat)) |det grad-hat Phi_K(xhat)|
 * with rho_h the (bi/tri)linear interpolant of the vertex values, which on
 * cell K is sum_v rho_{K,v} w_v(xhat).  Written operation order (the GPU
 * evaluates the same sequence of IEEE operations, so that the acceptance
 * decisions agree exactly): rho_h summed over local vertices v = 0..2^d-1
 * with w_v the product over axes in order (vertex_weight); J_ij summed over v
 * in order of X_{K,v,i} * dw_v/dt_j (phi_jacobian); det by det_small. */
static double rho_hat(const orc_mesh *m, int64_t K, const double *rho, const double *t) {
  int d = m->dim;
  double r = 0.0, J[3][3] = {{0}};
  for (int v = 0; v < (1 << d); ++v) r = r + rho[cell_vertex_index(m, K, v)] * vertex_weight(d, v, t);
  phi_jacobian(m, K, t, J);
  return r * fabs(det_small(d, J));
}

/* Cell weights w_K = int_K rho_h dx (first loop of the Sec. 2.2 listing),
 * by the tensor 2-point Gauss rule on the reference cell: nodes
 * 1/2 -+ 1/(2 sqrt 3), weights 1/2 per axis.  rho_h |det J| has degree <= 3
 * in each reference coordinate on (bi/tri)linear cells, so the rule is
 * exact.  rho is [nverts]; w is [ncells]. */
void orc_cell_weights(const orc_mesh *m, const double *rho, double *w) {
  int d = m->dim;
  double g[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
  for (int64_t K = 0; K < m->ncells; ++K) {
    double s = 0.0;
    for (int q = 0; q < (1 << d); ++q) {
      double t[3] = {g[q & 1], g[(q >> 1) & 1], g[(q >> 2) & 1]};
      double wq = 1.0;
      for (int j = 0; j < d; ++j) wq = wq * 0.5;
      s = s + wq * rho_hat(m, K, rho, t);
    }
    w[K] = s;
  }
}

/* Particles per cell from cell weights (the second and third parts of the
 * Sec. 2.2 listing, on one process): acc_K = w_0 + ... + w_K as a left fold,
 * W = acc_{C-1}; draw i = 0..N-1 takes u_i = top 53 bits of SplitMix64
 * output i times 2^-53, r_i = W u_i, and goes to the first cell with
 * acc_K > r_i (reading R19: "first accumulated weight above r" rather than
 * "not below", so that a cell of zero weight is never chosen), or, if fl(W
 * u_i) rounded up to W, to the last cell of positive weight.  Weights must be
 * finite and >= 0 with W > 0.  counts is [ncells]. */
void orc_draw_cell_counts(int64_t C, const double *w, int64_t N, uint64_t seed, int64_t *counts) {
  double *acc = (double *)malloc(sizeof(double) * (size_t)(C > 0 ? C : 1));
  double s = 0.0;
  int64_t last = -1;
  for (int64_t K = 0; K < C; ++K) {
    s = s + w[K];
    acc[K] = s;
    counts[K] = 0;
    if (w[K] > 0.0) last = K;
  }
  double W = s;
  for (int64_t i = 0; i < N; ++i) {
    double u = (double)(orc_splitmix64(seed, (uint64_t)i) >> 11) * 0x1.0p-53;
    double r = W * u;
    int64_t lo = 0, hi = C; /* first K in [lo, hi) with acc[K] > r */
    while (lo < hi) {
      int64_t mid = lo + (hi - lo) / 2;
      if (acc[mid] > r)
        hi = mid;
      else
        lo = mid + 1;
    }
    counts[lo < C ? lo : last] += 1;
  }
  free(acc);
}

/* In-cell Metropolis-Hastings generation (Sec. 2.2, MH paragraph): in cell
 * K with n_K particles, a chain on the reference cell with target rho-hat
 * and uniform proposals, started at the cell centre, of length J n_K
 * (J = thinning); every J-th state (states J, 2J, ..) becomes a particle.
 * Step s of the chain (global step g = J * first_K + s, first_K the number
 * of particles of the cells before K) draws SplitMix64 outputs
 * g (dim+1) + j: j < dim the proposal's coordinates (top 53 bits times
 * 2^-53), j = dim the acceptance uniform u.  The proposal y is accepted
 * when u rho-hat(current) < rho-hat(y) (reading R20: a fixed thinning J
 * stands in for the paper's J chosen above the longest stretch of repeated
 * states, which is known only after the run).
 * x = Phi_K(xhat), ids first_id + (creation index).  Outputs particle-major
 * as in orc_seed.  Returns N. */
int64_t orc_seed_mh(const orc_mesh *m, const uint32_t *per_cell, const double *rho, uint32_t thinning,
                    uint64_t seed, uint64_t first_id, double *x, double *xhat, int64_t *cell, uint64_t *id) {
  int d = m->dim;
  int64_t g = 0;
  for (int64_t K = 0; K < m->ncells; ++K) {
    uint32_t nk = per_cell[K];
    if (nk == 0) continue;
    double cur[3] = {0.5, 0.5, 0.5};
    double rc = rho_hat(m, K, rho, cur);
    uint64_t step0 = (uint64_t)thinning * (uint64_t)g;
    for (uint64_t s = 0; s < (uint64_t)thinning * nk; ++s) {
      uint64_t gs = step0 + s;
      double y[3] = {0.5, 0.5, 0.5};
      for (int j = 0; j < d; ++j)
        y[j] = (double)(orc_splitmix64(seed, gs * (uint64_t)(d + 1) + (uint64_t)j) >> 11) * 0x1.0p-53;
      double u = (double)(orc_splitmix64(seed, gs * (uint64_t)(d + 1) + (uint64_t)d) >> 11) * 0x1.0p-53;
      double ry = rho_hat(m, K, rho, y);
      if (u * rc < ry) {
        for (int j = 0; j < d; ++j) cur[j] = y[j];
        rc = ry;
      }
      if ((s + 1) % thinning == 0) {
        double p[3] = {0, 0, 0};
        orc_phi(m, K, cur, p);
        for (int j = 0; j < d; ++j) {
          x[g * d + j] = p[j];
          xhat[g * d + j] = cur[j];
        }
        cell[g] = K;
        id[g] = first_id + (uint64_t)g;
        ++g;
      }
    }
  }
  return g;
}

/* Prescribed particle locations (Sec. 2.2, second listing): for k = 0..n-1
 * in order, the point x_k becomes a particle of its owner cell (the lowest-
 * index cell holding it, reading R4) with xhat = Phi_K^{-1}(x_k) and the
 * next id; points in no cell are skipped.  The result is ordered by
 * (cell, id) (R9).  x is [n][dim]; outputs particle-major; returns the
 * number created. */
int64_t orc_import(const orc_mesh *m, int64_t n, const double *x, uint64_t first_id, double *xo, double *xhato,
                   int64_t *cello, uint64_t *ido) {
  int d = m->dim;
  orc_particle *P = (orc_particle *)calloc(n > 0 ? n : 1, sizeof(orc_particle));
  int64_t c = 0;
  uint64_t next_id = first_id;
  for (int64_t k = 0; k < n; ++k) {
    double t[3] = {0, 0, 0};
    int64_t K = orc_owner(m, x + k * d, t);
    if (K < 0) continue;
    P[c].id = next_id++;
    P[c].cell = K;
    for (int j = 0; j < d; ++j) {
      P[c].x[j] = x[k * d + j];
      P[c].xhat[j] = t[j];
    }
    ++c;
  }
  qsort(P, (size_t)c, sizeof(orc_particle), cmp_cell_id);
  for (int64_t i = 0; i < c; ++i) {
    for (int j = 0; j < d; ++j) {
      xo[i * d + j] = P[i].x[j];
      xhato[i * d + j] = P[i].xhat[j];
    }
    cello[i] = P[i].cell;
    ido[i] = P[i].id;
  }
  free(P);
  return c;
}
