/*
 * csph_oracle.c -- plain FP64 CPU oracle for contact SPH with Voronoi dynamic
 * domain decomposition (arXiv 1805.05128).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark.  It shares no code with the CUDA library.
 * Single-threaded, FP64, built with -ffp-contract=off.  Each routine names the
 * passage of the paper it follows.  Points where the paper is silent take the
 * readings listed here in the routine comments:
 *   - the pair Riemann solver is the linearised (acoustic) solver at the
 *     particle-centre states, no reconstruction (Sec. 4.1 cites it only);
 *   - the time integrator is kick-drift-kick leapfrog with one rate
 *     evaluation per step and dt = CFL * min_i eta d_i / (c_i + |v_i|);
 *   - h_ij = eta (d_i + d_j) / 2, eta multiplying eq. (SmoothingLengthDef);
 *   - g_kl of eq. (BalancingOffset) is g_k - g_l;
 *   - the double sum of eq. (BalancingOffsetPlusRot) visits each triangle
 *     {k, l, m} of mutually adjacent units once per k;
 *   - the three-body term is applied only for 2D decompositions.
 *
 * Parity of every routine here is pinned by the "not gpu" tests against
 * closed forms, brute force, library routines or invariants (see tests/).
 */
#include "csph_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

static double get(const double* a, int64_t i) { return a ? a[i] : 0.0; }

/* ------------------------------------------------------------------------ */
/* Smoothing kernels (Sec. 4.1).  W(r, h) and dW/dr.                         */
/* ------------------------------------------------------------------------ */

/* Cubic spline M4 with support 2h.  Normalisation 2/3 (1D), 10/(7 pi) (2D),
 * 1/pi (3D), each divided by h^dim. */
static double cubic_norm(int dim, double h) {
  if (dim == 1) return 2.0 / (3.0 * h);
  if (dim == 2) return 10.0 / (7.0 * ORC_PI * h * h);
  return 1.0 / (ORC_PI * h * h * h);
}

/* Wendland C2 (Dehnen & Aly 2012), used by the paper with radius kappa = 1.936
 * (Sec. 4.1): W = n_D / H^D * (1-s)^4 (1+4s) for D = 2, 3 and
 * n_1 / H * (1-s)^3 (1+3s) for D = 1, with s = r/H and H = kappa h.
 * n_1 = 5/4, n_2 = 7/pi, n_3 = 21/(2 pi). */
static double wendland_norm(int dim, double H) {
  if (dim == 1) return 1.25 / H;
  if (dim == 2) return 7.0 / (ORC_PI * H * H);
  return 21.0 / (2.0 * ORC_PI * H * H * H);
}

double orc_kernel_w(int kernel, int dim, double kappa, double r, double h) {
  if (kernel == ORC_KERNEL_CUBIC) {
    double q = r / h;
    double sig = cubic_norm(dim, h);
    if (q < 1.0) return sig * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
    if (q < 2.0) { double t = 2.0 - q; return sig * 0.25 * t * t * t; }
    return 0.0;
  } else {
    double H = kappa * h;
    double s = r / H;
    if (s >= 1.0) return 0.0;
    double t = 1.0 - s;
    if (dim == 1) return wendland_norm(1, H) * t * t * t * (1.0 + 3.0 * s);
    return wendland_norm(dim, H) * t * t * t * t * (1.0 + 4.0 * s);
  }
}

double orc_kernel_dw(int kernel, int dim, double kappa, double r, double h) {
  if (kernel == ORC_KERNEL_CUBIC) {
    double q = r / h;
    double sig = cubic_norm(dim, h) / h;
    if (q < 1.0) return sig * (-3.0 * q + 2.25 * q * q);
    if (q < 2.0) { double t = 2.0 - q; return sig * (-0.75 * t * t); }
    return 0.0;
  } else {
    double H = kappa * h;
    double s = r / H;
    if (s >= 1.0) return 0.0;
    double t = 1.0 - s;
    /* d/ds[(1-s)^4 (1+4s)] = -20 s (1-s)^3 ; d/ds[(1-s)^3 (1+3s)] = -12 s (1-s)^2 */
    if (dim == 1) return wendland_norm(1, H) / H * (-12.0 * s * t * t);
    return wendland_norm(dim, H) / H * (-20.0 * s * t * t * t);
  }
}

/* ------------------------------------------------------------------------ */
/* Equations of state.  Ideal gas, stiffened gas and Tait are the closures of
 * the synthetic workloads; Mie-Grueneisen with the linear u_s-u_p Hugoniot is
 * eqs. (mie_gruneisen_eos), (mie_gruneisen_reference) of Sec. 7.            */
/* ------------------------------------------------------------------------ */
int orc_eos(const orc_material* mat, double rho, double e, double* P, double* c) {
  double p, c2;
  switch (mat->eos) {
    case ORC_EOS_IDEAL:
      p = (mat->gamma - 1.0) * rho * e;
      c2 = mat->gamma * p / rho;
      break;
    case ORC_EOS_STIFFENED:
      p = (mat->gamma - 1.0) * rho * e - mat->gamma * mat->p_inf;
      c2 = mat->gamma * (p + mat->p_inf) / rho;
      break;
    case ORC_EOS_TAIT: {
      double B = mat->rho0 * mat->c0 * mat->c0 / mat->gamma;
      double r = rho / mat->rho0;
      p = B * (pow(r, mat->gamma) - 1.0);
      c2 = mat->c0 * mat->c0 * pow(r, mat->gamma - 1.0);
      break;
    }
    case ORC_EOS_MIE_GRUNEISEN: {
      /* x = rho0/rho; P = P_r(x) + Gamma rho (e - e_r(x));
       * P_r = rho0 ca^2 (1-x)/[1 - sa(1-x)]^2, e_r = ca^2/2 (1-x)^2/[1 - sa(1-x)]^2.
       * c^2 = dP/drho|_e + (P/rho^2) dP/de|_rho, with dP/de|_rho = Gamma rho. */
      double G = mat->gamma, ca = mat->c0, sa = mat->s_a;
      double x = mat->rho0 / rho;
      double u = 1.0 - x;                 /* compression 1 - x */
      double D = 1.0 - sa * u;
      double Pr = mat->rho0 * ca * ca * u / (D * D);
      double er = 0.5 * ca * ca * u * u / (D * D);
      double du_drho = x / rho;           /* d(1-x)/drho */
      double dPr = mat->rho0 * ca * ca * (1.0 + sa * u) / (D * D * D) * du_drho;
      double der = ca * ca * u / (D * D * D) * du_drho;
      p = Pr + G * rho * (e - er);
      c2 = dPr + G * (e - er) - G * rho * der + G * p / rho;
      break;
    }
    default:
      p = NAN; c2 = NAN;
  }
  *P = p;
  if (c2 < 0.0) { *c = 0.0; return 1; }
  *c = sqrt(c2);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Pair Riemann solver.  Sec. 4.1 uses "the Riemann solver" of the cited CSPH
 * scheme between the left state i and right state j along e^R = (r_j - r_i)/|..|.
 * Reading: the linearised (acoustic) solution of that Riemann problem with
 * impedances Z = rho c:  the contact pressure and velocity satisfy
 *   P* - P_i = -Z_i (v* - v_i^R)   (left-facing wave)
 *   P* - P_j = +Z_j (v* - v_j^R)   (right-facing wave).                     */
/* ------------------------------------------------------------------------ */
void orc_riemann_acoustic(double Pi, double Pj, double Zi, double Zj, double vRi, double vRj,
                          double* Pstar, double* vstar) {
  double zs = Zi + Zj;
  *Pstar = (Zj * Pi + Zi * Pj + Zi * Zj * (vRi - vRj)) / zs;
  *vstar = (Zi * vRi + Zj * vRj + Pi - Pj) / zs;
}

/* Alternative pair solver ("acoustic/HLL" in the specification of the
 * workloads; Sec. 4.1 names no solver form).  Reading: the two-wave HLL
 * state of the linearised Lagrangian acoustic system, d v/dt + dP/dm = 0,
 * dP/dt + C^2 dv/dm = 0 along e^R, with the Davis wave-speed estimate
 * S_L = -C, S_R = +C, C = max(Z_i, Z_j):
 *   P* = (P_i + P_j)/2 + C (v_i^R - v_j^R)/2,
 *   v* = (v_i^R + v_j^R)/2 + (P_i - P_j) / (2 C).
 * Equal impedances give the acoustic solution; otherwise it is the more
 * dissipative of the two.  Exchange-symmetric like the acoustic form.       */
void orc_riemann_hll(double Pi, double Pj, double Zi, double Zj, double vRi, double vRj,
                     double* Pstar, double* vstar) {
  double C = Zi > Zj ? Zi : Zj;
  *Pstar = 0.5 * (Pi + Pj) + 0.5 * C * (vRi - vRj);
  *vstar = 0.5 * (vRi + vRj) + (Pi - Pj) / (2.0 * C);
}

/* ------------------------------------------------------------------------ */
/* Derived per-particle quantities: e = E - v^2/2 (Sec. 4.1, below
 * eq. SPH:Energy), P and c from the EOS, d = (m/rho)^(1/dim)
 * (eq. SmoothingLengthDef uses the cube root in 3D).                         */
/* ------------------------------------------------------------------------ */
int64_t orc_derive(const orc_params* p, orc_state* s) {
  int64_t bad = 0;
  for (int64_t i = 0; i < s->n; ++i) {
    double vx = get(s->vx, i), vy = get(s->vy, i), vz = get(s->vz, i);
    double e = s->E[i] - 0.5 * (vx * vx + vy * vy + vz * vz);
    int mi = s->mat ? s->mat[i] : 0;
    bad += orc_eos(&p->mat[mi], s->rho[i], e, &s->P[i], &s->c[i]);
    double vol = s->m[i] / s->rho[i];
    if (p->dim == 1) s->d[i] = vol;
    else if (p->dim == 2) s->d[i] = sqrt(vol);
    else s->d[i] = cbrt(vol);
  }
  return bad;
}

/* CFL time step: dt = cfl * min_i (eta d_i) / (c_i + |v_i|).  Uses s->d, s->c. */
double orc_dt(const orc_params* p, const orc_state* s) {
  double best = INFINITY;
  for (int64_t i = 0; i < s->n; ++i) {
    double vx = get(s->vx, i), vy = get(s->vy, i), vz = get(s->vz, i);
    double vmag = sqrt(vx * vx + vy * vy + vz * vz);
    double dti = (p->eta * s->d[i]) / (s->c[i] + vmag);
    if (dti < best) best = dti;
  }
  return p->cfl * best;
}

/* ------------------------------------------------------------------------ */
/* Neighbour search (Sec. 4.2).                                             */
/* ------------------------------------------------------------------------ */

/* Interaction test.  The pair {i, j} interacts when r_ij < kappa h_ij with
 * h_ij = eta (d_i + d_j)/2 (eq. SmoothingLengthDef and the support statement
 * below it).  Written as r^2 < R^2 with R = (0.5 kappa eta)(d_i + d_j); the
 * operation order is fixed so that the decision is reproducible bit for bit. */
static double kh_of(const orc_params* p) { return (0.5 * p->kappa) * p->eta; }

static int pair_accept(const orc_params* p, const orc_state* s, double kh, int64_t i, int64_t j) {
  double dx = s->x[j] - s->x[i];
  double r2 = dx * dx;
  if (p->dim >= 2) { double dy = s->y[j] - s->y[i]; r2 = r2 + dy * dy; }
  if (p->dim >= 3) { double dz = s->z[j] - s->z[i]; r2 = r2 + dz * dz; }
  double R = kh * (s->d[i] + s->d[j]);
  return r2 < R * R;
}

/* All unordered pairs i < j by direct O(N^2) search (Sec. 4.2, first paragraph). */
int64_t orc_pairs_brute(const orc_params* p, const orc_state* s, int64_t cap, int32_t* pi, int32_t* pj) {
  double kh = kh_of(p);
  int64_t np = 0;
  for (int64_t i = 0; i < s->n; ++i)
    for (int64_t j = i + 1; j < s->n; ++j)
      if (pair_accept(p, s, kh, i, j)) {
        if (np < cap) { pi[np] = (int32_t)i; pj[np] = (int32_t)j; }
        ++np;
      }
  return np;
}

/* Dense cell mesh of eq. (Dcell): D^c = 1/2 (1 + beta) kappa (d1 + d2) with d1,
 * d2 the two largest particle sizes (here with the factor eta of h_ij and a
 * relative safety margin of 2^-20 so that rounding in the cell index can never
 * separate an interacting pair by two cells).  The origin is the componentwise
 * minimum of the positions.  If the mesh would exceed cell_cap cells, D^c is
 * doubled until it fits (a larger cell still holds every neighbour in the
 * 3^dim block B_i).  Cell index per axis: floor((x - x0) / D^c), computed as a
 * product with 1/D^c; linear index cx + nx (cy + ny cz). */
int orc_cell_grid(const orc_params* p, const orc_state* s, orc_grid* g, int64_t* cell_of) {
  const double* X[3] = {s->x, s->y, s->z};
  double xmax[3] = {0, 0, 0};
  for (int a = 0; a < 3; ++a) { g->x0[a] = 0.0; g->dims[a] = 1; }
  g->ncells = 0;
  if (s->n == 0) return 0;
  for (int a = 0; a < p->dim; ++a) {
    g->x0[a] = INFINITY; xmax[a] = -INFINITY;
    for (int64_t i = 0; i < s->n; ++i) {
      if (X[a][i] < g->x0[a]) g->x0[a] = X[a][i];
      if (X[a][i] > xmax[a]) xmax[a] = X[a][i];
    }
  }
  double d1 = 0.0, d2 = 0.0;
  for (int64_t i = 0; i < s->n; ++i) {
    double d = s->d[i];
    if (d > d1) { d2 = d1; d1 = d; }
    else if (d > d2) d2 = d;
  }
  if (s->n < 2) d2 = d1;
  double dc = kh_of(p) * (d1 + d2);
  dc = dc * (1.0 + p->cell_beta);
  dc = dc * (1.0 + 0x1p-20);
  if (!(dc > 0.0) || !isfinite(dc)) return -1;
  for (;;) {
    double inv = 1.0 / dc;
    int64_t tot = 1;
    for (int a = 0; a < 3; ++a) {
      g->dims[a] = (a < p->dim) ? (int64_t)floor((xmax[a] - g->x0[a]) * inv) + 1 : 1;
      tot *= g->dims[a];
    }
    if (tot <= p->cell_cap) { g->dc = dc; g->inv_dc = inv; g->ncells = tot; break; }
    dc = dc * 2.0;
  }
  if (cell_of) {
    for (int64_t i = 0; i < s->n; ++i) {
      int64_t c[3] = {0, 0, 0};
      for (int a = 0; a < p->dim; ++a) c[a] = (int64_t)floor((X[a][i] - g->x0[a]) * g->inv_dc);
      cell_of[i] = c[0] + g->dims[0] * (c[1] + g->dims[1] * c[2]);
    }
  }
  return 0;
}

/* Pair search through the cell mesh and a linked list (Sec. 4.2: head array
 * over the mesh, "next" vector over particles, 0-terminated chains; here -1
 * terminated).  Each particle scans the 3^dim cells of its block B_i; the
 * pair is kept from the lower index only. */
int64_t orc_pairs_cells(const orc_params* p, const orc_state* s, int64_t cap, int32_t* pi, int32_t* pj) {
  orc_grid g;
  if (s->n == 0) return 0;
  int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)s->n);
  if (orc_cell_grid(p, s, &g, cell) != 0) { free(cell); return -1; }
  int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)g.ncells);
  int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)s->n);
  for (int64_t c = 0; c < g.ncells; ++c) head[c] = -1;
  for (int64_t i = s->n - 1; i >= 0; --i) { next[i] = head[cell[i]]; head[cell[i]] = i; }
  double kh = kh_of(p);
  int64_t np = 0;
  int64_t nx = g.dims[0], ny = g.dims[1], nz = g.dims[2];
  for (int64_t i = 0; i < s->n; ++i) {
    int64_t ci = cell[i];
    int64_t cx = ci % nx, cy = (ci / nx) % ny, cz = ci / (nx * ny);
    for (int64_t oz = -1; oz <= 1; ++oz) {
      int64_t z = cz + oz; if (z < 0 || z >= nz) continue;
      for (int64_t oy = -1; oy <= 1; ++oy) {
        int64_t y = cy + oy; if (y < 0 || y >= ny) continue;
        for (int64_t ox = -1; ox <= 1; ++ox) {
          int64_t x = cx + ox; if (x < 0 || x >= nx) continue;
          for (int64_t j = head[x + nx * (y + ny * z)]; j >= 0; j = next[j]) {
            if (j <= i) continue;
            if (pair_accept(p, s, kh, i, j)) {
              if (np < cap) { pi[np] = (int32_t)i; pj[np] = (int32_t)j; }
              ++np;
            }
          }
        }
      }
    }
  }
  free(cell); free(head); free(next);
  return np;
}

/* ------------------------------------------------------------------------ */
/* CSPH rates over a pair list: eqs. (SPH:Conti), (SPH:Pulse), (SPH:Energy)
 * with e^R = (r_j - r_i)/|r_j - r_i|, v^R = v . e^R and
 * grad_i W_ij = -e^R W'_ij (Sec. 4.1).  Each pair contributes to both
 * particles; from j's side e^R flips sign, so v*^R flips and P* is unchanged. */
/* ------------------------------------------------------------------------ */
/* Second-order variant (order = 2).  Sec. 4.1 feeds the particle values
 * v_i^R, v_j^R (and P_i, P_j) to the Riemann solver; the cited CSPH scheme
 * may instead reconstruct the states at the contact point between the two
 * particles, and the paper gives no formula for it.  Reading used here:
 *  - SPH gradients of P and of the velocity over the same pair set, h_ij and
 *    W' as the rates:  grad q_i = sum_j V_j (q_j - q_i) (-W'_ij) e^R_ij
 *    (exact for a linear field when the kernel is normalised);
 *  - linear extrapolation of P and v^R from each particle to the pair
 *    midpoint, each increment limited by minmod against the pair jump:
 *      q_L = q_i + 1/2 minmod(r e.grad q_i, q_j - q_i)
 *      q_R = q_j - 1/2 minmod(r e.grad q_j, q_j - q_i)
 *    with e.grad v^R = e . (grad v) . e; so q_i <= q_L <= q_R <= q_j (or the
 *    reverse) and a linear field gives q_L = q_R = its midpoint value;
 *  - the acoustic solver on (P_L, v_L; P_R, v_R) with the particles' Z.
 * The reconstruction is exchange-symmetric (from j's side e^R flips and L, R
 * swap), so the fluxes keep their antisymmetry.                              */
static double minmod(double a, double b) {
  if (a > 0.0 && b > 0.0) return a < b ? a : b;
  if (a < 0.0 && b < 0.0) return a > b ? a : b;
  return 0.0;
}

/* grad P (3 per particle) and grad v (9 per particle, [a][b] = d v_a / d x_b). */
void orc_pair_gradients(const orc_params* p, const orc_state* s, int64_t npairs, const int32_t* pi,
                           const int32_t* pj, double* gP, double* gV) {
  for (int64_t i = 0; i < 3 * s->n; ++i) gP[i] = 0.0;
  for (int64_t i = 0; i < 9 * s->n; ++i) gV[i] = 0.0;
  for (int64_t k = 0; k < npairs; ++k) {
    int64_t i = pi[k], j = pj[k];
    double e[3] = {s->x[j] - s->x[i], p->dim >= 2 ? s->y[j] - s->y[i] : 0.0, p->dim >= 3 ? s->z[j] - s->z[i] : 0.0};
    double r = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    if (r == 0.0) continue;
    for (int a = 0; a < 3; ++a) e[a] /= r;
    double hij = p->eta * (s->d[i] + s->d[j]) * 0.5;
    double w = -orc_kernel_dw(p->kernel, p->dim, p->kappa, r, hij);   /* -W' >= 0 */
    double Vi = s->m[i] / s->rho[i], Vj = s->m[j] / s->rho[j];
    double dP = s->P[j] - s->P[i];
    double dv[3] = {get(s->vx, j) - get(s->vx, i), get(s->vy, j) - get(s->vy, i), get(s->vz, j) - get(s->vz, i)};
    /* from j's side both (q_i - q_j) and e^R change sign: the same product */
    for (int b = 0; b < 3; ++b) {
      gP[3 * i + b] += Vj * dP * w * e[b];
      gP[3 * j + b] += Vi * dP * w * e[b];
      for (int a = 0; a < 3; ++a) {
        gV[9 * i + 3 * a + b] += Vj * dv[a] * w * e[b];
        gV[9 * j + 3 * a + b] += Vi * dv[a] * w * e[b];
      }
    }
  }
}

void orc_rates(const orc_params* p, orc_state* s, int64_t npairs, const int32_t* pi, const int32_t* pj) {
  for (int64_t i = 0; i < s->n; ++i) {
    s->drho[i] = 0.0; s->dE[i] = 0.0; s->ax[i] = 0.0;
    if (s->ay) s->ay[i] = 0.0;
    if (s->az) s->az[i] = 0.0;
  }
  double *gP = NULL, *gV = NULL;
  if (p->order == 2) {
    gP = (double*)malloc(sizeof(double) * 3 * (size_t)(s->n > 0 ? s->n : 1));
    gV = (double*)malloc(sizeof(double) * 9 * (size_t)(s->n > 0 ? s->n : 1));
    orc_pair_gradients(p, s, npairs, pi, pj, gP, gV);
  }
  for (int64_t k = 0; k < npairs; ++k) {
    int64_t i = pi[k], j = pj[k];
    double dx = s->x[j] - s->x[i];
    double dy = p->dim >= 2 ? s->y[j] - s->y[i] : 0.0;
    double dz = p->dim >= 3 ? s->z[j] - s->z[i] : 0.0;
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (r == 0.0) continue;  /* coincident particles: e^R undefined, no interaction */
    double ex = dx / r, ey = dy / r, ez = dz / r;
    double vRi = get(s->vx, i) * ex + get(s->vy, i) * ey + get(s->vz, i) * ez;
    double vRj = get(s->vx, j) * ex + get(s->vy, j) * ey + get(s->vz, j) * ez;
    double Zi = s->rho[i] * s->c[i], Zj = s->rho[j] * s->c[j];
    double PL = s->P[i], PR = s->P[j], vL = vRi, vR = vRj;
    if (p->order == 2) {
      const double e[3] = {ex, ey, ez};
      double sPi = 0.0, sPj = 0.0, svi = 0.0, svj = 0.0;
      for (int b = 0; b < 3; ++b) {
        sPi += gP[3 * i + b] * e[b];
        sPj += gP[3 * j + b] * e[b];
        for (int a = 0; a < 3; ++a) {
          svi += e[a] * gV[9 * i + 3 * a + b] * e[b];
          svj += e[a] * gV[9 * j + 3 * a + b] * e[b];
        }
      }
      double dP = s->P[j] - s->P[i], dv = vRj - vRi;
      PL = s->P[i] + 0.5 * minmod(r * sPi, dP);
      PR = s->P[j] - 0.5 * minmod(r * sPj, dP);
      vL = vRi + 0.5 * minmod(r * svi, dv);
      vR = vRj - 0.5 * minmod(r * svj, dv);
    }
    double Ps, vs;
    if (Zi + Zj > 0.0) {
      if (p->solver == ORC_SOLVER_HLL) orc_riemann_hll(PL, PR, Zi, Zj, vL, vR, &Ps, &vs);
      else orc_riemann_acoustic(PL, PR, Zi, Zj, vL, vR, &Ps, &vs);
    }
    else { Ps = 0.5 * (PL + PR); vs = 0.5 * (vL + vR); }
    double hij = p->eta * (s->d[i] + s->d[j]) * 0.5;
    double dW = orc_kernel_dw(p->kernel, p->dim, p->kappa, r, hij);   /* W'_ij <= 0 */
    double Vi = s->m[i] / s->rho[i], Vj = s->m[j] / s->rho[j];
    /* SPH:Conti: drho_i/dt = 2 rho_i sum_j V_j (v_i^R - v*) e.grad_i W, e.grad_i W = -W' */
    s->drho[i] += 2.0 * s->rho[i] * Vj * (vRi - vs) * (-dW);
    s->drho[j] += 2.0 * s->rho[j] * Vi * (vs - vRj) * (-dW);
    /* SPH:Pulse: dv_i/dt = -(2/rho_i) sum_j V_j P* grad_i W = (2/rho_i) sum_j V_j P* W' e */
    double fi = 2.0 / s->rho[i] * Vj * Ps * dW;
    double fj = 2.0 / s->rho[j] * Vi * Ps * dW;
    s->ax[i] += fi * ex; s->ax[j] -= fj * ex;
    if (s->ay) { s->ay[i] += fi * ey; s->ay[j] -= fj * ey; }
    if (s->az) { s->az[i] += fi * ez; s->az[j] -= fj * ez; }
    /* SPH:Energy: dE_i/dt = -(2/rho_i) sum_j V_j P* v* e.grad_i W = (2/rho_i) sum_j V_j P* v* W' */
    s->dE[i] += fi * vs;
    s->dE[j] -= fj * vs;
  }
  free(gP);
  free(gV);
}

/* Derive e, P, c, d, search pairs through cells, evaluate rates. */
int64_t orc_eval_rates(const orc_params* p, orc_state* s) {
  orc_derive(p, s);
  int64_t np = orc_pairs_cells(p, s, 0, NULL, NULL);
  if (np < 0) return np;
  int32_t* pi = (int32_t*)malloc(sizeof(int32_t) * (size_t)(np > 0 ? np : 1));
  int32_t* pj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(np > 0 ? np : 1));
  orc_pairs_cells(p, s, np, pi, pj);
  orc_rates(p, s, np, pi, pj);
  free(pi); free(pj);
  return np;
}

/* ------------------------------------------------------------------------ */
/* Time update.  Alg. 1 only says "renew particle positions and states and
 * make global synchronization of SPH time step"; the integrator is the
 * reading KDK leapfrog with one rate evaluation per step:
 *   dt   = cfl min_i eta d_i/(c_i + |v_i|)              (state n)
 *   q^h  = q^n + dt/2 * dq^n        for q in {v, rho, E}
 *   x'   = x^n + dt * v^h
 *   q~   = q^h + dt/2 * dq^n        (predicted state at n+1)
 *   dq'  = rates(x', v~, rho~, E~)
 *   q'   = q^h + dt/2 * dq'
 * The rates dq' are kept and used as dq^n of the next step.                */
/* ------------------------------------------------------------------------ */
int orc_step(const orc_params* p, orc_state* s, int n_steps, int rates_valid, double* t, double* dt_out) {
  int64_t n = s->n;
  int dim = p->dim;
  if (!rates_valid) { if (orc_eval_rates(p, s) < 0) return -1; }
  size_t bytes = sizeof(double) * (size_t)(n > 0 ? n : 1);
  double *vh[3], *vp[3], *ap[3];
  for (int a = 0; a < 3; ++a) { vh[a] = malloc(bytes); vp[a] = malloc(bytes); ap[a] = malloc(bytes); }
  double *rh = malloc(bytes), *Eh = malloc(bytes), *rp = malloc(bytes), *Ep = malloc(bytes);
  double *drp = malloc(bytes), *dEp = malloc(bytes);
  double *dp = malloc(bytes), *Pp = malloc(bytes), *cp = malloc(bytes);
  double* V[3] = {s->vx, s->vy, s->vz};
  double* X[3] = {s->x, s->y, s->z};
  double* A[3] = {s->ax, s->ay, s->az};
  for (int st = 0; st < n_steps; ++st) {
    orc_derive(p, s);
    double dt = orc_dt(p, s);
    double hdt = 0.5 * dt;
    for (int64_t i = 0; i < n; ++i) {
      for (int a = 0; a < dim; ++a) {
        vh[a][i] = V[a][i] + hdt * A[a][i];
        X[a][i] = X[a][i] + dt * vh[a][i];
        vp[a][i] = vh[a][i] + hdt * A[a][i];
      }
      rh[i] = s->rho[i] + hdt * s->drho[i];
      Eh[i] = s->E[i] + hdt * s->dE[i];
      rp[i] = rh[i] + hdt * s->drho[i];
      Ep[i] = Eh[i] + hdt * s->dE[i];
    }
    orc_state pr;
    memset(&pr, 0, sizeof(pr));
    pr.n = n; pr.x = s->x; pr.y = s->y; pr.z = s->z;
    pr.vx = vp[0]; pr.vy = dim >= 2 ? vp[1] : NULL; pr.vz = dim >= 3 ? vp[2] : NULL;
    pr.rho = rp; pr.E = Ep; pr.m = s->m; pr.mat = s->mat;
    pr.ax = ap[0]; pr.ay = dim >= 2 ? ap[1] : NULL; pr.az = dim >= 3 ? ap[2] : NULL;
    pr.drho = drp; pr.dE = dEp; pr.d = dp; pr.P = Pp; pr.c = cp;
    if (orc_eval_rates(p, &pr) < 0) return -1;
    for (int64_t i = 0; i < n; ++i) {
      for (int a = 0; a < dim; ++a) {
        V[a][i] = vh[a][i] + hdt * ap[a][i];
        A[a][i] = ap[a][i];
      }
      s->rho[i] = rh[i] + hdt * drp[i];
      s->E[i] = Eh[i] + hdt * dEp[i];
      s->drho[i] = drp[i];
      s->dE[i] = dEp[i];
      s->d[i] = dp[i]; s->P[i] = Pp[i]; s->c[i] = cp[i];
    }
    if (t) *t += dt;
    if (dt_out) dt_out[st] = dt;
  }
  for (int a = 0; a < 3; ++a) { free(vh[a]); free(vp[a]); free(ap[a]); }
  free(rh); free(Eh); free(rp); free(Ep); free(drp); free(dEp); free(dp); free(Pp); free(cp);
  return 0;
}

/* FP64 sums of mass, momentum and total energy m E, in index order. */
void orc_conservation(const orc_state* s, double out5[5]) {
  for (int a = 0; a < 5; ++a) out5[a] = 0.0;
  for (int64_t i = 0; i < s->n; ++i) {
    double m = s->m[i];
    out5[0] += m;
    out5[1] += m * get(s->vx, i);
    out5[2] += m * get(s->vy, i);
    out5[3] += m * get(s->vz, i);
    out5[4] += m * s->E[i];
  }
}

/* ------------------------------------------------------------------------ */
/* Voronoi assignment, eq. (VoronoiDefinition) with the tie rule of Sec. 3.1:
 * a particle at equal distance from several generators belongs to the one of
 * smallest index.  Squared distance in the first gdim coordinates, summed in
 * axis order. */
/* ------------------------------------------------------------------------ */
void orc_voronoi_assign(int64_t n, int dim, const double* x, const double* y, const double* z,
                        int K, const double* gen, int32_t* unit) {
  for (int64_t i = 0; i < n; ++i) {
    int best = 0;
    double bd = INFINITY;
    for (int k = 0; k < K; ++k) {
      double dx = x[i] - gen[k * dim + 0];
      double d2 = dx * dx;
      if (dim >= 2) { double dy = y[i] - gen[k * dim + 1]; d2 = d2 + dy * dy; }
      if (dim >= 3) { double dz = z[i] - gen[k * dim + 2]; d2 = d2 + dz * dz; }
      if (d2 < bd) { bd = d2; best = k; }
    }
    unit[i] = best;
  }
}

/* ------------------------------------------------------------------------ */
/* Per-unit statistics for the balancing step (Alg. 1, Secs. 3.2, 4.2, 4.3):
 *  load[k]   L_k = number of interacting pairs handled by unit k, a pair
 *            that crosses units counting 1/2 to each (the interaction-count
 *            load named in the introduction as an alternative to timing);
 *  adj[k,l]  1 when some interacting pair joins a particle of k and one of l;
 *  dsh[k,l]  eq. (Horizon): max(max_{i in k} R^hrz_i, max_{i in l} R^hrz_i),
 *            R^hrz_i = (1 + beta) R^int_i,
 *            R^int_i = 1/2 kappa eta (d_i + max_{j neighbour of i} d_j);
 *            an isolated particle takes its own d as the neighbour maximum;
 *  centroid  eq. (VoronoiGeomCenters) over the current particle positions
 *            (r_c,k + Delta r_c,k of eq. TotalOffset);
 *  count[k]  N_k.                                                            */
/* ------------------------------------------------------------------------ */
int orc_unit_stats(const orc_params* p, const orc_state* s, const int32_t* unit, int K, int gdim,
                   int64_t npairs, const int32_t* pi, const int32_t* pj, double beta,
                   double* load, uint8_t* adj, double* dsh, double* centroid, int64_t* count) {
  const double* X[3] = {s->x, s->y, s->z};
  double kh = kh_of(p);
  double* dmax = (double*)malloc(sizeof(double) * (size_t)(s->n > 0 ? s->n : 1));
  double* rmax = (double*)calloc((size_t)K, sizeof(double));
  for (int k = 0; k < K; ++k) {
    load[k] = 0.0; count[k] = 0;
    for (int a = 0; a < gdim; ++a) centroid[k * gdim + a] = 0.0;
    for (int l = 0; l < K; ++l) { adj[k * K + l] = 0; dsh[k * K + l] = 0.0; }
  }
  for (int64_t i = 0; i < s->n; ++i) dmax[i] = -1.0;
  for (int64_t q = 0; q < npairs; ++q) {
    int64_t i = pi[q], j = pj[q];
    int ui = unit[i], uj = unit[j];
    load[ui] += 0.5; load[uj] += 0.5;
    if (ui != uj) { adj[ui * K + uj] = 1; adj[uj * K + ui] = 1; }
    if (s->d[j] > dmax[i]) dmax[i] = s->d[j];
    if (s->d[i] > dmax[j]) dmax[j] = s->d[i];
  }
  for (int64_t i = 0; i < s->n; ++i) {
    int u = unit[i];
    double dm = dmax[i] < 0.0 ? s->d[i] : dmax[i];
    double rhrz = (1.0 + beta) * (kh * (s->d[i] + dm));
    if (rhrz > rmax[u]) rmax[u] = rhrz;
    count[u] += 1;
    for (int a = 0; a < gdim; ++a) centroid[u * gdim + a] += X[a][i];
  }
  for (int k = 0; k < K; ++k) {
    if (count[k] > 0)
      for (int a = 0; a < gdim; ++a) centroid[k * gdim + a] /= (double)count[k];
    for (int l = 0; l < K; ++l) dsh[k * K + l] = rmax[k] > rmax[l] ? rmax[k] : rmax[l];
  }
  free(dmax); free(rmax);
  return 0;
}

/* Rotation of v about the axis a by the angle alpha (right-handed, Rodrigues).
 * A zero axis leaves v unchanged. */
static void rotate3(const double a[3], double alpha, const double v[3], double out[3]) {
  double na = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  if (na == 0.0) { out[0] = v[0]; out[1] = v[1]; out[2] = v[2]; return; }
  double u[3] = {a[0] / na, a[1] / na, a[2] / na};
  double c = cos(alpha), sn = sin(alpha);
  double uxv[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
  double udv = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
  for (int q = 0; q < 3; ++q) out[q] = v[q] * c + uxv[q] * sn + u[q] * udv * (1.0 - c);
}

static void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------ */
/* One balancing update of all generators (Secs. 3.2-3.4):
 *   two-body   eq. (BalancingOffset):
 *              dg2_k = sum_{l~k} Dsh_kl (L_k - L_l)/(L_k + L_l) g_kl/|g_kl|,
 *              g_kl = g_k - g_l;
 *   three-body eq. (BalancingOffsetRot), 2D only:
 *              dg_klm = -c_k + M(c_k x c_m, a_m) M(c_k x c_l, a_l) c_k,
 *              c_p = g_p - o_klm, o_klm the circumcentre of g_k, g_l, g_m,
 *              a_l = pi/3 (L_l - L_k)/(L_k + L_l + L_m), same for a_m,
 *              summed over each triangle of mutually adjacent units once, and
 *              the sum limited in length to max_l Dsh_kl;
 *   combined   eq. (BalancingOffsetPlusRot): dg = (1 - sigma) dg2 + sigma dg3;
 *   cumulative eq. (TotalOffset):
 *              g^_k = (1 - theta)(g_k + gamma dg_k) + theta (r_c,k + dr_c,k),
 *              the last term the current centroid (g_k for an empty unit).
 * Returns sum_k |g^_k - g_k| (eq. VDConvergence).  gen is updated in place. */
/* ------------------------------------------------------------------------ */
/* Four-body term for 3D decompositions (Sec. 3.3 names it, "a rotation on
 * the circumsphere of four generators", without a formula).  Reading: for
 * each set {k, l, m, n} of mutually adjacent units (each once per k,
 * l < m < n) with o the centre of the sphere through g_k, g_l, g_m, g_n,
 *   dg_klmn = -c_k + M(w, |w|) c_k,  w = sum_{p = l, m, n} a_p unit(c_k x c_p),
 *   c_p = g_p - o,  a_p = (T/2) (L_p - L_k) / (L_k + L_l + L_m + L_n),
 * T = arccos(-1/3), the angle between the generators of a regular
 * tetrahedron seen from its centre: the 2D form's pi/3 is half of the 120
 * degrees of three subdomains around a point.  One rotation about the summed
 * rotation vector: in 2D all the axes are the plane normal and this is the
 * product of the paper's rotations; in 3D rotations do not commute, and a
 * product would depend on the labels of l, m, n.  The rotation keeps |c_k|,
 * so the generator stays on the sphere and o stays the common point; the
 * summed term is length-limited like the 2D one.  Skipped when the four
 * generators are (nearly) coplanar. */
static void four_body(const double gk[3], const double gl[3], const double gm[3], const double gn[3],
                      double Lk, double Ll, double Lm, double Ln, double dg[3]) {
  double a[3], b[3], c[3];
  for (int q = 0; q < 3; ++q) { a[q] = gl[q] - gk[q]; b[q] = gm[q] - gk[q]; c[q] = gn[q] - gk[q]; }
  double bc[3], ca[3], ab[3];
  cross3(b, c, bc);
  cross3(c, a, ca);
  cross3(a, b, ab);
  double det = a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2];
  double a2 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
  double b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  double c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
  double s2 = a2 > b2 ? a2 : b2;
  s2 = s2 > c2 ? s2 : c2;
  if (fabs(det) < 1e-12 * s2 * sqrt(s2)) return;        /* coplanar: no circumsphere */
  double Ls = Lk + Ll + Lm + Ln;
  if (!(Ls > 0.0)) return;
  double o[3];
  for (int q = 0; q < 3; ++q) o[q] = gk[q] + (a2 * bc[q] + b2 * ca[q] + c2 * ab[q]) / (2.0 * det);
  double half_t = 0.5 * acos(-1.0 / 3.0);
  double al = half_t * (Ll - Lk) / Ls, am = half_t * (Lm - Lk) / Ls, an = half_t * (Ln - Lk) / Ls;
  double ck[3], cl[3], cm[3], cn[3];
  for (int q = 0; q < 3; ++q) { ck[q] = gk[q] - o[q]; cl[q] = gl[q] - o[q]; cm[q] = gm[q] - o[q]; cn[q] = gn[q] - o[q]; }
  const double* cp[3] = {cl, cm, cn};
  const double ap[3] = {al, am, an};
  double w[3] = {0.0, 0.0, 0.0};
  for (int t = 0; t < 3; ++t) {
    double ax[3];
    cross3(ck, cp[t], ax);
    double na = sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
    if (na == 0.0) continue;
    for (int q = 0; q < 3; ++q) w[q] += ap[t] * ax[q] / na;
  }
  double nw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  if (nw == 0.0) return;
  double r[3];
  rotate3(w, nw, ck, r);
  for (int q = 0; q < 3; ++q) dg[q] += r[q] - ck[q];
}

double orc_balance(int K, int gdim, double* gen, const double* load, const uint8_t* adj,
                   const double* dsh, const double* centroid, const int64_t* count,
                   double theta, double sigma, double gamma_b, double* dg_out) {
  double sig = (gdim >= 2) ? sigma : 0.0;   /* three-body terms in 2D, four-body terms in 3D */
  double* newg = (double*)malloc(sizeof(double) * (size_t)K * (size_t)gdim);
  double shift = 0.0;
  for (int k = 0; k < K; ++k) {
    double gk[3] = {0, 0, 0};
    for (int a = 0; a < gdim; ++a) gk[a] = gen[k * gdim + a];
    double dg2[3] = {0, 0, 0}, dg3[3] = {0, 0, 0};
    double maxd = 0.0;
    for (int l = 0; l < K; ++l) {
      if (l == k || !adj[k * K + l]) continue;
      if (dsh[k * K + l] > maxd) maxd = dsh[k * K + l];
      double den = load[k] + load[l];
      if (!(den > 0.0)) continue;
      double gkl[3] = {0, 0, 0};
      for (int a = 0; a < gdim; ++a) gkl[a] = gk[a] - gen[l * gdim + a];
      double nrm = sqrt(gkl[0] * gkl[0] + gkl[1] * gkl[1] + gkl[2] * gkl[2]);
      if (nrm == 0.0) continue;
      double f = dsh[k * K + l] * ((load[k] - load[l]) / den) / nrm;
      for (int a = 0; a < 3; ++a) dg2[a] += f * gkl[a];
    }
    if (sig != 0.0 && gdim == 3) {
      for (int l = 0; l < K; ++l) {
        if (l == k || !adj[k * K + l]) continue;
        for (int m = l + 1; m < K; ++m) {
          if (m == k || !adj[k * K + m] || !adj[l * K + m]) continue;
          for (int n4 = m + 1; n4 < K; ++n4) {
            if (n4 == k || !adj[k * K + n4] || !adj[l * K + n4] || !adj[m * K + n4]) continue;
            four_body(gk, &gen[l * 3], &gen[m * 3], &gen[n4 * 3], load[k], load[l], load[m], load[n4], dg3);
          }
        }
      }
      double n3 = sqrt(dg3[0] * dg3[0] + dg3[1] * dg3[1] + dg3[2] * dg3[2]);
      if (n3 > maxd && n3 > 0.0) {
        double f = maxd / n3;
        for (int a = 0; a < 3; ++a) dg3[a] *= f;
      }
    } else if (sig != 0.0) {
      for (int l = 0; l < K; ++l) {
        if (l == k || !adj[k * K + l]) continue;
        for (int m = l + 1; m < K; ++m) {
          if (m == k || !adj[k * K + m] || !adj[l * K + m]) continue;
          double gl[3] = {gen[l * gdim], gen[l * gdim + 1], 0.0};
          double gm[3] = {gen[m * gdim], gen[m * gdim + 1], 0.0};
          double ax = gl[0] - gk[0], ay = gl[1] - gk[1];
          double bx = gm[0] - gk[0], by = gm[1] - gk[1];
          double a2 = ax * ax + ay * ay, b2 = bx * bx + by * by;
          double crs = ax * by - ay * bx;
          double scale2 = a2 > b2 ? a2 : b2;
          if (fabs(crs) < 1e-12 * scale2) continue;     /* collinear: no circumcircle */
          double D = 2.0 * crs;
          double ox = gk[0] + (by * a2 - ay * b2) / D;
          double oy = gk[1] + (ax * b2 - bx * a2) / D;
          double Ls = load[k] + load[l] + load[m];
          if (!(Ls > 0.0)) continue;
          double al = ORC_PI / 3.0 * (load[l] - load[k]) / Ls;
          double am = ORC_PI / 3.0 * (load[m] - load[k]) / Ls;
          double ck[3] = {gk[0] - ox, gk[1] - oy, 0.0};
          double cl[3] = {gl[0] - ox, gl[1] - oy, 0.0};
          double cm[3] = {gm[0] - ox, gm[1] - oy, 0.0};
          double axl[3], axm[3], r1[3], r2[3];
          cross3(ck, cl, axl);
          cross3(ck, cm, axm);
          rotate3(axl, al, ck, r1);
          rotate3(axm, am, r1, r2);
          for (int a = 0; a < 3; ++a) dg3[a] += r2[a] - ck[a];
        }
      }
      double n3 = sqrt(dg3[0] * dg3[0] + dg3[1] * dg3[1] + dg3[2] * dg3[2]);
      if (n3 > maxd && n3 > 0.0) {
        double f = maxd / n3;
        for (int a = 0; a < 3; ++a) dg3[a] *= f;
      }
    }
    double dg[3];
    for (int a = 0; a < 3; ++a) dg[a] = (1.0 - sig) * dg2[a] + sig * dg3[a];
    double dist2 = 0.0;
    for (int a = 0; a < gdim; ++a) {
      double rc = count[k] > 0 ? centroid[k * gdim + a] : gk[a];
      double ng = (1.0 - theta) * (gk[a] + gamma_b * dg[a]) + theta * rc;
      newg[k * gdim + a] = ng;
      if (dg_out) dg_out[k * gdim + a] = dg[a];
      dist2 += (ng - gk[a]) * (ng - gk[a]);
    }
    shift += sqrt(dist2);
  }
  memcpy(gen, newg, sizeof(double) * (size_t)K * (size_t)gdim);
  free(newg);
  return shift;
}

/* ------------------------------------------------------------------------ */
/* Reverse mode (adjoint) of the CSPH step, written by hand from the
 * formulas above.  Readings: the pair set and the dt sequence of the
 * forward run are held fixed (dt is a stop-gradient); the cubic-spline W'
 * and W'' vanish at q = 2, so the gradient is continuous when pairs enter or
 * leave.  Supported closures: cubic-spline kernel; ideal and stiffened gas,
 * the parameters being (c0, gamma) of material 0 with P_inf = rho0 c0^2 / gamma
 * for the stiffened gas.                                                   */
/* ------------------------------------------------------------------------ */

/* cubic spline: W' = s h^-(D+1) g(q), dW'/dr = s h^-(D+2) g'(q),
 * dW'/dh = s h^-(D+2) (-(D+1) g(q) - q g'(q)), s = 2/3, 10/(7 pi), 1/pi */
static void cubic_dw_derivs(int dim, double r, double h, double* dw, double* dwdr, double* dwdh) {
  double s = dim == 1 ? 2.0 / 3.0 : (dim == 2 ? 10.0 / (7.0 * ORC_PI) : 1.0 / ORC_PI);
  double q = r / h, g, gp;
  if (q < 1.0) { g = -3.0 * q + 2.25 * q * q; gp = -3.0 + 4.5 * q; }
  else if (q < 2.0) { double t = 2.0 - q; g = -0.75 * t * t; gp = 1.5 * t; }
  else { g = 0.0; gp = 0.0; }
  double hp1 = pow(h, (double)(dim + 1));
  *dw = s * g / hp1;
  *dwdr = s * gp / (hp1 * h);
  *dwdh = s * (-(double)(dim + 1) * g - q * gp) / (hp1 * h);
}

/* VJP of orc_rates at the state s (with d, P, c from orc_derive) for the pair
 * list: given ga (3n, dL/da), gr (n, dL/d drho/dt), gE (n, dL/d dE/dt),
 * ADD dL/dx (bx, 3n), dL/dv (bv, 3n), dL/drho (brho), dL/dE (bE) and
 * dL/d(c0, gamma) of material 0 (bpar[2]).  Arrays of dimension 3 use the
 * layout [3*i + a]. */
int orc_rates_vjp(const orc_params* p, const orc_state* s, int64_t npairs, const int32_t* pi, const int32_t* pj,
                  const double* ga, const double* gr, const double* gE,
                  double* bx, double* bv, double* brho, double* bE, double* bpar) {
  if (p->order == 2 || p->solver == ORC_SOLVER_HLL) return -2;   /* first order, acoustic solver only */
  int64_t n = s->n;
  int dim = p->dim;
  if (p->kernel != ORC_KERNEL_CUBIC) return -1;
  for (int k = 0; k < p->n_mat; ++k)
    if (p->mat[k].eos != ORC_EOS_IDEAL && p->mat[k].eos != ORC_EOS_STIFFENED) return -2;
  double* bP = calloc((size_t)n, sizeof(double));
  double* bZ = calloc((size_t)n, sizeof(double));
  double* bV = calloc((size_t)n, sizeof(double));
  double* bd = calloc((size_t)n, sizeof(double));
  const double* X[3] = {s->x, s->y, s->z};
  const double* Vv[3] = {s->vx, s->vy, s->vz};
  for (int64_t k = 0; k < npairs; ++k) {
    int64_t i = pi[k], j = pj[k];
    double dxv[3] = {0, 0, 0}, e[3] = {0, 0, 0}, vi[3] = {0, 0, 0}, vj[3] = {0, 0, 0};
    double r2 = 0.0;
    for (int a = 0; a < dim; ++a) { dxv[a] = X[a][j] - X[a][i]; r2 += dxv[a] * dxv[a]; }
    double r = sqrt(r2);
    if (r == 0.0) continue;
    for (int a = 0; a < dim; ++a) { e[a] = dxv[a] / r; vi[a] = Vv[a][i]; vj[a] = Vv[a][j]; }
    double vRi = 0.0, vRj = 0.0;
    for (int a = 0; a < dim; ++a) { vRi += vi[a] * e[a]; vRj += vj[a] * e[a]; }
    double Zi = s->rho[i] * s->c[i], Zj = s->rho[j] * s->c[j], zs = Zi + Zj;
    double Pi = s->P[i], Pj = s->P[j], Ps, vs;
    if (zs > 0.0) orc_riemann_acoustic(Pi, Pj, Zi, Zj, vRi, vRj, &Ps, &vs);
    else { Ps = 0.5 * (Pi + Pj); vs = 0.5 * (vRi + vRj); }
    double hij = p->eta * (s->d[i] + s->d[j]) * 0.5;
    double W, Wr, Wh;
    cubic_dw_derivs(dim, r, hij, &W, &Wr, &Wh);
    double Vi = s->m[i] / s->rho[i], Vj = s->m[j] / s->rho[j];
    double rhoi = s->rho[i], rhoj = s->rho[j];
    double F = 2.0 * Vi * Vj * Ps * W;
    double dA[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) dA[a] = ga[3 * i + a] / s->m[i] - ga[3 * j + a] / s->m[j];
    double dB = gE[i] / s->m[i] - gE[j] / s->m[j];
    double Ci = gr[i], Cj = gr[j];
    /* outputs of the pair: F e (a), F v* (E), G_i, G_j (rho) */
    double gF = dB * vs, ge[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) { gF += dA[a] * e[a]; ge[a] = F * dA[a]; }
    double gvs = F * dB + 2.0 * W * rhoi * Vj * Ci - 2.0 * W * rhoj * Vi * Cj;
    double gvRi = -2.0 * W * rhoi * Vj * Ci;
    double gvRj = 2.0 * W * rhoj * Vi * Cj;
    double gW = gF * 2.0 * Vi * Vj * Ps - Ci * 2.0 * rhoi * Vj * (vRi - vs) - Cj * 2.0 * rhoj * Vi * (vs - vRj);
    double gPs = gF * 2.0 * Vi * Vj * W;
    bV[i] += gF * 2.0 * Vj * Ps * W + Cj * 2.0 * rhoj * (vs - vRj) * (-W);
    bV[j] += gF * 2.0 * Vi * Ps * W + Ci * 2.0 * rhoi * (vRi - vs) * (-W);
    brho[i] += Ci * 2.0 * Vj * (vRi - vs) * (-W);
    brho[j] += Cj * 2.0 * Vi * (vs - vRj) * (-W);
    /* acoustic solver */
    double gPi, gPj, gZi = 0.0, gZj = 0.0;
    if (zs > 0.0) {
      gPi = gPs * Zj / zs + gvs / zs;
      gPj = gPs * Zi / zs - gvs / zs;
      gvRi += gPs * Zi * Zj / zs + gvs * Zi / zs;
      gvRj += -gPs * Zi * Zj / zs + gvs * Zj / zs;
      gZi = gPs * ((Pj + Zj * (vRi - vRj)) - Ps) / zs + gvs * (vRi - vs) / zs;
      gZj = gPs * ((Pi + Zi * (vRi - vRj)) - Ps) / zs + gvs * (vRj - vs) / zs;
    } else {
      gPi = 0.5 * gPs; gPj = 0.5 * gPs;
      gvRi += 0.5 * gvs; gvRj += 0.5 * gvs;
    }
    bP[i] += gPi; bP[j] += gPj; bZ[i] += gZi; bZ[j] += gZj;
    /* v^R = v . e */
    for (int a = 0; a < dim; ++a) {
      bv[3 * i + a] += gvRi * e[a];
      bv[3 * j + a] += gvRj * e[a];
      ge[a] += gvRi * vi[a] + gvRj * vj[a];
    }
    /* geometry: e = dx / r, W'(r, h_ij), h_ij = eta (d_i + d_j) / 2 */
    double gr_ = gW * Wr;
    double gh = gW * Wh;
    double ede = 0.0;
    for (int a = 0; a < dim; ++a) ede += ge[a] * e[a];
    for (int a = 0; a < dim; ++a) {
      double gdx = (ge[a] - ede * e[a]) / r + gr_ * e[a];
      bx[3 * j + a] += gdx;
      bx[3 * i + a] -= gdx;
    }
    bd[i] += gh * p->eta * 0.5;
    bd[j] += gh * p->eta * 0.5;
  }
  /* per-particle chain: V = m/rho, d = (m/rho)^(1/dim), Z = rho c, EOS, e = E - v^2/2 */
  for (int64_t i = 0; i < n; ++i) {
    const orc_material* mt = &p->mat[s->mat ? s->mat[i] : 0];
    double rho = s->rho[i], c = s->c[i], P = s->P[i];
    double g = mt->gamma, pinf = mt->eos == ORC_EOS_STIFFENED ? mt->p_inf : 0.0;
    double V = s->m[i] / rho;
    brho[i] += bV[i] * (-V / rho);
    brho[i] += bd[i] * (-s->d[i] / ((double)dim * rho));
    brho[i] += bZ[i] * c;
    double bc = bZ[i] * rho;
    double bPi = bP[i], bPinf = 0.0, bg = 0.0;
    if (c > 0.0) {
      double bc2 = bc / (2.0 * c);
      bPi += bc2 * g / rho;
      brho[i] += bc2 * (-c * c / rho);
      bPinf += bc2 * g / rho;
      bg += bc2 * (P + pinf) / rho;
    }
    double v2 = 0.0;
    for (int a = 0; a < dim; ++a) v2 += Vv[a][i] * Vv[a][i];
    double e_int = s->E[i] - 0.5 * v2;
    brho[i] += bPi * (g - 1.0) * e_int;
    double be = bPi * (g - 1.0) * rho;
    bg += bPi * (rho * e_int - pinf);
    bPinf += -g * bPi;
    bE[i] += be;
    for (int a = 0; a < dim; ++a) bv[3 * i + a] -= be * Vv[a][i];
    if ((s->mat ? s->mat[i] : 0) == 0) {
      if (mt->eos == ORC_EOS_STIFFENED) {   /* P_inf = rho0 c0^2 / gamma */
        bpar[0] += bPinf * 2.0 * mt->rho0 * mt->c0 / g;
        bg += bPinf * (-pinf / g);
      }
      bpar[1] += bg;
    }
  }
  free(bP); free(bZ); free(bV); free(bd);
  return 0;
}

/* Forward steps with a prescribed dt sequence (replay of a recorded run). */
int orc_step_replay(const orc_params* p, orc_state* s, int n_steps, int rates_valid, const double* dts) {
  /* identical to orc_step with dt taken from dts */
  orc_params q = *p;
  int64_t n = s->n;
  int dim = p->dim;
  if (!rates_valid) { if (orc_eval_rates(&q, s) < 0) return -1; }
  size_t bytes = sizeof(double) * (size_t)(n > 0 ? n : 1);
  double *vh[3], *vp[3], *ap[3];
  for (int a = 0; a < 3; ++a) { vh[a] = malloc(bytes); vp[a] = malloc(bytes); ap[a] = malloc(bytes); }
  double *rh = malloc(bytes), *Eh = malloc(bytes), *rp = malloc(bytes), *Ep = malloc(bytes);
  double *drp = malloc(bytes), *dEp = malloc(bytes), *dp = malloc(bytes), *Pp = malloc(bytes), *cp = malloc(bytes);
  double* V[3] = {s->vx, s->vy, s->vz};
  double* X[3] = {s->x, s->y, s->z};
  double* A[3] = {s->ax, s->ay, s->az};
  for (int st = 0; st < n_steps; ++st) {
    double dt = dts[st], hdt = 0.5 * dt;
    for (int64_t i = 0; i < n; ++i) {
      for (int a = 0; a < dim; ++a) {
        vh[a][i] = V[a][i] + hdt * A[a][i];
        X[a][i] = X[a][i] + dt * vh[a][i];
        vp[a][i] = vh[a][i] + hdt * A[a][i];
      }
      rh[i] = s->rho[i] + hdt * s->drho[i];
      Eh[i] = s->E[i] + hdt * s->dE[i];
      rp[i] = rh[i] + hdt * s->drho[i];
      Ep[i] = Eh[i] + hdt * s->dE[i];
    }
    orc_state pr;
    memset(&pr, 0, sizeof(pr));
    pr.n = n; pr.x = s->x; pr.y = s->y; pr.z = s->z;
    pr.vx = vp[0]; pr.vy = dim >= 2 ? vp[1] : NULL; pr.vz = dim >= 3 ? vp[2] : NULL;
    pr.rho = rp; pr.E = Ep; pr.m = s->m; pr.mat = s->mat;
    pr.ax = ap[0]; pr.ay = dim >= 2 ? ap[1] : NULL; pr.az = dim >= 3 ? ap[2] : NULL;
    pr.drho = drp; pr.dE = dEp; pr.d = dp; pr.P = Pp; pr.c = cp;
    if (orc_eval_rates(&q, &pr) < 0) return -1;
    for (int64_t i = 0; i < n; ++i) {
      for (int a = 0; a < dim; ++a) { V[a][i] = vh[a][i] + hdt * ap[a][i]; A[a][i] = ap[a][i]; }
      s->rho[i] = rh[i] + hdt * drp[i];
      s->E[i] = Eh[i] + hdt * dEp[i];
      s->drho[i] = drp[i]; s->dE[i] = dEp[i];
      s->d[i] = dp[i]; s->P[i] = Pp[i]; s->c[i] = cp[i];
    }
  }
  for (int a = 0; a < 3; ++a) { free(vh[a]); free(vp[a]); free(ap[a]); }
  free(rh); free(Eh); free(rp); free(Ep); free(drp); free(dEp); free(dp); free(Pp); free(cp);
  return 0;
}

/* VJP of one KDK step (orc_step with the given dt) at the state s (x, v,
 * rho, E and the held rates a, drho, dE; s is not modified).  The adjoint y
 * = (x, v [3n each, layout 3i+a], rho, E, a [3n], drho, dE) of the state
 * after the step is replaced in place by the adjoint of the state before it;
 * bpar (2) accumulates dL/d(c0, gamma). */
int orc_step_vjp(const orc_params* p, const orc_state* s, double dt, double* yx, double* yv, double* yrho,
                 double* yE, double* ya, double* ydrho, double* ydE, double* bpar) {
  if (p->order == 2 || p->solver == ORC_SOLVER_HLL) return -2;   /* first order, acoustic solver only */
  int64_t n = s->n;
  int dim = p->dim;
  double hdt = 0.5 * dt;
  size_t b3 = sizeof(double) * 3 * (size_t)(n > 0 ? n : 1), b1 = sizeof(double) * (size_t)(n > 0 ? n : 1);
  /* predicted state at the end of the drift */
  double *xp[3], *vp[3];
  for (int a = 0; a < 3; ++a) { xp[a] = malloc(b1); vp[a] = malloc(b1); }
  double *rp = malloc(b1), *Ep = malloc(b1), *dp = malloc(b1), *Pp = malloc(b1), *cp = malloc(b1);
  double *apx = malloc(b1), *apy = malloc(b1), *apz = malloc(b1), *drp = malloc(b1), *dEp = malloc(b1);
  const double* X[3] = {s->x, s->y, s->z};
  const double* V[3] = {s->vx, s->vy, s->vz};
  const double* A[3] = {s->ax, s->ay, s->az};
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < 3; ++a) { xp[a][i] = 0.0; vp[a][i] = 0.0; }
    for (int a = 0; a < dim; ++a) {
      double vh = V[a][i] + hdt * A[a][i];
      xp[a][i] = X[a][i] + dt * vh;
      vp[a][i] = vh + hdt * A[a][i];
    }
    double rh = s->rho[i] + hdt * s->drho[i], Eh = s->E[i] + hdt * s->dE[i];
    rp[i] = rh + hdt * s->drho[i];
    Ep[i] = Eh + hdt * s->dE[i];
  }
  orc_state pr;
  memset(&pr, 0, sizeof(pr));
  pr.n = n; pr.x = xp[0]; pr.y = dim >= 2 ? xp[1] : NULL; pr.z = dim >= 3 ? xp[2] : NULL;
  pr.vx = vp[0]; pr.vy = dim >= 2 ? vp[1] : NULL; pr.vz = dim >= 3 ? vp[2] : NULL;
  pr.rho = rp; pr.E = Ep; pr.m = s->m; pr.mat = s->mat;
  pr.ax = apx; pr.ay = apy; pr.az = apz; pr.drho = drp; pr.dE = dEp; pr.d = dp; pr.P = Pp; pr.c = cp;
  orc_derive(p, &pr);
  int64_t np = orc_pairs_cells(p, &pr, 0, NULL, NULL);
  int32_t* pi = malloc(sizeof(int32_t) * (size_t)(np > 0 ? np : 1));
  int32_t* pj = malloc(sizeof(int32_t) * (size_t)(np > 0 ? np : 1));
  orc_pairs_cells(p, &pr, np, pi, pj);
  /* v' = v^h + h a', rho' = rho^h + h drho', E' = E^h + h dE' */
  double *gvh = malloc(b3), *grh = malloc(b1), *gEh = malloc(b1);
  double *ga = malloc(b3), *gr = malloc(b1), *gE = malloc(b1);
  double *bx = calloc(3 * (size_t)n, sizeof(double)), *bv = calloc(3 * (size_t)n, sizeof(double));
  double *bro = calloc((size_t)n, sizeof(double)), *bEE = calloc((size_t)n, sizeof(double));
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < 3; ++a) {
      gvh[3 * i + a] = yv[3 * i + a];
      ga[3 * i + a] = ya[3 * i + a] + hdt * yv[3 * i + a];
    }
    grh[i] = yrho[i]; gr[i] = ydrho[i] + hdt * yrho[i];
    gEh[i] = yE[i]; gE[i] = ydE[i] + hdt * yE[i];
  }
  /* rates at the predicted state */
  int rc = orc_rates_vjp(p, &pr, np, pi, pj, ga, gr, gE, bx, bv, bro, bEE, bpar);
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < dim; ++a) {
      double gxp = yx[3 * i + a] + bx[3 * i + a];       /* x' */
      double gvp = bv[3 * i + a];                        /* v~ */
      double gvha = gvh[3 * i + a] + gvp + dt * gxp;     /* v^h: from v', v~ and x' */
      double gah = hdt * gvp + hdt * gvha;               /* a enters v~ and v^h */
      yx[3 * i + a] = gxp;
      yv[3 * i + a] = gvha;
      ya[3 * i + a] = gah;
    }
    double grp = bro[i], gEp = bEE[i];
    double grha = grh[i] + grp, gEha = gEh[i] + gEp;
    yrho[i] = grha;
    ydrho[i] = hdt * grp + hdt * grha;
    yE[i] = gEha;
    ydE[i] = hdt * gEp + hdt * gEha;
  }
  for (int a = 0; a < 3; ++a) { free(xp[a]); free(vp[a]); }
  free(rp); free(Ep); free(dp); free(Pp); free(cp); free(apx); free(apy); free(apz); free(drp); free(dEp);
  free(pi); free(pj); free(gvh); free(grh); free(gEh); free(ga); free(gr); free(gE);
  free(bx); free(bv); free(bro); free(bEE);
  return rc;
}
