/*
 * csph_oracle.h -- plain FP64 CPU oracle for the contact-SPH (CSPH) hot path
 * with Voronoi dynamic domain decomposition (VD3), arXiv 1805.05128.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the correctness reference that
 * the CUDA path is compared against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library, and the product path never calls it.
 *
 * Every routine is single-threaded, FP64, compiled with -ffp-contract=off, and
 * written to be checked by eye against the paper:
 *   Sec. 3.1  eq. (VoronoiDefinition) + tie rule   -> orc_voronoi_assign
 *   Sec. 3.2-3.4 eqs. (BalancingOffset), (BalancingOffsetPlusRot),
 *            (BalancingOffsetRot), (TotalOffset)   -> orc_balance
 *   Sec. 4.1 eqs. (SPH:Conti), (SPH:Pulse), (SPH:Energy),
 *            (SmoothingLengthDef)                  -> orc_rates
 *   Sec. 4.2 eq. (Dcell), linked-list cells, R^int/R^hrz -> orc_cell_grid,
 *            orc_pairs_cells, orc_unit_stats
 *   Sec. 4.3 eq. (Horizon)                         -> orc_unit_stats
 *   Sec. 7   eqs. (mie_gruneisen_eos), (mie_gruneisen_reference) -> orc_eos
 */
#ifndef CSPH_ORACLE_H
#define CSPH_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_KERNEL_CUBIC = 0, ORC_KERNEL_WENDLAND_C2 = 1 };
enum { ORC_EOS_IDEAL = 0, ORC_EOS_STIFFENED = 1, ORC_EOS_TAIT = 2, ORC_EOS_MIE_GRUNEISEN = 3 };
enum { ORC_MAX_MAT = 4 };
enum { ORC_SOLVER_ACOUSTIC = 0, ORC_SOLVER_HLL = 1 };

typedef struct {
  int eos;        /* ORC_EOS_* */
  double gamma;   /* ideal/stiffened: adiabatic index; Tait: exponent; MG: Grueneisen Gamma */
  double rho0;    /* reference density */
  double c0;      /* reference sound speed (stiffened, Tait); MG: c_a of u_s = c_a + s_a u_p */
  double p_inf;   /* stiffened gas: P_inf */
  double s_a;     /* MG: Hugoniot slope s_a */
} orc_material;

typedef struct {
  int dim;        /* spatial dimension of the particles: 1, 2 or 3 */
  int kernel;     /* ORC_KERNEL_* */
  double kappa;   /* kernel support radius in units of h (2 cubic, 1.936 Wendland) */
  double eta;     /* h_ij = eta (d_i + d_j) / 2 */
  double cfl;     /* dt = cfl * min_i eta d_i / (c_i + |v_i|) */
  double cell_beta; /* buffer beta used in the cell size eq. (Dcell) */
  int64_t cell_cap; /* maximum number of cells of the dense grid */
  int n_mat;
  orc_material mat[ORC_MAX_MAT];
  int order;      /* 1 (particle-centre states, Sec. 4.1 as written) or 2 (states reconstructed
                     to the pair midpoint, the NEXT variant; see orc_rates) */
  int solver;     /* ORC_SOLVER_ACOUSTIC (default) or ORC_SOLVER_HLL */
} orc_params;

/* Particle state, structure of arrays, host memory.  For dim < 3 the unused
 * components (y/z, vy/vz, ay/az) may be NULL and are then taken as zero. */
typedef struct {
  int64_t n;
  double *x, *y, *z;
  double *vx, *vy, *vz;
  double *rho, *E, *m;        /* density, specific total energy e + v^2/2, mass */
  int32_t *mat;               /* material index per particle (NULL = 0) */
  double *ax, *ay, *az, *drho, *dE;   /* time derivatives at this state */
  double *d, *P, *c;          /* particle size, pressure, sound speed */
} orc_state;

/* Cell grid of eq. (Dcell) on the dense mesh. */
typedef struct {
  double x0[3];     /* origin = componentwise minimum of the positions */
  double dc;        /* cell edge D^c */
  double inv_dc;    /* 1 / D^c */
  int64_t dims[3];  /* cells per axis (1 for unused axes) */
  int64_t ncells;
} orc_grid;

/* ---- closure: kernel, EOS, pair Riemann solver ---- */
double orc_kernel_w(int kernel, int dim, double kappa, double r, double h);
double orc_kernel_dw(int kernel, int dim, double kappa, double r, double h);
/* returns 1 if c^2 < 0 (c is then set to 0 and the event is counted by callers) */
int orc_eos(const orc_material* mat, double rho, double e, double* P, double* c);
void orc_riemann_acoustic(double Pi, double Pj, double Zi, double Zj, double vRi, double vRj,
                          double* Pstar, double* vstar);
/* The two-wave HLL state of the same linearised problem with Davis wave
 * speeds +-max(Z_i, Z_j) (see the .c file). */
void orc_riemann_hll(double Pi, double Pj, double Zi, double Zj, double vRi, double vRj,
                     double* Pstar, double* vstar);

/* ---- per-particle derived quantities: e, P, c, d ---- */
int64_t orc_derive(const orc_params* p, orc_state* s);
double orc_dt(const orc_params* p, const orc_state* s);

/* ---- neighbour search ---- */
int orc_cell_grid(const orc_params* p, const orc_state* s, orc_grid* g, int64_t* cell_of /*n or NULL*/);
int64_t orc_pairs_brute(const orc_params* p, const orc_state* s, int64_t cap, int32_t* pi, int32_t* pj);
int64_t orc_pairs_cells(const orc_params* p, const orc_state* s, int64_t cap, int32_t* pi, int32_t* pj);

/* ---- CSPH rates over a pair list ---- */
void orc_rates(const orc_params* p, orc_state* s, int64_t npairs, const int32_t* pi, const int32_t* pj);
/* SPH gradients used by the order-2 reconstruction: gP (3 per particle) and
 * gV (9 per particle, [a][b] = d v_a / d x_b), grad q_i = sum_j V_j (q_j - q_i)
 * (-W'_ij) e^R_ij over the pair list, at the state's d, P. */
void orc_pair_gradients(const orc_params* p, const orc_state* s, int64_t npairs, const int32_t* pi,
                        const int32_t* pj, double* gP, double* gV);
int64_t orc_eval_rates(const orc_params* p, orc_state* s);   /* derive + pairs + rates; returns npairs or <0 */

/* ---- KDK leapfrog ---- */
int orc_step(const orc_params* p, orc_state* s, int n_steps, int rates_valid, double* t, double* dt_out);

/* ---- FP64 conservation sums: M, px, py, pz, E_tot ---- */
void orc_conservation(const orc_state* s, double out5[5]);

/* ---- VD3 ---- */
void orc_voronoi_assign(int64_t n, int dim, const double* x, const double* y, const double* z,
                        int K, const double* gen, int32_t* unit);
int orc_unit_stats(const orc_params* p, const orc_state* s, const int32_t* unit, int K, int gdim,
                   int64_t npairs, const int32_t* pi, const int32_t* pj, double beta,
                   double* load, uint8_t* adj, double* dsh, double* centroid, int64_t* count);
double orc_balance(int K, int gdim, double* gen, const double* load, const uint8_t* adj,
                   const double* dsh, const double* centroid, const int64_t* count,
                   double theta, double sigma, double gamma_b, double* dg_out);

/* ---- reverse mode (pair set and dt held fixed); cubic kernel, ideal / stiffened gas ---- */
int orc_rates_vjp(const orc_params* p, const orc_state* s, int64_t npairs, const int32_t* pi, const int32_t* pj,
                  const double* ga, const double* gr, const double* gE,
                  double* bx, double* bv, double* brho, double* bE, double* bpar);
int orc_step_replay(const orc_params* p, orc_state* s, int n_steps, int rates_valid, const double* dts);
int orc_step_vjp(const orc_params* p, const orc_state* s, double dt, double* yx, double* yv, double* yrho,
                 double* yE, double* ya, double* ydrho, double* ydE, double* bpar);

#ifdef __cplusplus
}
#endif
#endif
