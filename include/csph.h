/*
 * csph.h -- C ABI of the GB300 contact-SPH (CSPH) hot path with Voronoi
 * dynamic domain decomposition (VD3), arXiv 1805.05128.
 *
 * Conventions for every entry point:
 *  - All functions are extern "C", return an int status (SPH_OK = 0 or an
 *    SPH_ERR_* code) and never throw.  sph_last_error() gives a message.
 *  - Array arguments are DEVICE pointers owned by the caller unless a comment
 *    says "host".  Arrays are dense, contiguous, one element per particle (or
 *    per generator), 8-byte aligned for doubles.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are asynchronous on that stream: they enqueue work and return.
 *    Only sph_read_status() synchronises.  Errors found on the host (bad
 *    arguments) are returned at once; errors found on the device (list or
 *    cell capacity exceeded, non-finite values, unit ids out of range) are
 *    latched in a device status word and reported by sph_read_status().  A
 *    kernel that latches an error keeps every access in bounds and returns
 *    normally; the results of that call are then not meaningful.
 *  - A handle owns only workspace (cell lists, packed operands, work-unit
 *    lists, reduction buffers), allocated in sph_init and freed in
 *    sph_destroy.  A handle is used from one host thread at a time.
 */
#ifndef CSPH_H
#define CSPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SPH_OK 0
#define SPH_ERR_INVALID 1    /* bad argument or unsupported combination */
#define SPH_ERR_CAPACITY 2   /* more particles / cells / pairs than the workspace holds */
#define SPH_ERR_NONFINITE 3  /* NaN or Inf found in the particle state */
#define SPH_ERR_CUDA 4       /* a CUDA runtime call failed */
#define SPH_ERR_TIMEOUT 5    /* reserved: no kernel of this library waits on another, so nothing sets it */

/* ---- enumerations ---- */
#define SPH_KERNEL_CUBIC 0        /* cubic spline M4, support 2h */
#define SPH_KERNEL_WENDLAND_C2 1  /* Wendland C2, support kappa h (paper: kappa = 1.936, Sec. 4.1) */

#define SPH_EOS_IDEAL 0          /* P = (gamma-1) rho e */
#define SPH_EOS_STIFFENED 1      /* P = (gamma-1) rho e - gamma P_inf */
#define SPH_EOS_TAIT 2           /* P = rho0 c0^2/gamma [(rho/rho0)^gamma - 1] */
#define SPH_EOS_MIE_GRUNEISEN 3  /* eqs. (mie_gruneisen_eos), (mie_gruneisen_reference), Sec. 7 */
#define SPH_EOS_STIFFENED_C0 4   /* stiffened gas given by (rho0, c0, gamma): sph_init sets
                                    P_inf = rho0 c0^2 / gamma, so that c = c0 and P = 0 at rho0 with
                                    e = gamma P_inf / ((gamma - 1) rho0); p_inf is ignored.  The form
                                    whose dL/d(c0, gamma) sph_step_adjoint returns. */

#define SPH_PREC_FP64 0   /* every pair flux in FP64 */
#define SPH_PREC_MIXED 1  /* FP32 pair fluxes on local-origin offsets and on velocities relative
                             to whole-m/s references (exact differences), Kahan-compensated
                             per-particle sums; FP64 positions, time, integration */

#define SPH_SOLVER_ACOUSTIC 0  /* pair Riemann solver: linearised acoustic, impedance-weighted (Sec. 4.1) */
#define SPH_SOLVER_HLL 1       /* two-wave HLL state of the same linearised problem with Davis speeds
                                  -+max(Z_i, Z_j): the acoustic formula with both Z set to max(Z_i, Z_j) */

#define SPH_LOAD_PAIRS 0       /* work-unit load L_k: the pair interactions of unit k (deterministic) */
#define SPH_LOAD_TIME 1        /* L_k: the useful time t^u_k of eq. (load), here the SM cycles the pair
                                  kernel spends on unit k's particles (timing-dependent, so the
                                  rebalancing is not reproducible bit for bit) */

#define SPH_SCHED_GLOBAL 0       /* list kernel: warps take groups of 32 slots (cell order) from one global
                                    counter, whatever their units */
#define SPH_SCHED_UNITS 1        /* the Voronoi units are the work partition (Secs. 3-4 recast on one GPU):
                                    at each list build the slots are ordered unit-major (cell order
                                    inside a unit), each unit owning one contiguous range; each CTA
                                    drains its home unit's queue, then steals from the following units */
#define SPH_SCHED_UNITS_OWNED 2  /* as SPH_SCHED_UNITS without stealing: a unit is processed by its own
                                    CTAs only (the paper's one subdomain per processor), so the step waits
                                    for the most loaded unit */

#define SPH_MAX_MAT 4
#define SPH_MAX_UNITS 256

typedef struct sph_material {
  int32_t eos;     /* SPH_EOS_* */
  int32_t pad_;
  double gamma;    /* ideal/stiffened: adiabatic index; Tait: exponent; MG: Grueneisen Gamma */
  double rho0;     /* reference density (stiffened: informative; Tait, MG: used) */
  double c0;       /* reference sound speed (Tait); MG: c_a */
  double p_inf;    /* stiffened gas P_inf */
  double s_a;      /* MG: Hugoniot slope */
} sph_material;

typedef struct sph_params {
  int32_t dim;        /* spatial dimension of the particles: 1, 2 or 3 */
  int32_t kernel;     /* SPH_KERNEL_* */
  int32_t precision;  /* SPH_PREC_* */
  int32_t n_mat;      /* materials used: 1..SPH_MAX_MAT in mat[], or up to 65536 with materials */
  double kappa;       /* kernel support in units of h */
  double eta;         /* h_ij = eta (d_i + d_j)/2, eq. (SmoothingLengthDef) times eta */
  double cfl;         /* dt = cfl min_i eta d_i / (c_i + |v_i|) */
  double cell_beta;   /* beta of eq. (Dcell); 0 = mesh and pairs found every step; > 0 = Verlet
                         lists over (1 + beta) kappa h_ij reused across steps (sph_list_builds) */
  int64_t cell_cap;   /* maximum cells of the dense mesh over all instances */
  sph_material mat[SPH_MAX_MAT];
  /* Voronoi work units (VD3).  n_units = 0 disables them. */
  int32_t n_units;    /* K <= SPH_MAX_UNITS */
  int32_t unit_dim;   /* dimension of the decomposition: 1, 2 or 3 (<= dim) */
  int32_t n_upd;      /* sph_step rebalances every n_upd steps (0 = never) */
  int32_t pair_blocks_per_sm; /* resident CTAs per SM of the persistent pair kernel (128 threads,
                                 one warp per home cell); 0 or more than fit = as many as fit */
  double theta;       /* eq. (TotalOffset) */
  double sigma;       /* eq. (BalancingOffsetPlusRot) */
  double gamma_b;     /* gamma of eq. (TotalOffset) */
  double beta_sh;     /* buffer beta of R^hrz used in D^sh, eq. (Horizon) */
  double* generators; /* device, K x unit_dim, read and updated by sph_step's rebalancing */
  const sph_material* materials; /* host, n_mat entries, or NULL to use mat[]; copied by sph_init
                                    (one material per instance gives per-instance EOS parameters) */
  int32_t order;      /* 1 (or 0): the particles' own P, v^R feed the pair Riemann solver (Sec. 4.1);
                         2: P and v^R extrapolated to the pair midpoint with SPH gradients, minmod-
                         limited against the pair jump (an extension; needs cell_beta = 0, no adjoint) */
  int32_t solver;     /* SPH_SOLVER_*: the pair Riemann solver (HLL: no adjoint) */
  int32_t load_measure; /* SPH_LOAD_*: what the work-unit loads of the balancing count */
  int32_t list_cap;   /* Verlet lists: entries held per particle; 0 = the default (twice the
                         neighbours of a uniform lattice within the buffered radius, plus 32);
                         otherwise at least 32 (SPH_ERR_INVALID below).  A list that would grow
                         past it is cut at the capacity and SPH_ERR_CAPACITY is latched. */
  int32_t unit_sched; /* SPH_SCHED_*: work partition of the list kernel (needs cell_beta > 0 and
                         n_units > 0; otherwise the global counter is used) */
  int32_t list_staging; /* 1: the list kernel (mixed precision) stages each next chunk's neighbour
                           operands in shared memory with cp.async while the current one is
                           evaluated; 0 (default): the operands are gathered through L1 */
} sph_params;

/* Particle state: structure of arrays in device memory, n elements each.
 * For dim < 3 the unused components (y, z, vy, vz, ay, az) may be NULL. */
typedef struct sph_state {
  int64_t n;
  double *x, *y, *z;            /* position (FP64) */
  double *vx, *vy, *vz;         /* velocity */
  double *rho, *E, *m;          /* density, specific total energy e + v^2/2, mass */
  int32_t* mat;                 /* material index, or NULL for material 0 */
  double *ax, *ay, *az, *drho, *dE; /* rates at this state (written by the library) */
  double *d, *P, *c;            /* particle size, pressure, sound speed (written) */
  int64_t* id;                  /* caller's particle identity, permuted along; may be NULL */
  int32_t* unit;                /* work unit of each particle (written by voronoi_assign); may be
                                   NULL when n_units = 0 */
} sph_state;

typedef struct sph_balance_params {
  double theta, sigma, gamma_b, beta_sh;
} sph_balance_params;

typedef struct sph_handle sph_handle;

/* A checkpoint of a forward run, for sph_step_adjoint. */
typedef struct sph_ckpt {
  sph_state state;            /* device: state at the checkpoint, including the held rates */
  const double* dt;           /* device: the dt of each step after the checkpoint (n_steps doubles),
                                 as recorded with sph_last_dt during the forward run */
  int32_t rates_from_state;   /* 1 if the held rates were evaluated at this very state
                                 (the run's first checkpoint), else 0 */
  int32_t reverse_fp64;       /* mixed-precision handle: 1 = pair derivatives in FP64 (FP32 forward
                                 replay, FP64 adjoint), 0 = in FP32 with Kahan sums; ignored in FP64 */
} sph_ckpt;

/* Create a handle for `s->n` particles split into n_instances independent
 * simulations; instance b owns particles [inst_offsets[b], inst_offsets[b+1])
 * (host array of n_instances+1 entries, inst_offsets[0] = 0,
 * inst_offsets[n_instances] = s->n).  Checks the parameters, allocates the
 * workspace and checks the state for non-finite values (this one call
 * synchronises the stream).  Problem statement: particles with mass,
 * position, velocity, density and energy interacting through pair Riemann
 * fluxes within kappa h_ij (Sec. 4.1).  Errors: SPH_ERR_INVALID for bad
 * parameters, SPH_ERR_NONFINITE, SPH_ERR_CUDA.  On error *h is NULL. */
int sph_init(sph_handle** h, const sph_params* p, int n_instances, const int64_t* inst_offsets,
             const sph_state* s, void* stream);

/* Derive d_i = (m_i/rho_i)^(1/dim), P_i and c_i, build the cell mesh of
 * eq. (Dcell) and renumber the particles so that each cell's particles are
 * contiguous and cells follow each other in mesh order (the locality
 * renumbering of Sec. 4.2).  Every array of `s` (including id, unit, mat and
 * the rates) is permuted in place, within each instance. */
int sph_build_cells(sph_handle* h, sph_state* s, void* stream);

/* Evaluate the CSPH rates of eqs. (SPH:Conti), (SPH:Pulse), (SPH:Energy) at
 * the current state: d, P, c, cell mesh, pair search within kappa h_ij,
 * acoustic pair Riemann fluxes, per-particle sums.  Writes ax, ay, az, drho,
 * dE, d, P, c.  Does not move particles or permute arrays.  When work units
 * are enabled it adds this evaluation's pair counts and unit adjacency to the
 * balancing accumulators. */
int sph_eval_rates(sph_handle* h, sph_state* s, void* stream);

/* Advance every instance by n_steps kick-drift-kick steps (Alg. 1, loop
 * "renew particle positions and states and make global synchronization of
 * SPH time step"): dt from the CFL condition reduced on the device, half
 * kick with the rates held in `s`, drift, rates at the predicted state, half
 * kick.  t_dev (device, n_instances doubles, may be NULL) accumulates time.
 * If the rates in `s` were not produced by this handle they are evaluated
 * first.  With work units and n_upd > 0, every n_upd steps it runs
 * voronoi_balance on p->generators, voronoi_assign and the renumbering of
 * sph_build_cells (Alg. 1, outer loop). */
int sph_step(sph_handle* h, sph_state* s, int n_steps, double* t_dev, void* stream);

/* sph_step with a prescribed time step: step k of instance b uses
 * dt_dev[k * n_instances + b] (device) instead of the CFL condition; no
 * rebalancing.  Replays a recorded run (e.g. for finite-difference checks of
 * sph_step_adjoint). */
int sph_step_dt(sph_handle* h, sph_state* s, int n_steps, const double* dt_dev, double* t_dev, void* stream);

/* Assign every particle to its nearest generator, eq. (VoronoiDefinition),
 * ties to the smaller index (Sec. 3.1), in the first `dim` coordinates.
 * gen: device, K x dim doubles.  unit_out: device, n int32 (may be s->unit).
 * unit_offsets: device, K+1 int32, or NULL: start of each unit in the
 * handle's unit-ordered particle list.  Resets the balancing accumulators.
 * Requires one instance.  Errors: SPH_ERR_INVALID (K, dim, instances). */
int voronoi_assign(sph_handle* h, const sph_state* s, const double* gen, int K, int dim,
                   int32_t* unit_out, int32_t* unit_offsets, void* stream);

/* voronoi_balance from unit statistics given by the caller (host arrays), for
 * a decomposition spread over several processes whose statistics are reduced
 * across them first: load (K), adj (K x K bytes, 0/1, symmetric), rmax (K:
 * max over the unit's particles of R^hrz_i, so that D^sh_kl = max(rmax_k,
 * rmax_l), eq. Horizon), centroid (K x dim: the mean position of the unit's
 * particles), count (K).  The same update as voronoi_balance (eqs.
 * BalancingOffset ... TotalOffset) on gen (device, K x dim, updated in place);
 * shift_sum_out (device double, may be NULL) receives sum_k |g^_k - g_k|.
 * Requires K = the handle's n_units and dim = its unit_dim; the handle's
 * accumulators are reset. */
int voronoi_balance_stats(sph_handle* h, double* gen, int K, int dim, const double* load, const uint8_t* adj,
                          const double* rmax, const double* centroid, const int64_t* count,
                          const sph_balance_params* bp, double* shift_sum_out, void* stream);

/* One balancing update of the generators (Secs. 3.2-3.4): loads L_k (device
 * `load`, K doubles, or NULL for the accumulated pair counts, a pair that
 * crosses units counting 1/2 to each), adjacency from the accumulated
 * interacting pairs, D^sh_kl of eq. (Horizon), two-body eq.
 * (BalancingOffset), three-body eq. (BalancingOffsetRot) for dim = 2 limited
 * to max_l D^sh_kl, combination eq. (BalancingOffsetPlusRot) and cumulative
 * movement eq. (TotalOffset) toward the current centroid of each unit's
 * particles.  gen (device, K x dim) is updated in place; shift_sum_out
 * (device double, may be NULL) receives sum_k |g^_k - g_k|, eq. (VDConvergence).
 * Uses s->unit, positions and d, and the neighbour statistics of the last
 * rate evaluation; resets the accumulators. */
int voronoi_balance(sph_handle* h, const sph_state* s, double* gen, int K, int dim, const double* load,
                    const sph_balance_params* bp, double* shift_sum_out, void* stream);

/* Reverse mode of n_steps steps of sph_step after the checkpoint ck, with
 * the pair set and the dt sequence of the forward run held fixed (dt as a
 * stop-gradient; the cubic-spline W' and W'' vanish at the support, so the
 * gradient is continuous when pairs enter or leave).  The forward steps are
 * replayed from ck in the handle's precision and kept in workspace; the
 * vector-Jacobian products of the rates (eqs. SPH:Conti, SPH:Pulse,
 * SPH:Energy with the acoustic pair solver) and of the kick-drift-kick
 * algebra are accumulated in FP64.
 *   adj_out: device arrays in sph_state layout holding dL/d(state after the
 *            n_steps): x, y, z (positions), vx, vy, vz, rho, E, and ax, ay,
 *            az, drho, dE (the held rates); other fields are ignored
 *   adj_in:  receives dL/d(state at the checkpoint) in the same layout (may
 *            be adj_out itself).  With ck->rates_from_state the adjoint of
 *            the held rates is folded into x, v, rho, E and the rate fields
 *            are returned as zero.
 *   adj_params: device, 2 doubles, ADDED dL/d(c0, gamma) of material 0
 *            (SPH_EOS_STIFFENED_C0, or SPH_EOS_STIFFENED read as
 *            P_inf = rho0 c0^2 / gamma; ideal gas: dL/dgamma only).
 * Scope, narrower than the forward step's: one instance, the cubic spline,
 * ideal or stiffened gas, the acoustic pair solver and order 1
 * (SPH_ERR_INVALID otherwise); the replay finds the pairs with the per-step
 * cell search whatever cell_beta is.  With reverse_fp64 = 0 on a mixed
 * handle the pair derivatives use FP32 packed volumes rescaled back to SI
 * units, which loses precision for particles far below a micrometre.  No
 * counterpart in the paper, which runs forward only; it differentiates the
 * paper's step. */
int sph_step_adjoint(sph_handle* h, const sph_ckpt* ck, int n_steps, const sph_state* adj_out,
                     sph_state* adj_in, double* adj_params, void* stream);

/* Declare that the rate arrays of the state (ax, ay, az, drho, dE) are the
 * held rates of the scheme for the next step (the rates of the previous
 * step's evaluation at its predicted state, e.g. received from the process
 * that evaluated them), so that sph_step and sph_step_dt use them instead of
 * evaluating rates at the current state first.  A decomposed run moves
 * particles between handles with their held rates. */
int sph_hold_rates(sph_handle* h);

/* The CFL time step of the current state without stepping (Alg. 1: each
 * process's bound before the global synchronisation of the SPH time step):
 * dt_out (device, n_instances doubles) receives cfl min_i eta d_i / (c_i + |v_i|)
 * per instance, the dt sph_step would take.  A rank of a decomposed run
 * reduces it with the other ranks' (minimum) and steps with sph_step_dt. */
int sph_cfl_dt(sph_handle* h, const sph_state* s, double* dt_out, void* stream);

/* Copy the dt of the last step (device, n_instances doubles) to dt_out (device),
 * asynchronously; used to record the schedule for sph_step_adjoint. */
int sph_last_dt(sph_handle* h, double* dt_out, void* stream);

/* FP64 totals per instance: out (device, n_instances x 5 doubles) receives
 * mass, momentum x/y/z and total energy sum m E, summed in a fixed order. */
int sph_conservation(sph_handle* h, const sph_state* s, double* out, void* stream);

/* Host-side copy of the balancing accumulators (for inspection and tests):
 * load_out (host, K doubles: pair counts with 1/2 per crossing end, or with
 * SPH_LOAD_TIME half the accumulated SM cycles) and
 * adj_out (host, K*K bytes, 0/1).  Synchronises the stream. */
int sph_unit_stats(sph_handle* h, double* load_out, uint8_t* adj_out, void* stream);

/* Per-unit timing of the last list evaluation run with SPH_SCHED_UNITS or
 * SPH_SCHED_UNITS_OWNED (the completion times whose spread the balancing of
 * Sec. 2 minimises): out (host, 2 K doubles) receives, for unit k, the start
 * of its first slot group and the end of its last, in ns from the earliest
 * start of any unit (%globaltimer).  An empty unit reports 0, 0.
 * Synchronises the stream.  Errors: SPH_ERR_INVALID if the handle does not
 * partition the list kernel by units. */
int sph_unit_times(sph_handle* h, double* out, void* stream);

/* Synchronise the handle's last stream and report the device status word
 * (SPH_OK or the first SPH_ERR_* latched by a kernel) in *device_status;
 * the return value is SPH_OK unless the synchronisation itself failed.
 * Clears the status word. */
int sph_read_status(sph_handle* h, int* device_status);

/* Message for the last host-side error on this handle ("" if none);
 * sph_last_error(NULL) gives the message of the last failed sph_init. */
const char* sph_last_error(const sph_handle* h);

/* Counters of the last call: accepted half pairs (i < j) of the last rate
 * evaluation, candidates tested, and pairs decided by the FP64 fallback. */
int sph_pair_counts(sph_handle* h, int64_t* half_pairs, int64_t* candidates, int64_t* fp64_checks,
                    void* stream);

/* Verlet lists (cell_beta = beta > 0; the pair list with buffer beta of
 * Sec. 4.2, reused over several steps): *builds = number of list builds since
 * sph_init, *capacity = list entries held per particle.  sph_step keeps the
 * mesh, the slot order and the lists while every particle satisfies
 * |x - x_b - U| + kh max(0, d - d_b) <= 0.95 beta kh d_b (x_b, d_b at the
 * last build, kh = kappa eta / 2, U one displacement shared by all particles
 * of the handle, chosen on the device to follow the bulk motion), which keeps
 * every pair within kappa h_ij listed, and rebuilds them otherwise (decided
 * on the device, per instance: an instance whose criterion fails rebuilds
 * its mesh, slots and lists, the others keep theirs), as well as after any
 * call that rebuilds the mesh and after a rebalance that renumbers
 * unit-major (SPH_SCHED_UNITS*, which also rebuilds every instance at
 * once); the renumbering into slot order of the other rebalances keeps
 * them.  *builds counts the steps with a rebuild.  Synchronises the
 * stream.
 * Errors: SPH_ERR_INVALID if the handle has no lists (cell_beta = 0). */
int sph_list_builds(sph_handle* h, int64_t* builds, int32_t* capacity, void* stream);

/* Inspection of the neighbour search (Sec. 4.2) at the current state,
 * for verification: derives d, builds the cell mesh of eq. (Dcell) and
 * writes, per particle in the state's order, the linear cell index
 * cx + nx (cy + ny cz) local to its instance (cell_out, device, n int32).
 * grid_out (host, may be NULL) receives per instance 8 doubles:
 * x0[3], D^c, nx, ny, nz, ncells.  Synchronises the stream. */
int sph_cell_index(sph_handle* h, const sph_state* s, int32_t* cell_out, double* grid_out, void* stream);

/* Inspection of the interacting pairs (Sec. 4.1-4.2) at the current state:
 * runs the rate evaluation of sph_eval_rates and also writes every
 * interacting unordered pair once as (i, j) particle indices with i < j
 * into pi_out/pj_out (device, cap int32 each, unordered).  *count_out
 * (host) receives the number of pairs; when it exceeds cap only cap pairs
 * are written and SPH_ERR_CAPACITY is returned.  Synchronises the stream. */
int sph_pair_list(sph_handle* h, sph_state* s, int64_t cap, int32_t* pi_out, int32_t* pj_out,
                  int64_t* count_out, void* stream);

/* Allocation-free voronoi_assign.  Some callers cannot call cudaMalloc: a
 * host loop that must not allocate (allocation synchronises the device and
 * can fail under memory pressure at a bad time), or code whose device memory
 * all belongs to another allocator or a fixed arena that it may not step
 * outside.  Such a caller cannot create a handle, whose workspace sph_init
 * allocates.  This entry point needs no handle and allocates nothing: its
 * scratch (per-unit counts, their scan, a counter) lives in one file-scope
 * device array of about 8.4 MB that every device which loads the library
 * keeps until the process exits.  The paper has no counterpart; the result
 * equals that of voronoi_assign on the same inputs, ties going to the
 * smaller generator index.
 *   x, y, z      device positions, n doubles each (y NULL for dim 1, z NULL
 *                for dim <= 2)
 *   gen          device, K x dim doubles
 *   unit_out     device, n int32: the owning unit of each particle
 *   unit_offsets device, K+1 int32, or NULL: start of each unit in unit_list
 *   unit_list    device, n int32, or NULL: particle indices grouped by unit,
 *                ascending inside each unit
 * Limits: 1 <= n <= 4,194,304 and 1 <= K <= 256 (else SPH_ERR_CAPACITY, or
 * SPH_ERR_INVALID for n < 1, K < 1, a bad dim or a missing pointer; see
 * sph_last_error(NULL)).  Unlike the handle path this call has no status
 * word: a particle with a NaN or infinite coordinate is given unit 0 and
 * nothing reports it.  The array is shared by all calls on a device: calls
 * whose work overlaps on the GPU (other streams, other host threads) race on
 * it; each call resets what it needs, so consecutive calls on one stream are
 * independent.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current and keeps it for
 * the life of the process.  After cudaDeviceReset the kept address is
 * stale: do not call this entry point on a device that has been reset. */
int voronoi_assign_static(int64_t n, const double* x, const double* y, const double* z, const double* gen,
                          int K, int dim, int32_t* unit_out, int32_t* unit_offsets, int32_t* unit_list,
                          void* stream);

/* Measurement support.  sph_profile(h, 1) starts recording CUDA events
 * around every launch of the pair kernel on the caller's stream and counts
 * every kernel launch of the library; sph_profile(h, 0) stops.  Resets the
 * records either way.  Pair-kernel launches issued while the stream is being
 * captured into a CUDA graph are counted as launches but not timed. */
int sph_profile(sph_handle* h, int enable);

/* Synchronise and report, since the last sph_profile/sph_profile_read: the
 * summed device duration of the pair-kernel launches in ms (pair_ms), their
 * number, and the number of kernel launches of the library.  Resets them. */
int sph_profile_read(sph_handle* h, double* pair_ms, int64_t* pair_launches, int64_t* kernel_launches);

void sph_destroy(sph_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* CSPH_H */
