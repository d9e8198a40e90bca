// csph_internal.cuh -- shared declarations of the CUDA implementation of the
// CSPH hot path (arXiv 1805.05128) for sm_103a.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "csph.h"

namespace csph {

constexpr int kBlock = 256;          // threads of the per-particle kernels
constexpr int kPairBlock = 128;      // threads of the pair kernel
constexpr int kListCap = 128;        // per-particle neighbour list capacity of the pair kernel (shared memory)
constexpr double kCellMargin = 1.0 + 0x1p-20;  // relative safety margin of D^c

// Per-instance cell mesh of eq. (Dcell) on the dense grid.
struct GridInfo {
  double x0[3];      // componentwise minimum of the positions
  double hi[3];      // componentwise maximum of the positions
  double dc;         // cell edge D^c
  double inv_dc;     // 1 / D^c
  double dmax1, dmax2;  // the two largest particle sizes
  int32_t dims[3];   // cells per axis
  int32_t pad;
  int64_t cell_off;  // first global cell of this instance
  int64_t ncells;
  float dc_f;        // D^c rounded to FP32 (offset shifts of the mixed kernel)
  float pad2;
};

// Per-block partial reductions of the segmented per-particle kernels.
// Values are order-preserving integer keys of the doubles (see k_step.cu).
struct BlockPart {
  long long lo[3], hi[3];  // bounding box
  long long d1, d2;        // two largest particle sizes
  long long dtmin;         // min_i eta d_i / (c_i + |v_i|)
};

// Verlet lists: the grid-wide maximum of the validity criterion and the box
// of the displacements of one kick-drift, accumulated by its blocks with
// atomics and read (then reset) by the step's flag kernel.
struct VAcc {
  long long viol;          // max_i of the criterion key (> 0: rebuild)
  int dlo[3], dhi[3];      // box of x - x_b - U (FP32 order keys)
};

// Material constants on the device.
struct Mat {
  int eos;
  double gamma, rho0, c0, p_inf, s_a;
  // Tait: B = rho0 c0^2 / gamma, and gamma as an int when it is a whole
  // number in [1, 16] (0 otherwise), so that r^gamma is a few products
  // instead of pow (FP64 pow costs ~100 operations of GB300's narrow FP64 pipe)
  double tait_B;
  int tait_n;
  // the constants rounded to FP32 once (the FP32 sound speed of the mixed
  // packs and of the CFL bound; a conversion per particle costs a slot of the
  // narrow FP64 pipe)
  float gamma_f, rho0_f, c0_f, p_inf_f, s_a_f;
};

// Host-side table entry of a material.
// SPH_EOS_STIFFENED_C0 becomes the stiffened gas with P_inf = rho0 c0^2 / gamma.
inline Mat make_mat(int eos, double gamma, double rho0, double c0, double p_inf, double s_a) {
  if (eos == SPH_EOS_STIFFENED_C0) {
    eos = SPH_EOS_STIFFENED;
    p_inf = rho0 * c0 * c0 / gamma;
  }
  Mat m{eos, gamma, rho0, c0, p_inf, s_a, 0.0, 0, (float)gamma, (float)rho0, (float)c0, (float)p_inf, (float)s_a};
  if (eos == SPH_EOS_TAIT) {
    m.tait_B = rho0 * c0 * c0 / gamma;
    m.tait_n = (gamma >= 1.0 && gamma <= 16.0 && gamma == (double)(int)gamma) ? (int)gamma : 0;
  }
  return m;
}

// x^n for n >= 1 by binary powering (a few products; the rounding of each
// product is the only difference from pow).
template <typename T>
__device__ __forceinline__ T ipow(T x, int n) {
  T r = T(1), b = x;
  while (n > 0) {
    if (n & 1) r *= b;
    n >>= 1;
    if (n) b *= b;
  }
  return r;
}

struct DevParams {
  int dim, kernel, precision, n_mat;
  double kappa, eta, cfl, cell_beta, kh;  // kh = (0.5 kappa) eta
  const Mat* mat;                         // device table of n_mat materials
  const double* vref;                     // Verlet lists: x, y, z, d at the last build (4 arrays of n), or NULL
  const double* vframe;                   // Verlet lists, 6 doubles per instance: this step's frame
                                          // displacement U (3), the number of steps since the build,
                                          // U as 3 floats; or NULL
  VAcc* vacc;                             // Verlet lists: the criterion's accumulators, one per
                                          // instance, or NULL
  int64_t n;                              // particles of the handle (stride of vref)
  double vscale;                          // mixed precision: packed volume = (m / rho) vscale (a power of two)
  float eta_f, kh_f, cell_beta_f, vscale_f;   // eta, kh, cell_beta, vscale rounded to FP32 once
  const double* slot_org;                 // mixed precision: origin (x, y, z: 3 arrays of n) of each
                                          // cell-order slot's cell, written at every mesh build
};
constexpr int kMaxMaterials = 65536;

// FP64 packed pair operands (slot order).
struct alignas(32) D4 { double x, y, z, w; };
struct alignas(16) D2 { double x, y; };

}  // namespace csph

struct sph_handle {
  sph_params p;
  csph::DevParams dp;
  int n_inst = 0;
  int64_t n = 0;
  std::vector<int64_t> inst_off_h;
  std::vector<int32_t> inst_blk_h;   // first segmented block of each instance (+ total)
  std::string err;
  cudaStream_t last_stream = nullptr;
  bool rates_valid = false;
  int steps_since_balance = 0;

  // segmented blocks: block b covers particles [blk_start[b], blk_end[b]) of instance blk_inst[b]
  int nblk = 0;
  int32_t* blk_inst = nullptr;
  int64_t* blk_start = nullptr;
  int64_t* blk_end = nullptr;
  int32_t* inst_blk = nullptr;   // [n_inst + 1]
  int64_t* inst_off = nullptr;   // [n_inst + 1]

  csph::BlockPart* part = nullptr;   // [nblk]
  csph::GridInfo* grid = nullptr;    // [n_inst]
  double* dt = nullptr;              // [n_inst]
  int64_t* inst_cap = nullptr;       // [n_inst] cell capacity share of each instance
  int64_t* total_cells = nullptr;    // device scalar

  // cell lists
  int64_t cell_cap = 0;
  int32_t* cell_count = nullptr;     // [cell_cap], kept zero between uses
  int32_t* cell_start = nullptr;     // [cell_cap + 1]
  int32_t* scan_sums = nullptr;      // block sums of the scan
  int32_t* cell_of = nullptr;        // [n] global cell of particle p
  int32_t* rank = nullptr;           // [n] arrival rank within the cell
  int32_t* perm = nullptr;           // [n] slot -> particle
  int32_t* slot_cell = nullptr;      // [n] global cell of slot s
  double* slot_org = nullptr;        // mixed: [3 n] cell origin of each cell-order slot (k_cell_sort)
  int32_t* slot_unit = nullptr;      // [n] work unit of slot s

  // packed operands in slot order (FP32 or FP64 by precision)
  void* packA = nullptr;
  void* packB = nullptr;
  void* packC = nullptr;
  double* rho_slot = nullptr;        // [n] density of slot s (FP64)

  long long* dt_key = nullptr;             // [n_inst] CFL keys left by the fused second kick
  double* dmax_nbr = nullptr;        // [n] largest neighbour size of particle p (last evaluation)

  // Voronoi work units
  int K = 0;
  int gdim = 0;
  unsigned long long* load_acc = nullptr;  // [K] accumulated full-list pair counts
  uint32_t* adj_bits = nullptr;            // [K * K/32 rounded up]
  int32_t* unit_off = nullptr;             // [K + 1]
  int32_t* unit_list = nullptr;            // [n]
  int32_t* unit_work = nullptr;            // partition scratch: counts, starts, scan sums
  int64_t* unit_total = nullptr;           // device scalar K * nb
  int64_t unit_work_total = 0;             // K * nb on the host
  double* unit_stats = nullptr;            // [K x 5] centroid, count, max R^hrz; [K x 4] balance scratch;
                                            // [K x 16 x 4] partial sums of the statistics

  // optional pair output of the pair kernel (sph_pair_list)
  bool collect_adj = true;                  // record unit adjacency in the next pair evaluation
  int32_t* pair_out_i = nullptr;
  int32_t* pair_out_j = nullptr;
  int64_t pair_out_cap = 0;

  // profiling: kernel launch count and CUDA events around each pair-kernel launch
  int64_t launches = 0;
  bool profiling = false;
  std::vector<cudaEvent_t> prof_events;     // pool, used in (start, stop) pairs
  size_t prof_used = 0;

  csph::Mat* mat_dev = nullptr;             // material table
  std::vector<csph::Mat> mat_h;

  int* status = nullptr;                    // device status word
  unsigned long long* counters = nullptr;   // [8] full-list pairs, candidates, fp64 checks, assign FP64
                                            // re-evaluations, listed pairs, pair-kernel work counter

  // renumbering scratch
  void* scratch = nullptr;
  size_t scratch_bytes = 0;

  // reverse mode (sph_step_adjoint), allocated on first use
  void* adj64_A = nullptr;            // FP64 operands of a mixed handle's FP64 reverse pass (D4, D4, D2)
  void* adj64_B = nullptr;
  void* adj64_C = nullptr;
  double* adj64_rho = nullptr;
  csph::D4* adj_G = nullptr;          // rate adjoints / m, slot order (float4 in mixed mode)
  csph::D2* adj_GR = nullptr;         // (dL/ddrho, rho) of the slot (float2 in mixed mode)
  double* adj_pair = nullptr;         // 11 per particle: own-side pair derivatives
  double* adj_par = nullptr;          // 2 per particle: parameter derivatives
  double* adj_W = nullptr;            // working state, 16 arrays of n
  double* adj_store = nullptr;        // replayed states, 13 arrays of n per step
  int adj_store_steps = 0;

  // Verlet lists (cell_beta > 0): every pair within (1 + beta) kappa h_ij at the
  // last build, in slot order, reused by sph_step while the validity criterion
  // holds for every particle (displacement plus size growth since the build
  // within the buffer); the mesh, slot order and lists are rebuilt otherwise.
  bool verlet = false;
  int vcap = 0;                       // list capacity per particle
  uint32_t* vlist = nullptr;          // [n][vcap]: entry k of slot i at i vcap + k = (slot j << 5) | cell code
  int32_t* vcnt = nullptr;            // [n] entries of slot i
  double* vref = nullptr;             // [4 n] x, y, z, d of each particle at the last build, then
                                      // per instance: [6] the frame of the validity criterion (U,
                                      // steps since the build, U in FP32: 3 floats in the last
                                      // two), then per instance [4] a VAcc
  double* vframe = nullptr;           // = vref + 4 n
  csph::VAcc* vacc = nullptr;         // = vref + 4 n + 6 n_inst (32 bytes each)
  int* vflag = nullptr;               // [0]: rebuild in this step; [1]: lists invalid; [2]: builds done
  int* vinst = nullptr;               // [n_inst]: instance rebuilt in this step (its mesh, slots and
                                      // lists; the others keep theirs)

  // Work units as the partition of the list kernel's work (Verlet lists with
  // n_units > 0 and unit_sched > 0): at every list build the cell-order slots
  // are stably partitioned by unit into an evaluation order in which every
  // unit owns one contiguous range of slots; the packed operands and the lists
  // are laid out in that order and the list kernel drains per-unit queues.
  int unit_sched = 0;                 // SPH_SCHED_*
  int32_t* e_of_c = nullptr;          // [n] evaluation slot of each cell-order slot
  int32_t* perm_e = nullptr;          // [n] particle of each evaluation slot
  int32_t* unit_eoff = nullptr;       // [K + 1] start of each unit's evaluation range
  void* packAc = nullptr;             // [n] cell-order copy of the position / size operand (list build)
  unsigned long long* unit_q = nullptr;   // [K] per-unit work counters of the list kernel
  unsigned long long* unit_t = nullptr;   // [2K] first group start and last group end per unit (ns)

  // order-2 reconstruction (sph_params.order = 2): SPH gradients in slot order,
  // the pair kernel's precision: grad P, then grad v_x, grad v_y, grad v_z
  bool order2 = false;
  int solver = SPH_SOLVER_ACOUSTIC;
  bool load_timed = false;           // SPH_LOAD_TIME: unit loads in SM cycles

  // mixed precision: scales (powers of two) of the packed volume and of W', set
  // by sph_init from the largest particle volume (1 in FP64 mode)
  double vscale = 1.0;
  double wscale = 1.0;
  void* grad_p = nullptr;             // [n] float4 / D4
  void* grad_v = nullptr;             // [3 n] float4 / D4
};

namespace csph {

// --------------------------------------------------------------------------
// Device closure: EOS, kernel derivative, acoustic solver
// --------------------------------------------------------------------------

// Returns P and c of material m at (rho, e).  A negative c^2 yields c = 0.
__device__ __forceinline__ void eos(const Mat& m, double rho, double e, double& P, double& c) {
  double c2;
  if (m.eos == SPH_EOS_IDEAL) {
    P = (m.gamma - 1.0) * rho * e;
    c2 = m.gamma * P / rho;
  } else if (m.eos == SPH_EOS_STIFFENED) {
    P = (m.gamma - 1.0) * rho * e - m.gamma * m.p_inf;
    c2 = m.gamma * (P + m.p_inf) / rho;
  } else if (m.eos == SPH_EOS_TAIT) {
    const double r = rho / m.rho0;
    if (m.tait_n > 0) {                                  // whole exponent: r^(n-1) and r^n by products
      const double rn1 = m.tait_n > 1 ? ipow(r, m.tait_n - 1) : 1.0;
      P = m.tait_B * (rn1 * r - 1.0);
      c2 = m.c0 * m.c0 * rn1;
    } else {
      P = m.tait_B * (pow(r, m.gamma) - 1.0);
      c2 = m.c0 * m.c0 * pow(r, m.gamma - 1.0);
    }
  } else {  // Mie-Grueneisen with the linear u_s-u_p Hugoniot reference curves
    double G = m.gamma, ca = m.c0, sa = m.s_a;
    double x = m.rho0 / rho;
    double u = 1.0 - x;
    double D = 1.0 - sa * u;
    double iD2 = 1.0 / (D * D);
    double Pr = m.rho0 * ca * ca * u * iD2;
    double er = 0.5 * ca * ca * u * u * iD2;
    double du = x / rho;
    double dPr = m.rho0 * ca * ca * (1.0 + sa * u) * iD2 / D * du;
    double der = ca * ca * u * iD2 / D * du;
    P = Pr + G * rho * (e - er);
    c2 = dPr + G * (e - er) - G * rho * der + G * P / rho;
  }
  c = c2 > 0.0 ? sqrt(c2) : 0.0;
}

// dW/dr of the cubic spline (support 2h) or the Wendland C2 kernel (support
// kappa h), for dimension DIM.
template <typename T, int DIM>
__device__ __forceinline__ T kernel_dw(int kernel, T kappa, T r, T h) {
  const T pi = T(3.14159265358979323846);
  if (kernel == SPH_KERNEL_CUBIC) {
    T ih = T(1) / h;
    T q = r * ih;
    T norm;
    if (DIM == 1) norm = T(2.0 / 3.0) * ih * ih;
    else if (DIM == 2) norm = T(10) / (T(7) * pi) * ih * ih * ih;
    else norm = ih * ih * ih * ih / pi;
    T f;
    if (q < T(1)) f = q * (T(2.25) * q - T(3));
    else if (q < T(2)) { T t = T(2) - q; f = T(-0.75) * t * t; }
    else f = T(0);
    return norm * f;
  } else {
    T H = kappa * h;
    T iH = T(1) / H;
    T s = r * iH;
    if (s >= T(1)) return T(0);
    T t = T(1) - s;
    if (DIM == 1) return T(1.25) * iH * iH * (T(-12) * s * t * t);
    T norm = (DIM == 2) ? T(7) / pi * iH * iH * iH : T(21) / (T(2) * pi) * iH * iH * iH * iH;
    return norm * (T(-20) * s * t * t * t);
  }
}

// --------------------------------------------------------------------------
// Programmatic dependent launch of a step's kernels: each is launched while
// its predecessor in the stream still runs (launch_chained), so that the
// launch overhead overlaps the predecessor.  Every kernel launched this way
// calls chain_entry() first: it waits for the predecessor's completion and
// memory (which, by the same rule one level up, implies every earlier
// kernel's), and only then lets its own successor launch.  Launched without
// the attribute, both instructions do nothing.
// --------------------------------------------------------------------------
__device__ __forceinline__ void chain_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// --------------------------------------------------------------------------
// Host helpers shared by the translation units
// --------------------------------------------------------------------------
inline int grid_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

// Message reported by sph_last_error(NULL) (entry points without a handle).
void set_global_error(const std::string& msg);

// Launchers (defined in k_step.cu, k_pair.cu, k_vd3.cu).  They enqueue on
// `st` and return the launch status.
cudaError_t launch_derive_dt(sph_handle* h, const sph_state& s, bool with_bbox, cudaStream_t st);
// from_key: the step's dt from the CFL keys that the previous step's fused second
// kick left in dt_key (else from the block partials); dt_key is reset either way
cudaError_t launch_reduce_dt(sph_handle* h, cudaStream_t st, bool from_key = false);
cudaError_t launch_kick_drift(sph_handle* h, const sph_state& s, cudaStream_t st);
// gate (Verlet mode): device flag, the mesh kernels return at once while gate[0] == 0
cudaError_t launch_build_grid(sph_handle* h, const sph_state& s, cudaStream_t st, const int* gate = nullptr);
cudaError_t launch_verlet_flag(sph_handle* h, cudaStream_t st);
// eorder: write the packs in the unit-major evaluation order of the last build (e_of_c), the
// particle of each evaluation slot (perm_e) and, at builds, the cell-order copy packAc
// list_counters: also zero the counters of the list build and list evaluation
// that follow in the step (which then need no memsets of their own)
cudaError_t launch_pack(sph_handle* h, const sph_state& s, bool predict, cudaStream_t st, bool eorder = false,
                        bool list_counters = false);
// next_dt: also leave the CFL block minima of the new state in h->part (the next
// step's dt without a k_derive pass)
cudaError_t launch_kick2(sph_handle* h, const sph_state& s, double* t_dev, cudaStream_t st, bool next_dt = false);
// order: the particle to place at each position (NULL: h->perm, the cell order of the last mesh)
cudaError_t launch_renumber(sph_handle* h, sph_state& s, cudaStream_t st, const int32_t* order = nullptr);
// rates VJP at the state packed by launch_pack (k_adjoint.cu); fp64_pairs: the
// operands were packed in FP64 by launch_pack_fp64 into adj64_* (mixed handle)
cudaError_t launch_rates_vjp(sph_handle* h, const sph_state& W, sph_state& adj, const double* dt, int predicted,
                             double* par, cudaStream_t st, bool fp64_pairs = false);
cudaError_t launch_pack_fp64(sph_handle* h, const sph_state& s, bool predict, void* A, void* B, void* C,
                             double* rho_out, cudaStream_t st);
// Exclusive scan of cnt[0, *total) into start[0, *total], start[*total] = n_total;
// cnt is zeroed; launched for up to `cap` elements.
// gate (may be NULL): the kernels return at once while gate[0] == 0
cudaError_t launch_exclusive_scan(int32_t* cnt, const int64_t* total, int32_t* sums, int32_t* start,
                                  int64_t n_total, int64_t cap, cudaStream_t st, const int* gate = nullptr);
cudaError_t launch_conservation(sph_handle* h, const sph_state& s, double* out, cudaStream_t st);
cudaError_t launch_check_finite(sph_handle* h, const sph_state& s, cudaStream_t st);
cudaError_t launch_max_volume(sph_handle* h, const sph_state& s, unsigned long long* out, cudaStream_t st);
cudaError_t launch_pair(sph_handle* h, const sph_state& s, cudaStream_t st);
// A64/B64/C64: FP64 operands replacing the handle's packs (FP64 kernel on a mixed handle)
cudaError_t launch_pair_vjp(sph_handle* h, const sph_state& s, const void* G, const void* GR2, double* out,
                            cudaStream_t st, const void* A64 = nullptr, const void* B64 = nullptr,
                            const void* C64 = nullptr);
// Verlet lists: build (k_pair over the (1 + beta) radius, returns at once unless vflag[0]) and
// the pair evaluation over the lists; both only after a launch_pack with list_counters in
// the same step, which zeroes their counters
cudaError_t launch_list_build(sph_handle* h, const sph_state& s, cudaStream_t st);
// kick2: also the second half kick of the step (and the instance time, and with
// next_dt the CFL keys of the new state), fused into the rate write
cudaError_t launch_pair_lists(sph_handle* h, const sph_state& s, cudaStream_t st, bool kick2 = false,
                              double* t_dev = nullptr, bool next_dt = false);
cudaError_t launch_assign(sph_handle* h, const sph_state& s, const double* gen, int K, int dim,
                          int32_t* unit_out, cudaStream_t st);
cudaError_t launch_unit_lists(sph_handle* h, const int32_t* unit, int32_t* unit_offsets, cudaStream_t st);
cudaError_t launch_balance(sph_handle* h, const sph_state& s, double* gen, int K, int dim,
                           const double* load, const sph_balance_params& bp, double* shift_out,
                           cudaStream_t st);
// The balancing update from statistics already on the device: stats [K x 5] (centroid, count,
// rmax), load [K] (device), the adjacency already in h->adj_bits.
cudaError_t launch_balance_given(sph_handle* h, double* gen, int K, int dim, const double* stats,
                                 const double* load, const sph_balance_params& bp, double* shift_out,
                                 cudaStream_t st);
// Evaluation order of the unit-partitioned list kernel (gated on vflag[0], at list builds only,
// unless forced): e_of_c, perm_e, unit_eoff from the cell-order slots and the units of their particles.
cudaError_t launch_eorder(sph_handle* h, const sph_state& s, cudaStream_t st, bool force = false);

}  // namespace csph
