// pair_common.cuh -- shared by the pair kernels (k_pair.cu: the cell search
// and its modes; k_pair_lists.cu: the evaluation over the Verlet lists): the
// launch arguments, the arithmetic helpers, the pair flux accumulator FwdAcc
// and the host-side argument set-up.  Everything has internal linkage (an
// unnamed namespace), so each translation unit holds its own copy.
#pragma once

#include "csph_internal.cuh"
#include "step_math.cuh"

namespace csph {

namespace {

struct PairArgs {
  int64_t n;
  const int64_t* total_cells_dev;
  int64_t total_cells;   // read from total_cells_dev by the kernel
  int n_inst;
  const int64_t* inst_off;
  const GridInfo* grid;
  const void* A;
  const void* B;
  const void* C;
  const double* rho_slot;
  const int32_t* slot_cell;
  const int32_t* slot_unit;
  const int32_t* cell_start;
  const int32_t* perm;
  // FP64 state for the exact fallback test
  const double *x, *y, *z, *d;
  const double* m;
  // outputs, particle order
  double *ax, *ay, *az, *drho, *dE;
  double* dmax_nbr;
  // work units
  int K;
  unsigned long long* load_acc;
  uint32_t* adj_bits;
  int adj_words;  // 32-bit words per row
  unsigned long long* counters;
  int* status;
  unsigned long long* work_counter;   // next cell for the persistent warps (zeroed per launch)
  const int* vinst;                    // list build: the instances rebuilt in this step, or NULL (all)
  int collect_adj;   // record unit adjacency in this evaluation
  int load_timed;    // unit loads in SM cycles (SPH_LOAD_TIME) instead of pair counts
  int32_t* pair_i;   // optional unordered pair output (particle indices, i < j)
  int32_t* pair_j;
  int64_t pair_cap;
  double kh;
  float kh_f, eta_half_f, kappa_f;
  double eta_half, kappa;
  int kernel;
  // reverse mode (k_pair<..., VJP = true>): adjoint operands in slot order,
  // G = ((dL/da)/m, (dL/ddE)/m), GR2 = (dL/ddrho, rho), and the 11 own-side
  // derivatives per particle (particle order) it writes
  const void* G;
  const void* GR2;
  double* vjp_out;
  // Verlet lists (k_pair in list mode writes them, k_pair_lists reads them)
  uint32_t* vlist;   // [n][vcap]: (slot j << 5) | neighbour-cell code, particle-major
  int32_t* vcnt;
  double* vref;      // x, y, z, d per particle at the build (4 arrays of n)
  int* vflag;        // [0] rebuild now, [1] lists invalid, [2] builds done
  int vcap;
  // order-2 reconstruction: SPH gradients in slot order, the kernel's precision;
  // gP: grad P; gV: grad v_x, grad v_y, grad v_z (three arrays of n, consecutive)
  void* gP;
  void* gV;
  // mixed precision: the packed volume is V' = V vscale and W' is used as
  // W'' = W' wscale (both powers of two chosen by sph_init), so that the FP32
  // products stay in the normal range at any length scale; fscale =
  // 2 / (vscale^2 wscale) undoes them in FP64 and applies the factor 2 of the
  // momentum and energy fluxes, rscale = 1 / (vscale wscale),
  // vinv = 1 / vscale.  In FP64 mode the scales are 1 (fscale 2).
  float wscale_f;
  double fscale, rscale, vinv;
  // second half kick fused into the list kernel's rate write (k_pair_lists):
  // v, rho, E advanced by dt/2 with the new rates (the arithmetic of k_kick2),
  // the instance time advanced by dt, and with kick2_cfl the CFL keys of the
  // new state min-reduced into dt_key[instance] for the next step
  int kick2, kick2_cfl;
  double *kx_vx, *kx_vy, *kx_vz, *kx_rho, *kx_E;
  const int32_t* kx_mat;
  const double* kx_dt;
  double* kx_t;
  long long* dt_key;
  DevParams dp;
  // unit-partitioned list evaluation (evaluation order): e_of_c maps a
  // cell-order slot to its evaluation slot (NULL: the two orders coincide),
  // Ac holds the position / size operand in cell order for the list build;
  // unit_sched > 0: warps drain per-unit queues (unit_q) over the units'
  // evaluation ranges (unit_eoff), with stealing when unit_sched == 1;
  // unit_t receives each unit's first group start and last group end
  const int32_t* e_of_c;
  const void* Ac;
  const int32_t* unit_eoff;
  unsigned long long* unit_q;
  unsigned long long* unit_t;
  int unit_sched;
};

constexpr int kModeFwd = 0;    // rates
constexpr int kModeVjp = 1;    // reverse mode of the rates
constexpr int kModeList = 2;   // Verlet list build over the (1 + beta) radius
constexpr int kModeGrad = 3;   // SPH gradients of P and v (order-2 reconstruction)
constexpr int kModeFwd2 = 4;   // rates with states reconstructed to the pair midpoint

template <bool MIXED>
struct Ops;

// Packed operands per slot: A = (x, y, z, d), B = (v, V = m/rho), C = (P, Z = rho c)
// and, mixed, the reference velocity of B's relative velocity (k_pack).
template <>
struct Ops<true> {
  using T = float;
  using V4 = float4;
  using V2 = float2;
  using VC = float4;   // P, Z, reference velocity (x and y in one word, z)
};

template <>
struct Ops<false> {
  using T = double;
  using V4 = D4;
  using V2 = D2;
  using VC = D2;       // P, Z
};

// Reference velocities of the mixed packs: B holds v - k with k the whole-m/s
// reference of the particle, C.z holds k_x + 32768 and k_y + 32768 in its low
// and high halves, C.w holds k_z as a float.  ref_x / ref_y give
// 2^23 + k + 32768 exactly, so the difference of two particles' values is the
// exact difference of their references.
__device__ __forceinline__ float ref_x(float w) { return __int_as_float(__byte_perm(__float_as_int(w), 0x4B00, 0x5410)); }
__device__ __forceinline__ float ref_y(float w) { return __int_as_float(__byte_perm(__float_as_int(w), 0x4B00, 0x5432)); }
// Component c of a mixed pack's reference velocity (m/s, exact).
__device__ __forceinline__ float ref_v(const float4& C, int c) {
  return c == 0 ? ref_x(C.z) - 8421376.0f : (c == 1 ? ref_y(C.z) - 8421376.0f : C.w);
}
// Component c of v_j - v_i from mixed packs: the relative velocities' difference
// plus the exact difference of the references (negated exactly when i and j swap).
__device__ __forceinline__ float dvel(float bi, float bj, const float4& Ci, const float4& Cj, int c) {
  const float du = c == 0 ? ref_x(Cj.z) - ref_x(Ci.z) : (c == 1 ? ref_y(Cj.z) - ref_y(Ci.z) : Cj.w - Ci.w);
  return __fadd_rn(__fsub_rn(bj, bi), du);
}

template <typename T>
struct Kahan {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T v) {
    T y = v - c;
    T t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

template <>
struct Kahan<double> {  // FP64 sums need no compensation at these sizes
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
};

// Reciprocal and reciprocal square root: FP32 uses the fast hardware
// approximations (relative error ~1e-7, far inside the 1e-4 tolerance of the
// mixed path); FP64 keeps correctly rounded operations.
__device__ __forceinline__ float rcp_(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }

__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

// Uncontracted arithmetic for the expressions whose exchange symmetry must
// hold bit for bit (the compiler may not fuse these into FMAs).
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }

// Paired FP32 arithmetic (Blackwell's FADD2 / FMUL2 / FFMA2: two independent
// single-precision operations in one instruction, each rounded to nearest
// exactly as the scalar operation would be).  The mixed pair loop is bound by
// instruction issue, so pairing the x and y components, the independent rate
// terms and the Kahan sums cuts its instruction count while every component
// keeps the scalar code's bits.  a - b is formed as b * (-1) + a, one
// rounding, as the scalar subtraction.  Pairs are formed where both halves
// already sit in adjacent registers (the x, y of a loaded float4, a pair of
// running sums): joining two unrelated scalars costs register moves that
// measured as much as the operation saved.
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// Two independent Kahan sums carried in the halves of paired operations.
struct Kahan2 {
  float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
  __device__ __forceinline__ void add(float2 v) {
    const float2 y = sub2(v, c);
    const float2 t = add2(s, y);
    c = sub2(sub2(t, s), y);
    s = t;
  }
};

// Exact FP64 interaction test on the global positions, operation order of the oracle.
__device__ __forceinline__ bool exact_accept(const PairArgs& a, int dim, int64_t pi, int64_t pj) {
  double dx = __dsub_rn(a.x[pj], a.x[pi]);
  double r2 = __dmul_rn(dx, dx);
  if (dim >= 2) { double dy = __dsub_rn(a.y[pj], a.y[pi]); r2 = __dadd_rn(r2, __dmul_rn(dy, dy)); }
  if (dim >= 3) { double dz = __dsub_rn(a.z[pj], a.z[pi]); r2 = __dadd_rn(r2, __dmul_rn(dz, dz)); }
  double R = __dmul_rn(a.kh, __dadd_rn(a.d[pi], a.d[pj]));
  return r2 < __dmul_rn(R, R);
}

// dW/dr of the cubic spline (support 2h) or Wendland C2 (support kappa h)
// with the reciprocals above, times ws, a power of two folded into the
// normalisation constant (so the result is exactly ws times the unscaled
// value: the mixed path's W'' = W' wscale at no extra multiply).
template <typename T, int DIM, int KERN = -1>
__device__ __forceinline__ T dw_fast(int kernel, T kappa, T r, T h, T ws) {
  const T pi = T(3.14159265358979323846);
  // KERN >= 0: the kernel fixed at compile time (one branch compiled); -1: chosen at run time
  const bool cubic = KERN >= 0 ? KERN == SPH_KERNEL_CUBIC : kernel == SPH_KERNEL_CUBIC;
  if (cubic) {
    const T ih = rcp_(h);
    const T q = r * ih;
    T norm;
    if (DIM == 1) norm = (T(2.0 / 3.0) * ws) * ih * ih;
    else if (DIM == 2) norm = (T(10.0 / (7.0 * 3.14159265358979323846)) * ws) * ih * ih * ih;
    else norm = (T(1.0 / 3.14159265358979323846) * ws) * (ih * ih) * (ih * ih);
    const T t = T(2) - q;
    const T f_in = q * (T(2.25) * q - T(3));
    const T f_out = T(-0.75) * t * t;
    const T f = q < T(1) ? f_in : (q < T(2) ? f_out : T(0));   // selects, no divergence
    return norm * f;
  } else {
    const T iH = rcp_(kappa * h);
    const T s = r * iH;
    if (s >= T(1)) return T(0);
    const T t = T(1) - s;
    if (DIM == 1) return (T(1.25) * ws) * iH * iH * (T(-12) * s * t * t);
    const T norm = (DIM == 2) ? (T(7) / pi * ws) * iH * iH * iH : (T(21) / (T(2) * pi) * ws) * (iH * iH) * (iH * iH);
    return norm * (T(-20) * s * t * t * t);
  }
}

// Cubic spline W'(r, h) = s h^-(D+1) g(q) and its derivatives
// dW'/dr = s h^-(D+2) g'(q), dW'/dh = s h^-(D+2) (-(D+1) g - q g'), q = r/h.
template <typename T, int DIM>
__device__ __forceinline__ void cubic_dw3(T r, T h, T& w, T& wr, T& wh) {
  const T ih = rcp_(h);
  const T q = r * ih;
  T norm;
  if (DIM == 1) norm = T(2.0 / 3.0) * ih * ih;
  else if (DIM == 2) norm = T(10.0 / (7.0 * 3.14159265358979323846)) * ih * ih * ih;
  else norm = T(1.0 / 3.14159265358979323846) * (ih * ih) * (ih * ih);
  const T t = T(2) - q;
  const T g = q < T(1) ? q * (T(2.25) * q - T(3)) : (q < T(2) ? T(-0.75) * t * t : T(0));
  const T gp = q < T(1) ? T(4.5) * q - T(3) : (q < T(2) ? T(1.5) * t : T(0));
  w = norm * g;
  const T nh = norm * ih;
  wr = nh * gp;
  wh = nh * (T(-(DIM + 1)) * g - q * gp);
}

template <bool MIXED, int DIM>
struct Pair {
  using T = typename Ops<MIXED>::T;
  using V4 = typename Ops<MIXED>::V4;
  using V2 = typename Ops<MIXED>::V2;
  using VC = typename Ops<MIXED>::VC;

  // Canonical separation lo -> hi.  sh: shift from i's cell to j's cell (mixed only).
  static __device__ __forceinline__ void sep(bool ilo, const V4& Ai, const V4& Aj, T sx, T sy, T sz, T& dx,
                                             T& dy, T& dz) {
    const V4& lo = ilo ? Ai : Aj;
    const V4& hi = ilo ? Aj : Ai;
    if (MIXED) {
      T s0 = ilo ? sx : -sx, s1 = ilo ? sy : -sy, s2 = ilo ? sz : -sz;
      dx = (hi.x + s0) - lo.x;
      dy = DIM >= 2 ? (hi.y + s1) - lo.y : T(0);
      dz = DIM >= 3 ? (hi.z + s2) - lo.z : T(0);
    } else {
      dx = __dsub_rn(hi.x, lo.x);
      dy = DIM >= 2 ? __dsub_rn(hi.y, lo.y) : 0.0;
      dz = DIM >= 3 ? __dsub_rn(hi.z, lo.z) : 0.0;
    }
  }

  static __device__ __forceinline__ T r2_of(T dx, T dy, T dz) {
    if (MIXED) {
      T r2 = dx * dx;
      if (DIM >= 2) r2 = fmaf(dy, dy, r2);
      if (DIM >= 3) r2 = fmaf(dz, dz, r2);
      return r2;
    } else {
      T r2 = __dmul_rn(dx, dx);
      if (DIM >= 2) r2 = __dadd_rn(r2, __dmul_rn(dy, dy));
      if (DIM >= 3) r2 = __dadd_rn(r2, __dmul_rn(dz, dz));
      return r2;
    }
  }
};

// Flux of the interacting pair (i, j) from i's side.  Every quantity
// that j computes for the same pair is the exact negative (e^R, the
// momentum flux; FP64: v^R, v* and the energy flux) or the exact same value
// (r, P*, h_ij, W'; mixed: the velocity jump (v_j - v_i) . e): dx =
// (off_j - off_i) + shift is the rounded negative of j's (off_i - off_j) -
// shift, IEEE rounding is sign-symmetric, and the sums that mix i and j are
// written with uncontracted operations in an order that is symmetric under
// the exchange.  So the momentum fluxes are antisymmetric bit for bit and
// momentum is conserved by the pair sums up to the per-particle summation.
// Mixed precision takes velocities only through differences (relative packs
// with exact whole-m/s references) and sums the energy flux as
// F (v* - v_i^R), the writer adding v_i . a_i: energy is exchanged exactly up
// to the rounding of those small terms.
//
// Order 2 (ORDER2): P and v^R are extrapolated from each particle to the pair
// midpoint with the SPH gradients, each increment limited by minmod against
// the pair jump (q_L = q_i + minmod(r e.grad q_i, q_j - q_i)/2, q_R = q_j -
// minmod(r e.grad q_j, q_j - q_i)/2, e.grad v^R = e.(grad v).e), and the
// acoustic solver takes (P_L, v_L; P_R, v_R).  Written with the same
// uncontracted, sign-symmetric operations, j's side sees exactly (P_R, P_L,
// -v_R, -v_L), so the antisymmetry is kept.
template <typename T>
__device__ __forceinline__ T minmod(T a, T b) {
  return (a > T(0) && b > T(0)) ? (a < b ? a : b) : ((a < T(0) && b < T(0)) ? (a > b ? a : b) : T(0));
}

// The energy fluxes of a mixed evaluation are summed as F_ij (v* - v_i^R);
// the rate adds v_i . a_i, which is sum_j F_ij v_i^R / m_i (v_i . e_ij =
// v_i^R), with v_i the packed velocity (relative part plus reference) in
// FP64.  Zero for FP64 packs, whose fluxes carry v* itself.
template <bool MIXED>
__device__ __forceinline__ double lab_power_of(const PairArgs& a, int64_t i, const double* acc) {
  if constexpr (MIXED) {
    const float4 Bi = reinterpret_cast<const float4*>(a.B)[i];
    const float4 Ci = reinterpret_cast<const float4*>(a.C)[i];
    return ((double)Bi.x + (double)ref_v(Ci, 0)) * acc[0] + ((double)Bi.y + (double)ref_v(Ci, 1)) * acc[1] +
           ((double)Bi.z + (double)Ci.w) * acc[2];
  } else {
    return 0.0;
  }
}

// EXTRA: also the side outputs of an evaluation, i.e. the largest neighbour
// size, the unit adjacency and the optional pair output.  Only the
// evaluations that feed a rebalance or a pair query need them, and leaving
// them out of the pair loop saves ~10 % of the list kernel.
// Per-block shared tile of the unit adjacency bits (K <= SPH_MAX_UNITS), for
// the list evaluation with side outputs: zeroed by the kernel before its
// work loop, merged into adj_bits after it.
__device__ __forceinline__ uint32_t* adj_tile() {
  __shared__ uint32_t tile[SPH_MAX_UNITS * (SPH_MAX_UNITS / 32)];
  return tile;
}

template <bool MIXED, int DIM, bool ORDER2 = false, bool HLL = false, bool EXTRA = true, int KERN = -1>
struct FwdAcc {
  using P = Pair<MIXED, DIM>;
  using T = typename P::T;
  using V4 = typename P::V4;
  using VC = typename P::VC;
  // mixed precision at order 1: the flux in paired FP32 operations
  static constexpr bool kX2 = MIXED && !ORDER2;
  Kahan<T> s_rho, s_fx, s_fy, s_fz, s_q;
  Kahan2 k_fxy, k_fzq;   // kX2: (a_x, a_y) and (a_z, E) sums in paired form, folded by fold()
  T dmax = T(0);
  int last_adj = -1;
  int uj_ld = -1;       // EXTRA: unit of the current listed neighbour, loaded with its operands
  bool adj_local = false;   // EXTRA: unit adjacency into the block's shared tile (adj_tile), not global
  V4 gPi{}, gVi[3]{};   // order 2: i's gradients (set by the caller)

  // Moves the paired sums into s_fx, s_fy, s_fz, s_q (call once, after the last pair).
  __device__ __forceinline__ void fold() {
    if constexpr (kX2) {
      s_fx.s = k_fxy.s.x; s_fx.c = k_fxy.c.x;
      s_fy.s = k_fxy.s.y; s_fy.c = k_fxy.c.y;
      s_fz.s = k_fzq.s.x; s_fz.c = k_fzq.c.x;
      s_q.s = k_fzq.s.y;  s_q.c = k_fzq.c.y;
    }
  }

  // e . g, in a fixed uncontracted order (sign-symmetric in e)
  static __device__ __forceinline__ T dot_e(const V4& g, T ex, T ey, T ez) {
    T s = mul_(g.x, ex);
    if (DIM >= 2) s = fma_(g.y, ey, s);
    if (DIM >= 3) s = fma_(g.z, ez, s);
    return s;
  }
  // e . (grad v) . e  (even in e)
  static __device__ __forceinline__ T dvv(const V4* gv, T ex, T ey, T ez) {
    T s = mul_(ex, dot_e(gv[0], ex, ey, ez));
    if (DIM >= 2) s = fma_(ey, dot_e(gv[1], ex, ey, ez), s);
    if (DIM >= 3) s = fma_(ez, dot_e(gv[2], ex, ey, ez), s);
    return s;
  }

  __device__ __forceinline__ void pair(const PairArgs& a, int64_t i, const V4& Ai, const V4& Bi, const VC& Ci,
                                       int ui, int64_t j, T sx, T sy, T sz) {
    const V4* __restrict__ A = reinterpret_cast<const V4*>(a.A);
    const V4* __restrict__ B = reinterpret_cast<const V4*>(a.B);
    const VC* __restrict__ C = reinterpret_cast<const VC*>(a.C);
    if (j == i) return;       // the scan keeps the self pair (r = 0); it has no flux
    const V4 Aj = A[j];
    const V4 Bj = B[j];
    const VC Cj = C[j];
    T dx, dy, dz;
    separation(Ai, Aj, sx, sy, sz, dx, dy, dz);
    flux_at(a, i, Ai, Bi, Ci, ui, j, Aj, Bj, Cj, dx, dy, dz, P::r2_of(dx, dy, dz));
  }

  // x_j - x_i of the flux (mixed: FP32 offsets plus the cell shift, in an
  // order that j's side negates exactly)
  static __device__ __forceinline__ void separation(const V4& Ai, const V4& Aj, T sx, T sy, T sz, T& dx, T& dy,
                                                    T& dz) {
    if constexpr (kX2) {
      const float2 dxy = add2(sub2(f2(Aj.x, Aj.y), f2(Ai.x, Ai.y)), f2(sx, sy));
      dx = dxy.x;
      dy = DIM >= 2 ? dxy.y : T(0);
      dz = DIM >= 3 ? (Aj.z - Ai.z) + sz : T(0);
    } else if (MIXED) {
      dx = (Aj.x - Ai.x) + sx;
      dy = DIM >= 2 ? (Aj.y - Ai.y) + sy : T(0);
      dz = DIM >= 3 ? (Aj.z - Ai.z) + sz : T(0);
    } else {
      dx = __dsub_rn(Aj.x, Ai.x);
      dy = DIM >= 2 ? __dsub_rn(Aj.y, Ai.y) : 0.0;
      dz = DIM >= 3 ? __dsub_rn(Aj.z, Ai.z) : 0.0;
    }
  }

  // A listed candidate j of slot i (never i itself): the interaction test of
  // the scan, then the flux of an interacting pair.  Mixed: FP32 test on the
  // flux's own separation, decided in FP64 (oracle order) within the band
  // |r^2 - (kappa h_ij)^2| <= band, where FP32 rounding could flip it; FP64:
  // the oracle's test.  Returns whether the pair interacts.
  __device__ __forceinline__ bool pair_listed(const PairArgs& a, int64_t i, const V4& Ai, const V4& Bi,
                                              const VC& Ci, int ui, int64_t j, T sx, T sy, T sz, T khdi,
                                              float band, unsigned& nexact, bool valid = true) {
    const V4* __restrict__ A = reinterpret_cast<const V4*>(a.A);
    const V4* __restrict__ B = reinterpret_cast<const V4*>(a.B);
    const VC* __restrict__ C = reinterpret_cast<const VC*>(a.C);
    const V4 Aj = A[j];
    const V4 Bj = B[j];       // requested with A[j]: most candidates interact
    const VC Cj = C[j];
    // the side outputs' unit of j, requested with the operands rather than
    // inside the branch that needs it (a dependent load per entry there)
    if constexpr (EXTRA) uj_ld = a.collect_adj ? a.slot_unit[j] : -1;
    return pair_listed_ops(a, i, Ai, Bi, Ci, ui, j, Aj, Bj, Cj, sx, sy, sz, khdi, band, nexact, valid);
  }

  // pair_listed with j's operands already at hand (staged by the caller).
  // valid = false: a lane without an entry in this chunk (its operands are a
  // stand-in); it runs the same instructions and accepts nothing.
  __device__ __forceinline__ bool pair_listed_ops(const PairArgs& a, int64_t i, const V4& Ai, const V4& Bi,
                                                  const VC& Ci, int ui, int64_t j, const V4& Aj, const V4& Bj,
                                                  const VC& Cj, T sx, T sy, T sz, T khdi, float band,
                                                  unsigned& nexact, bool valid = true) {
    T dx, dy, dz;
    separation(Ai, Aj, sx, sy, sz, dx, dy, dz);
    const T r2 = P::r2_of(dx, dy, dz);
    bool acc;
    if (MIXED) {
      const T R = fmaf((T)a.kh_f, Aj.w, khdi);
      const T diff = fmaf(-R, R, r2);
      acc = valid && diff < T(0);
      if (valid && fabsf(diff) <= band) {
        ++nexact;
        acc = exact_accept(a, DIM, a.perm[i], a.perm[j]);
      }
    } else {
      T ex, ey, ez;
      P::sep(true, Ai, Aj, T(0), T(0), T(0), ex, ey, ez);   // x_j - x_i, oracle order
      const double R = __dmul_rn(a.kh, __dadd_rn(Ai.w, Aj.w));
      acc = valid && P::r2_of(ex, ey, ez) < __dmul_rn(R, R);
    }
    if constexpr (kX2) {
      // Branch-free: every listed entry runs the flux arithmetic, and the
      // kernel derivative is set to zero where the pair does not interact
      // (such entries lie at q >= kappa, where W' vanishes anyway; the select
      // keeps the exact pair set).  With ~86 % of the entries interacting the
      // lanes would run the flux almost always; the branches and their
      // reconvergence cost more than the idle arithmetic.  The side outputs
      // (rare: a unit boundary, a pair query) keep their branch.
      flux_x2(a, Ai, Bi, Ci, Aj, Bj, Cj, dx, dy, dz, r2, acc && r2 > T(0));
      if constexpr (EXTRA) {
        if (acc) dmax = Aj.w > dmax ? Aj.w : dmax;
        if (acc && r2 > T(0)) side_outputs(a, i, ui, j);
      }
    } else {
      if (acc) flux_at(a, i, Ai, Bi, Ci, ui, j, Aj, Bj, Cj, dx, dy, dz, r2);
    }
    return acc;
  }

  // The mixed order-1 flux of flux_at below, in paired operations: the same
  // rounded operations per component, so the same bits and the same exchange
  // symmetry (e, the velocity jump and the momentum flux negate exactly on j's
  // side, P* and W' are the same bits).
  // live = false: the terms are computed with W' = 0 (and a positive stand-in
  // for r^2 = 0), so they add zeros; the caller then needs no branch.
  __device__ __forceinline__ void flux_x2(const PairArgs& a, const float4& Ai, const float4& Bi,
                                          const float4& Ci, const float4& Aj, const float4& Bj, const float4& Cj,
                                          float dx, float dy, float dz, float r2, bool live = true) {
    if (!(r2 > 0.f)) r2 = 1.f;                       // coincident particles: no direction (live is false)
    const float ir = rsqrtf(r2);
    const float r = r2 * ir;
    const float2 exy = mul2(f2(dx, dy), f2(ir, ir));
    const float ez = dz * ir;
    float Zi = Ci.y, Zj = Cj.y;
    if constexpr (HLL) { const float Zm = Zi > Zj ? Zi : Zj; Zi = Zm; Zj = Zm; }
    const float zs = add_(Zi, Zj);
    // v_j - v_i: relative packs plus the exact difference of the references
    const float2 kij = sub2(f2(ref_x(Cj.z), ref_y(Cj.z)), f2(ref_x(Ci.z), ref_y(Ci.z)));
    const float2 gxy = add2(sub2(f2(Bj.x, Bj.y), f2(Bi.x, Bi.y)), kij);
    float gR = mul_(gxy.x, exy.x);
    if (DIM >= 2) gR = fma_(gxy.y, exy.y, gR);
    if (DIM >= 3) gR = fma_(__fadd_rn(__fsub_rn(Bj.z, Bi.z), Cj.w - Ci.w), ez, gR);
    const float Pl = Ci.x, Pr = Cj.x;
    float Ps, du;                                     // P*; v* - v_i^R
    {
      // the impedance-weighted state, and the plain averages when Z_i + Z_j = 0
      // (selected, both evaluated: no branch)
      const bool zp0 = zs > 0.f;
      const float izs = rcp_(zp0 ? zs : 1.f);
      const float numP = add_(add_(mul_(Zj, Pl), mul_(Zi, Pr)), mul_(mul_(Zi, Zj), -gR));
      const float numu = add_(mul_(Zj, gR), sub_(Pl, Pr));
      Ps = zp0 ? mul_(numP, izs) : mul_(0.5f, add_(Pl, Pr));
      du = zp0 ? mul_(numu, izs) : mul_(0.5f, gR);
    }
    const float hij = a.eta_half_f * add_(Ai.w, Aj.w);
    float dW = dw_fast<float, DIM, KERN>(a.kernel, a.kappa_f, r, hij, a.wscale_f);
    dW = live ? dW : 0.f;
    // momentum flux along e, without its factor 2 (carried by fscale; exact)
    const float F = mul_(mul_(mul_(Bi.w, Bj.w), Ps), dW);
    s_rho.add(Bj.w * (-du) * (-dW));
    k_fxy.add(mul2(f2(F, F), exy));
    k_fzq.add(f2(mul_(F, ez), mul_(F, du)));
  }

  __device__ __forceinline__ void flux_at(const PairArgs& a, int64_t i, const V4& Ai, const V4& Bi, const VC& Ci,
                                          int ui, int64_t j, const V4& Aj, const V4& Bj, const VC& Cj, T dx, T dy,
                                          T dz, T r2) {
    if constexpr (EXTRA) dmax = Aj.w > dmax ? Aj.w : dmax;
    if (!(r2 > T(0))) return;  // coincident particles: no direction, no flux
    if constexpr (kX2) {
      flux_x2(a, Ai, Bi, Ci, Aj, Bj, Cj, dx, dy, dz, r2);
      side_outputs(a, i, ui, j);
      return;
    }
    const T ir = rsqrt_(r2);
    const T r = r2 * ir;
    const T ex = dx * ir, ey = dy * ir, ez = dz * ir;
    T Zi = Ci.y, Zj = Cj.y;
    // HLL with Davis speeds -+max(Z_i, Z_j) is the acoustic state with both
    // impedances set to that maximum (exchange-symmetric, so P* stays the
    // same bits on both sides)
    if constexpr (HLL) { const T Zm = Zi > Zj ? Zi : Zj; Zi = Zm; Zj = Zm; }
    const T zs = add_(Zi, Zj);
    T Ps, cr, qv;   // P*; v_i^R - v* (continuity); the velocity of the energy flux
    if constexpr (MIXED) {
      // Velocities only through differences.  g = v_j - v_i from the relative
      // packs plus the exact reference difference, gR = g . e: j's side
      // negates g and e exactly, so gR and P* are the same bits there.  The
      // energy flux is summed as F (v* - v_i^R); the writer adds v_i . a_i,
      // which is sum_j F v_i^R.
      T gR = mul_(dvel(Bi.x, Bj.x, Ci, Cj, 0), ex);
      if (DIM >= 2) gR = fma_(dvel(Bi.y, Bj.y, Ci, Cj, 1), ey, gR);
      if (DIM >= 3) gR = fma_(dvel(Bi.z, Bj.z, Ci, Cj, 2), ez, gR);
      T Pl = Ci.x, Pr = Cj.x, jump = -gR;         // jump = w_i - w_j
      T hi = T(0), hj = T(0);
      if constexpr (ORDER2) {
        const V4* __restrict__ GP = reinterpret_cast<const V4*>(a.gP);
        const V4* __restrict__ GV = reinterpret_cast<const V4*>(a.gV);
        V4 gvj[3];
        gvj[0] = GV[j];
        if (DIM >= 2) gvj[1] = GV[a.n + j];
        if (DIM >= 3) gvj[2] = GV[2 * a.n + j];
        const T dP = sub_(Pr, Pl);
        const T sPi = mul_(r, dot_e(gPi, ex, ey, ez)), sPj = mul_(r, dot_e(GP[j], ex, ey, ez));
        const T svi = mul_(r, dvv(gVi, ex, ey, ez)), svj = mul_(r, dvv(gvj, ex, ey, ez));
        Pl = add_(Ci.x, mul_(T(0.5), minmod(sPi, dP)));
        Pr = sub_(Cj.x, mul_(T(0.5), minmod(sPj, dP)));
        hi = mul_(T(0.5), minmod(svi, gR));
        hj = mul_(T(0.5), minmod(svj, gR));
        jump = add_(jump, add_(hi, hj));           // j adds the same two increments the other way round
      }
      T du;                                        // v* - v_i^R
      if (zs > T(0)) {
        const T izs = rcp_(zs);
        Ps = mul_(add_(add_(mul_(Zj, Pl), mul_(Zi, Pr)), mul_(mul_(Zi, Zj), jump)), izs);
        if constexpr (ORDER2) du = mul_(add_(add_(mul_(Zi, hi), mul_(Zj, sub_(gR, hj))), sub_(Pl, Pr)), izs);
        else du = mul_(add_(mul_(Zj, gR), sub_(Pl, Pr)), izs);
      } else {
        Ps = mul_(T(0.5), add_(Pl, Pr));
        du = ORDER2 ? mul_(T(0.5), add_(hi, sub_(gR, hj))) : mul_(T(0.5), gR);
      }
      cr = -du;
      qv = du;
    } else {
      T vi = Bi.x * ex, vj = Bj.x * ex;
      if (DIM >= 2) { vi = fma_(Bi.y, ey, vi); vj = fma_(Bj.y, ey, vj); }
      if (DIM >= 3) { vi = fma_(Bi.z, ez, vi); vj = fma_(Bj.z, ez, vj); }
      T Pi = Ci.x, Pj = Cj.x, wi = vi, wj = vj;   // states fed to the solver
      if constexpr (ORDER2) {
        const V4* __restrict__ GP = reinterpret_cast<const V4*>(a.gP);
        const V4* __restrict__ GV = reinterpret_cast<const V4*>(a.gV);
        V4 gvj[3];
        gvj[0] = GV[j];
        if (DIM >= 2) gvj[1] = GV[a.n + j];
        if (DIM >= 3) gvj[2] = GV[2 * a.n + j];
        const T dP = sub_(Pj, Pi), dv = sub_(vj, vi);
        const T sPi = mul_(r, dot_e(gPi, ex, ey, ez)), sPj = mul_(r, dot_e(GP[j], ex, ey, ez));
        const T svi = mul_(r, dvv(gVi, ex, ey, ez)), svj = mul_(r, dvv(gvj, ex, ey, ez));
        Pi = add_(Ci.x, mul_(T(0.5), minmod(sPi, dP)));
        Pj = sub_(Cj.x, mul_(T(0.5), minmod(sPj, dP)));
        wi = add_(vi, mul_(T(0.5), minmod(svi, dv)));
        wj = sub_(vj, mul_(T(0.5), minmod(svj, dv)));
      }
      T vs;
      if (zs > T(0)) {
        const T izs = rcp_(zs);
        Ps = mul_(add_(add_(mul_(Zj, Pi), mul_(Zi, Pj)), mul_(mul_(Zi, Zj), sub_(wi, wj))), izs);
        vs = mul_(add_(add_(mul_(Zi, wi), mul_(Zj, wj)), sub_(Pi, Pj)), izs);
      } else {
        Ps = mul_(T(0.5), add_(Pi, Pj));
        vs = mul_(T(0.5), add_(wi, wj));
      }
      cr = vi - vs;
      qv = vs;
    }
    const T hij = (MIXED ? (T)a.eta_half_f : (T)a.eta_half) * add_(Ai.w, Aj.w);
    const T dW = MIXED ? dw_fast<T, DIM, KERN>(a.kernel, (T)a.kappa_f, r, hij, (T)a.wscale_f)
                       : kernel_dw<T, DIM>(a.kernel, (T)a.kappa, r, hij);
    // momentum flux along e, without its factor 2 (carried by fscale; exact)
    const T F = mul_(mul_(mul_(Bi.w, Bj.w), Ps), dW);
    s_rho.add(Bj.w * cr * (-dW));
    s_fx.add(mul_(F, ex));
    if (DIM >= 2) s_fy.add(mul_(F, ey));
    if (DIM >= 3) s_fz.add(mul_(F, ez));
    s_q.add(mul_(F, qv));
    side_outputs(a, i, ui, j);
  }

  // EXTRA: the optional pair output and the unit adjacency of an interacting pair.
  __device__ __forceinline__ void side_outputs(const PairArgs& a, int64_t i, int ui, int64_t j) {
    if constexpr (!EXTRA) return;
    if (a.pair_i) {
      const int32_t pi = a.perm[i], pj = a.perm[j];
      if (pi < pj) {
        const unsigned long long q = atomicAdd(&a.counters[4], 1ull);
        if ((int64_t)q < a.pair_cap) { a.pair_i[q] = pi; a.pair_j[q] = pj; }
      }
    }
    if (a.collect_adj) {
      const int uj = uj_ld >= 0 ? uj_ld : a.slot_unit[j];
      if (uj != ui && uj != last_adj) {
        const int w = ui * a.adj_words + (uj >> 5);
        const uint32_t bit = 1u << (uj & 31);
        if (adj_local) {
          // the block's tile, merged into adj_bits once at the end: global
          // atomics on the K x K bits from every boundary entry contend on a
          // few hundred words
          uint32_t* tile = adj_tile();
          if (!(tile[w] & bit)) atomicOr(&tile[w], bit);
        } else {
          atomicOr(&a.adj_bits[w], bit);
        }
        last_adj = uj;
      }
    }
  }

  // Rates of home slot i (particle perm[i]) from the sums; nfull: its interacting pairs.
  __device__ __forceinline__ void write(const PairArgs& a, int64_t i, unsigned nfull) const {
    const int64_t p = a.perm[i];
    a.drho[p] = 2.0 * a.rho_slot[i] * ((double)s_rho.s * a.rscale);
    const double im = a.fscale / a.m[p];
    const double acc[3] = {(double)s_fx.s * im, DIM >= 2 ? (double)s_fy.s * im : 0.0,
                           DIM >= 3 ? (double)s_fz.s * im : 0.0};
    a.ax[p] = acc[0];
    if (DIM >= 2) a.ay[p] = acc[1];
    if (DIM >= 3) a.az[p] = acc[2];
    a.dE[p] = (double)s_q.s * im + lab_power_of<MIXED>(a, i, acc);
    if (EXTRA) a.dmax_nbr[p] = nfull ? (double)dmax : -1.0;
  }
};

// Pair counters and work-unit loads (full-list pairs per unit), aggregated per warp.
// With timed loads, cyc is the SM cycles the warp spent on its home chunk,
// shared evenly by the chunk's particles.
__device__ __forceinline__ void warp_counters(const PairArgs& a, bool act, unsigned nfull, unsigned ncand,
                                              unsigned nexact, int ui, int lane, unsigned cyc = 0) {
  const unsigned tf = __reduce_add_sync(0xffffffffu, act ? nfull : 0u);
  const unsigned tc = __reduce_add_sync(0xffffffffu, ncand);
  const unsigned te = __reduce_add_sync(0xffffffffu, nexact);
  if (lane == 0) {
    atomicAdd(&a.counters[0], (unsigned long long)tf);
    atomicAdd(&a.counters[1], (unsigned long long)tc);
    atomicAdd(&a.counters[2], (unsigned long long)te);
  }
  if (a.K > 0) {
    const int u0 = __shfl_sync(0xffffffffu, ui, 0);
    const unsigned nact = __popc(__ballot_sync(0xffffffffu, act));
    const unsigned mine = a.load_timed ? (nact ? cyc / nact : 0u) : nfull;
    if (__all_sync(0xffffffffu, !act || ui == u0)) {
      if (lane == 0) atomicAdd(&a.load_acc[u0], (unsigned long long)(a.load_timed ? mine * nact : tf));
    } else if (act) {
      atomicAdd(&a.load_acc[ui], (unsigned long long)mine);
    }
  }
}

constexpr int kWarps = kPairBlock / 32;

// CUDA events around a pair-kernel launch when profiling (sph_profile).
// Launches captured into a CUDA graph are not timed: a record under capture
// only orders the graph's nodes, and its event has no time to read.
cudaError_t prof_record(sph_handle* h, bool start, cudaStream_t st) {
  if (!h->profiling) return cudaSuccess;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t ce = cudaStreamIsCapturing(st, &cap);
  if (ce != cudaSuccess) return ce;
  if (cap != cudaStreamCaptureStatusNone) return cudaSuccess;
  if (start && h->prof_used + 2 > h->prof_events.size()) {
    for (int k = 0; k < 64; ++k) {
      cudaEvent_t ev;
      cudaError_t e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return e;
      h->prof_events.push_back(ev);
    }
  }
  return cudaEventRecord(h->prof_events[h->prof_used++], st);
}

PairArgs make_args(sph_handle* h, const sph_state& s) {
  PairArgs a{};
  a.n = h->n;
  a.total_cells_dev = h->total_cells;
  a.total_cells = 0;
  a.n_inst = h->n_inst;
  a.inst_off = h->inst_off;
  a.grid = h->grid;
  a.A = h->packA;
  a.B = h->packB;
  a.C = h->packC;
  a.rho_slot = h->rho_slot;
  a.slot_cell = h->slot_cell;
  a.slot_unit = h->slot_unit;
  a.cell_start = h->cell_start;
  a.perm = h->perm;
  a.x = s.x; a.y = s.y; a.z = s.z; a.d = s.d; a.m = s.m;
  a.ax = s.ax; a.ay = s.ay; a.az = s.az; a.drho = s.drho; a.dE = s.dE;
  a.dmax_nbr = h->dmax_nbr;
  a.K = h->K;
  a.load_acc = h->load_acc;
  a.adj_bits = h->adj_bits;
  a.adj_words = (h->K + 31) / 32;
  a.counters = h->counters;
  a.work_counter = &h->counters[5];
  a.vinst = nullptr;
  a.status = h->status;
  a.collect_adj = (h->K > 0 && h->collect_adj) ? 1 : 0;
  a.load_timed = h->load_timed ? 1 : 0;
  a.pair_i = h->pair_out_i;
  a.pair_j = h->pair_out_j;
  a.pair_cap = h->pair_out_cap;
  a.kh = h->dp.kh;
  a.kh_f = (float)h->dp.kh;
  a.eta_half = h->dp.eta * 0.5;
  a.eta_half_f = (float)(h->dp.eta * 0.5);
  a.kappa = h->dp.kappa;
  a.kappa_f = (float)h->dp.kappa;
  a.kernel = h->dp.kernel;
  a.vlist = h->vlist;
  a.vcnt = h->vcnt;
  a.vref = h->vref;
  a.vflag = h->vflag;
  a.vcap = h->vcap;
  a.gP = h->grad_p;
  a.gV = h->grad_v;
  a.wscale_f = (float)h->wscale;
  a.fscale = 2.0 / (h->vscale * h->vscale * h->wscale);   // with the factor 2 of the momentum flux
  a.rscale = 1.0 / (h->vscale * h->wscale);
  a.vinv = 1.0 / h->vscale;
  a.e_of_c = nullptr;       // set by the Verlet-list launchers when the units partition the work
  a.Ac = nullptr;
  a.unit_eoff = nullptr;
  a.unit_q = nullptr;
  a.unit_t = nullptr;
  a.unit_sched = SPH_SCHED_GLOBAL;
  return a;
}

}  // namespace

}  // namespace csph
