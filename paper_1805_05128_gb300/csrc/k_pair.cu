// k_pair.cu -- the CSPH pair loop (Sec. 4.1-4.2): neighbour search in the
// 3^dim cells of the block B_i, acoustic pair Riemann solver, and the
// per-particle sums of eqs. (SPH:Conti), (SPH:Pulse), (SPH:Energy).
//
// A warp handles one home cell at a time, one lane per home particle (see
// k_pair below): candidates are staged in shared memory row by row, tested
// against every lane's particle, and the interacting ones are kept in a
// per-lane list; the fluxes are evaluated over the lists, so the flux
// arithmetic runs on converged lanes instead of under the ~17% acceptance
// of the candidate test.
//
// Antisymmetry: the momentum flux F_ij e^R and energy flux Q_ij that i and
// j apply are bitwise negatives of each other (see pair_flux).
//
// Mixed precision: the candidate test and the flux run in FP32 on offsets
// from each particle's own cell origin (FP32 keeps ~7 digits of a cell edge,
// not of the domain).  The FP32 test decides r^2 < R^2 whenever r^2 lies
// outside a band of 2^-12 D^c^2 around R^2, which bounds the accumulated
// FP32 error of both sides (<= ~1e-5 D^c^2); inside the band the pair is
// decided by the FP64 test on the global positions, with the same operation
// order as the oracle, so the pair set is the FP64 one.  Per-particle sums
// are Kahan-compensated.
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
  int collect_adj;   // record unit adjacency in this evaluation
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
};

constexpr int kModeFwd = 0;    // rates
constexpr int kModeVjp = 1;    // reverse mode of the rates
constexpr int kModeList = 2;   // Verlet list build over the (1 + beta) radius
constexpr int kModeGrad = 3;   // SPH gradients of P and v (order-2 reconstruction)
constexpr int kModeFwd2 = 4;   // rates with states reconstructed to the pair midpoint

template <bool MIXED>
struct Ops;

template <>
struct Ops<true> {
  using T = float;
  using V4 = float4;
  using V2 = float2;
};

template <>
struct Ops<false> {
  using T = double;
  using V4 = D4;
  using V2 = D2;
};

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
template <typename T, int DIM>
__device__ __forceinline__ T dw_fast(int kernel, T kappa, T r, T h, T ws) {
  const T pi = T(3.14159265358979323846);
  if (kernel == SPH_KERNEL_CUBIC) {
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
// that j computes for the same pair is the exact negative (e^R, v^R, v*,
// momentum and energy fluxes) or the exact same value (r, P*, h_ij, W'):
// dx = (off_j - off_i) + shift is the rounded negative of j's
// (off_i - off_j) - shift, IEEE rounding is sign-symmetric, and the sums
// that mix i and j are written with uncontracted operations in an order
// that is symmetric under the exchange.  So the applied fluxes are
// antisymmetric bit for bit and momentum and energy are conserved by the
// pair sums up to the per-particle summation.
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

// EXTRA: also the side outputs of an evaluation, i.e. the largest neighbour
// size, the unit adjacency and the optional pair output.  Only the
// evaluations that feed a rebalance or a pair query need them, and leaving
// them out of the pair loop saves ~10 % of the list kernel.
template <bool MIXED, int DIM, bool ORDER2 = false, bool HLL = false, bool EXTRA = true>
struct FwdAcc {
  using P = Pair<MIXED, DIM>;
  using T = typename P::T;
  using V4 = typename P::V4;
  using V2 = typename P::V2;
  Kahan<T> s_rho, s_fx, s_fy, s_fz, s_q;
  T dmax = T(0);
  int last_adj = -1;
  V4 gPi{}, gVi[3]{};   // order 2: i's gradients (set by the caller)

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

  __device__ __forceinline__ void pair(const PairArgs& a, int64_t i, const V4& Ai, const V4& Bi, const V2& Ci,
                                       int ui, int64_t j, T sx, T sy, T sz) {
    const V4* __restrict__ A = reinterpret_cast<const V4*>(a.A);
    const V4* __restrict__ B = reinterpret_cast<const V4*>(a.B);
    const V2* __restrict__ C = reinterpret_cast<const V2*>(a.C);
    if (j == i) return;       // the scan keeps the self pair (r = 0); it has no flux
    const V4 Aj = A[j];
    const V4 Bj = B[j];
    const V2 Cj = C[j];
    T dx, dy, dz;
    separation(Ai, Aj, sx, sy, sz, dx, dy, dz);
    flux_at(a, i, Ai, Bi, Ci, ui, j, Aj, Bj, Cj, dx, dy, dz, P::r2_of(dx, dy, dz));
  }

  // x_j - x_i of the flux (mixed: FP32 offsets plus the cell shift, in an
  // order that j's side negates exactly)
  static __device__ __forceinline__ void separation(const V4& Ai, const V4& Aj, T sx, T sy, T sz, T& dx, T& dy,
                                                    T& dz) {
    if (MIXED) {
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
                                              const V2& Ci, int ui, int64_t j, T sx, T sy, T sz, T khdi,
                                              float band, unsigned& nexact) {
    const V4* __restrict__ A = reinterpret_cast<const V4*>(a.A);
    const V4* __restrict__ B = reinterpret_cast<const V4*>(a.B);
    const V2* __restrict__ C = reinterpret_cast<const V2*>(a.C);
    const V4 Aj = A[j];
    const V4 Bj = B[j];       // requested with A[j]: most candidates interact
    const V2 Cj = C[j];
    T dx, dy, dz;
    separation(Ai, Aj, sx, sy, sz, dx, dy, dz);
    const T r2 = P::r2_of(dx, dy, dz);
    bool acc;
    if (MIXED) {
      const T R = fmaf((T)a.kh_f, Aj.w, khdi);
      const T diff = fmaf(-R, R, r2);
      acc = diff < T(0);
      if (fabsf(diff) <= band) {
        ++nexact;
        acc = exact_accept(a, DIM, a.perm[i], a.perm[j]);
      }
    } else {
      T ex, ey, ez;
      P::sep(true, Ai, Aj, T(0), T(0), T(0), ex, ey, ez);   // x_j - x_i, oracle order
      const double R = __dmul_rn(a.kh, __dadd_rn(Ai.w, Aj.w));
      acc = P::r2_of(ex, ey, ez) < __dmul_rn(R, R);
    }
    if (acc) flux_at(a, i, Ai, Bi, Ci, ui, j, Aj, Bj, Cj, dx, dy, dz, r2);
    return acc;
  }

  __device__ __forceinline__ void flux_at(const PairArgs& a, int64_t i, const V4& Ai, const V4& Bi, const V2& Ci,
                                          int ui, int64_t j, const V4& Aj, const V4& Bj, const V2& Cj, T dx, T dy,
                                          T dz, T r2) {
    if constexpr (EXTRA) dmax = Aj.w > dmax ? Aj.w : dmax;
    if (!(r2 > T(0))) return;  // coincident particles: no direction, no flux
    const T ir = rsqrt_(r2);
    const T r = r2 * ir;
    const T ex = dx * ir, ey = dy * ir, ez = dz * ir;
    T vi = Bi.x * ex, vj = Bj.x * ex;
    if (DIM >= 2) { vi = fma_(Bi.y, ey, vi); vj = fma_(Bj.y, ey, vj); }
    if (DIM >= 3) { vi = fma_(Bi.z, ez, vi); vj = fma_(Bj.z, ez, vj); }
    T Zi = Ci.y, Zj = Cj.y;
    // HLL with Davis speeds -+max(Z_i, Z_j) is the acoustic state with both
    // impedances set to that maximum (exchange-symmetric, so the flux keeps
    // its bitwise antisymmetry)
    if constexpr (HLL) { const T Zm = Zi > Zj ? Zi : Zj; Zi = Zm; Zj = Zm; }
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
    const T zs = add_(Zi, Zj);
    T Ps, vs;
    if (zs > T(0)) {
      const T izs = rcp_(zs);
      Ps = mul_(add_(add_(mul_(Zj, Pi), mul_(Zi, Pj)), mul_(mul_(Zi, Zj), sub_(wi, wj))), izs);
      vs = mul_(add_(add_(mul_(Zi, wi), mul_(Zj, wj)), sub_(Pi, Pj)), izs);
    } else {
      Ps = mul_(T(0.5), add_(Pi, Pj));
      vs = mul_(T(0.5), add_(wi, wj));
    }
    const T hij = (MIXED ? (T)a.eta_half_f : (T)a.eta_half) * add_(Ai.w, Aj.w);
    const T dW = MIXED ? dw_fast<T, DIM>(a.kernel, (T)a.kappa_f, r, hij, (T)a.wscale_f)
                       : kernel_dw<T, DIM>(a.kernel, (T)a.kappa, r, hij);
    // momentum flux along e, without its factor 2 (carried by fscale; exact)
    const T F = mul_(mul_(mul_(Bi.w, Bj.w), Ps), dW);
    s_rho.add(Bj.w * (vi - vs) * (-dW));
    s_fx.add(mul_(F, ex));
    if (DIM >= 2) s_fy.add(mul_(F, ey));
    if (DIM >= 3) s_fz.add(mul_(F, ez));
    s_q.add(mul_(F, vs));
    if constexpr (!EXTRA) return;
    if (a.pair_i) {
      const int32_t pi = a.perm[i], pj = a.perm[j];
      if (pi < pj) {
        const unsigned long long q = atomicAdd(&a.counters[4], 1ull);
        if ((int64_t)q < a.pair_cap) { a.pair_i[q] = pi; a.pair_j[q] = pj; }
      }
    }
    if (a.collect_adj) {
      const int uj = a.slot_unit[j];
      if (uj != ui && uj != last_adj) {
        atomicOr(&a.adj_bits[ui * a.adj_words + (uj >> 5)], 1u << (uj & 31));
        last_adj = uj;
      }
    }
  }

  // Rates of home slot i (particle perm[i]) from the sums; nfull: its interacting pairs.
  __device__ __forceinline__ void write(const PairArgs& a, int64_t i, unsigned nfull) const {
    const int64_t p = a.perm[i];
    a.drho[p] = 2.0 * a.rho_slot[i] * ((double)s_rho.s * a.rscale);
    const double im = a.fscale / a.m[p];
    a.ax[p] = (double)s_fx.s * im;
    if (DIM >= 2) a.ay[p] = (double)s_fy.s * im;
    if (DIM >= 3) a.az[p] = (double)s_fz.s * im;
    a.dE[p] = (double)s_q.s * im;
    if (EXTRA) a.dmax_nbr[p] = nfull ? (double)dmax : -1.0;
  }
};

// Pair counters and work-unit loads (full-list pairs per unit), aggregated per warp.
__device__ __forceinline__ void warp_counters(const PairArgs& a, bool act, unsigned nfull, unsigned ncand,
                                              unsigned nexact, int ui, int lane) {
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
    if (__all_sync(0xffffffffu, !act || ui == u0)) {
      if (lane == 0) atomicAdd(&a.load_acc[u0], (unsigned long long)tf);
    } else if (act) {
      atomicAdd(&a.load_acc[ui], (unsigned long long)nfull);
    }
  }
}

// One warp per home cell, lane l owning home particle start_c + chunk + l.
// For each neighbour row (the 3 x-consecutive cells at (oy, oz), contiguous
// in slot order) the warp stages 32 candidates at a time in shared memory,
// one loaded per lane (position relative to the home cell origin in mixed
// mode, global in FP64); every lane then tests its own home particle against
// each staged candidate, a broadcast read, and appends the accepted ones to
// its list in candidate order (no ballots or shuffles in the test loop).
// A list entry is 16 bits: the neighbour-cell code (ox+1) + 3 (oy+1) +
// 9 (oz+1) and the offset inside that cell.  Lists are rows of padded
// stride in shared memory; after the scan (or when some list could overflow
// during the next chunk) each lane evaluates the fluxes of its own row.
constexpr int kWarps = kPairBlock / 32;
// List staging per home particle in shared memory: kListCap entries for the
// flux modes, kBuildCap for the list build (whose rows are flushed to the
// global lists, so a shorter row only means more frequent flushes and frees
// shared memory for more resident blocks).  Row stride: cap + 2 16-bit
// entries, an odd number of words, so lane rows fall in distinct banks.
// Measured on the 1.125M plate: rows of 64 or 96 entries with 7-8 resident
// blocks made the step 0.3-3 % slower than 128 entries with 6 blocks.
constexpr int kBuildCap = 128;
constexpr int kBuildBlocks = 6;      // resident blocks per SM of the mixed list build

template <bool MIXED, int DIM, int MODE, bool HLL = false, bool EXTRA = true>
__global__ void __launch_bounds__(kPairBlock, (MODE == kModeVjp || MODE == kModeFwd2) ? (MIXED ? 4 : 2)
                                                 : (MODE == kModeGrad ? (MIXED ? 5 : 3)
                                                 : (MODE == kModeList ? (MIXED ? kBuildBlocks : 4) : (MIXED ? 6 : 4))))
    k_pair(PairArgs a) {
  constexpr bool VJP = MODE == kModeVjp;
  constexpr bool LIST = MODE == kModeList;
  constexpr bool GRAD = MODE == kModeGrad;
  using P = Pair<MIXED, DIM>;
  using T = typename P::T;
  using V4 = typename P::V4;
  using V2 = typename P::V2;
  constexpr int kCap = MODE == kModeList ? kBuildCap : kListCap;
  __shared__ uint16_t list[kWarps][32][kCap + 2];           // [warp][home particle][entry]
  __shared__ V4 home[kWarps][LIST ? 1 : 32];                 // home particles: x, y, z, kh d (mixed) or d (FP64)
  __shared__ V4 cand[kWarps][32];                            // list build: candidates (shifted in mixed), d
  __shared__ uint16_t cand_ent[kWarps][32];                  // list build: their list entries
  __shared__ int32_t nb_start[kWarps][27];                   // start slot of each neighbour cell
  __shared__ float4 nb_tab[kWarps][27];                      // per neighbour cell: start (bits), shift x, y, z

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t total = *a.total_cells_dev;
  const V4* __restrict__ A = reinterpret_cast<const V4*>(a.A);
  const V4* __restrict__ B = reinterpret_cast<const V4*>(a.B);
  const V2* __restrict__ C = reinterpret_cast<const V2*>(a.C);
  if constexpr (LIST) {
    if (a.vflag[0] == 0) return;                 // lists still valid: nothing to build
    if (blockIdx.x == 0 && threadIdx.x == 0) { a.vflag[1] = 0; a.vflag[2] += 1; }
  }
  // Persistent warps: each takes the next cell from a global counter, so the
  // work spreads evenly whatever the mix of empty and crowded cells.
  for (;;) {
  int64_t cell_g = 0;
  if (lane == 0) cell_g = (int64_t)atomicAdd(a.work_counter, 1ull);
  cell_g = __shfl_sync(0xffffffffu, cell_g, 0);
  if (cell_g >= total) break;
  const int hs = a.cell_start[cell_g], he = a.cell_start[cell_g + 1];
  if (hs == he) continue;                                    // empty cell (warp-uniform)

  int b = 0;
  if (a.n_inst > 1) {  // instance of this cell: binary search of the slot offsets
    int lo = 0, hi = a.n_inst;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (a.inst_off[mid] <= hs) lo = mid; else hi = mid;
    }
    b = lo;
  }
  const GridInfo& g = a.grid[b];
  const int nx = g.dims[0], ny = g.dims[1], nz = g.dims[2];
  const int64_t lc = cell_g - g.cell_off;
  const int cx = (int)(lc % nx), cy = (int)((lc / nx) % ny), cz = (int)(lc / ((int64_t)nx * ny));
  const T dcs = MIXED ? (T)g.dc_f : T(0);
  const float band = MIXED ? 0x1p-12f * g.dc_f * g.dc_f : 0.f;

  // starts of the 27 neighbour cells (index (ox+1) + 3 (oy+1) + 9 (oz+1)); -1 outside the mesh
  if (lane < 27) {
    const int ox = lane % 3 - 1, oy = (lane / 3) % 3 - 1, oz = lane / 9 - 1;
    const int xx = cx + ox, yy = cy + oy, zz = cz + oz;
    const bool in = xx >= 0 && xx < nx && yy >= 0 && yy < ny && zz >= 0 && zz < nz;
    const int st0 = in ? a.cell_start[g.cell_off + xx + (int64_t)nx * (yy + (int64_t)ny * zz)] : -1;
    nb_start[warp][lane] = st0;
    // the shift from the home cell's origin to this cell's, exact (ox, oy, oz in {-1, 0, 1})
    nb_tab[warp][lane] = make_float4(__int_as_float(st0), MIXED ? (float)ox * (float)dcs : 0.f,
                                     MIXED ? (float)oy * (float)dcs : 0.f, MIXED ? (float)oz * (float)dcs : 0.f);
  }

  for (int h0 = hs; h0 < he; h0 += 32) {
    const int i = h0 + lane;
    const bool act = i < he;
    const int nh = min(32, he - h0);
    const int ii = act ? i : hs;
    const V4 Ai = A[ii];
    const T khdi = MIXED ? (T)a.kh_f * Ai.w : T(0);
    if constexpr (!LIST) {
      V4 hv = Ai;
      if (MIXED) hv.w = khdi;
      home[warp][lane] = hv;
      __syncwarp();
    }
    int cnt = 0, vc = 0;
    unsigned nfull = 0, ncand = 0, nexact = 0;
    const int ui = a.K > 0 ? a.slot_unit[ii] : 0;
    const V4 Bi = B[ii];
    const V2 Ci = C[ii];
    // reverse mode: i's adjoint operands and the 11 own-side sums
    const V4* __restrict__ Gp = reinterpret_cast<const V4*>(a.G);
    const V2* __restrict__ Rp = reinterpret_cast<const V2*>(a.GR2);
    V4 Gi{};
    V2 Ri{};
    if constexpr (VJP) { Gi = Gp[ii]; Ri = Rp[ii]; }
    Kahan<T> s_bx[3], s_bv[3], s_bP, s_bZ, s_bV, s_bd, s_brho;

    FwdAcc<MIXED, DIM, MODE == kModeFwd2, HLL, EXTRA> fw;
    if constexpr (MODE == kModeFwd2) {
      fw.gPi = reinterpret_cast<const V4*>(a.gP)[ii];
      const V4* GV = reinterpret_cast<const V4*>(a.gV);
      fw.gVi[0] = GV[ii];
      if (DIM >= 2) fw.gVi[1] = GV[a.n + ii];
      if (DIM >= 3) fw.gVi[2] = GV[2 * a.n + ii];
    }
    auto pair_flux = [&](int64_t j, T sx, T sy, T sz) { fw.pair(a, i, Ai, Bi, Ci, ui, j, sx, sy, sz); };

    // SPH gradients (GRAD): grad q_i = sum_j V_j (q_j - q_i) (-W'_ij) e^R for q = P, v_x, v_y, v_z
    T gP[3] = {T(0), T(0), T(0)}, gV[3][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
    auto pair_grad = [&](int64_t j, T sx, T sy, T sz) {
      if (j == i) return;
      const V4 Aj = A[j];
      const V4 Bj = B[j];
      const V2 Cj = C[j];
      T dx, dy, dz;
      if (MIXED) {
        dx = (Aj.x - Ai.x) + sx;
        dy = DIM >= 2 ? (Aj.y - Ai.y) + sy : T(0);
        dz = DIM >= 3 ? (Aj.z - Ai.z) + sz : T(0);
      } else {
        dx = __dsub_rn(Aj.x, Ai.x);
        dy = DIM >= 2 ? __dsub_rn(Aj.y, Ai.y) : 0.0;
        dz = DIM >= 3 ? __dsub_rn(Aj.z, Ai.z) : 0.0;
      }
      const T r2 = P::r2_of(dx, dy, dz);
      if (!(r2 > T(0))) return;
      const T ir = rsqrt_(r2);
      const T r = r2 * ir;
      const T e[3] = {dx * ir, dy * ir, dz * ir};
      const T hij = (MIXED ? (T)a.eta_half_f : (T)a.eta_half) * (Ai.w + Aj.w);
      const T w = -(MIXED ? dw_fast<T, DIM>(a.kernel, (T)a.kappa_f, r, hij, (T)a.wscale_f)
                          : kernel_dw<T, DIM>(a.kernel, (T)a.kappa, r, hij));
      const T f = Bj.w * w;
      const T dP = Cj.x - Ci.x;
      const T dv[3] = {Bj.x - Bi.x, Bj.y - Bi.y, Bj.z - Bi.z};
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        gP[b] += f * dP * e[b];
#pragma unroll
        for (int c = 0; c < DIM; ++c) gV[c][b] += f * dv[c] * e[b];
      }
    };

    // Reverse mode of the pair's contributions (VJP = true): the derivative of
    // the pair's terms in a, drho, dE of both i and j, contracted with their
    // adjoints, with respect to i's own variables: position (through r, e and
    // W'), v (through v^R), P and Z = rho c (through the acoustic solver),
    // V = m/rho, d (through h_ij) and the rho factor of the continuity term.
    auto pair_vjp = [&](int64_t j, T sx, T sy, T sz) {
      if (j == i) return;
      const V4 Aj = A[j];
      const V4 Bj = B[j];
      const V2 Cj = C[j];
      const V4 Gj = Gp[j];
      const V2 Rj = Rp[j];
      T dx, dy, dz;
      if (MIXED) {
        dx = (Aj.x - Ai.x) + sx;
        dy = DIM >= 2 ? (Aj.y - Ai.y) + sy : T(0);
        dz = DIM >= 3 ? (Aj.z - Ai.z) + sz : T(0);
      } else {
        dx = __dsub_rn(Aj.x, Ai.x);
        dy = DIM >= 2 ? __dsub_rn(Aj.y, Ai.y) : 0.0;
        dz = DIM >= 3 ? __dsub_rn(Aj.z, Ai.z) : 0.0;
      }
      const T r2 = P::r2_of(dx, dy, dz);
      if (!(r2 > T(0))) return;
      const T ir = rsqrt_(r2);
      const T r = r2 * ir;
      const T e[3] = {dx * ir, dy * ir, dz * ir};
      const T vi[3] = {Bi.x, Bi.y, Bi.z}, vj[3] = {Bj.x, Bj.y, Bj.z};
      T vRi = T(0), vRj = T(0);
#pragma unroll
      for (int q = 0; q < DIM; ++q) { vRi += vi[q] * e[q]; vRj += vj[q] * e[q]; }
      const T Zi = Ci.y, Zj = Cj.y, zs = Zi + Zj, Pi = Ci.x, Pj = Cj.x;
      T Ps, vs, izs = T(0);
      if (zs > T(0)) {
        izs = rcp_(zs);
        Ps = (Zj * Pi + Zi * Pj + Zi * Zj * (vRi - vRj)) * izs;
        vs = (Zi * vRi + Zj * vRj + Pi - Pj) * izs;
      } else {
        Ps = T(0.5) * (Pi + Pj);
        vs = T(0.5) * (vRi + vRj);
      }
      const T eh = MIXED ? (T)a.eta_half_f : (T)a.eta_half;
      const T hij = eh * (Ai.w + Aj.w);
      T W, Wr, Wh;
      cubic_dw3<T, DIM>(r, hij, W, Wr, Wh);
      const T Vi = Bi.w * (T)a.vinv, Vj = Bj.w * (T)a.vinv;     // the packed volumes are scaled
      const T GRi = Ri.x, rhoi = Ri.y, GRj = Rj.x, rhoj = Rj.y;
      const T F = T(2) * Vi * Vj * Ps * W;
      const T dA[3] = {Gi.x - Gj.x, Gi.y - Gj.y, Gi.z - Gj.z};
      const T dB = Gi.w - Gj.w;
      T gF = dB * vs, ge[3] = {T(0), T(0), T(0)};
#pragma unroll
      for (int q = 0; q < DIM; ++q) { gF += dA[q] * e[q]; ge[q] = F * dA[q]; }
      const T ti = T(2) * W * rhoi * Vj * GRi;          // continuity terms of i and of j
      const T tj = T(2) * W * rhoj * Vi * GRj;
      const T gvs = F * dB + ti - tj;
      T gvRi = -ti, gvRj = tj;
      const T gW = gF * T(2) * Vi * Vj * Ps - GRi * T(2) * rhoi * Vj * (vRi - vs) - GRj * T(2) * rhoj * Vi * (vs - vRj);
      const T gPs = gF * T(2) * Vi * Vj * W;
      s_bV.add(gF * T(2) * Vj * Ps * W - GRj * T(2) * rhoj * (vs - vRj) * W);
      s_brho.add(-(GRi * T(2) * Vj * (vRi - vs) * W));
      T gPi, gZi = T(0);
      if (zs > T(0)) {
        gPi = (gPs * Zj + gvs) * izs;
        gvRi += (gPs * Zi * Zj + gvs * Zi) * izs;
        gvRj += (gvs * Zj - gPs * Zi * Zj) * izs;
        gZi = (gPs * ((Pj + Zj * (vRi - vRj)) - Ps) + gvs * (vRi - vs)) * izs;
      } else {
        gPi = T(0.5) * gPs;
        gvRi += T(0.5) * gvs;
        gvRj += T(0.5) * gvs;
      }
      s_bP.add(gPi);
      s_bZ.add(gZi);
      T ede = T(0);
#pragma unroll
      for (int q = 0; q < DIM; ++q) {
        s_bv[q].add(gvRi * e[q]);
        ge[q] += gvRi * vi[q] + gvRj * vj[q];
        ede += ge[q] * e[q];
      }
      const T grr = gW * Wr;
#pragma unroll
      for (int q = 0; q < DIM; ++q) s_bx[q].add(-((ge[q] - ede * e[q]) * ir + grr * e[q]));
      s_bd.add(gW * Wh * eh);
    };

    // List build: the warp writes each home particle's new entries together,
    // 32 consecutive entries of one row per store (the self pair dropped by
    // a ballot, list order kept), instead of one entry of 32 rows per store.
    auto flush_lists = [&]() {
      nfull += (unsigned)cnt;
      for (int hp = 0; hp < nh; ++hp) {
        const int n = __shfl_sync(0xffffffffu, cnt, hp);
        int v0 = __shfl_sync(0xffffffffu, vc, hp);
        const int64_t ih = h0 + hp;
        for (int k0 = 0; k0 < n; k0 += 32) {
          const int k = k0 + lane;
          uint32_t word = 0;
          bool w = false;
          if (k < n) {
            const unsigned ent = list[warp][hp][k];
            const int64_t j = (int64_t)__float_as_int(nb_tab[warp][ent >> 11].x) + (ent & 2047u);
            w = j != ih;
            word = ((uint32_t)j << 5) | (ent >> 11);
          }
          const unsigned m = __ballot_sync(0xffffffffu, w);
          const int pos = v0 + __popc(m & lt);
          if (w && pos < a.vcap) a.vlist[ih * a.vcap + pos] = word;
          v0 += __popc(m);
        }
        if (lane == hp) vc = v0;
      }
      cnt = 0;
    };

    auto flush = [&]() {
      nfull += (unsigned)cnt;
      for (int k = 0; k < cnt; ++k) {
        const unsigned ent = list[warp][lane][k];
        const float4 t = nb_tab[warp][ent >> 11];
        const int64_t j = (int64_t)__float_as_int(t.x) + (ent & 2047u);
        if constexpr (VJP) {
          pair_vjp(j, (T)t.y, (T)t.z, (T)t.w);
        } else if constexpr (GRAD) {
          pair_grad(j, (T)t.y, (T)t.z, (T)t.w);
        } else {
          pair_flux(j, (T)t.y, (T)t.z, (T)t.w);
        }
      }
      cnt = 0;
    };

    for (int oz = (DIM >= 3 ? -1 : 0); oz <= (DIM >= 3 ? 1 : 0); ++oz) {
      for (int oy = (DIM >= 2 ? -1 : 0); oy <= (DIM >= 2 ? 1 : 0); ++oy) {
        const int rc = 3 * (oy + 1) + 9 * (oz + 1);     // index of the row's ox = -1 cell
        const int s_m = nb_start[warp][rc], s_0 = nb_start[warp][rc + 1], s_p = nb_start[warp][rc + 2];
        if (s_0 < 0) continue;                           // row outside the mesh
        // contiguous slot range of the row: from the first existing cell to the end of the last
        const int r0 = s_m >= 0 ? s_m : s_0;
        const int xe = s_p >= 0 ? cx + 2 : cx + 1;       // one past the last existing cell in x
        const int64_t rowc = g.cell_off + (int64_t)nx * ((cy + oy) + (int64_t)ny * (cz + oz));
        const int r1 = a.cell_start[rowc + xe];
        const int b1 = a.cell_start[rowc + cx + 1];      // end of the ox = 0 cell
        ncand += act ? (unsigned)(r1 - r0) : 0u;
        for (int base = r0; base < r1; base += 32) {
          // a chunk adds at most 32 entries to a list: flush first if one could overflow
          if (__any_sync(0xffffffffu, cnt > kCap - 32)) {
            if constexpr (LIST) flush_lists();
            else if (act) flush();
          }
          const int j = base + lane;
          const bool jv = j < r1;
          V4 S = A[jv ? j : r0];
          uint32_t ent = 0;
          if (jv) {
            const int ox = j < s_0 ? -1 : (j < b1 ? 0 : 1);
            if (MIXED) { S.x += ox * dcs; S.y += oy * dcs; S.z += oz * dcs; }
            const int off = j - (ox < 0 ? s_m : (ox == 0 ? s_0 : b1));
            if (off > 2047) set_status(a.status, SPH_ERR_CAPACITY);   // cell over 2047 particles
            ent = ((uint32_t)(rc + ox + 1) << 11) | (uint32_t)(off & 2047);
          }
          if constexpr (LIST) {
            cand[warp][lane] = S;
            cand_ent[warp][lane] = (uint16_t)ent;
            __syncwarp();
            // each lane tests its home particle against the chunk's candidates,
            // broadcast from shared memory, and appends the accepted ones to its
            // own list in candidate order
            const int nc = min(32, r1 - base);
#pragma unroll 4
            for (int c = 0; c < nc; ++c) {
              const V4 Sc = cand[warp][c];
              bool acc;
              if (MIXED) {
                const T dx = Sc.x - Ai.x;
                const T dy = DIM >= 2 ? Sc.y - Ai.y : T(0);
                const T dz = DIM >= 3 ? Sc.z - Ai.z : T(0);
                const T r2 = P::r2_of(dx, dy, dz);
                const T R = fmaf((T)a.kh_f, Sc.w, khdi);
                const T diff = fmaf(-R, R, r2);          // r^2 - R^2
                acc = diff < band;                        // superset of the (1 + beta) radius
              } else {
                T dx, dy, dz;
                P::sep(true, Ai, Sc, T(0), T(0), T(0), dx, dy, dz);   // x_j - x_i, oracle order
                const T r2 = P::r2_of(dx, dy, dz);
                const double R = __dmul_rn(a.kh, __dadd_rn(Ai.w, Sc.w));
                acc = r2 < __dmul_rn(R, R);
              }
              if (acc && act) list[warp][lane][cnt++] = cand_ent[warp][c];
            }
            __syncwarp();   // the candidate buffer is rewritten by the next chunk
          } else {
            // transposed test: each lane tests its candidate against home particle
            // hp, broadcast from shared memory; a ballot collects the accepted lanes
            // and each writes its entry at the next free position of hp's list
#pragma unroll 4
            for (int hp = 0; hp < nh; ++hp) {
              const V4 H = home[warp][hp];
              bool acc;
              if (MIXED) {
                const T dx = S.x - H.x;
                const T dy = DIM >= 2 ? S.y - H.y : T(0);
                const T dz = DIM >= 3 ? S.z - H.z : T(0);
                const T r2 = P::r2_of(dx, dy, dz);
                const T R = fmaf((T)a.kh_f, S.w, H.w);
                const T diff = fmaf(-R, R, r2);          // r^2 - R^2
                acc = diff < T(0);
                if (fabsf(diff) <= band && jv) {          // too close to call in FP32: FP64 decides
                  ++nexact;
                  acc = (j == h0 + hp) || exact_accept(a, DIM, a.perm[h0 + hp], a.perm[j]);
                }
              } else {
                T dx, dy, dz;
                P::sep(true, H, S, T(0), T(0), T(0), dx, dy, dz);   // x_j - x_i, oracle order
                const T r2 = P::r2_of(dx, dy, dz);
                const double R = __dmul_rn(a.kh, __dadd_rn(H.w, S.w));
                acc = r2 < __dmul_rn(R, R);
              }
              acc = acc && jv;
              const unsigned mask = __ballot_sync(0xffffffffu, acc);
              if (mask) {
                const int c = __shfl_sync(0xffffffffu, cnt, hp);
                if (acc) list[warp][hp][c + __popc(mask & lt)] = (uint16_t)ent;
                if (lane == hp) cnt += __popc(mask);
              }
            }
          }
        }
      }
    }
    if constexpr (LIST) flush_lists();
    else if (act) flush();

    if constexpr (GRAD) {
      if (act) {
        V4* GP = reinterpret_cast<V4*>(a.gP);
        V4* GV = reinterpret_cast<V4*>(a.gV);
        const T rs = (T)a.rscale;                      // undo the volume and W' scales (powers of two)
        V4 q{};
        q.x = gP[0] * rs; q.y = gP[1] * rs; q.z = gP[2] * rs;
        GP[i] = q;
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          V4 g{};
          g.x = gV[c][0] * rs; g.y = gV[c][1] * rs; g.z = gV[c][2] * rs;
          GV[(int64_t)c * a.n + i] = g;
        }
      }
      __syncwarp();
      continue;
    }
    if constexpr (LIST) {
      if (act) {
        if (vc > a.vcap) set_status(a.status, SPH_ERR_CAPACITY);
        a.vcnt[i] = vc < a.vcap ? vc : a.vcap;
        const int64_t p = a.perm[i];
        a.vref[p] = a.x[p];
        if (DIM >= 2) a.vref[a.n + p] = a.y[p];
        if (DIM >= 3) a.vref[2 * a.n + p] = a.z[p];
        a.vref[3 * a.n + p] = a.d[p];
      }
      __syncwarp();
      continue;
    }
    if constexpr (VJP) {
      if (act) {
        double* o = a.vjp_out + 11 * (int64_t)a.perm[i];
#pragma unroll
        for (int q = 0; q < 3; ++q) { o[q] = (double)s_bx[q].s; o[3 + q] = (double)s_bv[q].s; }
        o[6] = (double)s_bP.s;
        o[7] = (double)s_bZ.s;
        o[8] = (double)s_bV.s;
        o[9] = (double)s_bd.s;
        o[10] = (double)s_brho.s;
      }
      __syncwarp();
      continue;
    }
    if (act) {
      nfull -= 1;   // the self pair
      fw.write(a, i, nfull);
    }
    warp_counters(a, act, nfull, ncand, nexact, ui, lane);
    __syncwarp();   // the home buffer is rewritten by the next chunk of home particles
  }
  __syncwarp();     // the neighbour-start buffer is rewritten by the next cell
  }
}

// Pair evaluation over the Verlet lists: four lanes per slot i (eight slots
// per warp: the per-slot reductions and set-up are shared by eight slots, and
// a list of ~90 entries fills its lanes to the last chunk), taken in groups
// of 32 consecutive slots from a global counter.  The slot's lanes read i's
// list four entries at a time (particle-major, so the reads are contiguous);
// each lane decides its entry as k_pair does (FP32 test outside the band of
// 2^-12 D^c^2, FP64 in the oracle's operation order inside it) and, if the
// pair interacts, adds its flux to the lane's Kahan sums (FwdAcc).  Test and
// flux share the loads and the separation; about 86 % of the entries of a
// list built with beta = 0.15 interact, so the lanes whose entry does not
// are cheaper than compacting the accepted ones first.  Each lane's Kahan
// sum takes about a quarter of the slot's pairs; the slot's four sums are
// combined by a fixed butterfly, and the FP64 scaling of the rates is done
// for the 32 slots of the group at once, one slot per lane.  Offsets stay
// relative to the cells of the build and each pair's shift comes from its
// neighbour-cell code, so the fluxes keep their bitwise antisymmetry; every
// order is fixed, so results are reproducible bit for bit.

// Lanes per slot of k_pair_lists (a divisor of 32): measured on the 1.125M
// plate impact, 16 / 8 / 4 / 2 lanes per slot take 0.89 / 0.81 / 0.75 / 0.76 ms.
constexpr int kSlotLanes = 4;
constexpr int kSlotsPerWarp = 32 / kSlotLanes;

// Sum over a slot's lanes of their Kahan sums (s - c), by a fixed butterfly.
template <typename T>
__device__ __forceinline__ T slot_sum(const Kahan<T>& k) {
  T v = k.s - k.c;
#pragma unroll
  for (int o = kSlotLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <bool MIXED, int DIM, bool HLL = false, bool EXTRA = true>
__global__ void __launch_bounds__(kPairBlock, MIXED ? (EXTRA ? 6 : 7) : 4) k_pair_lists(PairArgs a) {
  using P = Pair<MIXED, DIM>;
  using T = typename P::T;
  using V4 = typename P::V4;
  using V2 = typename P::V2;
  __shared__ float res[kWarps][6][32];            // per slot of the group: sums of rho, a (3), E, and dmax
  __shared__ double res64[kWarps][6][MIXED ? 1 : 32];
  __shared__ unsigned res_n[kWarps][32];
  // unit shifts (-1, 0, 1) per axis of each neighbour-cell code; a table read
  // and three multiplies are cheaper than the integer divisions and
  // conversions of the decode, and give the same FP32 shifts bit for bit
  __shared__ float4 unit_shift[32];
  if (threadIdx.x < 32) {
    const int c = threadIdx.x;
    unit_shift[c] = make_float4((float)(c % 3 - 1), (float)((c / 3) % 3 - 1), (float)(c / 9 - 1), 0.f);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int half = lane / kSlotLanes, hl = lane % kSlotLanes;   // the slot's group of lanes, lane in it
  const unsigned hmask = (kSlotLanes == 32 ? 0xffffffffu : ((1u << kSlotLanes) - 1u)) << (half * kSlotLanes);
  const V4* __restrict__ A = reinterpret_cast<const V4*>(a.A);
  for (;;) {
    int64_t g0 = 0;
    if (lane == 0) g0 = (int64_t)atomicAdd(a.work_counter, 32ull);
    g0 = __shfl_sync(0xffffffffu, g0, 0);
    if (g0 >= a.n) break;
    const int64_t g1 = g0 + 32 < a.n ? g0 + 32 : a.n;
    int unit_run = -1;
    unsigned unit_load = 0;
    unsigned tf = 0, tc = 0, te = 0;
    // Half h of the warp takes slots g0 + 2q + h, q = 0..15.  The list reads
    // are software-pipelined: the next chunk of entries (and, across slots,
    // the next slot's first chunk and count) is requested before the current
    // one is evaluated, so the DRAM latency of the lists overlaps the L2
    // gathers and the arithmetic.  vcap >= 32, so the first chunk of any row
    // is in bounds.
    uint32_t e_pre = 0u;
    int cnt_pre = 0;
    if (g0 + half < g1) {
      e_pre = a.vlist[(g0 + half) * (int64_t)a.vcap + hl];
      cnt_pre = a.vcnt[g0 + half];
    }
    for (int q = 0; g0 + kSlotsPerWarp * q < g1; ++q) {   // warp-uniform
      const int64_t i = g0 + kSlotsPerWarp * q + half;       // this group's slot
      const bool iv = i < g1;                                // uniform in the group
      const int cnt = iv ? cnt_pre : 0;
      uint32_t e_cur = e_pre;
      if (i + kSlotsPerWarp < g1) {
        e_pre = a.vlist[(i + kSlotsPerWarp) * (int64_t)a.vcap + hl];
        cnt_pre = a.vcnt[i + kSlotsPerWarp];
      }
      const int64_t ii = iv ? i : g0;                 // a valid slot for the loads
      int b = 0;
      if (a.n_inst > 1) {
        int lo = 0, hi = a.n_inst;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (a.inst_off[mid] <= ii) lo = mid; else hi = mid;
        }
        b = lo;
      }
      const GridInfo& g = a.grid[b];
      const T dcs = MIXED ? (T)g.dc_f : T(0);
      const float band = MIXED ? 0x1p-12f * g.dc_f * g.dc_f : 0.f;
      const V4 Ai = A[ii];
      const V4 Bi = reinterpret_cast<const V4*>(a.B)[ii];
      const V2 Ci = reinterpret_cast<const V2*>(a.C)[ii];
      const T khdi = MIXED ? (T)a.kh_f * Ai.w : T(0);
      const int ui = a.K > 0 ? a.slot_unit[ii] : 0;
      const uint32_t* __restrict__ row = a.vlist + ii * (int64_t)a.vcap;
      FwdAcc<MIXED, DIM, false, HLL, EXTRA> fw;
      unsigned nacc = 0;                              // accepted pairs of i (uniform in the group)
      int cmax = cnt;                                 // chunks run by the whole warp
#pragma unroll
      for (int o = kSlotLanes; o < 32; o <<= 1) {
        const int other = __shfl_xor_sync(0xffffffffu, cmax, o);
        cmax = cmax > other ? cmax : other;
      }
      for (int base = 0; base < cmax; base += kSlotLanes) {
        const int k = base + hl;
        const bool kv = k < cnt;
        const uint32_t e = kv ? e_cur : 0u;
        if (base + kSlotLanes < cnt) e_cur = (k + kSlotLanes < cnt) ? row[k + kSlotLanes] : 0u;   // next chunk, requested now
        bool acc = false;
        if (kv) {
          T sx = T(0), sy = T(0), sz = T(0);
          if (MIXED) {
            const float4 U = unit_shift[e & 31u];
            sx = (T)U.x * dcs;
            sy = (T)U.y * dcs;
            sz = (T)U.z * dcs;
          }
          acc = fw.pair_listed(a, ii, Ai, Bi, Ci, ui, (int64_t)(e >> 5), sx, sy, sz, khdi, band, te);
        }
        nacc += __popc(__ballot_sync(0xffffffffu, acc) & hmask);
      }
      // combine the half's sums (fixed butterfly order); the rates are scaled below, per lane
      const T srho = slot_sum(fw.s_rho), sfx = slot_sum(fw.s_fx);
      const T sfy = DIM >= 2 ? slot_sum(fw.s_fy) : T(0), sfz = DIM >= 3 ? slot_sum(fw.s_fz) : T(0);
      const T sq = slot_sum(fw.s_q);
      T dm = fw.dmax;
      if constexpr (EXTRA) {
#pragma unroll
        for (int o = kSlotLanes / 2; o > 0; o >>= 1) {
          const T ot = __shfl_xor_sync(0xffffffffu, dm, o);
          dm = ot > dm ? ot : dm;
        }
      }
      if (iv) {
        if (hl == 0) {
          const int r = (int)(i - g0);
          const T vals[6] = {srho, sfx, sfy, sfz, sq, dm};
#pragma unroll
          for (int qv = 0; qv < 6; ++qv) {
            if constexpr (MIXED) res[warp][qv][r] = (float)vals[qv];
            else res64[warp][qv][r] = (double)vals[qv];
          }
          res_n[warp][r] = nacc;
          tf += nacc;
          tc += (unsigned)cnt;
        }
        if (a.K > 0) {                                 // loads per unit, flushed when the unit changes
          if (ui != unit_run && unit_run >= 0 && hl == 0 && unit_load)
            atomicAdd(&a.load_acc[unit_run], (unsigned long long)unit_load);
          if (ui != unit_run) { unit_run = ui; unit_load = 0; }
          unit_load += nacc;
        }
      }
    }
    if (a.K > 0 && hl == 0 && unit_run >= 0 && unit_load)
      atomicAdd(&a.load_acc[unit_run], (unsigned long long)unit_load);
    __syncwarp();
    {
      const int64_t i = g0 + lane;                     // one slot of the group per lane
      long long key = LLONG_MAX;
      int bi = 0;
      if (i < g1) {
        auto rv = [&](int qv) -> double {
          if constexpr (MIXED) return (double)res[warp][qv][lane];
          else return res64[warp][qv][lane];
        };
        const int64_t p = a.perm[i];
        const double drho = 2.0 * a.rho_slot[i] * (rv(0) * a.rscale);
        const double im = a.fscale / a.m[p];
        const double acc[3] = {rv(1) * im, DIM >= 2 ? rv(2) * im : 0.0, DIM >= 3 ? rv(3) * im : 0.0};
        const double dE = rv(4) * im;
        a.drho[p] = drho;
        a.ax[p] = acc[0];
        if (DIM >= 2) a.ay[p] = acc[1];
        if (DIM >= 3) a.az[p] = acc[2];
        a.dE[p] = dE;
        if (EXTRA) a.dmax_nbr[p] = res_n[warp][lane] ? rv(5) : -1.0;
        if (a.kick2) {
          if (a.n_inst > 1) {
            int lo = 0, hi = a.n_inst;
            while (hi - lo > 1) {
              const int mid = (lo + hi) >> 1;
              if (a.inst_off[mid] <= i) lo = mid; else hi = mid;
            }
            bi = lo;
          }
          const double dt = a.kx_dt[bi];
          const double hdt = 0.5 * dt;
          double* V[3] = {a.kx_vx, a.kx_vy, a.kx_vz};
          double v[3] = {0.0, 0.0, 0.0};
#pragma unroll
          for (int c = 0; c < DIM; ++c) v[c] = V[c][p];
          const double rho0 = a.kx_rho[p], E0 = a.kx_E[p];
#pragma unroll
          for (int c = 0; c < DIM; ++c) v[c] = axpy<MIXED>(hdt, acc[c], v[c]);
          const double rho = axpy<MIXED>(hdt, drho, rho0);
          const double E = axpy<MIXED>(hdt, dE, E0);
#pragma unroll
          for (int c = 0; c < DIM; ++c) V[c][p] = v[c];
          a.kx_rho[p] = rho;
          a.kx_E[p] = E;
          if (a.kx_t && i == a.inst_off[bi]) a.kx_t[bi] += dt;    // one slot per instance
          if (a.kick2_cfl) key = cfl_key(a.dp, v[0], v[1], v[2], E, rho, a.m[p], a.kx_mat ? a.kx_mat[p] : 0);
        }
      }
      if (a.kick2_cfl) {
        // one atomic per warp when the group lies in one instance (the usual case)
        const int b0 = __shfl_sync(0xffffffffu, bi, 0);
        if (__all_sync(0xffffffffu, i >= g1 || bi == b0)) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const long long q = __shfl_xor_sync(0xffffffffu, key, o);
            key = q < key ? q : key;
          }
          if (lane == 0) atomicMin(&a.dt_key[b0], key);
        } else if (i < g1) {
          atomicMin(&a.dt_key[bi], key);
        }
      }
    }
    __syncwarp();
    te = __reduce_add_sync(0xffffffffu, te);
    tf = __reduce_add_sync(0xffffffffu, tf);
    tc = __reduce_add_sync(0xffffffffu, tc);
    if (lane == 0) {
      atomicAdd(&a.counters[0], (unsigned long long)tf);
      atomicAdd(&a.counters[1], (unsigned long long)tc);
      atomicAdd(&a.counters[2], (unsigned long long)te);
    }
  }
}

// Persistent grid: SMs x resident CTAs per SM, capped by the handle's
// pair_blocks_per_sm (0 = as many as fit).
template <bool MIXED, int DIM, int MODE, bool HLL, bool EXTRA = true>
cudaError_t launch_one(const PairArgs& args, int blocks_per_sm, cudaStream_t st) {
  static int sms = 0, per_sm = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair<MIXED, DIM, MODE, HLL, EXTRA>, kPairBlock, 0);
    if (per_sm < 1) per_sm = 1;
  }
  const int b = (blocks_per_sm > 0 && blocks_per_sm < per_sm) ? blocks_per_sm : per_sm;
  k_pair<MIXED, DIM, MODE, HLL, EXTRA><<<sms * b, kPairBlock, 0, st>>>(args);
  return cudaGetLastError();
}

template <bool MIXED, int MODE, bool HLL, bool EXTRA>
cudaError_t launch_dim3(sph_handle* h, const PairArgs& args, cudaStream_t st) {
  const int b = h->p.pair_blocks_per_sm;
  switch (h->dp.dim) {
    case 1: return launch_one<MIXED, 1, MODE, HLL, EXTRA>(args, b, st);
    case 2: return launch_one<MIXED, 2, MODE, HLL, EXTRA>(args, b, st);
    default: return launch_one<MIXED, 3, MODE, HLL, EXTRA>(args, b, st);
  }
}

// The pair solver and the side outputs (neighbour sizes, unit adjacency, pair
// output) are template parameters of the flux modes: as run-time branches in
// the pair loop they cost ~1 % and ~10 % of the kernel.
template <bool MIXED, int MODE>
cudaError_t launch_dim(sph_handle* h, const PairArgs& args, cudaStream_t st) {
  constexpr bool kFlux = MODE == kModeFwd || MODE == kModeFwd2;
  if constexpr (!kFlux) {
    return launch_dim3<MIXED, MODE, false, true>(h, args, st);
  } else {
    const bool extra = args.collect_adj || args.pair_i;
    if (h->solver == SPH_SOLVER_HLL)
      return extra ? launch_dim3<MIXED, MODE, true, true>(h, args, st) : launch_dim3<MIXED, MODE, true, false>(h, args, st);
    return extra ? launch_dim3<MIXED, MODE, false, true>(h, args, st) : launch_dim3<MIXED, MODE, false, false>(h, args, st);
  }
}

template <bool MIXED, int DIM, bool HLL, bool EXTRA>
cudaError_t launch_lists_one(const PairArgs& args, int blocks_per_sm, cudaStream_t st) {
  static int sms = 0, per_sm = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair_lists<MIXED, DIM, HLL, EXTRA>, kPairBlock, 0);
    if (per_sm < 1) per_sm = 1;
  }
  const int b = (blocks_per_sm > 0 && blocks_per_sm < per_sm) ? blocks_per_sm : per_sm;
  k_pair_lists<MIXED, DIM, HLL, EXTRA><<<sms * b, kPairBlock, 0, st>>>(args);
  return cudaGetLastError();
}

template <bool MIXED, bool HLL, bool EXTRA>
cudaError_t launch_lists_dim3(sph_handle* h, const PairArgs& args, cudaStream_t st) {
  const int b = h->p.pair_blocks_per_sm;
  switch (h->dp.dim) {
    case 1: return launch_lists_one<MIXED, 1, HLL, EXTRA>(args, b, st);
    case 2: return launch_lists_one<MIXED, 2, HLL, EXTRA>(args, b, st);
    default: return launch_lists_one<MIXED, 3, HLL, EXTRA>(args, b, st);
  }
}

// The side outputs (neighbour sizes, unit adjacency, pair output) only when
// this evaluation must produce them.
template <bool MIXED>
cudaError_t launch_lists_dim(sph_handle* h, const PairArgs& args, cudaStream_t st) {
  const bool extra = args.collect_adj || args.pair_i;
  if (h->solver == SPH_SOLVER_HLL)
    return extra ? launch_lists_dim3<MIXED, true, true>(h, args, st) : launch_lists_dim3<MIXED, true, false>(h, args, st);
  return extra ? launch_lists_dim3<MIXED, false, true>(h, args, st) : launch_lists_dim3<MIXED, false, false>(h, args, st);
}

// CUDA events around a pair-kernel launch when profiling (sph_profile).
cudaError_t prof_record(sph_handle* h, bool start, cudaStream_t st) {
  if (!h->profiling) return cudaSuccess;
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
  a.status = h->status;
  a.collect_adj = (h->K > 0 && h->collect_adj) ? 1 : 0;
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
  return a;
}

}  // namespace

// Reverse mode over the same pair set: the mesh and packs of the state s
// (k_pack of the handle's precision) and the adjoint operands G, GR2 (slot
// order, same precision) must be in place; writes 11 doubles per particle.
cudaError_t launch_pair_vjp(sph_handle* h, const sph_state& s, const void* G, const void* GR2, double* out,
                            cudaStream_t st, const void* A64, const void* B64, const void* C64) {
  PairArgs a = make_args(h, s);
  a.K = 0;
  a.collect_adj = 0;
  a.pair_i = a.pair_j = nullptr;
  a.G = G;
  a.GR2 = GR2;
  a.vjp_out = out;
  const bool fp64 = A64 != nullptr || h->dp.precision != SPH_PREC_MIXED;
  if (A64) {                       // FP64 operands of a mixed handle: unscaled volumes
    a.A = A64;
    a.B = B64;
    a.C = C64;
    a.vinv = 1.0;
  }
  cudaError_t e = cudaMemsetAsync(&h->counters[5], 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  e = fp64 ? launch_dim<false, kModeVjp>(h, a, st) : launch_dim<true, kModeVjp>(h, a, st);
  h->launches += 1;
  return e;
}

// Verlet list build: the pair kernel over the radius (1 + beta) kappa h_ij;
// returns at once on the device unless vflag[0] is set.
cudaError_t launch_list_build(sph_handle* h, const sph_state& s, cudaStream_t st) {
  PairArgs a = make_args(h, s);
  a.K = 0;
  a.collect_adj = 0;
  a.pair_i = a.pair_j = nullptr;
  const double khl = h->dp.kh * (1.0 + h->dp.cell_beta);
  a.kh = khl;
  a.kh_f = (float)khl;
  cudaError_t e = cudaMemsetAsync(&h->counters[5], 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  e = h->dp.precision == SPH_PREC_MIXED ? launch_dim<true, kModeList>(h, a, st)
                                        : launch_dim<false, kModeList>(h, a, st);
  h->launches += 1;
  return e;
}

// Pair evaluation over the Verlet lists (rates, counters, unit loads).
cudaError_t launch_pair_lists(sph_handle* h, const sph_state& s, cudaStream_t st, bool kick2, double* t_dev,
                              bool next_dt) {
  PairArgs a = make_args(h, s);
  a.kick2 = kick2 ? 1 : 0;
  a.kick2_cfl = kick2 && next_dt ? 1 : 0;
  a.kx_vx = s.vx;
  a.kx_vy = s.vy;
  a.kx_vz = s.vz;
  a.kx_rho = s.rho;
  a.kx_E = s.E;
  a.kx_mat = s.mat;
  a.kx_dt = h->dt;
  a.kx_t = t_dev;
  a.dt_key = h->dt_key;
  a.dp = h->dp;
  cudaError_t e = cudaMemsetAsync(h->counters, 0, 3 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(&h->counters[5], 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if ((e = prof_record(h, true, st)) != cudaSuccess) return e;
  e = h->dp.precision == SPH_PREC_MIXED ? launch_lists_dim<true>(h, a, st) : launch_lists_dim<false>(h, a, st);
  h->launches += 1;
  if (e == cudaSuccess) e = prof_record(h, false, st);
  return e;
}

cudaError_t launch_pair(sph_handle* h, const sph_state& s, cudaStream_t st) {
  PairArgs a = make_args(h, s);
  cudaError_t e = cudaMemsetAsync(h->counters, 0, 3 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(&h->counters[4], 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (h->order2) {
    // SPH gradients first (their own pass over the same pair set), then the rates
    a.gP = h->grad_p;
    a.gV = h->grad_v;
    e = h->dp.precision == SPH_PREC_MIXED ? launch_dim<true, kModeGrad>(h, a, st)
                                          : launch_dim<false, kModeGrad>(h, a, st);
    h->launches += 1;
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&h->counters[5], 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  if ((e = prof_record(h, true, st)) != cudaSuccess) return e;
  if (h->order2)
    e = h->dp.precision == SPH_PREC_MIXED ? launch_dim<true, kModeFwd2>(h, a, st)
                                          : launch_dim<false, kModeFwd2>(h, a, st);
  else
    e = h->dp.precision == SPH_PREC_MIXED ? launch_dim<true, kModeFwd>(h, a, st)
                                          : launch_dim<false, kModeFwd>(h, a, st);
  h->launches += 1;
  if (e == cudaSuccess) e = prof_record(h, false, st);
  return e;
}

}  // namespace csph
