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
};

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
// with the reciprocals above.
template <typename T, int DIM>
__device__ __forceinline__ T dw_fast(int kernel, T kappa, T r, T h) {
  const T pi = T(3.14159265358979323846);
  if (kernel == SPH_KERNEL_CUBIC) {
    const T ih = rcp_(h);
    const T q = r * ih;
    T norm;
    if (DIM == 1) norm = T(2.0 / 3.0) * ih * ih;
    else if (DIM == 2) norm = T(10.0 / (7.0 * 3.14159265358979323846)) * ih * ih * ih;
    else norm = T(1.0 / 3.14159265358979323846) * (ih * ih) * (ih * ih);
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
    if (DIM == 1) return T(1.25) * iH * iH * (T(-12) * s * t * t);
    const T norm = (DIM == 2) ? T(7) / pi * iH * iH * iH : T(21) / (T(2) * pi) * (iH * iH) * (iH * iH);
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

// One warp per home cell, lane l owning home particle start_c + chunk + l.
// Candidate test, transposed: for each neighbour row (the 3 x-consecutive
// cells at (oy, oz), contiguous in slot order) the warp takes 32 candidates
// at a time, one per lane (position relative to the home cell origin in
// mixed mode, global in FP64), and loops over the home particles, whose data
// is broadcast from shared memory.  Each lane tests its candidate against
// home particle hp; a ballot collects the accepted lanes and each writes its
// entry at the next free positions of hp's list (prefix popcount), so the
// 32 lanes are busy in every test and consecutive tests are independent.
// A list entry is 16 bits: the neighbour-cell code (ox+1) + 3 (oy+1) +
// 9 (oz+1) and the offset inside that cell.  Lists are rows of padded
// stride in shared memory; after the scan (or when some list could overflow
// during the next chunk) each lane evaluates the fluxes of its own row.
constexpr int kWarps = kPairBlock / 32;
constexpr int kRow = kListCap + 2;   // padded row stride (16-bit entries): lane rows fall in distinct banks

template <bool MIXED, int DIM, bool VJP>
__global__ void __launch_bounds__(kPairBlock, VJP ? (MIXED ? 4 : 2) : (MIXED ? 6 : 4)) k_pair(PairArgs a) {
  using P = Pair<MIXED, DIM>;
  using T = typename P::T;
  using V4 = typename P::V4;
  using V2 = typename P::V2;
  __shared__ uint16_t list[kWarps][32][kRow];               // [warp][home particle][entry]
  __shared__ V4 home[kWarps][32];                            // home particles: x, y, z, kh d (mixed) or d (FP64)
  __shared__ int32_t nb_start[kWarps][27];                   // start slot of each neighbour cell

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t total = *a.total_cells_dev;
  const V4* __restrict__ A = reinterpret_cast<const V4*>(a.A);
  const V4* __restrict__ B = reinterpret_cast<const V4*>(a.B);
  const V2* __restrict__ C = reinterpret_cast<const V2*>(a.C);
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
    nb_start[warp][lane] = in ? a.cell_start[g.cell_off + xx + (int64_t)nx * (yy + (int64_t)ny * zz)] : -1;
  }

  for (int h0 = hs; h0 < he; h0 += 32) {
    const int i = h0 + lane;
    const bool act = i < he;
    const int nh = min(32, he - h0);
    const int ii = act ? i : hs;
    const V4 Ai = A[ii];
    const T khdi = MIXED ? (T)a.kh_f * Ai.w : T(0);
    {
      V4 hv = Ai;
      if (MIXED) hv.w = khdi;
      home[warp][lane] = hv;
    }
    __syncwarp();
    int cnt = 0;
    unsigned nfull = 0, ncand = 0, nexact = 0;
    T dmax = T(0);
    const int ui = a.K > 0 ? a.slot_unit[ii] : 0;
    int last_adj = -1;
    Kahan<T> s_rho, s_fx, s_fy, s_fz, s_q;
    const V4 Bi = B[ii];
    const V2 Ci = C[ii];
    // reverse mode: i's adjoint operands and the 11 own-side sums
    const V4* __restrict__ Gp = reinterpret_cast<const V4*>(a.G);
    const V2* __restrict__ Rp = reinterpret_cast<const V2*>(a.GR2);
    V4 Gi{};
    V2 Ri{};
    if constexpr (VJP) { Gi = Gp[ii]; Ri = Rp[ii]; }
    Kahan<T> s_bx[3], s_bv[3], s_bP, s_bZ, s_bV, s_bd, s_brho;

    // Flux of the interacting pair (i, j) from i's side.  Every quantity
    // that j computes for the same pair is the exact negative (e^R, v^R, v*,
    // momentum and energy fluxes) or the exact same value (r, P*, h_ij, W'):
    // dx = (off_j - off_i) + shift is the rounded negative of j's
    // (off_i - off_j) - shift, IEEE rounding is sign-symmetric, and the sums
    // that mix i and j are written with uncontracted operations in an order
    // that is symmetric under the exchange.  So the applied fluxes are
    // antisymmetric bit for bit and momentum and energy are conserved by the
    // pair sums up to the per-particle summation.
    auto pair_flux = [&](int64_t j, int ox, int oy, int oz) {
      if (j == i) return;       // the scan keeps the self pair (r = 0); it has no flux
      const V4 Aj = A[j];
      const V4 Bj = B[j];
      const V2 Cj = C[j];
      T dx, dy, dz;
      if (MIXED) {
        dx = (Aj.x - Ai.x) + ox * dcs;
        dy = DIM >= 2 ? (Aj.y - Ai.y) + oy * dcs : T(0);
        dz = DIM >= 3 ? (Aj.z - Ai.z) + oz * dcs : T(0);
      } else {
        dx = __dsub_rn(Aj.x, Ai.x);
        dy = DIM >= 2 ? __dsub_rn(Aj.y, Ai.y) : 0.0;
        dz = DIM >= 3 ? __dsub_rn(Aj.z, Ai.z) : 0.0;
      }
      const T r2 = P::r2_of(dx, dy, dz);
      dmax = Aj.w > dmax ? Aj.w : dmax;
      if (!(r2 > T(0))) return;  // coincident particles: no direction, no flux
      const T ir = rsqrt_(r2);
      const T r = r2 * ir;
      const T ex = dx * ir, ey = dy * ir, ez = dz * ir;
      T vi = Bi.x * ex, vj = Bj.x * ex;
      if (DIM >= 2) { vi = fma_(Bi.y, ey, vi); vj = fma_(Bj.y, ey, vj); }
      if (DIM >= 3) { vi = fma_(Bi.z, ez, vi); vj = fma_(Bj.z, ez, vj); }
      const T Zi = Ci.y, Zj = Cj.y, Pi = Ci.x, Pj = Cj.x;
      const T zs = add_(Zi, Zj);
      T Ps, vs;
      if (zs > T(0)) {
        const T izs = rcp_(zs);
        Ps = mul_(add_(add_(mul_(Zj, Pi), mul_(Zi, Pj)), mul_(mul_(Zi, Zj), sub_(vi, vj))), izs);
        vs = mul_(add_(add_(mul_(Zi, vi), mul_(Zj, vj)), sub_(Pi, Pj)), izs);
      } else {
        Ps = mul_(T(0.5), add_(Pi, Pj));
        vs = mul_(T(0.5), add_(vi, vj));
      }
      const T hij = (MIXED ? (T)a.eta_half_f : (T)a.eta_half) * add_(Ai.w, Aj.w);
      const T dW = MIXED ? dw_fast<T, DIM>(a.kernel, (T)a.kappa_f, r, hij)
                         : kernel_dw<T, DIM>(a.kernel, (T)a.kappa, r, hij);
      const T F = mul_(mul_(mul_(T(2), mul_(Bi.w, Bj.w)), Ps), dW);   // momentum flux along e
      s_rho.add(Bj.w * (vi - vs) * (-dW));
      s_fx.add(mul_(F, ex));
      if (DIM >= 2) s_fy.add(mul_(F, ey));
      if (DIM >= 3) s_fz.add(mul_(F, ez));
      s_q.add(mul_(F, vs));
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
    };

    // Reverse mode of the pair's contributions (VJP = true): the derivative of
    // the pair's terms in a, drho, dE of both i and j, contracted with their
    // adjoints, with respect to i's own variables: position (through r, e and
    // W'), v (through v^R), P and Z = rho c (through the acoustic solver),
    // V = m/rho, d (through h_ij) and the rho factor of the continuity term.
    auto pair_vjp = [&](int64_t j, int ox, int oy, int oz) {
      if (j == i) return;
      const V4 Aj = A[j];
      const V4 Bj = B[j];
      const V2 Cj = C[j];
      const V4 Gj = Gp[j];
      const V2 Rj = Rp[j];
      T dx, dy, dz;
      if (MIXED) {
        dx = (Aj.x - Ai.x) + ox * dcs;
        dy = DIM >= 2 ? (Aj.y - Ai.y) + oy * dcs : T(0);
        dz = DIM >= 3 ? (Aj.z - Ai.z) + oz * dcs : T(0);
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
      const T Vi = Bi.w, Vj = Bj.w, GRi = Ri.x, rhoi = Ri.y, GRj = Rj.x, rhoj = Rj.y;
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

    auto flush = [&]() {
      nfull += (unsigned)cnt;
      for (int k = 0; k < cnt; ++k) {
        const unsigned ent = list[warp][lane][k];
        const int code = ent >> 11;
        const int oz = code / 9, oy = (code - 9 * oz) / 3, ox = code - 9 * oz - 3 * oy;
        const int64_t j = (int64_t)nb_start[warp][code] + (ent & 2047u);
        if constexpr (VJP) pair_vjp(j, ox - 1, oy - 1, oz - 1);
        else pair_flux(j, ox - 1, oy - 1, oz - 1);
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
          if (__any_sync(0xffffffffu, cnt > kListCap - 32)) {
            if (act) flush();
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
    if (act) flush();

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
      const int64_t p = a.perm[i];
      a.drho[p] = 2.0 * a.rho_slot[i] * (double)s_rho.s;
      const double im = 1.0 / a.m[p];
      a.ax[p] = (double)s_fx.s * im;
      if (DIM >= 2) a.ay[p] = (double)s_fy.s * im;
      if (DIM >= 3) a.az[p] = (double)s_fz.s * im;
      a.dE[p] = (double)s_q.s * im;
      a.dmax_nbr[p] = nfull ? (double)dmax : -1.0;
    }
    // counters and work-unit loads, aggregated per warp
    unsigned tf = __reduce_add_sync(0xffffffffu, act ? nfull : 0u);
    unsigned tc = __reduce_add_sync(0xffffffffu, ncand);
    unsigned te = __reduce_add_sync(0xffffffffu, nexact);
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
    __syncwarp();   // the home buffer is rewritten by the next chunk of home particles
  }
  __syncwarp();     // the neighbour-start buffer is rewritten by the next cell
  }
}

// Persistent grid: SMs x resident CTAs per SM, capped by the handle's
// pair_blocks_per_sm (0 = as many as fit).
template <bool MIXED, int DIM, bool VJP>
cudaError_t launch_one(const PairArgs& args, int blocks_per_sm, cudaStream_t st) {
  static int sms = 0, per_sm = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair<MIXED, DIM, VJP>, kPairBlock, 0);
    if (per_sm < 1) per_sm = 1;
  }
  const int b = (blocks_per_sm > 0 && blocks_per_sm < per_sm) ? blocks_per_sm : per_sm;
  k_pair<MIXED, DIM, VJP><<<sms * b, kPairBlock, 0, st>>>(args);
  return cudaGetLastError();
}

template <bool MIXED, bool VJP>
cudaError_t launch_dim(sph_handle* h, const PairArgs& args, cudaStream_t st) {
  const int b = h->p.pair_blocks_per_sm;
  switch (h->dp.dim) {
    case 1: return launch_one<MIXED, 1, VJP>(args, b, st);
    case 2: return launch_one<MIXED, 2, VJP>(args, b, st);
    default: return launch_one<MIXED, 3, VJP>(args, b, st);
  }
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
  return a;
}

}  // namespace

// Reverse mode over the same pair set: the mesh and packs of the state s
// (k_pack of the handle's precision) and the adjoint operands G, GR2 (slot
// order, same precision) must be in place; writes 11 doubles per particle.
cudaError_t launch_pair_vjp(sph_handle* h, const sph_state& s, const void* G, const void* GR2, double* out,
                            cudaStream_t st) {
  PairArgs a = make_args(h, s);
  a.K = 0;
  a.collect_adj = 0;
  a.pair_i = a.pair_j = nullptr;
  a.G = G;
  a.GR2 = GR2;
  a.vjp_out = out;
  cudaError_t e = cudaMemsetAsync(&h->counters[5], 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  e = h->dp.precision == SPH_PREC_MIXED ? launch_dim<true, true>(h, a, st) : launch_dim<false, true>(h, a, st);
  h->launches += 1;
  return e;
}

cudaError_t launch_pair(sph_handle* h, const sph_state& s, cudaStream_t st) {
  PairArgs a = make_args(h, s);
  cudaError_t e = cudaMemsetAsync(h->counters, 0, 3 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(&h->counters[4], 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h->profiling) {
    if (h->prof_used + 2 > h->prof_events.size()) {
      for (int k = 0; k < 64; ++k) {
        cudaEvent_t ev;
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return e;
        h->prof_events.push_back(ev);
      }
    }
    e0 = h->prof_events[h->prof_used++];
    e1 = h->prof_events[h->prof_used++];
    e = cudaEventRecord(e0, st);
    if (e != cudaSuccess) return e;
  }
  e = h->dp.precision == SPH_PREC_MIXED ? launch_dim<true, false>(h, a, st) : launch_dim<false, false>(h, a, st);
  h->launches += 1;
  if (e == cudaSuccess && h->profiling) e = cudaEventRecord(e1, st);
  return e;
}

}  // namespace csph
