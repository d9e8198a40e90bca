// k_pair.cu -- the CSPH pair loop (Sec. 4.1-4.2): neighbour search in the
// 3^dim cells of the block B_i, acoustic pair Riemann solver, and the
// per-particle sums of eqs. (SPH:Conti), (SPH:Pulse), (SPH:Energy).
//
// One thread owns one slot i (slots are particles in cell order).  The
// thread scans the candidate slots of its neighbour cells, keeps the
// interacting ones in a private list in shared memory (16-bit entries stored
// transposed so the lanes of a warp hit distinct banks), and evaluates the
// fluxes over that list after the scan, so the flux arithmetic runs on dense,
// converged lanes instead of under the ~17% acceptance of the candidate
// test.  The list holds 128 entries; only a particle with more interacting
// neighbours flushes it early.
//
// Antisymmetry: every pair flux is evaluated in the canonical orientation
// lo -> hi (lo = the smaller slot) with the same instruction sequence from
// both sides, so the momentum flux F_ij and energy flux Q_ij that i and j
// apply are bitwise negatives of each other.
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
  int collect_adj;   // record unit adjacency in this evaluation
  int32_t* pair_i;   // optional unordered pair output (particle indices, i < j)
  int32_t* pair_j;
  int64_t pair_cap;
  double kh;
  float kh_f, eta_half_f, kappa_f;
  double eta_half, kappa;
  int kernel;
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
    T f;
    if (q < T(1)) f = q * (T(2.25) * q - T(3));
    else if (q < T(2)) { const T t = T(2) - q; f = T(-0.75) * t * t; }
    else f = T(0);
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

template <bool MIXED, int DIM>
__global__ void __launch_bounds__(kPairBlock, MIXED ? 8 : 4) k_pair(PairArgs a) {
  using P = Pair<MIXED, DIM>;
  using T = typename P::T;
  using V4 = typename P::V4;
  using V2 = typename P::V2;
  // Per-thread neighbour list, 16-bit entries: 5-bit neighbour-cell code
  // (ox, oy, oz in {-1,0,1}^3) and 11-bit offset inside that cell.
  __shared__ uint16_t list[kListCap * kPairBlock];

  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const V4* __restrict__ A = reinterpret_cast<const V4*>(a.A);
  const V4* __restrict__ B = reinterpret_cast<const V4*>(a.B);
  const V2* __restrict__ C = reinterpret_cast<const V2*>(a.C);

  int b = 0;
  if (a.n_inst > 1) {  // instance of slot i: binary search of the slot offsets
    int lo = 0, hi = a.n_inst;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (a.inst_off[mid] <= i) lo = mid; else hi = mid;
    }
    b = lo;
  }
  const GridInfo& g = a.grid[b];
  const int nx = g.dims[0], ny = g.dims[1], nz = g.dims[2];
  const int64_t lc = (int64_t)a.slot_cell[i] - g.cell_off;
  const int cx = (int)(lc % nx), cy = (int)((lc / nx) % ny), cz = (int)(lc / ((int64_t)nx * ny));
  const T dcs = MIXED ? (T)g.dc_f : T(0);
  const float band = MIXED ? 0x1p-12f * g.dc_f * g.dc_f : 0.f;

  const V4 Ai = A[i];
  const V4 Bi = B[i];
  const V2 Ci = C[i];
  const T khdi = MIXED ? (T)a.kh_f * Ai.w : T(0);
  const int lane_base = threadIdx.x;
  int cnt = 0;
  unsigned nfull = 0, ncand = 0, nexact = 0;
  T dmax = T(0);
  const int ui = a.K > 0 ? a.slot_unit[i] : 0;
  int last_adj = -1;
  Kahan<T> s_rho, s_fx, s_fy, s_fz, s_q;

  // Flux of the interacting pair (i, j), evaluated in the canonical
  // orientation lo -> hi, applied to i with i's sign.
  auto pair_flux = [&](int64_t j, int ox, int oy, int oz) {
    if (j == i) return;       // the scan keeps the self pair (r = 0); it has no flux
    const V4 Aj = A[j];
    const V4 Bj = B[j];
    const V2 Cj = C[j];
    const bool ilo = i < j;
    T dx, dy, dz;
    P::sep(ilo, Ai, Aj, ox * dcs, oy * dcs, oz * dcs, dx, dy, dz);
    const T r2 = P::r2_of(dx, dy, dz);
    dmax = Aj.w > dmax ? Aj.w : dmax;
    if (!(r2 > T(0))) return;  // coincident particles: no direction, no flux
    const T ir = rsqrt_(r2);
    const T r = r2 * ir;
    const T ex = dx * ir, ey = dy * ir, ez = dz * ir;
    const V4& Bl = ilo ? Bi : Bj;
    const V4& Bh = ilo ? Bj : Bi;
    const V2& Cl = ilo ? Ci : Cj;
    const V2& Ch = ilo ? Cj : Ci;
    T vl = Bl.x * ex, vh = Bh.x * ex;
    if (DIM >= 2) { vl += Bl.y * ey; vh += Bh.y * ey; }
    if (DIM >= 3) { vl += Bl.z * ez; vh += Bh.z * ez; }
    const T Zl = Cl.y, Zh = Ch.y, Pl = Cl.x, Ph = Ch.x;
    const T zs = Zl + Zh;
    T Ps, vs;
    if (zs > T(0)) {
      const T izs = rcp_(zs);
      Ps = (Zh * Pl + Zl * Ph + Zl * Zh * (vl - vh)) * izs;
      vs = (Zl * vl + Zh * vh + Pl - Ph) * izs;
    } else {
      Ps = T(0.5) * (Pl + Ph);
      vs = T(0.5) * (vl + vh);
    }
    const V4& Al = ilo ? Ai : Aj;
    const V4& Ah = ilo ? Aj : Ai;
    const T hij = (MIXED ? (T)a.eta_half_f : (T)a.eta_half) * (Al.w + Ah.w);
    const T dW = MIXED ? dw_fast<T, DIM>(a.kernel, (T)a.kappa_f, r, hij)
                       : kernel_dw<T, DIM>(a.kernel, (T)a.kappa, r, hij);
    const T F = T(2) * (Bl.w * Bh.w) * Ps * dW;   // momentum flux lo <- hi along e
    const T Q = F * vs;                            // energy flux
    if (ilo) {
      s_rho.add(Bj.w * (vl - vs) * (-dW));
      s_fx.add(F * ex);
      if (DIM >= 2) s_fy.add(F * ey);
      if (DIM >= 3) s_fz.add(F * ez);
      s_q.add(Q);
    } else {
      s_rho.add(Bj.w * (vs - vh) * (-dW));
      s_fx.add(-(F * ex));
      if (DIM >= 2) s_fy.add(-(F * ey));
      if (DIM >= 3) s_fz.add(-(F * ez));
      s_q.add(-Q);
    }
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

  auto rare = [&](int64_t j, int ox, int oy, int oz) {
    ++nfull;
    pair_flux(j, ox, oy, oz);
  };

  auto flush = [&]() {
    nfull += (unsigned)cnt;
    for (int k = 0; k < cnt; ++k) {
      const unsigned ent = list[k * kPairBlock + lane_base];
      const int code = ent >> 11;
      const int ox = code % 3 - 1, oy = (code / 3) % 3 - 1, oz = code / 9 - 1;
      const int64_t c = g.cell_off + (cx + ox) + (int64_t)nx * ((cy + oy) + (int64_t)ny * (cz + oz));
      pair_flux((int64_t)a.cell_start[c] + (ent & 2047u), ox, oy, oz);
    }
    cnt = 0;
  };

  for (int oz = (DIM >= 3 ? -1 : 0); oz <= (DIM >= 3 ? 1 : 0); ++oz) {
    const int zz = cz + oz;
    if (zz < 0 || zz >= nz) continue;
    for (int oy = (DIM >= 2 ? -1 : 0); oy <= (DIM >= 2 ? 1 : 0); ++oy) {
      const int yy = cy + oy;
      if (yy < 0 || yy >= ny) continue;
      for (int ox = -1; ox <= 1; ++ox) {
        const int xx = cx + ox;
        if (xx < 0 || xx >= nx) continue;
        const int64_t c = g.cell_off + xx + (int64_t)nx * (yy + (int64_t)ny * zz);
        const int s0 = a.cell_start[c], s1 = a.cell_start[c + 1];
        const int code = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
        ncand += (unsigned)(s1 - s0);
        // j's offset relative to i's cell origin minus i's offset: q + off_j
        const T qx = ox * dcs - Ai.x, qy = oy * dcs - Ai.y, qz = oz * dcs - Ai.z;
        for (int j = s0; j < s1; ++j) {
          const V4 Aj = A[j];
          bool acc;
          if (MIXED) {
            // Not the canonical orientation: the band makes the decision the
            // exact FP64 one from either side, so the set stays symmetric.
            const T dx = Aj.x + qx;
            const T dy = DIM >= 2 ? Aj.y + qy : T(0);
            const T dz = DIM >= 3 ? Aj.z + qz : T(0);
            const T r2 = P::r2_of(dx, dy, dz);
            const T R = fmaf((T)a.kh_f, Aj.w, khdi);
            const T diff = fmaf(-R, R, r2);            // r^2 - R^2
            if (fabsf(diff) > band) acc = diff < T(0);
            else {
              ++nexact;
              acc = (j == i) || exact_accept(a, DIM, a.perm[i], a.perm[j]);
            }
          } else {
            T dx, dy, dz;
            P::sep(true, Ai, Aj, T(0), T(0), T(0), dx, dy, dz);
            const T r2 = P::r2_of(dx, dy, dz);
            const double R = __dmul_rn(a.kh, __dadd_rn(Ai.w, Aj.w));
            acc = r2 < __dmul_rn(R, R);
          }
          if (acc) {
            const int off = j - s0;
            if (off < 2048) {
              list[cnt * kPairBlock + lane_base] = (uint16_t)((code << 11) | off);
              if (++cnt == kListCap) flush();
            } else {
              rare(j, ox, oy, oz);   // cell of more than 2047 particles: no list entry
            }
          }
        }
      }
    }
  }
  flush();
  nfull -= 1;   // the self pair

  const int64_t p = a.perm[i];
  a.drho[p] = 2.0 * a.rho_slot[i] * (double)s_rho.s;
  const double im = 1.0 / a.m[p];
  a.ax[p] = (double)s_fx.s * im;
  if (DIM >= 2) a.ay[p] = (double)s_fy.s * im;
  if (DIM >= 3) a.az[p] = (double)s_fz.s * im;
  a.dE[p] = (double)s_q.s * im;
  a.dmax_nbr[p] = nfull ? (double)dmax : -1.0;

  // counters and work-unit loads, aggregated per warp
  const unsigned mask = __activemask();
  const int leader = __ffs(mask) - 1;
  const int lane = threadIdx.x & 31;
  unsigned tf = __reduce_add_sync(mask, nfull);
  unsigned tc = __reduce_add_sync(mask, ncand);
  unsigned te = __reduce_add_sync(mask, nexact);
  if (lane == leader) {
    atomicAdd(&a.counters[0], (unsigned long long)tf);
    atomicAdd(&a.counters[1], (unsigned long long)tc);
    atomicAdd(&a.counters[2], (unsigned long long)te);
  }
  if (a.K > 0) {
    const int u0 = __shfl_sync(mask, ui, leader);
    if (__all_sync(mask, ui == u0)) {
      if (lane == leader) atomicAdd(&a.load_acc[u0], (unsigned long long)tf);
    } else {
      atomicAdd(&a.load_acc[ui], (unsigned long long)nfull);
    }
  }
}

template <bool MIXED>
cudaError_t launch_dim(sph_handle* h, const PairArgs& args, cudaStream_t st) {
  int g = grid_for(h->n, kPairBlock);
  switch (h->dp.dim) {
    case 1: k_pair<MIXED, 1><<<g, kPairBlock, 0, st>>>(args); break;
    case 2: k_pair<MIXED, 2><<<g, kPairBlock, 0, st>>>(args); break;
    default: k_pair<MIXED, 3><<<g, kPairBlock, 0, st>>>(args); break;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pair(sph_handle* h, const sph_state& s, cudaStream_t st) {
  PairArgs a;
  a.n = h->n;
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
  cudaError_t e = cudaMemsetAsync(h->counters, 0, 3 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(&h->counters[4], 0, sizeof(unsigned long long), st);
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
  e = h->dp.precision == SPH_PREC_MIXED ? launch_dim<true>(h, a, st) : launch_dim<false>(h, a, st);
  h->launches += 1;
  if (e == cudaSuccess && h->profiling) e = cudaEventRecord(e1, st);
  return e;
}

}  // namespace csph
