// k_vd3.cu -- Voronoi dynamic decomposition recast as the work-unit
// partition of one GPU (Secs. 3.1-3.4, 4.3): nearest-generator assignment,
// stable per-unit particle lists, per-unit statistics (centroid, D^sh) and
// the balancing update of the generators.
#include <cfloat>
#include <mutex>
#include <string>

#include "csph_internal.cuh"

namespace csph {

namespace {

constexpr int kUnitBlock = 1024;   // particles per block of the unit partition kernels

// ---------------------------------------------------------------------------
// Nearest generator, eq. (VoronoiDefinition), ties to the smaller index.
// FP32 pass on offsets from the generators' mean o: with M = max(|x - o|_inf,
// max_k |g_k - o|_inf) each squared distance carries an error below
// dim M^2 2^-19; every k within 3 such bounds of the FP32 minimum is then
// re-evaluated in FP64 with the oracle's operation order (dx = x - g,
// squares summed in axis order), the smallest with strict < winning.
// ---------------------------------------------------------------------------
// The block's prologue (the generators' mean o, per axis in index order; their
// FP32 offsets and the largest of them) is shared out over the threads, and a
// capped grid strides over the particles, so that it runs once per resident
// block: done serially by one thread in every block of a one-particle-per-
// thread grid, its FP64 chain dominated the kernel.
template <int DIM>
__global__ void k_assign(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                         const double* __restrict__ z, const double* __restrict__ gen, int K,
                         int32_t* unit, unsigned long long* n_exact) {
  __shared__ double gd[SPH_MAX_UNITS * 3];
  __shared__ float gf[SPH_MAX_UNITS * 3];
  __shared__ double org[3];
  __shared__ float gred[kBlock / 32];
  for (int k = threadIdx.x; k < K * DIM; k += blockDim.x) gd[k] = gen[k];
  __syncthreads();
  if (threadIdx.x < DIM) {
    const int a = threadIdx.x;
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += gd[k * DIM + a];
    org[a] = s / K;
  }
  __syncthreads();
  float gm = 0.f;
  for (int k = threadIdx.x; k < K * DIM; k += blockDim.x) {
    const float v = (float)(gd[k] - org[k % DIM]);
    gf[k] = v;
    gm = fmaxf(gm, fabsf(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
  if ((threadIdx.x & 31) == 0) gred[threadIdx.x >> 5] = gm;
  __syncthreads();
  float gmax = 0.f;
  for (int w = 0; w < kBlock / 32; ++w) gmax = fmaxf(gmax, gred[w]);
  const double* X[3] = {x, y, z};
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    float xf[3] = {0.f, 0.f, 0.f};
    float M = gmax;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      xf[a] = (float)(X[a][p] - org[a]);
      M = fmaxf(M, fabsf(xf[a]));
    }
    // inflate M by a relative 2^-20 for the rounding of M itself
    M = M * (1.0f + 0x1p-20f);
    const float B = (float)DIM * M * M * 0x1p-19f;
    float best = FLT_MAX;
    for (int k = 0; k < K; ++k) {
      float d2 = 0.f;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        float t = xf[a] - gf[k * DIM + a];
        d2 = fmaf(t, t, d2);
      }
      best = fminf(best, d2);
    }
    const float lim = best + 3.0f * B;
    int first = -1, ncand = 0;
    for (int k = 0; k < K; ++k) {
      float d2 = 0.f;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        float t = xf[a] - gf[k * DIM + a];
        d2 = fmaf(t, t, d2);
      }
      if (d2 <= lim) {
        if (first < 0) first = k;
        ++ncand;
      }
    }
    int win = first;
    if (ncand > 1) {
      atomicAdd(n_exact, 1ull);
      double bd = DBL_MAX;
      for (int k = first; k < K; ++k) {
        float d2f = 0.f;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          float t = xf[a] - gf[k * DIM + a];
          d2f = fmaf(t, t, d2f);
        }
        if (d2f > lim) continue;
        double dx = __dsub_rn(X[0][p], gd[k * DIM + 0]);
        double d2 = __dmul_rn(dx, dx);
        if (DIM >= 2) { double dy = __dsub_rn(X[1][p], gd[k * DIM + 1]); d2 = __dadd_rn(d2, __dmul_rn(dy, dy)); }
        if (DIM >= 3) { double dz = __dsub_rn(X[2][p], gd[k * DIM + 2]); d2 = __dadd_rn(d2, __dmul_rn(dz, dz)); }
        if (d2 < bd) { bd = d2; win = k; }
      }
    }
    unit[p] = win < 0 ? 0 : win;   // no candidate only for non-finite input (latched elsewhere)
  }
}

// Grid of the assignment: particles in blocks of kBlock, at most 8 resident
// blocks' worth per SM (the blocks stride over the rest).
int assign_grid(int64_t n) {
  static int cap = 0;
  if (cap == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cap = 8 * (sms > 0 ? sms : 1);
  }
  const int64_t want = (n + kBlock - 1) / kBlock;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

cudaError_t launch_assign_kernel(int64_t n, int dim, const double* x, const double* y, const double* z,
                                 const double* gen, int K, int32_t* unit, unsigned long long* n_exact,
                                 cudaStream_t st) {
  const int g = assign_grid(n);
  if (dim == 1) k_assign<1><<<g, kBlock, 0, st>>>(n, x, y, z, gen, K, unit, n_exact);
  else if (dim == 2) k_assign<2><<<g, kBlock, 0, st>>>(n, x, y, z, gen, K, unit, n_exact);
  else k_assign<3><<<g, kBlock, 0, st>>>(n, x, y, z, gen, K, unit, n_exact);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Stable partition of the particles by unit.  Block b of kUnitBlock
// particles counts each unit per warp; counts[u * nb + b] feed an exclusive
// scan; the scatter ranks each particle by (warp, lane) inside its block, so
// each unit's list keeps ascending particle order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_unit_counts(const int32_t* unit, int64_t n, int K, int* wcnt,
                                                 int& my_unit, int& rank_in_warp) {
  // wcnt: [32 warps][K] in shared memory, zeroed by the caller
  int64_t p = (int64_t)blockIdx.x * kUnitBlock + threadIdx.x;
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  my_unit = (p < n) ? unit[p] : -1;
  if (p < n && (my_unit < 0 || my_unit >= K)) my_unit = 0;   // stays in bounds; k_pack latches the error
  unsigned same = __match_any_sync(0xffffffffu, my_unit);
  rank_in_warp = __popc(same & ((1u << lane) - 1u));
  if (my_unit >= 0 && rank_in_warp == 0) wcnt[w * K + my_unit] = __popc(same);
}

__global__ void k_unit_hist(const int32_t* __restrict__ unit, int64_t n, int K, int nb, int32_t* counts,
                            const int* __restrict__ gate = nullptr) {
  if (gate && gate[0] == 0) return;   // evaluation order: only at list builds
  extern __shared__ int wcnt[];
  for (int k = threadIdx.x; k < 32 * K; k += blockDim.x) wcnt[k] = 0;
  __syncthreads();
  int u, r;
  warp_unit_counts(unit, n, K, wcnt, u, r);
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    int s = 0;
    for (int w = 0; w < 32; ++w) s += wcnt[w * K + k];
    counts[(int64_t)k * nb + blockIdx.x] = s;
  }
}

__global__ void k_unit_scatter(const int32_t* __restrict__ unit, int64_t n, int K, int nb,
                               const int32_t* __restrict__ start, int32_t* list, const int* __restrict__ gate = nullptr) {
  if (gate && gate[0] == 0) return;
  extern __shared__ int wcnt[];
  for (int k = threadIdx.x; k < 32 * K; k += blockDim.x) wcnt[k] = 0;
  __syncthreads();
  int u, r;
  warp_unit_counts(unit, n, K, wcnt, u, r);
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {  // exclusive prefix over warps
    int s = 0;
    for (int w = 0; w < 32; ++w) { int c = wcnt[w * K + k]; wcnt[w * K + k] = s; s += c; }
  }
  __syncthreads();
  int64_t p = (int64_t)blockIdx.x * kUnitBlock + threadIdx.x;
  if (p < n) {
    int w = threadIdx.x >> 5;
    list[start[(int64_t)u * nb + blockIdx.x] + wcnt[w * K + u] + r] = (int32_t)p;
  }
}

__global__ void k_unit_offsets(const int32_t* __restrict__ start, int K, int nb, int64_t n, int32_t* unit_off,
                               int32_t* out_copy, const int* __restrict__ gate = nullptr) {
  if (gate && gate[0] == 0) return;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > K) return;
  int32_t v = (k < K) ? start[(int64_t)k * nb] : (int32_t)n;
  unit_off[k] = v;
  if (out_copy) out_copy[k] = v;
}

// ---------------------------------------------------------------------------
// Per-unit statistics, one block per unit, fixed summation order:
// centroid (eq. VoronoiGeomCenters over the current positions), count, and
// max_{i in k} R^hrz_i with R^hrz_i = (1 + beta)(kh (d_i + max_j d_j)).
// ---------------------------------------------------------------------------
// S blocks per unit (blockIdx.x = k S + s) each sum a strided share of the
// unit's particles into part[(k S + s) x 4] (position sums, max R^hrz); a
// second kernel adds the S partials of each unit in order.  One block per
// unit left most SMs idle (64 units) on a kernel bound by FP64 adds.
constexpr int kUnitSplit = 16;

__global__ void k_unit_stats(const int32_t* __restrict__ unit_off, const int32_t* __restrict__ list,
                             const double* __restrict__ x, const double* __restrict__ y,
                             const double* __restrict__ z, const double* __restrict__ d,
                             const double* __restrict__ dmax_nbr, int gdim, double kh, double beta, int S,
                             double* part) {
  const int k = blockIdx.x / S, sp = blockIdx.x % S;
  int b = unit_off[k], e = unit_off[k + 1];
  double acc[3] = {0, 0, 0};
  double rmax = 0.0;
  const double* X[3] = {x, y, z};
  for (int q = b + sp * (int)blockDim.x + threadIdx.x; q < e; q += S * (int)blockDim.x) {
    int64_t p = list[q];
    for (int a = 0; a < gdim; ++a) acc[a] += X[a][p];
    double dm = dmax_nbr[p] < 0.0 ? d[p] : dmax_nbr[p];
    double r = (1.0 + beta) * (kh * (d[p] + dm));
    rmax = fmax(rmax, r);
  }
  __shared__ double sh[4][kBlock];
  for (int a = 0; a < 3; ++a) sh[a][threadIdx.x] = acc[a];
  sh[3][threadIdx.x] = rmax;
  __syncthreads();
  for (int w = kBlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      for (int a = 0; a < 3; ++a) sh[a][threadIdx.x] += sh[a][threadIdx.x + w];
      sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* o = part + (size_t)blockIdx.x * 4;
    for (int a = 0; a < 4; ++a) o[a] = sh[a][0];
  }
}

// Per unit: the S partials in order -> out[k x 5] = centroid (3), count, max R^hrz.
__global__ void k_unit_stats_final(const int32_t* __restrict__ unit_off, int K, int S,
                                   const double* __restrict__ part, double* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  double acc[3] = {0, 0, 0}, rmax = 0.0;
  for (int sp = 0; sp < S; ++sp) {
    const double* q = part + ((size_t)k * S + sp) * 4;
    for (int a = 0; a < 3; ++a) acc[a] += q[a];
    rmax = fmax(rmax, q[3]);
  }
  const int cnt = unit_off[k + 1] - unit_off[k];
  for (int a = 0; a < 3; ++a) out[k * 5 + a] = cnt > 0 ? acc[a] / (double)cnt : 0.0;
  out[k * 5 + 3] = (double)cnt;
  out[k * 5 + 4] = rmax;
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ void rotate3(const double ax[3], double alpha, const double v[3], double out[3]) {
  double na = sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
  if (na == 0.0) { out[0] = v[0]; out[1] = v[1]; out[2] = v[2]; return; }
  const double ina = 1.0 / na;
  double u[3] = {ax[0] * ina, ax[1] * ina, ax[2] * ina};
  double c, s;
  sincos(alpha, &s, &c);
  double uxv[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
  double udv = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
  for (int q = 0; q < 3; ++q) out[q] = v[q] * c + uxv[q] * s + u[q] * udv * (1.0 - c);
}

// ---------------------------------------------------------------------------
// Balancing update (one block per generator k, then one block to apply):
//   eq. (BalancingOffset)       two-body, g_kl = g_k - g_l
//   eq. (BalancingOffsetRot)    three-body for 2D decompositions, each
//                               triangle of mutually adjacent units once,
//                               length limited to max_l D^sh_kl; for 3D
//                               decompositions four-body terms instead:
//                               -c_k + M(w, |w|) c_k about the centre of the
//                               sphere through g_k, g_l, g_m, g_n, with
//                               w = sum_p a_p unit(c_k x c_p) and
//                               a_p = (arccos(-1/3)/2)(L_p - L_k)/(L_k+L_l+L_m+L_n)
//   eq. (BalancingOffsetPlusRot), eq. (TotalOffset)
// D^sh_kl = max(rmax_k, rmax_l) (eq. Horizon).  Loads: caller's, else half
// the accumulated full-list pair counts.  Resets the accumulators.
// ---------------------------------------------------------------------------
// Butterfly sum / max over the warp (every lane gets the result).
__device__ __forceinline__ void warp_sum3(double* v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] += __shfl_xor_sync(0xffffffffu, v[a], o);
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double q = __shfl_xor_sync(0xffffffffu, v, o);
    v = q > v ? q : v;
  }
  return v;
}

// Unit k's update (one warp per unit, the terms spread over its lanes): the
// balancing offsets of unit k and its new generator, into scratch
// (3 coordinates, then the shift length, per unit).
__global__ void k_balance_unit(int K, int gdim, const double* __restrict__ gen, const double* __restrict__ load_in,
                               const unsigned long long* __restrict__ load_acc,
                               const uint32_t* __restrict__ adj_bits, int adj_words,
                               const double* __restrict__ stats, double theta, double sigma, double gamma_b,
                               double* scratch) {
  __shared__ double L[SPH_MAX_UNITS];
  __shared__ double G[SPH_MAX_UNITS * 3];
  __shared__ uint32_t AB[SPH_MAX_UNITS * (SPH_MAX_UNITS / 32)];   // the adjacency bitmap, staged
  const double pi = 3.14159265358979323846;
  for (int q = threadIdx.x; q < K; q += blockDim.x) {
    L[q] = load_in ? load_in[q] : 0.5 * (double)load_acc[q];
    for (int a = 0; a < 3; ++a) G[q * 3 + a] = a < gdim ? gen[q * gdim + a] : 0.0;
  }
  for (int q = threadIdx.x; q < K * adj_words; q += blockDim.x) AB[q] = adj_bits[q];
  __syncthreads();
  const int k = blockIdx.x;
  if (k >= K) return;
  const int lane = threadIdx.x & 31;   // one warp per unit
  double sig = (gdim >= 2) ? sigma : 0.0;   // three-body terms in 2D, four-body terms in 3D
  // The neighbours of a unit are walked as the set bits of its bitmap row, in
  // increasing index order; the warp's lanes take every 32nd neighbour l, and
  // every 32nd three- or four-body set in that walk, and the lanes' partial
  // sums are added by a butterfly.
  auto dsh = [&](int r, int c) -> double {
    double a = stats[r * 5 + 4], b = stats[c * 5 + 4];
    return a > b ? a : b;
  };
  const double* gk = &G[k * 3];
  double dg2[3] = {0, 0, 0}, dg3[3] = {0, 0, 0};
  double maxd = 0.0;
  int nth = 0;
  for (int w = 0; w < adj_words; ++w)
  for (uint32_t bits = AB[k * adj_words + w]; bits; bits &= bits - 1) {
    const int l = w * 32 + __ffs(bits) - 1;
    if (l == k || l >= K) continue;
    if ((nth++ & 31) != lane) continue;
    double D = dsh(k, l);
    if (D > maxd) maxd = D;
    double den = L[k] + L[l];
    if (!(den > 0.0)) continue;
    double gkl[3] = {gk[0] - G[l * 3], gk[1] - G[l * 3 + 1], gk[2] - G[l * 3 + 2]};
    double nrm = sqrt(gkl[0] * gkl[0] + gkl[1] * gkl[1] + gkl[2] * gkl[2]);
    if (nrm == 0.0) continue;
    double f = D * ((L[k] - L[l]) / den) / nrm;
    for (int a = 0; a < 3; ++a) dg2[a] += f * gkl[a];
  }
  if (sig != 0.0 && gdim == 3) {
    // four-body terms: each set {k, l, m, n} of mutually adjacent units once
    // (l < m < n), a rotation of c_k on the circumsphere of the four generators
    const double half_t = 0.5 * acos(-1.0 / 3.0);
    int nset = 0;
    for (int wl = 0; wl < adj_words; ++wl)
    for (uint32_t bl = AB[k * adj_words + wl]; bl; bl &= bl - 1) {
      const int l = wl * 32 + __ffs(bl) - 1;
      if (l == k || l >= K) continue;
      for (int wm = (l + 1) >> 5; wm < adj_words; ++wm)
      for (uint32_t bm = AB[k * adj_words + wm] & AB[l * adj_words + wm] &
                         (wm == ((l + 1) >> 5) ? (~0u << ((l + 1) & 31)) : ~0u);
           bm; bm &= bm - 1) {
        const int m = wm * 32 + __ffs(bm) - 1;
        if (m == k || m >= K) continue;
        for (int wn = (m + 1) >> 5; wn < adj_words; ++wn)
        for (uint32_t bn = AB[k * adj_words + wn] & AB[l * adj_words + wn] & AB[m * adj_words + wn] &
                           (wn == ((m + 1) >> 5) ? (~0u << ((m + 1) & 31)) : ~0u);
             bn; bn &= bn - 1) {
          const int n4 = wn * 32 + __ffs(bn) - 1;
          if (n4 == k || n4 >= K) continue;
          if ((nset++ & 31) != lane) continue;
          const double* gl = &G[l * 3];
          const double* gm = &G[m * 3];
          const double* gn = &G[n4 * 3];
          double a[3], b[3], c[3];
          for (int q = 0; q < 3; ++q) { a[q] = gl[q] - gk[q]; b[q] = gm[q] - gk[q]; c[q] = gn[q] - gk[q]; }
          double bc[3], ca[3], ab[3];
          cross3(b, c, bc);
          cross3(c, a, ca);
          cross3(a, b, ab);
          const double det = a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2];
          const double a2 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
          const double b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
          const double c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
          double s2 = a2 > b2 ? a2 : b2;
          s2 = s2 > c2 ? s2 : c2;
          if (fabs(det) < 1e-12 * s2 * sqrt(s2)) continue;          // coplanar: no circumsphere
          const double Ls = L[k] + L[l] + L[m] + L[n4];
          if (!(Ls > 0.0)) continue;
          double o[3];
          for (int q = 0; q < 3; ++q) o[q] = gk[q] + (a2 * bc[q] + b2 * ca[q] + c2 * ab[q]) / (2.0 * det);
          const double al = half_t * (L[l] - L[k]) / Ls, am = half_t * (L[m] - L[k]) / Ls;
          const double an = half_t * (L[n4] - L[k]) / Ls;
          double ck[3], cl[3], cm[3], cn[3];
          for (int q = 0; q < 3; ++q) { ck[q] = gk[q] - o[q]; cl[q] = gl[q] - o[q]; cm[q] = gm[q] - o[q]; cn[q] = gn[q] - o[q]; }
          // one rotation about the summed rotation vector (label independent)
          const double* cp[3] = {cl, cm, cn};
          const double ap[3] = {al, am, an};
          double w[3] = {0.0, 0.0, 0.0};
          for (int t = 0; t < 3; ++t) {
            double ax[3];
            cross3(ck, cp[t], ax);
            const double na = sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
            if (na == 0.0) continue;
            for (int q = 0; q < 3; ++q) w[q] += ap[t] * ax[q] / na;
          }
          const double nw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
          if (nw == 0.0) continue;
          double rr[3];
          rotate3(w, nw, ck, rr);
          for (int q = 0; q < 3; ++q) dg3[q] += rr[q] - ck[q];
        }
      }
    }
    warp_sum3(dg3);
    maxd = warp_max(maxd);
    double n3 = sqrt(dg3[0] * dg3[0] + dg3[1] * dg3[1] + dg3[2] * dg3[2]);
    if (n3 > maxd && n3 > 0.0) {
      double f = maxd / n3;
      for (int a = 0; a < 3; ++a) dg3[a] *= f;
    }
  } else if (sig != 0.0) {
    int nset = 0;
    for (int wl = 0; wl < adj_words; ++wl)
    for (uint32_t bl = AB[k * adj_words + wl]; bl; bl &= bl - 1) {
      const int l = wl * 32 + __ffs(bl) - 1;
      if (l == k || l >= K) continue;
      for (int wm = (l + 1) >> 5; wm < adj_words; ++wm)
      for (uint32_t bm = AB[k * adj_words + wm] & AB[l * adj_words + wm] &
                         (wm == ((l + 1) >> 5) ? (~0u << ((l + 1) & 31)) : ~0u);
           bm; bm &= bm - 1) {
        const int m = wm * 32 + __ffs(bm) - 1;
        if (m == k || m >= K) continue;
        if ((nset++ & 31) != lane) continue;
        const double* gl = &G[l * 3];
        const double* gm = &G[m * 3];
        double ax = gl[0] - gk[0], ay = gl[1] - gk[1];
        double bx = gm[0] - gk[0], by = gm[1] - gk[1];
        double a2 = ax * ax + ay * ay, b2 = bx * bx + by * by;
        double crs = ax * by - ay * bx;
        double scale2 = a2 > b2 ? a2 : b2;
        if (fabs(crs) < 1e-12 * scale2) continue;
        double Dd = 2.0 * crs;
        double ox = gk[0] + (by * a2 - ay * b2) / Dd;
        double oy = gk[1] + (ax * b2 - bx * a2) / Dd;
        double Ls = L[k] + L[l] + L[m];
        if (!(Ls > 0.0)) continue;
        double al = pi / 3.0 * (L[l] - L[k]) / Ls;
        double am = pi / 3.0 * (L[m] - L[k]) / Ls;
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
    warp_sum3(dg3);
    maxd = warp_max(maxd);
    double n3 = sqrt(dg3[0] * dg3[0] + dg3[1] * dg3[1] + dg3[2] * dg3[2]);
    if (n3 > maxd && n3 > 0.0) {
      double f = maxd / n3;
      for (int a = 0; a < 3; ++a) dg3[a] *= f;
    }
  }
  warp_sum3(dg2);
  if (lane != 0) return;
  double cnt = stats[k * 5 + 3];
  double dist2 = 0.0;
  for (int a = 0; a < gdim; ++a) {
    double dg = (1.0 - sig) * dg2[a] + sig * dg3[a];
    double rc = cnt > 0.0 ? stats[k * 5 + a] : gk[a];
    double ng = (1.0 - theta) * (gk[a] + gamma_b * dg) + theta * rc;
    scratch[k * 4 + a] = ng;
    dist2 += (ng - gk[a]) * (ng - gk[a]);
  }
  scratch[k * 4 + 3] = sqrt(dist2);
}

// New generators, the summed shift (fixed order) and the reset of the load
// and adjacency accumulators.
__global__ void k_balance_apply(int K, int gdim, double* gen, const double* __restrict__ scratch,
                                unsigned long long* load_acc, uint32_t* adj_bits, int adj_words, double* shift_out) {
  const int k = threadIdx.x;
  if (k < K) {
    for (int a = 0; a < gdim; ++a) gen[k * gdim + a] = scratch[k * 4 + a];
    load_acc[k] = 0ull;
    for (int w = 0; w < adj_words; ++w) adj_bits[k * adj_words + w] = 0u;
  }
  if (k == 0) {
    double s = 0.0;
    for (int q = 0; q < K; ++q) s += scratch[q * 4 + 3];
    if (shift_out) *shift_out = s;
  }
}

}  // namespace

cudaError_t launch_assign(sph_handle* h, const sph_state& s, const double* gen, int K, int dim,
                          int32_t* unit_out, cudaStream_t st) {
  h->launches += 1;
  return launch_assign_kernel(h->n, dim, s.x, s.y, s.z, gen, K, unit_out, &h->counters[3], st);
}

cudaError_t launch_unit_lists(sph_handle* h, const int32_t* unit, int32_t* unit_offsets, cudaStream_t st) {
  int K = h->K;
  int nb = grid_for(h->n, kUnitBlock);
  size_t smem = sizeof(int) * 32 * K;
  int32_t* counts = h->unit_work;                 // [K * nb]
  int32_t* starts = counts + (size_t)K * nb;       // [K * nb + 1]
  int32_t* sums = starts + (size_t)K * nb + 1;     // [K * nb / 1024 + 1]
  int64_t tot = h->unit_work_total;                // = K * nb, also in h->unit_total
  cudaError_t e;
  k_unit_hist<<<nb, kUnitBlock, smem, st>>>(unit, h->n, K, nb, counts);
  e = launch_exclusive_scan(counts, h->unit_total, sums, starts, h->n, tot, st);
  if (e != cudaSuccess) return e;
  k_unit_scatter<<<nb, kUnitBlock, smem, st>>>(unit, h->n, K, nb, starts, h->unit_list);
  k_unit_offsets<<<grid_for(K + 1, kBlock), kBlock, 0, st>>>(starts, K, nb, h->n, h->unit_off, unit_offsets);
  h->launches += 6;
  return cudaGetLastError();
}

namespace {

// Unit of each cell-order slot (clamped into range, as k_pack does).
__global__ void k_slot_units(int64_t n, const int32_t* __restrict__ perm, const int32_t* __restrict__ unit, int K,
                             int32_t* slot_u, const int* __restrict__ gate) {
  if (gate && gate[0] == 0) return;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    int u = unit[perm[c]];
    slot_u[c] = (u < 0 || u >= K) ? 0 : u;
  }
}

// Inverse of the partition (the evaluation slot of each cell-order slot) and
// the particle of each evaluation slot.
__global__ void k_eorder_inverse(int64_t n, const int32_t* __restrict__ c_of_e, const int32_t* __restrict__ perm,
                                 int32_t* e_of_c, int32_t* perm_e, const int* __restrict__ gate) {
  if (gate && gate[0] == 0) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = c_of_e[e];
    e_of_c[c] = (int32_t)e;
    perm_e[e] = perm[c];
  }
}

}  // namespace

// The unit-major evaluation order: a stable partition of the cell-order slots
// by the unit of their particle (so cell order, and with it locality, is kept
// inside each unit), the same block-histogram / scan / scatter as the unit
// lists.  Gated on vflag[0] (it runs only when the lists are rebuilt) unless
// forced (at a rebalance, where the state is then renumbered in this order).
cudaError_t launch_eorder(sph_handle* h, const sph_state& s, cudaStream_t st, bool force) {
  const int K = h->K;
  const int nb = grid_for(h->n, kUnitBlock);
  const size_t smem = sizeof(int) * 32 * K;
  int32_t* counts = h->unit_work;                 // [K * nb]
  int32_t* starts = counts + (size_t)K * nb;       // [K * nb + 1]
  int32_t* sums = starts + (size_t)K * nb + 1;
  int32_t* slot_u = h->rank;                        // free between a cell sort and the next one
  int32_t* c_of_e = reinterpret_cast<int32_t*>(h->scratch);   // free outside the renumbering
  const int* gate = force ? nullptr : h->vflag;
  const int g = assign_grid(h->n);
  k_slot_units<<<g, kBlock, 0, st>>>(h->n, h->perm, s.unit, K, slot_u, gate);
  k_unit_hist<<<nb, kUnitBlock, smem, st>>>(slot_u, h->n, K, nb, counts, gate);
  cudaError_t e = launch_exclusive_scan(counts, h->unit_total, sums, starts, h->n, h->unit_work_total, st, gate);
  if (e != cudaSuccess) return e;
  k_unit_scatter<<<nb, kUnitBlock, smem, st>>>(slot_u, h->n, K, nb, starts, c_of_e, gate);
  k_unit_offsets<<<grid_for(K + 1, kBlock), kBlock, 0, st>>>(starts, K, nb, h->n, h->unit_eoff, nullptr, gate);
  k_eorder_inverse<<<g, kBlock, 0, st>>>(h->n, c_of_e, h->perm, h->e_of_c, h->perm_e, gate);
  h->launches += 8;
  return cudaGetLastError();
}

cudaError_t launch_balance_given(sph_handle* h, double* gen, int K, int dim, const double* stats,
                                 const double* load, const sph_balance_params& bp, double* shift_out,
                                 cudaStream_t st) {
  double* scratch = h->unit_stats + (size_t)5 * K;
  k_balance_unit<<<K, 32, 0, st>>>(K, dim, gen, load, h->load_acc, h->adj_bits, (K + 31) / 32, stats, bp.theta,
                                   bp.sigma, bp.gamma_b, scratch);
  k_balance_apply<<<1, SPH_MAX_UNITS, 0, st>>>(K, dim, gen, scratch, h->load_acc, h->adj_bits, (K + 31) / 32,
                                               shift_out);
  h->launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_balance(sph_handle* h, const sph_state& s, double* gen, int K, int dim, const double* load,
                           const sph_balance_params& bp, double* shift_out, cudaStream_t st) {
  cudaError_t e = launch_unit_lists(h, s.unit, nullptr, st);
  if (e != cudaSuccess) return e;
  double* stats = h->unit_stats;
  // blocks per unit: about four per SM in total, at most kUnitSplit
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
  }
  int S = (4 * sms + K - 1) / K;
  S = S < 1 ? 1 : (S > kUnitSplit ? kUnitSplit : S);
  double* part = stats + (size_t)9 * K;
  k_unit_stats<<<K * S, kBlock, 0, st>>>(h->unit_off, h->unit_list, s.x, s.y, s.z, s.d, h->dmax_nbr, dim,
                                         h->dp.kh, bp.beta_sh, S, part);
  k_unit_stats_final<<<(K + 63) / 64, 64, 0, st>>>(h->unit_off, K, S, part, stats);
  double* scratch = stats + (size_t)5 * K;
  k_balance_unit<<<K, 32, 0, st>>>(K, dim, gen, load, h->load_acc, h->adj_bits, (K + 31) / 32, stats, bp.theta,
                                   bp.sigma, bp.gamma_b, scratch);
  k_balance_apply<<<1, SPH_MAX_UNITS, 0, st>>>(K, dim, gen, scratch, h->load_acc, h->adj_bits, (K + 31) / 32,
                                               shift_out);
  h->launches += 4;
  return cudaGetLastError();
}

}  // namespace csph

// ---------------------------------------------------------------------------
// Allocation-free Voronoi assignment for callers that cannot allocate device
// memory (no counterpart in the paper): a host loop that must not call
// cudaMalloc (an allocation synchronises the device and may fail under memory
// pressure), or code whose device memory is all owned by another pool (a
// framework's caching allocator, a fixed arena).  Such a caller cannot create
// a handle, whose workspace sph_init allocates.  This entry point takes only
// the caller's positions, generators and output arrays and keeps its scratch
// (per-unit counts, their scan and a counter) in one file-scope device array
// of fixed size, so it allocates nothing.
// ---------------------------------------------------------------------------
namespace csph {
namespace {

constexpr int64_t kStaticMaxN = int64_t(1) << 22;                                     // 4,194,304 particles
constexpr int64_t kStaticMaxCounts = int64_t(SPH_MAX_UNITS) * (kStaticMaxN / kUnitBlock);   // 1,048,576
constexpr int64_t kStaticSums = kStaticMaxCounts / 1024 + 2;
// int32 layout: counts | starts (+1) | scan sums | unit offsets (K+1) | pad to 8 bytes | total, exact counter
constexpr int64_t kOffCounts = 0;
constexpr int64_t kOffStarts = kOffCounts + kStaticMaxCounts;
constexpr int64_t kOffSums = kOffStarts + kStaticMaxCounts + 1;
constexpr int64_t kOffUnitOff = kOffSums + kStaticSums;
constexpr int64_t kOffTail = ((kOffUnitOff + SPH_MAX_UNITS + 1) + 1) & ~int64_t(1);  // even: 8-byte aligned
constexpr int64_t kStaticWords = kOffTail + 4;                                        // int64 total + uint64 counter

// The scratch shared by every call on a device (about 8.4 MB, held until exit).
static __device__ __align__(256) int32_t g_assign_scratch[kStaticWords];

__global__ void k_static_reset(int64_t* total, unsigned long long* exact, int64_t tot) {
  *total = tot;
  *exact = 0ull;
}

std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
int32_t* g_static_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, resolved once per
// device with that device current and kept for the life of the process
// (stale after cudaDeviceReset, which unloads the module).
cudaError_t static_scratch(int32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_assign_scratch);
    if (e != cudaSuccess) return e;
    g_static_addr[dev] = reinterpret_cast<int32_t*>(p);
  }
  *out = g_static_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace csph

extern "C" int voronoi_assign_static(int64_t n, const double* x, const double* y, const double* z,
                                     const double* gen, int K, int dim, int32_t* unit_out,
                                     int32_t* unit_offsets, int32_t* unit_list, void* stream) {
  using namespace csph;
  if (n < 1 || K < 1 || dim < 1 || dim > 3 || !x || !gen || !unit_out || (dim >= 2 && !y) || (dim >= 3 && !z)) {
    set_global_error("voronoi_assign_static: need n >= 1, 1 <= K, dim in 1..3 and non-NULL x (y, z for dim >= 2, 3), "
                     "gen and unit_out");
    return SPH_ERR_INVALID;
  }
  if (n > kStaticMaxN || K > SPH_MAX_UNITS) {
    set_global_error("voronoi_assign_static: at most 4,194,304 particles and 256 units (fixed scratch size)");
    return SPH_ERR_CAPACITY;
  }
  int32_t* scr = nullptr;
  cudaError_t e = static_scratch(&scr);
  if (e != cudaSuccess) {
    set_global_error(std::string("voronoi_assign_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    return SPH_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = grid_for(n, kUnitBlock);
  const int64_t tot = (int64_t)K * nb;
  int32_t* counts = scr + kOffCounts;
  int32_t* starts = scr + kOffStarts;
  int32_t* sums = scr + kOffSums;
  int64_t* total = reinterpret_cast<int64_t*>(scr + kOffTail);
  unsigned long long* exact = reinterpret_cast<unsigned long long*>(scr + kOffTail + 2);
  const size_t smem = sizeof(int) * 32 * K;
  // every launch is checked as soon as it is issued, so a failure is reported
  // by the launch that caused it
  k_static_reset<<<1, 1, 0, st>>>(total, exact, tot);   // the previous call left its values here
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_assign_kernel(n, dim, x, y, z, gen, K, unit_out, exact, st);
  if (e == cudaSuccess) {
    k_unit_hist<<<nb, kUnitBlock, smem, st>>>(unit_out, n, K, nb, counts);   // writes every count
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_exclusive_scan(counts, total, sums, starts, n, tot, st);
  if (e == cudaSuccess && unit_list) {
    k_unit_scatter<<<nb, kUnitBlock, smem, st>>>(unit_out, n, K, nb, starts, unit_list);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_unit_offsets<<<grid_for(K + 1, kBlock), kBlock, 0, st>>>(starts, K, nb, n,
                                                             unit_offsets ? unit_offsets : scr + kOffUnitOff, nullptr);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_global_error(std::string("voronoi_assign_static: ") + cudaGetErrorString(e));
    return SPH_ERR_CUDA;
  }
  return SPH_OK;
}
