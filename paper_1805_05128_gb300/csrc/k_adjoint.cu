// k_adjoint.cu -- reverse mode of the CSPH step (FP64 accumulation), with the
// pair set and the dt sequence of the forward run held fixed.
//
// For one step from state S (x, v, rho, E and the held rates a, drho, dE) with
// time step dt and h = dt/2 the forward map is
//   v^h = v + h a, rho^h = rho + h drho, E^h = E + h dE, x' = x + dt v^h,
//   v~ = v^h + h a, rho~ = rho^h + h drho, E~ = E^h + h dE,
//   (a', drho', dE') = R(x', v~, rho~, E~), v' = v^h + h a', rho', E' alike.
// Its transpose, applied to the adjoint of (x', v', rho', E', a', drho', dE'),
// needs the vector-Jacobian product of the rates R of eqs. (SPH:Conti),
// (SPH:Pulse), (SPH:Energy) with the acoustic pair solver: k_pair_vjp takes,
// for every interacting pair (i, j) seen from i, the derivative of the pair's
// contributions to (a, drho, dE) of both particles with respect to i's own
// variables (positions, v^R, P, Z = rho c, V = m/rho, d, and the rho factor of
// the continuity term); k_vjp_chain carries those through V, d, Z, the EOS
// and e = E - v^2/2 and then through the kick-drift-kick algebra above.
// Supported closures: cubic spline, ideal and stiffened gas (parameters c0,
// gamma of material 0, P_inf = rho0 c0^2 / gamma).
#include <cfloat>

#include "csph_internal.cuh"

namespace csph {

namespace {

struct AdjArgs {
  int64_t n;
  int n_inst;
  const int64_t* inst_off;
  const GridInfo* grid;
  const int64_t* total_cells;
  const int32_t* cell_start;
  const int32_t* slot_cell;
  const int32_t* perm;
  const D4* A;       // x, y, z, d       (slot order, FP64)
  const D4* B;       // v, V = m/rho
  const D2* C;       // P, Z = rho c
  const double* rho; // density of the slot
  const D4* G;       // (dL/da)/m, (dL/ddE)/m of the slot
  const double* GR;  // dL/ddrho of the slot
  double* out;       // particle order, 11 per particle: bx[3], bv[3], bP, bZ, bV, bd, brho
  double kh, eta;
  int dim;
};

// cubic spline: W' = s h^-(D+1) g(q), dW'/dr = s h^-(D+2) g'(q), dW'/dh = s h^-(D+2) (-(D+1) g - q g')
__device__ __forceinline__ void cubic_dw3(int dim, double r, double h, double& w, double& wr, double& wh) {
  const double pi = 3.14159265358979323846;
  const double s = dim == 1 ? 2.0 / 3.0 : (dim == 2 ? 10.0 / (7.0 * pi) : 1.0 / pi);
  const double q = r / h;
  double g, gp;
  if (q < 1.0) { g = -3.0 * q + 2.25 * q * q; gp = -3.0 + 4.5 * q; }
  else if (q < 2.0) { const double t = 2.0 - q; g = -0.75 * t * t; gp = 1.5 * t; }
  else { g = 0.0; gp = 0.0; }
  double hp1 = h * h;
  if (dim >= 2) hp1 *= h;
  if (dim >= 3) hp1 *= h;
  w = s * g / hp1;
  wr = s * gp / (hp1 * h);
  wh = s * (-(double)(dim + 1) * g - q * gp) / (hp1 * h);
}

// One thread per slot i: scan the 3^dim cells, FP64 interaction test in the
// oracle's operation order, own-side derivative of every interacting pair.
template <int DIM>
__global__ void __launch_bounds__(128) k_pair_vjp(AdjArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  int b = 0;
  if (a.n_inst > 1) {
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
  const D4 Ai = a.A[i], Bi = a.B[i], Gi = a.G[i];
  const D2 Ci = a.C[i];
  const double rhoi = a.rho[i], GRi = a.GR[i];
  double bx[3] = {0, 0, 0}, bv[3] = {0, 0, 0}, bP = 0, bZ = 0, bV = 0, bd = 0, brho = 0;
  for (int oz = (DIM >= 3 ? -1 : 0); oz <= (DIM >= 3 ? 1 : 0); ++oz) {
    const int zz = cz + oz;
    if (zz < 0 || zz >= nz) continue;
    for (int oy = (DIM >= 2 ? -1 : 0); oy <= (DIM >= 2 ? 1 : 0); ++oy) {
      const int yy = cy + oy;
      if (yy < 0 || yy >= ny) continue;
      const int x0 = cx > 0 ? cx - 1 : 0, x1 = cx + 1 < nx ? cx + 1 : nx - 1;
      const int64_t rowc = g.cell_off + (int64_t)nx * (yy + (int64_t)ny * zz);
      const int s0 = a.cell_start[rowc + x0], s1 = a.cell_start[rowc + x1 + 1];
      for (int j = s0; j < s1; ++j) {
        if (j == i) continue;
        const D4 Aj = a.A[j];
        double dxv[3];
        dxv[0] = __dsub_rn(Aj.x, Ai.x);
        dxv[1] = DIM >= 2 ? __dsub_rn(Aj.y, Ai.y) : 0.0;
        dxv[2] = DIM >= 3 ? __dsub_rn(Aj.z, Ai.z) : 0.0;
        double r2 = __dmul_rn(dxv[0], dxv[0]);
        if (DIM >= 2) r2 = __dadd_rn(r2, __dmul_rn(dxv[1], dxv[1]));
        if (DIM >= 3) r2 = __dadd_rn(r2, __dmul_rn(dxv[2], dxv[2]));
        const double R = __dmul_rn(a.kh, __dadd_rn(Ai.w, Aj.w));
        if (!(r2 < __dmul_rn(R, R)) || r2 == 0.0) continue;
        const D4 Bj = a.B[j], Gj = a.G[j];
        const D2 Cj = a.C[j];
        const double rhoj = a.rho[j], GRj = a.GR[j];
        const double r = sqrt(r2);
        double e[3] = {dxv[0] / r, dxv[1] / r, dxv[2] / r};
        const double vi[3] = {Bi.x, Bi.y, Bi.z}, vj[3] = {Bj.x, Bj.y, Bj.z};
        double vRi = 0, vRj = 0;
        for (int q = 0; q < DIM; ++q) { vRi += vi[q] * e[q]; vRj += vj[q] * e[q]; }
        const double Zi = Ci.y, Zj = Cj.y, zs = Zi + Zj, Pi = Ci.x, Pj = Cj.x;
        double Ps, vs;
        if (zs > 0.0) {
          Ps = (Zj * Pi + Zi * Pj + Zi * Zj * (vRi - vRj)) / zs;
          vs = (Zi * vRi + Zj * vRj + Pi - Pj) / zs;
        } else {
          Ps = 0.5 * (Pi + Pj);
          vs = 0.5 * (vRi + vRj);
        }
        const double hij = a.eta * (Ai.w + Aj.w) * 0.5;
        double W, Wr, Wh;
        cubic_dw3(DIM, r, hij, W, Wr, Wh);
        const double Vi = Bi.w, Vj = Bj.w;
        const double F = 2.0 * Vi * Vj * Ps * W;
        const double dA[3] = {Gi.x - Gj.x, Gi.y - Gj.y, Gi.z - Gj.z};
        const double dB = Gi.w - Gj.w;
        double gF = dB * vs, ge[3] = {0, 0, 0};
        for (int q = 0; q < DIM; ++q) { gF += dA[q] * e[q]; ge[q] = F * dA[q]; }
        const double gvs = F * dB + 2.0 * W * rhoi * Vj * GRi - 2.0 * W * rhoj * Vi * GRj;
        double gvRi = -2.0 * W * rhoi * Vj * GRi;
        double gvRj = 2.0 * W * rhoj * Vi * GRj;
        const double gW = gF * 2.0 * Vi * Vj * Ps - GRi * 2.0 * rhoi * Vj * (vRi - vs) - GRj * 2.0 * rhoj * Vi * (vs - vRj);
        const double gPs = gF * 2.0 * Vi * Vj * W;
        bV += gF * 2.0 * Vj * Ps * W + GRj * 2.0 * rhoj * (vs - vRj) * (-W);
        brho += GRi * 2.0 * Vj * (vRi - vs) * (-W);
        double gPi, gZi = 0.0;
        if (zs > 0.0) {
          gPi = gPs * Zj / zs + gvs / zs;
          gvRi += gPs * Zi * Zj / zs + gvs * Zi / zs;
          gvRj += -gPs * Zi * Zj / zs + gvs * Zj / zs;
          gZi = gPs * ((Pj + Zj * (vRi - vRj)) - Ps) / zs + gvs * (vRi - vs) / zs;
        } else {
          gPi = 0.5 * gPs;
          gvRi += 0.5 * gvs;
          gvRj += 0.5 * gvs;
        }
        bP += gPi;
        bZ += gZi;
        for (int q = 0; q < DIM; ++q) {
          bv[q] += gvRi * e[q];
          ge[q] += gvRi * vi[q] + gvRj * vj[q];
        }
        const double grr = gW * Wr, gh = gW * Wh;
        double ede = 0.0;
        for (int q = 0; q < DIM; ++q) ede += ge[q] * e[q];
        for (int q = 0; q < DIM; ++q) bx[q] -= (ge[q] - ede * e[q]) / r + grr * e[q];
        bd += gh * a.eta * 0.5;
      }
    }
  }
  double* o = a.out + 11 * (int64_t)a.perm[i];
  for (int q = 0; q < 3; ++q) { o[q] = bx[q]; o[3 + q] = bv[q]; }
  o[6] = bP; o[7] = bZ; o[8] = bV; o[9] = bd; o[10] = brho;
}

// Adjoint operands in slot order: G = (dL/da' / m, dL/ddE' / m), GR = dL/ddrho'.
// With predicted = 1 the rates are those after a step: their adjoints are the
// incoming ones plus h times the adjoints of v', E', rho' (v' = v^h + h a').
__global__ void k_adj_pack(int64_t n, int dim, const int32_t* __restrict__ perm, const sph_state adj,
                           const double* __restrict__ m, const double* __restrict__ dt, int predicted, D4* G,
                           double* GR) {
  int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= n) return;
  int64_t p = perm[sl];
  double hdt = predicted ? 0.5 * dt[0] : 0.0;
  double ga[3] = {adj.ax[p], dim >= 2 ? adj.ay[p] : 0.0, dim >= 3 ? adj.az[p] : 0.0};
  double gv[3] = {adj.vx[p], dim >= 2 ? adj.vy[p] : 0.0, dim >= 3 ? adj.vz[p] : 0.0};
  double im = 1.0 / m[p];
  G[sl] = D4{(ga[0] + hdt * gv[0]) * im, (ga[1] + hdt * gv[1]) * im, (ga[2] + hdt * gv[2]) * im,
             (adj.dE[p] + hdt * adj.E[p]) * im};
  GR[sl] = adj.drho[p] + hdt * adj.rho[p];
}

// Per particle: chain from (V, d, Z, P) to (rho, e) through the EOS, then to
// (E, v); then (predicted = 1) the transpose of the kick-drift-kick algebra,
// replacing the adjoint of the state after the step by that of the state
// before it, or (predicted = 0) the adjoint of the held rates folded into the
// state itself.  W holds the state as left by k_kick_drift (x', v^h, rho^h,
// E^h, the held rates, and d~, P~, c~ of the predicted state) or, with
// predicted = 0, the state itself with its d, P, c.
__global__ void k_vjp_chain(int64_t n, DevParams P, const sph_state W, sph_state adj, const double* __restrict__ pv,
                            const double* __restrict__ dt, int predicted, double* par_out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int dim = P.dim;
  const double* o = pv + 11 * i;
  const double hdt = predicted ? 0.5 * dt[0] : 0.0;
  const double* Wv[3] = {W.vx, W.vy, W.vz};
  const double* Wa[3] = {W.ax, W.ay, W.az};
  double v[3] = {0, 0, 0};
  for (int q = 0; q < dim; ++q) v[q] = Wv[q][i] + hdt * Wa[q][i];   // v~ (or v)
  const double rho = W.rho[i] + hdt * W.drho[i];                   // rho~
  const double E = W.E[i] + hdt * W.dE[i];                         // E~
  const int mi = W.mat ? W.mat[i] : 0;
  const Mat& mt = P.mat[mi];
  const double g = mt.gamma, pinf = mt.eos == SPH_EOS_STIFFENED ? mt.p_inf : 0.0;
  const double c = W.c[i], Pp = W.P[i], d = W.d[i], m = W.m[i];
  const double V = m / rho;
  double brho = o[10];
  brho += o[8] * (-V / rho);
  brho += o[9] * (-d / ((double)dim * rho));
  brho += o[7] * c;
  const double bc = o[7] * rho;
  double bP = o[6], bPinf = 0.0, bg = 0.0;
  if (c > 0.0) {
    const double bc2 = bc / (2.0 * c);
    bP += bc2 * g / rho;
    brho += bc2 * (-c * c / rho);
    bPinf += bc2 * g / rho;
    bg += bc2 * (Pp + pinf) / rho;
  }
  double v2 = 0.0;
  for (int q = 0; q < dim; ++q) v2 += v[q] * v[q];
  const double e_int = E - 0.5 * v2;
  brho += bP * (g - 1.0) * e_int;
  const double be = bP * (g - 1.0) * rho;
  bg += bP * (rho * e_int - pinf);
  bPinf += -g * bP;
  double bv[3];
  for (int q = 0; q < 3; ++q) bv[q] = o[3 + q] - (q < dim ? be * v[q] : 0.0);
  const double bE = be;
  double bc0 = 0.0;
  if (mi == 0) {
    if (mt.eos == SPH_EOS_STIFFENED) {
      bc0 = bPinf * 2.0 * mt.rho0 * mt.c0 / g;
      bg += bPinf * (-pinf / g);
    }
  } else {
    bg = 0.0;
  }
  par_out[2 * i] = bc0;
  par_out[2 * i + 1] = bg;

  double* AX[3] = {adj.x, adj.y, adj.z};
  double* AV[3] = {adj.vx, adj.vy, adj.vz};
  double* AA[3] = {adj.ax, adj.ay, adj.az};
  if (predicted) {
    const double h = dt[0];
    for (int q = 0; q < dim; ++q) {
      const double gxp = AX[q][i] + o[q];
      const double gvp = bv[q];
      const double gvha = AV[q][i] + gvp + h * gxp;
      AX[q][i] = gxp;
      AV[q][i] = gvha;
      AA[q][i] = hdt * gvp + hdt * gvha;
    }
    const double grha = adj.rho[i] + brho;
    adj.drho[i] = hdt * brho + hdt * grha;
    adj.rho[i] = grha;
    const double gEha = adj.E[i] + bE;
    adj.dE[i] = hdt * bE + hdt * gEha;
    adj.E[i] = gEha;
  } else {
    for (int q = 0; q < dim; ++q) {
      AX[q][i] += o[q];
      AV[q][i] += bv[q];
      AA[q][i] = 0.0;
    }
    adj.rho[i] += brho;
    adj.E[i] += bE;
    adj.drho[i] = 0.0;
    adj.dE[i] = 0.0;
  }
}

// Fixed-order sum of the per-particle parameter adjoints into out[0..1] (+=).
__global__ void k_sum_params(int64_t n, const double* __restrict__ par, double* out) {
  __shared__ double sh[2][1024];
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) { s0 += par[2 * i]; s1 += par[2 * i + 1]; }
  sh[0][threadIdx.x] = s0;
  sh[1][threadIdx.x] = s1;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) { sh[0][threadIdx.x] += sh[0][threadIdx.x + w]; sh[1][threadIdx.x] += sh[1][threadIdx.x + w]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] += sh[0][0]; out[1] += sh[1][0]; }
}

}  // namespace

// Rates VJP at the state in W (already packed in FP64 into A, B, C, rho by
// launch_pack_fp64), given the adjoint in adj; updates adj and adds the
// parameter gradient to par.
cudaError_t launch_rates_vjp(sph_handle* h, const sph_state& W, sph_state& adj, const double* dt, int predicted,
                             double* par, cudaStream_t st) {
  const int64_t n = h->n;
  k_adj_pack<<<grid_for(n, kBlock), kBlock, 0, st>>>(n, h->dp.dim, h->perm, adj, W.m, dt, predicted, h->adj_G,
                                                      h->adj_GR);
  AdjArgs a;
  a.n = n;
  a.n_inst = h->n_inst;
  a.inst_off = h->inst_off;
  a.grid = h->grid;
  a.total_cells = h->total_cells;
  a.cell_start = h->cell_start;
  a.slot_cell = h->slot_cell;
  a.perm = h->perm;
  a.A = h->adj_A;
  a.B = h->adj_B;
  a.C = h->adj_C;
  a.rho = h->adj_rho;
  a.G = h->adj_G;
  a.GR = h->adj_GR;
  a.out = h->adj_pair;
  a.kh = h->dp.kh;
  a.eta = h->dp.eta;
  a.dim = h->dp.dim;
  const int g = grid_for(n, 128);
  switch (h->dp.dim) {
    case 1: k_pair_vjp<1><<<g, 128, 0, st>>>(a); break;
    case 2: k_pair_vjp<2><<<g, 128, 0, st>>>(a); break;
    default: k_pair_vjp<3><<<g, 128, 0, st>>>(a); break;
  }
  k_vjp_chain<<<grid_for(n, kBlock), kBlock, 0, st>>>(n, h->dp, W, adj, h->adj_pair, dt, predicted, h->adj_par);
  k_sum_params<<<1, 1024, 0, st>>>(n, h->adj_par, par);
  h->launches += 4;
  return cudaGetLastError();
}

}  // namespace csph
