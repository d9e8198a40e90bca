// k_adjoint.cu -- reverse mode of the CSPH step, with the pair set and the dt
// sequence of the forward run held fixed.
//
// For one step from state S (x, v, rho, E and the held rates a, drho, dE) with
// time step dt and h = dt/2 the forward map is
//   v^h = v + h a, rho^h = rho + h drho, E^h = E + h dE, x' = x + dt v^h,
//   v~ = v^h + h a, rho~ = rho^h + h drho, E~ = E^h + h dE,
//   (a', drho', dE') = R(x', v~, rho~, E~), v' = v^h + h a', rho', E' alike.
// Its transpose, applied to the adjoint of (x', v', rho', E', a', drho', dE'),
// needs the vector-Jacobian product of the rates R of eqs. (SPH:Conti),
// (SPH:Pulse), (SPH:Energy) with the acoustic pair solver: the pair kernel in
// its reverse mode (k_pair<..., VJP = true> in k_pair.cu, the same candidate
// test and so the same pair set as the forward evaluation) takes, for every
// interacting pair (i, j) seen from i, the derivative of the pair's
// contributions to (a, drho, dE) of both particles with respect to i's own
// variables (positions, v^R, P, Z = rho c, V = m/rho, d, and the rho factor of
// the continuity term), in the handle's precision (FP32 with Kahan sums in
// mixed mode, FP64 otherwise); k_vjp_chain carries those, in FP64, through V,
// d, Z, the EOS and e = E - v^2/2 and then through the kick-drift-kick
// algebra above.
// Supported closures: cubic spline, ideal and stiffened gas (parameters c0,
// gamma of material 0, P_inf = rho0 c0^2 / gamma).
#include <cfloat>

#include "csph_internal.cuh"

namespace csph {

namespace {

// Adjoint operands in slot order, in the pair kernel's precision T:
// G = (dL/da' / m, dL/ddE' / m), GR2 = (dL/ddrho', rho of the slot).
// With predicted = 1 the rates are those after a step: their adjoints are the
// incoming ones plus h times the adjoints of v', E', rho' (v' = v^h + h a').
template <typename T, typename V4, typename V2>
__global__ void k_adj_pack(int64_t n, int dim, const int32_t* __restrict__ perm, const sph_state adj,
                           const double* __restrict__ m, const double* __restrict__ rho_slot,
                           const double* __restrict__ dt, int predicted, V4* G, V2* GR2) {
  int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= n) return;
  int64_t p = perm[sl];
  double hdt = predicted ? 0.5 * dt[0] : 0.0;
  double ga[3] = {adj.ax[p], dim >= 2 ? adj.ay[p] : 0.0, dim >= 3 ? adj.az[p] : 0.0};
  double gv[3] = {adj.vx[p], dim >= 2 ? adj.vy[p] : 0.0, dim >= 3 ? adj.vz[p] : 0.0};
  double im = 1.0 / m[p];
  V4 g;
  g.x = (T)((ga[0] + hdt * gv[0]) * im);
  g.y = (T)((ga[1] + hdt * gv[1]) * im);
  g.z = (T)((ga[2] + hdt * gv[2]) * im);
  g.w = (T)((adj.dE[p] + hdt * adj.E[p]) * im);
  G[sl] = g;
  V2 r;
  r.x = (T)(adj.drho[p] + hdt * adj.rho[p]);
  r.y = (T)rho_slot[sl];
  GR2[sl] = r;
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

// Rates VJP at the state in W (mesh and operands already built by
// launch_build_grid and launch_pack in the handle's precision), given the
// adjoint in adj; updates adj and adds the parameter gradient to par.
cudaError_t launch_rates_vjp(sph_handle* h, const sph_state& W, sph_state& adj, const double* dt, int predicted,
                             double* par, cudaStream_t st, bool fp64_pairs) {
  const int64_t n = h->n;
  const int g = grid_for(n, kBlock);
  if (fp64_pairs) {
    k_adj_pack<double, D4, D2><<<g, kBlock, 0, st>>>(n, h->dp.dim, h->perm, adj, W.m, h->adj64_rho, dt, predicted,
                                                      h->adj_G, h->adj_GR);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_pair_vjp(h, W, h->adj_G, h->adj_GR, h->adj_pair, st, h->adj64_A, h->adj64_B, h->adj64_C);
    if (e != cudaSuccess) return e;
    k_vjp_chain<<<g, kBlock, 0, st>>>(n, h->dp, W, adj, h->adj_pair, dt, predicted, h->adj_par);
    k_sum_params<<<1, 1024, 0, st>>>(n, h->adj_par, par);
    h->launches += 3;
    return cudaGetLastError();
  }
  if (h->dp.precision == SPH_PREC_MIXED)
    k_adj_pack<float, float4, float2><<<g, kBlock, 0, st>>>(n, h->dp.dim, h->perm, adj, W.m, h->rho_slot, dt,
                                                             predicted, reinterpret_cast<float4*>(h->adj_G),
                                                             reinterpret_cast<float2*>(h->adj_GR));
  else
    k_adj_pack<double, D4, D2><<<g, kBlock, 0, st>>>(n, h->dp.dim, h->perm, adj, W.m, h->rho_slot, dt, predicted,
                                                      h->adj_G, h->adj_GR);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_pair_vjp(h, W, h->adj_G, h->adj_GR, h->adj_pair, st);
  if (e != cudaSuccess) return e;
  k_vjp_chain<<<g, kBlock, 0, st>>>(n, h->dp, W, adj, h->adj_pair, dt, predicted, h->adj_par);
  k_sum_params<<<1, 1024, 0, st>>>(n, h->adj_par, par);
  h->launches += 3;
  return cudaGetLastError();
}

}  // namespace csph
