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
// Antisymmetry: the momentum flux F_ij e^R that i and j apply are bitwise
// negatives of each other, and so are the energy fluxes Q_ij of FP64
// handles; mixed handles sum the energy flux from velocity differences
// (FwdAcc in pair_common.cuh).
//
// Modes of the kernel: the rates (optionally with order-2 states), the SPH
// gradients of order 2, the reverse mode, and the Verlet list build; the
// evaluation over the lists is k_pair_lists.cu.
//
// Mixed precision: the candidate test and the flux run in FP32 on offsets
// from each particle's own cell origin (FP32 keeps ~7 digits of a cell edge,
// not of the domain).  The FP32 test decides r^2 < R^2 whenever r^2 lies
// outside a band of 2^-12 D^c^2 around R^2, which bounds the accumulated
// FP32 error of both sides (<= ~1e-5 D^c^2); inside the band the pair is
// decided by the FP64 test on the global positions, with the same operation
// order as the oracle, so the pair set is the FP64 one.  Per-particle sums
// are Kahan-compensated.
#include "pair_common.cuh"

namespace csph {

namespace {

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
  chain_entry();
  constexpr bool VJP = MODE == kModeVjp;
  constexpr bool LIST = MODE == kModeList;
  constexpr bool GRAD = MODE == kModeGrad;
  using P = Pair<MIXED, DIM>;
  using T = typename P::T;
  using V4 = typename P::V4;
  using V2 = typename P::V2;
  using VC = typename P::VC;
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
  // the list build reads the cell-order copy of the positions when the lists
  // are laid out in the unit-major evaluation order
  const V4* __restrict__ A = reinterpret_cast<const V4*>(LIST && a.Ac ? a.Ac : a.A);
  const V4* __restrict__ B = reinterpret_cast<const V4*>(a.B);
  const VC* __restrict__ C = reinterpret_cast<const VC*>(a.C);
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
  if (LIST && a.vinst && a.vinst[b] == 0) continue;   // the instance keeps its lists (warp-uniform)
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
    const long long t_start = a.load_timed ? clock64() : 0;   // timed unit loads
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
    // list build: the home group's bounding box and largest kh d, a warp-wide cull of candidates
    float bxl = 0.f, bxh = 0.f, byl = 0.f, byh = 0.f, bzl = 0.f, bzh = 0.f, bkh = 0.f;
    if constexpr (LIST && MIXED) {
      bxl = (float)Ai.x; bxh = bxl; byl = (float)Ai.y; byh = byl; bzl = (float)Ai.z; bzh = bzl; bkh = (float)khdi;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        bxl = fminf(bxl, __shfl_xor_sync(0xffffffffu, bxl, o)); bxh = fmaxf(bxh, __shfl_xor_sync(0xffffffffu, bxh, o));
        byl = fminf(byl, __shfl_xor_sync(0xffffffffu, byl, o)); byh = fmaxf(byh, __shfl_xor_sync(0xffffffffu, byh, o));
        bzl = fminf(bzl, __shfl_xor_sync(0xffffffffu, bzl, o)); bzh = fmaxf(bzh, __shfl_xor_sync(0xffffffffu, bzh, o));
        bkh = fmaxf(bkh, __shfl_xor_sync(0xffffffffu, bkh, o));
      }
    }
    const int ui = a.K > 0 ? a.slot_unit[ii] : 0;
    const V4 Bi = B[ii];
    const VC Ci = C[ii];
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
      const VC Cj = C[j];
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
      T dv[3];
      if constexpr (MIXED) {   // relative velocities plus the exact reference difference
        dv[0] = dvel(Bi.x, Bj.x, Ci, Cj, 0);
        dv[1] = dvel(Bi.y, Bj.y, Ci, Cj, 1);
        dv[2] = dvel(Bi.z, Bj.z, Ci, Cj, 2);
      } else {
        dv[0] = Bj.x - Bi.x;
        dv[1] = Bj.y - Bi.y;
        dv[2] = Bj.z - Bi.z;
      }
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
      const VC Cj = C[j];
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
      T vi[3] = {Bi.x, Bi.y, Bi.z}, vj[3] = {Bj.x, Bj.y, Bj.z};
      if constexpr (MIXED) {   // lab-frame velocities: relative ones plus the references
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          vi[q] += ref_v(Ci, q);
          vj[q] += ref_v(Cj, q);
        }
      }
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
        const int64_t ih = a.e_of_c ? (int64_t)a.e_of_c[h0 + hp] : (int64_t)(h0 + hp);   // the row's slot
        const int64_t ihc = h0 + hp;                                                          // cell order
        for (int k0 = 0; k0 < n; k0 += 32) {
          const int k = k0 + lane;
          uint32_t word = 0;
          bool w = false;
          if (k < n) {
            const unsigned ent = list[warp][hp][k];
            const int64_t j = (int64_t)__float_as_int(nb_tab[warp][ent >> 11].x) + (ent & 2047u);
            w = j != ihc;
            const int64_t je = a.e_of_c ? (int64_t)a.e_of_c[j] : j;
            word = ((uint32_t)je << 5) | (ent >> 11);
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
            int nc = min(32, r1 - base);
            if constexpr (MIXED) {
              // keep only the candidates within reach of the home group's box
              // (a superset: every rounding below is monotone in the distance)
              const float ex = fmaxf(0.f, fmaxf((float)S.x - bxh, bxl - (float)S.x));
              const float ey = DIM >= 2 ? fmaxf(0.f, fmaxf((float)S.y - byh, byl - (float)S.y)) : 0.f;
              const float ez = DIM >= 3 ? fmaxf(0.f, fmaxf((float)S.z - bzh, bzl - (float)S.z)) : 0.f;
              const float Rm = fmaf(a.kh_f, (float)S.w, bkh);
              const bool keep = jv && fmaf(-Rm, Rm, P::r2_of(ex, ey, ez)) < band;
              const unsigned km = __ballot_sync(0xffffffffu, keep);
              if (keep) {
                const int q = __popc(km & lt);
                cand[warp][q] = S;
                cand_ent[warp][q] = (uint16_t)ent;
              }
              nc = __popc(km);
            } else {
              cand[warp][lane] = S;
              cand_ent[warp][lane] = (uint16_t)ent;
            }
            __syncwarp();
            // each lane tests its home particle against the chunk's candidates,
            // broadcast from shared memory, and appends the accepted ones to its
            // own list in candidate order
#pragma unroll 8
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
        a.vcnt[a.e_of_c ? a.e_of_c[i] : i] = vc < a.vcap ? vc : a.vcap;
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
      fw.fold();
      fw.write(a, i, nfull);
    }
    warp_counters(a, act, nfull, ncand, nexact, ui, lane,
                  a.load_timed ? (unsigned)(clock64() - t_start) : 0u);
    __syncwarp();   // the home buffer is rewritten by the next chunk of home particles
  }
  __syncwarp();     // the neighbour-start buffer is rewritten by the next cell
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
  return launch_chained(k_pair<MIXED, DIM, MODE, HLL, EXTRA>, dim3(sms * b), dim3(kPairBlock), st, args);
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
  if (h->unit_sched != SPH_SCHED_GLOBAL) {   // rows and entries in the unit-major evaluation order
    a.e_of_c = h->e_of_c;
    a.Ac = h->packAc;
  }
  // work counter zeroed by the step's k_pack (launch_pack with list_counters)
  a.work_counter = &h->counters[7];
  a.vinst = h->n_inst > 1 ? h->vinst : nullptr;   // only the instances whose lists are rebuilt
  cudaError_t e = h->dp.precision == SPH_PREC_MIXED ? launch_dim<true, kModeList>(h, a, st)
                                                    : launch_dim<false, kModeList>(h, a, st);
  h->launches += 1;
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
