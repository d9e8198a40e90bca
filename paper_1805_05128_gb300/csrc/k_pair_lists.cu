// k_pair_lists.cu -- the CSPH pair rates over the Verlet lists (Sec. 4.1-4.2
// with the buffered horizon of eq. (Dcell)): each list entry is tested as the
// cell search does, the fluxes of the interacting pairs (pair_common.cuh's
// FwdAcc) are summed per particle, and the step's second half kick is applied
// with the new rates.
#include "pair_common.cuh"

namespace csph {

namespace {

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
// neighbour-cell code, so the momentum fluxes stay antisymmetric bit for bit; every
// order is fixed, so results are reproducible bit for bit.

// Lanes per slot of k_pair_lists (a divisor of 32): measured on the 1.125M
// plate impact, 16 / 8 / 4 / 2 lanes per slot take 0.89 / 0.81 / 0.75 / 0.76 ms.
constexpr int kSlotLanes = 4;
constexpr int kSlotsPerWarp = 32 / kSlotLanes;

// Optional staging of the neighbour operands (sph_params.list_staging): the
// operands of the next chunk's entries are copied into shared memory with
// cp.async (16-byte copies, .ca: kept in L1 too) while the current chunk is
// evaluated, so their L2 latency overlaps the arithmetic without holding
// them in registers.  Each lane reads back only what it copied, after
// cp.async.wait_group, so no barrier is needed.  Measured slower than the
// plain gathers on GB300 (more instructions, shared-memory latency, a
// smaller L1 for the gathers that hit), so the default gathers through L1.
__device__ __forceinline__ void cp16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Sum over a slot's lanes of their Kahan sums (s - c), by a fixed butterfly.
template <typename T>
__device__ __forceinline__ T slot_sum(const Kahan<T>& k) {
  T v = k.s - k.c;
#pragma unroll
  for (int o = kSlotLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <bool MIXED, int DIM, bool HLL = false, bool EXTRA = true, bool STAGE = false, int KERN = SPH_KERNEL_CUBIC>
__global__ void __launch_bounds__(kPairBlock, MIXED ? 7 : 4) k_pair_lists(PairArgs a) {
  chain_entry();
  using P = Pair<MIXED, DIM>;
  using T = typename P::T;
  using V4 = typename P::V4;
  using VC = typename P::VC;
  __shared__ float res[kWarps][6][32];            // per slot of the group: sums of rho, a (3), E, and dmax
  __shared__ double res64[kWarps][6][MIXED ? 1 : 32];
  __shared__ unsigned res_n[kWarps][32];
  __shared__ long long t_start[kWarps];          // timed loads: start of the warp's slot iteration
  // unit shifts (-1, 0, 1) per axis of each neighbour-cell code; a table read
  // and three multiplies are cheaper than the integer divisions and
  // conversions of the decode, and give the same FP32 shifts bit for bit
  __shared__ float4 unit_shift[32];
  // STAGE: [warp][stage][16-byte chunk][lane]: A_j, B_j, C_j (3 chunks mixed, 5 in FP64)
  constexpr int kChA = (int)(sizeof(V4) / 16), kChC = (int)(sizeof(VC) / 16), kCh = 2 * kChA + kChC;
  __shared__ __align__(16) float4 stg[STAGE ? kWarps : 1][2][kCh][32];
  if (threadIdx.x < 32) {
    const int c = threadIdx.x;
    unit_shift[c] = make_float4((float)(c % 3 - 1), (float)((c / 3) % 3 - 1), (float)(c / 9 - 1), 0.f);
  }
  const int adj_n = EXTRA && a.collect_adj ? a.K * a.adj_words : 0;   // the block's adjacency tile
  if constexpr (EXTRA)
    for (int w = threadIdx.x; w < adj_n; w += blockDim.x) adj_tile()[w] = 0u;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int half = lane / kSlotLanes, hl = lane % kSlotLanes;   // the slot's group of lanes, lane in it
  const V4* __restrict__ A = reinterpret_cast<const V4*>(a.A);
  // Work partition.  SPH_SCHED_GLOBAL: groups of 32 consecutive slots from one
  // global counter.  Units: each unit owns a contiguous range of evaluation
  // slots and a counter; CTA b starts on unit b K / gridDim.x (the CTAs are
  // spread evenly over the units), takes groups of 32 slots of that unit and,
  // with SPH_SCHED_UNITS, moves on to the following units once it is drained
  // (each unit tried once; a drained unit is recognised by a plain read).  With
  // SPH_SCHED_UNITS_OWNED a warp stops when its home unit is drained.  Every
  // loop is bounded: no warp waits on another.
  // The scheduling state lives in shared memory (lane 0 of each warp), which
  // keeps the registers of the pair loop free.
  __shared__ int u_cur[kWarps], u_left[kWarps];
  __shared__ unsigned long long t_grp[kWarps];
  if (lane == 0) {
    // Home unit.  With stealing: from the SM the CTA runs on (the CTAs of one
    // SM share its L1, so they work on one unit's neighbourhood).  Owned: the
    // grid is K times the CTAs per unit and CTA b serves unit b / (gridDim.x / K),
    // so that every unit has the same resources and the step waits only for
    // the most loaded unit.
    int u = 0;
    if (a.unit_sched == SPH_SCHED_UNITS) {
      unsigned smid, nsm;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
      asm volatile("mov.u32 %0, %%nsmid;" : "=r"(nsm));
      u = (int)(((long long)smid * a.K) / (nsm > 0 ? nsm : 1));
    } else if (a.unit_sched == SPH_SCHED_UNITS_OWNED) {
      const int per = (int)gridDim.x / a.K;
      u = (int)blockIdx.x / (per > 0 ? per : 1);
    }
    u_cur[warp] = u < a.K ? u : a.K - 1;
    u_left[warp] = a.K;
  }
  for (;;) {
    // slots in 32 bits: list entries hold slot indices in 27 bits
    int g0 = 0, g1 = 0;
    if (a.unit_sched == SPH_SCHED_GLOBAL) {
      unsigned long long gw = 0;
      if (lane == 0) gw = atomicAdd(a.work_counter, 32ull);
      gw = __shfl_sync(0xffffffffu, gw, 0);
      if ((int64_t)gw >= a.n) break;
      g0 = (int)gw;
      g1 = (int64_t)g0 + 32 < a.n ? g0 + 32 : (int)a.n;
    } else {
      int ok = 0;
      if (lane == 0) {
        int u = u_cur[warp];
        for (;;) {
          const int ub = a.unit_eoff[u], ue = a.unit_eoff[u + 1];
          const unsigned long long size = (unsigned long long)(ue - ub);
          if (*reinterpret_cast<volatile unsigned long long*>(&a.unit_q[u]) < size) {
            const unsigned long long old = atomicAdd(&a.unit_q[u], 32ull);
            if (old < size) {
              g0 = ub + (int)old;
              g1 = g0 + 32 < ue ? g0 + 32 : ue;
              ok = 1;
              break;
            }
          }
          if (a.unit_sched == SPH_SCHED_UNITS_OWNED || --u_left[warp] <= 0) break;
          u = u + 1 == a.K ? 0 : u + 1;
        }
        u_cur[warp] = u;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        t_grp[warp] = t;
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      g0 = __shfl_sync(0xffffffffu, g0, 0);
      g1 = __shfl_sync(0xffffffffu, g1, 0);
    }
    int unit_run = -1;
    unsigned unit_load = 0;
    unsigned tf = 0, tc = 0, te = 0;
    // Half h of the warp takes slots g0 + 2q + h, q = 0..15.  The list reads
    // are software-pipelined: the next chunk of entries (and, across slots,
    // the next slot's first chunk and count) is requested before the current
    // one is evaluated, so the DRAM latency of the lists overlaps the L2
    // gathers and the arithmetic.  vcap >= 32, so the first chunk of any row
    // is in bounds.
    uint32_t e_pre = 0u, e_pre1 = 0u;
    int cnt_pre = 0;
    const V4* __restrict__ Bp = reinterpret_cast<const V4*>(a.B);
    const VC* __restrict__ Cp = reinterpret_cast<const VC*>(a.C);
    int stage = 0;
    // STAGE: copy the operands of entry e (or of slot `self`, a stand-in that
    // accepts nothing, for a lane without an entry) into stage st
    auto stage_ops = [&](int st, bool has, uint32_t e, int self) {
      const int64_t j = has ? (int64_t)(e >> 5) : (int64_t)self;
      const char* ga = reinterpret_cast<const char*>(A + j);
      const char* gb = reinterpret_cast<const char*>(Bp + j);
      const char* gc = reinterpret_cast<const char*>(Cp + j);
#pragma unroll
      for (int c = 0; c < kChA; ++c) cp16(&stg[warp][st][c][lane], ga + 16 * c);
#pragma unroll
      for (int c = 0; c < kChA; ++c) cp16(&stg[warp][st][kChA + c][lane], gb + 16 * c);
#pragma unroll
      for (int c = 0; c < kChC; ++c) cp16(&stg[warp][st][2 * kChA + c][lane], gc + 16 * c);
    };
    if (g0 + half < g1) {
      e_pre = a.vlist[(g0 + half) * (int64_t)a.vcap + hl];
      cnt_pre = a.vcnt[g0 + half];
      if constexpr (STAGE) e_pre1 = a.vlist[(g0 + half) * (int64_t)a.vcap + hl + kSlotLanes];
    }
    if constexpr (STAGE) {
      stage_ops(stage, g0 + half < g1 && hl < cnt_pre, e_pre, g0 + half < g1 ? g0 + half : g0);
      cp_commit();
    }
    for (int q = 0; g0 + kSlotsPerWarp * q < g1; ++q) {   // warp-uniform
      if (a.load_timed) {                                    // kept in shared memory: frees registers
        __syncwarp();
        if (lane == 0) t_start[warp] = clock64();
        __syncwarp();
      }
      const int i = g0 + kSlotsPerWarp * q + half;           // this group's slot
      const bool iv = i < g1;                                // uniform in the group
      const int cnt = iv ? cnt_pre : 0;
      uint32_t e_cur = e_pre;
      uint32_t e_nx = e_pre1;                                // STAGE: entry of this slot's chunk 1
      const bool nv = i + kSlotsPerWarp < g1;                // the group's next slot exists
      if (STAGE) cnt_pre = 0;
      if (nv) {
        e_pre = a.vlist[(i + kSlotsPerWarp) * (int64_t)a.vcap + hl];
        cnt_pre = a.vcnt[i + kSlotsPerWarp];
        if constexpr (STAGE) e_pre1 = a.vlist[(i + kSlotsPerWarp) * (int64_t)a.vcap + hl + kSlotLanes];
      }
      const int ii = iv ? i : g0;                     // a valid slot for the loads
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
      const V4 Bi = Bp[ii];
      const VC Ci = Cp[ii];
      const T khdi = MIXED ? (T)a.kh_f * Ai.w : T(0);
      const int ui = a.K > 0 ? a.slot_unit[ii] : 0;
      const uint32_t* __restrict__ row = a.vlist + (int64_t)ii * a.vcap;
      FwdAcc<MIXED, DIM, false, HLL, EXTRA, KERN> fw;
      fw.adj_local = true;
      unsigned nacc = 0;                              // accepted pairs of i (the slot's total after the loop)
      int cmax = cnt;                                 // chunks run by the whole warp
#pragma unroll
      for (int o = kSlotLanes; o < 32; o <<= 1) {
        const int other = __shfl_xor_sync(0xffffffffu, cmax, o);
        cmax = cmax > other ? cmax : other;
      }
      if constexpr (STAGE) {
        // the operands of chunk base are in stage `stage`; the next chunk's
        // (or, at the slot's last chunk, the next slot's first) are copied now
        const int inext = nv ? i + kSlotsPerWarp : ii;
        for (int base = 0; base < cmax; base += kSlotLanes) {
          const int k = base + hl;
          const bool kv = k < cnt;
          const uint32_t e_nn = row[k + 2 * kSlotLanes < a.vcap ? k + 2 * kSlotLanes : k];
          if (base + kSlotLanes < cmax) stage_ops(stage ^ 1, k + kSlotLanes < cnt, e_nx, ii);
          else stage_ops(stage ^ 1, hl < cnt_pre, e_pre, inext);
          cp_commit();
          cp_wait<1>();
          V4 Aj;
          V4 Bj;
          VC Cj;
          if constexpr (MIXED) {
            Aj = stg[warp][stage][0][lane];
            Bj = stg[warp][stage][1][lane];
            Cj = stg[warp][stage][2][lane];
          } else {
            const double2 a0 = reinterpret_cast<const double2&>(stg[warp][stage][0][lane]);
            const double2 a1 = reinterpret_cast<const double2&>(stg[warp][stage][1][lane]);
            const double2 b0 = reinterpret_cast<const double2&>(stg[warp][stage][2][lane]);
            const double2 b1 = reinterpret_cast<const double2&>(stg[warp][stage][3][lane]);
            const double2 c0 = reinterpret_cast<const double2&>(stg[warp][stage][4][lane]);
            Aj = V4{a0.x, a0.y, a1.x, a1.y};
            Bj = V4{b0.x, b0.y, b1.x, b1.y};
            Cj = VC{c0.x, c0.y};
          }
          const uint32_t e = kv ? e_cur : 0u;
          T sx = T(0), sy = T(0), sz = T(0);
          if constexpr (MIXED) {
            const float4 U = unit_shift[e & 31u];
            const float2 sxy = mul2(f2(U.x, U.y), f2(dcs, dcs));
            sx = sxy.x;
            sy = sxy.y;
            sz = U.z * dcs;
          }
          const bool acc = fw.pair_listed_ops(a, ii, Ai, Bi, Ci, ui, kv ? (int64_t)(e >> 5) : (int64_t)ii, Aj, Bj,
                                              Cj, sx, sy, sz, khdi, band, te, kv);
          nacc += acc ? 1u : 0u;
          stage ^= 1;
          e_cur = e_nx;
          e_nx = e_nn;
        }
        if (cmax == 0) {                              // no chunk ran: stage the next slot's first chunk here
          stage_ops(stage ^ 1, hl < cnt_pre, e_pre, inext);
          cp_commit();
          stage ^= 1;
        }
      }
      for (int base = 0; !STAGE && base < cmax; base += kSlotLanes) {
        const int k = base + hl;
        const bool kv = k < cnt;
        const uint32_t e = kv ? e_cur : 0u;
        // next chunk's entry, requested now (always inside the row: vcap >= 32;
        // past the slot's count it is read but not used)
        e_cur = row[k + kSlotLanes < a.vcap ? k + kSlotLanes : k];
        bool acc;
        {
          // lanes past their slot's last entry (e = 0) evaluate a stand-in and
          // accept nothing: no branch around the pair
          T sx = T(0), sy = T(0), sz = T(0);
          if constexpr (MIXED) {
            const float4 U = unit_shift[e & 31u];
            const float2 sxy = mul2(f2(U.x, U.y), f2(dcs, dcs));
            sx = sxy.x;
            sy = sxy.y;
            sz = U.z * dcs;
          }
          acc = fw.pair_listed(a, ii, Ai, Bi, Ci, ui, (int64_t)(e >> 5), sx, sy, sz, khdi, band, te, kv);
        }
        nacc += acc ? 1u : 0u;                        // this lane's accepted entries
      }
      fw.fold();
#pragma unroll
      for (int o = kSlotLanes / 2; o > 0; o >>= 1) nacc += __shfl_xor_sync(0xffffffffu, nacc, o);   // slot total
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
          const int r = i - g0;
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
          // timed loads: the iteration's SM cycles (the eight slots share them)
          unit_load += a.load_timed ? (unsigned)((clock64() - t_start[warp]) / kSlotsPerWarp) : nacc;
        }
      }
    }
    if constexpr (STAGE) cp_wait<0>();              // the last slot's stand-in copy, before the stages are reused
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
        double im;
        if constexpr (MIXED) {   // 1/m from the FP32 reciprocal and one FP64 Newton step (~1e-14 relative)
          const double mm = a.m[p];
          double r = (double)__frcp_rn((float)mm);
          r = r * __fma_rn(-mm, r, 2.0);
          im = a.fscale * r;
        } else {
          im = a.fscale / a.m[p];
        }
        const double acc[3] = {rv(1) * im, DIM >= 2 ? rv(2) * im : 0.0, DIM >= 3 ? rv(3) * im : 0.0};
        const double dE = rv(4) * im + lab_power_of<MIXED>(a, i, acc);
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
      if (a.unit_sched != SPH_SCHED_GLOBAL) {         // the unit's first start and last end
        unsigned long long t_end;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
        atomicMin(&a.unit_t[u_cur[warp]], t_grp[warp]);
        atomicMax(&a.unit_t[a.K + u_cur[warp]], t_end);
      }
    }
  }
  if constexpr (EXTRA) {                            // the block's adjacency bits into adj_bits
    __syncthreads();
    for (int w = threadIdx.x; w < adj_n; w += blockDim.x) {
      const uint32_t v = adj_tile()[w];
      if (v) atomicOr(&a.adj_bits[w], v);
    }
  }
}

template <bool MIXED, int DIM, bool HLL, bool EXTRA, bool STAGE, int KERN>
cudaError_t launch_lists_one(const PairArgs& args, int blocks_per_sm, cudaStream_t st) {
  static int sms = 0, per_sm = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair_lists<MIXED, DIM, HLL, EXTRA, STAGE, KERN>,
                                                  kPairBlock, 0);
    if (per_sm < 1) per_sm = 1;
  }
  const int b = (blocks_per_sm > 0 && blocks_per_sm < per_sm) ? blocks_per_sm : per_sm;
  int grid = sms * b;
  if (args.unit_sched == SPH_SCHED_UNITS_OWNED && args.K > 0)   // the same number of CTAs for every unit
    grid = args.K * (grid / args.K > 0 ? grid / args.K : 1);
  // A plain launch, not chained to the list build before it: chained, the
  // persistent list kernel made the step 8 % longer on the 1.125M plate
  // impact (1.20 against 1.11 ms) and 27 % on the 256-instance ensemble.  Its
  // entry still lets the next step's kernels launch early.
  k_pair_lists<MIXED, DIM, HLL, EXTRA, STAGE, KERN><<<grid, kPairBlock, 0, st>>>(args);
  return cudaGetLastError();
}

// The smoothing kernel as a template parameter: one derivative compiled in
// the pair loop instead of a run-time choice (1.5 % of the list kernel).
template <bool MIXED, bool HLL, bool EXTRA, bool STAGE, int KERN>
cudaError_t launch_lists_dim3k(sph_handle* h, const PairArgs& args, cudaStream_t st) {
  const int b = h->p.pair_blocks_per_sm;
  switch (h->dp.dim) {
    case 1: return launch_lists_one<MIXED, 1, HLL, EXTRA, STAGE, KERN>(args, b, st);
    case 2: return launch_lists_one<MIXED, 2, HLL, EXTRA, STAGE, KERN>(args, b, st);
    default: return launch_lists_one<MIXED, 3, HLL, EXTRA, STAGE, KERN>(args, b, st);
  }
}

template <bool MIXED, bool HLL, bool EXTRA, bool STAGE>
cudaError_t launch_lists_dim3(sph_handle* h, const PairArgs& args, cudaStream_t st) {
  return h->dp.kernel == SPH_KERNEL_WENDLAND_C2
             ? launch_lists_dim3k<MIXED, HLL, EXTRA, STAGE, SPH_KERNEL_WENDLAND_C2>(h, args, st)
             : launch_lists_dim3k<MIXED, HLL, EXTRA, STAGE, SPH_KERNEL_CUBIC>(h, args, st);
}

// Staged operands only for the mixed evaluations without side outputs (the
// benchmark's form); every other form gathers through L1.
template <bool MIXED, bool HLL, bool EXTRA>
cudaError_t launch_lists_stage(sph_handle* h, const PairArgs& args, cudaStream_t st) {
  if constexpr (MIXED && !EXTRA) {
    if (h->p.list_staging) return launch_lists_dim3<MIXED, HLL, EXTRA, true>(h, args, st);
  }
  return launch_lists_dim3<MIXED, HLL, EXTRA, false>(h, args, st);
}

// The side outputs (neighbour sizes, unit adjacency, pair output) only when
// this evaluation must produce them.
template <bool MIXED>
cudaError_t launch_lists_dim(sph_handle* h, const PairArgs& args, cudaStream_t st) {
  const bool extra = args.collect_adj || args.pair_i;
  if (h->solver == SPH_SOLVER_HLL)
    return extra ? launch_lists_stage<MIXED, true, true>(h, args, st) : launch_lists_stage<MIXED, true, false>(h, args, st);
  return extra ? launch_lists_stage<MIXED, false, true>(h, args, st) : launch_lists_stage<MIXED, false, false>(h, args, st);
}

}  // namespace

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
  // pair counts and work counter zeroed by the step's k_pack (launch_pack with list_counters)
  cudaError_t e = cudaSuccess;
  if (h->unit_sched != SPH_SCHED_GLOBAL) {
    // operands, lists and rows in the unit-major evaluation order; per-unit
    // queues and times reset for this launch (starts to the maximum, ends to 0)
    a.perm = h->perm_e;
    a.e_of_c = h->e_of_c;
    a.unit_eoff = h->unit_eoff;
    a.unit_q = h->unit_q;
    a.unit_t = h->unit_t;
    a.unit_sched = h->unit_sched;
    if ((e = cudaMemsetAsync(h->unit_q, 0, sizeof(unsigned long long) * h->K, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(h->unit_t, 0xff, sizeof(unsigned long long) * h->K, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(h->unit_t + h->K, 0, sizeof(unsigned long long) * h->K, st)) != cudaSuccess) return e;
  }
  if ((e = prof_record(h, true, st)) != cudaSuccess) return e;
  e = h->dp.precision == SPH_PREC_MIXED ? launch_lists_dim<true>(h, a, st) : launch_lists_dim<false>(h, a, st);
  h->launches += 1;
  if (e == cudaSuccess) e = prof_record(h, false, st);
  return e;
}

}  // namespace csph
