// k_step.cu -- per-particle kernels of the CSPH step (HBM-bound): CFL time
// step, kick-drift-kick updates, the cell mesh of eq. (Dcell) with a
// counting sort into cells, operand packing for the pair kernel, the
// renumbering of Sec. 4.2 and the FP64 conservation sums.
//
// Every per-particle kernel runs on "segmented" blocks: block b covers the
// particles [blk_start[b], blk_end[b]) of one instance, so per-instance
// reductions are fixed-order reductions over whole blocks (no atomics).
#include <cfloat>
#include <climits>

#include "csph_internal.cuh"
#include "step_math.cuh"

namespace csph {

namespace {

__device__ __forceinline__ double ld(const double* a, int64_t i) { return a ? a[i] : 0.0; }

// Return the status of a failed launch from the enclosing launcher.
#define CKL(call)                            \
  do {                                       \
    const cudaError_t ckl_e_ = (call);       \
    if (ckl_e_ != cudaSuccess) return ckl_e_; \
  } while (0)

__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

// Merge the top-2 multisets (a1 >= a2) and (b1 >= b2).
__device__ __forceinline__ void top2_merge(long long& a1, long long& a2, long long b1, long long b2) {
  if (a1 >= b1) { a2 = a2 > b1 ? a2 : b1; }
  else { a2 = b2 > a1 ? b2 : a1; a1 = b1; }
}

// Order keys of FP32 values (integer order = numeric order), as dkey.
__device__ __forceinline__ int fkey(float x) {
  const int b = __float_as_int(x);
  return b < 0 ? b ^ 0x7fffffff : b;
}
__device__ __forceinline__ float funkey(int k) { return __int_as_float(k < 0 ? k ^ 0x7fffffff : k); }

struct Red {
  long long lo[3], hi[3], d1, d2, dtmin, viol;
  int dlo[3], dhi[3];
};

__device__ __forceinline__ void red_init(Red& r) {
  for (int a = 0; a < 3; ++a) { r.lo[a] = LLONG_MAX; r.hi[a] = LLONG_MIN; r.dlo[a] = INT_MAX; r.dhi[a] = INT_MIN; }
  r.d1 = 0; r.d2 = 0; r.dtmin = LLONG_MAX; r.viol = LLONG_MIN;
}

__device__ __forceinline__ void red_merge(Red& a, const Red& b) {
  for (int k = 0; k < 3; ++k) {
    a.lo[k] = a.lo[k] < b.lo[k] ? a.lo[k] : b.lo[k];
    a.hi[k] = a.hi[k] > b.hi[k] ? a.hi[k] : b.hi[k];
    a.dlo[k] = min(a.dlo[k], b.dlo[k]);
    a.dhi[k] = max(a.dhi[k], b.dhi[k]);
  }
  top2_merge(a.d1, a.d2, b.d1, b.d2);
  a.dtmin = a.dtmin < b.dtmin ? a.dtmin : b.dtmin;
  a.viol = a.viol > b.viol ? a.viol : b.viol;
}

__device__ __forceinline__ Red shfl_red(const Red& r, int o) {
  Red q;
  for (int a = 0; a < 3; ++a) {
    q.lo[a] = __shfl_xor_sync(0xffffffffu, r.lo[a], o);
    q.hi[a] = __shfl_xor_sync(0xffffffffu, r.hi[a], o);
    q.dlo[a] = __shfl_xor_sync(0xffffffffu, r.dlo[a], o);
    q.dhi[a] = __shfl_xor_sync(0xffffffffu, r.dhi[a], o);
  }
  q.d1 = __shfl_xor_sync(0xffffffffu, r.d1, o);
  q.d2 = __shfl_xor_sync(0xffffffffu, r.d2, o);
  q.dtmin = __shfl_xor_sync(0xffffffffu, r.dtmin, o);
  q.viol = __shfl_xor_sync(0xffffffffu, r.viol, o);
  return q;
}

// Block-wide reduction of Red: butterfly within each warp, then the warp
// results through shared memory; result in thread 0.  Every merge is a
// min / max / top-2 of integer keys, so the order does not change the result.
__device__ void block_reduce(Red& r) {
  __shared__ Red sh[kBlock / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) red_merge(r, shfl_red(r, o));
  const int t = threadIdx.x;
  if ((t & 31) == 0) sh[t >> 5] = r;
  __syncthreads();
  if (t == 0)
    for (int w = 1; w < kBlock / 32; ++w) red_merge(r, sh[w]);
}

// Block minimum of the dt keys only (a step's k_derive); result in thread 0.
__device__ long long block_min_key(long long k) {
  __shared__ long long sh[kBlock / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long q = __shfl_xor_sync(0xffffffffu, k, o);
    k = q < k ? q : k;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = k;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < kBlock / 32; ++w) k = sh[w] < k ? sh[w] : k;
  return k;
}

__device__ __forceinline__ void write_part(BlockPart* part, const Red& r) {
  BlockPart& b = part[blockIdx.x];
  for (int a = 0; a < 3; ++a) { b.lo[a] = r.lo[a]; b.hi[a] = r.hi[a]; }
  b.d1 = r.d1; b.d2 = r.d2; b.dtmin = r.dtmin;
}

// ---------------------------------------------------------------------------
// d, P, c at the current state, dt_i = eta d_i / (c_i + |v_i|) (cfl_key),
// optional bbox.
// ---------------------------------------------------------------------------
__global__ void k_derive(DevParams P, sph_state s, const int64_t* __restrict__ blk_start,
                         const int64_t* __restrict__ blk_end, BlockPart* part, int write_derived,
                         int with_bbox) {
  chain_entry();
  int64_t p = blk_start[blockIdx.x] + threadIdx.x;
  Red r;
  red_init(r);
  if (p < blk_end[blockIdx.x] && !with_bbox && !write_derived) {
    // a step's CFL bound only (every load issued before the arithmetic)
    const double vx = ld(s.vx, p), vy = ld(s.vy, p), vz = ld(s.vz, p);
    const double E = s.E[p], rho = s.rho[p], m = s.m[p];
    const int mi = s.mat ? s.mat[p] : 0;
    r.dtmin = cfl_key(P, vx, vy, vz, E, rho, m, mi);
  } else if (p < blk_end[blockIdx.x]) {
    double vx = ld(s.vx, p), vy = ld(s.vy, p), vz = ld(s.vz, p);
    double v2 = vx * vx + vy * vy + vz * vz;
    double e = s.E[p] - 0.5 * v2;
    int mi = s.mat ? s.mat[p] : 0;
    double Pp, cp;
    eos(P.mat[mi], s.rho[p], e, Pp, cp);
    double d = size_of(P.dim, s.m[p], s.rho[p]);
    if (write_derived) { s.d[p] = d; s.P[p] = Pp; s.c[p] = cp; }
    r.dtmin = dkey((P.eta * d) / (cp + sqrt(v2)));
    if (with_bbox) {
      r.lo[0] = r.hi[0] = dkey(s.x[p]);
      if (P.dim >= 2) r.lo[1] = r.hi[1] = dkey(s.y[p]);
      if (P.dim >= 3) r.lo[2] = r.hi[2] = dkey(s.z[p]);
      r.d1 = dkey(d);
    }
  }
  if (!with_bbox) {   // a step's dt: only the minimum is read (the other partials come from k_kick_drift)
    const long long k = block_min_key(r.dtmin);
    if (threadIdx.x == 0) part[blockIdx.x].dtmin = k;
    return;
  }
  block_reduce(r);
  if (threadIdx.x == 0) write_part(part, r);
}

// One block per instance: the step's dt = cfl * (minimum of the instance's
// block minima).  Only the dtmin fields are read, four independent loads in
// flight per thread.
__global__ void k_reduce_dt(const int32_t* __restrict__ inst_blk, const BlockPart* __restrict__ part, double cfl,
                            double* dt, long long* dt_key, int from_key) {
  chain_entry();
  const int b = blockIdx.x;
  if (from_key) {   // the fused second kick's keys: already the instance minimum
    if (threadIdx.x == 0) {
      dt[b] = cfl * dunkey(dt_key[b]);
      dt_key[b] = LLONG_MAX;
    }
    return;
  }
  const int k0 = inst_blk[b], k1 = inst_blk[b + 1];
  long long m = LLONG_MAX;
  for (int k = k0 + threadIdx.x; k < k1; k += 4 * blockDim.x) {
    long long q[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int kk = k + u * blockDim.x;
      q[u] = kk < k1 ? part[kk].dtmin : LLONG_MAX;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) m = q[u] < m ? q[u] : m;
  }
  m = block_min_key(m);
  if (threadIdx.x == 0) {
    dt[b] = cfl * dunkey(m);
    dt_key[b] = LLONG_MAX;   // the next accumulation starts afresh
  }
}

// One block per instance: the bounding box and the two largest sizes of the
// instance from its block partials, into the grid record.
// vinst (Verlet steps): an instance that keeps its lists keeps its mesh geometry.
__global__ void k_reduce_inst(const int32_t* __restrict__ inst_blk, const BlockPart* __restrict__ part,
                              GridInfo* grid, const int* __restrict__ gate, const int* __restrict__ vinst) {
  chain_entry();
  if (gate && gate[0] == 0) return;   // Verlet mode: mesh kept from the last build
  int b = blockIdx.x;
  if (vinst && vinst[b] == 0) return;
  Red r;
  red_init(r);
  for (int k = inst_blk[b] + threadIdx.x; k < inst_blk[b + 1]; k += blockDim.x) {
    Red q;
    for (int a = 0; a < 3; ++a) { q.lo[a] = part[k].lo[a]; q.hi[a] = part[k].hi[a]; }
    q.d1 = part[k].d1; q.d2 = part[k].d2; q.dtmin = part[k].dtmin;
    red_merge(r, q);
  }
  block_reduce(r);
  if (threadIdx.x == 0) {
    GridInfo& g = grid[b];
    for (int a = 0; a < 3; ++a) { g.x0[a] = dunkey(r.lo[a]); g.hi[a] = dunkey(r.hi[a]); }
    g.dmax1 = dunkey(r.d1);
    g.dmax2 = dunkey(r.d2);
  }
}

// Cell mesh per instance (one block, a thread per instance): D^c of eq.
// (Dcell) with the safety margin, doubled until the instance's share of the
// cell capacity holds the mesh; dims per axis; then the global cell offsets
// in instance order.  Matches the oracle bit for bit.
// vinst (Verlet steps): an instance that keeps its lists keeps its geometry and
// only moves to its new cell offset.
__global__ void k_grid_setup(DevParams P, int n_inst, const int64_t* __restrict__ inst_off,
                             const int64_t* __restrict__ inst_cap, GridInfo* grid, int64_t* total_cells,
                             int* status, const int* __restrict__ gate, const int* __restrict__ vinst) {
  chain_entry();
  if (gate && gate[0] == 0) return;   // Verlet mode: mesh kept from the last build
  // the instances' meshes, one thread per instance
  for (int b = threadIdx.x; b < n_inst; b += blockDim.x) {
    GridInfo& g = grid[b];
    if (vinst && vinst[b] == 0) continue;
    double hi[3];
    for (int a = 0; a < 3; ++a) hi[a] = g.hi[a];
    for (int a = P.dim; a < 3; ++a) { g.x0[a] = 0.0; g.hi[a] = 0.0; hi[a] = 0.0; }
    double d1 = g.dmax1, d2 = g.dmax2;
    if (inst_off[b + 1] - inst_off[b] < 2) d2 = d1;
    double dc = __dmul_rn(P.kh, __dadd_rn(d1, d2));
    dc = __dmul_rn(dc, 1.0 + P.cell_beta);
    dc = __dmul_rn(dc, kCellMargin);
    if (!(dc > 0.0) || !isfinite(dc)) { set_status(status, SPH_ERR_NONFINITE); dc = 1.0; }
    int64_t tot;
    double inv;
    int64_t dims[3];
    for (int iter = 0; iter < 2100; ++iter) {
      inv = 1.0 / dc;
      tot = 1;
      for (int a = 0; a < 3; ++a) {
        dims[a] = (a < P.dim) ? (int64_t)floor(__dmul_rn(__dsub_rn(hi[a], g.x0[a]), inv)) + 1 : 1;
        tot *= dims[a];
      }
      if (tot <= inst_cap[b]) break;
      dc = dc * 2.0;
    }
    g.dc = dc;
    g.inv_dc = inv;
    for (int a = 0; a < 3; ++a) g.dims[a] = (int32_t)dims[a];
    g.ncells = tot;
    g.dc_f = (float)dc;
  }
  __syncthreads();
  if (n_inst == 1) {
    if (threadIdx.x == 0) {
      grid[0].cell_off = 0;
      *total_cells = grid[0].ncells;
    }
    return;
  }
  // global cell offsets in instance order (a kept instance only moves): an
  // exclusive scan of the cell counts over the block (warp scans, then the
  // warps' totals), a chunk of instances at a time
  __shared__ long long wsum[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  long long carry = 0;
  for (int base = 0; base < n_inst; base += blockDim.x) {
    const int b = base + (int)threadIdx.x;
    const long long v = b < n_inst ? (long long)grid[b].ncells : 0;
    long long x = v;                                   // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    long long before = 0, chunk = 0;                   // the earlier warps' totals, the chunk's total
    for (int k = 0; k < nw; ++k) {
      if (k < w) before += wsum[k];
      chunk += wsum[k];
    }
    if (b < n_inst) grid[b].cell_off = carry + before + x - v;
    carry += chunk;
    __syncthreads();                                   // wsum is rewritten by the next chunk
  }
  if (threadIdx.x == 0) *total_cells = carry;
}

__device__ __forceinline__ int64_t local_cell(const GridInfo& g, int dim, double x, double y, double z,
                                              int32_t c[3]) {
  c[0] = (int32_t)floor(__dmul_rn(__dsub_rn(x, g.x0[0]), g.inv_dc));
  c[1] = dim >= 2 ? (int32_t)floor(__dmul_rn(__dsub_rn(y, g.x0[1]), g.inv_dc)) : 0;
  c[2] = dim >= 3 ? (int32_t)floor(__dmul_rn(__dsub_rn(z, g.x0[2]), g.inv_dc)) : 0;
  return (int64_t)c[0] + (int64_t)g.dims[0] * ((int64_t)c[1] + (int64_t)g.dims[1] * c[2]);
}

// vinst (Verlet steps): the particles of an instance that keeps its lists are
// counted at their positions of its last build (vref), with its kept
// geometry, which reproduces that build's cells, slots and in-cell order.
__global__ void k_cell_count(int dim, sph_state s, const int64_t* __restrict__ blk_start,
                             const int64_t* __restrict__ blk_end, const int32_t* __restrict__ blk_inst, int nblk,
                             const GridInfo* __restrict__ grid, int32_t* cell_count, int32_t* cell_of,
                             int32_t* rank, int* status, const int* __restrict__ gate, const int* __restrict__ vinst,
                             const double* __restrict__ vref, int64_t n) {
  chain_entry();
  if (gate && gate[0] == 0) return;   // Verlet mode: mesh kept from the last build
  // a capped grid strides over the segmented blocks (cheap to launch when gated)
  for (int lb = blockIdx.x; lb < nblk; lb += gridDim.x) {
    const int64_t p = blk_start[lb] + threadIdx.x;
    if (p >= blk_end[lb]) continue;
    const int b = blk_inst[lb];
    const GridInfo& g = grid[b];
    const bool kept = vinst && vinst[b] == 0;
    const double px = kept ? vref[p] : s.x[p];
    const double py = dim >= 2 ? (kept ? vref[n + p] : s.y[p]) : 0.0;
    const double pz = dim >= 3 ? (kept ? vref[2 * n + p] : s.z[p]) : 0.0;
    int32_t c[3];
    int64_t lc = local_cell(g, dim, px, py, pz, c);
    bool ok = true;
    for (int a = 0; a < 3; ++a) ok = ok && c[a] >= 0 && c[a] < g.dims[a];
    if (!ok) {  // only a non-finite position can leave the mesh: latch it, stay in bounds
      set_status(status, SPH_ERR_NONFINITE);
      lc = 0;
    }
    const int32_t gc = (int32_t)(g.cell_off + lc);
    cell_of[p] = gc;
    rank[p] = atomicAdd(&cell_count[gc], 1);
  }
}

// Exclusive scan of cell_count[0, total) into cell_start, 1024 cells per tile.
constexpr int kScanTile = 1024;

__global__ void k_scan_reduce(const int32_t* __restrict__ cnt, const int64_t* __restrict__ total,
                              int32_t* sums, const int* __restrict__ gate) {
  chain_entry();
  if (gate && gate[0] == 0) return;   // Verlet mode: mesh kept from the last build
  const int64_t tot = *total;
  __shared__ int sh[kBlock];
  // grid-stride over the tiles the current mesh has (the grid is sized for the capacity,
  // capped at a few waves)
  for (int64_t t = blockIdx.x; t * kScanTile < tot; t += gridDim.x) {
    const int64_t base = t * kScanTile;
    int v = 0;
    for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
      int64_t c = base + k;
      if (c < tot) v += cnt[c];
    }
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) sums[t] = sh[0];
    __syncthreads();
  }
}

// Single block: exclusive scan of the tile sums in place.
__global__ void k_scan_sums(int32_t* sums, const int64_t* __restrict__ total, const int* __restrict__ gate) {
  chain_entry();
  if (gate && gate[0] == 0) return;   // Verlet mode: mesh kept from the last build
  int64_t ntiles = (*total + kScanTile - 1) / kScanTile;
  __shared__ int carry;
  __shared__ int sh[1024];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < ntiles; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int v = (i < ntiles) ? sums[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
      int add = threadIdx.x >= (unsigned)off ? sh[threadIdx.x - off] : 0;
      __syncthreads();
      sh[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < ntiles) sums[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += sh[threadIdx.x];
    __syncthreads();
  }
}

// Per tile: exclusive scan plus tile offset; zero the counts for the next use.
__global__ void k_scan_down(int32_t* cnt, const int64_t* __restrict__ total, const int32_t* __restrict__ sums,
                            int32_t* start, int64_t n_total, const int* __restrict__ gate) {
  chain_entry();
  if (gate && gate[0] == 0) return;   // Verlet mode: mesh kept from the last build
  const int64_t tot = *total;
  constexpr int per = kScanTile / kBlock;  // 4 cells per thread
  __shared__ int sh[kBlock];
  for (int64_t t = blockIdx.x; t * kScanTile < tot; t += gridDim.x) {
    const int64_t base = t * kScanTile;
    int vals[per];
    int run = 0;
    for (int k = 0; k < per; ++k) {
      int64_t c = base + threadIdx.x * per + k;
      vals[k] = (c < tot) ? cnt[c] : 0;
      run += vals[k];
    }
    sh[threadIdx.x] = run;
    __syncthreads();
    for (int off = 1; off < kBlock; off <<= 1) {
      int add = threadIdx.x >= (unsigned)off ? sh[threadIdx.x - off] : 0;
      __syncthreads();
      sh[threadIdx.x] += add;
      __syncthreads();
    }
    int acc = sums[t] + sh[threadIdx.x] - run;
    for (int k = 0; k < per; ++k) {
      int64_t c = base + threadIdx.x * per + k;
      if (c < tot) {
        start[c] = acc;
        acc += vals[k];
        cnt[c] = 0;
      }
    }
    if (base + kScanTile >= tot && threadIdx.x == 0) start[tot] = (int32_t)n_total;
    __syncthreads();
  }
}

// vinst (Verlet steps): the slots of an instance that keeps its lists keep
// their particles (its cells' starts come out as before), so its particles
// are not scattered, and its cells are not sorted below.
__global__ void k_cell_scatter(int64_t n, const int32_t* __restrict__ cell_of, const int32_t* __restrict__ rank,
                               const int32_t* __restrict__ start, int32_t* perm, const int* __restrict__ gate,
                               const int* __restrict__ vinst, const int64_t* __restrict__ inst_off, int n_inst) {
  chain_entry();
  if (gate && gate[0] == 0) return;   // Verlet mode: mesh kept from the last build
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    if (vinst) {
      int lo = 0, hi = n_inst;                       // the particle's instance
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (inst_off[mid] <= p) lo = mid; else hi = mid;
      }
      if (vinst[lo] == 0) continue;
    }
    perm[start[cell_of[p]] + rank[p]] = (int32_t)p;
  }
}

// Within each cell, order the particles by index (the atomic arrival order is
// not reproducible; this makes the slot order a function of the state only).
// Mixed precision: also the origin of each cell, o = x0 + c dc per axis, for
// every slot of the cell (slot_org; k_pack takes the FP32 offsets from it).
__global__ void k_cell_sort(const int64_t* __restrict__ total, const int32_t* __restrict__ start, int32_t* perm,
                            const int* __restrict__ gate, const GridInfo* __restrict__ grid, int n_inst, int dim,
                            int64_t nslots, double* slot_org, const int* __restrict__ vinst) {
  chain_entry();
  if (gate && gate[0] == 0) return;   // Verlet mode: mesh kept from the last build
  // One warp per cell: each lane holds up to kSortPer of the cell's particle
  // indices and counts, by broadcasts, the cell's indices smaller than each
  // (indices are distinct), which is its position in ascending order.  Cells
  // above 32 kSortPer particles (never on a sane mesh: the cell code admits
  // 2047) are sorted by one lane.
  constexpr int kSortPer = 4;
  const int64_t tot = *total;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = w0; c < tot; c += nw) {
    const int b = start[c], e = start[c + 1], n = e - b;
    if (n <= 0) continue;
    int bi = 0;                                      // the cell's instance
    if (n_inst > 1 && (slot_org || vinst)) {
      int lo = 0, hi = n_inst;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (grid[mid].cell_off <= c) lo = mid; else hi = mid;
      }
      bi = lo;
    }
    if (vinst && vinst[bi] == 0) continue;          // kept: slots, order and origins as they are
    if (slot_org) {
      const GridInfo& g = grid[bi];
      const int64_t lc = c - g.cell_off;
      const int64_t cc[3] = {lc % g.dims[0], (lc / g.dims[0]) % g.dims[1], lc / ((int64_t)g.dims[0] * g.dims[1])};
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (a < dim) {
          const double o = __fma_rn((double)cc[a], g.dc, g.x0[a]);
          for (int k = b + lane; k < e; k += 32) slot_org[(int64_t)a * nslots + k] = o;
        }
    }
    if (n <= 1) continue;
    if (n > 32 * kSortPer) {
      if (lane == 0)
        for (int i = b + 1; i < e; ++i) {
          int32_t v = perm[i];
          int j = i - 1;
          while (j >= b && perm[j] > v) { perm[j + 1] = perm[j]; --j; }
          perm[j + 1] = v;
        }
      __syncwarp();
      continue;
    }
    int32_t v[kSortPer];
    int rank[kSortPer];
#pragma unroll
    for (int q = 0; q < kSortPer; ++q) {
      v[q] = lane + 32 * q < n ? perm[b + lane + 32 * q] : INT_MAX;
      rank[q] = 0;
    }
    const int rounds = (n + 31) >> 5;
    for (int r = 0; r < rounds; ++r) {
      const int cnt = min(32, n - 32 * r);
      int32_t mine = INT_MAX;
#pragma unroll
      for (int q = 0; q < kSortPer; ++q)
        if (q == r) mine = v[q];
      for (int k = 0; k < cnt; ++k) {
        const int32_t t = __shfl_sync(0xffffffffu, mine, k);
#pragma unroll
        for (int q = 0; q < kSortPer; ++q) rank[q] += t < v[q] ? 1 : 0;
      }
    }
    __syncwarp();   // every index read before any is written back
#pragma unroll
    for (int q = 0; q < kSortPer; ++q)
      if (lane + 32 * q < n) perm[b + rank[q]] = v[q];
  }
}

// ---------------------------------------------------------------------------
// Kick-drift: v <- v + dt/2 a, x <- x + dt v, rho, E half kicks; predicted
// size d~ from rho~ = rho^h + dt/2 drho; bounding box and sizes for the mesh.
// ---------------------------------------------------------------------------
template <bool MIXED>
__global__ void __launch_bounds__(kBlock, 4) k_kick_drift(DevParams P, sph_state s, const int64_t* __restrict__ blk_start,
                             const int64_t* __restrict__ blk_end, const int32_t* __restrict__ blk_inst,
                             const double* __restrict__ dt, BlockPart* part, int* status) {
  chain_entry();
  int64_t p = blk_start[blockIdx.x] + threadIdx.x;
  Red r;
  red_init(r);
  if (p < blk_end[blockIdx.x]) {
    const int dim = P.dim;
    const double h = dt[blk_inst[blockIdx.x]];
    const double hdt = 0.5 * h;
    double* X[3] = {s.x, s.y, s.z};
    double* V[3] = {s.vx, s.vy, s.vz};
    const double* A[3] = {s.ax, s.ay, s.az};
    // Every load is issued before the first store: the state arrays may alias
    // as far as the compiler can tell, so a load placed after a store would
    // wait for it, one memory round trip per component.
    double x[3] = {0.0, 0.0, 0.0}, v[3] = {0.0, 0.0, 0.0}, acc[3] = {0.0, 0.0, 0.0}, xb[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a < dim) {
        x[a] = X[a][p];
        v[a] = V[a][p];
        acc[a] = A[a][p];
        if (P.vref) xb[a] = P.vref[(int64_t)a * P.n + p];
      }
    const double rho0 = s.rho[p], drho = s.drho[p], E0 = s.E[p], dE = s.dE[p], m = s.m[p];
    const double db = P.vref ? P.vref[3 * P.n + p] : 0.0;
    bool finite = true;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a < dim) {
        v[a] = axpy<MIXED>(hdt, acc[a], v[a]);
        x[a] = axpy<MIXED>(h, v[a], x[a]);
        r.lo[a] = r.hi[a] = dkey(x[a]);
        finite = finite && finite_bits(x[a]);
      }
    const double rh = axpy<MIXED>(hdt, drho, rho0);
    const double En = axpy<MIXED>(hdt, dE, E0);
    const double rp = axpy<MIXED>(hdt, drho, rh);
    const double d = MIXED ? size_of_mixed(dim, m, rp) : size_of(dim, m, rp);
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a < dim) { V[a][p] = v[a]; X[a][p] = x[a]; }
    s.rho[p] = rh;
    s.E[p] = En;
    s.d[p] = d;
    r.d1 = dkey(d);
    if (P.vref) {
      // Verlet-list validity: a listed superset of the pairs within kappa h_ij holds as long
      // as |x_i - x_i^b - U| + kh max(0, d_i - d_i^b) <= beta kh d_i^b for every particle
      // (b: the last build).  U is one displacement shared by all particles, any vector:
      // the separation of a pair changes by (x_j - x_j^b - U) - (x_i - x_i^b - U), so
      // summing the bounds of i and j covers the pair.  U follows the bulk motion (the
      // midpoint of the displacement box, extrapolated from the previous step), so a body
      // in uniform motion keeps its lists.  Kept with a 5 % margin (differences in FP64,
      // the bound itself in FP32: the 5 % margin dwarfs its rounding).
      // (The displacement and U in FP32: their rounding, ~1e-7 of each, is far
      // inside the margin.)  The box is that of x - x^b - U.
      const float* Uf = reinterpret_cast<const float*>(P.vframe + 6 * blk_inst[blockIdx.x] + 4);
      float dsq = 0.0f;
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (a < dim) {
          const float dx = f32_rn(x[a] - xb[a]) - Uf[a];
          dsq += dx * dx;
          r.dlo[a] = r.dhi[a] = fkey(dx);
        }
      const float kh = P.kh_f;
      const float crit = sqrtf(dsq) + kh * fmaxf(f32_rn(d - db), 0.0f) - 0.95f * P.cell_beta_f * kh * f32_rn(db);
      r.viol = dkey(f64_of(crit));
    }
    if (!finite || !finite_bits(d)) set_status(status, SPH_ERR_NONFINITE);
  }
  block_reduce(r);
  if (threadIdx.x == 0) {
    write_part(part, r);
    if (P.vacc) {                  // the criterion's maximum and displacement box of the instance
      VAcc* va = P.vacc + blk_inst[blockIdx.x];
      atomicMax(&va->viol, r.viol);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        atomicMin(&va->dlo[a], r.dlo[a]);
        atomicMax(&va->dhi[a], r.dhi[a]);
      }
    }
  }
}

// Second half kick with the rates of the predicted state; instance time.
// With part, also the block minima of the CFL keys at the new state, which
// the next step of the same sph_step call takes instead of a k_derive pass.
template <bool MIXED>
__global__ void k_kick2(DevParams P, sph_state s, const int64_t* __restrict__ blk_start,
                        const int64_t* __restrict__ blk_end, const int32_t* __restrict__ blk_inst,
                        const int32_t* __restrict__ inst_blk, const double* __restrict__ dt, double* t_dev,
                        BlockPart* part) {
  chain_entry();
  const int64_t p = blk_start[blockIdx.x] + threadIdx.x;
  const int b = blk_inst[blockIdx.x];
  if (t_dev && threadIdx.x == 0 && inst_blk[b] == (int)blockIdx.x) t_dev[b] += dt[b];
  long long key = LLONG_MAX;
  if (p < blk_end[blockIdx.x]) {
    const int dim = P.dim;
    const double hdt = 0.5 * dt[b];
    double* V[3] = {s.vx, s.vy, s.vz};
    const double* A[3] = {s.ax, s.ay, s.az};
    double v[3] = {0.0, 0.0, 0.0}, acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a < dim) { v[a] = V[a][p]; acc[a] = A[a][p]; }
    const double rho0 = s.rho[p], drho = s.drho[p], E0 = s.E[p], dE = s.dE[p];
    double m = 0.0;
    int mi = 0;
    if (part) { m = s.m[p]; mi = s.mat ? s.mat[p] : 0; }
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a < dim) v[a] = axpy<MIXED>(hdt, acc[a], v[a]);
    const double rho = axpy<MIXED>(hdt, drho, rho0);
    const double E = axpy<MIXED>(hdt, dE, E0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a < dim) V[a][p] = v[a];
    s.rho[p] = rho;
    s.E[p] = E;
    if (part) key = cfl_key(P, v[0], v[1], v[2], E, rho, m, mi);
  }
  if (part) {   // uniform over the grid: every thread reaches the block barrier
    const long long k = block_min_key(key);
    if (threadIdx.x == 0) part[blockIdx.x].dtmin = k;
  }
}

// ---------------------------------------------------------------------------
// Pack the pair operands in slot order.  With predict, the state holds the
// half-step values q^h and the rates q' of the previous evaluation and the
// operands are the predicted q~ = q^h + dt/2 q'.  P and c of the packed state
// are written back to the particle arrays.
//   mixed: A = {x - o, y - o, z - o, d} (FP32 offsets from the particle's own
//          cell origin o, the local-origin idea of Sec. 3.1), B = {v, m/rho},
//          C = {P, rho c}
//   fp64 : A = {x, y, z, d} (global positions), B, C in FP64
// ---------------------------------------------------------------------------
template <bool MIXED>
__global__ void __launch_bounds__(kBlock, 4) k_pack(DevParams P, sph_state s, const int64_t* __restrict__ blk_start,
                       const int64_t* __restrict__ blk_end, const int32_t* __restrict__ blk_inst,
                       const GridInfo* __restrict__ grid, const double* __restrict__ dt, int predict,
                       const int32_t* __restrict__ perm, const int32_t* __restrict__ cell_of,
                       void* packA, void* packB, void* packC, double* rho_slot, int32_t* slot_cell,
                       int32_t* slot_unit, int n_units, int* status, const int32_t* __restrict__ e_of_c,
                       int32_t* perm_e, void* packAc, const int* __restrict__ gate,
                       unsigned long long* list_counters) {
  chain_entry();
  // the counters of the list build and the list evaluation that follow (the
  // evaluation's pair counts and work counter, the build's work counter)
  if (list_counters && blockIdx.x == 0 && threadIdx.x == 0) {
    list_counters[0] = 0ull;
    list_counters[1] = 0ull;
    list_counters[2] = 0ull;
    list_counters[5] = 0ull;
    list_counters[7] = 0ull;
  }
  const int64_t sc = blk_start[blockIdx.x] + threadIdx.x;     // cell-order slot
  if (sc >= blk_end[blockIdx.x]) return;
  // the operands go to the slot's evaluation position (unit-major order of the
  // last list build), or to the cell-order slot itself
  const int64_t sl = e_of_c ? (int64_t)e_of_c[sc] : sc;
  const bool build = packAc && gate && gate[0] != 0;          // a list build follows: cell-order copy of A
  int b = blk_inst[blockIdx.x];
  int64_t p = perm[sc];
  if (perm_e) perm_e[sl] = (int32_t)p;
  // every load of the gathered particle first (the stores to P and c below
  // would otherwise hold back the loads placed after them)
  const bool pr = predict != 0;
  double v[3] = {ld(s.vx, p), ld(s.vy, p), ld(s.vz, p)};
  double acc[3] = {0.0, 0.0, 0.0};
  if (pr) {
    acc[0] = s.ax[p];
    if (P.dim >= 2) acc[1] = s.ay[p];
    if (P.dim >= 3) acc[2] = s.az[p];
  }
  const double rho0 = s.rho[p], E0 = s.E[p];
  const double drho = pr ? s.drho[p] : 0.0, dE = pr ? s.dE[p] : 0.0;
  const int mi = s.mat ? s.mat[p] : 0;
  const double d = s.d[p];
  const double m = s.m[p];
  const double X[3] = {s.x[p], P.dim >= 2 ? s.y[p] : 0.0, P.dim >= 3 ? s.z[p] : 0.0};
  const int32_t gc = cell_of[p];
  int32_t u = s.unit ? s.unit[p] : 0;
  const double hdt = pr ? 0.5 * dt[b] : 0.0;
  if (pr) {
    v[0] = axpy<MIXED>(hdt, acc[0], v[0]);
    if (P.dim >= 2) v[1] = axpy<MIXED>(hdt, acc[1], v[1]);
    if (P.dim >= 3) v[2] = axpy<MIXED>(hdt, acc[2], v[2]);
  }
  double rho = pr ? axpy<MIXED>(hdt, drho, rho0) : rho0;
  double E = pr ? axpy<MIXED>(hdt, dE, E0) : E0;
  double e = E - 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  double Pp, cp;
  float cf = 0.0f;
  const Mat& mt = P.mat[mi];
  const bool fast = MIXED && predict &&
                    (mt.eos == SPH_EOS_IDEAL || mt.eos == SPH_EOS_STIFFENED || (mt.eos == SPH_EOS_TAIT && mt.tait_n > 0));
  if (fast) {
    // a mixed step packs FP32 operands: P in FP64 (the stiffened-gas and Tait
    // differences of two large terms, the expressions of eos()), c in FP32
    if (mt.eos == SPH_EOS_TAIT) Pp = mt.tait_B * (ipow(rho / mt.rho0, mt.tait_n) - 1.0);
    else Pp = (mt.gamma - 1.0) * rho * e - (mt.eos == SPH_EOS_STIFFENED ? mt.gamma * mt.p_inf : 0.0);
    cf = sound_speed_f32(mt, f32_rn(rho), f32_rn(e));
    cp = f64_of(cf);
  } else {
    eos(mt, rho, e, Pp, cp);
    cf = (float)cp;
  }
  s.P[p] = Pp;
  s.c[p] = cp;
  slot_cell[sl] = gc;
  if (u < 0 || u >= n_units) { if (n_units > 0) set_status(status, SPH_ERR_INVALID); u = 0; }
  slot_unit[sl] = u;
  rho_slot[sl] = rho;
  if (MIXED) {
    // FP32 offsets from the slot's cell origin (written at the mesh build)
    float off[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a < P.dim) off[a] = f32_rn(X[a] - P.slot_org[(int64_t)a * P.n + sc]);
    const float4 Arec = make_float4(off[0], off[1], off[2], f32_rn(d));
    reinterpret_cast<float4*>(packA)[sl] = Arec;
    if (build) reinterpret_cast<float4*>(packAc)[sc] = Arec;
    const float Vp = fast ? (f32_rn(m) / f32_rn(rho)) * P.vscale_f : (float)((m / rho) * P.vscale);
    // FP32 velocities relative to a reference velocity of whole m/s per
    // particle (k = v truncated, |k| <= 32767): v - k is exact in FP64 and
    // small, so FP32 keeps the velocity differences between neighbours to
    // ~1e-8 m/s instead of one ulp of the bulk velocity.  The references are
    // stored exactly: x and y biased by 32768 in the halves of one word,
    // z as a float.
    int k[3] = {0, 0, 0};
    float vr[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a < P.dim) vr[a] = f32_rn(v[a] - trunc_ref(v[a], k[a]));
    const uint32_t kxy = (uint32_t)(k[0] + 32768) | ((uint32_t)(k[1] + 32768) << 16);
    reinterpret_cast<float4*>(packB)[sl] = make_float4(vr[0], vr[1], vr[2], Vp);
    reinterpret_cast<float4*>(packC)[sl] = make_float4(f32_rn(Pp), fast ? f32_rn(rho) * cf : (float)(rho * cp),
                                                       __uint_as_float(kxy), (float)k[2]);
  } else {
    reinterpret_cast<D4*>(packA)[sl] = D4{X[0], X[1], X[2], d};
    if (build) reinterpret_cast<D4*>(packAc)[sc] = D4{X[0], X[1], X[2], d};
    reinterpret_cast<D4*>(packB)[sl] = D4{v[0], v[1], v[2], m / rho};
    reinterpret_cast<D2*>(packC)[sl] = D2{Pp, rho * cp};
  }
}

// ---------------------------------------------------------------------------
// Renumbering: gather every per-particle array through perm, copy back.
// ---------------------------------------------------------------------------
constexpr int kMaxPermArrays = 24;
struct PermArrays {
  void* ptr[kMaxPermArrays];
  int bytes[kMaxPermArrays];   // element size: 4 or 8
  int count;
};

__global__ void k_gather(int64_t n, const int32_t* __restrict__ perm, PermArrays a, char* scratch) {
  int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= n) return;
  int64_t p = perm[sl];
  size_t off = 0;
  for (int k = 0; k < a.count; ++k) {
    if (a.bytes[k] == 8) reinterpret_cast<uint64_t*>(scratch + off)[sl] = reinterpret_cast<const uint64_t*>(a.ptr[k])[p];
    else reinterpret_cast<uint32_t*>(scratch + off)[sl] = reinterpret_cast<const uint32_t*>(a.ptr[k])[p];
    off += (size_t)a.bytes[k] * n;
  }
}

// Writes the gathered arrays back; with perm, also makes the slot order the
// identity (particle sl now sits in slot sl).
__global__ void k_scatter_back(int64_t n, PermArrays a, const char* scratch, int32_t* perm) {
  int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= n) return;
  size_t off = 0;
  for (int k = 0; k < a.count; ++k) {
    if (a.bytes[k] == 8) reinterpret_cast<uint64_t*>(a.ptr[k])[sl] = reinterpret_cast<const uint64_t*>(scratch + off)[sl];
    else reinterpret_cast<uint32_t*>(a.ptr[k])[sl] = reinterpret_cast<const uint32_t*>(scratch + off)[sl];
    off += (size_t)a.bytes[k] * n;
  }
  if (perm) perm[sl] = (int32_t)sl;
}

// ---------------------------------------------------------------------------
// FP64 conservation sums per instance, fixed order: thread t sums particles
// t, t + blockDim, ...; then a tree over threads.
// ---------------------------------------------------------------------------
__global__ void k_conservation(sph_state s, const int64_t* __restrict__ inst_off, double* out) {
  int b = blockIdx.x;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int64_t p = inst_off[b] + threadIdx.x; p < inst_off[b + 1]; p += blockDim.x) {
    double m = s.m[p];
    acc[0] += m;
    acc[1] += m * ld(s.vx, p);
    acc[2] += m * ld(s.vy, p);
    acc[3] += m * ld(s.vz, p);
    acc[4] += m * s.E[p];
  }
  __shared__ double sh[5][kBlock];
  for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kBlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) out[b * 5 + k] = sh[k][0];
}

__global__ void k_check_finite(int dim, sph_state s, int64_t n, int* status) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  bool ok = isfinite(s.x[p]) && isfinite(s.vx[p]) && isfinite(s.rho[p]) && isfinite(s.E[p]) &&
            isfinite(s.m[p]) && s.rho[p] > 0.0 && s.m[p] > 0.0;
  if (dim >= 2) ok = ok && isfinite(s.y[p]) && isfinite(s.vy[p]);
  if (dim >= 3) ok = ok && isfinite(s.z[p]) && isfinite(s.vz[p]);
  if (!ok) set_status(status, SPH_ERR_NONFINITE);
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// Grids over the mesh capacity, whose kernels read the live cell count on the
// device and stride over it: at most 8 blocks of kBlock per SM, so a generous
// capacity costs no empty waves.
static int capped_grid(int want) {
  static int cap = 0;
  if (cap == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cap = 8 * (sms > 0 ? sms : 1);
  }
  return want < cap ? (want > 0 ? want : 1) : cap;
}

cudaError_t launch_derive_dt(sph_handle* h, const sph_state& s, bool with_bbox, cudaStream_t st) {
  CKL(launch_chained(k_derive, dim3(h->nblk), dim3(kBlock), st, h->dp, s, h->blk_start, h->blk_end, h->part, with_bbox ? 1 : 0,
                                       with_bbox ? 1 : 0));
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_reduce_dt(sph_handle* h, cudaStream_t st, bool from_key) {
  CKL(launch_chained(k_reduce_dt, dim3(h->n_inst), dim3(kBlock), st, h->inst_blk, h->part, h->dp.cfl, h->dt, h->dt_key, from_key ? 1 : 0));
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_kick_drift(sph_handle* h, const sph_state& s, cudaStream_t st) {
  if (h->dp.precision == SPH_PREC_MIXED)
    CKL(launch_chained(k_kick_drift<true>, dim3(h->nblk), dim3(kBlock), st, h->dp, s, h->blk_start, h->blk_end, h->blk_inst, h->dt, h->part,
                                                   h->status));
  else
    CKL(launch_chained(k_kick_drift<false>, dim3(h->nblk), dim3(kBlock), st, h->dp, s, h->blk_start, h->blk_end, h->blk_inst, h->dt, h->part,
                                                    h->status));
  h->launches += 1;
  return cudaGetLastError();
}

// Mesh from the block partials left by k_derive(with_bbox) or k_kick_drift,
// then the counting sort of particles into cells.
cudaError_t launch_build_grid(sph_handle* h, const sph_state& s, cudaStream_t st, const int* gate) {
  // per-instance rebuilds only inside the Verlet sequence (gated) of a batched
  // handle; any other build is global (one instance: the same thing)
  const int* vinst = gate && h->n_inst > 1 ? h->vinst : nullptr;
  CKL(launch_chained(k_reduce_inst, dim3(h->n_inst), dim3(kBlock), st, h->inst_blk, h->part, h->grid, gate, vinst));
  CKL(launch_chained(k_grid_setup, dim3(1), dim3(h->n_inst < 1024 ? 32 * ((h->n_inst + 31) / 32) : 1024), st,
                     h->dp, h->n_inst, h->inst_off, h->inst_cap, h->grid, h->total_cells, h->status, gate, vinst));
  CKL(launch_chained(k_cell_count, dim3(capped_grid(h->nblk)), dim3(kBlock), st, h->dp.dim, s, h->blk_start,
                     h->blk_end, h->blk_inst, h->nblk, h->grid, h->cell_count, h->cell_of, h->rank, h->status, gate,
                     vinst, (const double*)h->vref, h->n));
  int tiles = capped_grid(grid_for(h->cell_cap, kScanTile));
  CKL(launch_chained(k_scan_reduce, dim3(tiles), dim3(kBlock), st, h->cell_count, h->total_cells, h->scan_sums, gate));
  CKL(launch_chained(k_scan_sums, dim3(1), dim3(1024), st, h->scan_sums, h->total_cells, gate));
  CKL(launch_chained(k_scan_down, dim3(tiles), dim3(kBlock), st, h->cell_count, h->total_cells, h->scan_sums, h->cell_start, h->n, gate));
  CKL(launch_chained(k_cell_scatter, dim3(capped_grid(grid_for(h->n, kBlock))), dim3(kBlock), st, h->n, h->cell_of,
                     h->rank, h->cell_start, h->perm, gate, vinst, h->inst_off, h->n_inst));
  CKL(launch_chained(k_cell_sort, dim3(capped_grid(grid_for(h->cell_cap * 32, kBlock))), dim3(kBlock), st,
                     h->total_cells, h->cell_start, h->perm, gate, h->grid, h->n_inst, h->dp.dim, h->n, h->slot_org,
                     vinst));
  h->launches += 8;
  // a mesh built outside the Verlet sequence changes the slot order under the lists
  if (!gate && h->verlet) return cudaMemsetAsync(&h->vflag[1], 0xff, sizeof(int), st);
  return cudaGetLastError();
}

// Verlet lists: vflag[0] = lists invalid (vflag[1]) or the validity criterion
// of k_kick_drift failed for some particle of any instance.
// Also sets, per instance (no pair joins two instances), the frame
// displacement U of the next step's criterion: the midpoint of this step's
// displacement box, which covers k steps since the build, extrapolated to
// k + 1 steps; after a build, one step's worth of it (the new reference is
// this step's state); 0 while the reference is void.  Any U keeps the
// criterion sound; a good one only makes builds rarer.
__global__ void k_verlet_flag(int* vflag, double* vframe, VAcc* vacc, int n_inst, int* vinst, int together) {
  chain_entry();
  // each instance whose criterion failed is rebuilt (its mesh, slots and lists;
  // the other instances keep theirs), or all of them when the lists are void or
  // the instances share an evaluation order (together)
  int fail = 0;
  for (int b = threadIdx.x; b < n_inst; b += blockDim.x) fail |= vacc[b].viol > 0 ? 1 : 0;
  const bool void_ref = vflag[1] != 0;
  const bool any = __syncthreads_or(fail) != 0 || void_ref;
  if (threadIdx.x == 0) vflag[0] = any ? 1 : 0;
  for (int b = threadIdx.x; b < n_inst; b += blockDim.x) {
    const bool rebuild = void_ref || (together ? any : vacc[b].viol > 0);
    vinst[b] = rebuild ? 1 : 0;
    VAcc& va = vacc[b];
    int bx[6];
#pragma unroll
    for (int a = 0; a < 3; ++a) { bx[a] = va.dlo[a]; bx[3 + a] = va.dhi[a]; }
    // reset for the next kick-drift
    va.viol = LLONG_MIN;
#pragma unroll
    for (int a = 0; a < 3; ++a) { va.dlo[a] = INT_MAX; va.dhi[a] = INT_MIN; }
    double* fr = vframe + 6 * b;
    const double ks = fr[3] >= 1.0 ? fr[3] : 1.0;   // steps covered by this step's displacements
    float* Uf = reinterpret_cast<float*>(fr + 4);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      // midpoint of the box of x - x^b, from that of x - x^b - U
      const double mid = bx[a] <= bx[3 + a] ? 0.5 * ((double)funkey(bx[a]) + (double)funkey(bx[3 + a])) + fr[a]
                                            : fr[a];
      fr[a] = void_ref ? 0.0 : (rebuild ? mid / ks : mid * (ks + 1.0) / ks);
      Uf[a] = (float)fr[a];
    }
    fr[3] = rebuild ? 1.0 : ks + 1.0;
  }
}

cudaError_t launch_verlet_flag(sph_handle* h, cudaStream_t st) {
  CKL(launch_chained(k_verlet_flag, dim3(1), dim3(h->n_inst < 1024 ? 32 * ((h->n_inst + 31) / 32) : 1024), st,
                     h->vflag, h->vframe, h->vacc, h->n_inst, h->vinst, h->unit_sched != SPH_SCHED_GLOBAL ? 1 : 0));
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_pack(sph_handle* h, const sph_state& s, bool predict, cudaStream_t st, bool eorder,
                        bool list_counters) {
  unsigned long long* lc = list_counters ? h->counters : nullptr;
  const int32_t* eoc = eorder ? h->e_of_c : nullptr;
  int32_t* pe = eorder ? h->perm_e : nullptr;
  void* Ac = eorder ? h->packAc : nullptr;
  if (h->dp.precision == SPH_PREC_MIXED)
    CKL(launch_chained(k_pack<true>, dim3(h->nblk), dim3(kBlock), st, h->dp, s, h->blk_start, h->blk_end, h->blk_inst, h->grid, h->dt,
                                             predict ? 1 : 0, h->perm, h->cell_of, h->packA, h->packB, h->packC,
                                             h->rho_slot, h->slot_cell, h->slot_unit, h->K, h->status, eoc, pe, Ac,
                                             h->vflag, lc));
  else
    CKL(launch_chained(k_pack<false>, dim3(h->nblk), dim3(kBlock), st, h->dp, s, h->blk_start, h->blk_end, h->blk_inst, h->grid, h->dt,
                                              predict ? 1 : 0, h->perm, h->cell_of, h->packA, h->packB, h->packC,
                                              h->rho_slot, h->slot_cell, h->slot_unit, h->K, h->status, eoc, pe, Ac,
                                              h->vflag, lc));
  h->launches += 1;
  return cudaGetLastError();
}


// k_pack's FP64 variant into the given operand arrays (the FP64 reverse pass
// of a mixed-precision handle).
cudaError_t launch_pack_fp64(sph_handle* h, const sph_state& s, bool predict, void* A, void* B, void* C,
                             double* rho_out, cudaStream_t st) {
  k_pack<false><<<h->nblk, kBlock, 0, st>>>(h->dp, s, h->blk_start, h->blk_end, h->blk_inst, h->grid, h->dt,
                                            predict ? 1 : 0, h->perm, h->cell_of, A, B, C, rho_out, h->slot_cell,
                                            h->slot_unit, h->K, h->status, nullptr, nullptr, nullptr, nullptr, nullptr);
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_kick2(sph_handle* h, const sph_state& s, double* t_dev, cudaStream_t st, bool next_dt) {
  BlockPart* part = next_dt ? h->part : nullptr;
  if (h->dp.precision == SPH_PREC_MIXED)
    CKL(launch_chained(k_kick2<true>, dim3(h->nblk), dim3(kBlock), st, h->dp, s, h->blk_start, h->blk_end, h->blk_inst, h->inst_blk, h->dt,
                                              t_dev, part));
  else
    CKL(launch_chained(k_kick2<false>, dim3(h->nblk), dim3(kBlock), st, h->dp, s, h->blk_start, h->blk_end, h->blk_inst, h->inst_blk, h->dt,
                                               t_dev, part));
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_renumber(sph_handle* h, sph_state& s, cudaStream_t st, const int32_t* order) {
  PermArrays a;
  a.count = 0;
  auto add = [&](void* ptr, int bytes) {
    if (ptr) { a.ptr[a.count] = ptr; a.bytes[a.count] = bytes; ++a.count; }
  };
  add(s.x, 8); add(s.y, 8); add(s.z, 8);
  add(s.vx, 8); add(s.vy, 8); add(s.vz, 8);
  add(s.rho, 8); add(s.E, 8); add(s.m, 8);
  add(s.ax, 8); add(s.ay, 8); add(s.az, 8); add(s.drho, 8); add(s.dE, 8);
  add(s.d, 8); add(s.P, 8); add(s.c, 8);
  add(s.id, 8);
  add(s.mat, 4); add(s.unit, 4);
  int g = grid_for(h->n, kBlock);
  k_gather<<<g, kBlock, 0, st>>>(h->n, order ? order : h->perm, a, reinterpret_cast<char*>(h->scratch));
  k_scatter_back<<<g, kBlock, 0, st>>>(h->n, a, reinterpret_cast<const char*>(h->scratch), nullptr);
  h->launches += 2;
  if (!h->verlet) return cudaGetLastError();
  // another order than the slot order (the unit-major evaluation order) moves
  // particles between slots under the Verlet lists: rebuild them
  if (order) return cudaMemsetAsync(&h->vflag[1], 0xff, sizeof(int), st);
  // In slot order the mesh, the slots and the lists stay as they are: particle
  // q is now the one in slot q, so the slot permutation becomes the identity,
  // and each particle's cell and the build-time positions and sizes of the
  // validity criterion follow their particles.
  PermArrays b;
  b.count = 0;
  for (int k = 0; k < 4; ++k)
    if (k < h->dp.dim || k == 3) {
      b.ptr[b.count] = h->vref + (size_t)k * h->n;
      b.bytes[b.count] = 8;
      ++b.count;
    }
  b.ptr[b.count] = h->cell_of;
  b.bytes[b.count] = 4;
  ++b.count;
  k_gather<<<g, kBlock, 0, st>>>(h->n, h->perm, b, reinterpret_cast<char*>(h->scratch));
  k_scatter_back<<<g, kBlock, 0, st>>>(h->n, b, reinterpret_cast<const char*>(h->scratch), h->perm);
  h->launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_exclusive_scan(int32_t* cnt, const int64_t* total, int32_t* sums, int32_t* start,
                                  int64_t n_total, int64_t cap, cudaStream_t st, const int* gate) {
  int tiles = capped_grid(grid_for(cap, kScanTile));
  k_scan_reduce<<<tiles, kBlock, 0, st>>>(cnt, total, sums, gate);
  k_scan_sums<<<1, 1024, 0, st>>>(sums, total, gate);
  k_scan_down<<<tiles, kBlock, 0, st>>>(cnt, total, sums, start, n_total, gate);
  return cudaGetLastError();
}
// (launch_exclusive_scan's three kernels are counted by its callers)

cudaError_t launch_conservation(sph_handle* h, const sph_state& s, double* out, cudaStream_t st) {
  k_conservation<<<h->n_inst, kBlock, 0, st>>>(s, h->inst_off, out);
  h->launches += 1;
  return cudaGetLastError();
}

// Largest particle volume m / rho (positive doubles order like their bit patterns).
__global__ void k_max_volume(int64_t n, const double* __restrict__ m, const double* __restrict__ rho,
                             unsigned long long* out) {
  unsigned long long b = 0ull;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const double v = m[p] / rho[p];
    if (v > 0.0 && v < 1e300) {
      const unsigned long long q = (unsigned long long)__double_as_longlong(v);
      b = q > b ? q : b;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long q = __shfl_xor_sync(0xffffffffu, b, o);
    b = q > b ? q : b;
  }
  if ((threadIdx.x & 31) == 0 && b) atomicMax(out, b);
}

cudaError_t launch_max_volume(sph_handle* h, const sph_state& s, unsigned long long* out, cudaStream_t st) {
  k_max_volume<<<capped_grid(grid_for(h->n, kBlock)), kBlock, 0, st>>>(h->n, s.m, s.rho, out);
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_check_finite(sph_handle* h, const sph_state& s, cudaStream_t st) {
  k_check_finite<<<grid_for(h->n, kBlock), kBlock, 0, st>>>(h->dp.dim, s, h->n, h->status);
  h->launches += 1;
  return cudaGetLastError();
}

}  // namespace csph
