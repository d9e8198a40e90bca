// csph_api.cu -- the C ABI of include/csph.h: argument checks, workspace
// ownership and the orchestration of the kernels of one CSPH step.
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "csph_internal.cuh"

using namespace csph;

namespace {

thread_local std::string g_init_error;

int fail(sph_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg; else g_init_error = msg;
  return code;
}

int cuda_fail(sph_handle* h, const char* what, cudaError_t e) {
  return fail(h, SPH_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                           \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail((h), #call, e_);  \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * count);
}

void free_all(sph_handle* h) {
  void* ptrs[] = {h->blk_inst, h->blk_start, h->blk_end, h->inst_blk, h->inst_off, h->part, h->grid, h->dt,
                  h->inst_cap, h->total_cells, h->cell_count, h->cell_start, h->scan_sums, h->cell_of, h->rank,
                  h->perm, h->slot_cell, h->slot_unit, h->packA, h->packB, h->packC, h->rho_slot, h->dmax_nbr,
                  h->load_acc, h->adj_bits, h->unit_off, h->unit_list, h->unit_work, h->unit_total, h->unit_stats,
                  h->status, h->counters, h->scratch, h->adj_G,
                  h->adj_GR, h->adj_pair, h->adj_par, h->adj_W, h->adj_store, h->mat_dev, h->vlist, h->vcnt,
                  h->vref, h->vflag, h->grad_p, h->grad_v, h->adj64_A, h->adj64_B, h->adj64_C,
                  h->adj64_rho, h->dt_key, h->e_of_c, h->perm_e, h->unit_eoff, h->packAc, h->unit_q, h->unit_t, h->slot_org, h->vinst};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

int check_state(sph_handle* h, const sph_state* s, int dim) {
  if (!s) return fail(h, SPH_ERR_INVALID, "state is NULL");
  if (!s->x || !s->vx || !s->rho || !s->E || !s->m || !s->ax || !s->drho || !s->dE || !s->d || !s->P || !s->c)
    return fail(h, SPH_ERR_INVALID, "state: a required array is NULL");
  if (dim >= 2 && (!s->y || !s->vy || !s->ay)) return fail(h, SPH_ERR_INVALID, "state: y/vy/ay NULL for dim >= 2");
  if (dim >= 3 && (!s->z || !s->vz || !s->az)) return fail(h, SPH_ERR_INVALID, "state: z/vz/az NULL for dim 3");
  return SPH_OK;
}

int check_handle_state(sph_handle* h, const sph_state* s) {
  if (!h) return SPH_ERR_INVALID;
  int rc = check_state(h, s, h->dp.dim);
  if (rc) return rc;
  if (s->n != h->n) return fail(h, SPH_ERR_INVALID, "state size differs from the handle's");
  if (h->K > 0 && !s->unit) return fail(h, SPH_ERR_INVALID, "state: unit array NULL with work units enabled");
  return SPH_OK;
}

// adjoint states carry x, v, rho, E and the rate fields only
int check_adjoint_state(sph_handle* h, const sph_state* a) {
  const int dim = h->dp.dim;
  if (!a || !a->x || !a->vx || !a->rho || !a->E || !a->ax || !a->drho || !a->dE)
    return fail(h, SPH_ERR_INVALID, "adjoint state: x, vx, rho, E, ax, drho, dE are required");
  if (dim >= 2 && (!a->y || !a->vy || !a->ay)) return fail(h, SPH_ERR_INVALID, "adjoint state: y/vy/ay for dim >= 2");
  if (dim >= 3 && (!a->z || !a->vz || !a->az)) return fail(h, SPH_ERR_INVALID, "adjoint state: z/vz/az for dim 3");
  return SPH_OK;
}

int eval_rates_impl(sph_handle* h, sph_state* s, cudaStream_t st) {
  CK(h, launch_derive_dt(h, *s, true, st));
  CK(h, launch_build_grid(h, *s, st));
  CK(h, launch_pack(h, *s, false, st));
  CK(h, launch_pair(h, *s, st));
  h->rates_valid = true;
  return SPH_OK;
}

int balance_impl(sph_handle* h, sph_state* s, double* gen, int K, int dim, const double* load,
                 const sph_balance_params& bp, double* shift_out, cudaStream_t st) {
  CK(h, launch_balance(h, *s, gen, K, dim, load, bp, shift_out, st));
  return SPH_OK;
}

int assign_impl(sph_handle* h, const sph_state* s, const double* gen, int K, int dim, int32_t* unit_out,
                int32_t* unit_offsets, cudaStream_t st) {
  CK(h, launch_assign(h, *s, gen, K, dim, unit_out, st));
  CK(h, launch_unit_lists(h, unit_out, unit_offsets, st));
  CK(h, cudaMemsetAsync(h->load_acc, 0, sizeof(unsigned long long) * K, st));
  CK(h, cudaMemsetAsync(h->adj_bits, 0, sizeof(uint32_t) * K * ((K + 31) / 32), st));
  return SPH_OK;
}

}  // namespace

void csph::set_global_error(const std::string& msg) { g_init_error = msg; }

extern "C" {

int sph_init(sph_handle** out, const sph_params* p, int n_instances, const int64_t* inst_offsets,
             const sph_state* s, void* stream) {
  if (!out) return fail(nullptr, SPH_ERR_INVALID, "handle pointer is NULL");
  *out = nullptr;
  if (!p) return fail(nullptr, SPH_ERR_INVALID, "params is NULL");
  if (p->dim < 1 || p->dim > 3) return fail(nullptr, SPH_ERR_INVALID, "dim must be 1, 2 or 3");
  if (p->kernel != SPH_KERNEL_CUBIC && p->kernel != SPH_KERNEL_WENDLAND_C2)
    return fail(nullptr, SPH_ERR_INVALID, "unknown kernel");
  if (p->precision != SPH_PREC_FP64 && p->precision != SPH_PREC_MIXED)
    return fail(nullptr, SPH_ERR_INVALID, "unknown precision");
  if (p->order < 0 || p->order > 2) return fail(nullptr, SPH_ERR_INVALID, "order must be 1 or 2");
  if (p->order == 2 && p->cell_beta > 0.0)
    return fail(nullptr, SPH_ERR_INVALID, "order 2 runs with the per-step neighbour search (cell_beta = 0)");
  if (p->solver != SPH_SOLVER_ACOUSTIC && p->solver != SPH_SOLVER_HLL)
    return fail(nullptr, SPH_ERR_INVALID, "unknown pair solver");
  if (p->load_measure != SPH_LOAD_PAIRS && p->load_measure != SPH_LOAD_TIME)
    return fail(nullptr, SPH_ERR_INVALID, "unknown load measure");
  if (p->list_staging != 0 && p->list_staging != 1) return fail(nullptr, SPH_ERR_INVALID, "list_staging must be 0 or 1");
  if (p->unit_sched < SPH_SCHED_GLOBAL || p->unit_sched > SPH_SCHED_UNITS_OWNED)
    return fail(nullptr, SPH_ERR_INVALID, "unknown unit_sched");
  if (p->list_cap != 0 && (p->list_cap < 32 || p->list_cap > 65536))
    return fail(nullptr, SPH_ERR_INVALID, "list_cap must be 0 (default) or in [32, 65536]");
  if (p->n_mat < 1 || p->n_mat > kMaxMaterials || (p->n_mat > SPH_MAX_MAT && !p->materials))
    return fail(nullptr, SPH_ERR_INVALID, "n_mat out of range (more than SPH_MAX_MAT need params.materials)");
  const sph_material* mats = p->materials ? p->materials : p->mat;
  for (int k = 0; k < p->n_mat; ++k) {
    if (mats[k].eos < SPH_EOS_IDEAL || mats[k].eos > SPH_EOS_STIFFENED_C0)
      return fail(nullptr, SPH_ERR_INVALID, "unknown EOS");
    if (mats[k].eos == SPH_EOS_STIFFENED_C0 && !(mats[k].rho0 > 0 && mats[k].c0 > 0 && mats[k].gamma > 0))
      return fail(nullptr, SPH_ERR_INVALID, "SPH_EOS_STIFFENED_C0 needs rho0, c0, gamma > 0");
  }
  if (!(p->kappa > 0) || !(p->eta > 0) || !(p->cfl > 0) || !(p->cell_beta >= 0))
    return fail(nullptr, SPH_ERR_INVALID, "kappa, eta, cfl must be > 0 and cell_beta >= 0");
  if (n_instances < 1 || !inst_offsets) return fail(nullptr, SPH_ERR_INVALID, "need n_instances >= 1 and offsets");
  int rc = check_state(nullptr, s, p->dim);
  if (rc) return rc;
  if (s->n < 1) return fail(nullptr, SPH_ERR_INVALID, "no particles");
  // pair-list entries hold a slot index in 26 bits
  if (s->n >= (int64_t(1) << 26)) return fail(nullptr, SPH_ERR_CAPACITY, "at most 2^26 - 1 particles per handle");
  if (inst_offsets[0] != 0 || inst_offsets[n_instances] != s->n)
    return fail(nullptr, SPH_ERR_INVALID, "instance offsets must start at 0 and end at n");
  for (int b = 0; b < n_instances; ++b)
    if (inst_offsets[b + 1] <= inst_offsets[b]) return fail(nullptr, SPH_ERR_INVALID, "empty or unordered instance");
  if (p->cell_cap < n_instances || p->cell_cap > (int64_t(1) << 31) - 2)
    return fail(nullptr, SPH_ERR_INVALID, "cell_cap must be in [n_instances, 2^31 - 2]");
  if (p->n_units < 0 || p->n_units > SPH_MAX_UNITS) return fail(nullptr, SPH_ERR_INVALID, "n_units out of range");
  if (p->n_units > 0) {
    if (n_instances != 1) return fail(nullptr, SPH_ERR_INVALID, "work units need a single instance");
    if (p->unit_dim < 1 || p->unit_dim > p->dim) return fail(nullptr, SPH_ERR_INVALID, "unit_dim out of range");
    if (!s->unit) return fail(nullptr, SPH_ERR_INVALID, "work units need state.unit");
    if (p->n_upd > 0 && !p->generators) return fail(nullptr, SPH_ERR_INVALID, "n_upd > 0 needs generators");
  }

  sph_handle* h = new sph_handle();
  h->p = *p;
  h->n = s->n;
  h->n_inst = n_instances;
  h->inst_off_h.assign(inst_offsets, inst_offsets + n_instances + 1);
  h->last_stream = (cudaStream_t)stream;
  DevParams& dp = h->dp;
  dp.dim = p->dim; dp.kernel = p->kernel; dp.precision = p->precision; dp.n_mat = p->n_mat;
  dp.kappa = p->kappa; dp.eta = p->eta; dp.cfl = p->cfl; dp.cell_beta = p->cell_beta;
  dp.kh = (0.5 * p->kappa) * p->eta;
  dp.eta_f = (float)dp.eta;
  dp.kh_f = (float)dp.kh;
  dp.cell_beta_f = (float)dp.cell_beta;
  dp.vscale_f = 1.0f;
  dp.slot_org = nullptr;
  dp.n = s->n;
  dp.vref = nullptr;
  dp.vframe = nullptr;
  dp.vacc = nullptr;
  dp.vscale = 1.0;
  for (int k = 0; k < p->n_mat; ++k) {
    const sph_material& m = mats[k];
    h->mat_h.push_back(make_mat(m.eos, m.gamma, m.rho0, m.c0, m.p_inf, m.s_a));
  }
  h->p.materials = nullptr;   // the caller's host array is not kept
  cudaStream_t st = (cudaStream_t)stream;
  auto bail = [&](int code) {
    g_init_error = h->err;
    free_all(h);
    delete h;
    return code;
  };
#define CKI(call)                                                         \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) { cuda_fail(h, #call, e_); return bail(SPH_ERR_CUDA); } \
  } while (0)

  CKI(dalloc(&h->mat_dev, h->mat_h.size()));
  CKI(cudaMemcpy(h->mat_dev, h->mat_h.data(), sizeof(Mat) * h->mat_h.size(), cudaMemcpyHostToDevice));
  dp.mat = h->mat_dev;

  // segmented blocks
  std::vector<int32_t> bi;
  std::vector<int64_t> bs, be;
  h->inst_blk_h.clear();
  for (int b = 0; b < n_instances; ++b) {
    h->inst_blk_h.push_back((int32_t)bi.size());
    for (int64_t q = inst_offsets[b]; q < inst_offsets[b + 1]; q += kBlock) {
      bi.push_back(b);
      bs.push_back(q);
      be.push_back(std::min(q + kBlock, inst_offsets[b + 1]));
    }
  }
  h->inst_blk_h.push_back((int32_t)bi.size());
  h->nblk = (int)bi.size();
  const int64_t n = h->n;
  CKI(dalloc(&h->blk_inst, h->nblk));
  CKI(dalloc(&h->blk_start, h->nblk));
  CKI(dalloc(&h->blk_end, h->nblk));
  CKI(dalloc(&h->inst_blk, n_instances + 1));
  CKI(dalloc(&h->inst_off, n_instances + 1));
  CKI(cudaMemcpy(h->blk_inst, bi.data(), sizeof(int32_t) * bi.size(), cudaMemcpyHostToDevice));
  CKI(cudaMemcpy(h->blk_start, bs.data(), sizeof(int64_t) * bs.size(), cudaMemcpyHostToDevice));
  CKI(cudaMemcpy(h->blk_end, be.data(), sizeof(int64_t) * be.size(), cudaMemcpyHostToDevice));
  CKI(cudaMemcpy(h->inst_blk, h->inst_blk_h.data(), sizeof(int32_t) * (n_instances + 1), cudaMemcpyHostToDevice));
  CKI(cudaMemcpy(h->inst_off, inst_offsets, sizeof(int64_t) * (n_instances + 1), cudaMemcpyHostToDevice));

  CKI(dalloc(&h->part, h->nblk));
  CKI(dalloc(&h->grid, n_instances));
  CKI(dalloc(&h->dt, n_instances));
  CKI(dalloc(&h->inst_cap, n_instances));
  CKI(dalloc(&h->total_cells, 1));
  std::vector<int64_t> caps(n_instances);
  for (int b = 0; b < n_instances; ++b) {
    int64_t nb = inst_offsets[b + 1] - inst_offsets[b];
    // share of the cell capacity: 1 + floor((cap - n_inst) n_b / n); the shares sum to <= cap
    // and a single instance gets the whole capacity
    caps[b] = n_instances == 1 ? p->cell_cap
                               : 1 + (int64_t)((double)(p->cell_cap - n_instances) * (double)nb / (double)n);
  }
  CKI(cudaMemcpy(h->inst_cap, caps.data(), sizeof(int64_t) * n_instances, cudaMemcpyHostToDevice));

  h->cell_cap = p->cell_cap;
  CKI(dalloc(&h->cell_count, h->cell_cap));
  CKI(cudaMemset(h->cell_count, 0, sizeof(int32_t) * h->cell_cap));
  CKI(dalloc(&h->cell_start, h->cell_cap + 1));
  CKI(dalloc(&h->scan_sums, h->cell_cap / 1024 + 2));
  CKI(dalloc(&h->cell_of, n));
  CKI(dalloc(&h->rank, n));
  CKI(dalloc(&h->perm, n));
  CKI(dalloc(&h->slot_cell, n));
  CKI(dalloc(&h->slot_unit, n));
  if (p->precision == SPH_PREC_MIXED) {
    CKI(dalloc(&h->slot_org, (size_t)3 * n));
    CKI(cudaMemset(h->slot_org, 0, sizeof(double) * 3 * n));
    h->dp.slot_org = h->slot_org;
    CKI(dalloc(reinterpret_cast<float4**>(&h->packA), n));
    CKI(dalloc(reinterpret_cast<float4**>(&h->packB), n));
    CKI(dalloc(reinterpret_cast<float4**>(&h->packC), n));
  } else {
    CKI(dalloc(reinterpret_cast<D4**>(&h->packA), n));
    CKI(dalloc(reinterpret_cast<D4**>(&h->packB), n));
    CKI(dalloc(reinterpret_cast<D2**>(&h->packC), n));
  }
  CKI(dalloc(&h->rho_slot, n));
  CKI(dalloc(&h->dmax_nbr, n));
  CKI(dalloc(&h->dt_key, (size_t)n_instances));
  {
    std::vector<long long> inf((size_t)n_instances, LLONG_MAX);
    CKI(cudaMemcpy(h->dt_key, inf.data(), sizeof(long long) * inf.size(), cudaMemcpyHostToDevice));
  }
  CKI(dalloc(&h->status, 1));
  CKI(cudaMemset(h->status, 0, sizeof(int)));
  CKI(dalloc(&h->counters, 8));
  CKI(cudaMemset(h->counters, 0, 8 * sizeof(unsigned long long)));
  h->scratch_bytes = (size_t)n * (18 * 8 + 8 + 4 + 4);
  CKI(cudaMalloc(&h->scratch, h->scratch_bytes));

  h->K = p->n_units;
  h->gdim = p->unit_dim;
  if (h->K > 0) {
    int K = h->K;
    int nb = grid_for(n, 1024);
    h->unit_work_total = (int64_t)K * nb;
    CKI(dalloc(&h->load_acc, K));
    CKI(cudaMemset(h->load_acc, 0, sizeof(unsigned long long) * K));
    CKI(dalloc(&h->adj_bits, (size_t)K * ((K + 31) / 32)));
    CKI(cudaMemset(h->adj_bits, 0, sizeof(uint32_t) * K * ((K + 31) / 32)));
    CKI(dalloc(&h->unit_off, K + 1));
    CKI(dalloc(&h->unit_list, n));
    CKI(dalloc(&h->unit_work, 2 * h->unit_work_total + h->unit_work_total / 1024 + 4));
    CKI(cudaMemset(h->unit_work, 0, sizeof(int32_t) * (2 * h->unit_work_total + h->unit_work_total / 1024 + 4)));
    CKI(dalloc(&h->unit_total, 1));
    CKI(cudaMemcpy(h->unit_total, &h->unit_work_total, sizeof(int64_t), cudaMemcpyHostToDevice));
    // 5 statistics + 4 balancing scratch per unit, then the statistics' partial sums
    // (up to 16 blocks per unit, 4 values each)
    CKI(dalloc(&h->unit_stats, (size_t)K * (9 + 16 * 4)));
  }

  // order-2 reconstruction: SPH gradients of P and v in slot order
  h->order2 = p->order == 2;
  h->solver = p->solver;
  h->load_timed = p->load_measure == SPH_LOAD_TIME;
  if (h->order2) {
    if (p->precision == SPH_PREC_MIXED) {
      CKI(dalloc(reinterpret_cast<float4**>(&h->grad_p), n));
      CKI(dalloc(reinterpret_cast<float4**>(&h->grad_v), (size_t)3 * n));
    } else {
      CKI(dalloc(reinterpret_cast<D4**>(&h->grad_p), n));
      CKI(dalloc(reinterpret_cast<D4**>(&h->grad_v), (size_t)3 * n));
    }
  }

  // Verlet lists (cell_beta > 0): capacity per particle from the neighbours of a uniform
  // lattice within (1 + beta) kappa eta spacings, with a margin for non-uniform spacing
  h->verlet = p->cell_beta > 0.0;
  if (h->verlet) {
    if (n >= (int64_t(1) << 27)) {
      fail(h, SPH_ERR_INVALID, "Verlet lists (cell_beta > 0) hold at most 2^27 - 1 particles");
      return bail(SPH_ERR_INVALID);
    }
    const double rr = p->kappa * p->eta * (1.0 + p->cell_beta);
    const double pi = 3.14159265358979323846;
    const double vol = p->dim == 1 ? 2.0 * rr : (p->dim == 2 ? pi * rr * rr : 4.0 / 3.0 * pi * rr * rr * rr);
    const double cap = p->list_cap > 0 ? (double)p->list_cap : std::ceil((p->dim == 3 ? 2.0 : 3.0) * vol + 32.0);
    h->vcap = (int)std::min(65536.0, std::ceil(cap / 32.0) * 32.0);
    CKI(dalloc(&h->vlist, (size_t)h->vcap * n));
    CKI(dalloc(&h->vcnt, n));
    const size_t ni = (size_t)n_instances;
    CKI(dalloc(&h->vref, (size_t)4 * n + 10 * ni));
    CKI(cudaMemset(h->vref, 0, sizeof(double) * (4 * n + 10 * ni)));
    // per instance: U = 0 (also its FP32 copy), one step since the build; empty accumulators
    h->vframe = h->vref + (size_t)4 * n;
    h->vacc = reinterpret_cast<VAcc*>(h->vframe + 6 * ni);
    std::vector<double> frame0(6 * ni, 0.0);
    for (size_t b = 0; b < ni; ++b) frame0[6 * b + 3] = 1.0;
    CKI(cudaMemcpy(h->vframe, frame0.data(), sizeof(double) * frame0.size(), cudaMemcpyHostToDevice));
    const VAcc acc0{LLONG_MIN, {INT_MAX, INT_MAX, INT_MAX}, {INT_MIN, INT_MIN, INT_MIN}};
    std::vector<VAcc> accs(ni, acc0);
    CKI(cudaMemcpy(h->vacc, accs.data(), sizeof(VAcc) * ni, cudaMemcpyHostToDevice));
    CKI(dalloc(&h->vflag, 4));
    CKI(dalloc(&h->vinst, ni));
    {
      std::vector<int> ones(ni, 1);
      CKI(cudaMemcpy(h->vinst, ones.data(), sizeof(int) * ni, cudaMemcpyHostToDevice));
    }
    const int flags[4] = {1, 1, 0, 0};    // lists invalid until the first build
    CKI(cudaMemcpy(h->vflag, flags, sizeof(flags), cudaMemcpyHostToDevice));
    dp.vref = h->vref;
    dp.vframe = h->vframe;
    dp.vacc = h->vacc;
    // the units as the list kernel's work partition
    h->unit_sched = h->K > 0 ? p->unit_sched : SPH_SCHED_GLOBAL;
    if (h->unit_sched != SPH_SCHED_GLOBAL) {
      CKI(dalloc(&h->e_of_c, n));
      CKI(dalloc(&h->perm_e, n));
      CKI(dalloc(&h->unit_eoff, h->K + 1));
      CKI(cudaMemset(h->unit_eoff, 0, sizeof(int32_t) * (h->K + 1)));
      if (p->precision == SPH_PREC_MIXED) CKI(dalloc(reinterpret_cast<float4**>(&h->packAc), n));
      else CKI(dalloc(reinterpret_cast<D4**>(&h->packAc), n));
      CKI(dalloc(&h->unit_q, h->K));
      CKI(dalloc(&h->unit_t, (size_t)2 * h->K));
      CKI(cudaMemset(h->unit_t, 0, sizeof(unsigned long long) * 2 * h->K));
    }
  }

  CKI(launch_check_finite(h, *s, st));
  int status = 0;
  CKI(cudaStreamSynchronize(st));
  CKI(cudaMemcpy(&status, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (status != 0) {
    fail(h, SPH_ERR_NONFINITE, "state holds a non-finite or non-positive value");
    return bail(SPH_ERR_NONFINITE);
  }
  if (p->precision == SPH_PREC_MIXED && n > 0) {
    // Scales of the FP32 pair arithmetic (powers of two, so they change no
    // rounding): the packed volume V vscale is ~1 for the largest particle and
    // W' wscale ~1 for its smoothing length, which keeps 2 V_i V_j P* W' in the
    // normal FP32 range at any length scale (at 0.1 um spacing V_i V_j ~ 1e-42
    // is below it).  The FP64 rate formation divides them out.
    unsigned long long* mx = reinterpret_cast<unsigned long long*>(h->counters + 6);
    CKI(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), st));
    CKI(launch_max_volume(h, *s, mx, st));
    unsigned long long bits = 0;
    CKI(cudaMemcpyAsync(&bits, mx, sizeof(bits), cudaMemcpyDeviceToHost, st));
    CKI(cudaStreamSynchronize(st));
    double vmax = 0.0;
    std::memcpy(&vmax, &bits, sizeof(vmax));
    if (vmax > 0.0) {
      int ev = 0;
      std::frexp(vmax, &ev);                               // vmax in [2^(ev-1), 2^ev)
      h->vscale = std::ldexp(1.0, -ev);
      const double href = p->eta * std::pow(vmax, 1.0 / p->dim);
      const int eh = (int)std::lround((p->dim + 1) * std::log2(href));
      h->wscale = std::ldexp(1.0, eh);
      dp.vscale = h->vscale;
    }
  } else {
    dp.vscale = 1.0;
  }
  dp.vscale_f = (float)dp.vscale;
#undef CKI
  *out = h;
  return SPH_OK;
}

int sph_build_cells(sph_handle* h, sph_state* s, void* stream) {
  int rc = check_handle_state(h, s);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  CK(h, launch_derive_dt(h, *s, true, st));
  CK(h, launch_build_grid(h, *s, st));
  CK(h, launch_renumber(h, *s, st));
  return SPH_OK;
}

int sph_eval_rates(sph_handle* h, sph_state* s, void* stream) {
  int rc = check_handle_state(h, s);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  return eval_rates_impl(h, s, st);
}

int sph_step(sph_handle* h, sph_state* s, int n_steps, double* t_dev, void* stream) {
  int rc = check_handle_state(h, s);
  if (rc) return rc;
  if (n_steps < 0) return fail(h, SPH_ERR_INVALID, "n_steps < 0");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  if (!h->rates_valid) {
    rc = eval_rates_impl(h, s, st);
    if (rc) return rc;
  }
  const bool vd3 = h->K > 0 && h->p.n_upd > 0;
  sph_balance_params bp{h->p.theta, h->p.sigma, h->p.gamma_b, h->p.beta_sh};
  bool dt_from_key = false;   // the previous step's fused second kick left the CFL keys
  for (int k = 0; k < n_steps; ++k) {
    // the CFL minima of the step's start state: from the previous step's second
    // kick inside this call (renumbering permutes an instance's particles and
    // leaves its minimum unchanged), else a k_derive pass
    if (k == 0) CK(h, launch_derive_dt(h, *s, false, st));
    CK(h, launch_reduce_dt(h, st, dt_from_key));
    CK(h, launch_kick_drift(h, *s, st));
    if (h->verlet) {
      // Verlet lists: the mesh, slot order and lists are rebuilt only when the device flag
      // says so (validity criterion failed or lists invalidated); the kernels read the flag
      CK(h, launch_verlet_flag(h, st));
      CK(h, launch_build_grid(h, *s, st, h->vflag));
      // unit-major evaluation order of the slots (at builds only)
      if (h->unit_sched != SPH_SCHED_GLOBAL) CK(h, launch_eorder(h, *s, st));
    } else {
      CK(h, launch_build_grid(h, *s, st));
    }
    CK(h, launch_pack(h, *s, true, st, h->verlet && h->unit_sched != SPH_SCHED_GLOBAL, h->verlet));
    // unit adjacency is needed only from the evaluation that precedes a rebalance
    h->collect_adj = !vd3 || h->steps_since_balance + 1 >= h->p.n_upd;
    const bool next_dt = k + 1 < n_steps;
    if (h->verlet) {
      // the second half kick, the time and the next CFL bound are fused into the
      // list kernel's rate write
      CK(h, launch_list_build(h, *s, st));
      CK(h, launch_pair_lists(h, *s, st, true, t_dev, next_dt));
      dt_from_key = next_dt;
    } else {
      CK(h, launch_pair(h, *s, st));
      CK(h, launch_kick2(h, *s, t_dev, st, next_dt));
      dt_from_key = false;
    }
    h->collect_adj = true;
    if (vd3 && ++h->steps_since_balance >= h->p.n_upd) {
      // Alg. 1 outer loop: shift generators, reassign, renumber
      h->steps_since_balance = 0;
      rc = balance_impl(h, s, h->p.generators, h->K, h->gdim, nullptr, bp, nullptr, st);
      if (rc) return rc;
      rc = assign_impl(h, s, h->p.generators, h->K, h->gdim, s->unit, nullptr, st);
      if (rc) return rc;
      if (h->verlet && h->unit_sched != SPH_SCHED_GLOBAL) {
        // renumber unit-major (cell order inside a unit), the evaluation order
        // of the new units, so that the list kernel walks the state in order
        CK(h, launch_eorder(h, *s, st, true));
        CK(h, launch_renumber(h, *s, st, h->perm_e));
      } else {
        CK(h, launch_renumber(h, *s, st));
      }
    }
  }
  return SPH_OK;
}

int sph_step_dt(sph_handle* h, sph_state* s, int n_steps, const double* dt_dev, double* t_dev, void* stream) {
  int rc = check_handle_state(h, s);
  if (rc) return rc;
  if (n_steps < 0 || (n_steps > 0 && !dt_dev)) return fail(h, SPH_ERR_INVALID, "need n_steps >= 0 and dt_dev");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  if (!h->rates_valid) {
    rc = eval_rates_impl(h, s, st);
    if (rc) return rc;
  }
  for (int k = 0; k < n_steps; ++k) {
    CK(h, cudaMemcpyAsync(h->dt, dt_dev + (size_t)k * h->n_inst, sizeof(double) * h->n_inst,
                          cudaMemcpyDeviceToDevice, st));
    CK(h, launch_kick_drift(h, *s, st));
    CK(h, launch_build_grid(h, *s, st));
    CK(h, launch_pack(h, *s, true, st));
    CK(h, launch_pair(h, *s, st));
    CK(h, launch_kick2(h, *s, t_dev, st));
  }
  return SPH_OK;
}

int voronoi_assign(sph_handle* h, const sph_state* s, const double* gen, int K, int dim, int32_t* unit_out,
                   int32_t* unit_offsets, void* stream) {
  int rc = check_handle_state(h, s);
  if (rc) return rc;
  if (h->K == 0 || K != h->K) return fail(h, SPH_ERR_INVALID, "K must equal the handle's n_units (> 0)");
  if (dim != h->gdim) return fail(h, SPH_ERR_INVALID, "dim must equal the handle's unit_dim");
  if (!gen || !unit_out) return fail(h, SPH_ERR_INVALID, "gen and unit_out are required");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  return assign_impl(h, s, gen, K, dim, unit_out, unit_offsets, st);
}

int voronoi_balance(sph_handle* h, const sph_state* s, double* gen, int K, int dim, const double* load,
                    const sph_balance_params* bp, double* shift_sum_out, void* stream) {
  int rc = check_handle_state(h, s);
  if (rc) return rc;
  if (h->K == 0 || K != h->K) return fail(h, SPH_ERR_INVALID, "K must equal the handle's n_units (> 0)");
  if (dim != h->gdim) return fail(h, SPH_ERR_INVALID, "dim must equal the handle's unit_dim");
  if (!gen || !bp) return fail(h, SPH_ERR_INVALID, "gen and balance params are required");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  return balance_impl(h, const_cast<sph_state*>(s), gen, K, dim, load, *bp, shift_sum_out, st);
}

int voronoi_balance_stats(sph_handle* h, double* gen, int K, int dim, const double* load, const uint8_t* adj,
                          const double* rmax, const double* centroid, const int64_t* count,
                          const sph_balance_params* bp, double* shift_sum_out, void* stream) {
  if (!h) return SPH_ERR_INVALID;
  if (h->K == 0 || K != h->K) return fail(h, SPH_ERR_INVALID, "K must equal the handle's n_units (> 0)");
  if (dim != h->gdim) return fail(h, SPH_ERR_INVALID, "dim must equal the handle's unit_dim");
  if (!gen || !load || !adj || !rmax || !centroid || !count || !bp)
    return fail(h, SPH_ERR_INVALID, "gen, load, adj, rmax, centroid, count and bp are required");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  // statistics in the layout of the handle's own: [K x 5] centroid (3), count, rmax; then the loads
  std::vector<double> stats((size_t)6 * K, 0.0);
  for (int k = 0; k < K; ++k) {
    for (int a = 0; a < dim; ++a) stats[(size_t)k * 5 + a] = centroid[(size_t)k * dim + a];
    stats[(size_t)k * 5 + 3] = (double)count[k];
    stats[(size_t)k * 5 + 4] = rmax[k];
    stats[(size_t)5 * K + k] = load[k];
  }
  const int words = (K + 31) / 32;
  std::vector<uint32_t> bits((size_t)K * words, 0u);
  for (int k = 0; k < K; ++k)
    for (int l = 0; l < K; ++l)
      if (adj[(size_t)k * K + l]) bits[(size_t)k * words + (l >> 5)] |= 1u << (l & 31);
  // the statistics' partial-sum area of unit_stats (free outside voronoi_balance) holds the copies
  double* dst = h->unit_stats + (size_t)9 * K;
  CK(h, cudaMemcpyAsync(dst, stats.data(), sizeof(double) * stats.size(), cudaMemcpyHostToDevice, st));
  CK(h, cudaMemcpyAsync(h->adj_bits, bits.data(), sizeof(uint32_t) * bits.size(), cudaMemcpyHostToDevice, st));
  CK(h, launch_balance_given(h, gen, K, dim, dst, dst + (size_t)5 * K, *bp, shift_sum_out, st));
  CK(h, cudaStreamSynchronize(st));     // the host copies above are stack-owned
  return SPH_OK;
}

int sph_hold_rates(sph_handle* h) {
  if (!h) return SPH_ERR_INVALID;
  h->rates_valid = true;
  return SPH_OK;
}

int sph_cfl_dt(sph_handle* h, const sph_state* s, double* dt_out, void* stream) {
  int rc = check_handle_state(h, s);
  if (rc) return rc;
  if (!dt_out) return fail(h, SPH_ERR_INVALID, "dt_out is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  CK(h, launch_derive_dt(h, *s, false, st));
  CK(h, launch_reduce_dt(h, st, false));
  CK(h, cudaMemcpyAsync(dt_out, h->dt, sizeof(double) * h->n_inst, cudaMemcpyDeviceToDevice, st));
  return SPH_OK;
}

int sph_conservation(sph_handle* h, const sph_state* s, double* out, void* stream) {
  int rc = check_handle_state(h, s);
  if (rc) return rc;
  if (!out) return fail(h, SPH_ERR_INVALID, "out is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  CK(h, launch_conservation(h, *s, out, st));
  return SPH_OK;
}

int sph_unit_stats(sph_handle* h, double* load_out, uint8_t* adj_out, void* stream) {
  if (!h) return SPH_ERR_INVALID;
  if (h->K == 0) return fail(h, SPH_ERR_INVALID, "work units are disabled");
  cudaStream_t st = (cudaStream_t)stream;
  int K = h->K, words = (K + 31) / 32;
  std::vector<unsigned long long> acc(K);
  std::vector<uint32_t> bits((size_t)K * words);
  CK(h, cudaMemcpyAsync(acc.data(), h->load_acc, sizeof(unsigned long long) * K, cudaMemcpyDeviceToHost, st));
  CK(h, cudaMemcpyAsync(bits.data(), h->adj_bits, sizeof(uint32_t) * bits.size(), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  for (int k = 0; k < K; ++k) {
    if (load_out) load_out[k] = 0.5 * (double)acc[k];
    if (adj_out)
      for (int l = 0; l < K; ++l) adj_out[k * K + l] = (bits[(size_t)k * words + (l >> 5)] >> (l & 31)) & 1u;
  }
  return SPH_OK;
}

int sph_unit_times(sph_handle* h, double* out, void* stream) {
  if (!h) return SPH_ERR_INVALID;
  if (h->unit_sched == SPH_SCHED_GLOBAL || !h->unit_t)
    return fail(h, SPH_ERR_INVALID, "the list kernel is not partitioned by units (unit_sched, cell_beta, n_units)");
  if (!out) return fail(h, SPH_ERR_INVALID, "out is NULL");
  std::vector<unsigned long long> t((size_t)2 * h->K);
  cudaStream_t st = (cudaStream_t)stream;
  CK(h, cudaMemcpyAsync(t.data(), h->unit_t, sizeof(unsigned long long) * t.size(), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  const int K = h->K;                    // starts in t[0, K), ends in t[K, 2K)
  unsigned long long t0 = ~0ull;
  for (int k = 0; k < K; ++k)
    if (t[K + k] > 0 && t[k] < t0) t0 = t[k];
  for (int k = 0; k < K; ++k) {
    const bool used = t[K + k] > 0;
    out[2 * k] = used ? (double)(t[k] - t0) : 0.0;
    out[2 * k + 1] = used ? (double)(t[K + k] - t0) : 0.0;
  }
  return SPH_OK;
}

int sph_read_status(sph_handle* h, int* device_status) {
  if (!h || !device_status) return SPH_ERR_INVALID;
  CK(h, cudaStreamSynchronize(h->last_stream));
  CK(h, cudaMemcpy(device_status, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  CK(h, cudaMemset(h->status, 0, sizeof(int)));
  return SPH_OK;
}

const char* sph_last_error(const sph_handle* h) { return h ? h->err.c_str() : g_init_error.c_str(); }

int sph_pair_counts(sph_handle* h, int64_t* half_pairs, int64_t* candidates, int64_t* fp64_checks, void* stream) {
  if (!h) return SPH_ERR_INVALID;
  unsigned long long c[4];
  cudaStream_t st = (cudaStream_t)stream;
  CK(h, cudaMemcpyAsync(c, h->counters, sizeof(c), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  if (half_pairs) *half_pairs = (int64_t)(c[0] / 2);
  if (candidates) *candidates = (int64_t)c[1];
  if (fp64_checks) *fp64_checks = (int64_t)c[2];
  return SPH_OK;
}

int sph_list_builds(sph_handle* h, int64_t* builds, int32_t* capacity, void* stream) {
  if (!h) return SPH_ERR_INVALID;
  if (!h->verlet) return fail(h, SPH_ERR_INVALID, "the handle keeps no Verlet lists (cell_beta = 0)");
  int f[4];
  cudaStream_t st = (cudaStream_t)stream;
  CK(h, cudaMemcpyAsync(f, h->vflag, sizeof(f), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  if (builds) *builds = f[2];
  if (capacity) *capacity = h->vcap;
  return SPH_OK;
}

int sph_cell_index(sph_handle* h, const sph_state* s, int32_t* cell_out, double* grid_out, void* stream) {
  int rc = check_handle_state(h, s);
  if (rc) return rc;
  if (!cell_out) return fail(h, SPH_ERR_INVALID, "cell_out is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  sph_state tmp = *s;
  CK(h, launch_derive_dt(h, tmp, true, st));
  CK(h, launch_build_grid(h, tmp, st));
  std::vector<GridInfo> g(h->n_inst);
  CK(h, cudaMemcpyAsync(g.data(), h->grid, sizeof(GridInfo) * h->n_inst, cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  std::vector<int32_t> cells(h->n);
  CK(h, cudaMemcpy(cells.data(), h->cell_of, sizeof(int32_t) * h->n, cudaMemcpyDeviceToHost));
  for (int b = 0; b < h->n_inst; ++b) {
    for (int64_t q = h->inst_off_h[b]; q < h->inst_off_h[b + 1]; ++q) cells[q] -= (int32_t)g[b].cell_off;
    if (grid_out) {
      double* o = grid_out + 8 * b;
      for (int a = 0; a < 3; ++a) o[a] = g[b].x0[a];
      o[3] = g[b].dc;
      for (int a = 0; a < 3; ++a) o[4 + a] = (double)g[b].dims[a];
      o[7] = (double)g[b].ncells;
    }
  }
  CK(h, cudaMemcpy(cell_out, cells.data(), sizeof(int32_t) * h->n, cudaMemcpyHostToDevice));
  return SPH_OK;
}

int sph_pair_list(sph_handle* h, sph_state* s, int64_t cap, int32_t* pi_out, int32_t* pj_out, int64_t* count_out,
                  void* stream) {
  int rc = check_handle_state(h, s);
  if (rc) return rc;
  if (!pi_out || !pj_out || !count_out || cap < 0) return fail(h, SPH_ERR_INVALID, "bad pair output arguments");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  h->pair_out_i = pi_out;
  h->pair_out_j = pj_out;
  h->pair_out_cap = cap;
  rc = eval_rates_impl(h, s, st);
  h->pair_out_i = h->pair_out_j = nullptr;
  h->pair_out_cap = 0;
  if (rc) return rc;
  unsigned long long c = 0;
  CK(h, cudaMemcpyAsync(&c, &h->counters[4], sizeof(c), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  *count_out = (int64_t)c;
  if ((int64_t)c > cap) return fail(h, SPH_ERR_CAPACITY, "more pairs than cap");
  return SPH_OK;
}

int sph_last_dt(sph_handle* h, double* dt_out, void* stream) {
  if (!h || !dt_out) return SPH_ERR_INVALID;
  CK(h, cudaMemcpyAsync(dt_out, h->dt, sizeof(double) * h->n_inst, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return SPH_OK;
}

namespace {

// 13 state arrays stored per replayed step; the working state W adds d, P, c
constexpr int kAdjStored = 13;
constexpr int kAdjW = 16;

sph_state adj_work_state(sph_handle* h, const sph_state& ck) {
  const int64_t n = h->n;
  double* w = h->adj_W;
  sph_state W{};
  W.n = n;
  double** f[kAdjW] = {&W.x, &W.y, &W.z, &W.vx, &W.vy, &W.vz, &W.rho, &W.E, &W.ax, &W.ay, &W.az, &W.drho, &W.dE,
                       &W.d, &W.P, &W.c};
  for (int k = 0; k < kAdjW; ++k) *f[k] = w + (size_t)k * n;
  if (h->dp.dim < 2) { W.y = W.vy = W.ay = nullptr; }
  if (h->dp.dim < 3) { W.z = W.vz = W.az = nullptr; }
  W.m = ck.m;
  W.mat = ck.mat;
  W.id = nullptr;
  W.unit = nullptr;
  return W;
}

// copy the 13 dynamic arrays (x, v, rho, E, rates) between two states
cudaError_t copy_dynamic(const sph_state& dst, const sph_state& src, int64_t n, cudaStream_t st) {
  double* d[kAdjStored] = {dst.x, dst.y, dst.z, dst.vx, dst.vy, dst.vz, dst.rho, dst.E, dst.ax, dst.ay, dst.az,
                           dst.drho, dst.dE};
  const double* s[kAdjStored] = {src.x, src.y, src.z, src.vx, src.vy, src.vz, src.rho, src.E, src.ax, src.ay,
                                 src.az, src.drho, src.dE};
  for (int k = 0; k < kAdjStored; ++k) {
    if (!d[k] || !s[k]) continue;
    cudaError_t e = cudaMemcpyAsync(d[k], s[k], sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

sph_state stored_state(sph_handle* h, int step, const sph_state& like) {
  const int64_t n = h->n;
  double* base = h->adj_store + (size_t)step * kAdjStored * n;
  sph_state S = like;
  double** f[kAdjStored] = {&S.x, &S.y, &S.z, &S.vx, &S.vy, &S.vz, &S.rho, &S.E, &S.ax, &S.ay, &S.az, &S.drho,
                            &S.dE};
  for (int k = 0; k < kAdjStored; ++k) *f[k] = base + (size_t)k * n;
  if (h->dp.dim < 2) { S.y = S.vy = S.ay = nullptr; }
  if (h->dp.dim < 3) { S.z = S.vz = S.az = nullptr; }
  return S;
}

}  // namespace

int sph_step_adjoint(sph_handle* h, const sph_ckpt* ck, int n_steps, const sph_state* adj_out, sph_state* adj_in,
                     double* adj_params, void* stream) {
  if (!h || !ck || !adj_out || !adj_in || !adj_params) return h ? fail(h, SPH_ERR_INVALID, "NULL argument") : SPH_ERR_INVALID;
  if (n_steps < 0 || (n_steps > 0 && !ck->dt)) return fail(h, SPH_ERR_INVALID, "need n_steps >= 0 and the dt record");
  if (h->n_inst != 1) return fail(h, SPH_ERR_INVALID, "the adjoint supports a single instance");
  if (h->order2) return fail(h, SPH_ERR_INVALID, "the adjoint covers the first-order scheme (order 1)");
  if (h->solver != SPH_SOLVER_ACOUSTIC) return fail(h, SPH_ERR_INVALID, "the adjoint covers the acoustic pair solver");
  if (h->dp.kernel != SPH_KERNEL_CUBIC) return fail(h, SPH_ERR_INVALID, "the adjoint supports the cubic spline");
  for (int k = 0; k < h->dp.n_mat; ++k)
    if (h->mat_h[k].eos != SPH_EOS_IDEAL && h->mat_h[k].eos != SPH_EOS_STIFFENED)
      return fail(h, SPH_ERR_INVALID, "the adjoint supports ideal and stiffened gas");
  int rc = check_handle_state(h, &ck->state);
  if (rc) return rc;
  rc = check_adjoint_state(h, adj_out);
  if (rc) return rc;
  rc = check_adjoint_state(h, adj_in);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  const int64_t n = h->n;
  if (!h->adj_G) {
    CK(h, dalloc(&h->adj_G, n));
    CK(h, dalloc(&h->adj_GR, n));
    CK(h, dalloc(&h->adj_pair, (size_t)11 * n));
    CK(h, dalloc(&h->adj_par, (size_t)2 * n));
    CK(h, dalloc(&h->adj_W, (size_t)kAdjW * n));
    CK(h, cudaMemsetAsync(h->adj_W, 0, sizeof(double) * kAdjW * n, st));
  }
  // FP64 pair derivatives on a mixed-precision handle (the forward replay stays mixed)
  const bool rev64 = h->dp.precision == SPH_PREC_MIXED && ck->reverse_fp64 != 0;
  if (rev64 && !h->adj64_A) {
    CK(h, dalloc(reinterpret_cast<D4**>(&h->adj64_A), n));
    CK(h, dalloc(reinterpret_cast<D4**>(&h->adj64_B), n));
    CK(h, dalloc(reinterpret_cast<D2**>(&h->adj64_C), n));
    CK(h, dalloc(&h->adj64_rho, n));
  }
  if (n_steps > h->adj_store_steps) {
    if (h->adj_store) CK(h, cudaFree(h->adj_store));
    h->adj_store = nullptr;
    CK(h, dalloc(&h->adj_store, (size_t)n_steps * kAdjStored * n));
    h->adj_store_steps = n_steps;
  }
  sph_state W = adj_work_state(h, ck->state);
  // forward replay from the checkpoint with the recorded dt, keeping every state
  CK(h, copy_dynamic(W, ck->state, n, st));
  for (int k = 0; k < n_steps; ++k) {
    CK(h, copy_dynamic(stored_state(h, k, W), W, n, st));
    CK(h, cudaMemcpyAsync(h->dt, ck->dt + k, sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(h, launch_kick_drift(h, W, st));
    CK(h, launch_build_grid(h, W, st));
    CK(h, launch_pack(h, W, true, st));
    CK(h, launch_pair(h, W, st));
    CK(h, launch_kick2(h, W, nullptr, st));
  }
  // adjoint, in place in adj_in
  if (adj_in != adj_out) CK(h, copy_dynamic(*adj_in, *adj_out, n, st));
  for (int k = n_steps - 1; k >= 0; --k) {
    CK(h, copy_dynamic(W, stored_state(h, k, W), n, st));
    CK(h, cudaMemcpyAsync(h->dt, ck->dt + k, sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(h, launch_kick_drift(h, W, st));
    CK(h, launch_build_grid(h, W, st));
    if (rev64) {
      CK(h, launch_pack_fp64(h, W, true, h->adj64_A, h->adj64_B, h->adj64_C, h->adj64_rho, st));
      CK(h, launch_rates_vjp(h, W, *adj_in, ck->dt + k, 1, adj_params, st, true));
    } else {
      CK(h, launch_pack(h, W, true, st));
      CK(h, launch_rates_vjp(h, W, *adj_in, ck->dt + k, 1, adj_params, st));
    }
  }
  if (ck->rates_from_state) {
    // the held rates at the checkpoint were evaluated at its own state
    CK(h, copy_dynamic(W, ck->state, n, st));
    CK(h, launch_derive_dt(h, W, true, st));
    CK(h, launch_build_grid(h, W, st));
    if (rev64) {
      CK(h, launch_pack_fp64(h, W, false, h->adj64_A, h->adj64_B, h->adj64_C, h->adj64_rho, st));
      CK(h, launch_rates_vjp(h, W, *adj_in, h->dt, 0, adj_params, st, true));
    } else {
      CK(h, launch_pack(h, W, false, st));
      CK(h, launch_rates_vjp(h, W, *adj_in, h->dt, 0, adj_params, st));
    }
  }
  return SPH_OK;
}

int sph_profile(sph_handle* h, int enable) {
  if (!h) return SPH_ERR_INVALID;
  h->profiling = enable != 0;
  h->prof_used = 0;
  h->launches = 0;
  return SPH_OK;
}

int sph_profile_read(sph_handle* h, double* pair_ms, int64_t* pair_launches, int64_t* kernel_launches) {
  if (!h) return SPH_ERR_INVALID;
  CK(h, cudaStreamSynchronize(h->last_stream));
  double tot = 0.0;
  for (size_t k = 0; k + 1 < h->prof_used; k += 2) {
    float ms = 0.f;
    CK(h, cudaEventElapsedTime(&ms, h->prof_events[k], h->prof_events[k + 1]));
    tot += ms;
  }
  if (pair_ms) *pair_ms = tot;
  if (pair_launches) *pair_launches = (int64_t)(h->prof_used / 2);
  if (kernel_launches) *kernel_launches = h->launches;
  h->prof_used = 0;
  h->launches = 0;
  return SPH_OK;
}

void sph_destroy(sph_handle* h) {
  if (!h) return;
  for (cudaEvent_t ev : h->prof_events) cudaEventDestroy(ev);
  free_all(h);
  delete h;
}

}  // extern "C"
