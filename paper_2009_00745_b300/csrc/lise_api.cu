// lise_api.cu -- host side of the C ABI declared in include/lise.h.
//
// A context owns the ABM history on the device:
//   y_n, y_{n-1}             two state slots (swapped every step), complex128
//   y'_n .. y'_{n-3}         a ring of four derivative slots, compute precision
//   m_{n+1}, p_n - c_n       modifier (Eq. m) and the difference it uses, compute precision
//   Q (complex128), R        the corrector's precombined history (lise_kernels.cuh)
//   T_xy scratch             the in-plane kinetic part of the current operand
// (the compute precision is FP64, or FP32 in the mixed path; values kept in it are
// formed in it, so they are stored without rounding)
// plus per-group density partial sums, reduced densities and the potentials
// W = U(n) - mu + V_ext and Delta of the operand of the next right-hand side.
//
// One ABM step (Eqs. p, m, c, y) is 6 launches (7 in the mixed path, see abm_step):
//   planes(m), pencils[CORRECT]        m' = -iHm; y_{n+1} = Q + k1 m', p - c; densities of y_{n+1}
//   reduce                             W, Delta of y_{n+1} at t_{n+1}
//   planes(y_{n+1}), pencils[DERIV_PREDICT]
//                                      y'_{n+1}; m_{n+2}, Q, R; densities of m_{n+2}
//   reduce                             W, Delta of m_{n+2} at t_{n+2}
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/lise.h"
#include "lise_internal.h"
#include "lise_kernels.cuh"

using namespace lise;

namespace lise {

int check_params(const lise_params* p) {
  if (!p) return LISE_EINVAL;
  if (p->nx != p->ny || p->ny != p->nz) return LISE_EINVAL;
  if (!supported_n(p->nx)) return LISE_EINVAL;
  if (!(p->dx > 0.0) || !std::isfinite(p->dx) || p->n_qp < 1) return LISE_EINVAL;
  if (p->precision != LISE_FP64 && p->precision != LISE_MIXED && p->precision != LISE_MIXED_STRICT)
    return LISE_EINVAL;
  if (!std::isfinite(p->alpha) || !std::isfinite(p->beta) || !std::isfinite(p->mu) ||
      !std::isfinite(p->g) || !std::isfinite(p->drive_A) || !std::isfinite(p->drive_Omega))
    return LISE_EINVAL;
  if (p->pair_lattice && !(p->alpha > 0.0)) return LISE_EINVAL;
  if (p->pair_alpha != 0.0 && !(std::isfinite(p->pair_alpha) && p->pair_n0 > 0.0 && std::isfinite(p->pair_n0)))
    return LISE_EINVAL;
  // Eq. geff: E_c > 0, at most the one-axis natural cutoff pi^2 / (2 m* a^2) of the lattice, and
  // not together with the lattice form of Eq. geff_3D
  if (!(p->pair_ec >= 0.0) || !std::isfinite(p->pair_ec)) return LISE_EINVAL;
  if (p->pair_ec > 0.0) {
    const double PI = 3.14159265358979323846;
    if (p->pair_lattice || !(p->alpha > 0.0) || p->pair_ec > p->alpha * PI * PI / (2.0 * p->dx * p->dx))
      return LISE_EINVAL;
  }
  return LISE_OK;
}

Pairing make_pairing(const lise_params* p) {
  Pairing r;
  r.g = p->g;
  r.alpha_n0 = p->pair_alpha != 0.0 ? p->pair_alpha / p->pair_n0 : 0.0;
  r.c = p->pair_lattice ? pairing_lattice_c(p->dx, p->alpha) : 0.0;
  r.ec = p->pair_ec;
  r.m = p->pair_ec > 0.0 ? 1.0 / p->alpha : 0.0;
  r.mu = p->mu;
  r.beta = p->beta;
  return r;
}

}  // namespace lise

struct lise_ctx {
  lise_params p;
  int N = 0;
  long nxyz = 0;
  long ns = 0;  // complex elements per state array
  int mixed = 0;   // FP32 compute precision (LISE_MIXED and LISE_MIXED_STRICT)
  int strict = 0;  // LISE_MIXED_STRICT: R and p - c in complex128, FP64 history arithmetic
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int qg = 0, n_groups = 0;
  double2* slot[2] = {nullptr, nullptr};
  int y0_slot = 0;                 // slot holding y_n
  void* D[4] = {nullptr, nullptr, nullptr, nullptr};  // D[k] = y'_{n-k}, compute precision
  void* M = nullptr;  // m_{n+1}, complex of the compute precision (only an H psi operand)
  double2* Q = nullptr;
  // R and p - c (compute precision) share one allocation, R first; during the start
  // procedure the block holds the complex128 predictor state instead
  void* RPC = nullptr;
  void *R = nullptr, *PC = nullptr;
  void* TXY = nullptr;
  // density partial sums [3][n_groups_all][N^3] (n, Re nu, Im nu) in one allocation; part_*
  // view this context's groups [first_group, first_group + n_groups) of each array
  double* parts = nullptr;
  double *part_n = nullptr, *part_nr = nullptr, *part_ni = nullptr;
  int n_groups_all = 0, first_group = 0;
  // sharded densities (lise_set_shard): the exchange that fills the other shards' groups
  lise_exchange_fn exch = nullptr;
  void* exch_user = nullptr;
  int exch_on_device = 0, exch_capturable = 0;
  double* host_parts = nullptr;  // pinned [3][n_groups_all][N^3] for a host-side exchange
  double* dn[2] = {nullptr, nullptr};
  double2* dnu[2] = {nullptr, nullptr};
  double* W = nullptr;
  double2* Dl = nullptr;
  double* v_static = nullptr;
  void *tw = nullptr, *hxy = nullptr, *hz = nullptr;
  uint32_t* ozb = nullptr;  // FP64 tensor-core kinetic operator: D2 digit fragments
  int oz_sD = 0;
  double* e_site = nullptr;
  int* err = nullptr;
  long wait_polls = 0;  // bounded device waits (PencilArgs::wait_polls): 0 = the default limit
  double t = 0.0, dt = 0.0;
  int ready = 0;
  int sticky = LISE_OK;
  double* host_e = nullptr;
  // trivial-phase removal: eta per state and its per-block partial sums
  double* eta = nullptr;
  double* eta_part = nullptr;
  int n_blocks_x = 0;
  // per-step renormalisation: norm partials [state][kNormBlocks] and the scale per state
  double* norm_part = nullptr;
  double* norm_scale = nullptr;
  // CUDA graphs of kGraphSteps ABM steps, one per history configuration (y-slot
  // parity x position of the derivative ring), replayed by lise_step
  cudaGraphExec_t graph[2][4] = {};
  double* drive_dev = nullptr;  // drive amplitudes of the reductions of one replay
  int drive_red = 0;  // reductions per captured ABM step (2); checked at capture
  int capturing = 0;            // > 0 while capturing: index of the next reduction
  void* D_base[4] = {nullptr, nullptr, nullptr, nullptr};  // the ring's allocations in ring order
  // per-launch timing (lise_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> rec_cls;  // class of record i uses events 2i, 2i+1
};

namespace {

constexpr int kNormBlocks = 32;  // blocks per state of the norm reduction (renormalisation)

struct Footprint {
  size_t state, txy, partials, small, total;
};

Footprint footprint(const lise_params* p) {
  Footprint f{};
  const long N = p->nx;
  const long nxyz = N * N * N;
  const long ns = (long)p->n_qp * 2 * nxyz;
  int qg, ng;
  choose_groups((int)N, p->n_qp, p->precision != LISE_FP64, &qg, &ng);
  // 2 y slots and Q in complex128; 4 y', m in the compute precision; R and P-C in the compute
  // precision (complex128 in the strict split)
  const bool mixed = p->precision != LISE_FP64;
  const size_t rc = mixed ? sizeof(float2) : sizeof(double2);
  const size_t rh = (p->precision == LISE_MIXED) ? sizeof(float2) : sizeof(double2);
  f.state = 3 * (size_t)ns * sizeof(double2) + 5 * (size_t)ns * rc + 2 * (size_t)ns * rh;
  f.txy = (size_t)ns * rc;
  f.partials = 3 * (size_t)ng * nxyz * sizeof(double);
  f.small = (size_t)nxyz * (2 * sizeof(double) + 2 * sizeof(double2) + sizeof(double) + sizeof(double2) +
                            sizeof(double) + 2 * sizeof(double)) +
            3 * (size_t)N * sizeof(double2) + 256;
  if (p->remove_phase) f.small += (size_t)p->n_qp * (1 + pencil_blocks_x((int)N, p->precision != LISE_FP64)) * sizeof(double);
  if (p->renormalize) f.small += (size_t)p->n_qp * (1 + kNormBlocks) * sizeof(double);
  f.total = f.state + f.txy + f.partials + f.small;
  return f;
}

// bytes per complex element of R and p - c: the compute precision, complex128 in the strict split
size_t hist_elem(const lise_ctx* c) { return (c->mixed && !c->strict) ? sizeof(float2) : sizeof(double2); }

double drive_at(const lise_ctx* c, double t) {
  return c->p.drive_A == 0.0 ? 0.0 : c->p.drive_A * std::sin(c->p.drive_Omega * t);
}

int cu(cudaError_t e) { return e == cudaSuccess ? LISE_OK : LISE_ECUDA; }

// Records a CUDA event pair around the launch made by f() when profiling is on.
template <typename F>
int timed(lise_ctx* c, int cls, F f) {
  if (!c->prof) return f();
  const size_t i = c->rec_cls.size();
  while (c->ev_pool.size() < 2 * (i + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return LISE_ECUDA;
    c->ev_pool.push_back(e);
  }
  if (cudaEventRecord(c->ev_pool[2 * i], c->stream) != cudaSuccess) return LISE_ECUDA;
  int rc = f();
  if (cudaEventRecord(c->ev_pool[2 * i + 1], c->stream) != cudaSuccess) return LISE_ECUDA;
  c->rec_cls.push_back(cls);
  return rc;
}

#define TRY(x)                  \
  do {                          \
    int rc__ = (x);             \
    if (rc__ != LISE_OK) {      \
      return rc__;              \
    }                           \
  } while (0)

PencilArgs pencil_base(const lise_ctx* c) {
  PencilArgs a;
  std::memset(&a, 0, sizeof(a));
  a.err = c->err;
  a.wait_polls = c->wait_polls;
  a.strict = c->strict;
  a.txy = c->TXY;
  a.W = c->W;
  a.D = c->Dl;
  a.tw = c->tw;
  a.hz = c->hz;
  a.ozb = c->ozb;
  a.oz_sD = c->oz_sD;
  a.n_qp = c->p.n_qp;
  a.qg = c->qg;
  a.part_n = c->part_n;
  a.part_nr = c->part_nr;
  a.part_ni = c->part_ni;
  a.eta = c->p.remove_phase ? c->eta : nullptr;
  return a;
}

PlanesArgs planes_args(const lise_ctx* c, const double2* x, const void* xr) {
  PlanesArgs a;
  a.x = x;
  a.xr = xr;
  a.txy = c->TXY;
  a.tw = c->tw;
  a.hxy = c->hxy;
  a.ozb = c->ozb;
  a.oz_sD = c->oz_sD;
  a.n_planes = (long)c->p.n_qp * 2 * c->N;
  a.err = c->err;
  a.wait_polls = c->wait_polls;
  return a;
}

int run_planes(lise_ctx* c, const double2* x, const void* xr = nullptr) {
  const PlanesArgs a = planes_args(c, x, xr);
  return timed(c, LISE_KC_PLANES, [&] { return launch_planes(c->N, c->mixed, a, c->stream) ? LISE_ECUDA : LISE_OK; });
}

int run_pencils(lise_ctx* c, int mode, const PencilArgs& a) {
  return timed(c, LISE_KC_PENCILS,
               [&] { return launch_pencils(c->N, c->mixed, mode, a, c->stream) ? LISE_ECUDA : LISE_OK; });
}

// eta_q = <x_q|H x_q> with the current potentials (T_xy x must be in the scratch);
// a no-op without trivial-phase removal.
int run_eta(lise_ctx* c, const double2* x, const void* xr = nullptr) {
  if (!c->p.remove_phase) return LISE_OK;
  PencilArgs a = pencil_base(c);
  a.eta = nullptr;
  a.x = x;
  a.xr = xr;
  a.eta_part = c->eta_part;
  TRY(run_pencils(c, M_ETA, a));
  const double a3 = c->p.dx * c->p.dx * c->p.dx;
  return timed(c, LISE_KC_REDUCE, [&] {
    return launch_eta_reduce(c->eta_part, c->p.n_qp, c->n_blocks_x, a3, c->eta, c->stream) ? LISE_ECUDA : LISE_OK;
  });
}

// The other shards' groups of the partial sums (a no-op for an unsharded context): a
// device exchange enqueues its work on the context stream; a host exchange gets this
// context's groups in a pinned host copy and fills in the others, which are copied back.
int exchange_parts(lise_ctx* c) {
  if (!c->exch) return LISE_OK;
  const size_t plane = (size_t)c->n_groups_all * c->nxyz;  // doubles per array
  if (c->exch_on_device)
    return c->exch(c->exch_user, c->parts, 1, (void*)c->stream, c->nxyz, c->first_group, c->n_groups, c->n_groups_all)
               ? LISE_EEXCHANGE
               : LISE_OK;
  const size_t off = (size_t)c->first_group * c->nxyz, cnt = (size_t)c->n_groups * c->nxyz;
  for (int k = 0; k < 3; ++k)
    TRY(cu(cudaMemcpyAsync(c->host_parts + k * plane + off, c->parts + k * plane + off, cnt * sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream)));
  TRY(cu(cudaStreamSynchronize(c->stream)));
  if (c->exch(c->exch_user, c->host_parts, 0, nullptr, c->nxyz, c->first_group, c->n_groups, c->n_groups_all))
    return LISE_EEXCHANGE;
  return cu(cudaMemcpyAsync(c->parts, c->host_parts, 3 * plane * sizeof(double), cudaMemcpyHostToDevice, c->stream));
}

// The reduction's arguments without the drive (drive = 0, no drive pointer): the partial
// sums of all shards' groups (or of this context's own with all_shards = false), densities
// into slot dslot, averaged with (avg_n, avg_nu) if given, potentials if requested.
ReduceArgs reduce_args(const lise_ctx* c, int dslot, const double* avg_n, const double2* avg_nu, bool potentials,
                       bool all_shards) {
  ReduceArgs r;
  if (all_shards) {
    const size_t plane = (size_t)c->n_groups_all * c->nxyz;
    r.part_n = c->parts;
    r.part_nr = c->parts + plane;
    r.part_ni = c->parts + 2 * plane;
    r.n_groups = c->n_groups_all;
  } else {
    r.part_n = c->part_n;
    r.part_nr = c->part_nr;
    r.part_ni = c->part_ni;
    r.n_groups = c->n_groups;
  }
  r.nxyz = c->nxyz;
  r.N = c->N;
  r.a = c->p.dx;
  r.n_out = c->dn[dslot];
  r.nu_out = c->dnu[dslot];
  r.avg_n = avg_n;
  r.avg_nu = avg_nu;
  r.W = potentials ? c->W : nullptr;
  r.D = potentials ? c->Dl : nullptr;
  r.v_static = c->v_static;
  r.drive = 0.0;
  r.drive_ptr = nullptr;
  r.beta = c->p.beta;
  r.mu = c->p.mu;
  r.pair = make_pairing(&c->p);
  r.err = c->err;
  return r;
}

// Reduce the density partials; optionally average with (avg_n, avg_nu); write
// the densities to slot `dslot` and, if potentials is true, W and Delta at t.
// all_shards = false reduces this context's own groups only (no exchange).
int run_reduce(lise_ctx* c, int dslot, const double* avg_n, const double2* avg_nu, bool potentials, double t,
               bool all_shards = true) {
  if (all_shards) TRY(exchange_parts(c));
  ReduceArgs r = reduce_args(c, dslot, avg_n, avg_nu, potentials, all_shards);
  r.drive = drive_at(c, t);
  if (c->capturing) {  // inside a graph: the amplitude is refreshed before every replay
    if (c->p.drive_A != 0.0) r.drive_ptr = c->drive_dev + (c->capturing - 1);
    ++c->capturing;
  }
  return timed(c, LISE_KC_REDUCE, [&] { return launch_reduce(r, c->stream) ? LISE_ECUDA : LISE_OK; });
}

int run_density(lise_ctx* c, const double2* src) {
  PointwiseArgs a;
  std::memset(&a, 0, sizeof(a));
  a.src = src;
  a.part_n = c->part_n;
  a.part_nr = c->part_nr;
  a.part_ni = c->part_ni;
  a.n_qp = c->p.n_qp;
  a.qg = c->qg;
  a.nxyz = c->nxyz;
  return timed(c, LISE_KC_POINTWISE, [&] { return launch_density(a, c->stream) ? LISE_ECUDA : LISE_OK; });
}

double2 cx(double re, double im) { return make_double2(re, im); }

// psi_out = sum_{j=0}^{4} (-i dt H)^j / j! psi_in with the current potentials
// (order-4 series of exp(-i H dt)).  If dslot != nullptr, also stores
// -i H psi_in there.  The last term's kernel accumulates the densities of
// psi_out into the partials.  The series term lives in the Q array, which the
// start procedure fills only at its end.
int taylor4(lise_ctx* c, const double2* psi_in, double2* psi_out, void* dslot, double dt) {
  TRY(run_planes(c, psi_in));
  TRY(run_eta(c, psi_in));  // eta of the starting state with this series' Hamiltonian
  PencilArgs a = pencil_base(c);
  a.x = psi_in;
  a.out = c->Q;
  a.acc = psi_out;
  a.dslot = dslot;
  a.coef = cx(0.0, -dt);
  TRY(run_pencils(c, M_TAYLOR_FIRST, a));
  for (int j = 2; j <= 4; ++j) {
    TRY(run_planes(c, c->Q));
    PencilArgs b = pencil_base(c);
    b.x = c->Q;
    b.out = c->Q;
    b.acc = psi_out;
    b.coef = cx(0.0, -dt / j);
    b.dens = (j == 4);
    TRY(run_pencils(c, M_TAYLOR, b));
  }
  return LISE_OK;
}

int fetch_err(lise_ctx* c) {
  if (c->sticky) return c->sticky;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    c->sticky = LISE_ECUDA;
    return c->sticky;
  }
  if (h) {
    c->sticky = (h & 4) ? LISE_ETIMEOUT : LISE_ENONFINITE;
    return c->sticky;
  }
  return LISE_OK;
}

PointwiseArgs predict_args(lise_ctx* c, const double2* y0, const double2* y1, const void* d0, const void* d1,
                           const void* d2, const void* d3, double h) {
  PointwiseArgs w;
  std::memset(&w, 0, sizeof(w));
  w.y0 = y0;
  w.y1 = y1;
  w.d0 = d0;
  w.d1 = d1;
  w.d2 = d2;
  w.d3 = d3;
  w.pc = c->PC;
  w.q = c->Q;
  w.r = c->R;
  w.m = c->M;
  w.mixed = c->mixed;
  w.strict = c->strict;
  w.h = h;
  w.part_n = c->part_n;
  w.part_nr = c->part_nr;
  w.part_ni = c->part_ni;
  w.n_qp = c->p.n_qp;
  w.qg = c->qg;
  w.nxyz = c->nxyz;
  return w;
}

// y_{n+1} (in the y_{n-1} slot) becomes y_n; y'_{n+1} (in D[3]) becomes D[0]
void rotate_history(lise_ctx* c, double t1) {
  c->y0_slot = 1 - c->y0_slot;
  void* d3 = c->D[3];
  c->D[3] = c->D[2];
  c->D[2] = c->D[1];
  c->D[1] = c->D[0];
  c->D[0] = d3;
  c->t = t1;
}

int start_procedure(lise_ctx* c, double t0, double dt) {
  // y_0 is in slot[0]; densities and potentials of y_0 at t0 into dn[0]
  double2* cur = c->slot[0];
  double2* nxt = c->slot[1];
  TRY(run_density(c, cur));
  TRY(run_reduce(c, 0, nullptr, nullptr, true, t0));
  for (int s = 0; s < 3; ++s) {
    const double ts = t0 + s * dt;
    // predictor with H(t_s): psi_pre into the R/P-C block (free until the end of the
    // start); y'_s = -i H(t_s) y_s into D[3 - s]
    TRY(taylor4(c, cur, static_cast<double2*>(c->RPC), c->D[3 - s], dt));
    // corrector densities (n_pre + n(t_s)) / 2, potentials at t_s + dt/2
    TRY(run_reduce(c, 1, c->dn[0], c->dnu[0], true, ts + 0.5 * dt));
    // psi(t_s + dt) = exp(-i H_cor dt) psi(t_s), densities into dn[0] at t_{s+1}
    TRY(taylor4(c, cur, nxt, nullptr, dt));
    TRY(run_reduce(c, 0, nullptr, nullptr, true, ts + dt));
    double2* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  // cur = y_3, nxt = y_2; y'_3 = f(t_3, y_3) into D[0]
  TRY(run_planes(c, cur));
  TRY(run_eta(c, cur));
  PencilArgs a = pencil_base(c);
  a.x = cur;
  a.out = nullptr;
  a.dslot = c->D[0];
  TRY(run_pencils(c, M_RHS, a));
  c->y0_slot = (cur == c->slot[0]) ? 0 : 1;
  // p_3 - c_3 := 0; predictor and modifier of the first ABM step
  TRY(cu(cudaMemsetAsync(c->PC, 0, (size_t)c->ns * hist_elem(c), c->stream)));
  PointwiseArgs w = predict_args(c, c->slot[c->y0_slot], c->slot[1 - c->y0_slot], c->D[0], c->D[1], c->D[2],
                                 c->D[3], dt);
  TRY(timed(c, LISE_KC_POINTWISE, [&] { return launch_predict(w, c->stream) ? LISE_ECUDA : LISE_OK; }));
  const double t3 = t0 + 3 * dt;
  TRY(run_reduce(c, 1, nullptr, nullptr, true, t3 + dt));
  c->t = t3;
  c->dt = dt;
  return LISE_OK;
}

int abm_step(lise_ctx* c) {
  const double h = c->dt;
  const double t1 = c->t + h;
  double2* yn = c->slot[c->y0_slot];
  double2* ynm1 = c->slot[1 - c->y0_slot];
  // RHS #1 on m_{n+1} (stored in the compute precision): Eq. c, Eq. y through Q, R;
  // y_{n+1} replaces y_{n-1}
  TRY(run_planes(c, nullptr, c->M));
  TRY(run_eta(c, nullptr, c->M));
  PencilArgs a = pencil_base(c);
  a.xr = c->M;
  a.h = h;
  a.q = c->Q;
  a.r = c->R;
  a.pc = c->PC;
  a.ynew = ynm1;
  a.dens = 1;
  TRY(run_pencils(c, M_CORRECT, a));
  if (c->p.renormalize) {
    // end of the step: each state of y_{n+1} to unit norm, and the densities of the scaled state
    const double a3 = c->p.dx * c->p.dx * c->p.dx;
    PointwiseArgs w;
    std::memset(&w, 0, sizeof(w));
    w.part_n = c->part_n;
    w.part_nr = c->part_nr;
    w.part_ni = c->part_ni;
    w.n_qp = c->p.n_qp;
    w.qg = c->qg;
    w.nxyz = c->nxyz;
    TRY(timed(c, LISE_KC_POINTWISE, [&] {
      return launch_norms(ynm1, c->p.n_qp, c->nxyz, a3, kNormBlocks, c->norm_part, c->norm_scale, c->stream) ||
                     launch_scale_density(ynm1, c->norm_scale, w, c->stream)
                 ? LISE_ECUDA
                 : LISE_OK;
    }));
  }
  TRY(run_reduce(c, 1, nullptr, nullptr, true, t1));
  // RHS #2 on y_{n+1}: y'_{n+1} into the y'_{n-3} slot, then Eq. p and Eq. m of step n+2
  TRY(run_planes(c, ynm1));
  TRY(run_eta(c, ynm1));
  if (c->mixed) {
    // memory-bound path: the pencils launch writes y'_{n+1} only; a streaming kernel then
    // forms m, Q, R and the densities of m from the history
    PencilArgs b = pencil_base(c);
    b.x = ynm1;
    b.out = nullptr;
    b.dslot = c->D[3];
    TRY(run_pencils(c, M_RHS, b));
    PointwiseArgs w = predict_args(c, ynm1, yn, c->D[3], c->D[0], c->D[1], c->D[2], h);
    TRY(timed(c, LISE_KC_POINTWISE, [&] { return launch_predict(w, c->stream) ? LISE_ECUDA : LISE_OK; }));
    TRY(run_reduce(c, 1, nullptr, nullptr, true, t1 + h));
    rotate_history(c, t1);
    return LISE_OK;
  }
  PencilArgs b = pencil_base(c);
  b.x = ynm1;
  b.h = h;
  b.y0 = yn;
  b.d0 = c->D[0];
  b.d1 = c->D[1];
  b.d2 = c->D[2];
  b.dslot = c->D[3];
  b.pc = c->PC;
  b.q = c->Q;
  b.r = c->R;
  b.m = c->M;
  b.dens = 1;
  TRY(run_pencils(c, M_DERIV_PREDICT, b));
  TRY(run_reduce(c, 1, nullptr, nullptr, true, t1 + h));
  rotate_history(c, t1);
  return LISE_OK;
}

constexpr int kGraphSteps = 4;  // the history configuration repeats every 4 steps

int ring_position(const lise_ctx* c) {
  for (int k = 0; k < 4; ++k)
    if (c->D[0] == c->D_base[k]) return k;
  return -1;
}

void drop_graphs(lise_ctx* c) {
  for (auto& row : c->graph)
    for (auto& g : row)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
}

// Capture kGraphSteps ABM steps from the current configuration into a graph.  The
// host-side history state (t, slot parity, ring) is restored afterwards; the
// caller launches the graph and then advances it.
int capture_graph(lise_ctx* c, cudaGraphExec_t* out) {
  const double t0 = c->t;
  const int slot0 = c->y0_slot;
  void* d0[4] = {c->D[0], c->D[1], c->D[2], c->D[3]};
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LISE_ECUDA;
  c->capturing = 1;
  int rc = LISE_OK;
  for (int k = 0; k < kGraphSteps && rc == LISE_OK; ++k) rc = abm_step(c);
  c->drive_red = c->capturing - 1;  // reductions captured (2 per ABM step)
  c->capturing = 0;
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  c->t = t0;
  c->y0_slot = slot0;
  for (int k = 0; k < 4; ++k) c->D[k] = d0[k];
  if (rc == LISE_OK && c->drive_red != 2 * kGraphSteps) rc = LISE_ECUDA;  // (the replay's drive table)
  if (rc != LISE_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess || !g) return LISE_ECUDA;
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e == cudaSuccess ? LISE_OK : LISE_ECUDA;
}

// kGraphSteps steps by one graph replay (capturing it on first use).
int graph_steps(lise_ctx* c) {
  const int rp = ring_position(c);
  if (rp < 0) return LISE_ECUDA;
  cudaGraphExec_t& g = c->graph[c->y0_slot][rp];
  if (!g) TRY(capture_graph(c, &g));
  if (c->p.drive_A != 0.0) {
    double amp[2 * kGraphSteps];
    // the times of a step's two reductions, t_{n+1} = t_n + dt and t_{n+1} + dt, accumulated
    // exactly as abm_step does, so that a replay is bitwise the plain launches
    double t = c->t;
    for (int j = 0; j < kGraphSteps; ++j) {
      const double t1 = t + c->dt;
      amp[2 * j] = drive_at(c, t1);
      amp[2 * j + 1] = drive_at(c, t1 + c->dt);
      t = t1;
    }
    TRY(cu(cudaMemcpyAsync(c->drive_dev, amp, sizeof(amp), cudaMemcpyHostToDevice, c->stream)));
  }
  TRY(cu(cudaGraphLaunch(g, c->stream)));
  for (int k = 0; k < kGraphSteps; ++k) rotate_history(c, c->t + c->dt);
  return LISE_OK;
}

void free_ctx(lise_ctx* c) {
  drop_graphs(c);
  void* ptrs[] = {c->norm_part, c->norm_scale, c->drive_dev, c->eta, c->eta_part, c->slot[0], c->slot[1], c->D[0], c->D[1], c->D[2], c->D[3], c->M, c->RPC, c->Q, c->TXY,
                  c->parts, c->dn[0], c->dn[1], c->dnu[0], c->dnu[1], c->W,
                  c->Dl, c->v_static, c->tw, c->hxy, c->hz, c->ozb, c->e_site, c->err};
  // stream-ordered frees: no device-wide synchronisation (work of other contexts,
  // e.g. the other requests of a server, keeps running)
  for (void* q : ptrs)
    if (q) cudaFreeAsync(q, c->stream);
  cudaStreamSynchronize(c->stream);
  if (c->host_parts) cudaFreeHost(c->host_parts);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  std::free(c->host_e);
}

}  // namespace

extern "C" {

size_t lise_footprint_bytes(const lise_params* p) {
  if (check_params(p) != LISE_OK) return 0;
  return footprint(p).total;
}

const char* lise_strerror(int s) {
  switch (s) {
    case LISE_OK: return "ok";
    case LISE_EINVAL: return "invalid argument";
    case LISE_ENOMEM: return "device memory budget exceeded or allocation failed";
    case LISE_ECUDA: return "CUDA error";
    case LISE_ENONFINITE: return "non-finite state or density";
    case LISE_ETIMEOUT: return "bounded device wait timed out";
    case LISE_ESTATE: return "call out of order (no state set)";
    case LISE_EEXCHANGE: return "the shard exchange callback failed";
    default: return "unknown status";
  }
}

int lise_create(const lise_params* p, lise_ctx** out) {
  if (!out) return LISE_EINVAL;
  *out = nullptr;
  TRY(check_params(p));
  Footprint f = footprint(p);
  if (p->hbm_budget_bytes && f.total > p->hbm_budget_bytes) return LISE_ENOMEM;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || p->device < 0 || p->device >= ndev) return LISE_EINVAL;
  if (cudaSetDevice(p->device) != cudaSuccess) return LISE_ECUDA;
  lise_ctx* c = new (std::nothrow) lise_ctx();
  if (!c) return LISE_ENOMEM;
  c->p = *p;
  c->p.v_static = nullptr;
  c->N = p->nx;
  c->nxyz = (long)c->N * c->N * c->N;
  c->ns = (long)p->n_qp * 2 * c->nxyz;
  c->mixed = p->precision != LISE_FP64;
  c->strict = p->precision == LISE_MIXED_STRICT;
  c->device = p->device;
  choose_groups(c->N, p->n_qp, c->mixed, &c->qg, &c->n_groups);
  int rc = LISE_OK;
  if (p->stream) {
    c->stream = (cudaStream_t)p->stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) rc = LISE_ECUDA;
    c->own_stream = true;
  }
  const size_t sb = (size_t)c->ns * sizeof(double2);
  // stream-ordered allocations from the device's default memory pool (cheap to
  // create and free while other contexts run; see free_ctx)
  auto alloc = [&](void** q, size_t bytes) {
    if (rc != LISE_OK) return;
    cudaError_t e = cudaMallocAsync(q, bytes, c->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      rc = (e == cudaErrorMemoryAllocation) ? LISE_ENOMEM : LISE_ECUDA;
    }
  };
  alloc((void**)&c->slot[0], sb);
  alloc((void**)&c->slot[1], sb);
  const size_t sr = (size_t)c->ns * (c->mixed ? sizeof(float2) : sizeof(double2));  // compute-precision array
  for (int k = 0; k < 4; ++k) alloc(&c->D[k], sr);
  for (int k = 0; k < 4; ++k) c->D_base[k] = c->D[k];
  alloc((void**)&c->drive_dev, 2 * kGraphSteps * sizeof(double));
  alloc(&c->M, sr);
  alloc((void**)&c->Q, sb);
  const size_t sh = (size_t)c->ns * hist_elem(c);  // R or P-C
  alloc(&c->RPC, 2 * sh);  // R, P-C; at least one complex128 state (start procedure)
  if (c->RPC) {
    c->R = c->RPC;
    c->PC = static_cast<char*>(c->RPC) + sh;
  }
  alloc(&c->TXY, (size_t)c->ns * (c->mixed ? sizeof(float2) : sizeof(double2)));
  c->n_groups_all = c->n_groups;
  alloc((void**)&c->parts, 3 * (size_t)c->n_groups * c->nxyz * sizeof(double));
  if (c->parts) {
    c->part_n = c->parts;
    c->part_nr = c->parts + (size_t)c->n_groups * c->nxyz;
    c->part_ni = c->parts + 2 * (size_t)c->n_groups * c->nxyz;
  }
  for (int k = 0; k < 2; ++k) {
    alloc((void**)&c->dn[k], c->nxyz * sizeof(double));
    alloc((void**)&c->dnu[k], c->nxyz * sizeof(double2));
  }
  alloc((void**)&c->W, c->nxyz * sizeof(double));
  alloc((void**)&c->Dl, c->nxyz * sizeof(double2));
  if (p->v_static) alloc((void**)&c->v_static, c->nxyz * sizeof(double));
  const size_t rs = c->mixed ? sizeof(float) : sizeof(double);
  alloc(&c->tw, 2 * c->N * rs);
  alloc(&c->hxy, c->N * rs);
  alloc(&c->hz, c->N * rs);
  alloc((void**)&c->e_site, 2 * c->nxyz * sizeof(double));
  std::vector<uint32_t> ozt;
  if (ozaki_path(c->N, c->mixed)) {
    ozt.resize(ozaki_table_words(c->N));
    c->oz_sD = ozaki_table(c->N, p->dx, p->alpha, ozt.data());
    alloc((void**)&c->ozb, ozt.size() * sizeof(uint32_t));
  }
  c->n_blocks_x = pencil_blocks_x(c->N, c->mixed);
  if (p->renormalize) {
    alloc((void**)&c->norm_part, (size_t)p->n_qp * kNormBlocks * sizeof(double));
    alloc((void**)&c->norm_scale, (size_t)p->n_qp * sizeof(double));
  }
  if (p->remove_phase) {
    alloc((void**)&c->eta, (size_t)p->n_qp * sizeof(double));
    alloc((void**)&c->eta_part, (size_t)p->n_qp * c->n_blocks_x * sizeof(double));
  }
  alloc((void**)&c->err, sizeof(int));
  c->host_e = (double*)std::malloc(2 * c->nxyz * sizeof(double));
  if (rc == LISE_OK && !c->host_e) rc = LISE_ENOMEM;
  if (rc == LISE_OK) {
    // tables
    std::vector<char> tw(2 * c->N * rs), hxy(c->N * rs), hz(c->N * rs);
    fill_fft_tables(c->N, p->dx, p->alpha, c->mixed, tw.data(), hxy.data(), hz.data());
    rc = cu(cudaMemcpyAsync(c->tw, tw.data(), tw.size(), cudaMemcpyHostToDevice, c->stream));
    if (rc == LISE_OK) rc = cu(cudaMemcpyAsync(c->hxy, hxy.data(), hxy.size(), cudaMemcpyHostToDevice, c->stream));
    if (rc == LISE_OK) rc = cu(cudaMemcpyAsync(c->hz, hz.data(), hz.size(), cudaMemcpyHostToDevice, c->stream));
    if (rc == LISE_OK && c->ozb)
      rc = cu(cudaMemcpyAsync(c->ozb, ozt.data(), ozt.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream));
    if (rc == LISE_OK && p->v_static)
      rc = cu(cudaMemcpyAsync(c->v_static, p->v_static, c->nxyz * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (rc == LISE_OK) rc = cu(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    if (rc == LISE_OK) rc = cu(cudaStreamSynchronize(c->stream));
  }
  if (rc != LISE_OK) {
    free_ctx(c);
    delete c;
    return rc;
  }
  *out = c;
  return LISE_OK;
}

// Pencil batch autotuning (once per process for each lattice size and precision): time the
// two pencils launches of an ABM step for every compiled batch size on this context's
// buffers, before the series start overwrites them, and keep the fastest.  Needs the
// input state in slot 0; uses the other arrays as scratch.  Results do not depend on it.
static std::mutex g_tune_mu;

// Planes per block of the FFT planes kernel (lattices that do not use the tensor-core
// planes kernels), tuned like the pencils batch size: every compiled candidate timed on
// this context's operand (3 launches after a warm-up), the fastest kept.
static int tune_planes(lise_ctx* c) {
  if (ozaki_path(c->N, c->mixed) || planes_pb_get(c->N, c->mixed)) return LISE_OK;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (planes_pb_get(c->N, c->mixed)) return LISE_OK;
  int cands[8], n_valid = 0;
  for (int pb : {1, 2, 4, 8, -1, -2, -4, -8})
    if (planes_pb_valid(c->N, c->mixed, pb)) cands[n_valid++] = pb;
  if (n_valid < 2) {
    if (n_valid == 1) planes_pb_set(c->N, c->mixed, cands[0]);
    return LISE_OK;
  }
  const PlanesArgs a = planes_args(c, c->slot[0], nullptr);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return LISE_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return LISE_ECUDA;
  }
  int best = 0, rc = LISE_OK;
  float best_ms = 0.f;
  for (int ci = 0; ci < n_valid && rc == LISE_OK; ++ci) {
    const int pb = cands[ci];
    if (launch_planes(c->N, c->mixed, a, c->stream, pb)) rc = LISE_ECUDA;  // warm-up
    cudaEventRecord(e0, c->stream);
    for (int k = 0; k < 3 && rc == LISE_OK; ++k)
      if (launch_planes(c->N, c->mixed, a, c->stream, pb)) rc = LISE_ECUDA;
    cudaEventRecord(e1, c->stream);
    float ms = 0.f;
    if (rc != LISE_OK || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = LISE_ECUDA;
      break;
    }
    if (!best || ms < best_ms) {
      best = pb;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == LISE_OK && best) planes_pb_set(c->N, c->mixed, best);
  return rc;
}

static int tune_pencils(lise_ctx* c, double t0) {
  TRY(tune_planes(c));
  if (pencil_qb_get(c->N, c->mixed)) return LISE_OK;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (pencil_qb_get(c->N, c->mixed)) return LISE_OK;
  // candidate states per batch: 2 and 4, and 1 for the FP64 tensor-core kernels
  // (whose per-state digit groups make one state per batch a valid tile)
  int cands[3], n_valid = 0;
  for (int qb : {1, 2, 4})
    if (pencil_qb_valid(c->N, c->mixed, qb)) cands[n_valid++] = qb;
  if (n_valid < 2) {  // nothing to choose
    if (n_valid == 1) pencil_qb_set(c->N, c->mixed, cands[0]);
    return LISE_OK;
  }
  // valid potentials and T_xy of the input for representative launches (this context's
  // own density groups: no shard exchange while tuning)
  TRY(run_density(c, c->slot[0]));
  TRY(run_reduce(c, 0, nullptr, nullptr, true, t0, false));
  TRY(run_planes(c, c->slot[0]));
  TRY(cu(cudaMemsetAsync(c->M, 0, (size_t)c->ns * (c->mixed ? sizeof(float2) : sizeof(double2)), c->stream)));
  PencilArgs a = pencil_base(c);  // corrector on m = 0: y_{n+1}, p - c into free arrays
  a.xr = c->M;
  a.h = c->dt != 0.0 ? c->dt : 0.005;
  a.q = c->Q;
  a.r = c->R;
  a.pc = c->PC;
  a.ynew = c->slot[1];
  a.dens = 1;
  PencilArgs b = pencil_base(c);  // derivative (and, FP64, predictor) on the input
  b.x = c->slot[0];
  b.h = a.h;
  b.y0 = c->slot[1];
  b.d0 = c->D[0];
  b.d1 = c->D[1];
  b.d2 = c->D[2];
  b.dslot = c->D[3];
  b.pc = c->PC;
  b.q = c->Q;
  b.r = c->R;
  b.m = c->M;
  b.dens = 1;
  const int mode_b = c->mixed ? M_RHS : M_DERIV_PREDICT;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return LISE_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return LISE_ECUDA;
  }
  int best = 0, rc = LISE_OK;
  float best_ms = 0.f;
  for (int ci = 0; ci < n_valid; ++ci) {
    const int qb = cands[ci];
    auto run = [&] {
      return launch_pencils(c->N, c->mixed, M_CORRECT, a, c->stream, qb) ||
             launch_pencils(c->N, c->mixed, mode_b, b, c->stream, qb);
    };
    if (run()) {  // warm-up (and the one-time launch set-up)
      rc = LISE_ECUDA;
      break;
    }
    cudaEventRecord(e0, c->stream);
    for (int k = 0; k < 3; ++k)
      if (run()) rc = LISE_ECUDA;
    cudaEventRecord(e1, c->stream);
    float ms = 0.f;
    if (rc != LISE_OK || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = LISE_ECUDA;
      break;
    }
    if (!best || ms < best_ms) {
      best = qb;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == LISE_OK && best) pencil_qb_set(c->N, c->mixed, best);
  return rc;
}

// A non-finite density or a bounded wait that ran out leaves the device and the context's
// memory intact: a new state (series start, fresh history) clears it.  A CUDA error stays.
static int clear_recoverable(lise_ctx* c) {
  if (c->sticky != LISE_ENONFINITE && c->sticky != LISE_ETIMEOUT) return c->sticky;
  TRY(cu(cudaStreamSynchronize(c->stream)));
  TRY(cu(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream)));
  TRY(cu(cudaStreamSynchronize(c->stream)));
  c->sticky = LISE_OK;
  return LISE_OK;
}

static int set_state_common(lise_ctx* c, const double* psi, double t0, double dt, cudaMemcpyKind kind) {
  if (!c || !psi || !(dt != 0.0) || !std::isfinite(dt) || !std::isfinite(t0)) return LISE_EINVAL;
  if (cudaSetDevice(c->device) != cudaSuccess) return LISE_ECUDA;
  TRY(clear_recoverable(c));
  c->ready = 0;
  TRY(cu(cudaMemcpyAsync(c->slot[0], psi, (size_t)c->ns * sizeof(double2), kind, c->stream)));
  TRY(launch_finite_check(c->slot[0], c->ns, c->err, c->stream) ? LISE_ECUDA : LISE_OK);
  int h = 0;
  TRY(cu(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream)));
  TRY(cu(cudaStreamSynchronize(c->stream)));
  if (h) {
    // reject the input; the context stays usable
    TRY(cu(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream)));
    TRY(cu(cudaStreamSynchronize(c->stream)));
    return LISE_ENONFINITE;
  }
  if (dt != c->dt) drop_graphs(c);  // the step is baked into the captured kernels
  TRY(tune_pencils(c, t0));
  int rc = start_procedure(c, t0, dt);
  if (rc != LISE_OK) {
    c->sticky = rc;
    return rc;
  }
  TRY(fetch_err(c));
  c->ready = 1;
  return LISE_OK;
}

int lise_set_state(lise_ctx* c, const double* psi, double t0, double dt) {
  return set_state_common(c, psi, t0, dt, cudaMemcpyHostToDevice);
}

int lise_set_state_enqueue(lise_ctx* c, const double* psi, double t0, double dt) {
  if (!c || !psi || !(dt != 0.0) || !std::isfinite(dt) || !std::isfinite(t0)) return LISE_EINVAL;
  if (c->sticky) return c->sticky;
  if (cudaSetDevice(c->device) != cudaSuccess) return LISE_ECUDA;
  c->ready = 0;
  TRY(cu(cudaMemcpyAsync(c->slot[0], psi, (size_t)c->ns * sizeof(double2), cudaMemcpyHostToDevice, c->stream)));
  TRY(launch_finite_check(c->slot[0], c->ns, c->err, c->stream) ? LISE_ECUDA : LISE_OK);
  if (dt != c->dt) drop_graphs(c);
  const int rc = start_procedure(c, t0, dt);
  if (rc != LISE_OK) {
    c->sticky = rc;
    return rc;
  }
  c->ready = 1;
  return LISE_OK;
}

int lise_set_state_device(lise_ctx* c, const double* psi_dev, double t0, double dt) {
  return set_state_common(c, psi_dev, t0, dt, cudaMemcpyDeviceToDevice);
}

int lise_pencil_batch(int N, int precision) {
  if (!supported_n(N) || (precision != LISE_FP64 && precision != LISE_MIXED && precision != LISE_MIXED_STRICT))
    return 0;
  return pencil_qb(N, precision != LISE_FP64);
}

int lise_set_pencil_batch(int N, int precision, int qb) {
  if (!supported_n(N) || (precision != LISE_FP64 && precision != LISE_MIXED && precision != LISE_MIXED_STRICT))
    return LISE_EINVAL;
  const int mixed = precision != LISE_FP64;
  if (qb != 0 && !pencil_qb_valid(N, mixed, qb)) return LISE_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  pencil_qb_set(N, mixed, qb);
  return LISE_OK;
}

int lise_planes_per_block(int N, int precision) {
  if (!supported_n(N) || (precision != LISE_FP64 && precision != LISE_MIXED && precision != LISE_MIXED_STRICT))
    return 0;
  const int mixed = precision != LISE_FP64;
  return ozaki_path(N, mixed) ? 0 : planes_pb(N, mixed);
}

int lise_set_planes_per_block(int N, int precision, int pb) {
  if (!supported_n(N) || (precision != LISE_FP64 && precision != LISE_MIXED && precision != LISE_MIXED_STRICT))
    return LISE_EINVAL;
  const int mixed = precision != LISE_FP64;
  if (pb != 0 && !planes_pb_valid(N, mixed, pb)) return LISE_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  planes_pb_set(N, mixed, pb);
  return LISE_OK;
}

int lise_currents(lise_ctx* c, double* j_out) {
  if (!c || !j_out) return LISE_EINVAL;
  if (c->sticky) return c->sticky;
  if (!c->ready) return LISE_ESTATE;
  if (cudaSetDevice(c->device) != cudaSuccess) return LISE_ECUDA;
  double d1h[64];
  first_derivative_table(c->N, c->p.dx, d1h);
  double* d1 = nullptr;
  double* out = nullptr;
  if (cudaMallocAsync((void**)&d1, c->N * sizeof(double), c->stream) != cudaSuccess ||
      cudaMallocAsync((void**)&out, 3 * c->nxyz * sizeof(double), c->stream) != cudaSuccess) {
    cudaGetLastError();
    if (d1) cudaFreeAsync(d1, c->stream);
    return LISE_ENOMEM;
  }
  int rc = cu(cudaMemcpyAsync(d1, d1h, c->N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  // the density partial arrays [group][site] serve as the three current partials
  if (rc == LISE_OK && launch_currents(c->slot[c->y0_slot], d1, c->N, c->p.n_qp, c->qg, c->part_n, c->part_nr,
                                       c->part_ni, c->stream))
    rc = LISE_ECUDA;
  if (rc == LISE_OK) rc = exchange_parts(c);
  const size_t plane = (size_t)c->n_groups_all * c->nxyz;
  if (rc == LISE_OK && launch_sum_groups3(c->parts, c->parts + plane, c->parts + 2 * plane, c->n_groups_all, c->nxyz,
                                          out, c->stream))
    rc = LISE_ECUDA;
  if (rc == LISE_OK)
    rc = cu(cudaMemcpyAsync(j_out, out, 3 * c->nxyz * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  cudaFreeAsync(d1, c->stream);
  cudaFreeAsync(out, c->stream);
  if (rc == LISE_OK) rc = cu(cudaStreamSynchronize(c->stream));
  return rc;
}

int lise_kick(lise_ctx* c, const double* chi) {
  if (!c || !chi) return LISE_EINVAL;
  if (c->sticky) return c->sticky;
  if (!c->ready) return LISE_ESTATE;
  for (long i = 0; i < c->nxyz; ++i)
    if (!std::isfinite(chi[i])) return LISE_EINVAL;
  if (cudaSetDevice(c->device) != cudaSuccess) return LISE_ECUDA;
  c->ready = 0;
  // chi into the energy scratch (2 nxyz doubles); the kicked y(t) into slot 0, where the
  // series start expects its initial state
  TRY(cu(cudaMemcpyAsync(c->e_site, chi, c->nxyz * sizeof(double), cudaMemcpyHostToDevice, c->stream)));
  TRY(launch_kick(c->slot[c->y0_slot], c->slot[0], c->e_site, c->p.n_qp, c->nxyz, c->stream) ? LISE_ECUDA
                                                                                                : LISE_OK);
  const int rc = start_procedure(c, c->t, c->dt);
  if (rc != LISE_OK) {
    c->sticky = rc;
    return rc;
  }
  TRY(fetch_err(c));
  c->ready = 1;
  return LISE_OK;
}

int lise_step(lise_ctx* c, int n_steps, double dt) {
  if (!c || n_steps < 0) return LISE_EINVAL;
  if (c->sticky) return c->sticky;
  if (!c->ready) return LISE_ESTATE;
  if (dt != c->dt) return LISE_EINVAL;
  if (cudaSetDevice(c->device) != cudaSuccess) return LISE_ECUDA;
  int k = 0;
  while (k < n_steps) {
    int rc;
    // replay captured graphs for runs of kGraphSteps steps (plain launches while profiling,
    // so that every kernel is bracketed by its own events)
    if (!c->prof && n_steps - k >= kGraphSteps && (!c->exch || (c->exch_on_device && c->exch_capturable))) {
      rc = graph_steps(c);
      k += kGraphSteps;
    } else {
      rc = abm_step(c);
      ++k;
    }
    if (rc != LISE_OK) {
      c->sticky = rc;
      return rc;
    }
  }
  return LISE_OK;
}

int lise_get_state(lise_ctx* c, double* psi_out) {
  if (!c || !psi_out) return LISE_EINVAL;
  if (!c->ready) return LISE_ESTATE;
  TRY(fetch_err(c));
  TRY(cu(cudaMemcpyAsync(psi_out, c->slot[c->y0_slot], (size_t)c->ns * sizeof(double2), cudaMemcpyDeviceToHost,
                         c->stream)));
  return cu(cudaStreamSynchronize(c->stream));
}

int lise_get_state_device(lise_ctx* c, double* psi_dev_out) {
  if (!c || !psi_dev_out) return LISE_EINVAL;
  if (!c->ready) return LISE_ESTATE;
  TRY(fetch_err(c));
  TRY(cu(cudaMemcpyAsync(psi_dev_out, c->slot[c->y0_slot], (size_t)c->ns * sizeof(double2),
                         cudaMemcpyDeviceToDevice, c->stream)));
  return cu(cudaStreamSynchronize(c->stream));
}

int lise_get_time(lise_ctx* c, double* t) {
  if (!c || !t) return LISE_EINVAL;
  *t = c->t;
  return LISE_OK;
}

int lise_densities(lise_ctx* c, double* n_out, double* nu_out) {
  if (!c || !n_out || !nu_out) return LISE_EINVAL;
  if (!c->ready) return LISE_ESTATE;
  if (c->sticky) return c->sticky;
  TRY(run_density(c, c->slot[c->y0_slot]));
  TRY(run_reduce(c, 0, nullptr, nullptr, false, c->t));
  TRY(cu(cudaMemcpyAsync(n_out, c->dn[0], c->nxyz * sizeof(double), cudaMemcpyDeviceToHost, c->stream)));
  TRY(cu(cudaMemcpyAsync(nu_out, c->dnu[0], c->nxyz * sizeof(double2), cudaMemcpyDeviceToHost, c->stream)));
  TRY(cu(cudaStreamSynchronize(c->stream)));
  return fetch_err(c);
}

int lise_energy(lise_ctx* c, double* E, double* Nout) {
  if (!c || !E || !Nout) return LISE_EINVAL;
  if (!c->ready) return LISE_ESTATE;
  if (c->sticky) return c->sticky;
  const double2* y = c->slot[c->y0_slot];
  TRY(run_density(c, y));
  TRY(run_reduce(c, 0, nullptr, nullptr, false, c->t));
  TRY(run_planes(c, y));
  PencilArgs a = pencil_base(c);
  a.eta = nullptr;
  a.x = y;
  a.dens = 1;
  TRY(run_pencils(c, M_ENERGY, a));
  TRY(exchange_parts(c));  // the other shards' kinetic partials
  TRY(launch_energy_sites(c->parts, c->n_groups_all, c->dn[0], c->dnu[0], c->v_static, drive_at(c, c->t),
                          make_pairing(&c->p), c->N, c->p.dx, c->e_site, c->stream)
          ? LISE_ECUDA
          : LISE_OK);
  TRY(cu(cudaMemcpyAsync(c->host_e, c->e_site, 2 * c->nxyz * sizeof(double), cudaMemcpyDeviceToHost, c->stream)));
  TRY(cu(cudaStreamSynchronize(c->stream)));
  TRY(fetch_err(c));
  // compensated (Neumaier) sums over sites
  double se = 0, ce = 0, sn = 0, cn = 0;
  for (long i = 0; i < c->nxyz; ++i) {
    double x = c->host_e[i];
    double t = se + x;
    ce += (std::fabs(se) >= std::fabs(x)) ? (se - t) + x : (x - t) + se;
    se = t;
    x = c->host_e[c->nxyz + i];
    t = sn + x;
    cn += (std::fabs(sn) >= std::fabs(x)) ? (sn - t) + x : (x - t) + sn;
    sn = t;
  }
  *E = se + ce;
  *Nout = sn + cn;
  return LISE_OK;
}

int lise_rhs(lise_ctx* c, const double* psi, double t, double* dpsi_out) {
  if (!c || !psi || !dpsi_out || !std::isfinite(t)) return LISE_EINVAL;
  if (c->sticky) return c->sticky;
  if (cudaSetDevice(c->device) != cudaSuccess) return LISE_ECUDA;
  c->ready = 0;
  double2* x = c->slot[0];
  TRY(cu(cudaMemcpyAsync(x, psi, (size_t)c->ns * sizeof(double2), cudaMemcpyHostToDevice, c->stream)));
  TRY(run_density(c, x));
  TRY(run_reduce(c, 0, nullptr, nullptr, true, t));
  TRY(run_planes(c, x));
  TRY(run_eta(c, x));
  PencilArgs a = pencil_base(c);
  a.x = x;
  a.out = c->slot[1];
  TRY(run_pencils(c, M_RHS, a));
  TRY(cu(cudaMemcpyAsync(dpsi_out, c->slot[1], (size_t)c->ns * sizeof(double2), cudaMemcpyDeviceToHost, c->stream)));
  TRY(cu(cudaStreamSynchronize(c->stream)));
  return fetch_err(c);
}

// ---------------------------------------------------------------- checkpoint --
namespace {
struct CkptHeader {
  char magic[8];        // "LISECKP3"
  int N, n_qp, precision, y0_slot_unused;
  double t, dt;
  long long ns, nxyz;
  char pad[8];
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header is 64 bytes");
const int kCkptArrays = 10;

void ckpt_arrays(lise_ctx* c, void* arr[kCkptArrays], size_t sz[kCkptArrays]) {
  arr[0] = c->slot[c->y0_slot];
  arr[1] = c->slot[1 - c->y0_slot];
  for (int k = 0; k < 4; ++k) arr[2 + k] = c->D[k];
  arr[6] = c->M;
  arr[7] = c->PC;
  arr[8] = c->Q;
  arr[9] = c->R;
  // y_n, y_{n-1} and Q are complex128; the y' ring and m the compute precision; P-C and R
  // the compute precision, complex128 in the strict split
  const size_t sr = (size_t)c->ns * (c->mixed ? sizeof(float2) : sizeof(double2));
  for (int k = 0; k < kCkptArrays; ++k) sz[k] = sr;
  sz[0] = sz[1] = sz[8] = (size_t)c->ns * sizeof(double2);
  sz[7] = sz[9] = (size_t)c->ns * hist_elem(c);
}
}  // namespace

size_t lise_checkpoint_bytes(const lise_ctx* c) {
  if (!c) return 0;
  return sizeof(CkptHeader) + 3 * (size_t)c->ns * sizeof(double2) +
         (kCkptArrays - 5) * (size_t)c->ns * (c->mixed ? sizeof(float2) : sizeof(double2)) +
         2 * (size_t)c->ns * hist_elem(c) +
         (size_t)c->nxyz * (sizeof(double) + sizeof(double2));
}

int lise_checkpoint_save(lise_ctx* c, void* buf, size_t bytes) {
  if (!c || !buf) return LISE_EINVAL;
  if (!c->ready) return LISE_ESTATE;
  if (bytes < lise_checkpoint_bytes(c)) return LISE_EINVAL;
  TRY(fetch_err(c));
  CkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, "LISECKP3", 8);
  hd.N = c->N;
  hd.n_qp = c->p.n_qp;
  hd.precision = c->p.precision;
  hd.t = c->t;
  hd.dt = c->dt;
  hd.ns = c->ns;
  hd.nxyz = c->nxyz;
  char* out = static_cast<char*>(buf);
  std::memcpy(out, &hd, sizeof(hd));
  size_t off = sizeof(hd);
  void* arr[kCkptArrays];
  size_t sz[kCkptArrays];
  ckpt_arrays(c, arr, sz);
  for (int k = 0; k < kCkptArrays; off += sz[k], ++k)
    TRY(cu(cudaMemcpyAsync(out + off, arr[k], sz[k], cudaMemcpyDeviceToHost, c->stream)));
  TRY(cu(cudaMemcpyAsync(out + off, c->W, c->nxyz * sizeof(double), cudaMemcpyDeviceToHost, c->stream)));
  off += c->nxyz * sizeof(double);
  TRY(cu(cudaMemcpyAsync(out + off, c->Dl, c->nxyz * sizeof(double2), cudaMemcpyDeviceToHost, c->stream)));
  return cu(cudaStreamSynchronize(c->stream));
}

int lise_checkpoint_load(lise_ctx* c, const void* buf, size_t bytes) {
  if (!c || !buf) return LISE_EINVAL;
  if (c->sticky) return c->sticky;
  if (bytes < lise_checkpoint_bytes(c)) return LISE_EINVAL;
  CkptHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  if (std::memcmp(hd.magic, "LISECKP3", 8) != 0 || hd.N != c->N || hd.n_qp != c->p.n_qp ||
      hd.precision != c->p.precision || hd.ns != c->ns || hd.nxyz != c->nxyz || !(hd.dt != 0.0))
    return LISE_EINVAL;
  if (cudaSetDevice(c->device) != cudaSuccess) return LISE_ECUDA;
  c->ready = 0;
  c->y0_slot = 0;
  void* arr[kCkptArrays];
  size_t sz[kCkptArrays];
  ckpt_arrays(c, arr, sz);
  const char* in = static_cast<const char*>(buf);
  size_t off = sizeof(hd);
  for (int k = 0; k < kCkptArrays; off += sz[k], ++k)
    TRY(cu(cudaMemcpyAsync(arr[k], in + off, sz[k], cudaMemcpyHostToDevice, c->stream)));
  TRY(cu(cudaMemcpyAsync(c->W, in + off, c->nxyz * sizeof(double), cudaMemcpyHostToDevice, c->stream)));
  off += c->nxyz * sizeof(double);
  TRY(cu(cudaMemcpyAsync(c->Dl, in + off, c->nxyz * sizeof(double2), cudaMemcpyHostToDevice, c->stream)));
  TRY(cu(cudaStreamSynchronize(c->stream)));
  if (hd.dt != c->dt) drop_graphs(c);
  c->t = hd.t;
  c->dt = hd.dt;
  c->ready = 1;
  return LISE_OK;
}

int lise_profile(lise_ctx* c, int enable) {
  if (!c) return LISE_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LISE_ECUDA;
  c->prof = enable != 0;
  if (c->prof) c->rec_cls.clear();
  return LISE_OK;
}

int lise_profile_read(lise_ctx* c, int cls, long* launches, double* total_ms) {
  if (!c || !launches || !total_ms || cls < 0 || cls >= LISE_KC_COUNT) return LISE_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LISE_ECUDA;
  long n = 0;
  double ms = 0.0;
  for (size_t i = 0; i < c->rec_cls.size(); ++i) {
    if (c->rec_cls[i] != cls) continue;
    float e = 0.f;
    if (cudaEventElapsedTime(&e, c->ev_pool[2 * i], c->ev_pool[2 * i + 1]) != cudaSuccess) return LISE_ECUDA;
    ms += e;
    ++n;
  }
  *launches = n;
  *total_ms = ms;
  return LISE_OK;
}

const char* lise_kernel_class_name(int cls) {
  static const char* names[LISE_KC_COUNT] = {"planes", "pencils", "reduce", "pointwise"};
  return (cls >= 0 && cls < LISE_KC_COUNT) ? names[cls] : nullptr;
}

int lise_set_shard(lise_ctx* c, const lise_shard* sh) {
  if (!c || !sh) return LISE_EINVAL;
  if (sh->group_size < 1 || sh->group_size > 64) return LISE_EINVAL;
  const int n_local = (c->p.n_qp + sh->group_size - 1) / sh->group_size;
  if (sh->first_group < 0 || sh->n_groups_all < 1 || (long)sh->first_group + n_local > (long)sh->n_groups_all)
    return LISE_EINVAL;
  if (cudaSetDevice(c->device) != cudaSuccess) return LISE_ECUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LISE_ECUDA;
  // new partial-sum arrays for all shards' groups (zeroed), and the host copy of a host exchange
  const size_t bytes = 3 * (size_t)sh->n_groups_all * c->nxyz * sizeof(double);
  double* parts = nullptr;
  double* host = nullptr;
  if (cudaMallocAsync((void**)&parts, bytes, c->stream) != cudaSuccess) {
    cudaGetLastError();
    return LISE_ENOMEM;
  }
  if (sh->exchange && !sh->on_device && cudaHostAlloc((void**)&host, bytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeAsync(parts, c->stream);
    return LISE_ENOMEM;
  }
  if (cudaMemsetAsync(parts, 0, bytes, c->stream) != cudaSuccess) {
    cudaFreeAsync(parts, c->stream);
    if (host) cudaFreeHost(host);
    return LISE_ECUDA;
  }
  cudaFreeAsync(c->parts, c->stream);
  if (c->host_parts) cudaFreeHost(c->host_parts);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LISE_ECUDA;
  drop_graphs(c);  // the captured launches point at the old arrays
  c->parts = parts;
  c->host_parts = host;
  c->qg = sh->group_size;
  c->n_groups = n_local;
  c->n_groups_all = sh->n_groups_all;
  c->first_group = sh->first_group;
  const size_t plane = (size_t)c->n_groups_all * c->nxyz, off = (size_t)c->first_group * c->nxyz;
  c->part_n = parts + off;
  c->part_nr = parts + plane + off;
  c->part_ni = parts + 2 * plane + off;
  c->exch = sh->exchange;
  c->exch_user = sh->user;
  c->exch_on_device = sh->on_device;
  c->exch_capturable = sh->capturable;
  c->ready = 0;  // the history was built with the old groups
  return LISE_OK;
}

int lise_set_wait_limit(lise_ctx* c, long polls) {
  if (!c) return LISE_EINVAL;
  const long w = polls < 0 ? 0 : (polls == 0 ? -1 : polls);
  if (w != c->wait_polls) {
    if (cudaSetDevice(c->device) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) return LISE_ECUDA;
    drop_graphs(c);  // the limit is a kernel parameter of the captured launches
    c->wait_polls = w;
  }
  return LISE_OK;
}

int lise_sync(lise_ctx* c) {
  if (!c) return LISE_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    c->sticky = LISE_ECUDA;
    return c->sticky;
  }
  if (cudaGetLastError() != cudaSuccess) {
    c->sticky = LISE_ECUDA;
    return c->sticky;
  }
  return fetch_err(c);
}

void lise_destroy(lise_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_ctx(c);
  delete c;
}

}  // extern "C"

// ------------------------------------------------------------------- batches --
// Several evolutions stepped together (FP32 compute precision): every kernel class of an
// ABM step runs as one launch per lattice size over all evolutions of that size, from a
// device work table (PencilBatch and friends in lise_kernels.cuh) holding each evolution's
// arguments for each of the four history configurations of a 4-step period; four steps
// are captured as one CUDA graph.  The arguments are exactly those of abm_step's mixed
// branch, so each evolution's result is bitwise that of lise_step on its own context.
namespace {

constexpr size_t kTableAlign = 256;  // (tensor maps need 64-byte alignment)

struct MixedStepArgs {
  PlanesArgs pl_m, pl_y;
  PencilArgs corr, deriv;
  PointwiseArgs pred;
  ReduceArgs red[2];
};

// abm_step's launches (mixed branch) for the history configuration (y0_slot, D).
MixedStepArgs mixed_step_args(lise_ctx* c, int y0_slot, void* const D[4]) {
  MixedStepArgs a;
  const double h = c->dt;
  double2* yn = c->slot[y0_slot];
  double2* ynm1 = c->slot[1 - y0_slot];
  a.pl_m = planes_args(c, nullptr, c->M);
  a.corr = pencil_base(c);
  a.corr.xr = c->M;
  a.corr.h = h;
  a.corr.q = c->Q;
  a.corr.r = c->R;
  a.corr.pc = c->PC;
  a.corr.ynew = ynm1;
  a.corr.dens = 1;
  a.red[0] = reduce_args(c, 1, nullptr, nullptr, true, true);
  a.pl_y = planes_args(c, ynm1, nullptr);
  a.deriv = pencil_base(c);
  a.deriv.x = ynm1;
  a.deriv.out = nullptr;
  a.deriv.dslot = D[3];
  a.pred = predict_args(c, ynm1, yn, D[3], D[0], D[1], D[2], h);
  a.red[1] = reduce_args(c, 1, nullptr, nullptr, true, true);
  return a;
}

}  // namespace

struct lise_batch {
  std::vector<lise_ctx*> ctx;
  std::vector<int> y0_slot0;          // each context's configuration at creation
  std::vector<std::array<void*, 4>> D0;
  int device = 0, strict = 0;
  cudaStream_t stream = nullptr;
  struct Size {                       // the evolutions of one lattice size
    int N = 0, qb = 0, pb = 0;         // pencils batch size, planes per block
    long nxyz = 0;
    std::vector<int> evo;             // their batch indices
    int n_items = 0;                  // (evolution, group) items of the pencils and predictor launches
    // pencils and planes arguments (host copies: the launches carry them in their parameters), per
    // history phase and evolution; the evolutions in chunks of at most kBatchInline, one launch each
    std::vector<PencilArgs> corr[4], deriv[4];
    std::vector<PlanesArgs> pl_m[4], pl_y[4];
    std::vector<int> chunk0;          // first evolution (index into evo) of each chunk, and the end
    std::vector<int> chunk_item0;     // first item of each chunk, and the end
    std::vector<long> pl_block0;      // first planes block of each evolution within its chunk
    std::vector<long> chunk_blocks;   // planes blocks of each chunk
    PointwiseArgs* pred[4] = {};
    int2* items = nullptr;            // items (evolution relative to its chunk, group), by chunk
    int2* items_abs = nullptr;        // the same items with the evolution's index in evo (predictor)
    ReduceArgs* red[4][2] = {};       // the reductions of these evolutions
    long* red_block0 = nullptr;
    long red_blocks = 0;
    cudaStream_t stream = nullptr;    // this size's launches (forked from and joined to the batch stream)
    cudaEvent_t done = nullptr;       // end of this size's launches of a chunk
  };
  cudaEvent_t fork = nullptr;
  std::vector<Size> sizes;
  double* drive_dev = nullptr;        // [4 phases][2 reductions][evolutions]
  std::vector<double> drive_host;
  void* tables = nullptr;
  long step = 0;                      // steps taken since creation
  cudaGraphExec_t graph[4] = {};      // 4 steps from phase k
};

namespace {

void free_batch(lise_batch* b) {
  for (auto& g : b->graph)
    if (g) cudaGraphExecDestroy(g);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& z : b->sizes) {
    if (z.stream) cudaStreamDestroy(z.stream);
    if (z.done) cudaEventDestroy(z.done);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->tables) cudaFree(b->tables);
  if (b->stream) cudaStreamDestroy(b->stream);
}

// The launches made by f(size, stream) for every lattice size, each size on its own stream
// (the sizes run independently on the device), forked from and joined back to the batch stream.
template <typename F>
int batch_per_size(lise_batch* b, F f) {
  if (b->sizes.size() == 1) return f(b->sizes[0], b->stream);
  if (cudaEventRecord(b->fork, b->stream) != cudaSuccess) return LISE_ECUDA;
  for (auto& z : b->sizes) {
    if (cudaStreamWaitEvent(z.stream, b->fork, 0) != cudaSuccess) return LISE_ECUDA;
    TRY(f(z, z.stream));
    if (cudaEventRecord(z.done, z.stream) != cudaSuccess) return LISE_ECUDA;
  }
  for (auto& z : b->sizes)
    if (cudaStreamWaitEvent(b->stream, z.done, 0) != cudaSuccess) return LISE_ECUDA;
  return LISE_OK;
}

// One planes launch per chunk of the evolutions of one lattice size (arguments a[e]).
int batch_planes(const lise_batch::Size& z, const std::vector<PlanesArgs>& a, cudaStream_t st) {
  PlanesBatch pb;
  for (size_t c = 0; c + 1 < z.chunk0.size(); ++c) {
    const int e0 = z.chunk0[c], ne = z.chunk0[c + 1] - e0;
    for (int j = 0; j < ne; ++j) {
      pb.seg[j] = a[e0 + j];
      pb.block0[j] = z.pl_block0[e0 + j];
    }
    pb.block0[ne] = z.chunk_blocks[c];
    pb.n_seg = ne;
    if (launch_planes_batch(z.N, z.pb, pb, z.chunk_blocks[c], st)) return LISE_ECUDA;
  }
  return LISE_OK;
}

// The same for a pencils launch in the given mode.
int batch_pencils(const lise_batch::Size& z, int mode, int strict, const std::vector<PencilArgs>& a, cudaStream_t st) {
  PencilBatch pb;
  for (size_t c = 0; c + 1 < z.chunk0.size(); ++c) {
    const int e0 = z.chunk0[c], ne = z.chunk0[c + 1] - e0;
    for (int j = 0; j < ne; ++j) pb.evo[j] = a[e0 + j];
    pb.items = z.items + z.chunk_item0[c];
    if (launch_pencils_batch(z.N, mode, strict, pb, z.chunk_item0[c + 1] - z.chunk_item0[c], z.qb, st))
      return LISE_ECUDA;
  }
  return LISE_OK;
}

// The launches of one ABM step in history phase k of the evolutions of one lattice size.
int batch_size_step(lise_batch* b, lise_batch::Size& z, int k, cudaStream_t st) {
  const int ne = (int)z.evo.size();
  TRY(batch_planes(z, z.pl_m[k], st));
  TRY(batch_pencils(z, M_CORRECT, b->strict, z.corr[k], st));
  if (launch_reduce_batch(ReduceBatch{z.red[k][0], z.red_block0, ne}, z.red_blocks, st)) return LISE_ECUDA;
  TRY(batch_planes(z, z.pl_y[k], st));
  TRY(batch_pencils(z, M_RHS, 0, z.deriv[k], st));
  if (launch_predict_batch(b->strict, PredictBatch{z.pred[k], z.items_abs}, z.nxyz, z.n_items, st) ||
      launch_reduce_batch(ReduceBatch{z.red[k][1], z.red_block0, ne}, z.red_blocks, st))
    return LISE_ECUDA;
  return LISE_OK;
}

// m ABM steps from history phase k0.
int batch_launch_steps(lise_batch* b, int k0, int m) {
  return batch_per_size(b, [&](lise_batch::Size& z, cudaStream_t st) {
    for (int j = 0; j < m; ++j) TRY(batch_size_step(b, z, (k0 + j) % 4, st));
    return LISE_OK;
  });
}

// Drive amplitudes of the reductions of the next m steps (phases step .. step + m - 1).
int batch_refresh_drive(lise_batch* b, int m) {
  const int E = (int)b->ctx.size();
  bool any = false;
  for (int e = 0; e < E; ++e) {
    lise_ctx* c = b->ctx[e];
    if (c->p.drive_A == 0.0) continue;
    any = true;
    double t = c->t;  // accumulated as abm_step does (bitwise the same times)
    for (int j = 0; j < m; ++j) {
      const int k = (int)((b->step + j) % 4);
      const double t1 = t + c->dt;
      b->drive_host[(size_t)(2 * k) * E + e] = drive_at(c, t1);
      b->drive_host[(size_t)(2 * k + 1) * E + e] = drive_at(c, t1 + c->dt);
      t = t1;
    }
  }
  if (!any) return LISE_OK;
  return cu(cudaMemcpyAsync(b->drive_dev, b->drive_host.data(), b->drive_host.size() * sizeof(double),
                            cudaMemcpyHostToDevice, b->stream));
}

}  // namespace

extern "C" {

static int batch_create(lise_ctx* const* ctxs, int n, lise_batch** out);

int lise_batch_create(lise_ctx* const* ctxs, int n, lise_batch** out) {
  try {  // (host containers: an allocation failure is reported, not thrown through the C ABI)
    return batch_create(ctxs, n, out);
  } catch (...) {
    if (out) *out = nullptr;
    return LISE_ENOMEM;
  }
}

}  // extern "C"

static int batch_create(lise_ctx* const* ctxs, int n, lise_batch** out) {
  if (!out) return LISE_EINVAL;
  *out = nullptr;
  if (!ctxs || n < 1) return LISE_EINVAL;
  for (int e = 0; e < n; ++e) {
    lise_ctx* c = ctxs[e];
    if (!c) return LISE_EINVAL;
    for (int f = 0; f < e; ++f)
      if (ctxs[f] == c) return LISE_EINVAL;
    if (!c->mixed || c->strict != ctxs[0]->strict || c->device != ctxs[0]->device) return LISE_EINVAL;
    if (c->p.remove_phase || c->p.renormalize || c->exch || c->n_groups_all != c->n_groups) return LISE_EINVAL;
    if (c->sticky) return c->sticky;
    if (!c->ready) return LISE_ESTATE;
  }
  lise_batch* b = new (std::nothrow) lise_batch();
  if (!b) return LISE_ENOMEM;
  b->device = ctxs[0]->device;
  b->strict = ctxs[0]->strict;
  int rc = cudaSetDevice(b->device) == cudaSuccess ? LISE_OK : LISE_ECUDA;
  for (int e = 0; e < n && rc == LISE_OK; ++e) {
    lise_ctx* c = ctxs[e];
    rc = cu(cudaStreamSynchronize(c->stream));  // the contexts' own work is done
    b->ctx.push_back(c);
    b->y0_slot0.push_back(c->y0_slot);
    b->D0.push_back({c->D[0], c->D[1], c->D[2], c->D[3]});
  }
  if (rc == LISE_OK && cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) rc = LISE_ECUDA;
  if (rc == LISE_OK && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) rc = LISE_ECUDA;
  // lattice sizes in order of first appearance
  for (int e = 0; e < n && rc == LISE_OK; ++e) {
    lise_ctx* c = ctxs[e];
    auto it = std::find_if(b->sizes.begin(), b->sizes.end(), [&](const lise_batch::Size& z) { return z.N == c->N; });
    if (it == b->sizes.end()) {
      lise_batch::Size z;
      z.N = c->N;
      z.nxyz = c->nxyz;
      z.qb = pencil_qb(c->N, 1);
      z.pb = planes_pb(c->N, 1);
      b->sizes.push_back(z);
      it = b->sizes.end() - 1;
    }
    it->evo.push_back(e);
  }
  for (auto& z : b->sizes) {
    if (rc == LISE_OK && cudaStreamCreateWithFlags(&z.stream, cudaStreamNonBlocking) != cudaSuccess) rc = LISE_ECUDA;
    if (rc == LISE_OK && cudaEventCreateWithFlags(&z.done, cudaEventDisableTiming) != cudaSuccess) rc = LISE_ECUDA;
  }
  // host image of every table, then one device copy
  std::vector<unsigned char> img;
  auto place = [&](size_t bytes) {
    const size_t off = (img.size() + kTableAlign - 1) / kTableAlign * kTableAlign;
    img.resize(off + bytes);
    return off;
  };
  struct Off {
    size_t pred[4], red[4][2], items, items_abs, red_block0;
  };
  std::vector<Off> off(b->sizes.size());
  for (size_t zi = 0; zi < b->sizes.size(); ++zi) {
    auto& z = b->sizes[zi];
    const size_t ne = z.evo.size();
    for (int k = 0; k < 4; ++k) {
      off[zi].pred[k] = place(ne * sizeof(PointwiseArgs));
      for (int r = 0; r < 2; ++r) off[zi].red[k][r] = place(ne * sizeof(ReduceArgs));
    }
    off[zi].red_block0 = place((ne + 1) * sizeof(long));
    z.n_items = 0;
    for (int e : z.evo) z.n_items += b->ctx[e]->n_groups;
    off[zi].items = place((size_t)z.n_items * sizeof(int2));
    off[zi].items_abs = place((size_t)z.n_items * sizeof(int2));
  }
  const size_t drive_off = place((size_t)8 * n * sizeof(double));
  if (rc == LISE_OK && cudaMalloc(&b->tables, img.size()) != cudaSuccess) {
    cudaGetLastError();
    rc = LISE_ENOMEM;
  }
  unsigned char* dev = static_cast<unsigned char*>(b->tables);
  // fill the image
  for (size_t zi = 0; zi < b->sizes.size() && rc == LISE_OK; ++zi) {
    auto& z = b->sizes[zi];
    const int ne = (int)z.evo.size();
    int2* items = reinterpret_cast<int2*>(img.data() + off[zi].items);
    int2* items_abs = reinterpret_cast<int2*>(img.data() + off[zi].items_abs);
    // chunks of at most kBatchInline evolutions: items and planes blocks counted per chunk
    z.chunk0.clear();
    z.chunk_item0.clear();
    z.chunk_blocks.clear();
    z.pl_block0.assign(ne, 0);
    int it = 0;
    for (int j = 0; j < ne; ++j) {
      if (j % kBatchInline == 0) {
        z.chunk0.push_back(j);
        z.chunk_item0.push_back(it);
        z.chunk_blocks.push_back(0);
      }
      lise_ctx* c = b->ctx[z.evo[j]];
      for (int g = 0; g < c->n_groups; ++g) {
        items[it] = make_int2(j % kBatchInline, g);
        items_abs[it++] = make_int2(j, g);
      }
      z.pl_block0[j] = z.chunk_blocks.back();
      z.chunk_blocks.back() += planes_blocks((long)c->p.n_qp * 2 * c->N, z.pb);
    }
    z.chunk0.push_back(ne);
    z.chunk_item0.push_back(it);
    for (int k = 0; k < 4 && rc == LISE_OK; ++k) {
      z.corr[k].resize(ne);
      z.deriv[k].resize(ne);
      z.pl_m[k].resize(ne);
      z.pl_y[k].resize(ne);
      std::vector<PencilArgs>& corr = z.corr[k];
      std::vector<PencilArgs>& deriv = z.deriv[k];
      std::vector<PlanesArgs>& plm = z.pl_m[k];
      std::vector<PlanesArgs>& ply = z.pl_y[k];
      PointwiseArgs* pred = reinterpret_cast<PointwiseArgs*>(img.data() + off[zi].pred[k]);
      for (size_t j = 0; j < z.evo.size(); ++j) {
        const int e = z.evo[j];
        lise_ctx* c = b->ctx[e];
        // the configuration after k steps: slot parity flips, the derivative ring rotates
        void* Dk[4];
        for (int q = 0; q < 4; ++q) Dk[q] = b->D0[e][(q - k + 4) % 4];
        MixedStepArgs a = mixed_step_args(c, (b->y0_slot0[e] + k) % 2, Dk);
        if (!pencils_batch_maps(z.N, M_CORRECT, b->strict, z.qb, &a.corr) ||
            !pencils_batch_maps(z.N, M_RHS, 0, z.qb, &a.deriv)) {
          rc = LISE_ECUDA;
          break;
        }
        corr[j] = a.corr;
        deriv[j] = a.deriv;
        plm[j] = a.pl_m;
        ply[j] = a.pl_y;
        pred[j] = a.pred;
        for (int r = 0; r < 2; ++r) {
          ReduceArgs ra = a.red[r];
          if (c->p.drive_A != 0.0)
            ra.drive_ptr = reinterpret_cast<const double*>(dev + drive_off) + (size_t)(2 * k + r) * n + e;
          reinterpret_cast<ReduceArgs*>(img.data() + off[zi].red[k][r])[j] = ra;
        }
      }
      z.pred[k] = reinterpret_cast<PointwiseArgs*>(dev + off[zi].pred[k]);
      for (int r = 0; r < 2; ++r) z.red[k][r] = reinterpret_cast<ReduceArgs*>(dev + off[zi].red[k][r]);
    }
    long* rb0 = reinterpret_cast<long*>(img.data() + off[zi].red_block0);
    rb0[0] = 0;
    for (size_t j = 0; j < z.evo.size(); ++j) rb0[j + 1] = rb0[j] + (b->ctx[z.evo[j]]->nxyz + 255) / 256;
    z.red_blocks = rb0[z.evo.size()];
    z.red_block0 = reinterpret_cast<long*>(dev + off[zi].red_block0);
    z.items = reinterpret_cast<int2*>(dev + off[zi].items);
    z.items_abs = reinterpret_cast<int2*>(dev + off[zi].items_abs);
  }
  if (rc == LISE_OK) {
    b->drive_dev = reinterpret_cast<double*>(dev + drive_off);
    b->drive_host.assign((size_t)8 * n, 0.0);
    rc = cu(cudaMemcpyAsync(b->tables, img.data(), img.size(), cudaMemcpyHostToDevice, b->stream));
    if (rc == LISE_OK) rc = cu(cudaStreamSynchronize(b->stream));
  }
  if (rc != LISE_OK) {
    free_batch(b);
    delete b;
    return rc;
  }
  *out = b;
  return LISE_OK;
}

extern "C" {

int lise_batch_step(lise_batch* b, int n_steps) {
  if (!b || n_steps < 0) return LISE_EINVAL;
  if (cudaSetDevice(b->device) != cudaSuccess) return LISE_ECUDA;
  // every member must still be where the batch left it (not stepped on its own)
  for (size_t e = 0; e < b->ctx.size(); ++e) {
    lise_ctx* c = b->ctx[e];
    if (c->sticky) return c->sticky;
    if (!c->ready || c->y0_slot != (int)((b->y0_slot0[e] + b->step) % 2) || c->D[0] != b->D0[e][(4 - b->step % 4) % 4])
      return LISE_ESTATE;
  }
  int done = 0;
  while (done < n_steps) {
    const int phase = (int)(b->step % 4);
    const int m = (n_steps - done >= 4) ? 4 : 1;
    TRY(batch_refresh_drive(b, m));
    if (m == 4) {
      cudaGraphExec_t& g = b->graph[phase];
      if (!g) {
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LISE_ECUDA;
        int rc = batch_launch_steps(b, phase, 4);
        const cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
        if (rc == LISE_OK && (e != cudaSuccess || !graph)) rc = LISE_ECUDA;
        if (rc == LISE_OK && cudaGraphInstantiate(&g, graph, 0) != cudaSuccess) rc = LISE_ECUDA;
        if (graph) cudaGraphDestroy(graph);
        TRY(rc);
      }
      TRY(cu(cudaGraphLaunch(g, b->stream)));
    } else {
      TRY(batch_launch_steps(b, phase, 1));
    }
    for (lise_ctx* c : b->ctx)
      for (int j = 0; j < m; ++j) rotate_history(c, c->t + c->dt);
    b->step += m;
    done += m;
  }
  return LISE_OK;
}

int lise_batch_sync(lise_batch* b) {
  if (!b) return LISE_EINVAL;
  if (cudaSetDevice(b->device) != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess) return LISE_ECUDA;
  int first = LISE_OK;
  for (lise_ctx* c : b->ctx) {
    const int rc = fetch_err(c);
    if (first == LISE_OK) first = rc;
  }
  return first;
}

void* lise_batch_stream(lise_batch* b) { return b ? (void*)b->stream : nullptr; }

void lise_batch_destroy(lise_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  free_batch(b);
  delete b;
}

}  // extern "C"
