// lise_noalloc.cu -- lise_rhs_noalloc: one right-hand side on caller-owned
// device buffers, with all scratch memory in a fixed device array.
//
// Who needs this: code that must not call cudaMalloc while it runs.  Examples
// are a host framework whose caching allocator already holds the free device
// memory (a stray cudaMalloc would fail or fragment its pool), a latency-
// critical loop where cudaMalloc's implicit device synchronisation and
// unbounded cost are not acceptable, and plug-ins that are only handed buffers
// and a stream.  Such callers pass the state and the output; everything else
// the right-hand side needs (the in-plane kinetic part, density partial sums,
// densities, potentials, FFT tables) lives in g_rhs_scratch below.
//
// g_rhs_scratch is a file-scope __device__ array: every GPU that loads this
// library keeps LISE_NOALLOC_SCRATCH_BYTES of device memory for it until the
// process exits.  In host code the name g_rhs_scratch is only a host-side
// stand-in; its device address is obtained once per device with
// cudaGetSymbolAddress (with that device current) and cached.
#include <cmath>
#include <cstring>

#include "../../include/lise.h"
#include "lise_internal.h"
#include "lise_kernels.cuh"

using namespace lise;

static __device__ __align__(256) unsigned char g_rhs_scratch[LISE_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
unsigned char* g_scratch_dev[kMaxDevices] = {};  // device address of g_rhs_scratch per device

// FFT twiddles and kinetic factors, built on the host into static storage (no
// heap allocation) and copied into the scratch array on every call.
alignas(16) double g_tab_d[4 * 64];
alignas(16) float g_tab_f[4 * 64];
// D2 digit fragments of the FP64 tensor-core path (largest lattice: 64)
alignas(16) uint32_t g_tab_oz[7 * 6 * 3 * 32 * 2 + 7 * 48 * 48 / 2];  // the largest table: N = 48

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int lise_rhs_noalloc(const lise_params* p, const double* psi_dev, double t, double* dpsi_dev) {
  if (!psi_dev || !dpsi_dev || !std::isfinite(t)) return LISE_EINVAL;
  if (check_params(p) != LISE_OK) return LISE_EINVAL;  // the same validation as lise_create
  if (p->device < 0 || p->device >= kMaxDevices) return LISE_EINVAL;
  const int N = p->nx;
  const long nxyz = (long)N * N * N;
  const long ns = (long)p->n_qp * 2 * nxyz;
  const bool mixed = p->precision != LISE_FP64;  // (one right-hand side: both mixed splits alike)
  // density groups: the rule of a context
  int qg = 0, n_groups = 0;
  choose_groups(N, p->n_qp, mixed, &qg, &n_groups);

  // carve the scratch array; reject problems that do not fit
  const size_t rs = mixed ? sizeof(float) : sizeof(double);
  size_t off = 0;
  const size_t o_txy = off;    off += up256((size_t)ns * 2 * rs);
  const size_t o_pn = off;     off += up256((size_t)n_groups * nxyz * sizeof(double));
  const size_t o_pr = off;     off += up256((size_t)n_groups * nxyz * sizeof(double));
  const size_t o_pi = off;     off += up256((size_t)n_groups * nxyz * sizeof(double));
  const size_t o_n = off;      off += up256((size_t)nxyz * sizeof(double));
  const size_t o_nu = off;     off += up256((size_t)nxyz * sizeof(double2));
  const size_t o_w = off;      off += up256((size_t)nxyz * sizeof(double));
  const size_t o_d = off;      off += up256((size_t)nxyz * sizeof(double2));
  const size_t o_v = off;      off += up256(p->v_static ? (size_t)nxyz * sizeof(double) : 0);
  const size_t o_tab = off;    off += up256(4 * (size_t)N * rs);
  const size_t o_err = off;    off += up256(sizeof(int));
  const bool use_oz = ozaki_path(N, mixed);
  const size_t oz_words = use_oz ? ozaki_table_words(N) : 0;
  const size_t o_oz = off;     off += up256(oz_words * sizeof(uint32_t));
  const int nbx = pencil_blocks_x(N, mixed);
  const size_t o_eta = off;    off += up256(p->remove_phase ? (size_t)p->n_qp * sizeof(double) : 0);
  const size_t o_etap = off;   off += up256(p->remove_phase ? (size_t)p->n_qp * nbx * sizeof(double) : 0);
  if (off > (size_t)LISE_NOALLOC_SCRATCH_BYTES) return LISE_ENOMEM;

  if (cudaSetDevice(p->device) != cudaSuccess) return LISE_ECUDA;
  // one-time set-up on this device: the device address of the scratch array
  if (!g_scratch_dev[p->device]) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_rhs_scratch) != cudaSuccess || !addr) return LISE_ECUDA;
    g_scratch_dev[p->device] = static_cast<unsigned char*>(addr);
  }
  unsigned char* base = g_scratch_dev[p->device];
  cudaStream_t s = (cudaStream_t)p->stream;

  // tables and the static potential into the scratch; the error word starts at zero
  void* tab_host;
  if (mixed) {
    fill_fft_tables(N, p->dx, p->alpha, 1, g_tab_f, g_tab_f + 2 * N, g_tab_f + 3 * N);
    tab_host = g_tab_f;
  } else {
    fill_fft_tables(N, p->dx, p->alpha, 0, g_tab_d, g_tab_d + 2 * N, g_tab_d + 3 * N);
    tab_host = g_tab_d;
  }
  if (cudaMemcpyAsync(base + o_tab, tab_host, 4 * (size_t)N * rs, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return LISE_ECUDA;
  if (p->v_static &&
      cudaMemcpyAsync(base + o_v, p->v_static, (size_t)nxyz * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return LISE_ECUDA;
  if (cudaMemsetAsync(base + o_err, 0, sizeof(int), s) != cudaSuccess) return LISE_ECUDA;
  int oz_sD = 0;
  if (use_oz) {
    if (oz_words > sizeof(g_tab_oz) / sizeof(uint32_t)) return LISE_EINVAL;
    oz_sD = ozaki_table(N, p->dx, p->alpha, g_tab_oz);
    if (cudaMemcpyAsync(base + o_oz, g_tab_oz, oz_words * sizeof(uint32_t), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return LISE_ECUDA;
  }
  const uint32_t* ozb = use_oz ? reinterpret_cast<const uint32_t*>(base + o_oz) : nullptr;

  const double2* x = reinterpret_cast<const double2*>(psi_dev);
  double* part_n = reinterpret_cast<double*>(base + o_pn);
  double* part_nr = reinterpret_cast<double*>(base + o_pr);
  double* part_ni = reinterpret_cast<double*>(base + o_pi);
  int* err = reinterpret_cast<int*>(base + o_err);
  const void* tw = base + o_tab;
  const void* hxy = base + o_tab + 2 * (size_t)N * rs;
  const void* hz = base + o_tab + 3 * (size_t)N * rs;

  // densities of psi -> U(n), Delta at t
  PointwiseArgs da;
  std::memset(&da, 0, sizeof(da));
  da.src = x;
  da.part_n = part_n;
  da.part_nr = part_nr;
  da.part_ni = part_ni;
  da.n_qp = p->n_qp;
  da.qg = qg;
  da.nxyz = nxyz;
  if (launch_density(da, s)) return LISE_ECUDA;
  ReduceArgs r;
  std::memset(&r, 0, sizeof(r));
  r.part_n = part_n;
  r.part_nr = part_nr;
  r.part_ni = part_ni;
  r.n_groups = n_groups;
  r.nxyz = nxyz;
  r.N = N;
  r.a = p->dx;
  r.n_out = reinterpret_cast<double*>(base + o_n);
  r.nu_out = reinterpret_cast<double2*>(base + o_nu);
  r.W = reinterpret_cast<double*>(base + o_w);
  r.D = reinterpret_cast<double2*>(base + o_d);
  r.v_static = p->v_static ? reinterpret_cast<const double*>(base + o_v) : nullptr;
  r.drive = p->drive_A == 0.0 ? 0.0 : p->drive_A * std::sin(p->drive_Omega * t);
  r.beta = p->beta;
  r.mu = p->mu;
  r.pair = make_pairing(p);
  r.err = err;
  if (launch_reduce(r, s)) return LISE_ECUDA;

  // T_xy psi, then z-pencils with the BdG apply: dpsi = -i H psi
  PlanesArgs pa;
  pa.x = x;
  pa.xr = nullptr;
  pa.txy = base + o_txy;
  pa.tw = tw;
  pa.hxy = hxy;
  pa.ozb = ozb;
  pa.oz_sD = oz_sD;
  pa.n_planes = (long)p->n_qp * 2 * N;
  pa.err = err;
  pa.wait_polls = 0;  // the default bound
  if (launch_planes(N, mixed, pa, s)) return LISE_ECUDA;
  PencilArgs ka;
  std::memset(&ka, 0, sizeof(ka));
  ka.x = x;
  ka.txy = base + o_txy;
  ka.W = r.W;
  ka.D = r.D;
  ka.tw = tw;
  ka.hz = hz;
  ka.ozb = ozb;
  ka.err = err;
  ka.oz_sD = oz_sD;
  ka.n_qp = p->n_qp;
  ka.qg = qg;
  ka.out = reinterpret_cast<double2*>(dpsi_dev);
  if (p->remove_phase) {  // eta_q = <psi_q|H psi_q> first, then -i (H - eta_q) psi_q
    PencilArgs ea = ka;
    ea.out = nullptr;
    ea.eta_part = reinterpret_cast<double*>(base + o_etap);
    if (launch_pencils(N, mixed, M_ETA, ea, s)) return LISE_ECUDA;
    if (launch_eta_reduce(ea.eta_part, p->n_qp, nbx, p->dx * p->dx * p->dx, reinterpret_cast<double*>(base + o_eta), s))
      return LISE_ECUDA;
    ka.eta = reinterpret_cast<const double*>(base + o_eta);
  }
  if (launch_pencils(N, mixed, M_RHS, ka, s)) return LISE_ECUDA;

  int h_err = 0;
  if (cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LISE_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return LISE_ECUDA;
  return h_err ? ((h_err & 4) ? LISE_ETIMEOUT : LISE_ENONFINITE) : LISE_OK;
}
