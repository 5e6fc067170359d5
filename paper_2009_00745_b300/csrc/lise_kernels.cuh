// lise_kernels.cuh -- device kernels of the two-component TDSLDA step.
//
// Operator split used on the device (exact in exact arithmetic):
//   T psi = -(alpha/2) lap psi = T_xy psi + T_z psi,
//   T_xy = F_xy^-1 [(alpha/2)(kx^2 + ky^2) F_xy],  T_z = F_z^-1 [(alpha/2) kz^2 F_z],
// which equals F^-1[(alpha/2)|k|^2 F] of Sec. "Discretization" because F_z
// commutes with the in-plane multiplier.  Kernel "planes" applies T_xy to every
// xy-plane of every (state, component) and writes it to a scratch array;
// kernel "pencils" applies T_z to z-pencils, adds the scratch, forms
//   H psi = [[h, Delta],[Delta*, -h*]] psi,  h = T + W   (Eq. tdslda),
// and finishes with a fused, mode-dependent epilogue (the ABM formulas of
// Eqs. p, m, c, y, the order-4 series terms of the start procedure, or a plain
// right-hand side) plus per-group partial sums of the densities
// n = 2 sum |v|^2 and nu = sum u v^* (Eqs. rho_t, nu_t).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lise_fft.cuh"

namespace lise {

// Bounded waits on the hardware (tensor-core completion, tensor-memory-accelerator copies):
// polls before a wait gives up.  The drain waits that let work already in flight finish
// before a block frees its tensor memory or exits always use kDrainPolls.
constexpr long kDefaultWaitPolls = 1L << 22;
constexpr long kDrainPolls = 1L << 22;
__host__ __device__ inline long wait_limit(long wait_polls) {
  return wait_polls == 0 ? kDefaultWaitPolls : (wait_polls < 0 ? 0L : wait_polls);
}

enum PencilMode : int {
  M_RHS = 0,            // out = -i H x
  M_TAYLOR_FIRST = 1,   // h = H x; [dslot = -i h]; term = coef h -> out; acc = x + term
  M_TAYLOR = 2,         // term = coef H x -> out (in place); acc += term; [densities of acc]
  M_CORRECT = 3,        // m' = -i H m; Eq. c and Eq. y through Q, R -> ynew, pc; densities of ynew
  M_DERIV_PREDICT = 4,  // d = -i H y_{n+1} -> dslot; Eq. p, Eq. m of the next step -> m, and
                        // the corrector's precombined Q, R; densities of m
  M_ENERGY = 5,         // part_n += sum_q 2 Re(conj(v) T v)
  M_ETA = 6,            // eta_part[q][block] = sum over the block's sites of Re(conj(x) . H x)
};

struct PencilArgs {
  const double2* x;       // operand state [q][c][z][y][x] (complex128), unless xr is set
  const void* xr;         // if non-null: the operand stored in the compute precision
                          // (the modifier m of the mixed path); x is then unused
  const void* txy;        // T_xy x, complex of the compute precision
  const double* W;        // h - T = U(n) - mu + V_ext  [site]
  const double2* D;       // Delta [site]
  const void* tw;         // forward twiddles of the compute precision, N entries
  const void* hz;         // (alpha/2) kz^2 / N, N entries, compute precision
  const uint32_t* ozb;    // FP64 tensor-core path: digit fragments of D2 (lise_ozaki.cuh)
  int oz_sD;              //   and their scale exponent
  int n_qp;
  int qg;                 // states per density group (one grid row per group)
  double2* out;           // complex128 output (M_RHS, Taylor terms); may be null in M_RHS
  double2* acc;
  void* dslot;            // y' ring slot, compute precision (M_RHS, M_TAYLOR_FIRST, M_DERIV_PREDICT)
  double2 coef;
  double h;               // time step
  const double2* y0;      // y_n
  const double2* y1;      // y_{n-1} (M_CORRECT)
  const void* d0;         // y'_n      (compute precision, like every y' slot)
  const void* d1;         // y'_{n-1}
  const void* d2;         // y'_{n-2}
  double2* q;             // Q, complex128 (read in M_CORRECT, written in M_DERIV_PREDICT), see below
  void* r;                // R, compute precision (likewise)
  void* pc;               // p - c, compute precision (written in M_CORRECT, read in M_DERIV_PREDICT)
  void* m;                // m in the compute precision (written in M_DERIV_PREDICT)
  double2* ynew;          // y_{n+1} (written in M_CORRECT; may alias y1)
  double* part_n;         // [group][site] partial sums
  double* part_nr;
  double* part_ni;
  int dens;               // accumulate density partials of the mode's output state
  const double* eta;      // if non-null: apply H - eta_q (trivial-phase removal), eta per state
  double* eta_part;       // M_ETA output: [state][block] partial sums
  int* err;               // device error word: bit 4 set when a bounded wait ran out
  long wait_polls;        // bounded waits: 0 = kDefaultWaitPolls, < 0 = give up at once, else polls
  int strict;             // FP32 compute precision: the strict split (LISE_MIXED_STRICT), R and
                          // p - c in complex128 (units of h/48), the corrector's update in FP64
  // FP32 compute precision: tensor maps of the batch staging copies (operand, T_xy, and the
  // corrector's Q and R), written by launch_pencils from the pointers above
  CUtensorMap tm_x;
  CUtensorMap tm_t;
  CUtensorMap tm_q;
  CUtensorMap tm_r;
};

struct PlanesArgs {
  const double2* x;       // operand state, n_planes consecutive N x N planes (complex128)
  const void* xr;         // or, if non-null, the operand in the compute precision
  void* txy;              // output T_xy x
  const void* tw;         // forward twiddles, N entries
  const void* hxy;        // (alpha/2) k^2 / N^2, N entries
  const uint32_t* ozb;    // FP64 tensor-core path: digit fragments of D2 (lise_ozaki.cuh)
  int oz_sD;
  long n_planes;
  int* err;               // device error word: bit 4 set when a bounded wait ran out
  long wait_polls;        // as in PencilArgs
};

// Pairing coupling of Eqs. g0, geff_3D and geff (hbar = 1), built once from the parameters.
struct Pairing {
  double g;         // bare coupling: Delta = -g_eff nu
  double alpha_n0;  // Eq. g0: g0 = g (1 - alpha_n0 n), alpha_n0 = pair_alpha / pair_n0
  double c;         // Eq. geff_3D: 1/g_eff = 1/g0 - c; 0 without the lattice form
  double ec;        // Eq. geff: spherical momentum cutoff at energy E_c > 0; 0 = off
  double m;         // m* = 1/alpha (dispersion alpha k^2 / 2), for Eq. geff
  double mu;        // chemical potential, for Eq. geff
  double beta;      // U(n) = beta (3 pi^2 n)^(2/3) / 2, whose n-dependence enters d g_eff / dn
};

struct ReduceArgs {
  const double* part_n;
  const double* part_nr;
  const double* part_ni;
  int n_groups;
  long nxyz;
  int N;
  double a;
  double* n_out;          // densities of this reduction [site]
  double2* nu_out;
  const double* avg_n;    // if non-null: n <- (n + avg_n)/2, nu likewise (start corrector)
  const double2* avg_nu;
  double* W;              // potentials out
  double2* D;
  const double* v_static; // may be null
  double drive;           // A sin(Omega t)
  const double* drive_ptr;  // if non-null, the drive amplitude is read from here (graph replays)
  double beta, mu;
  Pairing pair;
  int* err;               // set bit 0 if a density is not finite
};

// Batched launches (lise_batch_*): the arguments of several evolutions and a work table mapping
// each block (row) to an evolution.  The pencils and planes launches carry up to kBatchInline
// evolutions' arguments in their kernel parameters (constant-bank reads, and the pencils
// kernel's tensor maps in parameter space, as in the per-context launches; larger groups take
// several launches); the reduction and predictor launches read theirs from device memory.
constexpr int kBatchInline = 16;
struct PencilBatch {
  PencilArgs evo[kBatchInline];  // per evolution (tensor maps of the staged FP32 path included)
  const int2* items;             // block row -> (index into evo, density group of that evolution)
};
struct PlanesBatch {
  PlanesArgs seg[kBatchInline];  // per evolution
  long block0[kBatchInline + 1]; // first block of each segment, n_seg + 1 entries
  int n_seg;
};
struct ReduceBatch {
  const ReduceArgs* evo;   // per evolution
  const long* block0;      // first block of each evolution, n + 1 entries
  int n;
};

// Effective pairing coupling g_eff and its total density derivative at a site of density n,
// cb2 = (3 pi^2 n)^(2/3), local potential u_loc = U(n) + V_ext (Eqs. g0, geff_3D, geff):
// 1/g_eff = 1/g0 - c.  The spherical-cutoff term of Eq. geff, with s = k_F^2 = 2 m* (mu - u_loc)
// and k_c^2 = s + 2 m* E_c, is the single analytic function
//   c = m* k_c / (2 pi^2) (1 - z A(z)),  z = s / k_c^2 < 1,
//   A(z) = artanh(sqrt z) / sqrt z (z > 0),  arctan(sqrt -z) / sqrt -z (z < 0),  1 (z = 0),
// which is the equation's logarithmic form for k_F^2 > 0 and its arctan form for k_F^2 < 0; its
// derivative is dc/du_loc = m*^2 A(z) / (2 pi^2 k_c).  c = 0 where k_c^2 <= 0 (no momenta below
// the cutoff).  d g_eff/dn = (dg0/dn) / (1 - c g0)^2 + g_eff^2 (dc/du_loc) dU/dn,
// dU/dn = beta cb2 / (3 n) (0 at n = 0).
__host__ __device__ inline void pairing_geff(const Pairing& P, double n, double cb2, double u_loc, double* geff,
                                             double* dgeff) {
  const double g0 = P.g * (1.0 - P.alpha_n0 * n);
  double c = P.c, dc = 0.0;
  if (P.ec > 0.0) {
    const double s = 2.0 * P.m * (P.mu - u_loc), kc2 = s + 2.0 * P.m * P.ec;
    c = 0.0;
    if (kc2 > 0.0) {
      const double kc = sqrt(kc2), z = s / kc2;
      double A = 1.0;
      if (z > 0.0) {
        const double r = sqrt(z);
        A = atanh(r) / r;
      } else if (z < 0.0) {
        const double r = sqrt(-z);
        A = atan(r) / r;
      }
      const double k2pi2 = 1.0 / (2.0 * 3.14159265358979323846 * 3.14159265358979323846);
      c = P.m * kc * k2pi2 * (1.0 - z * A);
      dc = P.m * P.m * A * k2pi2 / kc;
    }
  }
  const double den = 1.0 - c * g0;
  const double ge = g0 / den;
  *geff = ge;
  *dgeff = (-P.g * P.alpha_n0) / (den * den) + (n > 0.0 ? ge * ge * dc * (P.beta * cb2 / (3.0 * n)) : 0.0);
}

struct PointwiseArgs {
  // predictor + modifier: p = Eq. p, m = Eq. m, and the corrector's Q, R
  const double2 *y0, *y1;  // complex128 states
  const void *d0, *d1, *d2, *d3, *pc;  // compute precision
  double2* q;              // complex128
  void* r;                 // compute precision
  void* m;                 // m in the compute precision of the path
  int mixed;
  int strict;              // mixed only: the strict split (k_predict's ST)
  double h;
  // density partials of `src` (for the plain density pass) or of m
  const double2* src;
  double* part_n;
  double* part_nr;
  double* part_ni;
  int n_qp, qg;
  long nxyz;
};

struct PredictBatch {
  const PointwiseArgs* evo;  // per evolution
  const int2* items;         // block row -> (evolution, density group)
};

// The corrector of Eq. c splits as c_{n+1} = cbase_{n+1} + (17 h/48) m'_{n+1} with
//   cbase_{n+1} = (y_n + y_{n-1})/2 + h/48 (51 y'_n + 3 y'_{n-1} + y'_{n-2}),
// which depends only on the history known at predictor time.  With
//   Q = (161/170) cbase + (9/170) p_{n+1},   R = p_{n+1} - cbase,
// Eq. y becomes y_{n+1} = Q + (161/170)(17 h/48) m'_{n+1} and
// p_{n+1} - c_{n+1} = R - (17 h/48) m'_{n+1} (algebraically identical to Eqs. c, y).
// Q and R are formed with the predictor, so the corrector reads 2 arrays, not 6.
//
// Storage precision of the history.  y_n, y_{n-1} and Q are states (complex128).
// The derivatives y', R = pt - ct and p - c are formed in the compute precision
// (FP32 in the mixed path: the FFT/BdG apply and the derivative combinations run
// there), so they are stored in it: exactly, without rounding.  Every sum with a
// state value runs in FP64.

// Host-side launchers (defined in lise_kernels.cu).
// pb: planes per block of the FFT planes kernel (0 = the tuned value, else the default)
int launch_planes(int N, int mixed, const PlanesArgs& a, cudaStream_t s, int pb = 0);
// Planes-per-block autotuning state of the FFT planes kernel (per process): tuned value per
// (precision, N), 0 = none; the value in use; whether a variant is compiled.  pb > 0: the
// shared-memory line FFTs with pb planes per block; pb < 0: the register-line variant with
// -pb planes per block (FP32 compute precision, N <= 48).  All give bitwise the same result.
int planes_pb_get(int N, int mixed);
void planes_pb_set(int N, int mixed, int pb);
int planes_pb(int N, int mixed);
bool planes_pb_valid(int N, int mixed, int pb);
// qb: states per batch of the step modes (2 or 4 where compiled); 0 = the tuned value,
// else the default for the lattice and precision
int launch_pencils(int N, int mixed, int mode, const PencilArgs& a, cudaStream_t s, int qb = 0);
// Pencil batch autotuning state (per process): tuned QB per (precision, N), 0 = none.
int pencil_qb_get(int N, int mixed);
void pencil_qb_set(int N, int mixed, int qb);
bool pencil_qb_valid(int N, int mixed, int qb);
int launch_reduce(const ReduceArgs& a, cudaStream_t s);
// Batched launches of the FP32 compute precision (lise_batch_*): one launch over several
// evolutions of lattice N (items / segments / blocks as in the batch structs); qb: the
// pencils batch size (2 or 4, the one the evolutions' tensor maps were encoded for).
int launch_pencils_batch(int N, int mode, int strict, const PencilBatch& b, int n_items, int qb, cudaStream_t s);
int launch_planes_batch(int N, int pb, const PlanesBatch& b, long n_blocks, cudaStream_t s);
long planes_blocks(long n_planes, int pb);  // blocks of the FFT planes kernel: |pb| planes per block
int launch_reduce_batch(const ReduceBatch& b, long n_blocks, cudaStream_t s);
int launch_predict_batch(int strict, const PredictBatch& b, long nxyz, int n_items, cudaStream_t s);
// Tensor maps of one evolution's staged pencils launch (FP32 compute precision) written
// into a->tm_* from its array pointers; false if the encoding fails.
bool pencils_batch_maps(int N, int mode, int strict, int qb, PencilArgs* a);
int launch_predict(const PointwiseArgs& a, cudaStream_t s);
int launch_density(const PointwiseArgs& a, cudaStream_t s);
int launch_energy_sites(const double* part_ekin, int n_groups, const double* n, const double2* nu,
                        const double* v_static, double drive, const Pairing& pair, int N, double a,
                        double* e_site, cudaStream_t s);
// pair_c of Eq. geff_3D for lattice constant a and kinetic coefficient alpha (meff = 1/alpha).
double pairing_lattice_c(double a, double alpha);
int launch_finite_check(const double2* x, long count, int* err, cudaStream_t s);
// Per-step renormalisation: norm partials [q][block] of a^3 sum(|u|^2 + |v|^2) over nb
// blocks per state, then scale[q] = 1 / sqrt(sum over blocks in order); then y *= scale
// in place with the density partials of the scaled state (groups of qg states).
int launch_norms(const double2* y, int n_qp, long nxyz, double a3, int nb, double* part, double* scale,
                 cudaStream_t s);
int launch_scale_density(double2* y, const double* scale, const PointwiseArgs& a, cudaStream_t s);
// Current density of Eq. j: per state group g, jx/jy/jz partial sums [g][site] of
// -2 Im(conj(v) D1 v) along each axis; d1 = first-derivative circulant (N entries,
// Nyquist coefficient dropped).  Then out[3][site] = sums over groups in group order.
int launch_currents(const double2* psi, const double* d1, int N, int n_qp, int qg, double* jx, double* jy,
                    double* jz, cudaStream_t s);
int launch_sum_groups3(const double* jx, const double* jy, const double* jz, int n_groups, long nxyz, double* out,
                       cudaStream_t s);
// d1[m] = (1/N) sum_j (i k_j) e^{i k_j m a} over j != N/2 (real), m = 0..N-1.
void first_derivative_table(int N, double a, double* d1);
// dst = Eq. kick of src: u e^{i chi}, v e^{-i chi} for n_qp states of nxyz sites (dst may alias src).
int launch_kick(const double2* src, double2* dst, const double* chi, int n_qp, long nxyz, cudaStream_t s);
// eta[q] = a^3 * sum over the pencil blocks of eta_part[q][block] (compensated).
int launch_eta_reduce(const double* eta_part, int n_qp, int n_blocks, double a3, double* eta, cudaStream_t s);
int pencil_blocks_x(int N, int mixed);
// FP64 kinetic operator on the tensor cores (lise_ozaki.cuh): used for the FP64
// path on lattices with N a multiple of 16.  The table holds the D2 digit
// fragments (ozaki_table_words(N) uint32 words); ozaki_table returns its scale
// exponent sD (D2 ~ I_D 2^sD).
bool ozaki_path(int N, int mixed);
size_t ozaki_table_words(int N);
int ozaki_table(int N, double a, double alpha, uint32_t* out);
// Tile width (x values per pencil block) and group width for a lattice.
int pencil_tx(int N, int mixed);
int pencil_qb(int N, int mixed);
bool supported_n(int N);
// Density groups of a context (and of the no-allocation right-hand side): at most 64 states
// per group, fewer while the pencils grid would have fewer than 2048 blocks.
void choose_groups(int N, int n_qp, int mixed, int* qg, int* n_groups);
// Host tables of the FFT kernels for lattice N, spacing a: twiddles tw[2 N]
// (tw[j2 N1 + k1] = exp(-2 pi i j2 k1 / N) of the four-step plan, re/im interleaved) and the
// kinetic factors hxy[k] = (alpha/2) k^2 / N^2, hz[k] = (alpha/2) k^2 / N (Sec.
// "Discretization" k grid), in the compute precision (float if mixed); no heap use.
void fill_fft_tables(int N, double a, double alpha, int mixed, void* tw, void* hxy, void* hz);

}  // namespace lise
