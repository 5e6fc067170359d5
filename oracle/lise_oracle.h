/*
 * lise_oracle.h -- FP64 CPU oracle for the two-component TDSLDA step.
 *
 * TEST INFRASTRUCTURE ONLY.  This plain, slow, deliberately unoptimised C
 * implementation exists to check the CUDA library against the paper.  Only the
 * test suite, the package smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, table or helper with the CUDA path.
 *
 * Method (arXiv:2009.00745, "LISE"):
 *   - lattice and momentum grid: Sec. "Discretization" (x_n = n a, k_n);
 *   - spectral derivatives: forward FFT unnormalised, inverse with 1/N,
 *     D^(2) f = F^-1[(ik)^2 F f] (Sec. "Discretization", FFT definitions);
 *   - quasiparticle equations i d(psi)/dt = H psi, H = [[h, Delta],[Delta*, -h*]]
 *     (Eq. tdslda, reduced to one (u, v) pair per state for spin-symmetric,
 *     spin-singlet pairing);
 *   - densities n = 2 sum_k |v_k|^2, nu = sum_k u_k v_k^* (Eqs. rho_t, nu_t);
 *   - potentials: h = -(alpha/2) lap + beta (3 pi^2 n)^(2/3)/2 - mu + V_ext,
 *     Delta = -g nu (Eq. pairingfield with a constant coupling; the unitary
 *     Fermi gas form of the SLDA);
 *   - time stepping: series-expansion predictor/corrector start (Sec. TDSLDA,
 *     "Time evolution", order-4 Taylor series with averaged densities) followed
 *     by the 5th-order Adams-Bashforth-Milne predictor-modifier-corrector
 *     (Eqs. p, m, c, y).
 *
 * Parity status of each function is given in its comment ("pinned by" names
 * the tests that tie it to something other than itself).
 *
 * All complex arrays are C99 double complex.  State layout (also the host
 * layout of the C ABI): psi[q][c][z][y][x], q < n_qp, c = 0 (u) or 1 (v),
 * x fastest.  Densities and potentials: [z][y][x].
 */
#ifndef LISE_ORACLE_H
#define LISE_ORACLE_H
#include <complex.h>
#include <stddef.h>

typedef struct {
  int nx, ny, nz;          /* periodic lattice */
  double a;                /* lattice constant dx = dy = dz = a */
  int n_qp;                /* number of (u, v) quasiparticle states */
  double alpha;            /* kinetic coefficient: h contains -(alpha/2) lap */
  double beta;             /* UFG coefficient: U = beta (3 pi^2 n)^(2/3) / 2 */
  double mu;               /* chemical potential (constant) */
  double g;                /* pairing coupling: Delta = -g nu */
  const double *v_static;  /* [nz][ny][nx] static external potential, or NULL */
  double drive_A;          /* V_ext += A sin(Omega t) z_c */
  double drive_Omega;
  int remove_phase;        /* 1: i dpsi_k/dt = (H - eta_k) psi_k, eta_k = <psi_k|H|psi_k> (Eq. sp_en) */
  double pair_alpha;       /* Eq. g0: g0(r) = g (1 - pair_alpha n(r) / pair_n0); 0 = constant g */
  double pair_n0;
  int pair_lattice;        /* 1: Eq. geff_3D, 1/g_eff = 1/g0(r) - meff (pi/a) K / (4 pi^2 hbar^2), meff = 1/alpha */
  int renormalize;         /* 1: at the end of every ABM step each state is scaled to a^3 sum(|u|^2+|v|^2) = 1
                              (the renormalisation remark that follows Eq. sp_en), before its y' is formed */
  double pair_ec;          /* > 0: Eq. geff, the spherical momentum cutoff at energy E_c (exclusive with
                              pair_lattice; 0 < E_c <= pi^2 / (2 meff a^2)); 0 = off */
} or_params;

/* K of Eq. geff_3D (the value printed with it). */
#define OR_GEFF_K 2.442749607806335

/* Effective coupling and its total density derivative at a site of density n whose local
 * potential (U(n) + V_ext, without -mu and without the pairing term) is u_loc:
 * g_eff = g0 / (1 - c g0) (the same as 1/g_eff = 1/g0 - c) with
 *   c = K / (4 pi a alpha)                       (pair_lattice, Eq. geff_3D),
 *   c = the spherical-cutoff term of Eq. geff    (pair_ec > 0; depends on u_loc),
 *   c = 0                                        (neither);
 * dgeff_dn = (dg0/dn) / (1 - c g0)^2 + g_eff^2 (dc/dU) (dU/dn), U(n) = beta (3 pi^2 n)^(2/3) / 2. */
void or_geff(const or_params *p, double n, double u_loc, double *geff, double *dgeff_dn);

/* 1D DFT of length n (any n >= 1), out-of-place, unnormalised.
 * sign = -1: sum_j x_j exp(-2 pi i j k / n); sign = +1: exp(+...). */
void or_dft1d(const double complex *in, double complex *out, int n, int sign);

/* 3D FFT in place.  sign = -1 forward (unnormalised); sign = +1 inverse,
 * including the 1/(nx ny nz) factor. */
void or_fft3d(double complex *vol, int nx, int ny, int nz, int sign);

/* k_n of Sec. "Discretization" along one axis of length n, spacing a. */
double or_kgrid(int idx, int n, double a);

/* T f = -(alpha/2) lap f = F^-1[(alpha/2) |k|^2 F f]  (Nyquist mode kept). */
void or_kinetic(const or_params *p, const double complex *in, double complex *out);

/* n(r) = 2 sum_k |v_k|^2, nu(r) = sum_k u_k v_k^*, compensated sums in qp order. */
void or_densities(const or_params *p, const double complex *psi, double *n,
                  double complex *nu);

/* V_ext(r, t) = v_static(r) + A sin(Omega t) (i_z - nz/2) a (z measured from the box
 * centre).  Pinned by tests/test_oracle_drive.py: with alpha = beta = g = 0 every site
 * rotates by the exact phase int (V_ext - mu) dt, which fixes the origin of z, the drive's
 * form and the times at which the integrator evaluates it (t_{n+1} for both right-hand
 * sides of an ABM step, t + dt/2 for the series start's corrector Hamiltonian). */
double or_vext(const or_params *p, int ix, int iy, int iz, double t);

/* W(r) = beta (3 pi^2 n)^(2/3)/2 + (d g_eff/dn) |nu|^2 - mu + V_ext(r, t) (the diagonal
 * of h besides T; the middle term is dE_pair/dn and vanishes for a constant
 * coupling); Delta(r) = -g_eff(n(r)) nu(r). */
void or_potentials(const or_params *p, const double *n, const double complex *nu,
                   double t, double *W, double complex *Delta);

/* hpsi = H psi with H = [[h, Delta],[Delta*, -h*]], h = T + W;
 * -h* v is formed literally as -conj(h conj(v)). */
void or_apply_h(const or_params *p, const double *W, const double complex *Delta,
                const double complex *psi, double complex *hpsi);

/* eta_k = <psi_k|hpsi_k> = a^3 sum_r [conj(u) (H psi)_u + conj(v) (H psi)_v], real part
 * (H is Hermitian), compensated sums; eta has n_qp entries. */
void or_eta(const or_params *p, const double complex *psi, const double complex *hpsi, double *eta);

/* dpsi = f(t, psi) = -i H[psi](t) psi (potentials from the densities of psi);
 * with remove_phase, -i (H - eta_k) psi_k. */
void or_rhs(const or_params *p, const double complex *psi, double t,
            double complex *dpsi);

/* Integrator (opaque). */
typedef struct or_solver or_solver;
or_solver *or_create(const or_params *p);
void or_destroy(or_solver *s);
/* Copies psi (host layout above) as y_0 at time t0, then runs the
 * series-expansion start (3 steps) and fills the ABM history. */
int or_set_state(or_solver *s, const double complex *psi, double t0, double dt);
/* n_steps ABM steps of size dt (must equal the set_state dt). */
int or_step(or_solver *s, int n_steps);
/* Loads an ABM history directly instead of running the series start, so that the
 * steps of Eqs. p, m, c, y can be tested on their own: y_n = yn, y_{n-1} = ynm1,
 * y'_{n-k} = d[k] (k = 0..3), p_n - c_n = pc (NULL: zero), current time t_n = t,
 * step dt (non-zero).  Copies every array. */
int or_set_history(or_solver *s, const double complex *yn, const double complex *ynm1,
                   const double complex *d0, const double complex *d1, const double complex *d2,
                   const double complex *d3, const double complex *pc, double t, double dt);
/* First derivative along axis (0 = x, 1 = y, 2 = z): F^-1[(ik) F f] with the
 * Nyquist coefficient set to zero (Sec. "Discretization", odd derivatives). */
void or_gradient(const or_params *p, const double complex *in, int axis, double complex *out);
/* Current density of Eq. j for the two-component states (spin factor 2):
 * j(r) = 2 sum_k Im(v_k grad v_k^*) = -2 sum_k Im(v_k^* grad v_k); j[3][z][y][x] (x, y, z). */
void or_currents(const or_params *p, const double complex *psi, double *j);
/* Eq. kick (Sec. "External boosts and external potentials"): u -> e^{i chi(r)} u,
 * v -> e^{-i chi(r)} v for every state, chi real [z][y][x]. */
void or_kick(const or_params *p, double complex *psi, const double *chi);
/* Kick the solver's current state and restart the history through the series
 * start at the current time with the current step (as after a set_state). */
int or_solver_kick(or_solver *s, const double *chi);
void or_get_state(const or_solver *s, double complex *psi_out);
double or_time(const or_solver *s);
void or_get_densities(const or_solver *s, double *n, double complex *nu);
/* E = a^3 sum_r [(alpha/2) tau + (3/10) beta (3 pi^2)^(2/3) n^(5/3) + g_eff(n) |nu|^2
 *     + V_ext n],  tau = 2 sum_k |grad v_k|^2 (spectral);  N = a^3 sum_r n.
 * The pairing term has the sign of Eq. pairing (E_pair = g_eff |kappa|^2 with
 * Delta = -g_eff kappa); U = dE/dn gives the beta term of h. */
void or_energy(const or_solver *s, double *E, double *N);
/* Same quantities for an arbitrary state at time t. */
void or_energy_of(const or_params *p, const double complex *psi, double t,
                  double *E, double *N);

/* One series-expansion start step (Sec. TDSLDA, "Time evolution"), exposed for
 * the order tests: psi_out = psi(t + dt). */
void or_series_step(const or_params *p, const double complex *psi, double t,
                    double dt, double complex *psi_out);

/* The four update formulas of the Adams-Bashforth-Milne step, elementwise over
 * ns complex values (Eqs. p, m, c, y); the integrator uses exactly these. */
void or_abm_predictor(long ns, double h, const double complex *yn, const double complex *ynm1,
                      const double complex *d0, const double complex *d1,
                      const double complex *d2, const double complex *d3, double complex *p);
void or_abm_modifier(long ns, const double complex *p, const double complex *pc,
                     double complex *m);
void or_abm_corrector(long ns, double h, const double complex *yn, const double complex *ynm1,
                      const double complex *mp, const double complex *d0,
                      const double complex *d1, const double complex *d2, double complex *c);
void or_abm_final(long ns, const double complex *p, const double complex *c, double complex *y,
                  double complex *pc);

/* Number of OpenMP threads the oracle runs with (1 if built without OpenMP). */
int or_num_threads(void);

#endif
