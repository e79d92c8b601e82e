/*
 * nbref — CPU oracle for the hybrid symplectic planet-formation step.
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, FP64 restatement of the
 * method (Grimm & Stadel, "Terrestrial planet formation in the era of GPU
 * computing", section "The hybrid symplectic integrator", Eqs. H, Ha, Hb, Hc
 * and rcrit). Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it. It shares no source with the CUDA library.
 *
 * Units: AU, day, solar mass. The star is implicit (mass m0); bodies carry
 * heliocentric positions x and barycentric velocities v (democratic
 * heliocentric coordinates, section "The hybrid symplectic integrator").
 *
 * All arrays are host memory. x and v are interleaved [n][3]. Return codes:
 * 0 ok, -1 invalid argument, -4 iteration cap reached (no convergence).
 */
#ifndef NBREF_H
#define NBREF_H

#ifdef __cplusplus
extern "C" {
#endif

#define NBREF_OK 0
#define NBREF_E_INVALID (-1)
#define NBREF_E_NOCONV (-4)

typedef struct {
  double G;            /* gravitational constant, AU^3 Msun^-1 day^-2 */
  double m0;           /* central mass */
  double dt_rcrit;     /* time step that enters the velocity term of Eq. rcrit */
  double hill_factor;  /* 3 in Eq. rcrit */
  double vel_factor;   /* 0.4 in Eq. rcrit */
  int vel_mode;        /* 0: speed relative to the local circular orbit; 1: |v| */
  int merge;           /* 1: perfect merging on contact */
  double bs_tol;       /* Bulirsch-Stoer relative tolerance */
  int bs_kmax;         /* extrapolation columns (substep sequence n_k = 2k) */
  int bs_max_halvings; /* cap on substep halvings inside one step */
  int kepler_max_iter; /* cap on Kepler-equation iterations */
  int rcrit_refresh;   /* 0: r_crit at start and for merged survivors; 1: every step (see step) */
  /* Gas drag, applied with the implicit midpoint method of Eq. implicit (see step). */
  int gas;             /* 1: gas drag on */
  double gas_rho0;     /* midplane gas density at 1 AU, Msun / AU^3 */
  double gas_p;        /* density power law rho = rho0 (s / 1 AU)^-p, s = cylindrical radius */
  double gas_eta;      /* gas rotates at (1 - eta) times the circular speed */
  double gas_cd;       /* drag coefficient C_D */
  int gas_iter;        /* cap on implicit-midpoint iterations */
  double eject_r;      /* bodies beyond this heliocentric distance are removed; 0 = never */
  /* Multi-level changeover (section "Increasing N"): ml_levels intermediate
   * levels between the step and the direct solver; level l uses critical
   * radii r_crit / ml_factor^l and steps dt / ml_factor^l. 0 = groups go to
   * the direct solver at once. */
  int ml_levels;
  int ml_factor;
} nbref_params;

typedef struct {
  long long steps;          /* integrator steps taken */
  long long force_evals;    /* full O(N^2) force evaluations */
  long long encounter_pairs;/* sum over steps of |E| */
  long long groups;         /* close-encounter groups integrated */
  long long bs_substeps;    /* accepted BS substeps */
  long long bs_halvings;    /* substep halvings */
  long long bs_derivs;      /* right-hand-side evaluations inside BS */
  long long merges;         /* perfect mergers */
  long long kepler_iters;   /* Kepler iterations summed over bodies and steps */
  long long ejections;      /* bodies removed beyond eject_r */
  double m_ejected;         /* their mass */
  long long ml_substeps;    /* substeps taken on the intermediate changeover levels */
  long long ml_groups;      /* groups formed on the intermediate levels */
} nbref_stats;

typedef struct nbref_system nbref_system;

void nbref_default_params(nbref_params* p);

/* Smooth changeover K(r) and dK/dr for a pair with critical radius rc. */
void nbref_changeover(double r, double rc, double* K, double* dKdr);

/* Stumpff functions c0..c3 at argument z. */
void nbref_stumpff(double z, double c[4]);

/* Kepler drift of one body about mass parameter mu by time h (in place).
 * Returns 0 or NBREF_E_NOCONV; *iters receives the iteration count. */
int nbref_kepler_drift(double mu, double x[3], double v[3], double h, int max_iter, int* iters);

/* Gauss f, g, fdot, gdot for the same drift (diagnostic entry). */
int nbref_kepler_fg(double mu, const double x[3], const double v[3], double h, int max_iter,
                    double fg[4]);

/* Critical radius of one body, Eq. rcrit under the stated velocity reading. */
double nbref_rcrit(const nbref_params* p, const double x[3], const double v[3], double m);

/* Kick accelerations (Eq. Hb gradient) and the close-pair flags of n bodies.
 * a receives [n][3]; pairs receives (i, j) index pairs with i < j, sorted,
 * up to cap pairs; *npairs is the total found. Returns 0. */
int nbref_forces(int n, const double* x, const double* m, const double* rc, double G,
                 double* a, int* pairs, int cap, int* npairs);

/* Kick acceleration of the listed targets (a: [nt][3]) and the flagged pairs
 * that involve a listed target, sorted unique (min, max) index pairs. */
int nbref_forces_targets(int n, const double* x, const double* m, const double* rc, double G,
                         const int* targets, int nt, double* a, int* pairs, int cap,
                         int* npairs);

/* Integrate the H_A flow restricted to a group of n bodies over h with the
 * Gragg-Bulirsch-Stoer method and perfect merging. Arrays are updated in
 * place; alive[k] = 0 marks a body absorbed by a merger. */
int nbref_bs_group(const nbref_params* p, int n, double* x, double* v, double* m, double* R,
                   double* rc, int* alive, double h, double* E_lost, nbref_stats* st);

nbref_system* nbref_create(const nbref_params* p, int n, const double* x, const double* v,
                           const double* m, const double* R, const double* rc_override,
                           const int* ids, int* status);
int nbref_step(nbref_system* s, int nsteps, double dt);
int nbref_energy_momentum(const nbref_system* s, double* E, double L[3], double P[3],
                          double* E_lost);
int nbref_n_active(const nbref_system* s);
int nbref_get_state(const nbref_system* s, double* x, double* v, double* m, double* R,
                    double* rc, int* ids, int* n_active);
int nbref_get_accel(const nbref_system* s, double* a);
/* Encounter pairs of the last nbref_step call as (step, id_i, id_j) triples,
 * sorted by step then ids. *count receives the total; at most cap written. */
int nbref_encounter_list(const nbref_system* s, int* step_ij, int cap, int* count);
int nbref_stats_get(const nbref_system* s, nbref_stats* st);
long long nbref_step_index(const nbref_system* s);
void nbref_destroy(nbref_system* s);

/* Host threads of the OpenMP loops (over target bodies only, so results do
 * not depend on it); n < 1 means 1. Used to time the oracle on 1 and on all
 * cores in one process. */
void nbref_set_threads(int n);

/* One close-encounter group over h by the multi-level changeover
 * (ml_levels levels; the direct solver of nbref_bs_group when 0). Arguments
 * as nbref_bs_group. */
int nbref_ml_group(const nbref_params* p, int n, double* x, double* v, double* m, double* R,
                   double* rc, int* alive, double h, double* E_lost, nbref_stats* st);

/* One body's gas-drag update by the implicit midpoint method (Eq. implicit):
 * vout = v + tau a_f(x, (v + vout) / 2); Pm0 = P / m0 (the star's velocity
 * is -Pm0). Returns 0 or NBREF_E_NOCONV after gas_iter iterations. */
int nbref_implicit_drag(const nbref_params* p, const double x[3], const double v[3],
                        const double Pm0[3], double m, double R, double tau, double vout[3]);

#ifdef __cplusplus
}
#endif
#endif
