/*
 * eslbm_oracle.h -- plain FP64 CPU oracle for the fourth-order entropy-stable
 * vectorial lattice Boltzmann scheme of Bellotti, Helluy and Navoret,
 * "Fourth-order entropy-stable lattice Boltzmann schemes for hyperbolic
 * systems" (arXiv 2403.13406).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, literal reference that
 * the CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and
 * the cpu_baseline / reference legs of bench.py may load it.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * Every routine applies the paper's operators literally, in double precision:
 * one unit shift at a time for the transport (eq. transportPhase), one
 * relaxation sweep per R (eq. relaxationDiscretizationOmega), the basic brick
 * of eq. basicBrickSplitting composed as in eq. splittingToUse, and a
 * dichotomy for the entropic relaxation parameter (eq. variableOmegaProblem,
 * Section 5.1).
 *
 * Layout: f[(k*M + m)*ncell + cell], cell = y*nx + x (x fastest); k indexes
 * the velocities in the paper's order (D1Q2: +V, -V; D2Q4: (+V,0), (0,+V),
 * (-V,0), (0,-V), Section 1.2.2), m the conserved component.
 */
#ifndef ESLBM_ORACLE_H
#define ESLBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_LINEAR = 0, OR_BURGERS = 1, OR_SW = 2, OR_EULER = 3 };
enum { OR_OMEGA_FIXED = 0, OR_OMEGA_ENTROPIC = 1 };
/* which relaxation a stage applies: the scheme's main one (fixed omega or
   entropic omega), or the projection on the equilibrium R_1 (Section 6.1) */
enum { OR_R_MAIN = 0, OR_R_PROJECT = 1 };
/* composite schemes: I-IV of Section 6.1, the standard second-order lattice
   Boltzmann scheme R T(kappa dx / V) of Section 2.1 (one stage per step; 24
   of its steps span one composite step, Section 3.1), and scheme (B) of
   Section 6.3 */
enum { OR_SCHEME_I = 1, OR_SCHEME_II = 2, OR_SCHEME_III = 3, OR_SCHEME_IV = 4,
       OR_SCHEME_PLAIN = 5, OR_SCHEME_B = 6 };

typedef struct {
    int dim;          /* 1 -> D1Q2, 2 -> D2Q4 */
    int system;       /* OR_LINEAR, OR_BURGERS, OR_SW */
    long nx, ny;      /* ny = 1 for dim = 1 */
    int kappa;        /* shift unit, V dt / (24 dx) (kappa = 1 in the paper) */
    double V;         /* lattice velocity */
    double a[2];      /* linear transport velocity a (x, y) */
    double c[2];      /* Burgers flux coefficients: phi^j = c_j u^2 / 2 */
    double g;         /* gravity (shallow water) */
    int omega_mode;   /* OR_OMEGA_FIXED or OR_OMEGA_ENTROPIC */
    double omega;     /* relaxation parameter in fixed mode */
    double t_max;     /* entropic mode: search omega - 1 in [0, t_max] */
    double gamma;     /* Euler: ratio of specific heats (fixed omega only; no kinetic entropy) */
} or_model;

typedef struct {
    long relaxations;   /* cell relaxations performed */
    long fallbacks;     /* entropic mode: cells where no root existed (omega = 1 used) */
    double omega_min, omega_max;
} or_stats;

int or_q(const or_model *m);
int or_M(const or_model *m);
long or_ncell(const or_model *m);
/* 0 if the model is well formed, -1 otherwise */
int or_check(const or_model *m);

/* --- per-cell physics and kinetic quantities (Sections 1.1-1.2) --- */
void or_flux(const or_model *m, int j, const double *u, double *phi);
double or_entropy_S(const or_model *m, const double *u);
void or_dual(const or_model *m, const double *u, double *p);
void or_equilibrium(const or_model *m, const double *u, double *feq /* q*M */);
/* dual kinetic entropy s*_k(p), its gradient and Hessian (M x M, row-major) */
double or_kinetic_dual(const or_model *m, int k, const double *p, double *grad, double *hess);
/* kinetic entropy s_k(f_k); p_hint = dual of the cell's conserved moments */
double or_kinetic_entropy(const or_model *m, int k, const double *fk, const double *p_hint);
/* Bregman divergence B_k(h) = s_k(feq_k + h) - s_k(feq_k) - p.h around the
   equilibrium of u, cancellation-free; delta_out (M, may be NULL) receives
   Delta = p - p' with grad s*_k(p') = feq_k + h.  NaN outside the domain. */
double or_bregman(const or_model *m, int k, const double *u, const double *h, double *delta_out);
/* microscopic entropy imbalance Delta Sigma(omega) = Sigma(R_omega f) - Sigma(f)
   for one cell (fcell[k*M + m]) */
double or_entropy_imbalance(const or_model *m, const double *fcell, double omega);
/* relaxation parameter for one cell (fixed value, or the entropic root) */
double or_omega(const or_model *m, const double *fcell, or_stats *st);

/* --- grid operators --- */
void or_init_equilibrium(const or_model *m, const double *u0 /* M*ncell */, double *f);
/* T(s): s unit shifts along each population's own velocity (negative s
   reverses the direction) */
int or_transport(const or_model *m, double *f, long s);
/* one relaxation sweep; kind = OR_R_MAIN or OR_R_PROJECT */
int or_relax(const or_model *m, double *f, int kind, or_stats *st);
/* basic brick psi(coef dt) with coef = num/den (eq. basicBrickSplitting);
   -1 if the shifts are not integers */
int or_brick(const or_model *m, double *f, long num, long den, or_stats *st);
/* nsteps composite steps of the given scheme */
int or_composite_steps(const or_model *m, double *f, int scheme, long nsteps, or_stats *st);
/* time advanced by one step of the scheme, in units of dx / V */
long or_step_length(const or_model *m, int scheme);

/* --- observables --- */
void or_moments(const or_model *m, const double *f, double *u /* M*ncell */);
/* total microscopic entropy sum_x Sigma(f(x)) and total entropy sum_x S(u(x)) */
void or_entropy_totals(const or_model *m, const double *f, double *sigma_total, double *S_total);

#ifdef __cplusplus
}
#endif
#endif
