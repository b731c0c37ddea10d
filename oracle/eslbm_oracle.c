/*
 * eslbm_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see the
 * header).  Built with -O2 -ffp-contract=off and without fast-math so that
 * every operation is a plain IEEE double operation on both x86 and Arm.
 *
 * Readings of the paper used here, where it is silent or ambiguous:
 *  - Negative time steps reverse the shift direction only; the relaxation is
 *    unchanged (Section 2.1, eq. symmetryCondition and the remark after it).
 *  - Kinetic entropies of the nonlinear D2Q4 models are not printed in the
 *    paper.  We use the dual construction s^*_k = S^* / q_d + sign_k G^{j,*} / (2V),
 *    which satisfies eqs. entropyDefinitionMinimization and
 *    transformationEntropyFlux and reproduces every example of Section 1.2.
 *  - The entropy imbalance of eq. variableOmegaProblem is evaluated through
 *    the identity Delta Sigma(omega) = sum_k [B_k((omega-1) delta_k) -
 *    B_k(-delta_k)], with B_k the Bregman divergence of s_k at the
 *    equilibrium; this is the cancellation-free evaluation the remark at the
 *    end of Section 5.1 asks for (factoring out the distance to equilibrium).
 *  - The dichotomy of Section 5.1 searches omega - 1 in [0, t_max] and
 *    returns the lower end of the final bracket (so the cell's microscopic
 *    entropy does not increase).  When no root exists in the convexity
 *    domain the projection omega = 1 is used and counted as a fallback.
 *  - Shallow water: the paper's cubic for the dual velocity (Example 3) has
 *    a sign misprint in its linear coefficient; this oracle does not use the
 *    cubic but solves grad s*_k(p) = f_k directly, which is equivalent to the
 *    corrected cubic (the tests check both statements).
 */
#include "eslbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Model geometry (Section 1.2)                                        */
/* ------------------------------------------------------------------ */

int or_q(const or_model *m) { return m->dim == 1 ? 2 : 4; }

int or_M(const or_model *m)
{
    if (m->system == OR_EULER) return 4;
    return m->system == OR_SW ? m->dim + 1 : 1;
}

long or_ncell(const or_model *m) { return m->nx * (m->dim == 1 ? 1 : m->ny); }

/* axis (0 = x, 1 = y) and sign of velocity k */
static int vel_axis(const or_model *m, int k) { return m->dim == 1 ? 0 : (k & 1); }
static int vel_sign(const or_model *m, int k)
{
    if (m->dim == 1) return k == 0 ? 1 : -1;
    return k < 2 ? 1 : -1;
}

int or_check(const or_model *m)
{
    if (!m) return -1;
    if (m->dim != 1 && m->dim != 2) return -1;
    if (m->system < OR_LINEAR || m->system > OR_EULER) return -1;
    if (m->system == OR_EULER && (m->dim != 2 || !(m->gamma > 1.0) || m->omega_mode != OR_OMEGA_FIXED))
        return -1;
    if (m->nx < 1 || (m->dim == 2 && m->ny < 1)) return -1;
    if (m->kappa < 1) return -1;
    if (!(m->V > 0.0)) return -1;
    if (m->system == OR_SW && !(m->g > 0.0)) return -1;
    if (m->omega_mode != OR_OMEGA_FIXED && m->omega_mode != OR_OMEGA_ENTROPIC) return -1;
    if (m->omega_mode == OR_OMEGA_ENTROPIC && !(m->t_max > 0.0)) return -1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Physics: fluxes, entropy, dual variables (Section 1.1, examples of   */
/* Section 1.2)                                                         */
/* ------------------------------------------------------------------ */

void or_flux(const or_model *m, int j, const double *u, double *phi)
{
    switch (m->system) {
    case OR_LINEAR:
        phi[0] = m->a[j] * u[0];
        break;
    case OR_BURGERS:
        phi[0] = m->c[j] * 0.5 * u[0] * u[0];
        break;
    case OR_EULER: { /* (rho, rho u, rho v, E), p = (gamma - 1)(E - rho |v|^2 / 2) (Section 6.3) */
        double rho = u[0], vx = u[1] / rho, vy = u[2] / rho, E = u[3];
        double p = (m->gamma - 1.0) * (E - 0.5 * rho * (vx * vx + vy * vy));
        double v = j == 0 ? vx : vy;
        phi[0] = rho * v;
        phi[1] = u[1] * v + (j == 0 ? p : 0.0);
        phi[2] = u[2] * v + (j == 1 ? p : 0.0);
        phi[3] = v * (E + p);
        break;
    }
    default: { /* shallow water (h, hu[, hv]) */
        double h = u[0];
        if (m->dim == 1) {
            phi[0] = u[1];
            phi[1] = u[1] * u[1] / h + 0.5 * m->g * h * h;
        } else if (j == 0) {
            phi[0] = u[1];
            phi[1] = u[1] * u[1] / h + 0.5 * m->g * h * h;
            phi[2] = u[1] * u[2] / h;
        } else {
            phi[0] = u[2];
            phi[1] = u[1] * u[2] / h;
            phi[2] = u[2] * u[2] / h + 0.5 * m->g * h * h;
        }
    }
    }
}

/* macroscopic entropy S(u): u^2/2 (linear, Burgers), h|v|^2/2 + g h^2/2
   (shallow water, Example 3) */
double or_entropy_S(const or_model *m, const double *u)
{
    if (m->system == OR_EULER) return NAN; /* no kinetic entropies for Euler in the paper */
    if (m->system != OR_SW) return 0.5 * u[0] * u[0];
    double h = u[0], ke = 0.0;
    for (int i = 1; i <= m->dim; ++i) ke += u[i] * u[i];
    return 0.5 * ke / h + 0.5 * m->g * h * h;
}

/* p = grad S(u); shallow water: p = (g h - |v|^2/2, v) (Example 3) */
void or_dual(const or_model *m, const double *u, double *p)
{
    if (m->system == OR_EULER) {
        for (int i = 0; i < 4; ++i) p[i] = NAN;
        return;
    }
    if (m->system != OR_SW) {
        p[0] = u[0];
        return;
    }
    double h = u[0], v2 = 0.0;
    for (int i = 1; i <= m->dim; ++i) {
        p[i] = u[i] / h;
        v2 += p[i] * p[i];
    }
    p[0] = m->g * h - 0.5 * v2;
}

/* equilibria f^eq_k = u/q_d + sign_k phi^{j_k}(u)/(2V): D1Q2 after the
   velocity choice of Section 1.2.1, D2Q4 of Section 1.2.2 */
void or_equilibrium(const or_model *m, const double *u, double *feq)
{
    int q = or_q(m), M = or_M(m);
    double phi[2][4] = {{0}};
    or_flux(m, 0, u, phi[0]);
    if (m->dim == 2) or_flux(m, 1, u, phi[1]);
    for (int k = 0; k < q; ++k) {
        int j = vel_axis(m, k), s = vel_sign(m, k);
        for (int i = 0; i < M; ++i)
            feq[k * M + i] = u[i] / (double)q + (double)s * phi[j][i] / (2.0 * m->V);
    }
}

/* ------------------------------------------------------------------ */
/* Dual kinetic entropies s*_k(p) with gradient and Hessian             */
/* ------------------------------------------------------------------ */

/* S^*(p) and G^{j,*}(p) (eqs. entropyDefinitionMinimization and
   transformationEntropyFlux): linear S^* = p^2/2, G^* = a_j p^2/2; Burgers
   S^* = p^2/2, G^* = c_j p^3/6; shallow water S^* = W^2/(8g) with
   W = 2 p_1 + |p_v|^2, G^{j,*} = p_{1+j} S^*. */
static void dual_pair(const or_model *m, int j, const double *p, double *Ss, double *gS,
                      double *hS, double *Gs, double *gG, double *hG)
{
    int M = or_M(m);
    for (int i = 0; i < M * M; ++i) hS[i] = hG[i] = 0.0;
    if (m->system == OR_LINEAR) {
        *Ss = 0.5 * p[0] * p[0];
        gS[0] = p[0];
        hS[0] = 1.0;
        *Gs = 0.5 * m->a[j] * p[0] * p[0];
        gG[0] = m->a[j] * p[0];
        hG[0] = m->a[j];
        return;
    }
    if (m->system == OR_BURGERS) {
        double cj = m->c[j];
        *Ss = 0.5 * p[0] * p[0];
        gS[0] = p[0];
        hS[0] = 1.0;
        *Gs = cj * p[0] * p[0] * p[0] / 6.0;
        gG[0] = 0.5 * cj * p[0] * p[0];
        hG[0] = cj * p[0];
        return;
    }
    /* shallow water */
    double W = 2.0 * p[0];
    for (int i = 1; i < M; ++i) W += p[i] * p[i];
    double dW[3], d2W[3] = {0.0, 2.0, 2.0};
    dW[0] = 2.0;
    for (int i = 1; i < M; ++i) dW[i] = 2.0 * p[i];
    double g = m->g;
    *Ss = W * W / (8.0 * g);
    for (int i = 0; i < M; ++i) gS[i] = W * dW[i] / (4.0 * g);
    for (int i = 0; i < M; ++i)
        for (int l = 0; l < M; ++l)
            hS[i * M + l] = (dW[i] * dW[l] + (i == l ? W * d2W[i] : 0.0)) / (4.0 * g);
    int d = 1 + j; /* component of p carrying the velocity along axis j */
    *Gs = p[d] * (*Ss);
    for (int i = 0; i < M; ++i) gG[i] = (i == d ? *Ss : 0.0) + p[d] * gS[i];
    for (int i = 0; i < M; ++i)
        for (int l = 0; l < M; ++l)
            hG[i * M + l] = (i == d ? gS[l] : 0.0) + (l == d ? gS[i] : 0.0) + p[d] * hS[i * M + l];
}

double or_kinetic_dual(const or_model *m, int k, const double *p, double *grad, double *hess)
{
    int M = or_M(m), q = or_q(m);
    if (m->system == OR_EULER) {
        for (int i = 0; i < M; ++i) {
            if (grad) grad[i] = NAN;
            for (int l = 0; l < M && hess; ++l) hess[i * M + l] = NAN;
        }
        return NAN;
    }
    int j = vel_axis(m, k);
    double sg = (double)vel_sign(m, k) / (2.0 * m->V);
    double Ss, Gs, gS[3], gG[3], hS[9], hG[9];
    dual_pair(m, j, p, &Ss, gS, hS, &Gs, gG, hG);
    if (grad)
        for (int i = 0; i < M; ++i) grad[i] = gS[i] / (double)q + sg * gG[i];
    if (hess)
        for (int i = 0; i < M * M; ++i) hess[i] = hS[i] / (double)q + sg * hG[i];
    return Ss / (double)q + sg * Gs;
}

/* ------------------------------------------------------------------ */
/* Small dense linear algebra (M <= 3)                                  */
/* ------------------------------------------------------------------ */

/* solve A x = b by Gaussian elimination with partial pivoting; -1 if singular */
static int solve_small(int n, const double *A_in, const double *b_in, double *x)
{
    double A[9], b[3];
    memcpy(A, A_in, sizeof(double) * (size_t)(n * n));
    memcpy(b, b_in, sizeof(double) * (size_t)n);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
        if (!(fabs(A[piv * n + c]) > 0.0)) return -1;
        if (piv != c) {
            for (int l = 0; l < n; ++l) {
                double t = A[c * n + l];
                A[c * n + l] = A[piv * n + l];
                A[piv * n + l] = t;
            }
            double t = b[c];
            b[c] = b[piv];
            b[piv] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            for (int l = c; l < n; ++l) A[r * n + l] -= f * A[c * n + l];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int l = r + 1; l < n; ++l) s -= A[r * n + l] * x[l];
        x[r] = s / A[r * n + r];
    }
    return 0;
}

/* Sylvester's criterion: all leading principal minors positive */
static int positive_definite(int n, const double *A)
{
    if (!(A[0] > 0.0)) return 0;
    if (n == 1) return 1;
    double m2 = A[0] * A[n + 1] - A[1] * A[n];
    if (!(m2 > 0.0)) return 0;
    if (n == 2) return 1;
    double m3 = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                A[2] * (A[3] * A[7] - A[4] * A[6]);
    return m3 > 0.0;
}

/* ------------------------------------------------------------------ */
/* Cancellation-free Bregman divergence of the kinetic entropies        */
/* ------------------------------------------------------------------ */

/* Gauss-Legendre nodes on [0,1]: the dual kinetic entropies of all the
   systems here are polynomials of degree <= 5 in p, so their Hessians are of
   degree <= 3 along a segment and the two rules below are exact. */
static const double GL2_T[2] = {0.21132486540518711775, 0.78867513459481288225};
static const double GL3_T[3] = {0.11270166537925831148, 0.5, 0.88729833462074168852};
static const double GL3_W[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};

/* dh(Delta) = grad s*_k(p - Delta) - grad s*_k(p) = -(int_0^1 H(p - t Delta) dt) Delta */
static void grad_increment(const or_model *m, int k, const double *p, const double *D, double *dh)
{
    int M = or_M(m);
    double Hbar[9] = {0}, H[9], pt[3];
    for (int n = 0; n < 2; ++n) {
        for (int i = 0; i < M; ++i) pt[i] = p[i] - GL2_T[n] * D[i];
        or_kinetic_dual(m, k, pt, NULL, H);
        for (int i = 0; i < M * M; ++i) Hbar[i] += 0.5 * H[i];
    }
    for (int i = 0; i < M; ++i) {
        double s = 0.0;
        for (int l = 0; l < M; ++l) s += Hbar[i * M + l] * D[l];
        dh[i] = -s;
    }
}

/* Solve grad s*_k(p - Delta) = grad s*_k(p) + h for Delta by Newton's method
   in the increment variables (no O(1) quantity is ever subtracted from
   another).  Returns 0 on success with grad s*_k convex at p - Delta. */
static int solve_delta(const or_model *m, int k, const double *p, const double *h, double *D)
{
    int M = or_M(m);
    double H[9], r[3], corr[3], pt[3], dh[3];
    or_kinetic_dual(m, k, p, NULL, H);
    double nh[3];
    for (int i = 0; i < M; ++i) nh[i] = -h[i];
    if (solve_small(M, H, nh, D)) return -1;
    double prev = INFINITY;
    int converged = 0;
    for (int it = 0; it < 100; ++it) {
        grad_increment(m, k, p, D, dh);
        for (int i = 0; i < M; ++i) r[i] = dh[i] - h[i];
        for (int i = 0; i < M; ++i) pt[i] = p[i] - D[i];
        or_kinetic_dual(m, k, pt, NULL, H);
        if (solve_small(M, H, r, corr)) return -1;
        double cn = 0.0, dn = 0.0;
        for (int i = 0; i < M; ++i) {
            D[i] += corr[i];
            cn += corr[i] * corr[i];
            dn += D[i] * D[i];
        }
        if (!isfinite(dn)) return -1;
        if (cn <= 1e-32 * dn || cn == 0.0) {
            converged = 1;
            break;
        }
        if (it >= 8 && cn >= prev) { /* stagnation at the rounding level */
            converged = cn <= 1e-20 * dn;
            break;
        }
        prev = cn;
    }
    if (!converged) return -1;
    for (int i = 0; i < M; ++i) pt[i] = p[i] - D[i];
    or_kinetic_dual(m, k, pt, NULL, H);
    return positive_definite(M, H) ? 0 : -1;
}

/* B = s*_k(p) - s*_k(p') - grad s*_k(p').(p - p') = int_0^1 t Delta^T H(p - t Delta) Delta dt */
static double bregman_dual(const or_model *m, int k, const double *p, const double *D)
{
    int M = or_M(m);
    double H[9], pt[3], B = 0.0;
    for (int n = 0; n < 3; ++n) {
        for (int i = 0; i < M; ++i) pt[i] = p[i] - GL3_T[n] * D[i];
        or_kinetic_dual(m, k, pt, NULL, H);
        double qf = 0.0;
        for (int i = 0; i < M; ++i)
            for (int l = 0; l < M; ++l) qf += D[i] * H[i * M + l] * D[l];
        B += GL3_W[n] * GL3_T[n] * qf;
    }
    return B;
}

double or_bregman(const or_model *m, int k, const double *u, const double *h, double *delta_out)
{
    int M = or_M(m);
    double p[3], D[3];
    or_dual(m, u, p);
    int zero = 1;
    for (int i = 0; i < M; ++i) zero &= (h[i] == 0.0);
    if (zero) {
        if (delta_out)
            for (int i = 0; i < M; ++i) delta_out[i] = 0.0;
        return 0.0;
    }
    if (solve_delta(m, k, p, h, D)) return NAN;
    if (delta_out)
        for (int i = 0; i < M; ++i) delta_out[i] = D[i];
    return bregman_dual(m, k, p, D);
}

/* ------------------------------------------------------------------ */
/* Kinetic entropies s_k(f_k) (examples of Section 1.2)                 */
/* ------------------------------------------------------------------ */

double or_kinetic_entropy(const or_model *m, int k, const double *fk, const double *p_hint)
{
    int M = or_M(m);
    double sgn = (double)vel_sign(m, k);
    if (m->system == OR_LINEAR) {
        /* quadratic: s_k(f) = f^2 / (2 s*_k'') -- Examples 1 and 4 */
        double H[9];
        or_kinetic_dual(m, k, p_hint, NULL, H);
        return 0.5 * fk[0] * fk[0] / H[0];
    }
    if (m->system == OR_BURGERS && m->dim == 1) {
        /* Example 2: s_pm(f) = V^2/6 ((1 pm 4f/V)^{3/2} mp 6f/V - 1) */
        double V = m->V, x = 1.0 + sgn * 4.0 * fk[0] / V;
        if (x < 0.0) return NAN;
        return V * V / 6.0 * (x * sqrt(x) - sgn * 6.0 * fk[0] / V - 1.0);
    }
    /* dual route of Example 3: s_k(f) = p.f - s*_k(p) with grad s*_k(p) = f */
    double p[3], gr[3], H[9], r[3], corr[3];
    for (int i = 0; i < M; ++i) p[i] = p_hint[i];
    int ok = 0;
    double prev = INFINITY;
    for (int it = 0; it < 100; ++it) {
        or_kinetic_dual(m, k, p, gr, H);
        for (int i = 0; i < M; ++i) r[i] = gr[i] - fk[i];
        if (solve_small(M, H, r, corr)) return NAN;
        double cn = 0.0, pn = 0.0;
        for (int i = 0; i < M; ++i) {
            p[i] -= corr[i];
            cn += corr[i] * corr[i];
            pn += p[i] * p[i];
        }
        if (!isfinite(pn)) return NAN;
        if (cn <= 1e-32 * (pn + 1e-300)) {
            ok = 1;
            break;
        }
        if (it >= 8 && cn >= prev) {
            ok = cn <= 1e-20 * (pn + 1e-300);
            break;
        }
        prev = cn;
    }
    if (!ok) return NAN;
    or_kinetic_dual(m, k, p, NULL, H);
    if (!positive_definite(M, H)) return NAN;
    double s = -or_kinetic_dual(m, k, p, NULL, NULL);
    for (int i = 0; i < M; ++i) s += p[i] * fk[i];
    return s;
}

/* ------------------------------------------------------------------ */
/* Entropic relaxation parameter (Section 5, eq. variableOmegaProblem)  */
/* ------------------------------------------------------------------ */

typedef struct {
    const or_model *m;
    double u[4];
    double delta[4 * 4]; /* delta_k = f^eq_k - f_k */
    double E0;           /* sum_k B_k(-delta_k) = Sigma(f) - S(u) */
} imbalance_ctx;

static int prepare(const or_model *m, const double *fcell, imbalance_ctx *c)
{
    int q = or_q(m), M = or_M(m);
    double feq[16];
    c->m = m;
    for (int i = 0; i < M; ++i) {
        double s = 0.0;
        for (int k = 0; k < q; ++k) s += fcell[k * M + i];
        c->u[i] = s;
    }
    or_equilibrium(m, c->u, feq);
    int zero = 1;
    for (int i = 0; i < q * M; ++i) {
        c->delta[i] = feq[i] - fcell[i];
        zero &= (c->delta[i] == 0.0);
    }
    return zero;
}

/* sum_k B_k(t delta_k) */
static double bregman_sum(const imbalance_ctx *c, double t)
{
    int q = or_q(c->m), M = or_M(c->m);
    double s = 0.0, h[3];
    for (int k = 0; k < q; ++k) {
        for (int i = 0; i < M; ++i) h[i] = t * c->delta[k * M + i];
        s += or_bregman(c->m, k, c->u, h, NULL);
    }
    return s;
}

double or_entropy_imbalance(const or_model *m, const double *fcell, double omega)
{
    imbalance_ctx c;
    if (prepare(m, fcell, &c)) return 0.0;
    return bregman_sum(&c, omega - 1.0) - bregman_sum(&c, -1.0);
}

static void note_omega(or_stats *st, double w)
{
    if (!st) return;
    st->relaxations += 1;
    if (w < st->omega_min) st->omega_min = w;
    if (w > st->omega_max) st->omega_max = w;
}

double or_omega(const or_model *m, const double *fcell, or_stats *st)
{
    if (m->omega_mode == OR_OMEGA_FIXED) {
        note_omega(st, m->omega);
        return m->omega;
    }
    imbalance_ctx c;
    if (prepare(m, fcell, &c)) { /* already at equilibrium: every omega is the identity */
        note_omega(st, 2.0);
        return 2.0;
    }
    c.E0 = bregman_sum(&c, -1.0);
    if (!isfinite(c.E0)) goto fallback;
    if (c.E0 <= 0.0) { /* the divergence underflowed: a quadratic neighbourhood */
        note_omega(st, 2.0);
        return 2.0;
    }
    double lo = 0.0, hi = m->t_max;
    double Fhi = bregman_sum(&c, hi) - c.E0;
    if (isfinite(Fhi) && Fhi <= 0.0) goto fallback; /* no root below t_max */
    /* dichotomy; a point outside the convexity domain (NaN) counts as above the root */
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double Fm = bregman_sum(&c, mid) - c.E0;
        if (isfinite(Fm) && Fm <= 0.0) {
            lo = mid;
        } else {
            hi = mid;
            Fhi = Fm;
        }
    }
    if (!isfinite(Fhi)) goto fallback; /* the root is not inside the convexity domain */
    note_omega(st, 1.0 + lo);
    return 1.0 + lo;
fallback:
    if (st) st->fallbacks += 1;
    note_omega(st, 1.0);
    return 1.0;
}

/* ------------------------------------------------------------------ */
/* Grid operators                                                       */
/* ------------------------------------------------------------------ */

void or_init_equilibrium(const or_model *m, const double *u0, double *f)
{
    int q = or_q(m), M = or_M(m);
    long n = or_ncell(m);
    double u[4], feq[16];
    for (long x = 0; x < n; ++x) {
        for (int i = 0; i < M; ++i) u[i] = u0[(long)i * n + x];
        or_equilibrium(m, u, feq);
        for (int k = 0; k < q; ++k)
            for (int i = 0; i < M; ++i) f[(long)(k * M + i) * n + x] = feq[k * M + i];
    }
}

/* one unit shift of one plane: value at x comes from x - dir along axis */
static void unit_shift_plane(const or_model *m, double *plane, int axis, int dir, double *tmp)
{
    long nx = m->nx, ny = m->dim == 1 ? 1 : m->ny;
    for (long y = 0; y < ny; ++y)
        for (long x = 0; x < nx; ++x) {
            long sx = x, sy = y;
            if (axis == 0) sx = ((x - dir) % nx + nx) % nx;
            else sy = ((y - dir) % ny + ny) % ny;
            tmp[y * nx + x] = plane[sy * nx + sx];
        }
    memcpy(plane, tmp, sizeof(double) * (size_t)(nx * ny));
}

int or_transport(const or_model *m, double *f, long s)
{
    int q = or_q(m), M = or_M(m);
    long n = or_ncell(m);
    long reps = s < 0 ? -s : s;
    int dir_t = s < 0 ? -1 : 1;
    int err = 0;
    /* the planes are independent: with OpenMP each thread shifts whole planes */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(| : err)
#endif
    for (int l = 0; l < q * M; ++l) {
        double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
        if (!tmp) {
            err = 1;
            continue;
        }
        int k = l / M;
        for (long r = 0; r < reps; ++r)
            unit_shift_plane(m, f + (long)l * n, vel_axis(m, k), dir_t * vel_sign(m, k), tmp);
        free(tmp);
    }
    return err ? -1 : 0;
}

static void merge_stats(or_stats *into, const or_stats *from)
{
    into->relaxations += from->relaxations;
    into->fallbacks += from->fallbacks;
    if (from->omega_min < into->omega_min) into->omega_min = from->omega_min;
    if (from->omega_max > into->omega_max) into->omega_max = from->omega_max;
}

/* f_k <- (1 - omega) f_k + omega f^eq_k(u)  (eq. relaxationDiscretizationOmega).
   Cells are independent: with OpenMP each thread relaxes a block of cells with the
   same arithmetic and keeps its own statistics, merged at the end. */
int or_relax(const or_model *m, double *f, int kind, or_stats *st)
{
    int q = or_q(m), M = or_M(m);
    long n = or_ncell(m);
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
        or_stats local = {0, 0, INFINITY, -INFINITY};
        or_stats *ls = st ? &local : NULL;
        double fc[16], u[4], feq[16];
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (long x = 0; x < n; ++x) {
            for (int l = 0; l < q * M; ++l) fc[l] = f[(long)l * n + x];
            double w;
            if (kind == OR_R_PROJECT) {
                w = 1.0;
            } else {
                w = or_omega(m, fc, ls);
            }
            for (int i = 0; i < M; ++i) {
                double s = 0.0;
                for (int k = 0; k < q; ++k) s += fc[k * M + i];
                u[i] = s;
            }
            or_equilibrium(m, u, feq);
            for (int l = 0; l < q * M; ++l) f[(long)l * n + x] = (1.0 - w) * fc[l] + w * feq[l];
        }
        if (st) {
#ifdef _OPENMP
#pragma omp critical
#endif
            merge_stats(st, &local);
        }
    }
    return 0;
}

/* psi(tau), tau = (num/den) dt and dt = 24 kappa dx / V (Section 2.3):
   T(tau/4) R T(tau/2) R T(tau/4) of eq. basicBrickSplitting, i.e. shifts of
   6 kappa num/den and 12 kappa num/den cells. */
int or_brick(const or_model *m, double *f, long num, long den, or_stats *st)
{
    long q4 = 6L * m->kappa * num;
    if (den == 0 || q4 % den) return -1;
    long s4 = q4 / den;
    if (or_transport(m, f, s4)) return -1;
    or_relax(m, f, OR_R_MAIN, st);
    if (or_transport(m, f, 2 * s4)) return -1;
    or_relax(m, f, OR_R_MAIN, st);
    if (or_transport(m, f, s4)) return -1;
    return 0;
}

/* modified brick of Scheme (IV): R_1 T R_2 T R_1 T R_2 T (applied right to left) */
static int brick_iv(const or_model *m, double *f, long num, long den, or_stats *st)
{
    long q4 = 6L * m->kappa * num;
    if (den == 0 || q4 % den) return -1;
    long s4 = q4 / den;
    for (int half = 0; half < 2; ++half) {
        if (or_transport(m, f, s4)) return -1;
        or_relax(m, f, OR_R_MAIN, st);
        if (or_transport(m, f, s4)) return -1;
        or_relax(m, f, OR_R_PROJECT, st);
    }
    return 0;
}

long or_step_length(const or_model *m, int scheme)
{
    if (scheme == OR_SCHEME_B) return 4L * m->kappa;
    if (scheme == OR_SCHEME_PLAIN) return (long)m->kappa;
    return 24L * m->kappa;
}

int or_composite_steps(const or_model *m, double *f, int scheme, long nsteps, or_stats *st)
{
    /* composition psi(alpha dt)^n psi(beta dt) psi(alpha dt)^n of eq. splitting with
       n = 4, alpha = 1/6, beta = -1/3 (eq. splittingToUse); check the order
       conditions 2 n alpha + beta = 1 and 2 n alpha^3 + beta^3 = 0 exactly. */
    const long n_outer = 4, a_num = 1, a_den = 6, b_num = -1, b_den = 3;
    if (2 * n_outer * a_num * b_den + b_num * a_den != a_den * b_den) return -1;
    if (2 * n_outer * a_num * a_num * a_num * b_den * b_den * b_den +
            b_num * b_num * b_num * a_den * a_den * a_den != 0)
        return -1;
    for (long step = 0; step < nsteps; ++step) {
        switch (scheme) {
        case OR_SCHEME_I:
        case OR_SCHEME_II:
        case OR_SCHEME_III:
        case OR_SCHEME_IV: {
            for (int part = 0; part < 3; ++part) {
                long reps = part == 1 ? 1 : n_outer;
                long num = part == 1 ? b_num : a_num, den = part == 1 ? b_den : a_den;
                for (long r = 0; r < reps; ++r) {
                    int rc = scheme == OR_SCHEME_IV ? brick_iv(m, f, num, den, st)
                                                    : or_brick(m, f, num, den, st);
                    if (rc) return -1;
                    if (scheme == OR_SCHEME_III) or_relax(m, f, OR_R_PROJECT, st);
                }
            }
            if (scheme == OR_SCHEME_II) or_relax(m, f, OR_R_PROJECT, st);
            break;
        }
        case OR_SCHEME_PLAIN: /* the standard scheme R T(kappa dx / V) of Section 2.1 */
            if (or_transport(m, f, m->kappa)) return -1;
            or_relax(m, f, OR_R_MAIN, st);
            break;
        case OR_SCHEME_B: /* R_1 T(dt/4) R_2 T(dt/2) R_2 T(dt/4), dt = 4 dx / V (Section 6.3) */
            if (or_transport(m, f, m->kappa)) return -1;
            or_relax(m, f, OR_R_MAIN, st);
            if (or_transport(m, f, 2L * m->kappa)) return -1;
            or_relax(m, f, OR_R_MAIN, st);
            if (or_transport(m, f, m->kappa)) return -1;
            or_relax(m, f, OR_R_PROJECT, st);
            break;
        default:
            return -1;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Observables                                                          */
/* ------------------------------------------------------------------ */

void or_moments(const or_model *m, const double *f, double *u)
{
    int q = or_q(m), M = or_M(m);
    long n = or_ncell(m);
    for (int i = 0; i < M; ++i)
        for (long x = 0; x < n; ++x) {
            double s = 0.0;
            for (int k = 0; k < q; ++k) s += f[(long)(k * M + i) * n + x];
            u[(long)i * n + x] = s;
        }
}

/* Section 4: total microscopic entropy and total entropy of the moments */
void or_entropy_totals(const or_model *m, const double *f, double *sigma_total, double *S_total)
{
    int q = or_q(m), M = or_M(m);
    if (m->system == OR_EULER) {
        *sigma_total = NAN;
        *S_total = NAN;
        return;
    }
    long n = or_ncell(m);
    double sig = 0.0, S = 0.0, u[3], p[3], fk[3];
    for (long x = 0; x < n; ++x) {
        for (int i = 0; i < M; ++i) {
            double s = 0.0;
            for (int k = 0; k < q; ++k) s += f[(long)(k * M + i) * n + x];
            u[i] = s;
        }
        or_dual(m, u, p);
        S += or_entropy_S(m, u);
        for (int k = 0; k < q; ++k) {
            for (int i = 0; i < M; ++i) fk[i] = f[(long)(k * M + i) * n + x];
            sig += or_kinetic_entropy(m, k, fk, p);
        }
    }
    *sigma_total = sig;
    *S_total = S;
}
