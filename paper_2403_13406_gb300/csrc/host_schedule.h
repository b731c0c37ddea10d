// host_schedule.h -- host-side helpers shared by the single-lattice and the
// batched C ABI: the paper's operator list of one step and the family of a
// configuration.
#pragma once

#include <stdint.h>

#include <vector>

#include "../../include/eslbm.h"
#include "launch.h"

namespace eslbm {

struct Op {
    bool relax;
    int64_t shift;
    int kind;
};

// Operator list of one step, in application order (operators compose right to
// left in the paper's formulas).
inline std::vector<Op> scheme_ops(int scheme, int64_t kappa)
{
    std::vector<Op> ops;
    auto T = [&](int64_t s) { ops.push_back({false, s, 0}); };
    auto R = [&](int kind) { ops.push_back({true, 0, kind}); };
    // psi(coef dt) = T(coef dt/4) R T(coef dt/2) R T(coef dt/4), dt = 24 kappa dx / V
    // (eq. basicBrickSplitting); T(coef dt/4) shifts 6 kappa coef cells.
    auto brick = [&](int64_t q4) {
        T(q4);
        R(KIND_MAIN);
        T(2 * q4);
        R(KIND_MAIN);
        T(q4);
    };
    // Scheme (IV): R_1 T R_2 T R_1 T R_2 T with quarter transports (Section 6.1)
    auto brick_iv = [&](int64_t q4) {
        for (int half = 0; half < 2; ++half) {
            T(q4);
            R(KIND_MAIN);
            T(q4);
            R(KIND_PROJECT);
        }
    };
    switch (scheme) {
    case ESLBM_SCHEME_I:
    case ESLBM_SCHEME_II:
    case ESLBM_SCHEME_III:
    case ESLBM_SCHEME_IV: {
        // eq. splittingToUse: psi(dt/6)^4 psi(-dt/3) psi(dt/6)^4 (n = 4, alpha = 1/6,
        // beta = -1/3 solve eqs. fourtOrderConditionOne/Two)
        const int64_t n_outer = 4, a_num = 1, a_den = 6, b_num = -1, b_den = 3;
        const int64_t qa = 6 * kappa * a_num / a_den, qb = 6 * kappa * b_num / b_den;
        for (int part = 0; part < 3; ++part) {
            const int64_t reps = part == 1 ? 1 : n_outer;
            const int64_t q4 = part == 1 ? qb : qa;
            for (int64_t r = 0; r < reps; ++r) {
                if (scheme == ESLBM_SCHEME_IV) brick_iv(q4);
                else brick(q4);
                if (scheme == ESLBM_SCHEME_III) R(KIND_PROJECT);
            }
        }
        if (scheme == ESLBM_SCHEME_II) R(KIND_PROJECT);
        break;
    }
    case ESLBM_SCHEME_PLAIN:  // R T(kappa dx/V), Section 2.1
        T(kappa);
        R(KIND_MAIN);
        break;
    case ESLBM_SCHEME_B:  // R_1 T(dt/4) R T(dt/2) R T(dt/4), dt = 4 kappa dx / V, Section 6.3
        T(kappa);
        R(KIND_MAIN);
        T(2 * kappa);
        R(KIND_MAIN);
        T(kappa);
        R(KIND_PROJECT);
        break;
    }
    return ops;
}

inline int64_t step_cells(int scheme, int64_t kappa)
{
    if (scheme == ESLBM_SCHEME_PLAIN) return kappa;
    if (scheme == ESLBM_SCHEME_B) return 4 * kappa;
    return 24 * kappa;
}

inline int family_of(const eslbm_config &c)
{
    switch (c.system) {
    case ESLBM_LINEAR: return c.dim == 1 ? FAM_LINEAR1 : FAM_LINEAR2;
    case ESLBM_BURGERS: return c.dim == 1 ? FAM_BURGERS1 : FAM_BURGERS2;
    case ESLBM_SHALLOW_WATER: return c.dim == 1 ? FAM_SW1 : FAM_SW2;
    default: return FAM_EULER2;
    }
}

// Omega mode of a configuration (launch.h)
inline int omega_mode_of(const eslbm_config &c)
{
    if (c.omega_mode != ESLBM_OMEGA_ENTROPIC) return OM_FIXED;
    return c.precision == ESLBM_FP32_MIXED ? OM_MIXED : OM_ENTROPIC;
}

// Whether launches record their relaxations for the per-cell check (diagnostics on an
// entropic nonlinear system).
inline bool records_of(const eslbm_config &c)
{
    return c.diagnostics && c.omega_mode == ESLBM_OMEGA_ENTROPIC &&
           (c.system == ESLBM_BURGERS || c.system == ESLBM_SHALLOW_WATER);
}

inline int64_t num_M(const eslbm_config &c)
{
    if (c.system == ESLBM_SHALLOW_WATER) return c.dim + 1;
    if (c.system == ESLBM_EULER) return 4;
    return 1;
}

// Kernel parameters of a configuration, with the reference equilibrium of the
// shifted storage; ESLBM_ERR_DOMAIN if cfg.u_ref is outside the domain.
inline eslbm_status params_of(const eslbm_config &c, Params &P)
{
    P = Params{};
    P.V = c.V;
    P.a[0] = c.a[0];
    P.a[1] = c.a[1];
    P.c[0] = c.c[0];
    P.c[1] = c.c[1];
    P.g = c.g;
    P.gamma = c.gamma;
    P.omega = c.omega;
    P.t_max = c.t_max > 0.0 ? c.t_max : 3.0;
    // quadratic kinetic entropies: the entropic omega is 2 exactly (Proposition 2)
    if (c.omega_mode == ESLBM_OMEGA_ENTROPIC && c.system == ESLBM_LINEAR) P.omega = 2.0;
    if (c.shifted && !reference_state(family_of(c), c.precision == ESLBM_FP64, c.u_ref, P)) return ESLBM_ERR_DOMAIN;
    return ESLBM_OK;
}

}  // namespace eslbm
