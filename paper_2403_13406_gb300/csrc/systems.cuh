// systems.cuh -- per-cell physics of the vectorial D1Q2 / D2Q4 schemes:
// fluxes, equilibria, domain checks, and the cancellation-free evaluation of
// the entropy imbalance used by the entropic relaxation parameter.
//
// Entropic omega (Section 4, eq. variableOmegaProblem).  With
// delta_k = f^eq_k - f_k and p = grad S(u) (the common dual of every
// equilibrium population), R_omega f = f^eq + t delta with t = omega - 1 and
//   Sigma(R_omega f) - Sigma(f) = sum_k [B_k(t delta_k) - B_k(-delta_k)],
// where B_k(h) = s_k(f^eq_k + h) - s_k(f^eq_k) - p.h >= 0 is the Bregman
// divergence of the kinetic entropy (valid because sum_k delta_k = 0).  B_k is
// evaluated from its Legendre dual s*_k in deviation variables Delta = p - p'
// (grad s*_k(p') = f^eq_k + h), so no O(1) quantity is subtracted from another
// and the imbalance keeps full relative precision as f approaches equilibrium
// (the remark closing Section 5.1 asks for exactly this).  d/dt B_k(t delta_k)
// = -Delta.delta_k comes for free.
#pragma once

#include "common.cuh"

namespace eslbm {

// Division in the kernel's arithmetic type: the FP32 path uses the fast
// reciprocal-based division (a few ulp; far below the storage rounding of the
// relaxed distributions), the FP64 path the correctly rounded one.
template <class R> __host__ __device__ __forceinline__ R qdiv(R a, R b) { return a / b; }
template <> __host__ __device__ __forceinline__ float qdiv<float>(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}

// a + b and a - b rounded once each and never merged with a product into a fused multiply-add
template <class R> __host__ __device__ __forceinline__ R add_rn(R a, R b)
{
#ifdef __CUDA_ARCH__
    if constexpr (sizeof(R) == 4)
        return __fadd_rn(a, b);
    else
        return __dadd_rn(a, b);
#else
    return a + b;
#endif
}
template <class R> __host__ __device__ __forceinline__ R sub_rn(R a, R b)
{
#ifdef __CUDA_ARCH__
    if constexpr (sizeof(R) == 4)
        return __fsub_rn(a, b);
    else
        return __dsub_rn(a, b);
#else
    return a - b;
#endif
}

// The equilibria base + d and base - d of two opposite populations (k and k + Q/2, same component),
// both from the same rounded d, so that every kernel that inlines them (whatever it contracts
// around them) computes the same values.  Their roundings need not sum to exactly 2 base: the
// relaxation takes the deviation of the last population of each component from the others
// (`deviations` in the kernels), so that this rounding never enters the conserved sums.
template <class R> __host__ __device__ __forceinline__ void eq_pair(R base, R d, R &plus, R &minus)
{
    plus = add_rn(base, d);
    minus = sub_rn(base, d);
}

// ---------------------------------------------------------------------------
// Scalar systems (M = 1): linear transport and Burgers.  Dual kinetic
// entropies s*_k(p) = p^2/(2Q) + sign_k G^{j*}(p)/(2V) (Examples 1, 2, 4 and
// their D2Q4 analogue), a cubic in p:
//   s*_k'' (p) = D2_k = 1/Q + sign_k (a_j | c_j p) / (2V),   s*_k''' = 12 beta_k,
//   12 beta_k = 0 (linear) or sign_k c_j / V (Burgers).
// For increment h the deviation solves 3 beta Delta^2 - D2 Delta - h = 0:
//   Delta = -2h / (D2 + sqrt(D2^2 + 12 beta h)),
//   B = Delta^2 (D2/2 - 2 beta Delta).
// ---------------------------------------------------------------------------

template <int DIM, bool BURGERS> struct Scalar {
    static constexpr int Q = Lattice<DIM>::Q;
    static constexpr int M = 1;
    static constexpr bool LINEAR = !BURGERS;

    template <class R> __host__ __device__ static R flux(const ParamsR<R> &P, int j, R u)
    {
        return BURGERS ? P.c[j] * R(0.5) * u * u : P.a[j] * u;
    }

    template <class R> __host__ __device__ static void equilibrium(const ParamsR<R> &P, const R *u, R *feq)
    {
        const R inv2V = P.inv2V;
        const R phi0 = flux<R>(P, 0, u[0]);
        const R phi1 = DIM == 2 ? flux<R>(P, 1, u[0]) : R(0);
        const R base = u[0] / R(Q);
        // populations k and k + Q/2 are opposite (+x/-x, +y/-y)
        eq_pair<R>(base, phi0 * inv2V, feq[0], feq[Q / 2]);
        if (DIM == 2) eq_pair<R>(base, phi1 * inv2V, feq[1], feq[3]);
    }

    // f^eq_k(ubar + du) - f^eq_k(ubar) (u = ubar + du) without cancellation:
    // phi(u) - phi(ubar) = c du (u + ubar) / 2 (Burgers), a du (linear)
    template <class R> __device__ static void equilibrium_dev(const ParamsR<R> &P, const R *du, const R *u, R *fd)
    {
        const R inv2V = P.inv2V;
        R dphi[2];
#pragma unroll
        for (int j = 0; j < DIM; ++j) dphi[j] = BURGERS ? P.c[j] * R(0.5) * du[0] * (u[0] + P.ubar[0]) : P.a[j] * du[0];
        const R base = du[0] / R(Q);
        eq_pair<R>(base, dphi[0] * inv2V, fd[0], fd[Q / 2]);
        if (DIM == 2) eq_pair<R>(base, dphi[1] * inv2V, fd[1], fd[3]);
    }

    // convexity of every s*_k at the equilibrium dual p = u
    // E[k] = d f^eq_k / d u
    template <class R> __device__ static void equilibrium_jacobian(const ParamsR<R> &P, const R *u, R *E)
    {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int j = Lattice<DIM>::axis(k);
            const R slope = BURGERS ? P.c[j] * u[0] : P.a[j];
            E[k] = R(1) / R(Q) + R(Lattice<DIM>::sign(k)) * slope * P.inv2V;
        }
    }

    template <class R> __host__ __device__ static bool admissible(const ParamsR<R> &P, const R *u)
    {
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const R slope = BURGERS ? P.c[j] * u[0] : P.a[j];
            if (!(fabs(slope) * R(Q) < R(2) * P.V)) return false;
        }
        return isfinite(u[0]);
    }

    template <class R> __device__ static R entropy(const ParamsR<R> &, const R *u) { return R(0.5) * u[0] * u[0]; }

    template <class R> struct Ctx {
        R D2[Q], b12[Q], d[Q];
    };

    template <class R> __device__ static void prepare(const ParamsR<R> &P, const R *u, const R *delta, Ctx<R> &cx)
    {
        const R p = u[0];
        const R inv2V = P.inv2V;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int j = Lattice<DIM>::axis(k);
            const R sg = R(Lattice<DIM>::sign(k));
            const R slope = BURGERS ? P.c[j] * p : P.a[j];
            cx.D2[k] = R(1) / R(Q) + sg * slope * inv2V;
            cx.b12[k] = BURGERS ? sg * P.c[j] * (R(2) * inv2V) : R(0);
            cx.d[k] = delta[k];
        }
    }

    // B = sum_k B_k(t delta_k), dB = d B / dt, and (if Dout) Delta_k = p - p'_k.
    // false outside the convexity domain.
    template <class R, int WARM = 0>
    __device__ static bool eval(const ParamsR<R> &, const Ctx<R> &cx, R t, R &B, R &dB, R *Dout = nullptr,
                                R * = nullptr)
    {
        B = R(0);
        dB = R(0);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const R h = t * cx.d[k];
            if (Dout) Dout[k] = R(0);
            if (h == R(0)) continue;
            const R D2 = cx.D2[k], b12 = cx.b12[k];
            const R disc = D2 * D2 + b12 * h;
            if (!(disc > R(0))) return false;
            const R Dl = R(-2) * h / (D2 + sqrt(disc));
            if (!(D2 - R(0.5) * b12 * Dl > R(0))) return false;  // s*'' at p - Delta
            B += Dl * Dl * (R(0.5) * D2 - b12 * Dl * R(1.0 / 6.0));
            dB -= Dl * cx.d[k];
            if (Dout) Dout[k] = Dl;
        }
        return true;
    }
};

// ---------------------------------------------------------------------------
// Shallow water (Example 3 and its D2Q4 analogue), M = DIM + 1, u = (h, hu[, hv]).
// p = (g h - |v|^2/2, v), W(p) = 2 p_1 + |p_v|^2 = 2 g h, and
//   s*_k(p) = W^2 (nu + sign_k p_d) / (16 g V),  nu = 2V/Q, d = axis of k.
// Writing c = nu + sign p_d and, for the dual p' = p - Delta of f' = f^eq + h,
// Delta_W = W(p) - W(p'), b = Delta_d (and c_t = Delta_t across the axis):
//   4 g V h_1        = -Delta_W (c - sign b) - sign b W
//   h_d - v_d h_1    = -b f'_1 - sign Delta_W (2W - Delta_W) / (16 g V)
//   h_t - v_t h_1    = -c_t f'_1                      (D2Q4 only)
//   16 g V B         = c Delta_W^2 + 2 W' ((c - sign b)(b^2 + c_t^2) + sign b Delta_W)
// with W' = W - Delta_W.  The first relation gives Delta_W(b); the second is a
// scalar equation G(b) = 0 with G'(b) = f'_1 (W'/(2 c'^2) - 1) < 0 on the
// convex branch, solved by Newton from its linearisation at b = 0.
// ---------------------------------------------------------------------------

template <int DIM> struct ShallowWater {
    static constexpr int Q = Lattice<DIM>::Q;
    static constexpr int M = DIM + 1;
    static constexpr bool LINEAR = false;

    template <class R> __host__ __device__ static void equilibrium(const ParamsR<R> &P, const R *u, R *feq)
    {
        const R h = u[0];
        const R g = P.g;
        const R inv2V = P.inv2V;
        const R hp = R(0.5) * g * h * h;
        R phi[2][3];
        const R rh = qdiv(R(1), h);
        const R vx = u[1] * rh;
        phi[0][0] = u[1];
        phi[0][1] = u[1] * vx + hp;
        if (DIM == 2) {
            const R vy = u[2] * rh;
            phi[0][2] = u[2] * vx;
            phi[1][0] = u[2];
            phi[1][1] = u[1] * vy;
            phi[1][2] = u[2] * vy + hp;
        }
        // populations k and k + Q/2 are opposite (+x/-x, +y/-y)
#pragma unroll
        for (int k = 0; k < Q / 2; ++k) {
            const int j = Lattice<DIM>::axis(k);
#pragma unroll
            for (int m = 0; m < M; ++m)
                eq_pair<R>(u[m] / R(Q), phi[j][m] * inv2V, feq[k * M + m], feq[(k + Q / 2) * M + m]);
        }
    }

    // f^eq_k(ubar + du) - f^eq_k(ubar) (u = ubar + du) without cancellation: with
    // v = q / h, dv = v - vbar = (dq - vbar dh) / h, q_a v_b - qbar_a vbar_b = dq_a v_b + qbar_a dv_b
    // and g h^2 / 2 - g hbar^2 / 2 = g dh (h + hbar) / 2
    // (P.aux[j] = vbar_j, the reference velocity)
    template <class R> __device__ static void equilibrium_dev(const ParamsR<R> &P, const R *du, const R *u, R *fd)
    {
        const R h = u[0], hb = P.ubar[0], dh = du[0];
        const R rh = qdiv(R(1), h);
        R v[2], dv[2];
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            v[j] = u[1 + j] * rh;
            dv[j] = (du[1 + j] - P.aux[j] * dh) * rh;
        }
        const R dhp = R(0.5) * P.g * dh * (h + hb);
        R dphi[2][3];
        dphi[0][0] = du[1];
        dphi[0][1] = du[1] * v[0] + P.ubar[1] * dv[0] + dhp;
        if (DIM == 2) {
            dphi[0][2] = du[2] * v[0] + P.ubar[2] * dv[0];
            dphi[1][0] = du[2];
            dphi[1][1] = du[1] * v[1] + P.ubar[1] * dv[1];
            dphi[1][2] = du[2] * v[1] + P.ubar[2] * dv[1] + dhp;
        }
        const R inv2V = P.inv2V;
#pragma unroll
        for (int k = 0; k < Q / 2; ++k) {
            const int j = Lattice<DIM>::axis(k);
#pragma unroll
            for (int m = 0; m < M; ++m)
                eq_pair<R>(du[m] / R(Q), dphi[j][m] * inv2V, fd[k * M + m], fd[(k + Q / 2) * M + m]);
        }
    }

    // E[(k*M + m)*M + n] = d f^eq_{k,m} / d u_n
    template <class R> __device__ static void equilibrium_jacobian(const ParamsR<R> &P, const R *u, R *E)
    {
        const R h = u[0], g = P.g;
        R A[2][3][3];  // d phi^j / d u
        const R vx = u[1] / h;
        const R vy = DIM == 2 ? u[2] / h : R(0);
        // phi^x = (q_x, q_x^2/h + g h^2/2, q_x q_y/h)
        A[0][0][0] = R(0); A[0][0][1] = R(1); A[0][0][2] = R(0);
        A[0][1][0] = g * h - vx * vx; A[0][1][1] = R(2) * vx; A[0][1][2] = R(0);
        A[0][2][0] = -vx * vy; A[0][2][1] = vy; A[0][2][2] = vx;
        // phi^y = (q_y, q_x q_y/h, q_y^2/h + g h^2/2)
        A[1][0][0] = R(0); A[1][0][1] = R(0); A[1][0][2] = R(1);
        A[1][1][0] = -vx * vy; A[1][1][1] = vy; A[1][1][2] = vx;
        A[1][2][0] = g * h - vy * vy; A[1][2][1] = R(0); A[1][2][2] = R(2) * vy;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int j = Lattice<DIM>::axis(k);
            const R s2V = R(Lattice<DIM>::sign(k)) * P.inv2V;
#pragma unroll
            for (int m = 0; m < M; ++m)
#pragma unroll
                for (int n = 0; n < M; ++n) {
                    // in 1D the second component is q_x: the flux rows/columns (0, 1) of phi^x
                    E[(k * M + m) * M + n] = (m == n ? R(1) / R(Q) : R(0)) + s2V * A[j][m][n];
                }
        }
    }

    // h > 0 and |v_j| + sqrt(g h) < 2V/Q along each axis (Example 3)
    template <class R> __host__ __device__ static bool admissible(const ParamsR<R> &P, const R *u)
    {
        const R h = u[0];
        if (!(h > R(0)) || !isfinite(h)) return false;
        const R cs = sqrt(P.g * h);
        const R nu = R(2) * P.V / R(Q);
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const R v = u[1 + j] / h;
            if (!(fabs(v) + cs < nu)) return false;
        }
        return true;
    }

    template <class R> __device__ static R entropy(const ParamsR<R> &P, const R *u)
    {
        R q2 = u[1] * u[1];
        if (DIM == 2) q2 += u[2] * u[2];
        return R(0.5) * q2 / u[0] + R(0.5) * P.g * u[0] * u[0];
    }

    template <class R> struct Ctx {
        R W, v[DIM], c[Q], f1[Q], d[Q][M];
        R rc[Q];      // 1 / c_k
        R rg0[Q];     // 1 / (f^eq_1 (W/(2c^2) - 1)): slope of the linearised equation in b
        // FP32: the t-independent parts of the evaluations, once per cell: r(t) = t r1, the
        // expansion b(t) = t beta1 + t^2 beta2 + ..., and the convergence scale |t| bs1 of b
        R r1[Q], beta1[Q], beta2[Q], bs1[Q];
    };

    template <class R> __device__ static void prepare(const ParamsR<R> &P, const R *u, const R *delta, Ctx<R> &cx)
    {
        const R h = u[0];
        cx.W = R(2) * P.g * h;
        const R rh = qdiv(R(1), h);
#pragma unroll
        for (int j = 0; j < DIM; ++j) cx.v[j] = u[1 + j] * rh;
        const R nu = R(2) * P.V / R(Q);
        const R inv2V = P.inv2V;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int dax = Lattice<DIM>::axis(k);
            const R sg = R(Lattice<DIM>::sign(k));
            const R ck = nu + sg * cx.v[dax];
            cx.c[k] = ck;
            cx.f1[k] = h * ck * inv2V;  // f^eq_1 of population k
            cx.rc[k] = qdiv(R(1), ck);  // only seeds the Newton guess
            cx.rg0[k] = qdiv(R(1), cx.f1[k] * (R(0.5) * cx.W * cx.rc[k] * cx.rc[k] - R(1)));
#pragma unroll
            for (int m = 0; m < M; ++m) cx.d[k][m] = delta[k * M + m];
            if constexpr (sizeof(R) == 4) {
                // linearised equation in b at b = 0: b = (r - lin) rg0, both terms linear in t
                const R r1 = cx.d[k][1 + dax] - cx.v[dax] * cx.d[k][0];
                const R lin1 = R(0.5) * sg * cx.W * cx.d[k][0] * cx.rc[k];
                const R beta1 = (r1 - lin1) * cx.rg0[k];
                // second-order term of b(t) from the expansion of G(b(t)) = 0: with
                // K = 4 g V d_1 + sign W beta_1 the t^2 terms give
                // beta_2 = (d_1 beta_1 - (2 W beta_1 + sign K) K / (16 g V c^2)) / (W^2/(8gVc) - f_1)
                const R K = P.gV4 * cx.d[k][0] + sg * cx.W * beta1;
                cx.r1[k] = r1;
                cx.beta1[k] = beta1;
                cx.beta2[k] = (cx.d[k][0] * beta1 -
                               (R(2) * cx.W * beta1 + sg * K) * K * P.inv16gV * cx.rc[k] * cx.rc[k]) * cx.rg0[k];
                cx.bs1[k] = (fabs(r1) + fabs(lin1)) * fabs(cx.rg0[k]);
            }
        }
    }

    // WARM (FP32 only): 0 = start from the linearised guess b = t beta_1; 1 = t is +1 and bio[0..Q)
    // holds b(-1): start from b(-1) + 2 beta_1; 2 = bio holds b(-1) and b(+1): start from the cubic
    // t beta_1 + t^2 beta_2 + t^3 beta_3 through them.  b(t) is odd-plus-even smooth in t with
    // b'(0) = beta_1, so these guesses are off by O(|delta|^3) and O(|delta|^4), and one Newton step
    // brings them to the rounding level.  The solution is stored in bio[Q * (t > 0) + k] when bio is set.
    template <class R, int WARM = 0>
    __device__ static bool eval(const ParamsR<R> &P, const Ctx<R> &cx, R t, R &B, R &dB, R *Dout = nullptr,
                                R *bio = nullptr)
    {
        constexpr bool FAST = sizeof(R) == 4;
        constexpr int warm = FAST ? WARM : 0;
        const R gV4 = P.gV4;
        const R inv16gV = P.inv16gV;
        const R W = cx.W;
        bool good = true;
        R h1[Q], r[Q], f1p[Q], b[Q], bscale[Q], db[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int dax = Lattice<DIM>::axis(k);
            const R sg = R(Lattice<DIM>::sign(k));
            h1[k] = t * cx.d[k][0];
            f1p[k] = cx.f1[k] + h1[k];
            good &= f1p[k] > R(0);
            db[k] = R(0);
            if constexpr (FAST) {
                const R beta1 = cx.beta1[k];
                r[k] = t * cx.r1[k];
                bscale[k] = fabs(t) * cx.bs1[k];
                if constexpr (warm == 0) {
                    b[k] = t * (beta1 + t * cx.beta2[k]);  // second-order guess
                } else if constexpr (warm == 1) {
                    b[k] = bio[k] + R(2) * beta1;
                } else {
                    const R beta2 = R(0.5) * (bio[Q + k] + bio[k]);
                    const R beta3 = R(0.5) * (bio[Q + k] - bio[k]) - beta1;
                    b[k] = t * (beta1 + t * (beta2 + t * beta3));
                }
            } else {
                const R hd = t * cx.d[k][1 + dax];
                r[k] = hd - cx.v[dax] * h1[k];
                // linearised guess at b = 0; the magnitude of its two terms is the convergence
                // scale of b (which itself can be far smaller when they cancel)
                const R lin = R(0.5) * sg * W * h1[k] * cx.rc[k];
                b[k] = (r[k] - lin) * cx.rg0[k];
                bscale[k] = (fabs(r[k]) + fabs(lin)) * fabs(cx.rg0[k]);
            }
        }
        // one Newton step on G(b) = -b f'_1 - sign dW (2W - dW)/(16 g V) - r for population k
        auto newton = [&](int k) {
            const R sg = R(Lattice<DIM>::sign(k));
            const R cp = cx.c[k] - sg * b[k];
            const R rcp = qdiv(R(1), cp);
            const R dW = -(gV4 * h1[k] + sg * b[k] * W) * rcp;
            const R Wp = W - dW;
            const R G = -b[k] * f1p[k] - sg * dW * (W + Wp) * inv16gV - r[k];
            const R Gp = f1p[k] * (R(0.5) * Wp * rcp * rcp - R(1));
            good &= (cp > R(0)) & (Wp > R(0)) & (Gp < R(0));
            db[k] = qdiv(G, Gp);
            b[k] -= db[k];
        };
        // min_inner steps for every population, in lockstep: straight-line code that the
        // scheduler can interleave across populations, and no divergence for smooth cells
        if constexpr (FAST) {  // second-order or warm guesses: one step, more only if the check asks
#pragma unroll
            for (int k = 0; k < Q; ++k) newton(k);
        } else {
#pragma unroll
            for (int it = 0; it < Tol<R>::min_inner; ++it)
#pragma unroll
                for (int k = 0; k < Q; ++k) newton(k);
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            R prev = fabs(db[k]);
            bool conv = prev <= Tol<R>::inner * (fabs(b[k]) + bscale[k]);
            for (int it = FAST ? 1 : Tol<R>::min_inner; !conv && it < Tol<R>::max_inner; ++it) {
                newton(k);
                const R ad = fabs(db[k]);
                if (ad <= Tol<R>::inner * (fabs(b[k]) + bscale[k])) {
                    conv = true;
                } else if (ad >= prev) {  // stalled at the rounding level
                    conv = ad <= Tol<R>::inner_accept * (fabs(b[k]) + bscale[k]);
                    break;
                }
                prev = ad;
            }
            // out of iterations while the steps hover at the rounding level (they need not grow, so
            // the stall test above may not fire): accept as at a stall
            if (!conv) conv = fabs(db[k]) <= Tol<R>::inner_accept * (fabs(b[k]) + bscale[k]);
            good &= conv;
        }
        B = R(0);
        dB = R(0);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int dax = Lattice<DIM>::axis(k);
            const R sg = R(Lattice<DIM>::sign(k));
            const R ck = cx.c[k];
            const R cp = ck - sg * b[k];
            const R dW = -(gV4 * h1[k] + sg * b[k] * W) * qdiv(R(1), cp);
            const R Wp = W - dW;
            R ct = R(0), vt = R(0);
            if (DIM == 2) {
                vt = cx.v[1 - dax];
                ct = qdiv(vt * h1[k] - t * cx.d[k][2 - dax], f1p[k]);
            }
            const R bk = b[k];
            const R D1 = R(0.5) * (dW - R(2) * cx.v[dax] * bk + bk * bk - R(2) * vt * ct + ct * ct);
            B += (ck * dW * dW + R(2) * Wp * (cp * (bk * bk + ct * ct) + sg * bk * dW)) * inv16gV;
            R dot = D1 * cx.d[k][0] + bk * cx.d[k][1 + dax];
            if (DIM == 2) dot += ct * cx.d[k][2 - dax];
            dB -= dot;
            if (Dout) {  // Delta_k = p - p'_k in the components (p_1, v_x[, v_y])
                Dout[k * M + 0] = D1;
                Dout[k * M + 1 + dax] = bk;
                if (DIM == 2) Dout[k * M + 2 - dax] = ct;
            }
            if constexpr (FAST && warm < 2)
                if (bio) bio[warm * Q + k] = bk;  // b(-1) (warm 0) or b(+1) (warm 1)
        }
        return good;
    }
};

// ---------------------------------------------------------------------------
// Euler (Section 6.3): (rho, rho u, rho v, E), p = (gamma - 1)(E - rho|v|^2/2).
// Fixed relaxation parameter only: the paper gives no kinetic entropies for it.
// ---------------------------------------------------------------------------

struct Euler2 {
    static constexpr int Q = 4;
    static constexpr int M = 4;
    static constexpr bool LINEAR = false;

    template <class R> __host__ __device__ static void equilibrium(const ParamsR<R> &P, const R *u, R *feq)
    {
        const R rho = u[0], mx = u[1], my = u[2], E = u[3];
        const R rr = qdiv(R(1), rho);
        const R vx = mx * rr, vy = my * rr;
        const R p = P.gamma_m1 * (E - R(0.5) * (mx * vx + my * vy));
        const R phx[4] = {mx, mx * vx + p, my * vx, vx * (E + p)};
        const R phy[4] = {my, mx * vy, my * vy + p, vy * (E + p)};
        const R inv2V = P.inv2V;
        // populations k and k + 2 are opposite (+x/-x, +y/-y)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            eq_pair<R>(u[m] * R(0.25), phx[m] * inv2V, feq[0 * 4 + m], feq[2 * 4 + m]);
            eq_pair<R>(u[m] * R(0.25), phy[m] * inv2V, feq[1 * 4 + m], feq[3 * 4 + m]);
        }
    }

    // f^eq_k(ubar + du) - f^eq_k(ubar) (u = ubar + du) without cancellation: with
    // v = m / rho, dv = (dm - vbar drho) / rho, m_a v_b - mbar_a vbar_b = dm_a v_b + mbar_a dv_b,
    // dp = (gamma - 1)(dE - (dm.v + mbar.dv) / 2) and
    // v_a (E + p) - vbar_a (Ebar + pbar) = dv_a (E + p) + vbar_a (dE + dp)
    // (P.aux = (vbar_x, vbar_y, pbar), the reference velocity and pressure)
    template <class R> __device__ static void equilibrium_dev(const ParamsR<R> &P, const R *du, const R *u, R *fd)
    {
        const R rho = u[0], rr = qdiv(R(1), u[0]);
        const R vx = u[1] * rr, vy = u[2] * rr;
        const R vbx = P.aux[0], vby = P.aux[1];
        const R dvx = (du[1] - vbx * du[0]) * rr, dvy = (du[2] - vby * du[0]) * rr;
        const R pb = P.aux[2];
        const R dK = R(0.5) * (du[1] * vx + du[2] * vy + P.ubar[1] * dvx + P.ubar[2] * dvy);
        const R dp = P.gamma_m1 * (du[3] - dK);
        const R Ep = u[3] + pb + dp;
        (void)rho;
        const R dphx[4] = {du[1], du[1] * vx + P.ubar[1] * dvx + dp, du[2] * vx + P.ubar[2] * dvx,
                           dvx * Ep + vbx * (du[3] + dp)};
        const R dphy[4] = {du[2], du[1] * vy + P.ubar[1] * dvy, du[2] * vy + P.ubar[2] * dvy + dp,
                           dvy * Ep + vby * (du[3] + dp)};
        const R inv2V = P.inv2V;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            eq_pair<R>(du[m] * R(0.25), dphx[m] * inv2V, fd[0 * 4 + m], fd[2 * 4 + m]);
            eq_pair<R>(du[m] * R(0.25), dphy[m] * inv2V, fd[1 * 4 + m], fd[3 * 4 + m]);
        }
    }

    template <class R> __device__ static void equilibrium_jacobian(const ParamsR<R> &P, const R *u, R *E)
    {
        const R rho = u[0], mx = u[1], my = u[2], En = u[3];
        const R vx = mx / rho, vy = my / rho, gm = P.gamma_m1;
        const R p = gm * (En - R(0.5) * (mx * vx + my * vy));
        const R dp[4] = {gm * R(0.5) * (vx * vx + vy * vy), -gm * vx, -gm * vy, gm};
        const R H = (En + p) / rho;  // total enthalpy
        R A[2][4][4];
        // phi^x = (m_x, m_x v_x + p, m_y v_x, v_x (E + p))
        A[0][0][0] = R(0); A[0][0][1] = R(1); A[0][0][2] = R(0); A[0][0][3] = R(0);
        A[0][1][0] = -vx * vx + dp[0]; A[0][1][1] = R(2) * vx + dp[1]; A[0][1][2] = dp[2]; A[0][1][3] = dp[3];
        A[0][2][0] = -vx * vy; A[0][2][1] = vy; A[0][2][2] = vx; A[0][2][3] = R(0);
        A[0][3][0] = -vx * H + vx * dp[0]; A[0][3][1] = H + vx * dp[1]; A[0][3][2] = vx * dp[2];
        A[0][3][3] = vx + vx * dp[3];
        // phi^y = (m_y, m_x v_y, m_y v_y + p, v_y (E + p))
        A[1][0][0] = R(0); A[1][0][1] = R(0); A[1][0][2] = R(1); A[1][0][3] = R(0);
        A[1][1][0] = -vx * vy; A[1][1][1] = vy; A[1][1][2] = vx; A[1][1][3] = R(0);
        A[1][2][0] = -vy * vy + dp[0]; A[1][2][1] = dp[1]; A[1][2][2] = R(2) * vy + dp[2]; A[1][2][3] = dp[3];
        A[1][3][0] = -vy * H + vy * dp[0]; A[1][3][1] = vy * dp[1]; A[1][3][2] = H + vy * dp[2];
        A[1][3][3] = vy + vy * dp[3];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = k & 1;
            const R s2V = (k < 2 ? R(1) : R(-1)) * P.inv2V;
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int n = 0; n < 4; ++n) E[(k * 4 + m) * 4 + n] = (m == n ? R(0.25) : R(0)) + s2V * A[j][m][n];
        }
    }

    template <class R> __host__ __device__ static bool admissible(const ParamsR<R> &P, const R *u)
    {
        const R rho = u[0];
        if (!(rho > R(0))) return false;
        const R p = P.gamma_m1 * (u[3] - R(0.5) * (u[1] * u[1] + u[2] * u[2]) / rho);
        return p > R(0) && isfinite(p);
    }

    template <class R> __device__ static R entropy(const ParamsR<R> &, const R *) { return R(NAN); }

    template <class R> struct Ctx {
        R unused;
    };
    template <class R> __device__ static void prepare(const ParamsR<R> &, const R *, const R *, Ctx<R> &) {}
    template <class R, int WARM = 0>
    __device__ static bool eval(const ParamsR<R> &, const Ctx<R> &, R, R &B, R &dB, R * = nullptr, R * = nullptr)
    {
        B = R(NAN);
        dB = R(NAN);
        return false;
    }
};

// ---------------------------------------------------------------------------
// Entropic relaxation parameter: root t* > 0 of the convex, increasing
// F(t) = B(t) - E0, B(t) = sum_k B_k(t delta_k), E0 = B(-1) (omega = 1 + t).
//  1. Evaluate B and B' at t = -1 and t = +1 (omega = 2 is exact for quadratic
//     entropies, Proposition 2, and close to the root for smooth data).
//  2. B(0) = B'(0) = 0, so these four values fix the quartic model
//     B(t) ~ b2 t^2 + b3 t^3 + b4 t^4; its root (a few polynomial Newton steps)
//     is within O(|delta|^3) of t*.
//  3. Safeguarded Newton on the exact F from there, keeping a bracket
//     [lo, hi] with F(lo) <= 0 < F(hi) (outside the convexity domain counts as
//     above the root).  FP32 stops after the first exact evaluation at the
//     model root (its O(|delta|^3) error is below the storage rounding of
//     omega delta), adding one at the Newton point when that evaluation fell
//     below the root with no upper point; FP64 iterates to a relative step of
//     1e-9 and evaluates once more.  In FP32 the inner solves of the evaluation at +1 and of the later
//     ones start from the deviations already found at -1 (and +1), which
//     leaves one inner Newton step to do instead of two.  In both precisions,
//     when the spare datum of the model certifies it to the rounding level of
//     the arithmetic (smooth data), the model root itself is returned, lowered
//     by the error estimate, without further evaluations.
//  4. Return the chord root of the final bracket: for a convex F it never
//     exceeds t*, so the cell's microscopic entropy does not increase.  If
//     Newton converged from below (every evaluation <= 0 at rounding level),
//     return lo.  No root inside (0, t_max] or inside the convexity domain:
//     fallback omega = 1 (projection).
// ---------------------------------------------------------------------------

template <class Sys, class R>
__device__ R entropic_omega(const ParamsR<R> &P, const typename Sys::template Ctx<R> &cx, bool &fallback,
                           R *Dm = nullptr, R *E0 = nullptr)
{
    // (Dm, E0: optional outputs of the evaluation at t = -1, the dual deviations and B(-1))
    fallback = false;
    R Em = R(0), dEm;
    R bw[2 * Sys::Q];  // deviations at t = -1 and t = +1: warm starts of the later evaluations
    bool warm2 = false;
    const bool okm = Sys::template eval<R, 0>(P, cx, R(-1), Em, dEm, Dm, bw);
    if (E0) *E0 = okm ? Em : R(0);
    if (!okm) {
        fallback = true;
        return R(1);
    }
    if (!(Em > R(0))) return R(2);  // at equilibrium (to rounding): every omega is the identity
    R lo = R(0), hi = P.t_max;
    R Flo = -Em, Fhi = R(0);
    bool hi_ok = false;
    R t;
    bool last = false, last_newton = false, extra = false;
    R Bp, dBp;
    if (R(1) < hi && Sys::template eval<R, 1>(P, cx, R(1), Bp, dBp, nullptr, bw)) {
        warm2 = true;
        const R F1 = Bp - Em;
        if (F1 == R(0)) return R(2);
        if (F1 < R(0)) {
            lo = R(1);
            Flo = F1;
        } else {
            hi = R(1);
            Fhi = F1;
            hi_ok = true;
        }
        // quartic model through B(0) = B'(0) = 0 and B, B' at t = -1, +1
        const R b3 = R(0.5) * (Bp - Em);
        const R b4 = R(0.25) * ((dBp - dEm) - R(2) * (Bp + Em));
        const R b2 = R(0.5) * (Bp + Em) - b4;
        R tm = R(1);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const R m = tm * tm * (b2 + tm * (b3 + tm * b4)) - Em;
            const R dm = tm * (R(2) * b2 + tm * (R(3) * b3 + R(4) * b4 * tm));
            tm -= qdiv(m, dm);
        }
        if (tm > lo && tm < hi) {
            if (fabs(tm - R(1)) <= R(0.25)) {
                // The four values fix the quartic model with one datum to spare.  Its
                // residual r = (B'(1) + B'(-1)) - 3 (B(1) - B(-1)) is the sum over odd n of
                // 2 (n - 3) c_n = 4 c5 + 8 c7 + ... for B(t) = sum_n c_n t^n, the odd content the
                // model misses.  When r is at the rounding level of B the model root is as good
                // as an exact evaluation at it would certify: return it, lowered by the model's
                // error bound over F'(tm) so that F stays <= 0.
                // The even content beyond the model is not measured: the model takes
                // b2 = c2 - c6, b4 = c4 + 2 c6, which leaves c6 t^2 (t^2 - 1)^2 + ..., about
                // 4 c6 (t - 1)^2 near t = 1.  The bound used, 6 c6 |t - 1| with c6 estimated from
                // the decay of the series, c6 ~ c4^2 / c2, over-bounds that term for |t - 1| <= 1/4
                // and must be at the rounding level too.
                const R r = (dBp + dEm) - R(3) * (Bp - Em);
                const R eps = sizeof(R) == 4 ? R(1.1920929e-7) : R(2.220446049250313e-16);
                const R tol = R(64) * eps * (Bp + Em);
                const R dm = tm * (R(2) * b2 + tm * (R(3) * b3 + R(4) * b4 * tm));
                const R even = R(6) * qdiv(b4 * b4, fabs(b2)) * fabs(tm - R(1));
                // and only for smooth cells (cubic term small against the quadratic one), where the
                // rounding-level difference between tm and the root is immaterial; rough cells take
                // the exact evaluation, whose chord is accurate to second order
                if (fabs(r) <= tol && even <= tol && dm > R(0) && fabs(b3) <= R(1e-3) * b2) {
                    const R tc = tm - qdiv(fabs(r) + even, dm);
                    return R(1) + (tc > R(0) ? tc : R(0));
                }
            }
            t = tm;
            last = sizeof(R) == 4;  // FP32: one exact evaluation at the model root
            last_newton = true;
        } else if (sizeof(R) == 4 && fabs(F1) <= R(64) * R(1.1920929e-7) * (Bp + Em)) {
            // FP32, model root on the wrong side of t = 1 with F(1) at the rounding level of B
            // (the odd part of B(t) is O(|delta|^3), below FP32 resolution for small
            // deviations): iterating on such values would only chase noise.  Take what the
            // two evaluations bracket: F(1) <= 0 allows omega = 2; F(1) > 0 gives the chord
            // through F(0) = -E0 and F(1), which does not exceed the root of a convex F.
            return F1 < R(0) ? R(2) : R(1) + Em / Bp;
        } else {
            const R tn = R(1) - F1 / dBp;
            t = (dBp > R(0) && tn > lo && tn < hi) ? tn : R(0.5) * (lo + hi);
        }
    } else {
        hi = R(1) < hi ? R(1) : hi;  // t = 1 leaves the convexity domain (or exceeds t_max)
        t = R(0.5) * hi;
    }
    for (int it = 0; it < Tol<R>::max_outer; ++it) {
        R F, dF;
        const bool ok = warm2 ? Sys::template eval<R, 2>(P, cx, t, F, dF, nullptr, bw)
                              : Sys::template eval<R, 0>(P, cx, t, F, dF);
        if (ok) F -= Em;
        if (ok && F <= R(0)) {
            lo = t;
            Flo = F;
        } else {
            hi = t;
            Fhi = F;
            hi_ok = ok;
        }
        if (ok && F == R(0)) break;
        if (last) {
            // FP32, the evaluation at the model root fell below the root with no upper point:
            // the Newton point from it lies above the root of the convex F, so when it is not
            // already within the rounding level one more evaluation there closes a bracket for
            // the chord (rough cells only; smooth ones are certified or bracketed already)
            if (sizeof(R) == 4 && !extra && !hi_ok && ok && dF > R(0)) {
                const R tn = t - F / dF;
                extra = true;
                if (tn - t > R(1e-6) * t && tn < hi) {
                    t = tn;
                    continue;
                }
            }
            break;
        }
        bool newton = ok && dF > R(0);
        R tn = newton ? t - F / dF : R(-1);
        if (!(tn > lo && tn < hi)) {
            tn = R(0.5) * (lo + hi);
            newton = false;
        }
        if (fabs(tn - t) <= Tol<R>::newton * tn) {
            last = true;
            last_newton = newton;
        }
        t = tn;
    }
    if (Flo == R(0) && lo > R(0)) return R(1) + lo;
    if (!hi_ok) {
        // Newton converged from below (every evaluation <= 0 within rounding): lo is the root;
        // otherwise the bracket collapsed on t_max or on the domain edge: no root
        if (last && last_newton) return R(1) + lo;
        fallback = true;
        return R(1);
    }
    const R tc = lo - Flo * (hi - lo) / (Fhi - Flo);
    return R(1) + tc;
}

}  // namespace eslbm
