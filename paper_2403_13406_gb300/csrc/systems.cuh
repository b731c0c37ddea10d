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

    template <class R> __device__ static R flux(const Params &P, int j, R u)
    {
        return BURGERS ? R(P.c[j]) * R(0.5) * u * u : R(P.a[j]) * u;
    }

    template <class R> __device__ static void equilibrium(const Params &P, const R *u, R *feq)
    {
        const R inv2V = R(0.5) / R(P.V);
        const R phi0 = flux<R>(P, 0, u[0]);
        const R phi1 = DIM == 2 ? flux<R>(P, 1, u[0]) : R(0);
        const R base = u[0] / R(Q);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const R phi = Lattice<DIM>::axis(k) == 0 ? phi0 : phi1;
            feq[k] = Lattice<DIM>::sign(k) > 0 ? base + phi * inv2V : base - phi * inv2V;
        }
    }

    // convexity of every s*_k at the equilibrium dual p = u
    template <class R> __device__ static bool admissible(const Params &P, const R *u)
    {
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const R slope = BURGERS ? R(P.c[j]) * u[0] : R(P.a[j]);
            if (!(fabs(slope) * R(Q) < R(2) * R(P.V))) return false;
        }
        return isfinite(u[0]);
    }

    template <class R> __device__ static R entropy(const Params &, const R *u) { return R(0.5) * u[0] * u[0]; }

    template <class R> struct Ctx {
        R D2[Q], b12[Q], d[Q];
    };

    template <class R> __device__ static void prepare(const Params &P, const R *u, const R *delta, Ctx<R> &cx)
    {
        const R p = u[0];
        const R inv2V = R(0.5) / R(P.V);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int j = Lattice<DIM>::axis(k);
            const R sg = R(Lattice<DIM>::sign(k));
            const R slope = BURGERS ? R(P.c[j]) * p : R(P.a[j]);
            cx.D2[k] = R(1) / R(Q) + sg * slope * inv2V;
            cx.b12[k] = BURGERS ? sg * R(P.c[j]) / R(P.V) : R(0);
            cx.d[k] = delta[k];
        }
    }

    // B = sum_k B_k(t delta_k), dB = d B / dt.  false outside the convexity domain.
    template <class R> __device__ static bool eval(const Params &, const Ctx<R> &cx, R t, R &B, R &dB)
    {
        B = R(0);
        dB = R(0);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const R h = t * cx.d[k];
            if (h == R(0)) continue;
            const R D2 = cx.D2[k], b12 = cx.b12[k];
            const R disc = D2 * D2 + b12 * h;
            if (!(disc > R(0))) return false;
            const R Dl = R(-2) * h / (D2 + sqrt(disc));
            if (!(D2 - R(0.5) * b12 * Dl > R(0))) return false;  // s*'' at p - Delta
            B += Dl * Dl * (R(0.5) * D2 - b12 * Dl * R(1.0 / 6.0));
            dB -= Dl * cx.d[k];
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

    template <class R> __device__ static void equilibrium(const Params &P, const R *u, R *feq)
    {
        const R h = u[0];
        const R g = R(P.g);
        const R inv2V = R(0.5) / R(P.V);
        const R hp = R(0.5) * g * h * h;
        R phi[2][3];
        const R vx = u[1] / h;
        phi[0][0] = u[1];
        phi[0][1] = u[1] * vx + hp;
        if (DIM == 2) {
            const R vy = u[2] / h;
            phi[0][2] = u[2] * vx;
            phi[1][0] = u[2];
            phi[1][1] = u[1] * vy;
            phi[1][2] = u[2] * vy + hp;
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int j = Lattice<DIM>::axis(k);
            const bool plus = Lattice<DIM>::sign(k) > 0;
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const R base = u[m] / R(Q);
                feq[k * M + m] = plus ? base + phi[j][m] * inv2V : base - phi[j][m] * inv2V;
            }
        }
    }

    // h > 0 and |v_j| + sqrt(g h) < 2V/Q along each axis (Example 3)
    template <class R> __device__ static bool admissible(const Params &P, const R *u)
    {
        const R h = u[0];
        if (!(h > R(0)) || !isfinite(h)) return false;
        const R cs = sqrt(R(P.g) * h);
        const R nu = R(2) * R(P.V) / R(Q);
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const R v = u[1 + j] / h;
            if (!(fabs(v) + cs < nu)) return false;
        }
        return true;
    }

    template <class R> __device__ static R entropy(const Params &P, const R *u)
    {
        R q2 = u[1] * u[1];
        if (DIM == 2) q2 += u[2] * u[2];
        return R(0.5) * q2 / u[0] + R(0.5) * R(P.g) * u[0] * u[0];
    }

    template <class R> struct Ctx {
        R W, v[DIM], c[Q], f1[Q], d[Q][M];
    };

    template <class R> __device__ static void prepare(const Params &P, const R *u, const R *delta, Ctx<R> &cx)
    {
        const R h = u[0];
        cx.W = R(2) * R(P.g) * h;
#pragma unroll
        for (int j = 0; j < DIM; ++j) cx.v[j] = u[1 + j] / h;
        const R nu = R(2) * R(P.V) / R(Q);
        const R inv2V = R(0.5) / R(P.V);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int dax = Lattice<DIM>::axis(k);
            const R sg = R(Lattice<DIM>::sign(k));
            cx.c[k] = nu + sg * cx.v[dax];
            cx.f1[k] = h * cx.c[k] * inv2V;  // f^eq_1 of population k
#pragma unroll
            for (int m = 0; m < M; ++m) cx.d[k][m] = delta[k * M + m];
        }
    }

    template <class R> __device__ static bool eval(const Params &P, const Ctx<R> &cx, R t, R &B, R &dB)
    {
        const R g = R(P.g), V = R(P.V);
        const R gV4 = R(4) * g * V;
        const R inv16gV = R(1) / (R(16) * g * V);
        const R W = cx.W;
        B = R(0);
        dB = R(0);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int dax = Lattice<DIM>::axis(k);
            const R sg = R(Lattice<DIM>::sign(k));
            const R h1 = t * cx.d[k][0];
            const R hd = t * cx.d[k][1 + dax];
            R ht = R(0);
            if (DIM == 2) ht = t * cx.d[k][2 - dax];
            if (h1 == R(0) && hd == R(0) && ht == R(0)) continue;
            const R vd = cx.v[dax];
            const R ck = cx.c[k];
            const R f1p = cx.f1[k] + h1;
            if (!(f1p > R(0))) return false;
            const R r = hd - vd * h1;
            // linearised guess at b = 0
            const R A0 = W / (R(2) * ck * ck) - R(1);
            R b = (r - sg * W * h1 / (R(2) * ck)) / (cx.f1[k] * A0);
            R cp, dW, Wp;
            bool conv = false;
            R prev = R(INFINITY);
            for (int it = 0; it < Tol<R>::max_inner; ++it) {
                cp = ck - sg * b;
                if (!(cp > R(0))) return false;
                dW = -(gV4 * h1 + sg * b * W) / cp;
                Wp = W - dW;
                if (!(Wp > R(0))) return false;
                const R G = -b * f1p - sg * dW * (W + Wp) * inv16gV - r;
                const R Gp = f1p * (Wp / (R(2) * cp * cp) - R(1));
                if (!(Gp < R(0))) return false;
                const R db = G / Gp;
                b -= db;
                const R ad = fabs(db);
                if (ad <= Tol<R>::inner * fabs(b)) {
                    conv = true;
                    break;
                }
                if (it >= 2 && ad >= prev) {  // stalled at the rounding level
                    conv = ad <= Tol<R>::inner_accept * fabs(b);
                    break;
                }
                prev = ad;
            }
            if (!conv) return false;
            cp = ck - sg * b;
            dW = -(gV4 * h1 + sg * b * W) / cp;
            Wp = W - dW;
            R ct = R(0);
            if (DIM == 2) ct = (cx.v[1 - dax] * h1 - ht) / f1p;
            R vt = R(0);
            if (DIM == 2) vt = cx.v[1 - dax];
            const R D1 = R(0.5) * (dW - R(2) * vd * b + b * b - R(2) * vt * ct + ct * ct);
            B += (ck * dW * dW + R(2) * Wp * (cp * (b * b + ct * ct) + sg * b * dW)) * inv16gV;
            R dot = D1 * cx.d[k][0] + b * cx.d[k][1 + dax];
            if (DIM == 2) dot += ct * cx.d[k][2 - dax];
            dB -= dot;
        }
        return true;
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

    template <class R> __device__ static void equilibrium(const Params &P, const R *u, R *feq)
    {
        const R rho = u[0], mx = u[1], my = u[2], E = u[3];
        const R vx = mx / rho, vy = my / rho;
        const R p = R(P.gamma - 1.0) * (E - R(0.5) * (mx * vx + my * vy));
        const R phx[4] = {mx, mx * vx + p, my * vx, vx * (E + p)};
        const R phy[4] = {my, mx * vy, my * vy + p, vy * (E + p)};
        const R inv2V = R(0.5) / R(P.V);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const R *phi = (k & 1) ? phy : phx;
            const bool plus = k < 2;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const R base = u[m] * R(0.25);
                feq[k * 4 + m] = plus ? base + phi[m] * inv2V : base - phi[m] * inv2V;
            }
        }
    }

    template <class R> __device__ static bool admissible(const Params &P, const R *u)
    {
        const R rho = u[0];
        if (!(rho > R(0))) return false;
        const R p = R(P.gamma - 1.0) * (u[3] - R(0.5) * (u[1] * u[1] + u[2] * u[2]) / rho);
        return p > R(0) && isfinite(p);
    }

    template <class R> __device__ static R entropy(const Params &, const R *) { return R(NAN); }

    template <class R> struct Ctx {
        R unused;
    };
    template <class R> __device__ static void prepare(const Params &, const R *, const R *, Ctx<R> &) {}
    template <class R> __device__ static bool eval(const Params &, const Ctx<R> &, R, R &B, R &dB)
    {
        B = R(NAN);
        dB = R(NAN);
        return false;
    }
};

// ---------------------------------------------------------------------------
// Entropic relaxation parameter: safeguarded Newton on the convex, increasing
// F(t) = sum_k B_k(t delta_k) - E0 over (0, t_max], E0 = sum_k B_k(-delta_k),
// started at t = 1 (omega = 2, exact for quadratic entropies, Proposition 2).
// The bracket [lo, hi] keeps F(lo) <= 0 < F(hi) (a point outside the convexity
// domain counts as above the root).  The result is the chord root of the final
// bracket, which never exceeds the true root for a convex F: the cell's
// microscopic entropy does not increase.  No root inside the domain (F stays
// <= 0 up to t_max or up to the domain edge): fallback to omega = 1.
// ---------------------------------------------------------------------------

template <class Sys, class R>
__device__ R entropic_omega(const Params &P, const typename Sys::template Ctx<R> &cx, bool &fallback)
{
    fallback = false;
    R E0, dE0;
    if (!Sys::template eval<R>(P, cx, R(-1), E0, dE0)) {
        fallback = true;
        return R(1);
    }
    if (!(E0 > R(0))) return R(2);  // at equilibrium (to rounding): every omega is the identity
    R lo = R(0), hi = R(P.t_max);
    R Flo = -E0, Fhi = R(0);
    bool hi_ok = false;
    R t = R(1) < hi ? R(1) : R(0.5) * hi;
    bool last = false;
    for (int it = 0; it < Tol<R>::max_outer; ++it) {
        R F, dF;
        const bool ok = Sys::template eval<R>(P, cx, t, F, dF);
        if (ok) F -= E0;
        if (ok && F <= R(0)) {
            lo = t;
            Flo = F;
        } else {
            hi = t;
            Fhi = F;
            hi_ok = ok;
        }
        if (last || (ok && F == R(0))) break;
        R tn = (ok && dF > R(0)) ? t - F / dF : R(-1);
        if (!(tn > lo && tn < hi)) tn = R(0.5) * (lo + hi);
        if (fabs(tn - t) <= Tol<R>::newton * tn) last = true;
        t = tn;
    }
    if (Flo == R(0) && lo > R(0)) return R(1) + lo;
    if (!hi_ok) {
        fallback = true;
        return R(1);
    }
    const R tc = lo - Flo * (hi - lo) / (Fhi - Flo);
    return R(1) + tc;
}

}  // namespace eslbm
