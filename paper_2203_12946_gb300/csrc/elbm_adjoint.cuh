// elbm_adjoint.cuh -- reverse-mode derivative (vector-Jacobian product) of one
// node's collision f* = f + alpha(f) beta (f^eq(f) - f) (Eq. fstar_def), with
// alpha from the closed form of Sec. III / Appendix C-D differentiated through
// every intermediate: the sign-split sums, alpha_Lower, the bound h, the
// coefficient a, and the positivity clamp.
//
// The paper defines no adjoint; this is the chain rule written out by hand.
// Membership in Omega+ / Omega- is held fixed (each restricted term is O(x^3),
// so the sums are twice differentiable across x = 0); the cutoff and the clamp
// are branches, differentiated on the side the forward pass took.
#pragma once

#include "elbm_device.cuh"

namespace eelbm {

// Positive root R(a, b, c) = 2c / (b + sqrt(b^2 - 4ac)) and its partials.
template <class T>
struct RootGrad {
    T r, ra, rb, rc;
};

template <class T>
__device__ __forceinline__ RootGrad<T> root_grad(T a, T b, T c)
{
    const T Dsc = sqrt(b * b - T(4) * a * c); // >= b > 0 because a <= 0 <= c
    const T den = b + Dsc;
    const T id = T(1) / den;
    RootGrad<T> g;
    g.r = T(2) * c * id;
    g.rc = T(2) * id + T(4) * a * c * id * id / Dsc;
    g.rb = -T(2) * c * id * id * (T(1) + b / Dsc);
    g.ra = T(4) * c * c * id * id / Dsc;
    return g;
}

// h = J^T g for the collision at one node (pre-collision populations F).
// With kForce the node map is C(F) + Phi(C(F)), Phi the body-force term of
// add_force (f^eq(rho, u + F_b/rho) - f^eq(rho, u)); the incoming adjoint passes
// through Phi first, and dforce[a] receives this node's d<g, C + Phi>/dF_b,a.
template <int D, class T, bool kForce = false>
__device__ void node_vjp(const T (&F)[Lattice<D>::Q], const T (&gin0)[Lattice<D>::Q], const CollideParams &p,
                         T (&h)[Lattice<D>::Q], T *dforce = nullptr)
{
    constexpr int Q = Lattice<D>::Q;
    const T beta = beta_of<T>(p);

    // ---- forward: moments and the equilibrium (Sec. I), in the forms the step uses ----
    // Deviations from k_i T(W) (exact), drho corrected for the rest of W, r = rho W in two
    // parts, and per axis eps(c) = -t, 2t +- 3u with t = s - 1 = 3u^2/(1+s): then
    // f^eq_i = k_i r (1 + E_i) and f^eq_i - F_i = (k_i r) E_i + (k_i r - F_i) with one
    // rounding.  The same care matters here as in the step: a VJP of f^eq built on
    // rounded weights maps the conserved adjoint modes (g_i = a + c_i . m) to (1 + e)
    // times themselves, and e ~ 1e-8 per step grows over a long reverse sweep.
    T dev[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) dev[i] = F[i] - T(weight_k(D, i)) * T(weight_unit(D));
    T drho = T(0), j[D];
#pragma unroll
    for (int a = 0; a < D; ++a) j[a] = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += dev[i];
#pragma unroll
        for (int a = 0; a < D; ++a) j[a] += T(vel(D, i, a)) * dev[i];
    }
    drho -= T(double(Q == 9 ? 36 : 216) * double(weight_unit_lo<D, T>()));
    const T rho = T(1) + drho;
    const T irho = T(1) / rho;
    const T rW = fma(rho, T(weight_unit(D)), rho * weight_unit_lo<D, T>());
    // eps[a][c+1] and its derivative d eps / d u_a: 6u/s - 3, -3u/s, 6u/s + 3
    T u[D], eps[D][3], deps[D][3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        u[a] = j[a] * irho;
        const T sq = sqrt(T(1) + T(3) * u[a] * u[a]);
        const T t = T(3) * u[a] * u[a] / (T(1) + sq);
        eps[a][0] = T(2) * t - T(3) * u[a];
        eps[a][1] = -t;
        eps[a][2] = T(2) * t + T(3) * u[a];
        const T v = T(3) * u[a] / sq;
        deps[a][0] = T(2) * v - T(3);
        deps[a][1] = -v;
        deps[a][2] = T(2) * v + T(3);
    }
    // E without axis `skip` (skip = D: all axes): prod (1 + eps) - 1, never rounding 1 + eps
    auto E_excl_at = [&](const T (&ep)[D][3], int i, int skip) -> T {
        T e = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (a != skip) {
                const T ea = ep[a][vel(D, i, a) + 1];
                e = e + ea + e * ea;
            }
        return e;
    };
    auto E_excl = [&](int i, int skip) -> T { return E_excl_at(eps, i, skip); };
    T feq[Q], x[Q], delta[Q];
    T xabs = T(0), xmin = T(0);
    int imin = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T kr = T(weight_k(D, i)) * rW;
        const T E = E_excl(i, D);
        delta[i] = fma(kr, E, kr - F[i]);
        feq[i] = F[i] + delta[i];
        x[i] = delta[i] / F[i];
        xabs = fmax(xabs, fabs(x[i]));
        if (x[i] < xmin) {
            xmin = x[i];
            imin = i;
        }
    }

    // ---- forward: the path length with its intermediates (Appendix D order) ----
    T alpha = T(2);
    int br = kBranchCutoff;
    T B1 = 0, C1 = 0, Cc = 0, S3 = 0, S4 = 0, S5 = 0, S6 = 0, aL = 0, kk = 0, Bp = 0, b = 0, a2 = 0, hh = 0, A = 0;
    if (p.mode != kModeLBGK && !(p.cutoff && xabs < T(kCutoff))) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T xi = x[i], fx2 = F[i] * xi * xi;
            B1 += fx2;
            C1 += fx2 / (T(2) + xi);
            Cc += fx2 * (T(60) + xi * (T(60) + T(11) * xi)) / (T(60) + xi * (T(90) + xi * (T(36) + T(3) * xi)));
            if (xi < T(0)) {
                const T fx3 = fx2 * xi;
                S3 += fx3;
                S4 += fx3 * xi;
                S5 += fx3 * xi * xi;
                S6 += fx3 * xi * xi * xi;
            }
        }
        B1 *= T(0.5);
        C1 *= T(2);
        if (B1 > T(0)) {
            aL = root_grad(T(0.5) * S3, B1, C1).r;
            if (p.mode == kModeLower) {
                alpha = aL;
            } else {
                kk = p.b_variant ? aL : aL * beta;
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    if (x[i] >= T(0)) {
                        const T t = kk * x[i];
                        Bp += F[i] * x[i] * x[i] * x[i] * (T(80) + t * (T(80) + T(19) * t)) /
                              (T(64) + t * (T(96) + t * (T(44) + T(6) * t)));
                    }
                b = B1 - T(2.0 / 15.0) * aL * beta * beta * Bp;
                a2 = beta * beta * S3 / T(6);
                hh = root_grad(a2, b, Cc).r;
                const T hb = hh * beta;
                A = beta * beta * (S3 / T(6) - hb * S4 / T(12) + hb * hb * S5 / T(20) - hb * hb * hb * S6 / T(5));
                alpha = root_grad(A, b, Cc).r;
            }
            br = kBranchSolved;
        }
    }
    bool clamped = false;
    if (p.mode != kModeLBGK && xmin < T(0) && alpha * beta * (-xmin) > T(1)) {
        const T amax = T(-1) / (beta * xmin);
        alpha = T(0.5) * (T(1) + amax);
        if (alpha > amax) alpha = T(0.5) * amax;
        clamped = true;
    }

    // ---- reverse: d alpha / d F into Fb (via x: xb) ----
    T Fb[Q], xb[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) Fb[i] = xb[i] = T(0);
    if (clamped) {
        // alpha = (1 + alpha_max)/2 or alpha_max/2: both carry half of d alpha_max / d x_min
        xb[imin] = T(0.5) / (beta * xmin * xmin);
    } else if (br == kBranchSolved) {
        T B1b = 0, C1b = 0, Ccb = 0, S3b = 0, S4b = 0, S5b = 0, S6b = 0, aLb = 0, Bpb = 0;
        if (p.mode == kModeLower) {
            aLb = T(1);
        } else {
            const RootGrad<T> ra = root_grad(A, b, Cc);
            const T Ab = ra.ra;
            T bb = ra.rb;
            Ccb = ra.rc;
            const T hb = hh * beta;
            const T dAdh = beta * beta * (-beta * S4 / T(12) + T(2) * hh * beta * beta * S5 / T(20) -
                                          T(3) * hh * hh * beta * beta * beta * S6 / T(5));
            const T hbar = Ab * dAdh;
            S3b += Ab * beta * beta / T(6);
            S4b += -Ab * beta * beta * hb / T(12);
            S5b += Ab * beta * beta * hb * hb / T(20);
            S6b += -Ab * beta * beta * hb * hb * hb / T(5);
            const RootGrad<T> rh = root_grad(a2, b, Cc);
            bb += hbar * rh.rb;
            Ccb += hbar * rh.rc;
            S3b += hbar * rh.ra * beta * beta / T(6);
            B1b += bb;
            aLb += -bb * T(2.0 / 15.0) * beta * beta * Bp;
            Bpb = -bb * T(2.0 / 15.0) * aL * beta * beta;
            // Omega+ Boole term: d/dF, d/dx, and through k = alpha_L beta (or alpha_L)
            T kb = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (x[i] >= T(0)) {
                    const T xi = x[i], t = kk * xi;
                    const T N = T(80) + t * (T(80) + T(19) * t), Np = T(80) + T(38) * t;
                    const T M = T(64) + t * (T(96) + t * (T(44) + T(6) * t));
                    const T Mp = T(96) + t * (T(88) + T(18) * t);
                    const T Bv = N / M, Bd = (Np * M - N * Mp) / (M * M);
                    const T x3 = xi * xi * xi;
                    Fb[i] += Bpb * x3 * Bv;
                    xb[i] += Bpb * F[i] * (T(3) * xi * xi * Bv + x3 * Bd * kk);
                    kb += Bpb * F[i] * x3 * Bd * xi;
                }
            aLb += kb * (p.b_variant ? T(1) : beta);
        }
        // alpha_Lower = R(S3/2, B1, C1)
        const RootGrad<T> rl = root_grad(T(0.5) * S3, B1, C1);
        S3b += aLb * rl.ra * T(0.5);
        B1b += aLb * rl.rb;
        C1b = aLb * rl.rc;
        // the sums: B1 = 1/2 <F,x^2>, C1 = 2 <F, x^2/(2+x)>, Cc = <F, x^2 P/Q>, S_k = <F, x^k>_-
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T xi = x[i], Fi = F[i], x2 = xi * xi;
            const T P = T(60) + xi * (T(60) + T(11) * xi), Pp = T(60) + T(22) * xi;
            const T Qx = T(60) + xi * (T(90) + xi * (T(36) + T(3) * xi)), Qp = T(90) + xi * (T(72) + T(9) * xi);
            const T r = x2 * P / Qx;
            const T rp = (T(2) * xi * P + x2 * Pp) / Qx - x2 * P * Qp / (Qx * Qx);
            const T q = T(2) + xi;
            Fb[i] += B1b * T(0.5) * x2 + C1b * T(2) * x2 / q + Ccb * r;
            xb[i] += B1b * Fi * xi + C1b * Fi * (T(8) * xi + T(2) * x2) / (q * q) + Ccb * Fi * rp;
            if (xi < T(0)) {
                const T x3 = x2 * xi;
                Fb[i] += S3b * x3 + S4b * x3 * xi + S5b * x3 * x2 + S6b * x3 * x2 * xi;
                xb[i] += Fi * (T(3) * S3b * x2 + T(4) * S4b * x3 + T(5) * S5b * x3 * xi + T(6) * S6b * x3 * x2);
            }
        }
    }
    // x_i = f^eq_i / F_i - 1 and the equilibrium's dependence on F through (rho, u)
    T lam[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        Fb[i] += -xb[i] * feq[i] / (F[i] * F[i]);
        lam[i] = xb[i] / F[i];
    }
    // VJP of f^eq = rho W k_i prod_a (1 + eps_a(c_ia; v)) at a velocity v = (j + F_b)/rho
    // (F_b = 0: v = u):
    //   sum_i l_i d feq_i / d F_j = G_rho + sum_a G_a (c_ja - v_a) / rho,
    //   G_rho = sum_i l_i feq_i / rho,
    //   G_a = sum_i l_i (k_i r) eps_a'(c_ia) prod_{b != a} (1 + eps_b(c_ib)).
    auto feq_vjp_at = [&](const T (&l)[Q], T (&out)[Q], const T (&ep)[D][3], const T (&dep)[D][3],
                          const T (&vv)[D], const T (&fq)[Q], T (&Ga)[D]) {
        T Gr = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) Ga[a] = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            Gr += l[i] * fq[i];
            const T lk = l[i] * (T(weight_k(D, i)) * rW);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const T q = lk * dep[a][vel(D, i, a) + 1];
                Ga[a] += fma(q, E_excl_at(ep, i, a), q);
            }
        }
        Gr *= irho;
        T base = Gr;
#pragma unroll
        for (int a = 0; a < D; ++a) base -= Ga[a] * vv[a] * irho;
#pragma unroll
        for (int jj = 0; jj < Q; ++jj) {
            T v = base;
#pragma unroll
            for (int a = 0; a < D; ++a) v += Ga[a] * T(vel(D, jj, a)) * irho;
            out[jj] = v;
        }
    };
    auto feq_vjp = [&](const T (&l)[Q], T (&out)[Q]) {
        T Ga[D];
        feq_vjp_at(l, out, eps, deps, u, feq, Ga);
    };
    T V[Q];
    feq_vjp(lam, V);
#pragma unroll
    for (int i = 0; i < Q; ++i) Fb[i] += V[i]; // Fb = d alpha / d F

    // ---- the body-force term: gin = (I + dPhi/df*)^T gin0, and d/dF_b ----
    T gin[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) gin[i] = gin0[i];
    if constexpr (kForce) {
        T v[D], epv[D][3], depv[D][3], feqv[Q], Gv[D], Gu[D], Vv[Q], Vu[Q];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            v[a] = u[a] + T(p.force[a]) * irho;
            const T sq = sqrt(T(1) + T(3) * v[a] * v[a]);
            const T t = T(3) * v[a] * v[a] / (T(1) + sq);
            epv[a][0] = T(2) * t - T(3) * v[a];
            epv[a][1] = -t;
            epv[a][2] = T(2) * t + T(3) * v[a];
            const T dv = T(3) * v[a] / sq;
            depv[a][0] = T(2) * dv - T(3);
            depv[a][1] = -dv;
            depv[a][2] = T(2) * dv + T(3);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T kr = T(weight_k(D, i)) * rW;
            feqv[i] = fma(kr, E_excl_at(epv, i, D), kr);
        }
        feq_vjp_at(gin0, Vv, epv, depv, v, feqv, Gv);
        feq_vjp_at(gin0, Vu, eps, deps, u, feq, Gu);
#pragma unroll
        for (int i = 0; i < Q; ++i) gin[i] += Vv[i] - Vu[i];
        if (dforce) {
#pragma unroll
            for (int a = 0; a < D; ++a) dforce[a] += Gv[a] * irho; // d v_a / d F_b,a = 1/rho
        }
    }

    // ---- the collision's VJP: h_j = g_j + beta (s dalpha/dF_j + alpha (feq_vjp(g)_j - g_j)) ----
    T s = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) s += gin[i] * delta[i];
    feq_vjp(gin, V);
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = gin[i] + beta * (s * Fb[i] + alpha * (V[i] - gin[i]));
}

} // namespace eelbm
