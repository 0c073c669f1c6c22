// Per-node collision operators on deviations d_i = f_i - w_i (registers).
//
//  bgk_collide   LBGK, Eq. lbgk relaxed toward f_eq (as in Algorithm cnp),
//                polynomial f_eq of Eq. equilibrium, Guo forcing Eq. guo_force
//                with the force-shifted velocity of Eq. edm_momentum.
//  mrt_collide   MRT, Eq. mrt_collision, in the orthogonal D3Q19 moment basis
//                of d'Humieres et al. (2002); Guo forcing in moment space,
//                (I - S/2) M F~, and M^-1 = M^T diag(1/|M_k|^2).
//  elbm_collide  entropic LBM, Eqs. elbm and alpha_cond: entropic equilibrium
//                (product form, read with sqrt(1 + 3 u^2), mass and momentum
//                restored on D3Q19), FP64 safeguarded Newton for alpha, EDM
//                forcing Eq. edm_force.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// First-order equilibrium coefficients b_i = 3 w_i, rounded so that
// sum_i b_i e_ia e_ib = delta_ab holds exactly in the compute type.  With
// 3 w_i simply rounded (1/6, 1/12 on D3Q19; 1/3, 1/12 on D2Q9) the sum misses
// 1 by ~1e-8 in FP32, so every collision would rescale the momentum of the
// equilibrium coherently at every node and the error would grow linearly in
// time (1.2e-5 relative after 1000 steps of the 256^3 vortex); with exact
// sums only incoherent per-element rounding is left.  The pairs used are
// exactly representable: on D3Q19 b_diag = fl(1/12), b_axis = (1 - 8 b_diag)/2;
// on D2Q9 b_axis = fl(1/3), b_diag = (1 - 2 b_axis)/4 (Sterbenz subtractions).
// ---------------------------------------------------------------------------
template <class L, class R>
__host__ __device__ constexpr R first_order_coef(int i)
{
    if (i == 0) return R(0);
    if (L::Q == 19) {
        constexpr R bd = R(1.0 / 12.0);
        return i < 7 ? (R(1) - R(8) * bd) / R(2) : bd;
    }
    constexpr R ba = R(1.0 / 3.0);
    return i < 5 ? ba : (R(1) - R(2) * ba) / R(4);
}

// ---------------------------------------------------------------------------
// LBGK
// ---------------------------------------------------------------------------
template <class L, class R>
__host__ __device__ __forceinline__ void bgk_collide(R (&d)[L::Q], R om, R F0, R F1, R F2, bool has_force,
                                            R& rho_out, R (&v)[3])
{
    R drho = 0, j[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        drho += d[i];
        if (L::ex(i)) j[0] += L::ex(i) * d[i];
        if (L::ey(i)) j[1] += L::ey(i) * d[i];
        if (L::ez(i)) j[2] += L::ez(i) * d[i];
    }
    const R rho = R(1) + drho;
    const R irho = R(1) / rho;
    v[0] = (j[0] + R(0.5) * F0) * irho;
    v[1] = (j[1] + R(0.5) * F1) * irho;
    v[2] = (L::D == 3) ? (j[2] + R(0.5) * F2) * irho : R(0);
    const R usq = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const R cf = R(1) - R(0.5) * om;
    const R vF = v[0] * F0 + v[1] * F1 + v[2] * F2;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const R wi = (R)L::w(i);
        const R bi = first_order_coef<L, R>(i);
        const R eu = L::ex(i) * v[0] + L::ey(i) * v[1] + L::ez(i) * v[2];
        // Eq. equilibrium minus w_i, written as w_i drho + 3 w_i rho e.u
        // + w_i rho (9/2 (e.u)^2 - 3/2 u^2)
        const R feq = wi * drho + bi * (rho * eu) + wi * (rho * (R(4.5) * eu * eu - R(1.5) * usq));
        R di = d[i] + om * (feq - d[i]);
        if (has_force) {
            const R eF = L::ex(i) * F0 + L::ey(i) * F1 + L::ez(i) * F2;
            di += cf * (bi * eF - R(3) * wi * vF + R(9) * wi * eu * eF);
        }
        d[i] = di;
    }
    rho_out = rho;
}

// ---------------------------------------------------------------------------
// MRT (D3Q19)
// ---------------------------------------------------------------------------
// Moment polynomials of d'Humieres et al. (2002), evaluated on this file's
// velocity set at compile time.  Row order: rho, e, eps, jx, qx, jy, qy, jz,
// qz, 3pxx, 3pixx, pww, piww, pxy, pyz, pxz, mx, my, mz.
__host__ __device__ constexpr int mrt_poly(int k, int x, int y, int z)
{
    const int e2 = x * x + y * y + z * z;
    return k == 0 ? 1
         : k == 1 ? 19 * e2 - 30
         : k == 2 ? (21 * e2 * e2 - 53 * e2 + 24) / 2
         : k == 3 ? x
         : k == 4 ? (5 * e2 - 9) * x
         : k == 5 ? y
         : k == 6 ? (5 * e2 - 9) * y
         : k == 7 ? z
         : k == 8 ? (5 * e2 - 9) * z
         : k == 9 ? 3 * x * x - e2
         : k == 10 ? (3 * e2 - 5) * (3 * x * x - e2)
         : k == 11 ? y * y - z * z
         : k == 12 ? (3 * e2 - 5) * (y * y - z * z)
         : k == 13 ? x * y
         : k == 14 ? y * z
         : k == 15 ? x * z
         : k == 16 ? x * (y * y - z * z)
         : k == 17 ? y * (z * z - x * x)
         : z * (x * x - y * y);
}
__host__ __device__ constexpr int mrt_M(int k, int i)
{
    return mrt_poly(k, D3Q19::ex(i), D3Q19::ey(i), D3Q19::ez(i));
}
__host__ __device__ constexpr int mrt_norm2(int k)
{
    int s = 0;
    for (int i = 0; i < 19; ++i) s += mrt_M(k, i) * mrt_M(k, i);
    return s;
}

template <class R>
__host__ __device__ __forceinline__ void mrt_collide(R (&d)[19], const StepParams& p, R& rho_out,
                                            R (&v)[3])
{
    using L = D3Q19;
    R drho = 0, j[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        drho += d[i];
        if (L::ex(i)) j[0] += L::ex(i) * d[i];
        if (L::ey(i)) j[1] += L::ey(i) * d[i];
        if (L::ez(i)) j[2] += L::ez(i) * d[i];
    }
    const R rho = R(1) + drho;
    const R irho = R(1) / rho;
    const R F0 = (R)p.F[0], F1 = (R)p.F[1], F2 = (R)p.F[2];
    v[0] = (j[0] + R(0.5) * F0) * irho;
    v[1] = (j[1] + R(0.5) * F1) * irho;
    v[2] = (j[2] + R(0.5) * F2) * irho;
    const R usq = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const R vF = v[0] * F0 + v[1] * F1 + v[2] * F2;
    // non-equilibrium part n_i = f_i - f_eq_i = d_i - (f_eq_i - w_i)
    R nq[19], Ft[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const R wi = (R)L::w(i);
        const R bi = first_order_coef<L, R>(i);
        const R eu = L::ex(i) * v[0] + L::ey(i) * v[1] + L::ez(i) * v[2];
        nq[i] = d[i] - (wi * drho + bi * (rho * eu) +
                        wi * (rho * (R(4.5) * eu * eu - R(1.5) * usq)));
        const R eF = L::ex(i) * F0 + L::ey(i) * F1 + L::ez(i) * F2;
        Ft[i] = bi * eF - R(3) * wi * vF + R(9) * wi * eu * eF;
    }
    R t[19];
#pragma unroll
    for (int k = 0; k < 19; ++k) {
        R m = 0, mf = 0;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            if (mrt_M(k, i) != 0) {
                m += R(mrt_M(k, i)) * nq[i];
                mf += R(mrt_M(k, i)) * Ft[i];
            }
        }
        t[k] = R(p.mrt_c[k]) * m - (p.has_force ? R(p.mrt_cf[k]) * mf : R(0));
    }
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        R s = 0;
#pragma unroll
        for (int k = 0; k < 19; ++k)
            if (mrt_M(k, i) != 0) s += R(mrt_M(k, i)) * t[k];
        d[i] -= s;
    }
    rho_out = rho;
}

// ---------------------------------------------------------------------------
// ELBM
// ---------------------------------------------------------------------------
// Entropic equilibrium, Sec. 2.1.3, with the first factor read as
// 2 - sqrt(1 + 3 u^2) and mass and momentum put back along the zeroth and
// first Hermite directions (variant 0); or the polynomial equilibrium
// (variant 1).  FP64.
template <class L>
__host__ __device__ __forceinline__ void elbm_feq(double rho, const double (&u)[3], int variant,
                                         double (&fe)[L::Q])
{
    if (variant == 1) {
        const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const double eu = L::ex(i) * u[0] + L::ey(i) * u[1] + L::ez(i) * u[2];
            fe[i] = rho * L::w(i) * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
        }
        return;
    }
    double c[3], r[3], ri[3];
#pragma unroll
    for (int a = 0; a < L::D; ++a) {
        const double s = sqrt(1.0 + 3.0 * u[a] * u[a]);
        c[a] = 2.0 - s;
        r[a] = (2.0 * u[a] + s) / (1.0 - u[a]);
        ri[a] = 1.0 / r[a];
    }
    const double c0 = (L::D == 3) ? rho * c[0] * c[1] * c[2] : rho * c[0] * c[1];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        double q = c0 * L::w(i);
        if (L::ex(i) == 1) q *= r[0];
        if (L::ex(i) == -1) q *= ri[0];
        if (L::ey(i) == 1) q *= r[1];
        if (L::ey(i) == -1) q *= ri[1];
        if (L::D == 3) {
            if (L::ez(i) == 1) q *= r[2];
            if (L::ez(i) == -1) q *= ri[2];
        }
        fe[i] = q;
    }
    {
        // put the residual mass and momentum back (zero up to rounding on
        // D2Q9, O(u^3) on D3Q19): the root of g shifts with f_eq's mass defect
        double m0 = 0, m1[3] = {0, 0, 0};
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            m0 += fe[i];
            m1[0] += L::ex(i) * fe[i];
            m1[1] += L::ey(i) * fe[i];
            m1[2] += L::ez(i) * fe[i];
        }
        const double dr = rho - m0;
        const double dj0 = rho * u[0] - m1[0], dj1 = rho * u[1] - m1[1],
                     dj2 = rho * u[2] - m1[2];
#pragma unroll
        for (int i = 0; i < L::Q; ++i)
            fe[i] += L::w(i) * (dr + 3.0 * (L::ex(i) * dj0 + L::ey(i) * dj1 + L::ez(i) * dj2));
    }
}

// g(a) = H(f + a Delta) - H(f) and g'(a), with Delta_i = f_i x_i:
//   g(a)  = a A + sum_i f_i (1 + a x_i) log1p(a x_i)
//   g'(a) = A + sum_i f_i x_i log1p(a x_i),      A = sum_i Delta_i ln(f_i / w_i)
// (the termwise form of the H difference; sum Delta_i = 0 removes the
// constant of dH/df).
template <class L>
__host__ __device__ __forceinline__ void elbm_g(const double (&f)[L::Q], const double (&x)[L::Q],
                                       double A, double a, double& g, double& gp)
{
    double s = 0, sp = 0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const double ax = a * x[i];
        const double l1 = log1p(ax);
        s += f[i] * (1.0 + ax) * l1;
        sp += f[i] * x[i] * l1;
    }
    g = a * A + s;
    gp = A + sp;
}

// Eight lattice-symmetry invariants fed to the alpha surrogate (FP64 in,
// FP32 out): t3..t6 = (a_k / rho) / eps^k with a_k = sum f x^k and
// eps = sqrt(a2 / rho), eps, max x / eps, min x / eps, A / a2.
template <class L>
__host__ __device__ __forceinline__ void elbm_features(const double (&f)[L::Q], const double (&x)[L::Q],
                                              double rho, double A, double (&feat)[8],
                                              double (&ak)[7])
{
    double a2 = 0, a3 = 0, a4 = 0, a5 = 0, a6 = 0, xmax = -1e300, xmin = 1e300;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const double xi = x[i];
        const double p2 = f[i] * xi * xi;
        a2 += p2;
        a3 += p2 * xi;
        a4 += p2 * xi * xi;
        a5 += p2 * xi * xi * xi;
        a6 += p2 * xi * xi * xi * xi;
        xmax = fmax(xmax, xi);
        xmin = fmin(xmin, xi);
    }
    const double eps = sqrt(a2 / rho);
    const double ie = 1.0 / eps;
    const double ie2 = ie * ie;
    const double ir = 1.0 / rho;
    feat[0] = a3 * ir * ie2 * ie;
    feat[1] = a4 * ir * ie2 * ie2;
    feat[2] = a5 * ir * ie2 * ie2 * ie;
    feat[3] = a6 * ir * ie2 * ie2 * ie2;
    feat[4] = eps;
    feat[5] = xmax * ie;
    feat[6] = xmin * ie;
    feat[7] = A / a2;
    ak[0] = ak[1] = 0;
    ak[2] = a2; ak[3] = a3; ak[4] = a4; ak[5] = a5; ak[6] = a6;
}

// MLP 8 -> 32 -> 32 -> 1 (tanh), parameters in shared memory (FP32 holding
// BF16-rounded weights), FP32 accumulation.  Returns the raw output.
__host__ __device__ __forceinline__ float mlp_eval(const float* __restrict__ P, const double (&feat)[8])
{
    const float* mean = P;
    const float* istd = P + 8;
    const float* W1 = P + 16;
    const float* b1 = W1 + 256;
    const float* W2 = b1 + 32;
    const float* b2 = W2 + 1024;
    const float* W3 = b2 + 32;
    const float* b3 = W3 + 32;
    float z[8], h1[32];
#pragma unroll
    for (int k = 0; k < 8; ++k) z[k] = ((float)feat[k] - mean[k]) * istd[k];
#pragma unroll
    for (int o = 0; o < 32; ++o) {
        float s = b1[o];
#pragma unroll
        for (int k = 0; k < 8; ++k) s = fmaf(W1[o * 8 + k], z[k], s);
        h1[o] = tanhf(s);
    }
    float out = b3[0];
#pragma unroll 4
    for (int o = 0; o < 32; ++o) {
        float s = b2[o];
#pragma unroll
        for (int k = 0; k < 32; ++k) s = fmaf(W2[o * 32 + k], h1[k], s);
        out = fmaf(W3[o], tanhf(s), out);
    }
    return out;
}

struct AlphaResult {
    double alpha;
    int evals;
    int status;
};

// Non-trivial root of g in [1, alpha_max) (Eq. alpha_cond).  Near-equilibrium
// nodes (max |x| < skip_eps) take alpha = 2.  Safeguarded Newton keeps a
// bracket [lo, hi]: g < 0 below the root, >= 0 at or above it (g is convex
// with g(0) = 0).  If the positivity limit hi is reached with g(hi) < 0 there
// is no root below it and alpha = hi = alpha_max (1 - 1e-10).
template <class L>
__host__ __device__ AlphaResult elbm_solve(const double (&f)[L::Q], const double (&x)[L::Q], double A,
                                  double rho, const StepParams& p, const float* smlp,
                                  double (&feat)[8], bool& have_feat)
{
    AlphaResult r{2.0, 0, ALPHA_SKIP};
    have_feat = false;
    if (p.alpha_mode == 3) return r;          // fixed alpha = 2
    double maxabs = 0, amax = 1e300;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        maxabs = fmax(maxabs, fabs(x[i]));
        if (x[i] < 0) amax = fmin(amax, -1.0 / x[i]);   // f + a f x > 0  <=>  a < -1/x
    }
    if (maxabs < p.skip_eps || !(amax < 1e300)) return r;
    double lo = 1.0, hi = amax * (1.0 - 1e-10);
    bool hi_known = false;
    int evals = 0;
    const bool guarded = (p.alpha_mode == 1 || p.alpha_mode == 2);
    if (guarded || p.pairs_X != nullptr) {
        double ak[7];
        elbm_features<L>(f, x, rho, A, feat, ak);
        have_feat = true;
        if (guarded) {
        double a;
        if (p.alpha_mode == 1)
            a = 2.0 + (ak[3] - 2.0 * ak[4]) / (3.0 * ak[2]) + 4.0 * ak[3] * ak[3] / (9.0 * ak[2] * ak[2]);
        else
            a = 2.0 + (double)smlp[MLP_NPARAM - 1] * (double)mlp_eval(smlp, feat) * feat[4];
        a = fmin(fmax(a, lo), hi);
        double corr = 1e300;
        for (int k = 0; k < p.guard_steps; ++k) {
            double g, gp;
            elbm_g<L>(f, x, A, a, g, gp);
            ++evals;
            double an = (gp > 0) ? a - g / gp : lo;
            an = fmin(fmax(an, lo), hi);
            corr = fabs(an - a);
            a = an;
        }
        if (corr <= p.guard_tol * a) {
            r.alpha = a;
            r.evals = evals;
            r.status = ALPHA_GUARDED;
            return r;
        }
        }
    }
    double a = 2.0;
    if (!(a < hi)) a = 0.5 * (lo + hi);
    int status = ALPHA_NOCONV;
    for (int it = 0; it < p.max_iter; ++it) {
        double g, gp;
        elbm_g<L>(f, x, A, a, g, gp);
        ++evals;
        if (g == 0.0) { status = ALPHA_CONV; break; }
        if (g < 0) lo = a;
        else { hi = a; hi_known = true; }
        double an = (gp > 0) ? a - g / gp : -1.0;
        // a step below the tolerance is the answer, even when rounding has
        // collapsed the bracket onto the root
        if (gp > 0 && fabs(an - a) <= p.tol * a) { a = an; status = ALPHA_CONV; break; }
        if (!(an > lo && an < hi)) {
            if (!hi_known && !(an < hi)) {
                double gh, gph;
                elbm_g<L>(f, x, A, hi, gh, gph);
                ++evals;
                if (gh < 0) { a = hi; status = ALPHA_CLAMP; break; }
                hi_known = true;
            }
            an = 0.5 * (lo + hi);
        }
        if (fabs(an - a) <= p.tol * a) { a = an; status = ALPHA_CONV; break; }
        a = an;
    }
    r.alpha = a;
    r.evals = evals;
    r.status = status;
    return r;
}

// ELBM collision of one node.  d (deviations, compute type R) in/out.
// Returns the per-node outcome for the counters.
template <class L, class R>
__host__ __device__ __forceinline__ AlphaResult elbm_collide(R (&d)[L::Q], const StepParams& p,
                                                    const float* smlp, R& rho_out, R (&vout)[3],
                                                    double (&feat)[8], bool& have_feat)
{
    double f[L::Q], x[L::Q];
    double drho = 0, j[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const double di = (double)d[i];
        f[i] = L::w(i) + di;
        drho += di;
        j[0] += L::ex(i) * di;
        j[1] += L::ey(i) * di;
        j[2] += L::ez(i) * di;
    }
    const double rho = 1.0 + drho;
    const double irho = 1.0 / rho;
    double u[3] = {j[0] * irho, j[1] * irho, (L::D == 3) ? j[2] * irho : 0.0};
    double fe[L::Q];
    elbm_feq<L>(rho, u, p.feq_variant, fe);
    double A = 0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const double Dl = fe[i] - f[i];
        x[i] = Dl / f[i];
        A += Dl * log(f[i] / L::w(i));
    }
    AlphaResult ar = elbm_solve<L>(f, x, A, rho, p, smlp, feat, have_feat);
    const double ab = ar.alpha * 0.5 * p.omega;     // alpha * beta, beta = 1/(2 tau)
#pragma unroll
    for (int i = 0; i < L::Q; ++i) d[i] = (R)((f[i] - L::w(i)) + ab * (f[i] * x[i]));
    if (p.has_force) {
        // EDM, Eq. edm_force: f_eq(rho, u + F/rho) - f_eq(rho, u)
        double us[3] = {u[0] + p.F[0] * irho, u[1] + p.F[1] * irho,
                        (L::D == 3) ? u[2] + p.F[2] * irho : 0.0};
        double fs[L::Q];
        elbm_feq<L>(rho, us, p.feq_variant, fs);
#pragma unroll
        for (int i = 0; i < L::Q; ++i)
            d[i] = (R)((f[i] - L::w(i)) + ab * (f[i] * x[i]) + (fs[i] - fe[i]));
    }
    rho_out = (R)rho;
    vout[0] = (R)(u[0] + 0.5 * p.F[0] * irho);
    vout[1] = (R)(u[1] + 0.5 * p.F[1] * irho);
    vout[2] = (L::D == 3) ? (R)(u[2] + 0.5 * p.F[2] * irho) : R(0);
    return ar;
}

}  // namespace lbm
