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
// Each operator reports the node's density as its deviation drho = rho - 1
// (the kernels store that in the rho output field; readback adds the 1 in
// FP64), so the output keeps the precision of the deviation form.
#pragma once

#include "fp_bits.cuh"
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
// on D2Q9 b_axis = fl(1/3), b_diag = (1 - 2 b_axis)/4 (Sterbenz subtractions);
// on D3Q15 b_axis = fl(1/3), b_corner = (1 - 2 b_axis)/8; on D3Q27
// b_axis = fl(2/9), b_edge = fl(1/18), b_corner = (1 - (2 b_axis + 8 b_edge))/8
// (in that order of evaluation, exact in FP32 and FP64).
// ---------------------------------------------------------------------------
template <class L, class R>
__host__ __device__ constexpr R first_order_coef(int i)
{
    if (i == 0) return R(0);
    if (L::Q == 19) {
        constexpr R bd = R(1.0 / 12.0);
        return i < 7 ? (R(1) - R(8) * bd) / R(2) : bd;
    }
    if (L::Q == 15) {                       // 2 b_axis + 8 b_corner = 1
        constexpr R ba = R(1.0 / 3.0);
        return i < 7 ? ba : (R(1) - R(2) * ba) / R(8);
    }
    if (L::Q == 27) {                       // 2 b_axis + 8 b_edge + 8 b_corner = 1
        constexpr R ba = R(2.0 / 9.0), be = R(1.0 / 18.0);
        return i < 7 ? ba : (i < 19 ? be : (R(1) - (R(2) * ba + R(8) * be)) / R(8));
    }
    constexpr R ba = R(1.0 / 3.0);
    return i < 5 ? ba : (R(1) - R(2) * ba) / R(4);
}

// e_i . (a0, a1, a2) with the lattice's constant components folded at
// compile time (IEEE arithmetic does not let the compiler drop 0 * a).
template <class L, class R>
__host__ __device__ __forceinline__ R edot(int i, R a0, R a1, R a2)
{
    const int x = L::ex(i), y = L::ey(i), z = L::ez(i);
    R s;
    if (x) {
        s = x > 0 ? a0 : -a0;
        if (y) s = y > 0 ? s + a1 : s - a1;
        if (z) s = z > 0 ? s + a2 : s - a2;
    } else if (y) {
        s = y > 0 ? a1 : -a1;
        if (z) s = z > 0 ? s + a2 : s - a2;
    } else if (z) {
        s = z > 0 ? a2 : -a2;
    } else {
        s = R(0);
    }
    return s;
}

// ---------------------------------------------------------------------------
// LBGK, Eq. lbgk relaxed toward Eq. equilibrium, Guo forcing Eq. guo_force.
// Opposite pairs (2q+1, 2q+2) share the even part of the equilibrium,
// w_i (drho + rho (9/2 (e.u)^2 - 3/2 u^2)), and the odd part b_i rho e.u
// changes sign, so each pair is computed once.  Multiply-adds are explicit
// (fma) so that the operation sequence does not depend on the compiler's
// contraction choices in different kernels.
// ---------------------------------------------------------------------------
template <class L, class R>
__host__ __device__ __forceinline__ void bgk_collide(R (&d)[L::Q], R om, R F0, R F1, R F2,
                                                     bool has_force, R& drho_out, R (&v)[3])
{
    constexpr int NP = (L::Q - 1) / 2;
    R S[NP], A[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        S[q] = d[2 * q + 1] + d[2 * q + 2];
        A[q] = d[2 * q + 1] - d[2 * q + 2];
    }
    R drho = d[0];
#pragma unroll
    for (int q = 0; q < NP; ++q) drho += S[q];
    R j[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int i = 2 * q + 1;
        if (L::ex(i)) j[0] = L::ex(i) > 0 ? j[0] + A[q] : j[0] - A[q];
        if (L::ey(i)) j[1] = L::ey(i) > 0 ? j[1] + A[q] : j[1] - A[q];
        if (L::ez(i)) j[2] = L::ez(i) > 0 ? j[2] + A[q] : j[2] - A[q];
    }
    const R rho = R(1) + drho;
    const R irho = R(1) / rho;
    v[0] = fma(R(0.5), F0, j[0]) * irho;
    v[1] = fma(R(0.5), F1, j[1]) * irho;
    v[2] = (L::D == 3) ? fma(R(0.5), F2, j[2]) * irho : R(0);
    const R usq = fma(v[0], v[0], fma(v[1], v[1], v[2] * v[2]));
    const R m15 = R(-1.5) * usq;
    const R cf = fma(R(-0.5), om, R(1));
    const R vF = fma(v[0], F0, fma(v[1], F1, v[2] * F2));
    // f' = (1 - om) f + om f_eq, with om folded into the equilibrium's
    // per-class factors (om w_i rho, om w_i drho, om b_i rho): two operations
    // fewer per pair than relaxing f_eq - f.  b_i keeps sum b_i e_i e_i = I
    // exact, so the equilibrium momentum om rho v is not rescaled coherently.
    const R c1 = R(1) - om;
    const R orho = om * rho, odrho = om * drho;
    {
        const R w0 = (R)L::w(0);
        R d0 = fma(c1, d[0], fma(w0 * orho, m15, w0 * odrho));
        if (has_force) d0 = fma(cf, R(-3) * w0 * vF, d0);
        d[0] = d0;
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int i = 2 * q + 1;
        const R wi = (R)L::w(i);
        const R bi = first_order_coef<L, R>(i);
        const R eu = edot<L, R>(i, v[0], v[1], v[2]);
        const R t = fma(R(4.5) * eu, eu, m15);
        const R even = fma(wi * orho, t, wi * odrho);
        const R odd = (bi * orho) * eu;
        R dp = fma(c1, d[i], even + odd);
        R dm = fma(c1, d[i + 1], even - odd);
        if (has_force) {
            const R eF = edot<L, R>(i, F0, F1, F2);
            const R ge = cf * wi * fma(R(9) * eu, eF, R(-3) * vF);   // even part of the Guo term
            const R go = cf * bi * eF;                                // odd part
            dp += ge + go;
            dm += ge - go;
        }
        d[i] = dp;
        d[i + 1] = dm;
    }
    drho_out = drho;
}

// ---------------------------------------------------------------------------
// Regularized LBGK (Sec. 2.1.1) and LBGK with the Smagorinsky subgrid model
// (Sec. 2.1.4).  Both need the non-equilibrium momentum flux
//   Pi_ab = sum_i (f_i - fe_i) e_ia e_ib
// about an equilibrium fe of the node's own mass; only the even (pair-sum)
// parts contribute.
//  REG:  fe = f_eq(rho, u), u = j / rho, so that f - fe has no mass and no
//        momentum; the populations become f~ = fe + f_reg,
//        f_reg_i = w_i / (2 c_s^4) (e_ia e_ib - c_s^2 delta_ab) Pi_ab, and the
//        LBGK collision with Guo's force acts on them:
//        f' = f~ + omega (f_eq(rho, v) - f~) + Guo term.
//  SMAG: fe = f_eq(rho, v), Pi = Q of Eq. taut,
//        tau = tau0 + tau_t, tau_t = (sqrt(tau0^2 + 4 C_S^2 |Q| / c_s^4) - tau0)/2,
//        |Q| = (Q_ab Q_ab)^(1/2); then LBGK with that tau.
// ---------------------------------------------------------------------------
// Even and odd parts of one opposite pair's equilibrium deviation at
// velocity u (m15 = -3/2 u^2), computed where they are used: the operators
// below recompute them in their update pass instead of keeping per-pair
// arrays alive across passes (registers, not FLOPs, limit these kernels).
template <class L, class R>
__host__ __device__ __forceinline__ void eq_pair(int i, R rho, R drho, R u0, R u1, R u2, R m15,
                                                 R& ev, R& od)
{
    const R wi = (R)L::w(i);
    const R eu = edot<L, R>(i, u0, u1, u2);
    ev = fma(wi * rho, fma(R(4.5) * eu, eu, m15), wi * drho);
    od = (first_order_coef<L, R>(i) * rho) * eu;
}

template <class L, class R, bool SMAG>
__host__ __device__ __forceinline__ void les_collide(R (&d)[L::Q], R om0, R tau0, R cs2smag,
                                                     R F0, R F1, R F2, bool has_force,
                                                     R& drho_out, R (&v)[3])
{
    constexpr int NP = (L::Q - 1) / 2;
    // pass 1: mass, momentum, and the flux about fe
    R drho = d[0], j0 = R(0), j1 = R(0), j2 = R(0);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int i = 2 * q + 1;
        drho += d[i] + d[i + 1];
        const R A = d[i] - d[i + 1];
        if (L::ex(i)) j0 = L::ex(i) > 0 ? j0 + A : j0 - A;
        if (L::ey(i)) j1 = L::ey(i) > 0 ? j1 + A : j1 - A;
        if (L::ez(i)) j2 = L::ez(i) > 0 ? j2 + A : j2 - A;
    }
    const R rho = R(1) + drho;
    const R irho = R(1) / rho;
    v[0] = fma(R(0.5), F0, j0) * irho;
    v[1] = fma(R(0.5), F1, j1) * irho;
    v[2] = (L::D == 3) ? fma(R(0.5), F2, j2) * irho : R(0);
    const R vF = fma(v[0], F0, fma(v[1], F1, v[2] * F2));
    // the velocity fe is taken at: v (SMAG), u = j / rho (REG)
    const R e0 = SMAG ? v[0] : j0 * irho, e1 = SMAG ? v[1] : j1 * irho,
            e2 = SMAG ? v[2] : ((L::D == 3) ? j2 * irho : R(0));
    const R m15e = R(-1.5) * fma(e0, e0, fma(e1, e1, e2 * e2));
    R P[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};   // xx yy zz xy xz yz
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int i = 2 * q + 1;
        R ev, od;
        eq_pair<L, R>(i, rho, drho, e0, e1, e2, m15e, ev, od);
        const R ns = fma(R(-2), ev, d[i] + d[i + 1]);   // pair sum of f - fe
        const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        if (ex) P[0] += ns;
        if (ey) P[1] += ns;
        if (ez) P[2] += ns;
        if (ex && ey) P[3] = (ex * ey > 0) ? P[3] + ns : P[3] - ns;
        if (ex && ez) P[4] = (ex * ez > 0) ? P[4] + ns : P[4] - ns;
        if (ey && ez) P[5] = (ey * ez > 0) ? P[5] + ns : P[5] - ns;
    }
    R om = om0;
    if (SMAG) {
        const R qq = fma(P[0], P[0], fma(P[1], P[1], P[2] * P[2])) +
                     R(2) * fma(P[3], P[3], fma(P[4], P[4], P[5] * P[5]));
        const R tau_t = R(0.5) * (sqrt(fma(tau0, tau0, R(36) * cs2smag * sqrt(qq))) - tau0);
        om = R(1) / (tau0 + tau_t);
    }
    const R cf = fma(R(-0.5), om, R(1));
    const R w0 = (R)L::w(0);
    const R m15v = R(-1.5) * fma(v[0], v[0], fma(v[1], v[1], v[2] * v[2]));
    const R e0v = fma(w0 * rho, m15v, w0 * drho);       // rest equilibrium at v
    // pass 2: relax, pair by pair
    if (SMAG) {
        R d0 = fma(om, e0v - d[0], d[0]);
        if (has_force) d0 = fma(cf, R(-3) * w0 * vF, d0);
        d[0] = d0;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const int i = 2 * q + 1;
            R ev, od;
            eq_pair<L, R>(i, rho, drho, v[0], v[1], v[2], m15v, ev, od);
            R dp = fma(om, (ev + od) - d[i], d[i]);
            R dm = fma(om, (ev - od) - d[i + 1], d[i + 1]);
            if (has_force) {
                const R wi = (R)L::w(i);
                const R eu = edot<L, R>(i, v[0], v[1], v[2]);
                const R eF = edot<L, R>(i, F0, F1, F2);
                const R ge = cf * wi * fma(R(9) * eu, eF, R(-3) * vF);
                const R go = cf * first_order_coef<L, R>(i) * eF;
                dp += ge + go;
                dm += ge - go;
            }
            d[i] = dp;
            d[i + 1] = dm;
        }
    } else {
        // f~ = fe + f_reg; f' = f~ + omega (f_eq(v) - f~) + Guo term
        const R tr3 = (P[0] + P[1] + P[2]) * R(1.0 / 3.0);
        {
            const R e0u = fma(w0 * rho, m15e, w0 * drho);
            const R ft = fma(w0 * R(4.5), -tr3, e0u);
            R d0 = fma(om, e0v - ft, ft);
            if (has_force) d0 = fma(cf, R(-3) * w0 * vF, d0);
            d[0] = d0;
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const int i = 2 * q + 1;
            const R wi = (R)L::w(i);
            // e.Pi.e for this pair (the same for both members)
            const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
            R ePe = R(0);
            if (ex) ePe += P[0];
            if (ey) ePe += P[1];
            if (ez) ePe += P[2];
            if (ex && ey) ePe = (ex * ey > 0) ? fma(R(2), P[3], ePe) : fma(R(-2), P[3], ePe);
            if (ex && ez) ePe = (ex * ez > 0) ? fma(R(2), P[4], ePe) : fma(R(-2), P[4], ePe);
            if (ey && ez) ePe = (ey * ez > 0) ? fma(R(2), P[5], ePe) : fma(R(-2), P[5], ePe);
            const R freg = wi * R(4.5) * (ePe - tr3);
            R evu, odu, evv, odv;
            eq_pair<L, R>(i, rho, drho, e0, e1, e2, m15e, evu, odu);
            if (has_force)
                eq_pair<L, R>(i, rho, drho, v[0], v[1], v[2], m15v, evv, odv);
            else {
                evv = evu;
                odv = odu;
            }
            const R ftp = (evu + odu) + freg, ftm = (evu - odu) + freg;
            R dp = fma(om, (evv + odv) - ftp, ftp);
            R dm = fma(om, (evv - odv) - ftm, ftm);
            if (has_force) {
                const R eu = edot<L, R>(i, v[0], v[1], v[2]);
                const R eF = edot<L, R>(i, F0, F1, F2);
                const R ge = cf * wi * fma(R(9) * eu, eF, R(-3) * vF);
                const R go = cf * first_order_coef<L, R>(i) * eF;
                dp += ge + go;
                dm += ge - go;
            }
            d[i] = dp;
            d[i + 1] = dm;
        }
    }
    drho_out = drho;
}

// ---------------------------------------------------------------------------
// Velocity and pressure boundary nodes (Sec. 2.3: equilibrium, Zou-He and
// regularized conditions).  Applied to the post-streaming deviations of a
// node marked with a condition, before its collision.  With n the inward
// normal, the populations with e_i . n > 0 came from outside and are unknown.
// The known ones fix the missing moment through
//   rho (1 - v_n) = S_0 + 2 S_out - F_n / 2
// (S_0: e.n = 0, S_out: e.n < 0; momentum j = rho v - F/2 as in Guo's scheme,
// so the collision reports exactly v).  Velocity condition: v given; pressure
// condition: rho given, v = v_n n.  Then, with f_eq at (rho, v):
//  equilibrium: f_i = f_eq_i - 3/2 w_i e_i . F;
//  Zou-He: unknown f_i = f_opp(i) + f_eq_i - f_eq_opp(i), and the momentum
//    still missing goes to the link along n (normal part) and, per tangential
//    axis t, evenly with sign e_it to the unknown links of smallest length
//    with e_it != 0 (two edge links; the four body diagonals on D3Q15);
//  regularized: unknown f_i as Zou-He before the correction, then
//    f_i = f_eq_i + w_i 9/2 (e_i e_i - I/3) : Pi^neq - 3/2 w_i e_i . F.
// Rare nodes; deviation-form arithmetic in the compute type, as in the collisions.
// ---------------------------------------------------------------------------
template <class L, class R>
__device__ __forceinline__ void bc_apply(R (&d)[L::Q], const BCEntry& b, R F0, R F1, R F2)
{
    // Deviation form throughout (d = f - w), like the collision operators:
    // on a symmetric lattice the weights of the e.n = 0 and e.n < 0 sets
    // satisfy W_0 + 2 W_out = 1, so S_0 + 2 S_out = 1 + (D_0 + 2 D_out) with D
    // the deviation sums; w_opp(i) = w_i, so the bounce-back of the
    // non-equilibrium part is d_i = d_opp(i) + (e_i - e_opp(i)) equilibrium
    // deviations; momenta are sums of e d.  The normal's axis is a run-time
    // value: components are picked with selects (no run-time indexed arrays,
    // which would live in local memory).
    constexpr int Q = L::Q, D = L::D;
    const int ax = b.axis, sg = b.sign;
    auto pick = [ax](R c0, R c1, R c2) { return ax == 0 ? c0 : (ax == 1 ? c1 : c2); };
    auto en = [&](int i) { return sg * (ax == 0 ? L::ex(i) : (ax == 1 ? L::ey(i) : L::ez(i))); };
    R D0 = R(0), Do = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int e = en(i);
        if (e == 0) D0 += d[i];
        else if (e < 0) Do += d[i];
    }
    const R Fax = pick(F0, F1, F2);
    const R Fn = sg > 0 ? Fax : -Fax;
    const R K = fma(R(2), Do, D0) - R(0.5) * Fn;    // S_0 + 2 S_out - F_n/2 - 1
    R rho, drho, v0, v1, v2;
    if (b.kind == 1) {
        v0 = sel<R>(b.val_f[0], b.val[0]);
        v1 = sel<R>(b.val_f[1], b.val[1]);
        v2 = D == 3 ? sel<R>(b.val_f[2], b.val[2]) : R(0);
        const R vax = pick(v0, v1, v2);
        const R vn = sg > 0 ? vax : -vax;
        drho = (K + vn) / (R(1) - vn);                // rho = (1 + K) / (1 - v_n)
        rho = R(1) + drho;
    } else {
        rho = sel<R>(b.val_f[0], b.val[0]);
        drho = rho - R(1);
        const R vn = (drho - K) / rho;                // 1 - (1 + K) / rho
        const R va = sg > 0 ? vn : -vn;
        v0 = ax == 0 ? va : R(0);
        v1 = ax == 1 ? va : R(0);
        v2 = ax == 2 ? va : R(0);
    }
    const R m15 = R(-1.5) * fma(v0, v0, fma(v1, v1, v2 * v2));
    R qe[Q];   // equilibrium deviations f_eq - w
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const R eu = edot<L, R>(i, v0, v1, v2);
        const R wi = (R)L::w(i);
        qe[i] = fma(wi * rho, fma(R(3), eu, fma(R(4.5) * eu, eu, m15)), wi * drho);
    }
    if (b.method == 0) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
            d[i] = fma(R(-1.5) * (R)L::w(i), edot<L, R>(i, F0, F1, F2), qe[i]);
        return;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i)
        if (en(i) > 0) d[i] = d[L::opp(i)] + (qe[i] - qe[L::opp(i)]);
    if (b.method == 1) {
        R J0 = R(0), J1 = R(0), J2 = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (L::ex(i)) J0 = L::ex(i) > 0 ? J0 + d[i] : J0 - d[i];
            if (L::ey(i)) J1 = L::ey(i) > 0 ? J1 + d[i] : J1 - d[i];
            if (L::ez(i)) J2 = L::ez(i) > 0 ? J2 + d[i] : J2 - d[i];
        }
        const R dJ0 = fma(rho, v0, R(-0.5) * F0) - J0;
        const R dJ1 = fma(rho, v1, R(-0.5) * F1) - J1;
        const R dJ2 = D == 3 ? fma(rho, v2, R(-0.5) * F2) - J2 : R(0);
        const R dJn = pick(dJ0, dJ1, dJ2);
        constexpr int tlen = (Q == 15) ? 3 : 2;      // shortest unknown links with e_t != 0
        constexpr R tshare = (Q == 15) ? R(0.25) : R(0.5);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (en(i) <= 0) continue;
            const int l2 = L::ex(i) * L::ex(i) + L::ey(i) * L::ey(i) + L::ez(i) * L::ez(i);
            if (l2 == 1) d[i] += sg > 0 ? dJn : -dJn;      // the link along n
            if (l2 == tlen) {
                if (L::ex(i) && ax != 0) d[i] = fma(L::ex(i) > 0 ? tshare : -tshare, dJ0, d[i]);
                if (L::ey(i) && ax != 1) d[i] = fma(L::ey(i) > 0 ? tshare : -tshare, dJ1, d[i]);
                if (L::ez(i) && ax != 2) d[i] = fma(L::ez(i) > 0 ? tshare : -tshare, dJ2, d[i]);
            }
        }
        return;
    }
    // regularized: Hermite coefficient a2 = sum (f - f_eq)(e e - I/3); the
    // node's mass defect m = sum (f - f_eq) (F_n/2 under a force) enters the
    // diagonal
    R P[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};   // xx yy zz xy xz yz
    R m = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const R nq = d[i] - qe[i];
        const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        m += nq;
        if (ex) P[0] += nq;
        if (ey) P[1] += nq;
        if (ez) P[2] += nq;
        if (ex && ey) P[3] = (ex * ey > 0) ? P[3] + nq : P[3] - nq;
        if (ex && ez) P[4] = (ex * ez > 0) ? P[4] + nq : P[4] - nq;
        if (ey && ez) P[5] = (ey * ez > 0) ? P[5] + nq : P[5] - nq;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) P[a] = fma(R(-1.0 / 3.0), m, P[a]);
    const R tr3 = (P[0] + P[1] + P[2]) * R(1.0 / 3.0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        R ePe = R(0);
        if (ex) ePe += P[0];
        if (ey) ePe += P[1];
        if (ez) ePe += P[2];
        if (ex && ey) ePe = (ex * ey > 0) ? fma(R(2), P[3], ePe) : fma(R(-2), P[3], ePe);
        if (ex && ez) ePe = (ex * ez > 0) ? fma(R(2), P[4], ePe) : fma(R(-2), P[4], ePe);
        if (ey && ez) ePe = (ey * ez > 0) ? fma(R(2), P[5], ePe) : fma(R(-2), P[5], ePe);
        const R wi = (R)L::w(i);
        d[i] = fma(R(4.5) * wi, ePe - tr3, fma(R(-1.5) * wi, edot<L, R>(i, F0, F1, F2), qe[i]));
    }
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

// Rows odd under e -> -e (momentum, energy flux and the third-order m moments);
// all other rows are even.
__host__ __device__ constexpr bool mrt_odd(int k)
{
    return (k >= 3 && k <= 8) || k >= 16;
}

// MRT collision, Eq. mrt_collision with Guo's term in moment space:
//   m' = m - S (m - m_eq) + (I - S/2) M F~,   f' = f + M^-1 (m' - m).
// Written in closed form for this basis instead of as generic 19 x 19
// products:
//  * the moments of the deviations d = f - w come from the opposite-pair
//    sums (even rows) and differences (odd rows) with the rows' small
//    integer coefficients (checked against mrt_poly at compile time);
//  * the equilibrium moments of the polynomial f_eq(rho, v) (Eq. equilibrium)
//    in this basis are, with the weights' own moments (e 11, eps 3) removed:
//      e: -11 drho + 19 rho v^2     eps: 3 drho - 11/2 rho v^2
//      3p_xx: rho (3 v_x^2 - v^2)   3pi_xx: -1/2 of 3p_xx
//      p_ww: rho (v_y^2 - v_z^2)    pi_ww: -1/2 of p_ww
//      p_ab: rho v_a v_b            q_a: -2/3 rho v_a     m_a: 0
//  * the moments of Guo's term F~_i = w_i [3 (e_i - v) + 9 (e_i.v) e_i].F are
//      rho 0, j_a F_a, e 38 v.F, eps -11 v.F, q_a -2/3 F_a, m_a 0,
//      3p_xx 2 G_x, 3pi_xx -G_x with G_x = 3 v_x F_x - v.F,
//      p_ww 2 G_w, pi_ww -G_w with G_w = v_y F_y - v_z F_z,
//      p_ab v_a F_b + v_b F_a
//    (the second-order terms follow from 4th-order isotropy, the 6th-order
//    sums for pi vanish on D3Q19 like those of its equilibrium);
//  * the conserved rows need no rate: m - m_eq is 0 for rho and -F/2 for j
//    (v is Guo's force-shifted velocity), so m' - m is 0 and F for any s;
//  * the inverse M^-1 = M^T diag(1/|M_k|^2) is applied per opposite pair:
//    an even part shared by both members and an odd part of opposite sign.
// t_k = c_k (m_k - m_eq_k) - cf_k mf_k with c_k = s_k/|M_k|^2 and
// cf_k = (1 - s_k/2)/|M_k|^2 from the host; f' = f - M^T t.
// ---------------------------------------------------------------------------
namespace mrt_check {
// pair q of D3Q19 has the directions 2q+1 (e_q) and 2q+2 (-e_q): three axis
// pairs x, y, z, then xy (1,1,0), (1,-1,0), xz (1,0,1), (1,0,-1),
// yz (0,1,1), (0,1,-1).  Every coefficient the operator uses, by row k and
// direction i:
constexpr bool rows_ok()
{
    // even rows: rest, axis x, y, z, xy+, xy-, xz+, xz-, yz+, yz-
    constexpr int ev[10][10] = {
        /* e     */ {-30, -11, -11, -11, 8, 8, 8, 8, 8, 8},
        /* eps   */ {12, -4, -4, -4, 1, 1, 1, 1, 1, 1},
        /* 3pxx  */ {0, 2, -1, -1, 1, 1, 1, 1, -2, -2},
        /* 3pixx */ {0, -4, 2, 2, 1, 1, 1, 1, -2, -2},
        /* pww   */ {0, 0, 1, -1, 1, 1, -1, -1, 0, 0},
        /* piww  */ {0, 0, -2, 2, 1, 1, -1, -1, 0, 0},
        /* pxy   */ {0, 0, 0, 0, 1, -1, 0, 0, 0, 0},
        /* pyz   */ {0, 0, 0, 0, 0, 0, 0, 0, 1, -1},
        /* pxz   */ {0, 0, 0, 0, 0, 0, 1, -1, 0, 0},
        /* rho   */ {1, 1, 1, 1, 1, 1, 1, 1, 1, 1}};
    constexpr int evk[10] = {1, 2, 9, 10, 11, 12, 13, 14, 15, 0};
    // odd rows on the first member of each pair
    constexpr int od[9][9] = {
        /* jx */ {1, 0, 0, 1, 1, 1, 1, 0, 0},
        /* qx */ {-4, 0, 0, 1, 1, 1, 1, 0, 0},
        /* jy */ {0, 1, 0, 1, -1, 0, 0, 1, 1},
        /* qy */ {0, -4, 0, 1, -1, 0, 0, 1, 1},
        /* jz */ {0, 0, 1, 0, 0, 1, -1, 1, -1},
        /* qz */ {0, 0, -4, 0, 0, 1, -1, 1, -1},
        /* mx */ {0, 0, 0, 1, 1, -1, -1, 0, 0},
        /* my */ {0, 0, 0, -1, 1, 0, 0, 1, 1},
        /* mz */ {0, 0, 0, 0, 0, 1, -1, -1, 1}};
    constexpr int odk[9] = {3, 4, 5, 6, 7, 8, 16, 17, 18};
    for (int r = 0; r < 10; ++r) {
        if (mrt_odd(evk[r])) return false;
        if (mrt_M(evk[r], 0) != ev[r][0]) return false;
        for (int q = 0; q < 9; ++q)
            if (mrt_M(evk[r], 2 * q + 1) != ev[r][q + 1] ||
                mrt_M(evk[r], 2 * q + 2) != ev[r][q + 1])
                return false;
    }
    for (int r = 0; r < 9; ++r) {
        if (!mrt_odd(odk[r]) || mrt_M(odk[r], 0) != 0) return false;
        for (int q = 0; q < 9; ++q)
            if (mrt_M(odk[r], 2 * q + 1) != od[r][q] || mrt_M(odk[r], 2 * q + 2) != -od[r][q])
                return false;
    }
    return mrt_norm2(3) == 10 && mrt_norm2(5) == 10 && mrt_norm2(7) == 10;
}
static_assert(rows_ok(), "closed-form MRT rows disagree with the basis polynomials");
}  // namespace mrt_check

template <class R>
__host__ __device__ __forceinline__ void mrt_collide(R (&d)[19], const StepParams& p, R& drho_out,
                                                     R (&v)[3])
{
    // pair sums and differences; axis pairs 0..2, then the diagonal pairs
    R S[9], A[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        S[q] = d[2 * q + 1] + d[2 * q + 2];
        A[q] = d[2 * q + 1] - d[2 * q + 2];
    }
    const R Dxy = S[3] + S[4], Dxz = S[5] + S[6], Dyz = S[7] + S[8];
    const R Sax = (S[0] + S[1]) + S[2], Sdg = (Dxy + Dxz) + Dyz;
    const R drho = (d[0] + Sax) + Sdg;
    // diagonal parts of the odd rows (shared by j and q)
    const R Jx = (A[3] + A[4]) + (A[5] + A[6]);
    const R Jy = (A[3] - A[4]) + (A[7] + A[8]);
    const R Jz = (A[5] - A[6]) + (A[7] - A[8]);
    const R j0 = A[0] + Jx, j1 = A[1] + Jy, j2 = A[2] + Jz;
    const R rho = R(1) + drho;
    const R irho = R(1) / rho;
    const R F0 = sel<R>(p.F_f[0], p.F[0]), F1 = sel<R>(p.F_f[1], p.F[1]),
            F2 = sel<R>(p.F_f[2], p.F[2]);
    const bool force = p.has_force != 0;
    // Guo: rho v = j + F/2
    const R jF0 = fma(R(0.5), F0, j0), jF1 = fma(R(0.5), F1, j1), jF2 = fma(R(0.5), F2, j2);
    v[0] = jF0 * irho;
    v[1] = jF1 * irho;
    v[2] = jF2 * irho;
    const R rx = jF0 * v[0], ry = jF1 * v[1], rz = jF2 * v[2];   // rho v_a^2
    const R rusq = (rx + ry) + rz;                                // rho v^2
    auto c = [&](int k) { return sel<R>(p.mrt_c_f[k], p.mrt_c[k]); };
    auto cf = [&](int k) { return sel<R>(p.mrt_cf_f[k], p.mrt_cf[k]); };

    // non-equilibrium moments
    const R ne = fma(R(-30), d[0], fma(R(-11), Sax, R(8) * Sdg)) -
                 fma(R(-11), drho, R(19) * rusq);
    const R neps = fma(R(12), d[0], fma(R(-4), Sax, Sdg)) - fma(R(3), drho, R(-5.5) * rusq);
    const R pxx_eq = fma(R(2), rx, -(ry + rz));                   // rho (3 v_x^2 - v^2)
    const R pww_eq = ry - rz;
    const R a1 = fma(R(2), S[0], -(S[1] + S[2]));                 // axis part of 3p_xx
    const R a2 = (Dxy + Dxz) - R(2) * Dyz;                        // diagonal part of both
    const R npxx = (a1 + a2) - pxx_eq;
    const R npixx = fma(R(-2), a1, a2) + R(0.5) * pxx_eq;
    const R b1 = S[1] - S[2], b2 = Dxy - Dxz;
    const R npww = (b1 + b2) - pww_eq;
    const R npiww = fma(R(-2), b1, b2) + R(0.5) * pww_eq;
    const R npxy = (S[3] - S[4]) - jF0 * v[1];
    const R npyz = (S[7] - S[8]) - jF1 * v[2];
    const R npxz = (S[5] - S[6]) - jF0 * v[2];
    constexpr R k23 = R(2) / R(3);
    const R nqx = fma(R(-4), A[0], Jx) + k23 * jF0;
    const R nqy = fma(R(-4), A[1], Jy) + k23 * jF1;
    const R nqz = fma(R(-4), A[2], Jz) + k23 * jF2;
    const R nmx = (A[3] + A[4]) - (A[5] + A[6]);
    const R nmy = (A[4] - A[3]) + (A[7] + A[8]);
    const R nmz = (A[5] - A[6]) - (A[7] - A[8]);

    R te = c(1) * ne, teps = c(2) * neps, tpxx = c(9) * npxx, tpixx = c(10) * npixx;
    R tpww = c(11) * npww, tpiww = c(12) * npiww;
    R tpxy = c(13) * npxy, tpyz = c(14) * npyz, tpxz = c(15) * npxz;
    R tqx = c(4) * nqx, tqy = c(6) * nqy, tqz = c(8) * nqz;
    const R tmx = c(16) * nmx, tmy = c(17) * nmy, tmz = c(18) * nmz;
    // momentum rows: m' - m = F, |M_j|^2 = 10
    R tjx = R(0), tjy = R(0), tjz = R(0);
    if (force) {
        const R vF = fma(v[0], F0, fma(v[1], F1, v[2] * F2));
        const R Gx = fma(R(3) * v[0], F0, -vF);
        const R Gw = fma(v[1], F1, -(v[2] * F2));
        te = fma(-cf(1), R(38) * vF, te);
        teps = fma(cf(2), R(11) * vF, teps);
        tpxx = fma(-cf(9), R(2) * Gx, tpxx);
        tpixx = fma(cf(10), Gx, tpixx);
        tpww = fma(-cf(11), R(2) * Gw, tpww);
        tpiww = fma(cf(12), Gw, tpiww);
        tpxy = fma(-cf(13), fma(v[0], F1, v[1] * F0), tpxy);
        tpyz = fma(-cf(14), fma(v[1], F2, v[2] * F1), tpyz);
        tpxz = fma(-cf(15), fma(v[0], F2, v[2] * F0), tpxz);
        tqx = fma(cf(4), k23 * F0, tqx);
        tqy = fma(cf(6), k23 * F1, tqy);
        tqz = fma(cf(8), k23 * F2, tqz);
        tjx = R(-0.1) * F0;
        tjy = R(-0.1) * F1;
        tjz = R(-0.1) * F2;
    }

    // inverse transform, f' = f - M^T t
    d[0] -= fma(R(-30), te, R(12) * teps);
    const R Eax = fma(R(-11), te, R(-4) * teps);
    const R Edg = fma(R(8), te, teps);
    const R P1 = fma(R(2), tpixx, -tpxx);            // y and z axis pairs; x gets -2 P1
    const R W = fma(R(-2), tpiww, tpww);             // +y, -z
    const R Q1 = tpxx + tpixx, Q2 = tpww + tpiww;    // diagonal pairs
    const R X = tjx + tqx, Y = tjy + tqy, Z = tjz + tqz;
    R ev[9], od[9];
    ev[0] = fma(R(-2), P1, Eax);
    ev[1] = (Eax + P1) + W;
    ev[2] = (Eax + P1) - W;
    od[0] = fma(R(-4), tqx, tjx);
    od[1] = fma(R(-4), tqy, tjy);
    od[2] = fma(R(-4), tqz, tjz);
    const R exy = (Edg + Q1) + Q2, exz = (Edg + Q1) - Q2, eyz = fma(R(-2), Q1, Edg);
    ev[3] = exy + tpxy;
    ev[4] = exy - tpxy;
    ev[5] = exz + tpxz;
    ev[6] = exz - tpxz;
    ev[7] = eyz + tpyz;
    ev[8] = eyz - tpyz;
    od[3] = (X + Y) + (tmx - tmy);
    od[4] = (X - Y) + (tmx + tmy);
    od[5] = (X + Z) + (tmz - tmx);
    od[6] = (X - Z) - (tmx + tmz);
    od[7] = (Y + Z) + (tmy - tmz);
    od[8] = (Y - Z) + (tmy + tmz);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        d[2 * q + 1] -= ev[q] + od[q];
        d[2 * q + 2] -= ev[q] - od[q];
    }
    drho_out = drho;
}

// ---------------------------------------------------------------------------
// ELBM
// ---------------------------------------------------------------------------
// FP64 sum of the lattice weights in index order, folded at compile time.
template <class L>
__host__ __device__ constexpr double weight_sum()
{
    double s = 0.0;
    for (int i = 0; i < L::Q; ++i) s += L::w(i);
    return s;
}

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
// constant of dH/df).  This is the definition; LogEval evaluates it.
template <class L>
struct LogEval {
    const double* f;
    const double* x;
    double A;
    __host__ __device__ bool valid(double) const { return true; }
    __host__ __device__ void operator()(double a, double& g, double& gp) const
    {
        double s = 0, sp = 0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const double ax = a * x[i];
            const double l1 = log1p(ax);
            s = fma(f[i] * (1.0 + ax), l1, s);
            sp = fma(f[i] * x[i], l1, sp);
        }
        g = a * A + s;
        gp = A + sp;
    }
};

// The same g as a power series in a.  With a_k = sum_i f_i x_i^k and
// (1 + y) log1p(y) = y + sum_{k>=2} (-1)^k y^k / (k (k-1)) (|y| < 1):
//   g(a)  = a (A + a_1) + sum_{k=2}^{K} c_k a^k,   c_k = (-1)^k a_k / (k (k-1)),
//   g'(a) = (A + a_1) + sum_{k=2}^{K} k c_k a^(k-1).
// After one pass of FP64 multiply-adds per node every Newton evaluation is a
// K-term polynomial instead of q logarithms.  Used when max|x| <= 0.03 and
// for a <= 0.1 / max|x|, where the terms beyond K = 14 are below 1e-17 of
// a_2 (the scale of g'); an iterate outside that range falls back to LogEval.
constexpr int kSeriesK = 14;
constexpr int kSeriesK64 = 6;    // moments above this order are accumulated in FP32
constexpr double kSeriesMaxX = 0.03;
struct SeriesEval {
    double c[kSeriesK + 1];      // c_k, k = 2..K
    double A1;                   // A + a_1
    double amax;                 // largest a the truncation is accurate for
    __host__ __device__ bool valid(double a) const { return a <= amax; }
    __host__ __device__ void operator()(double a, double& g, double& gp) const
    {
        double p = c[kSeriesK], q = kSeriesK * c[kSeriesK];
#pragma unroll
        for (int k = kSeriesK - 1; k >= 2; --k) {
            p = fma(p, a, c[k]);
            q = fma(q, a, k * c[k]);
        }
        // p = sum c_k a^(k-2), q = sum k c_k a^(k-2)
        g = a * fma(a, p, A1);
        gp = fma(a, q, A1);
    }
};

// Eight lattice-symmetry invariants fed to the alpha surrogate, from the
// moments a_k = sum f x^k (k = 2..6), the extremes of x and A:
// t_k = (a_k / rho) / eps^k (k = 3..6), eps = sqrt(a_2 / rho),
// max x / eps, min x / eps, A / a_2.
// The features are inputs of an FP32 network and are stored as FP32 pairs,
// so they are formed in FP32 from the FP64 moments rounded to FP32.
__host__ __device__ __forceinline__ void elbm_features(const double (&ak)[7], double xmax,
                                                       double xmin, double rho, double A,
                                                       float (&feat)[8])
{
    const float a2 = narrow(ak[2]), ir = 1.0f / narrow(rho);
    const float eps = sqrtf(a2 * ir);
    const float ie = 1.0f / eps;
    const float ie2 = ie * ie;
    feat[0] = narrow(ak[3]) * ir * ie2 * ie;
    feat[1] = narrow(ak[4]) * ir * ie2 * ie2;
    feat[2] = narrow(ak[5]) * ir * ie2 * ie2 * ie;
    feat[3] = narrow(ak[6]) * ir * ie2 * ie2 * ie2;
    feat[4] = eps;
    feat[5] = narrow(xmax) * ie;
    feat[6] = narrow(xmin) * ie;
    feat[7] = narrow(A) / a2;
}

// MLP 8 -> 32 -> 32 -> 1 (tanh), parameters in shared memory (FP32 holding
// BF16-rounded weights), FP32 accumulation.  Returns the raw output.
__host__ __device__ __forceinline__ float mlp_eval(const float* __restrict__ P, const float (&feat)[8])
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
    for (int k = 0; k < 8; ++k) z[k] = (feat[k] - mean[k]) * istd[k];
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

// Guesses of the guarded alpha modes, from the moments a_k = sum f x^k
// (ak[0..6]) and A1 = A + a_1:
//   1  s2: the root of g(alpha)/alpha expanded about 2 to second order for an
//      f_eq that minimises H (then A = -sum f x ln(1 + x)),
//      s2 = 2 + (a_3 - 2 a_4) / (3 a_2) + 4 a_3^2 / (9 a_2^2);
//   2  s2 + scale * out: the surrogate learns what s2 misses;
//   4  the root of g(alpha)/alpha with g's series truncated after a_6 and the
//      node's own A (exact for any f_eq; three Newton steps from s2 on
//      h(a) = A1 + sum_{k=2}^{6} (-1)^k a_k a^(k-1) / (k (k-1))).
// A guess only seeds the FP64 Newton solve, which takes it after one FP64
// correction of at most guard_tol * alpha, so it is formed in FP32, on the
// moments divided by a_2: its rounding (~1e-7 of alpha) is well inside that
// bound, and the corrected alpha is off by about the correction squared.
// Below a_2 = 1e-30 (FP32's normal range ends at 1.2e-38) the guess is 2.
__host__ __device__ __forceinline__ double alpha_guess(const StepParams& p, const float* smlp,
                                                       const double (&ak)[7], double A1,
                                                       const float (&feat)[8])
{
    const float a2 = (float)ak[2];
    if (!(a2 > 1e-30f)) return 2.0;
    const float ia2 = 1.0f / a2;
    const float q3 = (float)ak[3] * ia2, q4 = (float)ak[4] * ia2;
    const float s2 = fmaf(4.0f / 9.0f, q3 * q3, fmaf(fmaf(-2.0f, q4, q3), 1.0f / 3.0f, 2.0f));
    if (p.alpha_mode == 2) return (double)fmaf(smlp[MLP_NPARAM - 1], mlp_eval(smlp, feat), s2);
    if (p.alpha_mode != 4) return (double)s2;
    // h / a_2 with c_2 / a_2 = 1/2
    const float c1 = (float)A1 * ia2, c3 = q3 * (-1.0f / 6.0f), c4 = q4 * (1.0f / 12.0f),
                c5 = (float)ak[5] * ia2 * (-1.0f / 20.0f), c6 = (float)ak[6] * ia2 * (1.0f / 30.0f);
    float a = s2;
#pragma unroll
    for (int it = 0; it < 3; ++it) {
        const float h = fmaf(a, fmaf(a, fmaf(a, fmaf(a, fmaf(a, c6, c5), c4), c3), 0.5f), c1);
        const float hp =
            fmaf(a, fmaf(a, fmaf(a, fmaf(a, 5.0f * c6, 4.0f * c5), 3.0f * c4), 2.0f * c3), 0.5f);
        a -= h / hp;
    }
    return (double)a;
}

struct AlphaResult {
    double alpha;
    int evals;
    int status;
    double resid;   // |g(alpha)| / a_2 with the logarithm form (diagnostic mode), else 0
};
constexpr int ALPHA_NEEDS_LOG = 100;   // internal: series range left, redo with logs

// Guarded alpha modes: start from a guess, and accept early.
__host__ __device__ __forceinline__ bool alpha_guarded(int mode)
{
    return mode == 1 || mode == 2 || mode == 4;
}

// Non-trivial root of g in [1, alpha_max) (Eq. alpha_cond) with evaluator ev.
// Safeguarded Newton keeps a bracket [lo, hi]: g < 0 below the root, >= 0 at
// or above it (g is convex with g(0) = 0).  If the positivity limit hi is
// reached with g(hi) < 0 there is no root below it and alpha = hi =
// alpha_max (1 - 1e-10).  Newton starts from alpha = 2, or in the guarded
// modes from the guess (second-order series, MLP or truncated-series root);
// these accept the first Newton correction of at most guard_tol * alpha
// within their first guard_steps evaluations (the corrected alpha is then
// off by about that correction squared), and otherwise continue from the
// bracket and iterate they have reached to the tolerance.
template <class Ev>
__host__ __device__ AlphaResult elbm_solve(const Ev& ev, double amax, const StepParams& p,
                                           double guess, int evals0)
{
    AlphaResult r{2.0, evals0, ALPHA_NOCONV};
    double lo = 1.0, hi = amax * (1.0 - 1e-10);
    bool hi_known = false;
    int evals = evals0;
    const bool guarded = alpha_guarded(p.alpha_mode);
    double a = guarded ? fmin(fmax(guess, lo), hi) : 2.0;
    if (!(a < hi)) a = 0.5 * (lo + hi);
    for (int it = 0; it < p.max_iter; ++it) {
        if (!ev.valid(a)) return AlphaResult{a, evals, ALPHA_NEEDS_LOG};
        double g, gp;
        ev(a, g, gp);
        ++evals;
        if (g == 0.0) { r.status = ALPHA_CONV; break; }
        if (g < 0) lo = a;
        else { hi = a; hi_known = true; }
        double an = (gp > 0) ? a - g / gp : -1.0;
        if (guarded && it < p.guard_steps && an > lo && an < hi &&
            fabs(an - a) <= p.guard_tol * a) {
            a = an;
            r.status = ALPHA_GUARDED;
            break;
        }
        // a step below the tolerance is the answer, even when rounding has
        // collapsed the bracket onto the root
        if (gp > 0 && fabs(an - a) <= p.tol * a) { a = an; r.status = ALPHA_CONV; break; }
        if (!(an > lo && an < hi)) {
            if (!hi_known && !(an < hi)) {
                if (!ev.valid(hi)) return AlphaResult{a, evals, ALPHA_NEEDS_LOG};
                double gh, gph;
                ev(hi, gh, gph);
                ++evals;
                if (gh < 0) { a = hi; r.status = ALPHA_CLAMP; break; }
                hi_known = true;
            }
            an = 0.5 * (lo + hi);
        }
        if (fabs(an - a) <= p.tol * a) { a = an; r.status = ALPHA_CONV; break; }
        a = an;
    }
    r.alpha = a;
    r.evals = evals;
    return r;
}

// Reciprocal in FP64 from an FP32 seed refined by two Newton-Raphson steps
// r <- r (2 - f r).  The seed, the FP32 reciprocal of f truncated to 24 bits,
// is within 2^-22 of 1/f; each step squares the relative error (2^-44, then
// below FP64 rounding).  f > 0, as the distributions of a valid state are.
__host__ __device__ __forceinline__ double recip_nr(double f);
// The same with one refinement step: relative error below 2^-46 (1.4e-14).
// The range is checked on the FP32 value the seed starts from, and the seed
// (a normal FP32 number there) is widened by integer operations: neither
// takes the FP64 pipe.
__host__ __device__ __forceinline__ double recip_nr1(double f)
{
    const float ff = (float)f;
    if (!(ff > 1e-30f && ff < 1e30f)) return 1.0 / f;   // outside the FP32 seed's range
    const double r = widen_normal(1.0f / ff);
    return r * fma(-f, r, 2.0);
}
// The same from an FP32 value fs of f formed without an FP64 conversion (the
// stored FP32 deviation plus the weight, in FP32): fs is within
// 2^-24 (1 + w / f) of f and the seed 1/fs within one more 2^-24, so one step
// leaves a relative error below (2 + w / f)^2 2^-48: 5.7e-14 where f >= w / 2,
// 5e-13 where f >= w / 10.
__host__ __device__ __forceinline__ double recip_nr1_seeded(double f, float fs)
{
    if (!(fs > 1e-30f && fs < 1e30f)) return 1.0 / f;   // outside the FP32 seed's range
    const double r = widen_normal(1.0f / fs);
    return r * fma(-f, r, 2.0);
}
__host__ __device__ __forceinline__ double recip_nr(double f)
{
    const float ff = narrow_trunc(f);   // 2^-23: two steps still reach FP64 rounding
    if (!(ff > 1e-30f && ff < 1e30f)) return 1.0 / f;   // outside the FP32 seed's range
    double r = widen_normal(1.0f / ff);
    r = r * fma(-f, r, 2.0);
    r = r * fma(-f, r, 2.0);
    return r;
}

// An FP64 result in the compute type R; to FP32 rounded to nearest on the
// integer pipes (the value of the conversion instruction).
template <class R>
__host__ __device__ __forceinline__ R to_compute(double v)
{
    if constexpr (sizeof(R) == 4)
        return narrow(v);
    else
        return (R)v;
}

// ELBM collision of one node.  d (deviations, compute type R) in/out.
// Returns the per-node outcome for the counters.
template <class L, class R>
__host__ __device__ __forceinline__ AlphaResult elbm_collide(R (&d)[L::Q], const StepParams& p,
                                                             const float* smlp, R& drho_out,
                                                             R (&vout)[3], float (&feat)[8],
                                                             bool& have_feat)
{
    double f[L::Q], x[L::Q], fe[L::Q], y[L::Q];
    double drho = 0, j[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        double di;
        if constexpr (sizeof(R) == 4)
            di = widen(d[i]);       // exact, on the integer pipes
        else
            di = (double)d[i];
        f[i] = L::w(i) + di;
        drho += di;
        j[0] += L::ex(i) * di;
        j[1] += L::ey(i) * di;
        j[2] += L::ez(i) * di;
    }
    const double rho = 1.0 + drho;
    const double irho = recip_nr(rho);
    double u[3] = {j[0] * irho, j[1] * irho, (L::D == 3) ? j[2] * irho : 0.0};
    // equilibrium; for the entropic form also its pieces: f_eq_i = P_i (1 + y_i)
    // with P_i = c0 w_i prod_a r_a^e_ia (ln(P_i / w_i) affine in e_i) and y_i the
    // relative mass/momentum restoration
    double lc0 = 0;
    const bool entropic = (p.feq_variant == 0);
    if (entropic) {
        double c[3], r[3], ri[3];
#pragma unroll
        for (int a = 0; a < L::D; ++a) {
            const double s = sqrt(1.0 + 3.0 * u[a] * u[a]);
            c[a] = 2.0 - s;
            r[a] = (2.0 * u[a] + s) * recip_nr(1.0 - u[a]);
            ri[a] = (1.0 - u[a]) * recip_nr(2.0 * u[a] + s);
        }
        const double c0 = (L::D == 3) ? rho * c[0] * c[1] * c[2] : rho * c[0] * c[1];
        const double ic0 = recip_nr(c0);
        double m0 = 0, m1[3] = {0, 0, 0};
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            double q = c0 * L::w(i), iq = ic0;        // P_i and (w_i / P_i)
            if (L::ex(i) == 1) { q *= r[0]; iq *= ri[0]; }
            if (L::ex(i) == -1) { q *= ri[0]; iq *= r[0]; }
            if (L::ey(i) == 1) { q *= r[1]; iq *= ri[1]; }
            if (L::ey(i) == -1) { q *= ri[1]; iq *= r[1]; }
            if (L::D == 3) {
                if (L::ez(i) == 1) { q *= r[2]; iq *= ri[2]; }
                if (L::ez(i) == -1) { q *= ri[2]; iq *= r[2]; }
            }
            fe[i] = q;
            y[i] = iq;
            m0 += q;
            m1[0] += L::ex(i) * q;
            m1[1] += L::ey(i) * q;
            m1[2] += L::ez(i) * q;
        }
        // put the residual mass and momentum back (zero up to rounding on
        // D2Q9, O(u^3) on D3Q19): the root of g shifts with f_eq's mass defect
        const double dr = rho - m0;
        const double dj0 = fma(rho, u[0], -m1[0]), dj1 = fma(rho, u[1], -m1[1]),
                     dj2 = fma(rho, u[2], -m1[2]);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const double corr = fma(3.0, L::ex(i) * dj0 + L::ey(i) * dj1 + L::ez(i) * dj2, dr);
            fe[i] = fma(L::w(i), corr, fe[i]);
            y[i] *= corr;                               // w_i corr / P_i
        }
        // ln c0 and ln r_a enter A only as ln c0 sum Delta and ln r_a
        // sum e_a Delta.  The restored f_eq carries f's momentum, so
        // sum e_a Delta vanishes up to rounding (~1e-19); its mass is
        // 1 + drho while f_i = w_i + d_i carries sum w_i + drho, so
        // sum Delta = 1 - sum w_i (an ulp of the FP64 weights) up to rounding.
        // A keeps ln c0 (1 - sum w_i); an FP32 logarithm changes it by ~1e-26.
        lc0 = (double)logf((float)c0);
    } else {
        elbm_feq<L>(rho, u, 1, fe);
    }
    // Delta_i = f_eq,i - f_i replaces f_eq in its registers; the update, A and
    // the moments take it as it is, and x_i = Delta_i / f_i
    double (&Dl)[L::Q] = fe;
    // extremes of x through integer order keys (exact; no FP64 comparisons)
    double xmin = 1e300, xmax = -1e300;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        // x_i to 1.4e-14 relative with FP64 storage: Delta_i = f_i x_i then
        // holds to FP64's own rounding level.  With FP32 storage, whose
        // stored values round at 6e-8, to ~6e-14 from an FP32 seed that needs
        // no FP64 conversion.
        Dl[i] = fe[i] - f[i];
        if constexpr (sizeof(R) == 4)   // FP32 storage: seed from the FP32 deviation
            x[i] = Dl[i] * recip_nr1_seeded(f[i], (float)L::w(i) + d[i]);
        else
            x[i] = Dl[i] * recip_nr1(f[i]);
        xmin = fmin(xmin, x[i]);
        xmax = fmax(xmax, x[i]);
    }
    const double maxabs = fmax(-xmin, xmax);   // max |x_i|, exactly
    AlphaResult ar{2.0, 0, ALPHA_SKIP};
    have_feat = false;
    // positivity limit: f_i + a f_i x_i > 0 for all i  <=>  a < -1 / min x
    const double amax = xmin < -1e-30 ? recip_nr(-xmin) : 1e300;
    if (p.alpha_mode != 3 && maxabs >= p.skip_eps && amax < 1e300) {
        // the invariant features feed the learned guess and the pair collection
        // only; the series and root guesses use the moments themselves
        const bool want_feat = p.alpha_mode == 2 || p.pairs_X != nullptr;
        double ak[7];
        double A = 0;
        bool solved = false;
        if (entropic && maxabs <= kSeriesMaxX) {
            // moments a_k and A from the series (no per-direction logarithm)
            // a_2..a_6 in FP64; a_7..a_14 in FP32.  With |a_k| <= max|x|^(k-2) a_2
            // and a max|x| <= 0.1 over the series' range, term k of g is at most
            // 2 (a max|x|)^(k-2) / (k (k-1)) of a^2 a_2 / 2: from k = 7 on below
            // 4.8e-7, so FP32's relative error (< 2e-6 after 14 products and 19
            // sums) moves g by less than 1e-12 of its scale, the Newton tolerance
            // on alpha, and by about 1e-13 at the roots met (alpha near 2 with
            // max|x| <= 0.03: a max|x| <= 0.07, term 7 below 4e-8).
            double a[kSeriesK + 1];
            float ahi[kSeriesK - kSeriesK64];
#pragma unroll
            for (int k = 0; k <= kSeriesK; ++k) a[k] = 0;
#pragma unroll
            for (int k = 0; k < kSeriesK - kSeriesK64; ++k) ahi[k] = 0.f;
            double sy = 0;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                double pw = Dl[i];
                a[1] += pw;
#pragma unroll
                for (int k = 2; k <= kSeriesK64; ++k) {
                    pw *= x[i];
                    a[k] += pw;
                }
                // x_i and f x^6 in FP32 without FP64 conversions: x_i
                // truncated to 24 bits by integer operations, f from the
                // stored deviation with FP32 storage (one more unit in the
                // last place, within the bound above)
                const float xf = narrow_trunc(x[i]);
                float pwf;
                if constexpr (sizeof(R) == 4) {
                    const float x3 = xf * xf * xf;
                    pwf = ((float)L::w(i) + d[i]) * (x3 * x3);
                } else {
                    pwf = (float)pw;
                }
#pragma unroll
                for (int k = 0; k < kSeriesK - kSeriesK64; ++k) {
                    pwf *= xf;
                    ahi[k] += pwf;
                }
                const double yi = y[i];
                sy = fma(Dl[i], yi * fma(-yi, fma(-yi, fma(-0.25, yi, 1.0 / 3.0), 0.5), 1.0), sy);
            }
#pragma unroll
            for (int k = 0; k < kSeriesK - kSeriesK64; ++k) a[kSeriesK64 + 1 + k] = widen(ahi[k]);
            // A = sum Delta ln(f_eq/w) - sum Delta log1p(x), with
            // sum Delta ln(f_eq/w) = ln c0 (1 - sum w) + sum Delta log1p(y)
            // (the ln r_a sum e_a Delta terms vanish, see above) and
            // sum Delta log1p(x) = sum_{n>=1} (-1)^(n+1) a_(n+1) / n
            double sl = 0;
#pragma unroll
            for (int n = kSeriesK - 1; n >= 1; --n)
                sl = fma(a[n + 1], ((n & 1) ? 1.0 : -1.0) * (1.0 / n), sl);
            A = fma(lc0, 1.0 - weight_sum<L>(), sy - sl);
            SeriesEval ev;
#pragma unroll
            for (int k = 2; k <= kSeriesK; ++k)
                ev.c[k] = a[k] * (((k & 1) ? -1.0 : 1.0) * (1.0 / (double)(k * (k - 1))));
            ev.c[0] = ev.c[1] = 0;
            ev.A1 = A + a[1];
            ev.amax = 0.1 / maxabs;
#pragma unroll
            for (int k = 0; k < 7; ++k) ak[k] = a[k];
            double guess = 2.0;
            if (want_feat) {
                elbm_features(ak, xmax, xmin, rho, A, feat);
                have_feat = true;
            }
            if (alpha_guarded(p.alpha_mode)) guess = alpha_guess(p, smlp, ak, ev.A1, feat);
            ar = elbm_solve(ev, amax, p, guess, 0);
            solved = (ar.status != ALPHA_NEEDS_LOG);
        }
        if (!solved) {
            // the definition: logarithms per direction
            A = 0;
#pragma unroll
            for (int k = 0; k < 7; ++k) ak[k] = 0;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                A += Dl[i] * log(f[i] / L::w(i));
                ak[1] += Dl[i];
                const double p2 = Dl[i] * x[i];
                ak[2] += p2;
                ak[3] += p2 * x[i];
                ak[4] += p2 * x[i] * x[i];
                ak[5] += p2 * x[i] * x[i] * x[i];
                ak[6] += p2 * x[i] * x[i] * x[i] * x[i];
            }
            double guess = 2.0;
            if (want_feat) {
                elbm_features(ak, xmax, xmin, rho, A, feat);
                have_feat = true;
            }
            if (alpha_guarded(p.alpha_mode)) guess = alpha_guess(p, smlp, ak, A + ak[1], feat);
            LogEval<L> ev{f, x, A};
            ar = elbm_solve(ev, amax, p, guess, ar.evals);
        }
        if (p.elbm_diag && (ar.status == ALPHA_CONV || ar.status == ALPHA_GUARDED)) {
            // entropy condition at the accepted alpha, by the definition
            // (per-direction logarithms): also measures the series truncation
            double Al = 0;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) Al = fma(Dl[i], log(f[i] / L::w(i)), Al);
            LogEval<L> evd{f, x, Al};
            double g, gp;
            evd(ar.alpha, g, gp);
            ar.resid = fabs(g) / ak[2];
        }
    }
    const double ab = ar.alpha * 0.5 * p.omega;     // alpha * beta, beta = 1/(2 tau)
    if (p.has_force) {
        // EDM, Eq. edm_force: f_eq(rho, u + F/rho) - f_eq(rho, u)
        double us[3] = {u[0] + p.F[0] * irho, u[1] + p.F[1] * irho,
                        (L::D == 3) ? u[2] + p.F[2] * irho : 0.0};
        double fs[L::Q];
        elbm_feq<L>(rho, us, p.feq_variant, fs);
#pragma unroll
        for (int i = 0; i < L::Q; ++i)   // f_eq(u + F/rho) - f_eq(u) added
            d[i] = to_compute<R>(fma(ab, Dl[i], f[i] - L::w(i)) + (fs[i] - (f[i] + Dl[i])));
    } else {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) d[i] = to_compute<R>(fma(ab, Dl[i], f[i] - L::w(i)));
    }
    drho_out = (R)drho;
    vout[0] = (R)(u[0] + 0.5 * p.F[0] * irho);
    vout[1] = (R)(u[1] + 0.5 * p.F[1] * irho);
    vout[2] = (L::D == 3) ? (R)(u[2] + 0.5 * p.F[2] * irho) : R(0);
    return ar;
}

}  // namespace lbm
