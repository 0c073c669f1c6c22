/*
 * Plain, slow FP64 CPU oracle of the lattice Boltzmann stream-and-collide step
 * (Januszewski & Kostur, "Sailfish: a flexible multi-GPU implementation of the
 * lattice Boltzmann method").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark load this file.  It shares no code, header, table
 * or constant with the CUDA library: its velocity sets are enumerated here from
 * {-1,0,1}^D, its MRT basis is evaluated here from the basis polynomials, and
 * the CUDA side has its own copies of everything.
 *
 * Every step is written in the paper's order and notation, node by node:
 *   streaming (pull form of the left side of Eq. lbgk; AB pattern, Sec. 3.3),
 *   half-way bounce-back (Sec. 2.3),
 *   moments (Eq. lb_macro), force-shifted velocity (Eq. edm_momentum),
 *   LBGK (Eq. lbgk with the relaxation toward f_eq as in Algorithm cnp),
 *   MRT (Eq. mrt_collision), ELBM (Eqs. elbm and alpha_cond),
 *   Guo forcing (Eq. guo_force) and EDM forcing (Eq. edm_force),
 *   regularized LBGK (Sec. 2.1.1) and LBGK with the Smagorinsky subgrid
 *   model (Sec. 2.1.4, Eqs. smagorinsky and taut).
 *
 * Readings of garbled or silent passages (each also listed in the design notes):
 *   - Eq. lbgk / Eq. elbm print "+(f - f_eq)/tau"; Algorithm cnp relaxes
 *     toward f_eq.  We relax toward f_eq.
 *   - The entropic equilibrium (Sec. 2.1.3) prints sqrt(1 + u^2) in its first
 *     factor; the form consistent with its own second factor and with the
 *     polynomial equilibrium at O(u^2) is sqrt(1 + 3 u^2).  We use 3 u^2.
 *   - On D3Q19 the product form is not the exact H-minimiser; we restore mass
 *     and momentum with f_eq_i += w_i (drho + 3 e_i . dj) (feq_variant 0), or
 *     use the polynomial f_eq (feq_variant 1).
 *   - alpha: non-trivial root of g(alpha) = H(f + alpha Delta) - H(f) in
 *     [1, alpha_max), found by safeguarded Newton; near-equilibrium nodes
 *     (max |x_i| < skip_eps) take alpha = 2; if no root lies below the
 *     positivity limit, alpha = alpha_max (1 - 1e-10).
 *   - MRT forcing: Guo's term in moment space with (I - S/2).  ELBM forcing:
 *     EDM with the model's own equilibrium.  Reported velocity is always
 *     v = (j + F/2) / rho.
 *   - MRT basis: the orthogonal D3Q19 moment polynomials of d'Humieres et al.
 *     (2002), the reference the MRT subsection defers to.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OQMAX 27

/* ------------------------------------------------------------------ */
/* Lattices: Sec. 2, Fig. lattices and Table bgkweights.               */
/* ------------------------------------------------------------------ */
typedef struct {
    int D, Q;
    int e[OQMAX][3];
    double w[OQMAX];
    int opp[OQMAX];
} olat;

/* Enumerate e in {-1,0,1}^D and keep the links whose squared length the
 * lattice uses (Sec. 2, Fig. lattices): D2Q9 all nine; D3Q15 lengths 0, 1,
 * sqrt 3; D3Q19 lengths 0, 1, sqrt 2; D3Q27 all.  Weights by link length from
 * Table bgkweights (a negative entry marks an unused length). */
static int olat_build(olat* L, int D, int Q)
{
    double w_by_len2[4];
    if (D == 2 && Q == 9) {
        w_by_len2[0] = 4.0 / 9.0; w_by_len2[1] = 1.0 / 9.0; w_by_len2[2] = 1.0 / 36.0;
        w_by_len2[3] = -1.0;
    } else if (D == 3 && Q == 15) {
        w_by_len2[0] = 2.0 / 9.0; w_by_len2[1] = 1.0 / 9.0; w_by_len2[2] = -1.0;
        w_by_len2[3] = 1.0 / 72.0;
    } else if (D == 3 && Q == 19) {
        w_by_len2[0] = 1.0 / 3.0; w_by_len2[1] = 1.0 / 18.0; w_by_len2[2] = 1.0 / 36.0;
        w_by_len2[3] = -1.0;
    } else if (D == 3 && Q == 27) {
        w_by_len2[0] = 8.0 / 27.0; w_by_len2[1] = 2.0 / 27.0; w_by_len2[2] = 1.0 / 54.0;
        w_by_len2[3] = 1.0 / 216.0;
    } else {
        return -1;
    }
    L->D = D;
    int q = 0;
    int zlo = (D == 3) ? -1 : 0, zhi = (D == 3) ? 1 : 0;
    for (int ez = zlo; ez <= zhi; ++ez)
        for (int ey = -1; ey <= 1; ++ey)
            for (int ex = -1; ex <= 1; ++ex) {
                int n2 = ex * ex + ey * ey + ez * ez;
                if (w_by_len2[n2] < 0.0) continue;
                L->e[q][0] = ex; L->e[q][1] = ey; L->e[q][2] = ez;
                L->w[q] = w_by_len2[n2];
                ++q;
            }
    L->Q = q;
    for (int i = 0; i < q; ++i)
        for (int k = 0; k < q; ++k)
            if (L->e[k][0] == -L->e[i][0] && L->e[k][1] == -L->e[i][1] &&
                L->e[k][2] == -L->e[i][2])
                L->opp[i] = k;
    return q;
}

/* Lattice by code: 2 = D2Q9, 3 = D3Q19 (the dimension's default), 15 =
 * D3Q15, 19 = D3Q19, 27 = D3Q27, 9 = D2Q9. */
static const olat* get_lattice(int code)
{
    static olat L9, L15, L19, L27;
    static int built = 0;
    if (!built) {           /* tables are tiny; building twice is harmless */
        olat_build(&L9, 2, 9);
        olat_build(&L15, 3, 15);
        olat_build(&L19, 3, 19);
        olat_build(&L27, 3, 27);
        built = 1;
    }
    switch (code) {
    case 2: case 9: return &L9;
    case 3: case 19: return &L19;
    case 15: return &L15;
    case 27: return &L27;
    default: return NULL;
    }
}

/* the lattice of a parameter block: q selects it, else the dimension's default */
#define PLAT(p) get_lattice((p)->q ? (p)->q : (p)->D)

static double edot(const olat* L, int i, const double* u)
{
    double s = 0.0;
    for (int a = 0; a < L->D; ++a) s += L->e[i][a] * u[a];
    return s;
}

/* ------------------------------------------------------------------ */
/* Equilibria.                                                          */
/* ------------------------------------------------------------------ */

/* Eq. equilibrium: rho w_i (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u^2). */
static void feq_poly(const olat* L, double rho, const double* u, double* feq)
{
    double u2 = 0.0;
    for (int a = 0; a < L->D; ++a) u2 += u[a] * u[a];
    for (int i = 0; i < L->Q; ++i) {
        double eu = edot(L, i, u);
        feq[i] = rho * L->w[i] * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * u2);
    }
}

/* Entropic equilibrium (Sec. 2.1.3), read with sqrt(1 + 3 u_a^2):
 *   rho w_i prod_a (2 - sqrt(1 + 3 u_a^2)) ((2 u_a + sqrt(1 + 3 u_a^2)) / (1 - u_a))^{e_ia}. */
static void feq_entropic_product(const olat* L, double rho, const double* u, double* feq)
{
    double c[3], r[3];
    for (int a = 0; a < L->D; ++a) {
        double s = sqrt(1.0 + 3.0 * u[a] * u[a]);
        c[a] = 2.0 - s;
        r[a] = (2.0 * u[a] + s) / (1.0 - u[a]);
    }
    for (int i = 0; i < L->Q; ++i) {
        double p = rho * L->w[i];
        for (int a = 0; a < L->D; ++a) {
            p *= c[a];
            if (L->e[i][a] == 1) p *= r[a];
            else if (L->e[i][a] == -1) p /= r[a];
        }
        feq[i] = p;
    }
}

/* The product form with the mass and momentum residuals put back along the
 * first two Hermite directions: f_i += w_i (drho + 3 e_i . dj).  On D2Q9 the
 * residuals are zero to rounding (the product form is the exact minimiser
 * there); on D3Q19 they are O(u^3). */
static void feq_entropic(const olat* L, double rho, const double* u, double* feq)
{
    feq_entropic_product(L, rho, u, feq);
    double m0 = 0.0, m1[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < L->Q; ++i) {
        m0 += feq[i];
        for (int a = 0; a < L->D; ++a) m1[a] += L->e[i][a] * feq[i];
    }
    double drho = rho - m0, dj[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < L->D; ++a) dj[a] = rho * u[a] - m1[a];
    for (int i = 0; i < L->Q; ++i)
        feq[i] += L->w[i] * (drho + 3.0 * edot(L, i, dj));
}

/* ------------------------------------------------------------------ */
/* MRT basis (D3Q19): the orthogonal moment polynomials of d'Humieres,  */
/* Ginzburg, Krafczyk, Lallemand and Luo (2002), in their moment order: */
/* rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy,    */
/* pyz, pxz, mx, my, mz.                                                */
/* ------------------------------------------------------------------ */
static double mrt_row(int k, int ex, int ey, int ez)
{
    double x = ex, y = ey, z = ez, e2 = x * x + y * y + z * z;
    switch (k) {
    case 0: return 1.0;
    case 1: return 19.0 * e2 - 30.0;
    case 2: return (21.0 * e2 * e2 - 53.0 * e2 + 24.0) / 2.0;
    case 3: return x;
    case 4: return (5.0 * e2 - 9.0) * x;
    case 5: return y;
    case 6: return (5.0 * e2 - 9.0) * y;
    case 7: return z;
    case 8: return (5.0 * e2 - 9.0) * z;
    case 9: return 3.0 * x * x - e2;
    case 10: return (3.0 * e2 - 5.0) * (3.0 * x * x - e2);
    case 11: return y * y - z * z;
    case 12: return (3.0 * e2 - 5.0) * (y * y - z * z);
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return x * (y * y - z * z);
    case 17: return y * (z * z - x * x);
    case 18: return z * (x * x - y * y);
    }
    return 0.0;
}

typedef struct {
    double M[19][19];
    double Minv[19][19];
} omrt;

/* Gauss-Jordan inverse with partial pivoting (a library-style step). */
static int invert19(double A[19][19], double Ainv[19][19])
{
    double a[19][38];
    for (int r = 0; r < 19; ++r)
        for (int c = 0; c < 38; ++c)
            a[r][c] = (c < 19) ? A[r][c] : (c - 19 == r ? 1.0 : 0.0);
    for (int col = 0; col < 19; ++col) {
        int piv = col;
        for (int r = col + 1; r < 19; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (fabs(a[piv][col]) < 1e-300) return -1;
        if (piv != col)
            for (int c = 0; c < 38; ++c) {
                double t = a[col][c]; a[col][c] = a[piv][c]; a[piv][c] = t;
            }
        double d = a[col][col];
        for (int c = 0; c < 38; ++c) a[col][c] /= d;
        for (int r = 0; r < 19; ++r) {
            if (r == col) continue;
            double m = a[r][col];
            if (m == 0.0) continue;
            for (int c = 0; c < 38; ++c) a[r][c] -= m * a[col][c];
        }
    }
    for (int r = 0; r < 19; ++r)
        for (int c = 0; c < 19; ++c) Ainv[r][c] = a[r][c + 19];
    return 0;
}

static const omrt* get_mrt(void)
{
    static omrt T;
    static int built = 0;
    if (!built) {
        const olat* L = get_lattice(3);
        for (int k = 0; k < 19; ++k)
            for (int i = 0; i < 19; ++i)
                T.M[k][i] = mrt_row(k, L->e[i][0], L->e[i][1], L->e[i][2]);
        invert19(T.M, T.Minv);
        built = 1;
    }
    return &T;
}

/* ------------------------------------------------------------------ */
/* Parameters (mirrored field by field by the Python loader).           */
/* ------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz;
    int D;            /* 2: D2Q9, 3: D3Q19 */
    int model;        /* 0 LBGK, 1 MRT, 2 ELBM */
    int alpha_mode;   /* ELBM: 0 Newton from 2, 1 series guess + guarded Newton,
                         2 MLP guess + guarded Newton, 3 alpha fixed at 2,
                         4 truncated-series root guess + guarded Newton */
    int max_iter;     /* Newton evaluation cap */
    int feq_variant;  /* ELBM: 0 entropic (restored on D3Q19), 1 polynomial */
    int nthreads;     /* OpenMP threads for oracle_run; 0 = runtime default */
    int guard_steps;  /* guarded modes: evaluations that may end in early acceptance */
    double tau;
    double force[3];
    double s[19];     /* MRT rates, d'Humieres moment order */
    double tol;       /* Newton: stop when |alpha_{n+1} - alpha_n| <= tol alpha_n */
    double skip_eps;  /* alpha = 2 when max_i |x_i| < skip_eps */
    double guard_tol; /* guarded modes: accept a correction <= guard_tol alpha */
    const double* mlp;/* MLP parameters for alpha_mode 2 */
    double smag_cs;   /* Smagorinsky constant C_S (model 4) */
    int q;            /* velocity set: 0 = D2Q9 / D3Q19 by D, or 9, 15, 19, 27 */
    /* velocity / pressure boundary conditions, entry k for mask code 2 + k */
    int bc_kind[15];      /* 1 velocity, 2 pressure */
    int bc_method[15];    /* 0 equilibrium, 1 Zou-He, 2 regularized */
    int bc_normal[15];    /* inward normal: +-1 x, +-2 y, +-3 z */
    double bc_val[15][3]; /* velocity, or the density in [0] */
} oracle_params;

/* Per-node ELBM outcome. */
enum { AL_CONV = 0, AL_SKIP = 1, AL_CLAMP = 2, AL_NOCONV = 3, AL_FIXED = 4, AL_GUARDED = 5 };

/* ------------------------------------------------------------------ */
/* ELBM: Eqs. elbm and alpha_cond.                                      */
/* ------------------------------------------------------------------ */

/* g(alpha) = H(f + alpha Delta) - H(f) with H = sum f ln(f/w), written
 * termwise: f_i + alpha Delta_i = f_i (1 + alpha x_i), x_i = Delta_i / f_i, so
 *   (f+aD) ln((f+aD)/w) - f ln(f/w) = a D ln(f/w) + (f + a D) log1p(a x).
 * g'(alpha) = sum D_i (ln(f_i/w_i) + log1p(alpha x_i) + 1). */
static void elbm_g(const olat* L, const double* f, const double* d, const double* lnfw,
                   double alpha, double* g, double* gp)
{
    double G = 0.0, Gp = 0.0;
    for (int i = 0; i < L->Q; ++i) {
        double x = d[i] / f[i];
        double l1 = log1p(alpha * x);
        G += alpha * d[i] * lnfw[i] + (f[i] + alpha * d[i]) * l1;
        Gp += d[i] * (lnfw[i] + l1 + 1.0);
    }
    *g = G;
    *gp = Gp;
}

/* Eight lattice-symmetry invariants of (f, Delta) that the alpha surrogate
 * reads, and the moments a_k = sum f x^k used by the series guess.
 *   eps = sqrt(a2 / rho), t_k = (a_k / rho) / eps^k (k = 3..6),
 *   xmax / eps, xmin / eps, A / a2 with A = sum Delta ln(f / w). */
static void elbm_features(const olat* L, const double* f, const double* d,
                          const double* lnfw, double rho, double* feat, double* ak)
{
    double a[7] = {0, 0, 0, 0, 0, 0, 0};
    double xmax = -1e300, xmin = 1e300, A = 0.0;
    for (int i = 0; i < L->Q; ++i) {
        double x = d[i] / f[i];
        double p = f[i] * x * x;
        for (int k = 2; k <= 6; ++k) {
            a[k] += p;
            p *= x;
        }
        if (x > xmax) xmax = x;
        if (x < xmin) xmin = x;
        A += d[i] * lnfw[i];
    }
    double eps = sqrt(a[2] / rho);
    feat[0] = (a[3] / rho) / (eps * eps * eps);
    feat[1] = (a[4] / rho) / (eps * eps * eps * eps);
    feat[2] = (a[5] / rho) / (eps * eps * eps * eps * eps);
    feat[3] = (a[6] / rho) / (eps * eps * eps * eps * eps * eps);
    feat[4] = eps;
    feat[5] = xmax / eps;
    feat[6] = xmin / eps;
    feat[7] = A / a[2];
    if (ak)
        for (int k = 0; k < 7; ++k) ak[k] = a[k];
}

/* Second-order small-deviation guess: the root of g(alpha)/alpha expanded
 * about alpha = 2 to second order in the moments a_k = sum f x^k, for an f_eq
 * that minimises H (then A = -sum f x ln(1 + x)). */
static double series2_guess(const double* ak)
{
    return 2.0 + (ak[3] - 2.0 * ak[4]) / (3.0 * ak[2]) + 4.0 * ak[3] * ak[3] / (9.0 * ak[2] * ak[2]);
}

/* Root of g(alpha)/alpha with the series of g truncated after a_6 and the
 * node's own A (exact for any f_eq, not only the H minimiser):
 *   h(alpha) = A + a_1 + sum_{k=2}^{6} (-1)^k a_k alpha^(k-1) / (k (k-1)),
 * three Newton steps on h from the second-order guess. */
static double series_root_guess(const double* ak, double A1)
{
    double a = series2_guess(ak);
    for (int it = 0; it < 3; ++it) {
        double h = A1, hp = 0.0;
        for (int k = 2; k <= 6; ++k) {
            const double c = ((k % 2) ? -1.0 : 1.0) * ak[k] / (double)(k * (k - 1));
            h += c * pow(a, k - 1);
            hp += (k - 1) * c * pow(a, k - 2);
        }
        a -= h / hp;
    }
    return a;
}

/* The same second-order guess from the surrogate's features (t_3, t_4 and
 * eps = sqrt(a_2 / rho)): (a_3 - 2 a_4) / (3 a_2) = (t_3 eps - 2 t_4 eps^2) / 3
 * and 4 a_3^2 / (9 a_2^2) = 4 t_3^2 eps^2 / 9. */
static double series2_from_features(const double* feat)
{
    const double t3 = feat[0], t4 = feat[1], eps = feat[4];
    return 2.0 + (t3 * eps - 2.0 * t4 * eps * eps) / 3.0 + 4.0 * t3 * t3 * eps * eps / 9.0;
}

/* MLP 8 -> 32 -> 32 -> 1, tanh hidden units (parameter layout documented in
 * the Python loader).  The network learns what the second-order guess s2
 * misses: alpha guess = s2 + scale * out. */
#define MLP_IN 8
#define MLP_H 32
static double mlp_guess(const double* P, const double* feat, double s2)
{
    const double* mean = P;
    const double* istd = P + 8;
    const double* W1 = P + 16;
    const double* b1 = W1 + MLP_H * MLP_IN;
    const double* W2 = b1 + MLP_H;
    const double* b2 = W2 + MLP_H * MLP_H;
    const double* W3 = b2 + MLP_H;
    const double* b3 = W3 + MLP_H;
    const double* scale = b3 + 1;
    double z[MLP_IN], h1[MLP_H], h2[MLP_H];
    for (int k = 0; k < MLP_IN; ++k) z[k] = (feat[k] - mean[k]) * istd[k];
    for (int o = 0; o < MLP_H; ++o) {
        double s = b1[o];
        for (int k = 0; k < MLP_IN; ++k) s += W1[o * MLP_IN + k] * z[k];
        h1[o] = tanh(s);
    }
    for (int o = 0; o < MLP_H; ++o) {
        double s = b2[o];
        for (int k = 0; k < MLP_H; ++k) s += W2[o * MLP_H + k] * h1[k];
        h2[o] = tanh(s);
    }
    double out = b3[0];
    for (int k = 0; k < MLP_H; ++k) out += W3[k] * h2[k];
    return s2 + scale[0] * out;
}

/* Solve Eq. alpha_cond for the non-trivial root.  out[0] = alpha,
 * out[1] = g evaluations, out[2] = status, out[3] = |g(alpha)| / a2 at the
 * returned alpha (one extra evaluation, diagnostics only). */
static void elbm_alpha(const olat* L, const oracle_params* p, const double* f,
                       const double* feq, double rho, double* out)
{
    double d[OQMAX], lnfw[OQMAX], x[OQMAX];
    double maxabs = 0.0, amax = INFINITY;
    for (int i = 0; i < L->Q; ++i) {
        d[i] = feq[i] - f[i];
        x[i] = d[i] / f[i];
        if (fabs(x[i]) > maxabs) maxabs = fabs(x[i]);
        if (d[i] < 0.0) {
            double lim = -f[i] / d[i];
            if (lim < amax) amax = lim;
        }
        lnfw[i] = log(f[i] / L->w[i]);
    }
    out[1] = 0.0;
    out[3] = 0.0;
    if (p->alpha_mode == 3) {
        out[0] = 2.0; out[2] = AL_FIXED;
        return;
    }
    if (maxabs < p->skip_eps || !(amax < INFINITY)) {
        out[0] = 2.0; out[2] = AL_SKIP;
        return;
    }
    double hi = amax * (1.0 - 1e-10), lo = 1.0;
    int hi_known = 0;          /* g(hi) >= 0 established */
    int evals = 0;
    double alpha = 2.0;
    int status = AL_NOCONV;

    double feat[8], ak[7];
    const int guarded = p->alpha_mode == 1 || p->alpha_mode == 2 || p->alpha_mode == 4;
    if (guarded) {
        elbm_features(L, f, d, lnfw, rho, feat, ak);
        double guess;
        if (p->alpha_mode == 1) {
            guess = series2_guess(ak);
        } else if (p->alpha_mode == 2) {
            guess = mlp_guess(p->mlp, feat, series2_guess(ak));
        } else {
            double A1 = 0.0;           /* A + a_1, a_1 = sum Delta */
            for (int i = 0; i < L->Q; ++i) A1 += d[i] * lnfw[i] + d[i];
            guess = series_root_guess(ak, A1);
        }
        alpha = guess;
        if (!(alpha > lo)) alpha = lo;
        if (!(alpha < hi)) alpha = hi;
    }

    /* Safeguarded Newton on the convex g (g(0) = 0, g < 0 on (0, alpha*),
     * g > 0 beyond) from 2, or from the guess: keep a bracket [lo, hi], step
     * by Newton when it stays inside, otherwise bisect.  The guarded modes
     * accept the first Newton correction of at most guard_tol alpha within
     * their first guard_steps evaluations (one more Newton step from there
     * squares that error); otherwise the solve continues to the tolerance. */
    if (!(alpha < hi)) alpha = 0.5 * (lo + hi);
    for (int it = 0; it < p->max_iter; ++it) {
        double g, gp;
        elbm_g(L, f, d, lnfw, alpha, &g, &gp);
        ++evals;
        if (g == 0.0) { status = AL_CONV; break; }
        if (g < 0.0) lo = alpha;
        else { hi = alpha; hi_known = 1; }
        double an = (gp > 0.0) ? alpha - g / gp : NAN;
        if (guarded && it < p->guard_steps && an > lo && an < hi &&
            fabs(an - alpha) <= p->guard_tol * alpha) {
            alpha = an;
            status = AL_GUARDED;
            break;
        }
        /* a step already below the tolerance ends the solve; testing the
         * bracket first would reject a sub-ulp step at the root itself */
        if (fabs(an - alpha) <= p->tol * alpha) { alpha = an; status = AL_CONV; break; }
        if (!(an > lo && an < hi)) {
            if (!hi_known && !(an < hi)) {
                /* Newton points past the positivity limit: is there a root? */
                double gh, gph;
                elbm_g(L, f, d, lnfw, hi, &gh, &gph);
                ++evals;
                if (gh < 0.0) { alpha = hi; status = AL_CLAMP; break; }
                hi_known = 1;
            }
            an = 0.5 * (lo + hi);
        }
        if (fabs(an - alpha) <= p->tol * alpha) { alpha = an; status = AL_CONV; break; }
        alpha = an;
    }
done:
    out[0] = alpha;
    out[1] = evals;
    out[2] = status;
    {
        double g, gp, a2 = 0.0;
        elbm_g(L, f, d, lnfw, alpha, &g, &gp);
        for (int i = 0; i < L->Q; ++i) a2 += f[i] * x[i] * x[i];
        out[3] = fabs(g) / a2;
    }
}

/* ------------------------------------------------------------------ */
/* Collision of one node (post-streaming f in, post-collision f out).   */
/* info = {alpha, evals, status, |g|/a2} for ELBM.                      */
/* ------------------------------------------------------------------ */
/* ------------------------------------------------------------------ */
/* Velocity and pressure boundary nodes (Sec. 2.3: equilibrium, Zou-He and  */
/* regularized variants).                                                   */
/* ------------------------------------------------------------------ */
/* A boundary node is a fluid node next to the outside of the domain; n is its
 * inward unit normal along a lattice axis.  After streaming, the populations
 * with e_i . n > 0 came from outside and are unknown; the others are known.
 * Mass and normal momentum of the known ones fix the missing moment:
 *   rho (1 - v_n) = S_0 + 2 S_out - F_n / 2,
 * S_0 = sum over e_i . n = 0, S_out = sum over e_i . n < 0, with the momentum
 * j = rho v - F/2 of Guo's scheme (Eq. edm_momentum read backwards), so that
 * the collision reports exactly the prescribed v.  Velocity condition: v
 * given, rho from the relation; pressure condition: rho given, v = v_n n with
 * v_n from the relation (no tangential velocity).  Then, with f_eq at (rho, v):
 *   equilibrium: f_i = f_eq_i - (3/2) w_i e_i . F (all i);
 *   Zou-He: unknown f_i = f_opp(i) + f_eq_i - f_eq_opp(i) (bounce-back of the
 *     non-equilibrium part), then the momentum left over, dJ = j - sum f e,
 *     goes to the unknown populations: its normal part to the one along n,
 *     each tangential part t split evenly, with sign e_it, over the unknown
 *     populations with e_it != 0 of the smallest |e| (D2Q9, D3Q19, D3Q27:
 *     the two edge links; D3Q15: the four body diagonals);
 *   regularized: unknown f_i as in Zou-He before the correction, then all
 *     f_i = f_eq_i + w_i / (2 c_s^4) (e_i e_i - c_s^2 I) : Pi^neq
 *     - (3/2) w_i e_i . F, Pi^neq = sum (f - f_eq) e e. */
static void bc_node(const olat* L, const oracle_params* p, int id, double* f)
{
    const int Q = L->Q, D = L->D;
    const int ax = abs(p->bc_normal[id]) - 1, sg = p->bc_normal[id] > 0 ? 1 : -1;
    const double* F = p->force;
    double S0 = 0.0, So = 0.0;
    for (int i = 0; i < Q; ++i) {
        int en = sg * L->e[i][ax];
        if (en == 0) S0 += f[i];
        else if (en < 0) So += f[i];
    }
    const double Fn = sg * F[ax];
    double rho, v[3] = {0.0, 0.0, 0.0};
    if (p->bc_kind[id] == 1) {
        for (int a = 0; a < D; ++a) v[a] = p->bc_val[id][a];
        rho = (S0 + 2.0 * So - 0.5 * Fn) / (1.0 - sg * v[ax]);
    } else {
        rho = p->bc_val[id][0];
        v[ax] = sg * (1.0 - (S0 + 2.0 * So - 0.5 * Fn) / rho);
    }
    double feq[OQMAX];
    feq_poly(L, rho, v, feq);
    const int method = p->bc_method[id];
    if (method == 0) {
        for (int i = 0; i < Q; ++i) f[i] = feq[i] - 1.5 * L->w[i] * edot(L, i, F);
        return;
    }
    for (int i = 0; i < Q; ++i)
        if (sg * L->e[i][ax] > 0) f[i] = f[L->opp[i]] + feq[i] - feq[L->opp[i]];
    if (method == 1) {
        double dJ[3];
        for (int a = 0; a < D; ++a) {
            double s = 0.0;
            for (int i = 0; i < Q; ++i) s += L->e[i][a] * f[i];
            dJ[a] = rho * v[a] - 0.5 * F[a] - s;
        }
        for (int i = 0; i < Q; ++i) {      /* the link along n */
            int on = 1;
            for (int a = 0; a < D; ++a) on &= (L->e[i][a] == (a == ax ? sg : 0));
            if (on) f[i] += sg * dJ[ax];
        }
        for (int t = 0; t < D; ++t) {
            if (t == ax) continue;
            int best = 99, cnt = 0;
            for (int i = 0; i < Q; ++i)
                if (sg * L->e[i][ax] > 0 && L->e[i][t] != 0) {
                    int n2 = 0;
                    for (int a = 0; a < D; ++a) n2 += L->e[i][a] * L->e[i][a];
                    if (n2 < best) { best = n2; cnt = 0; }
                    if (n2 == best) ++cnt;
                }
            for (int i = 0; i < Q; ++i)
                if (sg * L->e[i][ax] > 0 && L->e[i][t] != 0) {
                    int n2 = 0;
                    for (int a = 0; a < D; ++a) n2 += L->e[i][a] * L->e[i][a];
                    if (n2 == best) f[i] += L->e[i][t] * dJ[t] / cnt;
                }
        }
        return;
    }
    double Pi[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b)
                Pi[a][b] += (f[i] - feq[i]) *
                            (L->e[i][a] * L->e[i][b] - (a == b ? 1.0 / 3.0 : 0.0));
    for (int i = 0; i < Q; ++i) {
        double pr = 0.0;
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b)
                pr += (L->e[i][a] * L->e[i][b] - (a == b ? 1.0 / 3.0 : 0.0)) * Pi[a][b];
        f[i] = feq[i] + 4.5 * L->w[i] * pr - 1.5 * L->w[i] * edot(L, i, F);
    }
}

static int collide_node(const olat* L, const oracle_params* p, double* f, double* rho_out,
                        double* v_out, double* info)
{
    int Q = L->Q, D = L->D;
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {           /* Eq. lb_macro */
        rho += f[i];
        for (int a = 0; a < D; ++a) j[a] += L->e[i][a] * f[i];
    }
    const double* F = p->force;
    double v[3] = {0.0, 0.0, 0.0}, u[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < D; ++a) {
        u[a] = j[a] / rho;                     /* Eq. lb_macro */
        v[a] = (j[a] + 0.5 * F[a]) / rho;      /* Eq. edm_momentum */
    }
    double feq[OQMAX];
    if (p->model == 0) {
        /* LBGK with Guo forcing: Eqs. lbgk, equilibrium, guo_force. */
        feq_poly(L, rho, v, feq);
        for (int i = 0; i < Q; ++i) {
            double ev = edot(L, i, v), fi = 0.0;
            for (int a = 0; a < D; ++a)
                fi += (3.0 * (L->e[i][a] - v[a]) + 9.0 * ev * L->e[i][a]) * F[a];
            f[i] = f[i] + (feq[i] - f[i]) / p->tau + (1.0 - 0.5 / p->tau) * L->w[i] * fi;
        }
    } else if (p->model == 1) {
        /* MRT, Eq. mrt_collision, with Guo's term taken to moment space:
         * m' = m - S (m - m_eq) + (I - S/2) M Ft,  f' = M^-1 m'. */
        if (L->Q != 19) return -1;
        const omrt* T = get_mrt();
        double Ft[OQMAX], m[19], meq[19], mF[19], mp[19];
        feq_poly(L, rho, v, feq);
        for (int i = 0; i < Q; ++i) {
            double ev = edot(L, i, v), fi = 0.0;
            for (int a = 0; a < D; ++a)
                fi += (3.0 * (L->e[i][a] - v[a]) + 9.0 * ev * L->e[i][a]) * F[a];
            Ft[i] = L->w[i] * fi;
        }
        for (int k = 0; k < 19; ++k) {
            m[k] = meq[k] = mF[k] = 0.0;
            for (int i = 0; i < 19; ++i) {
                m[k] += T->M[k][i] * f[i];
                meq[k] += T->M[k][i] * feq[i];
                mF[k] += T->M[k][i] * Ft[i];
            }
            mp[k] = m[k] - p->s[k] * (m[k] - meq[k]) + (1.0 - 0.5 * p->s[k]) * mF[k];
        }
        for (int i = 0; i < 19; ++i) {
            double s = 0.0;
            for (int k = 0; k < 19; ++k) s += T->Minv[i][k] * mp[k];
            f[i] = s;
        }
    } else if (p->model == 2) {
        /* ELBM, Eq. elbm: f' = f + alpha beta (f_eq - f), beta = 1/(2 tau),
         * then EDM forcing, Eq. edm_force. */
        if (p->feq_variant == 0) feq_entropic(L, rho, u, feq);
        else feq_poly(L, rho, u, feq);
        double al[4];
        elbm_alpha(L, p, f, feq, rho, al);
        double beta = 0.5 / p->tau;
        for (int i = 0; i < Q; ++i) f[i] = f[i] + al[0] * beta * (feq[i] - f[i]);
        if (F[0] != 0.0 || F[1] != 0.0 || F[2] != 0.0) {
            double us[3] = {0.0, 0.0, 0.0}, fs[OQMAX];
            for (int a = 0; a < D; ++a) us[a] = u[a] + F[a] / rho;
            if (p->feq_variant == 0) feq_entropic(L, rho, us, fs);
            else feq_poly(L, rho, us, fs);
            for (int i = 0; i < Q; ++i) f[i] += fs[i] - feq[i];
        }
        if (info)
            for (int k = 0; k < 4; ++k) info[k] = al[k];
    } else if (p->model == 3 || p->model == 4) {
        /* Non-equilibrium momentum flux Pi_ab = sum_i (f_i - fe_i)(e_ia e_ib
         * - delta_ab c_s^2), c_s^2 = 1/3, about an equilibrium fe of the
         * node's own mass (so the delta term drops out):
         *  REG (Sec. 2.1.1): fe = f_eq(rho, u), u = j / rho, so that f - fe
         *    carries no mass and no momentum; the populations are replaced by
         *    fe_i + f_reg_i, f_reg_i = w_i / (2 c_s^4) (e_ia e_ib - c_s^2
         *    delta_ab) Pi_ab, and the LBGK collision with Guo's force then
         *    acts on them: f' = f~ + (f_eq(rho, v) - f~) / tau + Guo term.
         *  SMAG (Sec. 2.1.4): fe = f_eq(rho, v), the collision's own
         *    equilibrium, Pi = Q of Eq. taut; LBGK with tau0 + tau_t. */
        feq_poly(L, rho, v, feq);
        double fe[OQMAX];
        if (p->model == 3) feq_poly(L, rho, u, fe);
        else
            for (int i = 0; i < Q; ++i) fe[i] = feq[i];
        double Pi[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int i = 0; i < Q; ++i) {
            double fn = f[i] - fe[i];
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b)
                    Pi[a][b] += fn * (L->e[i][a] * L->e[i][b] - (a == b ? 1.0 / 3.0 : 0.0));
        }
        double tau = p->tau;
        if (p->model == 4) {
            /* Eq. taut: tau_t = (sqrt(tau0^2 + 4 C_S^2 |Q| / c_s^4) - tau0) / 2,
             * |Q| = (Q_ab Q_ab)^(1/2); total relaxation time tau0 + tau_t
             * (Eq. smagorinsky with nu_t = tau_t / 3). */
            double qq = 0.0;
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) qq += Pi[a][b] * Pi[a][b];
            double tau_t = 0.5 * (sqrt(p->tau * p->tau + 4.0 * 9.0 * p->smag_cs * p->smag_cs *
                                       sqrt(qq)) - p->tau);
            tau = p->tau + tau_t;
            if (info) info[0] = tau;
        }
        for (int i = 0; i < Q; ++i) {
            double ev = edot(L, i, v), fi = 0.0;
            for (int a = 0; a < D; ++a)
                fi += (3.0 * (L->e[i][a] - v[a]) + 9.0 * ev * L->e[i][a]) * F[a];
            double guo = (1.0 - 0.5 / tau) * L->w[i] * fi;
            double ft = f[i];
            if (p->model == 3) {
                double pr = 0.0;
                for (int a = 0; a < D; ++a)
                    for (int b = 0; b < D; ++b)
                        pr += (L->e[i][a] * L->e[i][b] - (a == b ? 1.0 / 3.0 : 0.0)) * Pi[a][b];
                ft = fe[i] + L->w[i] * 4.5 * pr;
            }
            f[i] = ft + (feq[i] - ft) / tau + guo;
        }
    } else {
        return -1;
    }
    *rho_out = rho;
    for (int a = 0; a < 3; ++a) v_out[a] = (a < D) ? v[a] : 0.0;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Public entry points (ctypes).                                        */
/* ------------------------------------------------------------------ */

/* Velocity set in this file's enumeration order.  Returns Q. */
int oracle_lattice(int D, int* e, double* w, int* opp)
{
    const olat* L = get_lattice(D);
    if (!L) return -1;
    for (int i = 0; i < L->Q; ++i) {
        for (int a = 0; a < 3; ++a) e[3 * i + a] = L->e[i][a];
        w[i] = L->w[i];
        opp[i] = L->opp[i];
    }
    return L->Q;
}

/* kind: 0 polynomial, 1 entropic product (as printed, with the 3u^2 reading),
 * 2 entropic with mass/momentum restored. */
int oracle_feq(int D, int kind, double rho, const double* u, double* feq)
{
    const olat* L = get_lattice(D);
    if (!L) return -1;
    double uu[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < L->D; ++a) uu[a] = u[a];
    if (kind == 0) feq_poly(L, rho, uu, feq);
    else if (kind == 1) feq_entropic_product(L, rho, uu, feq);
    else if (kind == 2) feq_entropic(L, rho, uu, feq);
    else return -1;
    return 0;
}

/* D3Q19 moment matrix and its inverse, columns in this file's velocity order. */
int oracle_mrt_matrix(double* M, double* Minv)
{
    const omrt* T = get_mrt();
    for (int k = 0; k < 19; ++k)
        for (int i = 0; i < 19; ++i) {
            M[19 * k + i] = T->M[k][i];
            Minv[19 * k + i] = T->Minv[k][i];
        }
    return 0;
}

/* One node: f (Q values, post-streaming) -> post-collision f in place. */
int oracle_collide(const oracle_params* p, double* f, double* rho, double* v, double* info)
{
    const olat* L = PLAT(p);
    if (!L) return -1;
    double inf4[4] = {0, 0, 0, 0};
    int r = collide_node(L, p, f, rho, v, inf4);
    if (info)
        for (int k = 0; k < 4; ++k) info[k] = inf4[k];
    return r;
}

/* One boundary node's reconstruction (condition id) on post-streaming f. */
int oracle_bc_node(const oracle_params* p, int id, double* f)
{
    const olat* L = PLAT(p);
    if (!L || id < 0 || id >= 15 || (p->bc_kind[id] != 1 && p->bc_kind[id] != 2)) return -1;
    bc_node(L, p, id, f);
    return 0;
}

/* g(alpha) and g'(alpha) for given f and f_eq (diagnostics / pins). */
int oracle_elbm_g(int D, const double* f, const double* feq, double alpha, double* g, double* gp)
{
    const olat* L = get_lattice(D);
    if (!L) return -1;
    double d[OQMAX], lnfw[OQMAX];
    for (int i = 0; i < L->Q; ++i) {
        d[i] = feq[i] - f[i];
        lnfw[i] = log(f[i] / L->w[i]);
    }
    elbm_g(L, f, d, lnfw, alpha, g, gp);
    return 0;
}

/* alpha solve for given f and f_eq; out = {alpha, evals, status, |g|/a2}. */
int oracle_elbm_alpha(const oracle_params* p, const double* f, const double* feq, double* out)
{
    const olat* L = PLAT(p);
    if (!L) return -1;
    double rho = 0.0;
    for (int i = 0; i < L->Q; ++i) rho += f[i];
    elbm_alpha(L, p, f, feq, rho, out);
    return 0;
}

/* Features (8) and a_k (k = 0..6) for given f and f_eq. */
int oracle_elbm_features(int D, const double* f, const double* feq, double* feat, double* ak)
{
    const olat* L = get_lattice(D);
    if (!L) return -1;
    double d[OQMAX], lnfw[OQMAX], rho = 0.0;
    for (int i = 0; i < L->Q; ++i) {
        d[i] = feq[i] - f[i];
        lnfw[i] = log(f[i] / L->w[i]);
        rho += f[i];
    }
    elbm_features(L, f, d, lnfw, rho, feat, ak);
    return 0;
}

/* MLP guess for a feature vector (FP64). */
double oracle_mlp_guess(const double* P, const double* feat)
{
    return mlp_guess(P, feat, series2_from_features(feat));
}

/* Truncated-series root guess from the moments a_0..a_6 and A + a_1. */
double oracle_series_root_guess(const double* ak, double A1)
{
    return series_root_guess(ak, A1);
}

/* F[q][z][y][x] = f_eq(rho, u) with the model's equilibrium (polynomial for
 * LBGK and MRT; ELBM's own for ELBM).  u is [D][z][y][x]. */
int oracle_init(const oracle_params* p, const double* rho, const double* u, double* F)
{
    const olat* L = PLAT(p);
    if (!L) return -1;
    size_t N = (size_t)p->nx * p->ny * p->nz;
    for (size_t n = 0; n < N; ++n) {
        double uu[3] = {0.0, 0.0, 0.0}, feq[OQMAX];
        for (int a = 0; a < L->D; ++a) uu[a] = u[a * N + n];
        if (p->model == 2 && p->feq_variant == 0) feq_entropic(L, rho[n], uu, feq);
        else feq_poly(L, rho[n], uu, feq);
        for (int i = 0; i < L->Q; ++i) F[i * N + n] = feq[i];
    }
    return 0;
}

/* nsteps AB steps: F (post-collision state at t) -> F at t + nsteps.
 * Ftmp is scratch of the same size.  rho, u ([D][z][y][x]) receive the
 * macroscopic fields of the last step; alpha (may be NULL) the last step's
 * per-node alpha.  mask (may be NULL): 0 fluid, 1 solid, 2 + k a boundary
 * node of condition k (bc_* entries of the parameters).  Solid nodes
 * get F = 0, rho = 0, u = 0.  stats (may be NULL, 6 doubles): total g
 * evaluations, skipped, clamped, not converged, guarded-accepted, nodes. */
int oracle_run(const oracle_params* p, double* F, double* Ftmp, const uint8_t* mask,
               int nsteps, double* rho, double* u, double* alpha, double* stats)
{
    const olat* L = PLAT(p);
    if (!L) return -1;
    if (p->model == 1 && L->Q != 19) return -1;
    const int nx = p->nx, ny = p->ny, nz = p->nz, Q = L->Q, D = L->D;
    const size_t N = (size_t)nx * ny * nz;
    double st[6] = {0, 0, 0, 0, 0, 0};
    if (p->model == 1) get_mrt();   /* build the tables before the parallel loop */
#ifdef _OPENMP
    if (p->nthreads > 0) omp_set_num_threads(p->nthreads);
#endif
    double* A = F;
    double* B = Ftmp;
    for (int step = 0; step < nsteps; ++step) {
        const int last = (step == nsteps - 1);
        double s_ev = 0, s_skip = 0, s_clamp = 0, s_nc = 0, s_gu = 0, s_n = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : s_ev, s_skip, s_clamp, s_nc, s_gu, s_n)
#endif
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    size_t n = ((size_t)z * ny + y) * nx + x;
                    if (mask && mask[n] == 1) {
                        for (int i = 0; i < Q; ++i) B[i * N + n] = 0.0;
                        if (last) {
                            rho[n] = 0.0;
                            for (int a = 0; a < D; ++a) u[a * N + n] = 0.0;
                            if (alpha) alpha[n] = 0.0;
                        }
                        continue;
                    }
                    /* Pull streaming with periodic wrap; half-way bounce-back
                     * when the upstream node is solid (Sec. 2.3). */
                    double f[OQMAX];
                    for (int i = 0; i < Q; ++i) {
                        int sx = ((x - L->e[i][0]) % nx + nx) % nx;
                        int sy = ((y - L->e[i][1]) % ny + ny) % ny;
                        int sz = ((z - L->e[i][2]) % nz + nz) % nz;
                        size_t src = ((size_t)sz * ny + sy) * nx + sx;
                        if (mask && mask[src] == 1) f[i] = A[L->opp[i] * N + n];
                        else f[i] = A[i * N + src];
                    }
                    if (mask && mask[n] >= 2) bc_node(L, p, mask[n] - 2, f);
                    double r, v[3], info[4] = {0, 0, 0, 0};
                    collide_node(L, p, f, &r, v, info);
                    for (int i = 0; i < Q; ++i) B[i * N + n] = f[i];
                    if (p->model == 2) {
                        s_ev += info[1];
                        s_skip += (info[2] == AL_SKIP);
                        s_clamp += (info[2] == AL_CLAMP);
                        s_nc += (info[2] == AL_NOCONV);
                        s_gu += (info[2] == AL_GUARDED);
                    }
                    s_n += 1;
                    if (last) {
                        rho[n] = r;
                        for (int a = 0; a < D; ++a) u[a * N + n] = v[a];
                        if (alpha) alpha[n] = info[0];
                    }
                }
        st[0] += s_ev; st[1] += s_skip; st[2] += s_clamp; st[3] += s_nc; st[4] += s_gu;
        st[5] += s_n;
        double* t = A; A = B; B = t;
    }
    if (A != F) memcpy(F, A, sizeof(double) * N * Q);
    if (stats)
        for (int k = 0; k < 6; ++k) stats[k] = st[k];
    return 0;
}

/* Number of OpenMP threads oracle_run would use (1 without OpenMP). */
int oracle_max_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) return nthreads;
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}
