/*
 * hsma_oracle.c -- plain, slow, FP64 CPU oracle of the harmonic surface mapping
 * algorithm (HSMA) for the reaction potential of a spherical cavity embedded in a
 * linearized Poisson-Boltzmann continuum (Fu & Gan, arXiv:1907.01724).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, import or call
 * this file: only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Every function follows the paper's definitions step by step, in the paper's
 * order and notation, with no blocking, fusion or reordering:
 *   Sec. 2.2  modified spherical Hankel function k_n (finite sum), S_n, Kirkwood M_n
 *   Sec. 2.3  decomposition M_n = gamma + dbar/(n+sigma) + hat M_n
 *   Sec. 2.4  modified Kelvin image q_K, modified coefficient hat M'_n,
 *             truncated correction potential, Green's second identity with the
 *             central difference for dG/dnu, Fibonacci quadrature, discrete images
 *   Sec. 4.1  self energy E_self = Phi_RF(x_s, x_s)/2
 *   fields    E = -grad phi of the same source set (the gradient of the
 *             potential the paper defines, for forces F_i = q_i E(x_i))
 *
 * Readings of the paper that this file takes (the paper is silent or ambiguous):
 *   - Units: the paper's expansions use Phi = q/(4 pi eps1 r).  The prefactor
 *     1/(4 pi) is the parameter coulomb_k (all results are linear in it).
 *   - hat M'_n depends on the charge through r_K,i (Sec. 2.4), so the correction
 *     potential is summed charge by charge.
 *   - The correction potential is evaluated with the addition theorem
 *     sum_m Y*_nm(x_i) Y_nm(y) = (2n+1)/(4 pi) P_n(cos angle), i.e. in Legendre
 *     pair form, which is algebraically the coefficient sum of Sec. 2.4.
 *   - Truncation at order p keeps n = 0..p.
 *   - A charge at the centre (r_i = 0) has its Kelvin image at infinity; its
 *     image term is the limit (coulomb_k/eps1)(q/a)(gamma - dbar/2), a constant,
 *     and only n = 0 survives in its correction series (with the limit
 *     hat M'_0 = M_0 - gamma + dbar/2).
 *   - The dipole shells use the quadrature weights of the auxiliary sphere
 *     (the central difference sits inside the integral over that sphere).
 *   - Energy: E_total = 1/2 sum_i q_i [ sum_{j != i} k q_j/(eps1 r_ij) + Phi_RF(x_i) ],
 *     E_RF = 1/2 sum_i q_i Phi_RF(x_i); Neumaier-compensated sums.
 *   - Images only near the interface (a variant the paper motivates in Sec. 2.3:
 *     the image terms matter for charges close to the interface): a charge with
 *     r_i < image_rel R gets no Kelvin image and no line image, and its whole
 *     reaction potential is the truncated series with the full M_n, i.e.
 *     hat M'_{n,i} = M_n (c_i = -gamma in the notation below); image_rel = 0 is
 *     the paper's method (every charge has its image).
 *   - dipole_form = 0 evaluates the three shells as literal point charges (eq.
 *     threeintegrals after quadrature); dipole_form = 1 evaluates the same
 *     difference (1/d_- - 1/d_+)/dy through the exact rewrite
 *     2 (R_tau - x.yhat) / (d_+ d_- (d_+ + d_-)), which avoids cancellation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846264338327950288

typedef struct {
    double a;          /* cavity radius R */
    double eps1;       /* dielectric constant inside */
    double eps2;       /* dielectric constant outside */
    double kappa;      /* inverse Debye length outside */
    int p;             /* truncation order, n = 0..p */
    int F1, F2;        /* successive Fibonacci numbers of the quadrature */
    double tau;        /* R_tau = (1 + tau) R */
    double dy_rel;     /* dy = dy_rel * R_tau */
    double coulomb_k;  /* 1/(4 pi) in the paper's units */
    int dipole_form;   /* 0 literal shells, 1 fused rewrite */
    int nthreads;      /* OpenMP threads (<= 0: library default) */
    double image_rel;  /* charges with r_i < image_rel R get no Kelvin image (0: every charge) */
} oracle_params;

/* ------------------------------------------------------------------------ */
/* Sec. 2.2: k_n(mu) = pi e^{-mu}/(2 mu) sum_{l=0}^{n} (n+l)!/(l!(n-l)!) (2mu)^{-l}.
 * S_n(mu) = k_n(mu) / (mu k_n'(mu)).
 * Differentiating the finite sum term by term,
 *   mu k_n'(mu) = pi e^{-mu}/2 * [ -(1 + 1/mu) sum_l c_l (2mu)^{-l}
 *                                 - (1/mu) sum_l l c_l (2mu)^{-l} ],
 * so that  S_n = - Sigma0 / ( (mu + 1) Sigma0 + Sigma1 )  with
 *   Sigma0 = sum_l c_l (2mu)^{-l},  Sigma1 = sum_l l c_l (2mu)^{-l}.
 * Both sums are divided by their common positive factor c_n (2mu)^{-n}, which
 * cancels in the ratio and keeps every term finite (also at mu = 0, where only
 * l = n survives and S_n = -1/(n+1)).  The terms t_l = c_l (2mu)^{n-l} / c_n
 * satisfy t_n = 1, t_l = t_{l+1} * 2 mu (l+1) / ((n+l+1)(n-l)).               */
double oracle_Sn(int n, double mu)
{
    double sigma0 = 0.0, sigma1 = 0.0, t = 1.0;
    for (int l = n; l >= 0; --l) {
        sigma0 += t;
        sigma1 += (double)l * t;
        if (l > 0)
            t = t * 2.0 * mu * (double)l / ((double)(n + l) * (double)(n - l + 1));
    }
    return -sigma0 / ((mu + 1.0) * sigma0 + sigma1);
}

/* Eq. Anuapp1: M_n = (eps (n+1) S_n + 1) / (eps n S_n - 1), eps = eps1/eps2. */
double oracle_Mn(int n, double eps, double mu)
{
    double S = oracle_Sn(n, mu);
    return (eps * (double)(n + 1) * S + 1.0) / (eps * (double)n * S - 1.0);
}

/* Sec. 2.3: gamma = (eps-1)/(eps+1), sigma = (1+mu)/(1+eps),
 * dbar = gamma (1 - sigma) - mu/(1+eps).                                    */
void oracle_decomposition(double eps, double mu, double* gamma, double* sigma, double* dbar)
{
    double g = (eps - 1.0) / (eps + 1.0);
    double s = (1.0 + mu) / (1.0 + eps);
    *gamma = g;
    *sigma = s;
    *dbar = g * (1.0 - s) - mu / (1.0 + eps);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.4, Fibonacci integration on a sphere of radius R:
 *   oint f dS ~ (2 pi R^2 / F2) sum_{j=0}^{F2} [1 + cos(pi z_j)] [f(y_{2j+1}) + f(y_{2j+2})],
 *   z_j = -1 + 2j/F2,  theta_j = arccos(z_j + sin(pi z_j)/pi),
 *   phi_{2j+1} = pi j F1/F2,  phi_{2j+2} = pi + pi j F1/F2.
 * Writes 2(F2+1) points (row-major x,y,z) on the sphere of radius R and their
 * weights; points y_{2j+1} and y_{2j+2} are stored at 2j and 2j+1.          */
int oracle_fibonacci(int F1, int F2, double R, double* pts, double* w)
{
    if (F2 <= 0 || F1 < 0) return -1;
    for (int j = 0; j <= F2; ++j) {
        double z = -1.0 + 2.0 * (double)j / (double)F2;
        double c = z + sin(ORACLE_PI * z) / ORACLE_PI;
        if (c > 1.0) c = 1.0;
        if (c < -1.0) c = -1.0;
        double theta = acos(c);
        double weight = 2.0 * ORACLE_PI * R * R / (double)F2 * (1.0 + cos(ORACLE_PI * z));
        for (int s = 0; s < 2; ++s) {
            double phi = ORACLE_PI * (double)j * (double)F1 / (double)F2 + (s ? ORACLE_PI : 0.0);
            double* y = pts + 3 * (2 * j + s);
            y[0] = R * sin(theta) * cos(phi);
            y[1] = R * sin(theta) * sin(phi);
            y[2] = R * cos(theta);
            w[2 * j + s] = weight;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.4 sources.  For each charge: Kelvin point r_K,i = (R/r_i)^2 x_i and the
 * trapezoid-modified image strength
 *   q_K,i = (q_i/R) [ gamma r_K,i + dbar (R_tau - r_K,i)/2 ].
 * The correction potential truncated at p (eq. phim with the addition theorem),
 *   Phi_corr(y) = sum_i k q_i/(eps1 R) sum_{n=0}^{p} hat M'_{n,i} (|y|/r_K,i)^n P_n(xhat_i . yhat),
 *   hat M'_{n,i} = M_n - gamma - dbar (R_tau - r_K,i)/(2 r_K,i),
 * and its radial derivative are evaluated at the Fibonacci points y_j of the
 * auxiliary sphere R_tau.  Outputs (any pointer may be NULL):
 *   kel_xyz [n*3], kel_q [n]     Kelvin image positions and q_K (not scaled by k/eps1;
 *                                zero strength for r_i = 0, whose term is r0_const)
 *   surf_xyz [M*3], surf_w [M]   Fibonacci points on the sphere R_tau and weights
 *   surf_phi [M], surf_dphi [M]  Phi_corr and dPhi_corr/dr at those points
 *   r0_const                     sum over centre charges of (k/eps1)(q/R)(gamma - dbar/2)
 * M = 2(F2+1).                                                              */
static double legendre_next(int n, double t, double Pn, double Pnm1)
{
    /* Bonnet: (n+1) P_{n+1} = (2n+1) t P_n - n P_{n-1} */
    return ((2.0 * n + 1.0) * t * Pn - (double)n * Pnm1) / (double)(n + 1);
}

int oracle_build(const oracle_params* P, int64_t n, const double* xyz, const double* q,
                 double* kel_xyz, double* kel_q,
                 double* surf_xyz, double* surf_w, double* surf_phi, double* surf_dphi,
                 double* r0_const)
{
    const double a = P->a;
    const double eps = P->eps1 / P->eps2;
    const double mu = P->kappa * a;
    const double Rtau = (1.0 + P->tau) * a;
    const int p = P->p;
    const int M = 2 * (P->F2 + 1);
    double gamma, sigma, dbar;
    oracle_decomposition(eps, mu, &gamma, &sigma, &dbar);
    (void)sigma;

    double* Mn = (double*)malloc(sizeof(double) * (size_t)(p + 1));
    for (int k = 0; k <= p; ++k) Mn[k] = oracle_Mn(k, eps, mu);

    /* Kelvin images */
    double c0 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double* x = xyz + 3 * i;
        double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        if (P->image_rel > 0.0 && r < P->image_rel * a) {
            /* no image: the charge's reaction potential is all in the series */
            if (kel_xyz) { kel_xyz[3 * i] = 0.0; kel_xyz[3 * i + 1] = 0.0; kel_xyz[3 * i + 2] = 0.0; }
            if (kel_q) kel_q[i] = 0.0;
            continue;
        }
        if (r == 0.0) {
            c0 += P->coulomb_k / P->eps1 * q[i] / a * (gamma - 0.5 * dbar);
            if (kel_xyz) { kel_xyz[3 * i] = 0.0; kel_xyz[3 * i + 1] = 0.0; kel_xyz[3 * i + 2] = 0.0; }
            if (kel_q) kel_q[i] = 0.0;
            continue;
        }
        double rK = a * a / r;
        double s = (a / r) * (a / r);
        if (kel_xyz) {
            kel_xyz[3 * i] = s * x[0];
            kel_xyz[3 * i + 1] = s * x[1];
            kel_xyz[3 * i + 2] = s * x[2];
        }
        if (kel_q) kel_q[i] = q[i] / a * (gamma * rK + dbar * (Rtau - rK) / 2.0);
    }
    if (r0_const) *r0_const = c0;

    /* Fibonacci points on the auxiliary sphere */
    double* pts = (double*)malloc(sizeof(double) * 3 * (size_t)M);
    double* w = (double*)malloc(sizeof(double) * (size_t)M);
    oracle_fibonacci(P->F1, P->F2, Rtau, pts, w);
    if (surf_xyz) memcpy(surf_xyz, pts, sizeof(double) * 3 * (size_t)M);
    if (surf_w) memcpy(surf_w, w, sizeof(double) * (size_t)M);

    /* Phi_corr and its radial derivative at the points (Legendre pair form) */
    if (surf_phi || surf_dphi) {
        int64_t Mj = M;
#ifdef _OPENMP
        if (P->nthreads > 0) omp_set_num_threads(P->nthreads);
#pragma omp parallel for schedule(static)
#endif
        for (int64_t j = 0; j < Mj; ++j) {
            const double* y = pts + 3 * j;
            double rho = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
            double phi = 0.0, dphi = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                const double* x = xyz + 3 * i;
                double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
                double pref = P->coulomb_k * q[i] / (P->eps1 * a);
                int no_image = P->image_rel > 0.0 && r < P->image_rel * a;
                if (r == 0.0) {
                    /* limit r_K -> infinity: only n = 0, hat M'_0 = M_0 - gamma + dbar/2
                       (M_0 for a charge without image) */
                    phi += pref * (no_image ? Mn[0] : Mn[0] - gamma + 0.5 * dbar);
                    continue;
                }
                double rK = a * a / r;
                double corr_i = no_image ? -gamma : dbar * (Rtau - rK) / (2.0 * rK);
                double t = (x[0] * y[0] + x[1] * y[1] + x[2] * y[2]) / (r * rho);
                double u = rho / rK; /* (|y| / r_K,i) */
                double Pn = 1.0, Pnm1 = 0.0, un = 1.0;
                double sphi = 0.0, sdphi = 0.0;
                for (int k = 0; k <= p; ++k) {
                    double Mhat = Mn[k] - gamma - corr_i;
                    sphi += Mhat * un * Pn;
                    /* d/d|y| (|y|/r_K)^k = k |y|^{k-1} / r_K^k = k u^k / |y| */
                    sdphi += Mhat * (double)k * un / rho * Pn;
                    double Pnext = legendre_next(k, t, Pn, Pnm1);
                    Pnm1 = Pn;
                    Pn = Pnext;
                    un *= u;
                }
                phi += pref * sphi;
                dphi += pref * sdphi;
            }
            if (surf_phi) surf_phi[j] = phi;
            if (surf_dphi) surf_dphi[j] = dphi;
        }
    }
    free(pts);
    free(w);
    free(Mn);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Potentials at nt target points (eq. phirffinall plus the Coulomb part):
 *   phi_coul(t) = sum_{j != self(t)} k q_j / (eps1 |t - x_j|)
 *   phi_rf(t)   = sum_j k q_K,j / (eps1 |t - r_K,j|) + r0_const
 *               + sum_l [ w_l dPhi_l/(4 pi) / |t - y_l|
 *                         + w_l Phi_l/(4 pi dy) ( 1/|t - y_l^-| - 1/|t - y_l^+| ) ]
 * with y_l^{+-} = (R_tau +- dy/2) yhat_l, dy = dy_rel R_tau (eqs. approxG,
 * threeintegrals, phicorrfinall).  self_index[t] is the charge that target t is
 * (excluded from the Coulomb sum), or -1; self_index may be NULL (no exclusion).
 * Any source array may be NULL to leave that part out.                      */
int oracle_eval(const oracle_params* P, int64_t n, const double* xyz, const double* q,
                const double* kel_xyz, const double* kel_q,
                int64_t M, const double* surf_xyz, const double* surf_w,
                const double* surf_phi, const double* surf_dphi, double r0_const,
                int64_t nt, const double* txyz, const int64_t* self_index,
                double* phi_coul, double* phi_rf)
{
    const double kc = P->coulomb_k / P->eps1;
    const double Rtau = (1.0 + P->tau) * P->a;
    const double dy = P->dy_rel * Rtau;
    const double inv4pi = 1.0 / (4.0 * ORACLE_PI);
#ifdef _OPENMP
    if (P->nthreads > 0) omp_set_num_threads(P->nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t t = 0; t < nt; ++t) {
        const double* x = txyz + 3 * t;
        int64_t self = self_index ? self_index[t] : -1;
        double pc = 0.0, pr = 0.0;
        if (xyz && q) {
            for (int64_t j = 0; j < n; ++j) {
                if (j == self) continue;
                double dx = x[0] - xyz[3 * j], dy_ = x[1] - xyz[3 * j + 1], dz = x[2] - xyz[3 * j + 2];
                pc += kc * q[j] / sqrt(dx * dx + dy_ * dy_ + dz * dz);
            }
        }
        if (kel_xyz && kel_q) {
            for (int64_t j = 0; j < n; ++j) {
                if (kel_q[j] == 0.0) continue; /* centre charge: image at infinity, in r0_const */
                double dx = x[0] - kel_xyz[3 * j], dy_ = x[1] - kel_xyz[3 * j + 1], dz = x[2] - kel_xyz[3 * j + 2];
                pr += kc * kel_q[j] / sqrt(dx * dx + dy_ * dy_ + dz * dz);
            }
        }
        pr += r0_const;
        if (surf_xyz) {
            for (int64_t l = 0; l < M; ++l) {
                const double* y = surf_xyz + 3 * l;
                double rho = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
                double yh[3] = {y[0] / rho, y[1] / rho, y[2] / rho};
                /* monopole layer at R_tau yhat */
                double dx = x[0] - y[0], dy_ = x[1] - y[1], dz = x[2] - y[2];
                double d = sqrt(dx * dx + dy_ * dy_ + dz * dz);
                pr += surf_w[l] * surf_dphi[l] * inv4pi / d;
                /* dipole layer from the central difference */
                double rm = Rtau - 0.5 * dy, rp = Rtau + 0.5 * dy;
                double xm[3] = {rm * yh[0], rm * yh[1], rm * yh[2]};
                double xp[3] = {rp * yh[0], rp * yh[1], rp * yh[2]};
                double ddm = sqrt((x[0] - xm[0]) * (x[0] - xm[0]) + (x[1] - xm[1]) * (x[1] - xm[1]) +
                                  (x[2] - xm[2]) * (x[2] - xm[2]));
                double ddp = sqrt((x[0] - xp[0]) * (x[0] - xp[0]) + (x[1] - xp[1]) * (x[1] - xp[1]) +
                                  (x[2] - xp[2]) * (x[2] - xp[2]));
                double strength = surf_w[l] * surf_phi[l] * inv4pi / dy;
                if (P->dipole_form == 0) {
                    pr += strength / ddm;
                    pr -= strength / ddp;
                } else {
                    /* (1/d_- - 1/d_+) = (d_+^2 - d_-^2)/(d_+ d_- (d_+ + d_-)),
                       d_+^2 - d_-^2 = 2 dy (R_tau - x.yhat) */
                    double xy = x[0] * yh[0] + x[1] * yh[1] + x[2] * yh[2];
                    pr += surf_w[l] * surf_phi[l] * inv4pi * 2.0 * (Rtau - xy) / (ddp * ddm * (ddp + ddm));
                }
            }
        }
        if (phi_coul) phi_coul[t] = pc;
        if (phi_rf) phi_rf[t] = pr;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Fields E = -grad phi at nt target points: the gradient, with every source held
 * fixed, of each term of oracle_eval.  A point source Q at s contributes
 *   Q (t - s) / |t - s|^3
 * (real charges except self(t), Kelvin images, monopole layer).  The dipole shells,
 * strength w Phi/(4 pi dy) at y^- and minus that at y^+, contribute
 *   dipole_form 0:  strength [ (t - y^-)/d_-^3 - (t - y^+)/d_+^3 ];
 *   dipole_form 1:  the same difference without cancellation.  With
 *     (t - y^-) - (t - y^+) = dy yhat  and  d_+^2 - d_-^2 = 2 dy (R_tau - t.yhat),
 *     d_+^3 - d_-^3 = (d_+ - d_-)(d_+^2 + d_+ d_- + d_-^2),
 *   it is (w Phi/(4 pi)) [ yhat/d_-^3
 *          + (t - y^+) 2 (R_tau - t.yhat)(d_+^2 + d_+ d_- + d_-^2) / ((d_+ + d_-) d_-^3 d_+^3) ].
 * The centre constant r0_const has no field.  Outputs are nt x 3, row-major.   */
int oracle_field(const oracle_params* P, int64_t n, const double* xyz, const double* q,
                 const double* kel_xyz, const double* kel_q,
                 int64_t M, const double* surf_xyz, const double* surf_w,
                 const double* surf_phi, const double* surf_dphi,
                 int64_t nt, const double* txyz, const int64_t* self_index,
                 double* E_coul, double* E_rf)
{
    const double kc = P->coulomb_k / P->eps1;
    const double Rtau = (1.0 + P->tau) * P->a;
    const double dy = P->dy_rel * Rtau;
    const double inv4pi = 1.0 / (4.0 * ORACLE_PI);
#ifdef _OPENMP
    if (P->nthreads > 0) omp_set_num_threads(P->nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t t = 0; t < nt; ++t) {
        const double* x = txyz + 3 * t;
        int64_t self = self_index ? self_index[t] : -1;
        double ec[3] = {0.0, 0.0, 0.0}, er[3] = {0.0, 0.0, 0.0};
        if (xyz && q) {
            for (int64_t j = 0; j < n; ++j) {
                if (self == j) continue;
                double u[3] = {x[0] - xyz[3 * j], x[1] - xyz[3 * j + 1], x[2] - xyz[3 * j + 2]};
                double d = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                double c = kc * q[j] / (d * d * d);
                for (int k = 0; k < 3; ++k) ec[k] += c * u[k];
            }
        }
        if (kel_xyz && kel_q) {
            for (int64_t j = 0; j < n; ++j) {
                if (kel_q[j] == 0.0) continue; /* centre charge: constant potential, no field */
                double u[3] = {x[0] - kel_xyz[3 * j], x[1] - kel_xyz[3 * j + 1], x[2] - kel_xyz[3 * j + 2]};
                double d = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                double c = kc * kel_q[j] / (d * d * d);
                for (int k = 0; k < 3; ++k) er[k] += c * u[k];
            }
        }
        if (surf_xyz) {
            for (int64_t l = 0; l < M; ++l) {
                const double* y = surf_xyz + 3 * l;
                double rho = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
                double yh[3] = {y[0] / rho, y[1] / rho, y[2] / rho};
                /* monopole layer at R_tau yhat */
                double u[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
                double d = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                double c = surf_w[l] * surf_dphi[l] * inv4pi / (d * d * d);
                for (int k = 0; k < 3; ++k) er[k] += c * u[k];
                /* dipole layer from the central difference */
                double rm = Rtau - 0.5 * dy, rp = Rtau + 0.5 * dy;
                double um[3] = {x[0] - rm * yh[0], x[1] - rm * yh[1], x[2] - rm * yh[2]};
                double up[3] = {x[0] - rp * yh[0], x[1] - rp * yh[1], x[2] - rp * yh[2]};
                double dm = sqrt(um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
                double dp = sqrt(up[0] * up[0] + up[1] * up[1] + up[2] * up[2]);
                if (P->dipole_form == 0) {
                    double strength = surf_w[l] * surf_phi[l] * inv4pi / dy;
                    for (int k = 0; k < 3; ++k)
                        er[k] += strength * (um[k] / (dm * dm * dm) - up[k] / (dp * dp * dp));
                } else {
                    double D = surf_w[l] * surf_phi[l] * inv4pi;
                    double xy = x[0] * yh[0] + x[1] * yh[1] + x[2] * yh[2];
                    double dm3 = dm * dm * dm, dp3 = dp * dp * dp;
                    double f = 2.0 * (Rtau - xy) * (dp * dp + dp * dm + dm * dm) / ((dp + dm) * dm3 * dp3);
                    for (int k = 0; k < 3; ++k) er[k] += D * (yh[k] / dm3 + up[k] * f);
                }
            }
        }
        for (int k = 0; k < 3; ++k) {
            if (E_coul) E_coul[3 * t + k] = ec[k];
            if (E_rf) E_rf[3 * t + k] = er[k];
        }
    }
    return 0;
}

/* Neumaier-compensated E_total = 1/2 sum q_i (phi_coul_i + phi_rf_i), E_RF = 1/2 sum q_i phi_rf_i. */
int oracle_energy(int64_t n, const double* q, const double* phi_coul, const double* phi_rf,
                  double* e_total, double* e_rf)
{
    double s1 = 0.0, c1 = 0.0, s2 = 0.0, c2 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double terms[2] = {0.5 * q[i] * (phi_coul[i] + phi_rf[i]), 0.5 * q[i] * phi_rf[i]};
        double* s[2] = {&s1, &s2};
        double* c[2] = {&c1, &c2};
        for (int k = 0; k < 2; ++k) {
            double t = *s[k] + terms[k];
            if (fabs(*s[k]) >= fabs(terms[k]))
                *c[k] += (*s[k] - t) + terms[k];
            else
                *c[k] += (terms[k] - t) + *s[k];
            *s[k] = t;
        }
    }
    if (e_total) *e_total = s1 + c1;
    if (e_rf) *e_rf = s2 + c2;
    return 0;
}

/* Whole method for one cavity: potentials at the charges and the energies. */
int oracle_hsma(const oracle_params* P, int64_t n, const double* xyz, const double* q,
                double* phi_coul, double* phi_rf, double* e_total, double* e_rf)
{
    const int64_t M = 2 * (int64_t)(P->F2 + 1);
    double* kel_xyz = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double* kel_q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* sxyz = (double*)malloc(sizeof(double) * 3 * (size_t)M);
    double* sw = (double*)malloc(sizeof(double) * (size_t)M);
    double* sphi = (double*)malloc(sizeof(double) * (size_t)M);
    double* sdphi = (double*)malloc(sizeof(double) * (size_t)M);
    int64_t* self = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double* pc = phi_coul ? phi_coul : (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* pr = phi_rf ? phi_rf : (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double c0 = 0.0;
    for (int64_t i = 0; i < n; ++i) self[i] = i;
    oracle_build(P, n, xyz, q, kel_xyz, kel_q, sxyz, sw, sphi, sdphi, &c0);
    oracle_eval(P, n, xyz, q, kel_xyz, kel_q, M, sxyz, sw, sphi, sdphi, c0, n, xyz, self, pc, pr);
    oracle_energy(n, q, pc, pr, e_total, e_rf);
    if (!phi_coul) free(pc);
    if (!phi_rf) free(pr);
    free(kel_xyz); free(kel_q); free(sxyz); free(sw); free(sphi); free(sdphi); free(self);
    return 0;
}

/* Threads an OpenMP region would use with the given request (for reporting). */
int oracle_threads(int requested)
{
#ifdef _OPENMP
    if (requested > 0) return requested;
    return omp_get_max_threads();
#else
    (void)requested;
    return 1;
#endif
}
