/*
 * rlb_oracle.c -- plain, slow, double-precision CPU oracle for one time step
 * of the ultra-relativistic lattice Boltzmann (RLB) method of Mohseni,
 * Mendoza, Succi and Herrmann, "Lattice Boltzmann model for ultra-relativistic
 * flows" (arXiv:1302.1125).
 *
 * TEST INFRASTRUCTURE ONLY: this is the reference the CUDA library is checked
 * against.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code with the CUDA library.
 * Build with -O2 -ffp-contract=off so that x86 and Arm give the same bits.
 *
 * Every step follows the paper in its own order and notation; nothing is
 * blocked, fused or reordered beyond what the equations say.  Where the paper
 * is silent, garbled or inconsistent the following readings are taken (the
 * CUDA library takes the same ones):
 *
 *  R1  nu = c/c_s is one global lattice constant, nu = sqrt(13), so that
 *      c_a = sqrt(13)/nu = 1 (Eq. 46): the lattice vectors are the integer
 *      vectors of Eq. 42 and c_t/c_0 = sqrt(27/13).  The paper notes that its
 *      quadrature needs only xi_x ~ 1 (Sec. II); c_a = 1 is also the only
 *      member of the lattice family for which every number-distribution
 *      weight of Eqs. 59-60 is non-negative and the upwind scheme for h is
 *      diffusive at every |u| < 1 (for nu = 1, w'_diag = 1/1092 - 3/280 < 0
 *      and the kinetic scheme for n is anti-diffusive once |u| > 0.05).
 *      Temperatures are in units of the workload's reference temperature
 *      and P = n T holds cell by cell (Sec. III).  The weights of Eqs. 43-45
 *      are nu-free: -539/676, 99/338, 9/2704.
 *  R2  f^{aR} (Eq. 50) is printed with Delta f^{a+}; it is read with
 *      Delta f^{a-}, the standard MUSCL minmod right state (for a
 *      population with p^a < 0, f^{a+} = 0 and the printed form would drop
 *      the limiter correction, breaking mirror symmetry).
 *  R3  h^a(x) of Eq. 48 is the flux through the interface x + 1/2; the
 *      divergence of Eq. 47 is read as the conservative difference
 *      h^a(x) - h^a(x - e_a) (the printed h^a(x+e_a) - h^a(x) is the same
 *      difference one cell downstream).
 *  R4  alpha (Eqs. 55-56) is one constant per run: alpha = 27 eta_b /(4 P nu^6)
 *      with eta_b = (zeta/s) s evaluated at the reference state T = 1,
 *      lambda = 1 (so s = 4 n, P = n and alpha = 27 (zeta/s) / nu^6), unless
 *      an alpha is given directly, as the paper does in Sec. III.
 *  R5  Eq. 57 needs f^eq(t - dt); at the first step f^eq(-dt) := f^eq(0) of
 *      the initial fields.  The previous macroscopic state (P, u', n) is kept
 *      per cell instead of 19 previous equilibria.
 *  R6  n is recovered from the number distribution as n = N^0 / gamma with
 *      N^0 = xi^0 sum_i h_i (Eq. 58 gives N^0 = n gamma for h = h^eq).
 *  R7  the entropy density s = n (4 - ln lambda) (Sec. III) turns negative
 *      for lambda > e^4; the factor (4 - ln lambda) is floored at S_MIN.
 *  R8  the equilibrium is the second-order polynomial in u' = gamma u whose
 *      discrete moments reproduce T_eq^{alpha beta} of Eq. 36 exactly (the
 *      expansion printed as Eq. 29 does not satisfy Eq. 36 on this lattice).
 *  R9  boundaries: "open" ends are zero-gradient (the ghost value is the
 *      value of the edge cell), transverse directions may be periodic, and an
 *      inlet face holds the ghost cells at the equilibrium of a fixed state
 *      (Sec. III, astrophysical application).
 *  R10 Euler (inviscid) mode replaces the collision by f <- f^eq, h <- h^eq of
 *      the streamed state (Sec. III).
 *  R11 solid cells (orc_solid_reset): every cell of the cloud is set to the
 *      equilibrium of its fixed state after every step.
 *  R13 the basic model (Sec. II, before the extension; model = 1) is the
 *      D3Q19 lattice with unit diagonals c_a (+-1, +-1, 0), weights of its
 *      own quadrature, c_a = sqrt(19)/nu and c_t/c_0 = sqrt(27)/nu; as R1,
 *      nu = sqrt(19) so that c_a = 1 and the weights are -44/361, 99/722,
 *      9/361.  Everything else is the same step (Eq. 57: limiter streaming,
 *      bulk term, implicit collision), so the two models differ only in the
 *      lattice.  The equilibrium is again the second-order polynomial matched
 *      to Eq. 36 (R8); the paper's constants make it exist on both lattices.
 *  R14 the paper gives number-distribution weights (Eqs. 59-60) only for
 *      the extended cell configuration; on the basic lattice the weights
 *      that give Eq. 58 the same moments (sum_i w'_i = 1 and
 *      sum_i w'_i c_ix^2 = 1/3, so that N^0 = n gamma) and fourth-order
 *      isotropy are the standard D3Q19 weights 1/3, 1/18, 1/36.
 */
#include "rlb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NU (L->nu)          /* the model's lattice constant nu: sqrt(13) (R1) or sqrt(19) (R13) */
#define D_G 16.0          /* gluon degeneracy, Sec. III */
#define S_MIN 1e-3        /* R7 */
#define T_REF 1.0         /* R1 / R4 */
#define PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Lattices: the extended D3Q19 configuration of Sec. II.A (model 0) and the */
/* basic D3Q19 lattice of Sec. II (model 1, R13).                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    double nu;             /* lattice constant nu = c/c_s (R1, R13) */
    int e[19][3];          /* unit direction of each population */
    double c[19][3];       /* spatial components c_i of xi_i (Eq. 42) */
    double w[19];          /* Eqs. 43-45 */
    double wh[19];         /* Eqs. 59-60 */
    double xi0;            /* time component c_t/c_0 (Eq. 46) */
    double c0_over_ct;
    double sigma2;         /* sum_i w_i c_ix^2 */
    double m4;             /* sum_i w_i c_ix^4 */
    double m22;            /* sum_i w_i c_ix^2 c_iy^2 */
} lattice_t;

static lattice_t L_models[2];
static const lattice_t *L = &L_models[0];

static void build_lattice(lattice_t *l, int basic)
{
    const double nu = basic ? sqrt(19.0) : sqrt(13.0);   /* R1, R13 */
    const double ca = (basic ? sqrt(19.0) : sqrt(13.0)) / nu;   /* Eq. 46 / Sec. II */
    const double ct_c0 = sqrt(27.0) / nu;                 /* Eq. 46 / Sec. II */
    const double dshell = basic ? 1.0 : 2.0;              /* diagonal length in units of c_a */
    int i = 0, a, b, s1, s2;
    memset(l, 0, sizeof(*l));
    l->nu = nu;
    /* i = 0: rest */
    i = 1;
    /* 1 <= i <= 6: c_a (+-1, 0, 0) fully symmetric */
    for (a = 0; a < 3; ++a)
        for (s1 = 1; s1 >= -1; s1 -= 2) {
            l->e[i][a] = s1;
            l->c[i][a] = ca * s1;
            ++i;
        }
    /* 7 <= i <= 18: 2 c_a (+-1, +-1, 0) (extended) or c_a (+-1, +-1, 0) (basic) */
    for (a = 0; a < 3; ++a)
        for (b = a + 1; b < 3; ++b)
            for (s1 = 1; s1 >= -1; s1 -= 2)
                for (s2 = 1; s2 >= -1; s2 -= 2) {
                    l->e[i][a] = s1;
                    l->e[i][b] = s2;
                    l->c[i][a] = dshell * ca * s1;
                    l->c[i][b] = dshell * ca * s2;
                    ++i;
                }
    /* weights written as printed with c_t/c_0, c_a, nu: Eqs. 43-45 (extended)
     * and the basic model's quadrature weights of Sec. II */
    {
        const double r2 = ct_c0 * ct_c0;  /* c_t^2 / c_0^2 */
        double w0, w1, w2;
        if (basic) {
            w0 = 1.0 + 4.0 * r2 * nu * nu / 361.0 - r2 / (ca * ca);
            w1 = r2 / (2166.0 * ca * ca) * (361.0 - 8.0 * ca * ca * nu * nu);
            w2 = r2 * nu * nu / 1083.0;
        } else {
            w0 = 1.0 + 7.0 * r2 * nu * nu / 676.0 - r2 / (ca * ca);
            w1 = r2 / (1014.0 * ca * ca) * (169.0 - 2.0 * ca * ca * nu * nu);
            w2 = r2 * nu * nu / 8112.0;
        }
        l->w[0] = w0;
        for (i = 1; i <= 6; ++i) l->w[i] = w1;
        for (i = 7; i <= 18; ++i) l->w[i] = w2;
    }
    /* number-distribution weights: Eqs. 59-60 (extended; c_a is the scalar of
     * Eq. 46), the standard D3Q19 weights on the basic lattice (R14) */
    if (basic) {
        l->wh[0] = 1.0 / 3.0;
        for (i = 1; i <= 6; ++i) l->wh[i] = 1.0 / 18.0;
        for (i = 7; i <= 18; ++i) l->wh[i] = 1.0 / 36.0;
    } else {
        l->wh[0] = 1.0 / 10.0;
        for (i = 1; i <= 6; ++i) l->wh[i] = 6.0 / 35.0 - 1.0 / (42.0 * ca * ca);
        for (i = 7; i <= 18; ++i) l->wh[i] = 1.0 / (84.0 * ca * ca) - 3.0 / 280.0;
    }
    l->xi0 = ct_c0;
    l->c0_over_ct = 1.0 / ct_c0;
    /* lattice moments used to solve the moment conditions of Eq. 36 (R8) */
    for (i = 0; i < 19; ++i) {
        l->sigma2 += l->w[i] * l->c[i][0] * l->c[i][0];
        l->m4 += l->w[i] * pow(l->c[i][0], 4);
        l->m22 += l->w[i] * l->c[i][0] * l->c[i][0] * l->c[i][1] * l->c[i][1];
    }
}

__attribute__((constructor)) static void build_lattices(void)
{
    build_lattice(&L_models[0], 0);
    build_lattice(&L_models[1], 1);
}

void orc_set_model(int model) { L = &L_models[model == 1 ? 1 : 0]; }
int orc_get_model(void) { return L == &L_models[1] ? 1 : 0; }

double orc_lattice(int *e, double *c, double *w, double *wh)
{
    int i, a;
    for (i = 0; i < 19; ++i) {
        for (a = 0; a < 3; ++a) {
            if (e) e[3 * i + a] = L->e[i][a];
            if (c) c[3 * i + a] = L->c[i][a];
        }
        if (w) w[i] = L->w[i];
        if (wh) wh[i] = L->wh[i];
    }
    return L->xi0;
}

double orc_nu(void) { return NU; }

static int g_threads = 1;
void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int orc_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------------ */
/* Equilibria                                                                */
/* ------------------------------------------------------------------------ */

/* f^eq (R8): f_i = w_i [a0 + a1 (c_i.u') + a2 sum_{a<b} c_ia c_ib u'_a u'_b
 *                     + a3 sum_a c_ia^2 u'_a^2 + a4 |u'|^2],
 * with the coefficients fixed by requiring, for the ultra-relativistic gas
 * eps = 3P (Eq. 38), that sum_i p_i^a p_i^b f_i = (eps+P) U^a U^b - P eta^ab
 * (Eq. 36) with p_i = (xi^0, c_i) and U = (gamma, u'):
 *   T^{0a}: xi0 a1 sigma2 u'_a             = 4 P gamma u'_a
 *   T^{ab}: a2 m22 u'_a u'_b  (a != b)      = 4 P u'_a u'_b
 *   T^{aa}: a0 sigma2 + a3 (m4 - m22) u'_a^2 + (a3 m22 + a4 sigma2)|u'|^2
 *                                           = P + 4 P u'_a^2
 * and T^{00} then holds because xi0^2 = 3 sigma2 on this lattice. */
void orc_feq(double P, const double up[3], double out[19])
{
    const double u2 = up[0] * up[0] + up[1] * up[1] + up[2] * up[2];
    const double gamma = sqrt(1.0 + u2);      /* Eq. 8 with nu = 1 */
    const double a0 = P / L->sigma2;
    const double a1 = 4.0 * P * gamma / (L->xi0 * L->sigma2);
    const double a2 = 4.0 * P / L->m22;
    const double a3 = 4.0 * P / (L->m4 - L->m22);
    const double a4 = -a3 * L->m22 / L->sigma2;
    int i;
    for (i = 0; i < 19; ++i) {
        const double *c = L->c[i];
        const double cu = c[0] * up[0] + c[1] * up[1] + c[2] * up[2];
        const double off = c[0] * c[1] * up[0] * up[1] + c[0] * c[2] * up[0] * up[2]
                         + c[1] * c[2] * up[1] * up[2];
        const double dia = c[0] * c[0] * up[0] * up[0] + c[1] * c[1] * up[1] * up[1]
                         + c[2] * c[2] * up[2] * up[2];
        out[i] = L->w[i] * (a0 + a1 * cu + a2 * off + a3 * dia + a4 * u2);
    }
}

/* h^eq, Eq. 58: w'_i n gamma (c0/ct + 3 c_i.u + 9/2 (c_i.u)^2 - 3/2 |u|^2),
 * u the three-velocity u'/gamma. */
void orc_heq(double n, const double up[3], double out[19])
{
    const double gamma = sqrt(1.0 + up[0] * up[0] + up[1] * up[1] + up[2] * up[2]);
    const double u[3] = {up[0] / gamma, up[1] / gamma, up[2] / gamma};
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    int i;
    for (i = 0; i < 19; ++i) {
        const double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
        out[i] = L->wh[i] * n * gamma * (L->c0_over_ct + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* ------------------------------------------------------------------------ */
/* Moments and Landau-frame recovery (Sec. II, Eqs. 36 and 38)               */
/* ------------------------------------------------------------------------ */

/* mom = (T^00, T^0x, T^0y, T^0z, N^0) with p_i^0 = xi0 for every i */
void orc_moments(const double f[19], const double h[19], double mom[5])
{
    int i, a;
    for (a = 0; a < 5; ++a) mom[a] = 0.0;
    for (i = 0; i < 19; ++i) {
        mom[0] += L->xi0 * L->xi0 * f[i];
        for (a = 0; a < 3; ++a) mom[1 + a] += L->xi0 * L->c[i][a] * f[i];
        mom[4] += L->xi0 * h[i];
    }
}

/* Landau frame: T^{mu nu} U_nu = eps U^mu with eps = 3P.  With E = T^00 and
 * M = T^0a this gives E = (eps+P) gamma^2 - P and M = (eps+P) gamma^2 u, so
 * (E + P) u = M and 3 X^2 - 4 E X + |M|^2 = 0 for X = E + P, whose physical
 * root is eps = -E + sqrt(4 E^2 - 3 |M|^2).  n = N^0 / gamma (R6).
 * macro = (P, u'_x, u'_y, u'_z, n).  Returns 1 for a non-physical state. */
int orc_recover(const double mom[5], double macro[5])
{
    const double E = mom[0];
    const double M2 = mom[1] * mom[1] + mom[2] * mom[2] + mom[3] * mom[3];
    const double eps = -E + sqrt(4.0 * E * E - 3.0 * M2);
    const double P = eps / 3.0;
    double u[3], u2, gamma;
    int a, bad;
    for (a = 0; a < 3; ++a) u[a] = mom[1 + a] / (E + P);
    u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    gamma = 1.0 / sqrt(1.0 - u2);
    macro[0] = P;
    for (a = 0; a < 3; ++a) macro[1 + a] = gamma * u[a];
    macro[4] = mom[4] / gamma;
    bad = !(E > 0.0) || !(E * E > M2) || !(eps > 0.0) || !(u2 < 1.0) || !isfinite(macro[4])
          || !isfinite(gamma);
    return bad;
}

/* tau from eta/s: Eq. 41, eta = (eps + P)(tau - 1/2)/nu^2, with
 * s = 4n - n ln(lambda), lambda = n/n_eq, n_eq = d_G T^3/pi^2 (Sec. III)
 * and T = P/n (Sec. III: P = n T). */
double orc_tau(const orc_params *p, double P, double n)
{
    orc_set_model(p->model);
    double T, neq, lam, sfac, s, eta;
    if (p->tau_override > 0.0) return p->tau_override;
    T = P / n;
    neq = D_G * T * T * T / (PI * PI);
    lam = n / neq;
    sfac = 4.0 - log(lam);
    if (sfac < S_MIN) sfac = S_MIN;  /* R7 */
    s = n * sfac;
    eta = p->eta_over_s * s;
    return 0.5 + NU * NU * eta / (4.0 * P);
}

/* alpha of Eq. 55 from zeta/s through Eq. 56 (R4) */
double orc_alpha(const orc_params *p)
{
    orc_set_model(p->model);
    double nref, sref, pref, eta_b;
    if (p->alpha_override >= 0.0) return p->alpha_override;
    nref = D_G * T_REF * T_REF * T_REF / (PI * PI);   /* lambda = 1 */
    sref = nref * (4.0 - log(1.0));
    pref = nref * T_REF;
    eta_b = p->zeta_over_s * sref;
    return 27.0 * eta_b / (4.0 * pref * pow(NU, 6));
}

/* ------------------------------------------------------------------------ */
/* Streaming: minmod flux limiter, Eqs. 47-53                                */
/* ------------------------------------------------------------------------ */

static double sgn(double v) { return (v > 0.0) - (v < 0.0); }

/* Eq. 53 */
double orc_minmod(double X, double Y)
{
    return 0.5 * fmin(fabs(X), fabs(Y)) * (sgn(X) + sgn(Y));
}

/* Eq. 51 */
static double fplus(double p, double q) { return 0.5 * (p + fabs(p)) * q; }
static double fminus(double p, double q) { return 0.5 * (p - fabs(p)) * q; }

/* h^a at the interface y + 1/2 from q(y-1), q(y), q(y+1), q(y+2): Eqs. 48-52 */
static double flux(double p, double qm1, double q0, double q1, double q2, int limiter)
{
    double fL = fplus(p, q0);     /* Eq. 49 */
    double fR = fminus(p, q1);    /* Eq. 50 */
    if (limiter == ORC_LIMITER_MINMOD) {
        const double dp_y = fplus(p, q1) - fplus(p, q0);       /* Delta f^{a+}(y) */
        const double dp_ym1 = fplus(p, q0) - fplus(p, qm1);    /* Delta f^{a+}(y-1) */
        const double dm_y = fminus(p, q1) - fminus(p, q0);     /* Delta f^{a-}(y) */
        const double dm_yp1 = fminus(p, q2) - fminus(p, q1);   /* Delta f^{a-}(y+1) */
        fL += 0.5 * orc_minmod(dp_y, dp_ym1);
        fR -= 0.5 * orc_minmod(dm_y, dm_yp1);                  /* R2 */
    }
    return fL + fR;               /* Eq. 48 */
}

/* ------------------------------------------------------------------------ */
/* State access with the boundary map (R9)                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    const void *base;
    int f32;
    long N;
} plane_ref;

static double get(const plane_ref *r, int i, long idx)
{
    if (r->f32) return (double)((const float *)r->base)[(long)i * r->N + idx];
    return ((const double *)r->base)[(long)i * r->N + idx];
}

/* map a coordinate that may lie up to two cells outside [0, n); -1 = inlet ghost */
static long map_coord(long c, long n, int lo, int hi)
{
    int bc;
    if (c >= 0 && c < n) return c;
    bc = c < 0 ? lo : hi;
    if (bc == ORC_BC_PERIODIC) {
        long m = c % n;
        return m < 0 ? m + n : m;
    }
    if (bc == ORC_BC_OUTFLOW) return c < 0 ? 0 : n - 1;
    return -1;
}

/* value of population i at cell (x, y, z) + d e_axis */
static double nb(const orc_grid *g, const plane_ref *r, int i, double ghost,
                 long x, long y, long z, int axis, int d)
{
    long c[3] = {x, y, z};
    const long n[3] = {g->nx, g->ny, g->nz};
    long m;
    c[axis] += d;
    m = map_coord(c[axis], n[axis], g->bc_lo[axis], g->bc_hi[axis]);
    if (m < 0) return ghost;
    c[axis] = m;
    return get(r, i, c[0] + n[0] * (c[1] + n[1] * c[2]));
}

/* -k sum_a [h^a(x) - h^a(x - e_a)] / dx  (Eq. 47 and R3; dx = 1) */
static double stream_at(const orc_params *p, const plane_ref *r, int i, double ghost,
                        const double pa[3], double k, long x, long y, long z)
{
    double s = 0.0;
    int a, d;
    for (a = 0; a < 3; ++a) {
        double q[5];
        if (pa[a] == 0.0) continue;  /* p^a = 0: f^{a+-} = 0, the flux vanishes */
        for (d = -2; d <= 2; ++d) q[d + 2] = nb(&p->g, r, i, ghost, x, y, z, a, d);
        s += flux(pa[a], q[1], q[2], q[3], q[4], p->limiter)
           - flux(pa[a], q[0], q[1], q[2], q[3], p->limiter);
    }
    return -k * s;
}

/* sum_a d^2 q / dx_a^2 by central differences (Eq. 54, dx = 1) */
static double lap_at(const orc_params *p, const plane_ref *r, int i, double ghost,
                     long x, long y, long z)
{
    double s = 0.0;
    int a;
    for (a = 0; a < 3; ++a)
        s += nb(&p->g, r, i, ghost, x, y, z, a, 1) - 2.0 * get(r, i, x + (long)p->g.nx * (y + (long)p->g.ny * z))
           + nb(&p->g, r, i, ghost, x, y, z, a, -1);
    return s;
}

void orc_stream(const orc_params *p, const double *q, double ghost,
                const double pa[3], double k, double *out)
{
    const long N = (long)p->g.nx * p->g.ny * p->g.nz;
    const plane_ref r = {q, 0, N};
    long idx;
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (idx = 0; idx < N; ++idx) {
        const long x = idx % p->g.nx, y = (idx / p->g.nx) % p->g.ny, z = idx / ((long)p->g.nx * p->g.ny);
        out[idx] = stream_at(p, &r, 0, ghost, pa, k, x, y, z);
    }
}

void orc_laplacian(const orc_params *p, const double *q, double ghost, double *out)
{
    const long N = (long)p->g.nx * p->g.ny * p->g.nz;
    const plane_ref r = {q, 0, N};
    long idx;
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (idx = 0; idx < N; ++idx) {
        const long x = idx % p->g.nx, y = (idx / p->g.nx) % p->g.ny, z = idx / ((long)p->g.nx * p->g.ny);
        out[idx] = lap_at(p, &r, 0, ghost, x, y, z);
    }
}

/* ------------------------------------------------------------------------ */
/* The time step, Eq. 57                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    double ghost_f[19], ghost_h[19];  /* inlet equilibria (R9) */
    double alpha;
} step_consts;

static void make_consts(const orc_params *p, step_consts *k)
{
    const double u2 = p->inlet_u[0] * p->inlet_u[0] + p->inlet_u[1] * p->inlet_u[1]
                    + p->inlet_u[2] * p->inlet_u[2];
    const double gamma = 1.0 / sqrt(1.0 - u2);
    const double up[3] = {gamma * p->inlet_u[0], gamma * p->inlet_u[1], gamma * p->inlet_u[2]};
    orc_feq(p->inlet_n * p->inlet_T, up, k->ghost_f);
    orc_heq(p->inlet_n, up, k->ghost_h);
    k->alpha = orc_alpha(p);
}

/* new f, h and the macros of time t at one cell */
static int update_cell(const orc_params *p, const step_consts *k, const plane_ref *F,
                       const plane_ref *H, const plane_ref *PV, long x, long y, long z,
                       double fo[19], double ho[19], double mo[5])
{
    const long idx = x + (long)p->g.nx * (y + (long)p->g.ny * z);
    const double dt = p->dt;
    /* prefactor of the flux term of Eq. 57: (c0/ct)(dt/dx); p_i^a = c_ia */
    const double kstream = L->c0_over_ct * dt;
    /* prefactor of the bulk term of Eq. 57 times lambda_i (Eq. 55, dx = 1) */
    const double kbulk = L->c0_over_ct * NU * dt * k->alpha;
    double f[19], h[19], sf[19], sh[19], mom[5], mac[5];
    int i, bad;

    for (i = 0; i < 19; ++i) {
        f[i] = get(F, i, idx);
        h[i] = get(H, i, idx);
        sf[i] = stream_at(p, F, i, k->ghost_f[i], L->c[i], kstream, x, y, z);
        if (i != 0) sf[i] += kbulk * lap_at(p, F, i, k->ghost_f[i], x, y, z);  /* lambda_0 = 0 */
        sh[i] = stream_at(p, H, i, k->ghost_h[i], L->c[i], kstream, x, y, z);  /* no lambda term */
    }

    if (p->euler_mode) {
        /* R10: f(t+dt) = f^eq of the streamed state */
        double fs[19], hs[19];
        for (i = 0; i < 19; ++i) {
            fs[i] = f[i] + sf[i];
            hs[i] = h[i] + sh[i];
        }
        orc_moments(fs, hs, mom);
        bad = orc_recover(mom, mac);
        orc_feq(mac[0], mac + 1, fo);
        orc_heq(mac[4], mac + 1, ho);
    } else {
        double feq[19], heq[19], feqp[19], heqp[19], pv[5], tau, omega;
        orc_moments(f, h, mom);
        bad = orc_recover(mom, mac);
        orc_feq(mac[0], mac + 1, feq);
        orc_heq(mac[4], mac + 1, heq);
        for (i = 0; i < 5; ++i) pv[i] = get(PV, i, idx);
        orc_feq(pv[0], pv + 1, feqp);   /* f^eq(x, t - dt) */
        orc_heq(pv[4], pv + 1, heqp);
        tau = orc_tau(p, mac[0], mac[4]);
        omega = L->c0_over_ct * NU * dt / tau;
        /* Eq. 57 solved for f(x, t + dt) */
        for (i = 0; i < 19; ++i) {
            fo[i] = (f[i] + sf[i] + omega * (2.0 * feq[i] - feqp[i])) / (1.0 + omega);
            ho[i] = (h[i] + sh[i] + omega * (2.0 * heq[i] - heqp[i])) / (1.0 + omega);
        }
    }
    for (i = 0; i < 5; ++i) mo[i] = mac[i];
    return bad;
}

void orc_init(const orc_params *p, const double *n, const double *T,
              const double *ux, const double *uy, const double *uz,
              double *f, double *h, double *prev)
{
    orc_set_model(p->model);
    const long N = (long)p->g.nx * p->g.ny * p->g.nz;
    long idx;
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (idx = 0; idx < N; ++idx) {
        const double u2 = ux[idx] * ux[idx] + uy[idx] * uy[idx] + uz[idx] * uz[idx];
        const double gamma = 1.0 / sqrt(1.0 - u2);
        const double up[3] = {gamma * ux[idx], gamma * uy[idx], gamma * uz[idx]};
        const double P = n[idx] * T[idx];
        double fe[19], he[19];
        int i;
        orc_feq(P, up, fe);
        orc_heq(n[idx], up, he);
        for (i = 0; i < 19; ++i) {
            f[(long)i * N + idx] = fe[i];
            h[(long)i * N + idx] = he[i];
        }
        prev[0 * N + idx] = P;
        prev[1 * N + idx] = up[0];
        prev[2 * N + idx] = up[1];
        prev[3 * N + idx] = up[2];
        prev[4 * N + idx] = n[idx];
    }
}

void orc_solid_reset(const orc_params *p, const unsigned char *mask, double n, double T,
                     double *f, double *h, double *prev)
{
    orc_set_model(p->model);
    const long N = (long)p->g.nx * p->g.ny * p->g.nz;
    const double rest[3] = {0.0, 0.0, 0.0};
    double fe[19], he[19];
    long idx;
    int i;
    orc_feq(n * T, rest, fe);
    orc_heq(n, rest, he);
    for (idx = 0; idx < N; ++idx) {
        if (!mask[idx]) continue;
        for (i = 0; i < 19; ++i) {
            f[(long)i * N + idx] = fe[i];
            h[(long)i * N + idx] = he[i];
        }
        prev[0 * N + idx] = n * T;
        prev[1 * N + idx] = 0.0;
        prev[2 * N + idx] = 0.0;
        prev[3 * N + idx] = 0.0;
        prev[4 * N + idx] = n;
    }
}

long orc_step(const orc_params *p, const double *f, const double *h,
              double *prev, double *fout, double *hout)
{
    orc_set_model(p->model);
    const long N = (long)p->g.nx * p->g.ny * p->g.nz;
    const plane_ref F = {f, 0, N}, H = {h, 0, N}, PV = {prev, 0, N};
    step_consts k;
    double *mnew = (double *)malloc(sizeof(double) * 5 * (size_t)N);
    long idx, bad = 0;
    make_consts(p, &k);
#pragma omp parallel for schedule(static) reduction(+ : bad) num_threads(g_threads)
    for (idx = 0; idx < N; ++idx) {
        const long x = idx % p->g.nx, y = (idx / p->g.nx) % p->g.ny, z = idx / ((long)p->g.nx * p->g.ny);
        double fo[19], ho[19], mo[5];
        int i;
        bad += update_cell(p, &k, &F, &H, &PV, x, y, z, fo, ho, mo);
        for (i = 0; i < 19; ++i) {
            fout[(long)i * N + idx] = fo[i];
            hout[(long)i * N + idx] = ho[i];
        }
        for (i = 0; i < 5; ++i) mnew[(long)i * N + idx] = mo[i];
    }
    memcpy(prev, mnew, sizeof(double) * 5 * (size_t)N);
    free(mnew);
    return bad;
}

long orc_step_cells(const orc_params *p, const void *f, const void *h,
                    const void *prev, int is_f32, long ncell, const long *cells,
                    double *fout, double *hout, double *mout)
{
    orc_set_model(p->model);
    const long N = (long)p->g.nx * p->g.ny * p->g.nz;
    const plane_ref F = {f, is_f32, N}, H = {h, is_f32, N}, PV = {prev, is_f32, N};
    step_consts k;
    long j, bad = 0;
    make_consts(p, &k);
#pragma omp parallel for schedule(static) reduction(+ : bad) num_threads(g_threads)
    for (j = 0; j < ncell; ++j) {
        const long idx = cells[j];
        const long x = idx % p->g.nx, y = (idx / p->g.nx) % p->g.ny, z = idx / ((long)p->g.nx * p->g.ny);
        bad += update_cell(p, &k, &F, &H, &PV, x, y, z, fout + 19 * j, hout + 19 * j, mout + 5 * j);
    }
    return bad;
}

long orc_macroscopic(const orc_params *p, const double *f, const double *h, double *out)
{
    orc_set_model(p->model);
    const long N = (long)p->g.nx * p->g.ny * p->g.nz;
    long idx, bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad) num_threads(g_threads)
    for (idx = 0; idx < N; ++idx) {
        double fl[19], hl[19], mom[5], mac[5], gamma;
        int i;
        for (i = 0; i < 19; ++i) {
            fl[i] = f[(long)i * N + idx];
            hl[i] = h[(long)i * N + idx];
        }
        orc_moments(fl, hl, mom);
        bad += orc_recover(mom, mac);
        gamma = sqrt(1.0 + mac[1] * mac[1] + mac[2] * mac[2] + mac[3] * mac[3]);
        out[0 * N + idx] = mac[4];
        out[1 * N + idx] = 3.0 * mac[0];
        out[2 * N + idx] = mac[1] / gamma;
        out[3 * N + idx] = mac[2] / gamma;
        out[4 * N + idx] = mac[3] / gamma;
        out[5 * N + idx] = gamma;
    }
    return bad;
}
