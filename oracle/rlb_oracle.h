/*
 * rlb_oracle.h -- interface of the plain double-precision CPU oracle for the
 * ultra-relativistic lattice Boltzmann (RLB) time step of Mohseni, Mendoza,
 * Succi and Herrmann, "Lattice Boltzmann model for ultra-relativistic flows"
 * (arXiv:1302.1125).
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle is what the CUDA library is checked
 * against.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code, header, table or constant
 * with the CUDA library; the only thing the two have in common is the
 * documented data layout (population order, structure-of-arrays planes,
 * x-fastest cell index), which is an interface, not code.
 *
 * Data layout (all arrays are plain double, structure of arrays):
 *   cell index    idx = x + nx * (y + ny * z)
 *   f, h          19 planes of N = nx*ny*nz values: f[i*N + idx]
 *   prev          5 planes: P, u'_x, u'_y, u'_z, n of the previous time level
 *                 (u' = gamma*u, the spatial part of U^mu)
 *   macroscopic   6 planes: n, e, u_x, u_y, u_z, gamma (u = 3-velocity)
 *
 * Lattice units: nu = sqrt(13) so c_a = 1; c_i = c_a * shell * direction
 * (basic lattice: nu = sqrt(19), c_a = 1, diagonals c_a (+-1, +-1, 0)).
 * Population order (extended lattice, Sec. II.A, Eq. 42):
 *   0        rest
 *   1..6     c_a * (+x, -x, +y, -y, +z, -z)
 *   7..10    2 c_a * (x,y) signs (+,+) (+,-) (-,+) (-,-)
 *   11..14   2 c_a * (x,z) signs (+,+) (+,-) (-,+) (-,-)
 *   15..18   2 c_a * (y,z) signs (+,+) (+,-) (-,+) (-,-)
 */
#ifndef RLB_ORACLE_H
#define RLB_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_PERIODIC = 0, ORC_BC_OUTFLOW = 1, ORC_BC_INLET = 2 };
enum { ORC_LIMITER_MINMOD = 0, ORC_LIMITER_NONE = 1 };

typedef struct {
    int nx, ny, nz;
    int bc_lo[3], bc_hi[3];      /* per axis x, y, z */
} orc_grid;

typedef struct {
    orc_grid g;
    double dt;                   /* delta t / delta x (delta x = 1) */
    double eta_over_s;
    double zeta_over_s;
    double tau_override;         /* > 0: use this tau everywhere */
    double alpha_override;       /* >= 0: use this alpha; < 0: derive from zeta/s */
    double inlet_n, inlet_T, inlet_u[3];  /* state of the inlet ghost cells */
    int limiter;                 /* ORC_LIMITER_* */
    int euler_mode;              /* 1: f <- f^eq of the streamed state (Sec. III) */
    int model;                   /* 0: extended lattice (Sec. II.A), 1: basic lattice (Sec. II, R13) */
} orc_params;

/* the lattice the functions below without an orc_params use: 0 extended
 * (default), 1 basic; the functions taking orc_params select p->model */
void orc_set_model(int model);
int orc_get_model(void);
double orc_nu(void);
/* lattice: e[19][3] unit directions, c[19][3] velocities, w[19], wh[19]; returns xi0 */
double orc_lattice(int *e, double *c, double *w, double *wh);
void orc_set_threads(int n);
int orc_get_threads(void);

void orc_feq(double P, const double up[3], double out[19]);
void orc_heq(double n, const double up[3], double out[19]);
void orc_moments(const double f[19], const double h[19], double mom[5]);
int orc_recover(const double mom[5], double macro[5]);
double orc_tau(const orc_params *p, double P, double n);
double orc_alpha(const orc_params *p);
double orc_minmod(double X, double Y);

/* streaming increment of one scalar plane q moving with p[3]:
 * out = -k * sum_a [h^a(x) - h^a(x - e_a)]; ghost = inlet ghost value */
void orc_stream(const orc_params *p, const double *q, double ghost,
                const double pa[3], double k, double *out);
/* out = sum_a (q(x+e_a) - 2 q(x) + q(x-e_a)) */
void orc_laplacian(const orc_params *p, const double *q, double ghost, double *out);

void orc_init(const orc_params *p, const double *n, const double *T,
              const double *ux, const double *uy, const double *uz,
              double *f, double *h, double *prev);
/* one time step; prev is read (t - dt) and overwritten with the macros of t.
 * returns the number of cells whose recovery was non-physical */
long orc_step(const orc_params *p, const double *f, const double *h,
              double *prev, double *fout, double *hout);
/* the same update for a list of cells only, reading full-size float or
 * double state; outputs are per listed cell: fout[19*k], hout[19*k], mout[5*k] */
long orc_step_cells(const orc_params *p, const void *f, const void *h,
                    const void *prev, int is_f32, long ncell, const long *cells,
                    double *fout, double *hout, double *mout);
long orc_macroscopic(const orc_params *p, const double *f, const double *h,
                     double *out);
/* solid cells (Sec. III, the astrophysical run: a fixed cloud whose cells
 * evolve to the equilibrium of the constant state n, T, u = 0): every cell
 * with mask[idx] != 0 is set to f^eq(P = n T, 0), h^eq(n, 0) with the
 * previous level (P, 0, 0, 0, n).  The time loop applies it after every
 * step (reading R11). */
void orc_solid_reset(const orc_params *p, const unsigned char *mask, double n, double T,
                     double *f, double *h, double *prev);

#ifdef __cplusplus
}
#endif
#endif
