/*
 * clusterlat_oracle.h -- plain serial FP64 CPU oracle of the staggered-leapfrog
 * evolution of interacting scalar fields on a periodic lattice (CLUSTEREASY,
 * arXiv:0712.0813, Sec. III "Parallel Algorithms").
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library against
 * an independent, obviously-correct implementation.  Only the test-suite, the
 * package smoke test and the benchmark's CPU-baseline leg may load it.  It
 * shares no source, header, helper or constant with the CUDA path, and the
 * product path never calls it.
 *
 * Conventions (all program units):
 *   - d = dims in {1,2,3}; N sites per side; S = N^d sites; dx = L/N.
 *   - One field array holds S doubles in row-major order, x fastest:
 *     3D index ((z*N)+y)*N+x, 2D y*N+x, 1D x.  A multi-field array is nf such
 *     arrays back to back (field 0 = phi, fields 1.. = chi_i).
 *   - Model: V = phi^4/4 + sum_i (q_i/2) phi^2 chi_i^2.
 *   - Staggering (Sec. III): f lives at integer time t, its derivative v = f'
 *     at t + dt/2.  The scale factor a lives at t, a' at t + dt/2.
 *
 * The paper states the scheme in words only; the Laplacian, the rescaled field
 * equation, the scale-factor equation and the start-up are the readings listed
 * in the design notes (c-1 .. c-14 there) and are repeated at each function.
 */
#ifndef CLUSTERLAT_ORACLE_H
#define CLUSTERLAT_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int dims;          /* 1, 2 or 3 */
  long long N;       /* sites per side, >= 3 */
  double L;          /* box side */
  double dt;         /* time step */
  int nf;            /* number of fields, 1..4 */
  double q[3];       /* couplings q_i of chi_i */
  int expansion;     /* 0: a == 1 fixed; 1: self-consistent a(t) */
  double kappa2;     /* (8 pi / 3) (phi0 / M_pl)^2 */
} orc_model;

typedef struct {
  double a;          /* a(t) */
  double ap;         /* a'(t + dt/2) */
  double app;        /* a''(t), from the last step (or start-up) */
  double t;          /* program time */
  long long step;    /* number of full steps taken */
} orc_scale;

/* Number of sites S = N^dims. */
long long orc_sites(const orc_model* m);

/* out = discrete Laplacian of one field array (periodic, 2d+1 points). */
void orc_laplacian(const orc_model* m, const double* f, double* out);

/* dV/df_i for the nf field values of one site. */
void orc_dvdf(const orc_model* m, const double* fsite, double* out);

/* V at one site. */
double orc_potential(const orc_model* m, const double* fsite);

/* F_i = lap f_i - dV/df_i + s f_i for all fields and sites (nf*S values). */
void orc_force(const orc_model* m, const double* f, double s, double* F);

/* Mean gradient energy G = (1/S) sum_x sum_i sum_d 1/2 ((f_i(x+e_d)-f_i(x))/dx)^2;
 * per_field (may be NULL) receives each field's share. */
double orc_gradient_mean(const orc_model* m, const double* f, double* per_field);

/* Mean potential energy V = (1/S) sum_x V(f(x)). */
double orc_potential_mean(const orc_model* m, const double* f);

/* Start-up.  In: f = f(0), v = u(0) = f' - (a'/a) f (synchronised).
 * Out: v = v(dt/2), sc = {a=1, a'(dt/2), a''(0), t=0, step=0}.
 * Returns 0, or -1 if the Friedmann equation has no real root. */
int orc_init(const orc_model* m, double* f, double* v, orc_scale* sc);

/* nsteps full leapfrog steps, in place.  Returns 0, or -1 on a negative
 * discriminant in the a' update. */
int orc_step(const orc_model* m, double* f, double* v, orc_scale* sc, long long nsteps);

/* Synchronised velocity v(t) = v(t+dt/2) - dt/2 F(f(t), a''/a). */
void orc_sync_velocity(const orc_model* m, const double* f, const double* v,
                       const orc_scale* sc, double* vsync);

/* u(t) = v(t) - (a'(t)/a(t)) f(t), with a'(t) = a'(t+dt/2) - dt/2 a''(t). */
void orc_sync_u(const orc_model* m, const double* f, const double* v,
                const orc_scale* sc, double* u);

/* Energies at integer time.  out[16]:
 *   0..3  K_i = <1/2 u_i^2>          4..7  G_i (gradient, per field)
 *   8     V = <V(f)>                 9     E = sum K + sum G + V
 *   10    a(t)                       11    a'(t)
 *   12    t                          13    Friedmann residual |a'^2/kappa2 - E|/E
 *                                          (0 without expansion)
 *   14,15 unused (0) */
void orc_energy(const orc_model* m, const double* f, const double* v,
                const orc_scale* sc, double* out);

/* Per-field mean and population variance (two-pass) of f. */
void orc_means_variances(const orc_model* m, const double* f, double* mean, double* var);

#ifdef __cplusplus
}
#endif
#endif
