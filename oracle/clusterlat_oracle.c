/*
 * clusterlat_oracle.c -- serial FP64 oracle (TEST INFRASTRUCTURE ONLY; see the
 * header).  Built with -O2 -ffp-contract=off so that every product and sum is
 * rounded exactly as written.
 *
 * It follows the scheme of arXiv:0712.0813 Sec. III literally: one array pair
 * (f, v) per field, evolved in place, f at integer time and v = f' half a step
 * later; each step first advances f by a full step with v, then evaluates the
 * second derivative from the new f and advances v by a full step.  No tiling,
 * no fusion, no reordering.
 */
#include "clusterlat_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

long long orc_sites(const orc_model* m) {
  long long s = 1;
  for (int d = 0; d < m->dims; ++d) s *= m->N;
  return s;
}

/* Index of the neighbour of site s one step along axis d (0 = x, 1 = y,
 * 2 = z) in direction dir = +1/-1, with the periodic wrap.  The paper's ghost
 * ("buffer") columns exist only to make these neighbours available to each
 * processor (Sec. III); on one array the wrap is the index arithmetic itself. */
static long long neighbour(const orc_model* m, long long s, int d, int dir) {
  long long N = m->N, stride = 1;
  for (int k = 0; k < d; ++k) stride *= N;
  long long c = (s / stride) % N;
  long long c2 = (c + dir + N) % N;
  return s + (c2 - c) * stride;
}

/* Reading c-1: the nearest-neighbour second difference
 *   lap f(x) = dx^-2 sum_d [ f(x+e_d) + f(x-e_d) - 2 f(x) ]. */
void orc_laplacian(const orc_model* m, const double* f, double* out) {
  long long S = orc_sites(m);
  double dx = m->L / (double)m->N;
  double inv_dx2 = 1.0 / (dx * dx);
  for (long long s = 0; s < S; ++s) {
    double acc = 0.0;
    for (int d = 0; d < m->dims; ++d) {
      double fp = f[neighbour(m, s, d, +1)];
      double fm = f[neighbour(m, s, d, -1)];
      acc += fp + fm - 2.0 * f[s];
    }
    out[s] = acc * inv_dx2;
  }
}

/* Model V = phi^4/4 + sum_i (q_i/2) phi^2 chi_i^2 (program units):
 *   dV/dphi   = phi^3 + phi sum_i q_i chi_i^2
 *   dV/dchi_i = q_i phi^2 chi_i */
void orc_dvdf(const orc_model* m, const double* fs, double* out) {
  double phi = fs[0];
  double coupling = 0.0;
  for (int i = 1; i < m->nf; ++i) coupling += m->q[i - 1] * fs[i] * fs[i];
  out[0] = phi * phi * phi + phi * coupling;
  for (int i = 1; i < m->nf; ++i) out[i] = m->q[i - 1] * phi * phi * fs[i];
}

double orc_potential(const orc_model* m, const double* fs) {
  double phi = fs[0];
  double v = 0.25 * phi * phi * phi * phi;
  for (int i = 1; i < m->nf; ++i) v += 0.5 * m->q[i - 1] * phi * phi * fs[i] * fs[i];
  return v;
}

/* Readings c-2/c-3: the conformally rescaled field equation
 *   f_i'' = lap f_i - dV/df_i + (a''/a) f_i ,   s = a''/a. */
void orc_force(const orc_model* m, const double* f, double s, double* F) {
  long long S = orc_sites(m);
  int nf = m->nf;
  for (int i = 0; i < nf; ++i) orc_laplacian(m, f + (long long)i * S, F + (long long)i * S);
  double fs[4], dv[4];
  for (long long x = 0; x < S; ++x) {
    for (int i = 0; i < nf; ++i) fs[i] = f[(long long)i * S + x];
    orc_dvdf(m, fs, dv);
    for (int i = 0; i < nf; ++i) {
      long long k = (long long)i * S + x;
      F[k] = F[k] - dv[i] + s * fs[i];
    }
  }
}

/* Reading c-4: G from forward differences. */
double orc_gradient_mean(const orc_model* m, const double* f, double* per_field) {
  long long S = orc_sites(m);
  double dx = m->L / (double)m->N;
  double total = 0.0;
  for (int i = 0; i < m->nf; ++i) {
    const double* fi = f + (long long)i * S;
    double acc = 0.0;
    for (long long x = 0; x < S; ++x) {
      for (int d = 0; d < m->dims; ++d) {
        double g = (fi[neighbour(m, x, d, +1)] - fi[x]) / dx;
        acc += 0.5 * g * g;
      }
    }
    acc /= (double)S;
    if (per_field) per_field[i] = acc;
    total += acc;
  }
  return total;
}

double orc_potential_mean(const orc_model* m, const double* f) {
  long long S = orc_sites(m);
  double fs[4];
  double acc = 0.0;
  for (long long x = 0; x < S; ++x) {
    for (int i = 0; i < m->nf; ++i) fs[i] = f[(long long)i * S + x];
    acc += orc_potential(m, fs);
  }
  return acc / (double)S;
}

/* Reading c-4: a'' = (-a'^2 + kappa2 (2 G + 3 V)) / a  (acceleration equation
 * with the kinetic term eliminated through the Friedmann equation). */
static double accel(const orc_model* m, double a, double ap, double G, double V) {
  return (-ap * ap + m->kappa2 * (2.0 * G + 3.0 * V)) / a;
}

/* Reading c-6: a(0) = 1, a'(0) = kappa sqrt(K+G+V) from the Friedmann equation
 * with the synchronised velocities u = f' - (a'/a) f; then f' = u + (a'/a) f,
 * and the half-step start v(dt/2) = f'(0) + dt/2 F(0), a'(dt/2) = a'(0) + dt/2 a''(0)
 * that puts v and a' half a step after f and a (Sec. III staggering). */
int orc_init(const orc_model* m, double* f, double* v, orc_scale* sc) {
  long long S = orc_sites(m);
  long long n = (long long)m->nf * S;
  double a = 1.0, ap0 = 0.0, app0 = 0.0;
  if (m->expansion) {
    double K = 0.0;
    for (long long k = 0; k < n; ++k) K += 0.5 * v[k] * v[k];
    K /= (double)S;
    double G = orc_gradient_mean(m, f, NULL);
    double V = orc_potential_mean(m, f);
    double rho = K + G + V;
    if (!(rho >= 0.0)) return -1;
    ap0 = sqrt(m->kappa2 * rho);
    for (long long k = 0; k < n; ++k) v[k] = v[k] + (ap0 / a) * f[k];
    app0 = accel(m, a, ap0, G, V);
  }
  double* F = (double*)malloc((size_t)n * sizeof(double));
  if (!F) return -2;
  orc_force(m, f, app0 / a, F);
  for (long long k = 0; k < n; ++k) v[k] = v[k] + 0.5 * m->dt * F[k];
  free(F);
  sc->a = a;
  sc->ap = ap0 + 0.5 * m->dt * app0;
  sc->app = app0;
  sc->t = 0.0;
  sc->step = 0;
  return 0;
}

/* One full step of the staggered leapfrog (Sec. III), in place:
 *   drift  f <- f + dt v                      (v at t+dt/2 moves f to t+dt)
 *   scale  a <- a + dt a'                     (a' at t+dt/2)
 *          G, V of the new f; a' and a'' at t+dt from the implicit midpoint
 *          a'_new - a'_old = dt (-(a'_mid)^2/a + Q), a'_mid = (a'_new+a'_old)/2,
 *          Q = kappa2 (2G+3V)/a, solved in closed form (reading c-4)
 *   kick   v <- v + dt F(f, a''/a)            (v moves to t+3dt/2) */
int orc_step(const orc_model* m, double* f, double* v, orc_scale* sc, long long nsteps) {
  long long S = orc_sites(m);
  long long n = (long long)m->nf * S;
  double dt = m->dt;
  double* F = (double*)malloc((size_t)n * sizeof(double));
  if (!F) return -2;
  int rc = 0;
  for (long long it = 0; it < nsteps; ++it) {
    for (long long k = 0; k < n; ++k) f[k] = f[k] + dt * v[k];
    double s = 0.0;
    if (m->expansion) {
      double a = sc->a + dt * sc->ap;
      double G = orc_gradient_mean(m, f, NULL);
      double V = orc_potential_mean(m, f);
      double Q = m->kappa2 * (2.0 * G + 3.0 * V) / a;
      double c = 2.0 * sc->ap + dt * Q;
      double disc = 1.0 + dt * c / a;
      if (!(disc >= 0.0)) { rc = -1; break; }
      double u = 2.0 * c / (1.0 + sqrt(disc));   /* u = a'_new + a'_old */
      double app = (u - 2.0 * sc->ap) / dt;
      sc->a = a;
      sc->ap = u - sc->ap;
      sc->app = app;
      s = app / a;
    }
    sc->t = sc->t + dt;
    sc->step += 1;
    orc_force(m, f, s, F);
    for (long long k = 0; k < n; ++k) v[k] = v[k] + dt * F[k];
  }
  free(F);
  return rc;
}

/* Reading c-7: outputs at integer time use the synchronised velocity. */
void orc_sync_velocity(const orc_model* m, const double* f, const double* v,
                       const orc_scale* sc, double* vsync) {
  long long n = (long long)m->nf * orc_sites(m);
  double s = m->expansion ? sc->app / sc->a : 0.0;
  orc_force(m, f, s, vsync);
  for (long long k = 0; k < n; ++k) vsync[k] = v[k] - 0.5 * m->dt * vsync[k];
}

void orc_sync_u(const orc_model* m, const double* f, const double* v,
                const orc_scale* sc, double* u) {
  long long n = (long long)m->nf * orc_sites(m);
  orc_sync_velocity(m, f, v, sc, u);
  if (m->expansion) {
    double ap_t = sc->ap - 0.5 * m->dt * sc->app;
    double h = ap_t / sc->a;
    for (long long k = 0; k < n; ++k) u[k] = u[k] - h * f[k];
  }
}

void orc_energy(const orc_model* m, const double* f, const double* v,
                const orc_scale* sc, double* out) {
  long long S = orc_sites(m);
  long long n = (long long)m->nf * S;
  for (int k = 0; k < 16; ++k) out[k] = 0.0;
  double* u = (double*)malloc((size_t)n * sizeof(double));
  if (!u) return;
  orc_sync_u(m, f, v, sc, u);
  double E = 0.0;
  for (int i = 0; i < m->nf; ++i) {
    double K = 0.0;
    for (long long x = 0; x < S; ++x) {
      double ui = u[(long long)i * S + x];
      K += 0.5 * ui * ui;
    }
    out[i] = K / (double)S;
    E += out[i];
  }
  free(u);
  double Gf[4] = {0, 0, 0, 0};
  orc_gradient_mean(m, f, Gf);
  for (int i = 0; i < m->nf; ++i) { out[4 + i] = Gf[i]; E += Gf[i]; }
  out[8] = orc_potential_mean(m, f);
  E += out[8];
  out[9] = E;
  double ap_t = m->expansion ? sc->ap - 0.5 * m->dt * sc->app : 0.0;
  out[10] = m->expansion ? sc->a : 1.0;
  out[11] = ap_t;
  out[12] = sc->t;
  out[13] = m->expansion ? fabs(ap_t * ap_t / m->kappa2 - E) / E : 0.0;
}

/* Reading c-10: per-field mean <f> and population variance <(f - <f>)^2>,
 * the textbook two-pass definition. */
void orc_means_variances(const orc_model* m, const double* f, double* mean, double* var) {
  long long S = orc_sites(m);
  for (int i = 0; i < m->nf; ++i) {
    const double* fi = f + (long long)i * S;
    double s1 = 0.0;
    for (long long x = 0; x < S; ++x) s1 += fi[x];
    double mu = s1 / (double)S;
    double s2 = 0.0;
    for (long long x = 0; x < S; ++x) s2 += (fi[x] - mu) * (fi[x] - mu);
    mean[i] = mu;
    var[i] = s2 / (double)S;
  }
}
