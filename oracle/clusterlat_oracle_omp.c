/*
 * clusterlat_oracle_omp.c -- the oracle's loops with OpenMP threads over the
 * sites, for TIMING ONLY (TEST INFRASTRUCTURE; see clusterlat_oracle.h).
 *
 * The benchmark times the oracle as the CPU baseline on all host cores.  This
 * file repeats the serial oracle's loops (clusterlat_oracle.c: one array pair
 * per field, in place, drift then kick, arXiv:0712.0813 Sec. III) with a
 * `parallel for` over the outermost site index and `reduction(+)` for the
 * global sums G and V (and K at start-up).  Nothing else changes: the same
 * neighbour index arithmetic, the same per-site operations, no tiling.
 * Because the reductions add in a different order, results agree with the
 * serial oracle to rounding (a CPU test checks that on a 32^3 lattice), not
 * bit for bit, so the parity tests keep using the serial oracle.
 */
#include "clusterlat_oracle.h"

#include <math.h>
#include <omp.h>
#include <stdlib.h>

static long long sites(const orc_model* m) {
  long long s = 1;
  for (int d = 0; d < m->dims; ++d) s *= m->N;
  return s;
}

static long long neighbour(const orc_model* m, long long s, int d, int dir) {
  long long N = m->N, stride = 1;
  for (int k = 0; k < d; ++k) stride *= N;
  long long c = (s / stride) % N;
  long long c2 = (c + dir + N) % N;
  return s + (c2 - c) * stride;
}

static void laplacian(const orc_model* m, const double* f, double* out) {
  long long S = sites(m);
  double dx = m->L / (double)m->N;
  double inv_dx2 = 1.0 / (dx * dx);
#pragma omp parallel for schedule(static)
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

static void dvdf(const orc_model* m, const double* fs, double* out) {
  double phi = fs[0];
  double coupling = 0.0;
  for (int i = 1; i < m->nf; ++i) coupling += m->q[i - 1] * fs[i] * fs[i];
  out[0] = phi * phi * phi + phi * coupling;
  for (int i = 1; i < m->nf; ++i) out[i] = m->q[i - 1] * phi * phi * fs[i];
}

static double potential(const orc_model* m, const double* fs) {
  double phi = fs[0];
  double v = 0.25 * phi * phi * phi * phi;
  for (int i = 1; i < m->nf; ++i) v += 0.5 * m->q[i - 1] * phi * phi * fs[i] * fs[i];
  return v;
}

static void force(const orc_model* m, const double* f, double s, double* F) {
  long long S = sites(m);
  int nf = m->nf;
  for (int i = 0; i < nf; ++i) laplacian(m, f + (long long)i * S, F + (long long)i * S);
#pragma omp parallel for schedule(static)
  for (long long x = 0; x < S; ++x) {
    double fs[4] = {0, 0, 0, 0}, dv[4];
    for (int i = 0; i < nf; ++i) fs[i] = f[(long long)i * S + x];
    dvdf(m, fs, dv);
    for (int i = 0; i < nf; ++i) {
      long long k = (long long)i * S + x;
      F[k] = F[k] - dv[i] + s * fs[i];
    }
  }
}

static double gradient_mean(const orc_model* m, const double* f) {
  long long S = sites(m);
  double dx = m->L / (double)m->N;
  double total = 0.0;
  for (int i = 0; i < m->nf; ++i) {
    const double* fi = f + (long long)i * S;
    double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
    for (long long x = 0; x < S; ++x) {
      for (int d = 0; d < m->dims; ++d) {
        double g = (fi[neighbour(m, x, d, +1)] - fi[x]) / dx;
        acc += 0.5 * g * g;
      }
    }
    total += acc / (double)S;
  }
  return total;
}

static double potential_mean(const orc_model* m, const double* f) {
  long long S = sites(m);
  double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
  for (long long x = 0; x < S; ++x) {
    double fs[4] = {0, 0, 0, 0};
    for (int i = 0; i < m->nf; ++i) fs[i] = f[(long long)i * S + x];
    acc += potential(m, fs);
  }
  return acc / (double)S;
}

static double accel(const orc_model* m, double a, double ap, double G, double V) {
  return (-ap * ap + m->kappa2 * (2.0 * G + 3.0 * V)) / a;
}

int orcp_threads(void) { return omp_get_max_threads(); }

void orcp_set_threads(int n) {
  if (n > 0) omp_set_num_threads(n);
}

/* Same start-up as orc_init. */
int orcp_init(const orc_model* m, double* f, double* v, orc_scale* sc) {
  long long S = sites(m);
  long long n = (long long)m->nf * S;
  double a = 1.0, ap0 = 0.0, app0 = 0.0;
  if (m->expansion) {
    double K = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : K)
    for (long long k = 0; k < n; ++k) K += 0.5 * v[k] * v[k];
    K /= (double)S;
    double G = gradient_mean(m, f);
    double V = potential_mean(m, f);
    double rho = K + G + V;
    if (!(rho >= 0.0)) return -1;
    ap0 = sqrt(m->kappa2 * rho);
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < n; ++k) v[k] = v[k] + (ap0 / a) * f[k];
    app0 = accel(m, a, ap0, G, V);
  }
  double* F = (double*)malloc((size_t)n * sizeof(double));
  if (!F) return -2;
  force(m, f, app0 / a, F);
#pragma omp parallel for schedule(static)
  for (long long k = 0; k < n; ++k) v[k] = v[k] + 0.5 * m->dt * F[k];
  free(F);
  sc->a = a;
  sc->ap = ap0 + 0.5 * m->dt * app0;
  sc->app = app0;
  sc->t = 0.0;
  sc->step = 0;
  return 0;
}

/* Same steps as orc_step: drift, scale factor from G and V of the new f, kick. */
int orcp_step(const orc_model* m, double* f, double* v, orc_scale* sc, long long nsteps) {
  long long S = sites(m);
  long long n = (long long)m->nf * S;
  double dt = m->dt;
  double* F = (double*)malloc((size_t)n * sizeof(double));
  if (!F) return -2;
  int rc = 0;
  for (long long it = 0; it < nsteps; ++it) {
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < n; ++k) f[k] = f[k] + dt * v[k];
    double s = 0.0;
    if (m->expansion) {
      double a = sc->a + dt * sc->ap;
      double G = gradient_mean(m, f);
      double V = potential_mean(m, f);
      double Q = m->kappa2 * (2.0 * G + 3.0 * V) / a;
      double c = 2.0 * sc->ap + dt * Q;
      double disc = 1.0 + dt * c / a;
      if (!(disc >= 0.0)) { rc = -1; break; }
      double u = 2.0 * c / (1.0 + sqrt(disc));
      double app = (u - 2.0 * sc->ap) / dt;
      sc->a = a;
      sc->ap = u - sc->ap;
      sc->app = app;
      s = app / a;
    }
    sc->t = sc->t + dt;
    sc->step += 1;
    force(m, f, s, F);
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < n; ++k) v[k] = v[k] + dt * F[k];
  }
  free(F);
  return rc;
}
