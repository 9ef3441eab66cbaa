/*
 * md_oracle.c -- plain, slow, FP64 CPU oracle for the long-range MD method of
 * arXiv 1212.0262 (Rocha Filho, "Molecular dynamics for long-range interacting
 * systems on Graphic Processing Units").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA path.
 *
 * Everything is written as the plain definition: direct pair sums over j != i
 * with sin/cos of the FP64 difference, sequential loops, no blocking, no
 * reordering.  Build with -O2 -ffp-contract=off so that every product and sum
 * is rounded exactly as written.
 *
 * Layout: positions q and momenta p are arrays of dim*N doubles.  dim = 1 for
 * HMF and Ring (q = theta), dim = 2 for the 2D model (q = [x_0..x_{N-1},
 * y_0..y_{N-1}], p = [px..., py...]), dim = 3 for 3D gravity (x block, y block,
 * z block).  A "harmonic" test model (f = -q) is included only to pin the
 * integrator's order.
 *
 * Readings of the paper taken here (each is pinned by a test):
 *  - Yoshida constants (Sec. 3, Eq. 4): the paper does not print B0, B1, D0,
 *    D1.  The symmetric 4-kick/3-drift split that is 4th order is the
 *    triple-jump composition of the kick-drift-kick leapfrog:
 *    w1 = 1/(2 - 2^(1/3)), w0 = -2^(1/3)/(2 - 2^(1/3)),
 *    B0 = w1/2, B1 = (w0 + w1)/2, D0 = w1, D1 = w0.
 *  - Step list of Sec. 3: the closing kick (item 11) uses the force at the new
 *    positions r(t+dt) from item 10, and item 12 carries that force into the
 *    next step's first kick (first-same-as-last).  The literal reading (stale
 *    f^(I), "f^(II) = f(t+dt)") breaks the scheme's symmetry.
 *  - Ring force sign: Eq. 8 prints +sin/(..)^(3/2); minus the gradient of the
 *    Hamiltonian of Eq. 1 gives the negative of that, which is what is used.
 *  - 2D force (not printed): f_i = -(2/N) sum_j r_ij / (|r_ij|^2 + eps), from
 *    Eq. 3 with the natural log.
 *  - Energies use i<j pair sums (Eqs. 1-3); self terms are excluded.
 *  - 3D self-gravitating particles (not in the paper; its introduction lists
 *    self-gravitating systems among the long-range models and its conclusion
 *    calls other N-particle systems a direct extension): unit masses with the
 *    Kac 1/N coupling and the additive softening of Eqs. 1-3,
 *    V = -(1/N) sum_{i<j} (|r_ij|^2 + eps)^(-1/2),
 *    f_i = -(1/N) sum_j r_ij (|r_ij|^2 + eps)^(-3/2).
 *  - 1D self-gravitating sheets (not one of the paper's three models; its
 *    introduction lists one-dimensional gravity of infinite uniform sheets among
 *    the long-range models): unit masses, Kac 1/N coupling,
 *    V = (1/N) sum_{i<j} |x_i - x_j| (eps = 0) or sqrt((x_i - x_j)^2 + eps) (eps > 0),
 *    f_i = -(1/N) sum_j sign(x_i - x_j) with sign(0) = 0 (eps = 0), or
 *    -(1/N) sum_j d / sqrt(d^2 + eps).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_HMF 0
#define ORA_RING 1
#define ORA_GRAV2D 2
#define ORA_GRAV3D 3
#define ORA_SHEET1D 4
#define ORA_HARMONIC 9

#define ORA_OBS_KINETIC 0
#define ORA_OBS_MAGNETIZATION 1

int ora_dim(int model) { return model == ORA_GRAV2D ? 2 : model == ORA_GRAV3D ? 3 : 1; }

/* Sec. 3, Eq. 4: B0, B1, D0, D1 from the closed form of the triple jump. */
void ora_yoshida(double c[4]) {
  double t = cbrt(2.0);
  double w1 = 1.0 / (2.0 - t);
  double w0 = -t / (2.0 - t);
  c[0] = 0.5 * w1;        /* B0 */
  c[1] = 0.5 * (w0 + w1); /* B1 */
  c[2] = w1;              /* D0 */
  c[3] = w0;              /* D1 */
}

/* ---------------------------------------------------------------- HMF ---- */

/* Eq. 7: Mx = (1/N) sum cos(theta_i), My = (1/N) sum sin(theta_i). */
void ora_magnetization(int64_t N, const double *th, double *mx, double *my) {
  double sx = 0.0, sy = 0.0;
  for (int64_t i = 0; i < N; i++) {
    sx += cos(th[i]);
    sy += sin(th[i]);
  }
  *mx = sx / (double)N;
  *my = sy / (double)N;
}

/* Eq. 6: f_i = cos(theta_i) My - sin(theta_i) Mx (mean-field form). */
void ora_force_hmf(int64_t N, const double *th, double *f) {
  double mx, my;
  ora_magnetization(N, th, &mx, &my);
  for (int64_t i = 0; i < N; i++) f[i] = cos(th[i]) * my - sin(th[i]) * mx;
}

/* Eq. 2 differentiated directly: f_i = -(1/N) sum_{j != i} sin(theta_i - theta_j). */
void ora_force_hmf_pairwise(int64_t N, const double *th, double *f) {
  for (int64_t i = 0; i < N; i++) {
    double s = 0.0;
    for (int64_t j = 0; j < N; j++)
      if (j != i) s += sin(th[i] - th[j]);
    f[i] = -s / (double)N;
  }
}

/* Eq. 5: V = (N/2)(1 - Mx^2 - My^2). */
double ora_potential_hmf(int64_t N, const double *th) {
  double mx, my;
  ora_magnetization(N, th, &mx, &my);
  return 0.5 * (double)N * (1.0 - mx * mx - my * my);
}

/* Eq. 2 directly: V = (1/N) sum_{i<j} [1 - cos(theta_i - theta_j)]. */
double ora_potential_hmf_pairwise(int64_t N, const double *th) {
  double v = 0.0;
  for (int64_t i = 0; i < N; i++)
    for (int64_t j = i + 1; j < N; j++) v += 1.0 - cos(th[i] - th[j]);
  return v / (double)N;
}

/* --------------------------------------------------------------- Ring ---- */

/* Minus the theta_i-gradient of Eq. 1:
 * f_i = -(1/(2 sqrt(2) N)) sum_{j != i} sin(d) / (1 - cos(d) + eps)^(3/2), d = theta_i - theta_j. */
void ora_force_ring(int64_t N, double eps, const double *th, double *f) {
  double c = 1.0 / (2.0 * sqrt(2.0) * (double)N);
  for (int64_t i = 0; i < N; i++) {
    double s = 0.0;
    for (int64_t j = 0; j < N; j++) {
      if (j == i) continue;
      double d = th[i] - th[j];
      double D = 1.0 - cos(d) + eps;
      s += sin(d) / (D * sqrt(D));
    }
    f[i] = -c * s;
  }
}

/* Eq. 1: V = -(1/N) sum_{i<j} 1 / (sqrt(2) sqrt(1 - cos(theta_i - theta_j) + eps)). */
double ora_potential_ring(int64_t N, double eps, const double *th) {
  double v = 0.0;
  for (int64_t i = 0; i < N; i++)
    for (int64_t j = i + 1; j < N; j++)
      v += 1.0 / (sqrt(2.0) * sqrt(1.0 - cos(th[i] - th[j]) + eps));
  return -v / (double)N;
}

/* ----------------------------------------------------------------- 2D ---- */

/* Minus the gradient of Eq. 3: f_i = -(2/N) sum_{j != i} r_ij / (|r_ij|^2 + eps). */
void ora_force_2d(int64_t N, double eps, const double *q, double *f) {
  const double *x = q, *y = q + N;
  for (int64_t i = 0; i < N; i++) {
    double sx = 0.0, sy = 0.0;
    for (int64_t j = 0; j < N; j++) {
      if (j == i) continue;
      double dx = x[i] - x[j], dy = y[i] - y[j];
      double s = dx * dx + dy * dy + eps;
      sx += dx / s;
      sy += dy / s;
    }
    f[i] = -2.0 * sx / (double)N;
    f[N + i] = -2.0 * sy / (double)N;
  }
}

/* Eq. 3: V = (1/N) sum_{i<j} log[(x_i - x_j)^2 + (y_i - y_j)^2 + eps] (natural log). */
double ora_potential_2d(int64_t N, double eps, const double *q) {
  const double *x = q, *y = q + N;
  double v = 0.0;
  for (int64_t i = 0; i < N; i++)
    for (int64_t j = i + 1; j < N; j++) {
      double dx = x[i] - x[j], dy = y[i] - y[j];
      v += log(dx * dx + dy * dy + eps);
    }
  return v / (double)N;
}

/* ----------------------------------------------------------------- 3D ---- */

/* Minus the gradient of V below: f_i = -(1/N) sum_{j != i} r_ij / (|r_ij|^2 + eps)^(3/2). */
void ora_force_3d(int64_t N, double eps, const double *q, double *f) {
  const double *x = q, *y = q + N, *z = q + 2 * N;
  for (int64_t i = 0; i < N; i++) {
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t j = 0; j < N; j++) {
      if (j == i) continue;
      double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
      double s = dx * dx + dy * dy + dz * dz + eps;
      double w = 1.0 / (s * sqrt(s));
      sx += dx * w;
      sy += dy * w;
      sz += dz * w;
    }
    f[i] = -sx / (double)N;
    f[N + i] = -sy / (double)N;
    f[2 * N + i] = -sz / (double)N;
  }
}

/* V = -(1/N) sum_{i<j} (|r_ij|^2 + eps)^(-1/2). */
double ora_potential_3d(int64_t N, double eps, const double *q) {
  const double *x = q, *y = q + N, *z = q + 2 * N;
  double v = 0.0;
  for (int64_t i = 0; i < N; i++)
    for (int64_t j = i + 1; j < N; j++) {
      double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
      v += 1.0 / sqrt(dx * dx + dy * dy + dz * dz + eps);
    }
  return -v / (double)N;
}

/* ------------------------------------------------------------ 1D sheets -- */

static double sgn(double d) { return d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0); }

/* f_i = -(1/N) sum_{j != i} sign(x_i - x_j) (eps = 0), -(1/N) sum_j d / sqrt(d^2 + eps). */
void ora_force_sheet(int64_t N, double eps, const double *x, double *f) {
  for (int64_t i = 0; i < N; i++) {
    double s = 0.0;
    for (int64_t j = 0; j < N; j++) {
      if (j == i) continue;
      double d = x[i] - x[j];
      s += eps > 0.0 ? d / sqrt(d * d + eps) : sgn(d);
    }
    f[i] = -s / (double)N;
  }
}

/* The eps = 0 force with every sign decided on the FP32-rounded positions (the
 * precision in which the FP32 pair kernel takes the decision). */
void ora_force_sheet_f32(int64_t N, const double *x, double *f) {
  for (int64_t i = 0; i < N; i++) {
    double s = 0.0;
    for (int64_t j = 0; j < N; j++) {
      if (j == i) continue;
      float a = (float)x[i], b = (float)x[j];
      s += a > b ? 1.0 : (a < b ? -1.0 : 0.0);
    }
    f[i] = -s / (double)N;
  }
}

/* V = (1/N) sum_{i<j} |x_i - x_j| (eps = 0) or sqrt((x_i - x_j)^2 + eps). */
double ora_potential_sheet(int64_t N, double eps, const double *x) {
  double v = 0.0;
  for (int64_t i = 0; i < N; i++)
    for (int64_t j = i + 1; j < N; j++) {
      double d = x[i] - x[j];
      v += eps > 0.0 ? sqrt(d * d + eps) : fabs(d);
    }
  return v / (double)N;
}

/* ------------------------------------------------------------ generic ---- */

void ora_force(int model, int64_t N, double eps, const double *q, double *f) {
  switch (model) {
  case ORA_HMF: ora_force_hmf(N, q, f); break;
  case ORA_RING: ora_force_ring(N, eps, q, f); break;
  case ORA_GRAV2D: ora_force_2d(N, eps, q, f); break;
  case ORA_GRAV3D: ora_force_3d(N, eps, q, f); break;
  case ORA_SHEET1D: ora_force_sheet(N, eps, q, f); break;
  case ORA_HARMONIC:
    for (int64_t i = 0; i < N; i++) f[i] = -q[i];
    break;
  }
}

double ora_potential(int model, int64_t N, double eps, const double *q) {
  switch (model) {
  case ORA_HMF: return ora_potential_hmf(N, q);
  case ORA_RING: return ora_potential_ring(N, eps, q);
  case ORA_GRAV2D: return ora_potential_2d(N, eps, q);
  case ORA_GRAV3D: return ora_potential_3d(N, eps, q);
  case ORA_SHEET1D: return ora_potential_sheet(N, eps, q);
  case ORA_HARMONIC: {
    double v = 0.0;
    for (int64_t i = 0; i < N; i++) v += 0.5 * q[i] * q[i];
    return v;
  }
  }
  return NAN;
}

/* K = (1/2) sum p^2 over all dim*N components (Eqs. 1-3). */
double ora_kinetic(int64_t n, const double *p) {
  double k = 0.0;
  for (int64_t i = 0; i < n; i++) k += p[i] * p[i];
  return 0.5 * k;
}

/* Per-particle scale of the force sum, sum_j |f_ij| (per component), used to
 * state the summation-order tolerance of a force comparison. */
void ora_force_abs(int model, int64_t N, double eps, const double *q, double *out) {
  if (model == ORA_HMF) {
    double ac = 0.0, as = 0.0;
    for (int64_t j = 0; j < N; j++) {
      ac += fabs(cos(q[j]));
      as += fabs(sin(q[j]));
    }
    for (int64_t i = 0; i < N; i++)
      out[i] = (fabs(cos(q[i])) * as + fabs(sin(q[i])) * ac) / (double)N;
  } else if (model == ORA_RING) {
    double c = 1.0 / (2.0 * sqrt(2.0) * (double)N);
    for (int64_t i = 0; i < N; i++) {
      double s = 0.0;
      for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        double d = q[i] - q[j];
        double D = 1.0 - cos(d) + eps;
        s += fabs(sin(d)) / (D * sqrt(D));
      }
      out[i] = c * s;
    }
  } else if (model == ORA_GRAV2D) {
    const double *x = q, *y = q + N;
    for (int64_t i = 0; i < N; i++) {
      double sx = 0.0, sy = 0.0;
      for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        double dx = x[i] - x[j], dy = y[i] - y[j];
        double s = dx * dx + dy * dy + eps;
        sx += fabs(dx) / s;
        sy += fabs(dy) / s;
      }
      out[i] = 2.0 * sx / (double)N;
      out[N + i] = 2.0 * sy / (double)N;
    }
  } else if (model == ORA_GRAV3D) {
    const double *x = q, *y = q + N, *z = q + 2 * N;
    for (int64_t i = 0; i < N; i++) {
      double sx = 0.0, sy = 0.0, sz = 0.0;
      for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
        double s = dx * dx + dy * dy + dz * dz + eps;
        double w = 1.0 / (s * sqrt(s));
        sx += fabs(dx) * w;
        sy += fabs(dy) * w;
        sz += fabs(dz) * w;
      }
      out[i] = sx / (double)N;
      out[N + i] = sy / (double)N;
      out[2 * N + i] = sz / (double)N;
    }
  } else if (model == ORA_SHEET1D) {
    for (int64_t i = 0; i < N; i++) {
      double s = 0.0;
      for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        double d = q[i] - q[j];
        s += eps > 0.0 ? fabs(d) / sqrt(d * d + eps) : fabs(sgn(d));
      }
      out[i] = s / (double)N;
    }
  } else {
    for (int64_t i = 0; i < N; i++) out[i] = fabs(q[i]);
  }
}

/* Forces on the particles listed in rows[0..nrows-1] only (same definitions as
 * ora_force; HMF uses the mean field of all N angles).  out has nrows*dim
 * entries: [f_row0.., (fy_row0..)]; out_abs (may be NULL) gets sum_j |f_ij| in
 * the same layout.  Used to check large systems on samples. */
void ora_force_rows(int model, int64_t N, double eps, const double *q, const int64_t *rows,
                    int64_t nrows, double *out, double *out_abs) {
  if (model == ORA_HMF) {
    double mx, my, ac = 0.0, as = 0.0;
    ora_magnetization(N, q, &mx, &my);
    for (int64_t j = 0; j < N; j++) {
      ac += fabs(cos(q[j]));
      as += fabs(sin(q[j]));
    }
    for (int64_t r = 0; r < nrows; r++) {
      double t = q[rows[r]];
      out[r] = cos(t) * my - sin(t) * mx;
      if (out_abs) out_abs[r] = (fabs(cos(t)) * as + fabs(sin(t)) * ac) / (double)N;
    }
  } else if (model == ORA_RING) {
    double c = 1.0 / (2.0 * sqrt(2.0) * (double)N);
    for (int64_t r = 0; r < nrows; r++) {
      int64_t i = rows[r];
      double s = 0.0, sa = 0.0;
      for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        double d = q[i] - q[j];
        double D = 1.0 - cos(d) + eps;
        s += sin(d) / (D * sqrt(D));
        sa += fabs(sin(d)) / (D * sqrt(D));
      }
      out[r] = -c * s;
      if (out_abs) out_abs[r] = c * sa;
    }
  } else if (model == ORA_GRAV2D) {
    const double *x = q, *y = q + N;
    for (int64_t r = 0; r < nrows; r++) {
      int64_t i = rows[r];
      double sx = 0.0, sy = 0.0, ax = 0.0, ay = 0.0;
      for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        double dx = x[i] - x[j], dy = y[i] - y[j];
        double s = dx * dx + dy * dy + eps;
        sx += dx / s;
        sy += dy / s;
        ax += fabs(dx) / s;
        ay += fabs(dy) / s;
      }
      out[r] = -2.0 * sx / (double)N;
      out[nrows + r] = -2.0 * sy / (double)N;
      if (out_abs) {
        out_abs[r] = 2.0 * ax / (double)N;
        out_abs[nrows + r] = 2.0 * ay / (double)N;
      }
    }
  } else if (model == ORA_GRAV3D) {
    const double *x = q, *y = q + N, *z = q + 2 * N;
    for (int64_t r = 0; r < nrows; r++) {
      int64_t i = rows[r];
      double sx = 0.0, sy = 0.0, sz = 0.0, ax = 0.0, ay = 0.0, az = 0.0;
      for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
        double s = dx * dx + dy * dy + dz * dz + eps;
        double w = 1.0 / (s * sqrt(s));
        sx += dx * w;
        sy += dy * w;
        sz += dz * w;
        ax += fabs(dx) * w;
        ay += fabs(dy) * w;
        az += fabs(dz) * w;
      }
      out[r] = -sx / (double)N;
      out[nrows + r] = -sy / (double)N;
      out[2 * nrows + r] = -sz / (double)N;
      if (out_abs) {
        out_abs[r] = ax / (double)N;
        out_abs[nrows + r] = ay / (double)N;
        out_abs[2 * nrows + r] = az / (double)N;
      }
    }
  } else if (model == ORA_SHEET1D) {
    for (int64_t r = 0; r < nrows; r++) {
      int64_t i = rows[r];
      double s = 0.0, a = 0.0;
      for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        double d = q[i] - q[j];
        double t = eps > 0.0 ? d / sqrt(d * d + eps) : sgn(d);
        s += t;
        a += fabs(t);
      }
      out[r] = -s / (double)N;
      if (out_abs) out_abs[r] = a / (double)N;
    }
  }
}

/* ------------------------------------------------------------ integrator -- */

static void kick(int64_t n, double coef, const double *f, double *p) {
  for (int64_t i = 0; i < n; i++) p[i] = p[i] + coef * f[i];
}
static void drift(int64_t n, double coef, const double *p, double *q) {
  for (int64_t i = 0; i < n; i++) q[i] = q[i] + coef * p[i];
}

/* The step list of Sec. 3 (items 1-12) with Eq. 4's splitting, taken nsteps
 * times in place.  Item 1 is computed once; items 10-12 hand the force at
 * r(t+dt) to the next step (first-same-as-last).  Returns 0, or -1 on
 * allocation failure. */
int ora_step(int model, int64_t N, double eps, double dt, int64_t nsteps, double *q, double *p) {
  int64_t n = (int64_t)ora_dim(model) * N;
  double c[4];
  ora_yoshida(c);
  double *f = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!f) return -1;
  ora_force(model, N, eps, q, f);       /* item 1 */
  for (int64_t s = 0; s < nsteps; s++) {
    kick(n, c[0] * dt, f, p);            /* item 2  */
    drift(n, c[2] * dt, p, q);           /* item 3  */
    ora_force(model, N, eps, q, f);      /* item 4  */
    kick(n, c[1] * dt, f, p);            /* item 5  */
    drift(n, c[3] * dt, p, q);           /* item 6  */
    ora_force(model, N, eps, q, f);      /* item 7  */
    kick(n, c[1] * dt, f, p);            /* item 8  */
    drift(n, c[2] * dt, p, q);           /* item 9  */
    ora_force(model, N, eps, q, f);      /* item 10 */
    kick(n, c[0] * dt, f, p);            /* item 11 */
  }
  free(f);
  return 0;
}

/* ----------------------------------------------- Jacobian-vector products -- */

/* out = J(q) v with J = df/dq (symmetric, equal to minus the Hessian of V),
 * written as the derivative of each pair term above. */
void ora_hvp(int model, int64_t N, double eps, const double *q, const double *v, double *out) {
  if (model == ORA_HMF) {
    /* f_i = -(1/N) sum_j sin(t_i - t_j):  (Jv)_i = -(1/N) sum_j cos(t_i - t_j)(v_i - v_j). */
    for (int64_t i = 0; i < N; i++) {
      double s = 0.0;
      for (int64_t j = 0; j < N; j++)
        if (j != i) s += cos(q[i] - q[j]) * (v[i] - v[j]);
      out[i] = -s / (double)N;
    }
  } else if (model == ORA_RING) {
    /* f_i = sum_j g(d_ij), g(d) = -c sin(d) D^(-3/2), D = 1 - cos d + eps;
     * g'(d) = -c [cos(d) D^(-3/2) - (3/2) sin(d)^2 D^(-5/2)]. */
    double c = 1.0 / (2.0 * sqrt(2.0) * (double)N);
    for (int64_t i = 0; i < N; i++) {
      double s = 0.0;
      for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        double d = q[i] - q[j];
        double D = 1.0 - cos(d) + eps;
        double sn = sin(d);
        double gp = -c * (cos(d) / (D * sqrt(D)) - 1.5 * sn * sn / (D * D * sqrt(D)));
        s += gp * (v[i] - v[j]);
      }
      out[i] = s;
    }
  } else if (model == ORA_GRAV2D) {
    /* phi(r) = -(2/N) r / s, s = |r|^2 + eps:  dphi/dr w = -(2/N)[w/s - 2 r (r.w)/s^2]. */
    const double *x = q, *y = q + N, *vx = v, *vy = v + N;
    for (int64_t i = 0; i < N; i++) {
      double ax = 0.0, ay = 0.0;
      for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        double dx = x[i] - x[j], dy = y[i] - y[j];
        double wx = vx[i] - vx[j], wy = vy[i] - vy[j];
        double s = dx * dx + dy * dy + eps;
        double rw = dx * wx + dy * wy;
        ax += wx / s - 2.0 * dx * rw / (s * s);
        ay += wy / s - 2.0 * dy * rw / (s * s);
      }
      out[i] = -2.0 * ax / (double)N;
      out[N + i] = -2.0 * ay / (double)N;
    }
  } else if (model == ORA_GRAV3D) {
    /* phi(r) = -(1/N) r s^(-3/2):  dphi/dr w = -(1/N)[w s^(-3/2) - 3 r (r.w) s^(-5/2)]. */
    const double *x = q, *y = q + N, *z = q + 2 * N, *vx = v, *vy = v + N, *vz = v + 2 * N;
    for (int64_t i = 0; i < N; i++) {
      double ax = 0.0, ay = 0.0, az = 0.0;
      for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
        double wx = vx[i] - vx[j], wy = vy[i] - vy[j], wz = vz[i] - vz[j];
        double s = dx * dx + dy * dy + dz * dz + eps;
        double s32 = s * sqrt(s), s52 = s * s * sqrt(s);
        double rw = dx * wx + dy * wy + dz * wz;
        ax += wx / s32 - 3.0 * dx * rw / s52;
        ay += wy / s32 - 3.0 * dy * rw / s52;
        az += wz / s32 - 3.0 * dz * rw / s52;
      }
      out[i] = -ax / (double)N;
      out[N + i] = -ay / (double)N;
      out[2 * N + i] = -az / (double)N;
    }
  } else if (model == ORA_SHEET1D) {
    /* eps > 0: phi(d) = -(1/N) d / sqrt(d^2 + eps), dphi/dd = -(1/N) eps (d^2 + eps)^(-3/2);
     * eps = 0: the sign force is piecewise constant, its derivative 0 between crossings. */
    for (int64_t i = 0; i < N; i++) {
      double a = 0.0;
      if (eps > 0.0)
        for (int64_t j = 0; j < N; j++) {
          if (j == i) continue;
          double d = q[i] - q[j];
          double sd = d * d + eps;
          a += eps / (sd * sqrt(sd)) * (v[i] - v[j]);
        }
      out[i] = -a / (double)N;
    }
  } else {
    for (int64_t i = 0; i < N; i++) out[i] = -v[i];
  }
}

/* Mean-field form of the HMF product, from Eqs. 6-7:
 * (Jv)_i = -(sin t_i My + cos t_i Mx) v_i + cos t_i A + sin t_i B,
 * A = (1/N) sum cos t_k v_k, B = (1/N) sum sin t_k v_k. */
void ora_hvp_hmf_meanfield(int64_t N, const double *q, const double *v, double *out) {
  double mx, my, a = 0.0, b = 0.0;
  ora_magnetization(N, q, &mx, &my);
  for (int64_t k = 0; k < N; k++) {
    a += cos(q[k]) * v[k];
    b += sin(q[k]) * v[k];
  }
  a /= (double)N;
  b /= (double)N;
  for (int64_t i = 0; i < N; i++)
    out[i] = -(sin(q[i]) * my + cos(q[i]) * mx) * v[i] + cos(q[i]) * a + sin(q[i]) * b;
}

/* out = df/d(eps) at q (zero for HMF and the harmonic model). */
void ora_dforce_deps(int model, int64_t N, double eps, const double *q, double *out) {
  if (model == ORA_RING) {
    /* d/deps of -c sin(d) D^(-3/2) = (3c/2) sin(d) D^(-5/2). */
    double c = 1.0 / (2.0 * sqrt(2.0) * (double)N);
    for (int64_t i = 0; i < N; i++) {
      double s = 0.0;
      for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        double d = q[i] - q[j];
        double D = 1.0 - cos(d) + eps;
        s += sin(d) / (D * D * sqrt(D));
      }
      out[i] = 1.5 * c * s;
    }
  } else if (model == ORA_GRAV2D) {
    /* d/deps of -(2/N) r/s = (2/N) r / s^2. */
    const double *x = q, *y = q + N;
    for (int64_t i = 0; i < N; i++) {
      double sx = 0.0, sy = 0.0;
      for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        double dx = x[i] - x[j], dy = y[i] - y[j];
        double s = dx * dx + dy * dy + eps;
        sx += dx / (s * s);
        sy += dy / (s * s);
      }
      out[i] = 2.0 * sx / (double)N;
      out[N + i] = 2.0 * sy / (double)N;
    }
  } else if (model == ORA_GRAV3D) {
    /* d/deps of -(1/N) r s^(-3/2) = (3/(2N)) r s^(-5/2). */
    const double *x = q, *y = q + N, *z = q + 2 * N;
    for (int64_t i = 0; i < N; i++) {
      double sx = 0.0, sy = 0.0, sz = 0.0;
      for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
        double s = dx * dx + dy * dy + dz * dz + eps;
        double s52 = s * s * sqrt(s);
        sx += dx / s52;
        sy += dy / s52;
        sz += dz / s52;
      }
      out[i] = 1.5 * sx / (double)N;
      out[N + i] = 1.5 * sy / (double)N;
      out[2 * N + i] = 1.5 * sz / (double)N;
    }
  } else if (model == ORA_SHEET1D && eps > 0.0) {
    /* d/deps of -(1/N) d (d^2 + eps)^(-1/2) = (1/(2N)) d (d^2 + eps)^(-3/2). */
    for (int64_t i = 0; i < N; i++) {
      double a = 0.0;
      for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        double d = q[i] - q[j];
        double sd = d * d + eps;
        a += d / (sd * sqrt(sd));
      }
      out[i] = 0.5 * a / (double)N;
    }
  } else {
    int64_t n = (int64_t)ora_dim(model) * N;
    for (int64_t i = 0; i < n; i++) out[i] = 0.0;
  }
}

/* ------------------------------------------------------- discrete adjoint -- */

static void hvp_fast(int model, int64_t N, double eps, const double *q, const double *v, double *out) {
  if (model == ORA_HMF)
    ora_hvp_hmf_meanfield(N, q, v, out);
  else
    ora_hvp(model, N, eps, q, v, out);
}

/* Observable at the final state and its gradient with respect to (q, p).
 * KINETIC: O = (1/2) sum p^2.  MAGNETIZATION (angle models): O = |M| of Eq. 7. */
static double observable(int model, int obs, int64_t N, const double *q, const double *p,
                         double *lq, double *lp) {
  int64_t n = (int64_t)ora_dim(model) * N;
  if (obs == ORA_OBS_KINETIC) {
    for (int64_t i = 0; i < n; i++) {
      lq[i] = 0.0;
      lp[i] = p[i];
    }
    return ora_kinetic(n, p);
  }
  double mx, my;
  ora_magnetization(N, q, &mx, &my);
  double m = sqrt(mx * mx + my * my);
  for (int64_t i = 0; i < N; i++) {
    lq[i] = (my * cos(q[i]) - mx * sin(q[i])) / ((double)N * m);
    lp[i] = 0.0;
  }
  return m;
}

/* Gradient of O(state after nsteps) with respect to the initial q0, p0 and eps,
 * by the exact reverse of the step list above.  The forward pass stores the
 * positions of every kick; the reverse pass applies, map by map from last to
 * first, the transposed Jacobians:
 *   drift q' = q + d dt p :  lp += d dt lq
 *   kick  p' = p + b dt f(q):  lq += b dt J(q) lp,  geps += b dt <lp, df/deps(q)>.
 * Returns 0, -1 on allocation failure, -2 for an unsupported observable. */
int ora_grad(int model, int64_t N, double eps, double dt, int64_t nsteps, int obs,
             const double *q0, const double *p0, double *gq, double *gp, double *geps,
             double *value) {
  if (obs == ORA_OBS_MAGNETIZATION && model != ORA_HMF && model != ORA_RING) return -2;
  int64_t n = (int64_t)ora_dim(model) * N;
  size_t nb = sizeof(double) * (size_t)n;
  double c[4];
  ora_yoshida(c);
  const double kb[4] = {c[0], c[1], c[1], c[0]}; /* kick coefficients in step order */
  const double dd[3] = {c[2], c[3], c[2]};       /* drift coefficients in step order */
  double *qs = (double *)malloc(nb * (size_t)(4 * nsteps + 1));
  double *q = (double *)malloc(nb), *p = (double *)malloc(nb), *f = (double *)malloc(nb);
  double *t1 = (double *)malloc(nb), *t2 = (double *)malloc(nb);
  if (!qs || !q || !p || !f || !t1 || !t2) {
    free(qs); free(q); free(p); free(f); free(t1); free(t2);
    return -1;
  }
  memcpy(q, q0, nb);
  memcpy(p, p0, nb);
  /* forward: kick k of step s happens at qs[4 s + k] */
  for (int64_t s = 0; s < nsteps; s++) {
    for (int k = 0; k < 4; k++) {
      memcpy(qs + (size_t)(4 * s + k) * (size_t)n, q, nb);
      ora_force(model, N, eps, q, f);
      kick(n, kb[k] * dt, f, p);
      if (k < 3) drift(n, dd[k] * dt, p, q);
    }
  }
  double *lq = gq, *lp = gp;
  *value = observable(model, obs, N, q, p, lq, lp);
  double ge = 0.0;
  for (int64_t s = nsteps - 1; s >= 0; s--) {
    for (int k = 3; k >= 0; k--) {
      if (k < 3)
        for (int64_t i = 0; i < n; i++) lp[i] = lp[i] + dd[k] * dt * lq[i];
      const double *qk = qs + (size_t)(4 * s + k) * (size_t)n;
      hvp_fast(model, N, eps, qk, lp, t1);
      ora_dforce_deps(model, N, eps, qk, t2);
      double dot = 0.0;
      for (int64_t i = 0; i < n; i++) {
        lq[i] = lq[i] + kb[k] * dt * t1[i];
        dot += lp[i] * t2[i];
      }
      ge += kb[k] * dt * dot;
    }
  }
  if (geps) *geps = ge;
  free(qs); free(q); free(p); free(f); free(t1); free(t2);
  return 0;
}

/* Observable after nsteps from (q0, p0), used by finite-difference checks. */
double ora_observable_after(int model, int64_t N, double eps, double dt, int64_t nsteps, int obs,
                            const double *q0, const double *p0) {
  int64_t n = (int64_t)ora_dim(model) * N;
  size_t nb = sizeof(double) * (size_t)n;
  double *q = (double *)malloc(nb), *p = (double *)malloc(nb);
  double *lq = (double *)malloc(nb), *lp = (double *)malloc(nb);
  double v = NAN;
  if (q && p && lq && lp) {
    memcpy(q, q0, nb);
    memcpy(p, p0, nb);
    if (ora_step(model, N, eps, dt, nsteps, q, p) == 0) v = observable(model, obs, N, q, p, lq, lp);
  }
  free(q); free(p); free(lq); free(lp);
  return v;
}
