/* Linked-cell CPU implementation of the method's force fields and integrator (FP64, OpenMP):
 * the CPU throughput baseline the GPU path is compared with.  It is neither the parity oracle nor
 * the product: the oracle (brute force, oracle/) pins it in tests, and it shares no code with the
 * oracle or with the CUDA library.
 *
 * What it computes (arXiv 2507.11172):
 *   - Lennard-Jones 12-6 forces and energy over every pair with r <= r_c2 (Sec. 2.1, Sec. 4.2.2);
 *   - Axilrod-Teller-Muto forces and energy over every triplet whose three pair distances are all
 *     <= r_c3 (Sec. 2.1; the cutoff rule of the caption of Fig. 2 and Sec. 4.2.2);
 *   - the single-loop r-RESPA integrator of Algorithm 2 (Sec. 4.1): F3 kicks of dt_outer / 2 around
 *     each outer step, velocity Verlet on F2 with dt = dt_outer / k inside it.
 * How: the traversal the paper's shared-memory Cutoff method uses (linked cells of edge >= the
 * largest cutoff, every particle against the 27 cells around its own, no Newton 3: each thread owns
 * the full force of its particles, so no two threads write the same sum).  A particle's ATM force is
 * the sum over the pairs (j, k) of its neighbours within r_c3 with r_jk <= r_c3; each triplet is
 * therefore met once from each of its three members.  Positions are periodic in a cube of side L;
 * displacements take the minimum image.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* cell grid: particles of cell c are idx[start[c]] .. idx[start[c + 1] - 1] */
typedef struct {
  int nc;
  double edge;
  int *start, *idx, *cell;
  double *xs;  /* positions folded into [0, L), in cell order (xs[3 q ..] belongs to particle idx[q]) */
} Grid;

static void grid_free(Grid *g) {
  free(g->start);
  free(g->idx);
  free(g->cell);
  free(g->xs);
  memset(g, 0, sizeof(*g));
}

static double fold(double x, double L) {
  double y = x - L * floor(x / L);
  return y >= L ? y - L : y;
}

/* cells of edge L / nc >= reach, nc >= 3 per side (so the 27 cells around any cell are distinct) */
static int grid_build(int64_t n, const double *x, double L, double reach, Grid *g) {
  memset(g, 0, sizeof(*g));
  const int nc = (int)floor(L / reach);
  if (nc < 3) return -1;
  g->nc = nc;
  g->edge = L / nc;
  const int64_t ncell = (int64_t)nc * nc * nc;
  g->start = (int *)calloc((size_t)ncell + 1, sizeof(int));
  g->idx = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
  g->cell = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
  g->xs = (double *)malloc((size_t)(n > 0 ? 3 * n : 1) * sizeof(double));
  if (!g->start || !g->idx || !g->cell || !g->xs) {
    grid_free(g);
    return -2;
  }
  for (int64_t i = 0; i < n; ++i) {
    int c[3];
    for (int a = 0; a < 3; ++a) {
      c[a] = (int)(fold(x[3 * i + a], L) / g->edge);
      if (c[a] >= nc) c[a] = nc - 1;
    }
    g->cell[i] = (c[2] * nc + c[1]) * nc + c[0];
    g->start[g->cell[i] + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) g->start[c + 1] += g->start[c];
  int *fill = (int *)malloc((size_t)ncell * sizeof(int));
  if (!fill) {
    grid_free(g);
    return -2;
  }
  memcpy(fill, g->start, (size_t)ncell * sizeof(int));
  for (int64_t i = 0; i < n; ++i) {
    const int q = fill[g->cell[i]]++;
    g->idx[q] = (int)i;
    for (int a = 0; a < 3; ++a) g->xs[3 * q + a] = fold(x[3 * i + a], L);
  }
  free(fill);
  return 0;
}

/* the 27 cells around cell c (periodic) and, per cell, the shift that brings its particles next to c:
 * a stencil cell across the box boundary holds the periodic images one box length away */
static void grid_stencil(const Grid *g, int c, double L, int out[27], double shift[27][3]) {
  const int nc = g->nc, cc[3] = {c % nc, (c / nc) % nc, c / (nc * nc)};
  int m = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int dd[3] = {dx, dy, dz};
        int w[3];
        for (int a = 0; a < 3; ++a) {
          const int t = cc[a] + dd[a];
          w[a] = t < 0 ? t + nc : (t >= nc ? t - nc : t);
          shift[m][a] = t < 0 ? -L : (t >= nc ? L : 0.0);
        }
        out[m++] = (w[2] * nc + w[1]) * nc + w[0];
      }
}

/* LJ: per particle, the full force from every neighbour within r_c; u = the pair energy (each pair
 * counted once), w = the pair virial sum r . F */
static void lj_pass(int64_t n, double L, const Grid *g, double eps, double sigma, double rc, double *f, double *u,
                    double *w) {
  const double rc2 = rc * rc, s2 = sigma * sigma;
  const double *xs = g->xs;
  double usum = 0.0, wsum = 0.0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : usum, wsum)
  for (int64_t qi = 0; qi < n; ++qi) {
    const int i = g->idx[qi];
    int st[27];
    double sh[27][3];
    grid_stencil(g, g->cell[i], L, st, sh);
    const double xi = xs[3 * qi], yi = xs[3 * qi + 1], zi = xs[3 * qi + 2];
    double fx = 0.0, fy = 0.0, fz = 0.0, ui = 0.0, wi = 0.0;
    for (int s = 0; s < 27; ++s) {
      const double ox = sh[s][0] - xi, oy = sh[s][1] - yi, oz = sh[s][2] - zi;
      for (int q = g->start[st[s]]; q < g->start[st[s] + 1]; ++q) {
        if (q == qi) continue;
        const double dx = xs[3 * q] + ox, dy = xs[3 * q + 1] + oy, dz = xs[3 * q + 2] + oz;  /* x_j - x_i */
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 > rc2) continue;
        const double sr2 = s2 / r2, sr6 = sr2 * sr2 * sr2;
        /* U = 4 eps (sr12 - sr6); F_i = -(dU/dr) (x_i - x_j) / r = -gs d with d = x_j - x_i */
        const double gs = 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r2;
        fx -= gs * dx;
        fy -= gs * dy;
        fz -= gs * dz;
        ui += 4.0 * eps * (sr6 * sr6 - sr6);
        wi += gs * r2;
      }
    }
    f[3 * i] = fx;
    f[3 * i + 1] = fy;
    f[3 * i + 2] = fz;
    usum += 0.5 * ui;
    wsum += 0.5 * wi;
  }
  *u = usum;
  *w = wsum;
}

/* ATM, squared-distance form: a = r_ij^2, b = r_ik^2, c = r_jk^2, s = abc, A = a + b - c,
 * B = a - b + c, C = -a + b + c, P = ABC (= 8 abc cos g_i cos g_j cos g_k by the law of cosines):
 *   phi = nu s^(-3/2) (1 + 3 P / (8 s)),
 *   dphi/da = s^(-5/2) (-3/2 nu bc + 3/8 nu dP/da - 15/16 nu P / a),  dP/da = BC + AC - AB,
 *   dphi/db = s^(-5/2) (-3/2 nu ac + 3/8 nu dP/db - 15/16 nu P / b),  dP/db = BC - AC + AB,
 * and with d_ij = x_j - x_i, d_ik = x_k - x_i: F_i = -grad_i phi = 2 dphi/da d_ij + 2 dphi/db d_ik.
 * Per particle: its share of the force from every triplet it belongs to; u = the triplet energy (each
 * triplet once), *ntrip = the number of triplets within the cutoff. */
static int atm_pass(int64_t n, double L, const Grid *g, double nu, double rc, double *f,
                    double *u, int64_t *ntrip) {
  const double rc2 = rc * rc;
  int maxc = 0;
  const int64_t ncell = (int64_t)g->nc * g->nc * g->nc;
  for (int64_t c = 0; c < ncell; ++c)
    if (g->start[c + 1] - g->start[c] > maxc) maxc = g->start[c + 1] - g->start[c];
  const int cap = maxc > 0 ? 27 * maxc : 1;  /* at most every particle of the 27 cells */
  double usum = 0.0;
  int64_t csum = 0;
  int bad = 0;
#pragma omp parallel reduction(+ : usum, csum) reduction(| : bad)
  {
    double *nd = (double *)malloc((size_t)cap * 4 * sizeof(double));  /* d (3) and |d|^2 per neighbour */
    if (!nd) bad = 1;
#pragma omp for schedule(dynamic, 64)
    for (int64_t qi = 0; qi < n; ++qi) {
      if (!nd) continue;
      const int i = g->idx[qi];
      int st[27], m = 0;
      double sh[27][3];
      grid_stencil(g, g->cell[i], L, st, sh);
      const double *xs = g->xs;
      for (int s = 0; s < 27; ++s) {
        const double ox = sh[s][0] - xs[3 * qi], oy = sh[s][1] - xs[3 * qi + 1], oz = sh[s][2] - xs[3 * qi + 2];
        for (int q = g->start[st[s]]; q < g->start[st[s] + 1]; ++q) {
          if (q == qi) continue;
          const double dx = xs[3 * q] + ox, dy = xs[3 * q + 1] + oy, dz = xs[3 * q + 2] + oz;  /* x_j - x_i */
          const double r2 = dx * dx + dy * dy + dz * dz;
          if (r2 > rc2) continue;
          nd[4 * m] = dx;
          nd[4 * m + 1] = dy;
          nd[4 * m + 2] = dz;
          nd[4 * m + 3] = r2;
          ++m;
        }
      }
      double fi[3] = {0.0, 0.0, 0.0}, ui = 0.0;
      int64_t ci = 0;
      for (int p = 0; p < m; ++p) {
        const double *dp = nd + 4 * p;
        const double a = dp[3];
        for (int q = p + 1; q < m; ++q) {
          const double *dq = nd + 4 * q;
          const double ex = dq[0] - dp[0], ey = dq[1] - dp[1], ez = dq[2] - dp[2];
          const double c = ex * ex + ey * ey + ez * ez;
          if (c > rc2) continue;
          const double b = dq[3];
          const double s = a * b * c;
          const double A = a + b - c, B = a - b + c, C = -a + b + c;
          const double P = A * B * C;
          const double is = 1.0 / s, r3 = is * sqrt(is), r5 = r3 * is;  /* s^(-3/2), s^(-5/2) */
          const double pa = r5 * nu * (-1.5 * b * c + 0.375 * (B * C + A * C - A * B) - 0.9375 * P / a);
          const double pb = r5 * nu * (-1.5 * a * c + 0.375 * (B * C - A * C + A * B) - 0.9375 * P / b);
          for (int k = 0; k < 3; ++k) fi[k] += 2.0 * pa * dp[k] + 2.0 * pb * dq[k];
          ui += nu * r3 * (1.0 + 0.375 * P * is);
          ++ci;
        }
      }
      for (int k = 0; k < 3; ++k) f[3 * i + k] = fi[k];
      usum += ui;
      csum += ci;
    }
    free(nd);
  }
  if (bad) return -2;
  *u = usum / 3.0;   /* each triplet was met from its three members */
  *ntrip = csum / 3;
  return 0;
}

/* F2 and F3 at x with their energies (and the LJ virial); returns 0, -1 for a box of fewer than three
 * cells per side of the largest cutoff, -2 when memory runs out */
int cells_forces(int64_t n, const double *x, double L, double eps, double sigma, double rc2, double nu, double rc3,
                 double *f2, double *f3, double *out) {
  if (n < 0 || !(L > 0.0) || !(rc2 > 0.0) || !(rc3 > 0.0) || !x || !f2 || !f3 || !out) return -1;
  Grid g;
  const int st = grid_build(n, x, L, rc2 > rc3 ? rc2 : rc3, &g);
  if (st) return st;
  double u2, w2, u3;
  int64_t nt = 0;
  lj_pass(n, L, &g, eps, sigma, rc2, f2, &u2, &w2);
  const int sa = atm_pass(n, L, &g, nu, rc3, f3, &u3, &nt);
  grid_free(&g);
  if (sa) return sa;
  out[0] = u2;
  out[1] = w2;
  out[2] = u3;
  out[3] = (double)nt;
  return 0;
}

static double now_s(void) {
#ifdef _OPENMP
  return omp_get_wtime();
#else
  return 0.0;
#endif
}

/* Algorithm 2 for n_outer outer steps of k inner steps (dt = dt_outer / k) from (x, v) in place, with
 * the forces F2b(x), F3b(x) at the start in f2, f3 (computed first when have_forces is 0) and left
 * there at the end.  out: [U2, U3 at the end, interacting triplets summed over the ATM evaluations,
 * seconds in LJ evaluations, seconds in ATM evaluations, number of ATM evaluations]. */
int cells_respa(int64_t n, double *x, double *v, double L, double mass, double eps, double sigma, double rc2,
                double nu, double rc3, int n_outer, int k, double dt_outer, double *f2, double *f3, int have_forces,
                double *out) {
  if (n < 0 || n_outer < 0 || k < 1 || !(dt_outer > 0.0) || !(mass > 0.0) || !x || !v || !f2 || !f3 || !out)
    return -1;
  const double reach = rc2 > rc3 ? rc2 : rc3;
  const double dt = dt_outer / k, h3 = dt * k / (2.0 * mass), h2 = dt / (2.0 * mass), hx = dt * dt / (2.0 * mass);
  double u2 = 0.0, w2 = 0.0, u3 = 0.0, trip = 0.0, t_lj = 0.0, t_atm = 0.0, n_atm = 0.0;
  double *fnew = (double *)malloc((size_t)(3 * n > 0 ? 3 * n : 1) * sizeof(double));
  if (!fnew) return -2;
  Grid g;
  int st = 0;
  if (!have_forces) {  /* F2b(x^0), F3b(x^0): not part of the timed steps */
    double o[4];
    st = cells_forces(n, x, L, eps, sigma, rc2, nu, rc3, f2, f3, o);
    if (st) goto done;
    u2 = o[0];
    u3 = o[2];
  }
  for (int64_t it = 0; it < (int64_t)n_outer * k; ++it) {
    if (it % k == 0) {
#pragma omp parallel for schedule(static)
      for (int64_t q = 0; q < 3 * n; ++q) v[q] += h3 * f3[q];
    }
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < 3 * n; ++q) x[q] = fold(x[q] + dt * v[q] + hx * f2[q], L);
    double t0 = now_s();
    if ((st = grid_build(n, x, L, reach, &g)) != 0) goto done;
    lj_pass(n, L, &g, eps, sigma, rc2, fnew, &u2, &w2);
    t_lj += now_s() - t0;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < 3 * n; ++q) {
      v[q] += h2 * (f2[q] + fnew[q]);
      f2[q] = fnew[q];
    }
    if ((it + 1) % k == 0) {
      int64_t nt = 0;
      t0 = now_s();
      st = atm_pass(n, L, &g, nu, rc3, f3, &u3, &nt);
      t_atm += now_s() - t0;
      if (st) {
        grid_free(&g);
        goto done;
      }
      trip += (double)nt;
      n_atm += 1.0;
#pragma omp parallel for schedule(static)
      for (int64_t q = 0; q < 3 * n; ++q) v[q] += h3 * f3[q];
    }
    grid_free(&g);
  }
done:
  free(fnew);
  out[0] = u2;
  out[1] = u3;
  out[2] = trip;
  out[3] = t_lj;
  out[4] = t_atm;
  out[5] = n_atm;
  return st;
}

int cells_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
