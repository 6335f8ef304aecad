/* CPU FP64 ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct brute-force evaluation of the two force
 * fields of arXiv 2507.11172 (Martin et al., "The Multiple Time-Stepping
 * Method for 3-Body Interactions in High Performance Molecular Dynamics
 * Simulations").  Only the tests, the smoke check and the benchmark's CPU
 * baseline may call it; the GPU library never does.  It shares no code,
 * header or table with the CUDA path.
 *
 * Definitions (paper, Sec. 2.1 and Sec. 4.1-4.2):
 *   phi2(i,j)   = 4 eps [ (sigma/r_ij)^12 - (sigma/r_ij)^6 ]            (LJ 12-6)
 *   phi3(i,j,k) = nu (1 + 3 cos(th_i) cos(th_j) cos(th_k)) / (r_ij r_ik r_jk)^3
 *                 with th_i the angle between vectors ij and ik          (ATM)
 *   F_i = -grad_i Phi, Phi = sum phi2 + sum phi3                        (Eq. 2, 3)
 *   A pair interacts iff r <= r_c; a triplet iff all three pair distances
 *   are <= r_c (Fig. 2 caption; Sec. 4.2.2).  Each unordered pair / triple
 *   is counted once (Newton's third law, Sec. 2.2).  Plain truncation, no
 *   shift.  Periodic cubic box, minimum image d - L rint(d/L) per axis.
 *
 * Numerics: everything in IEEE double; built with -ffp-contract=off so no
 * fused multiply-add changes a rounding.  Squared distances are formed as
 * dx*dx + dy*dy + dz*dz left to right and compared with rc*rc.
 *
 * Virial W = sum over interactions of sum over members r_a . F_a with the
 * members placed at their minimum-image positions around the first member.
 *
 * Every function returns 0 on success, -1 on bad arguments.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

static double min_image(double d, double L) { return d - L * rint(d / L); }

/* minimum-image vector b - a and its squared length */
static double mi_vec(const double *a, const double *b, double L, double out[3]) {
  out[0] = min_image(b[0] - a[0], L);
  out[1] = min_image(b[1] - a[1], L);
  out[2] = min_image(b[2] - a[2], L);
  return out[0] * out[0] + out[1] * out[1] + out[2] * out[2];
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ---------------- Lennard-Jones 12-6 (Sec. 2.1) ---------------- */

/* energy of one pair at squared distance r2 and the factor g with
 * F_i = -g * d, F_j = +g * d for d = x_j - x_i, i.e. g = -(dphi/dr)/r. */
static void lj_pair(double r2, double eps, double sigma, double *phi, double *g) {
  double sr2 = (sigma * sigma) / r2;
  double sr6 = sr2 * sr2 * sr2;
  double sr12 = sr6 * sr6;
  *phi = 4.0 * eps * (sr12 - sr6);
  *g = 24.0 * eps * (2.0 * sr12 - sr6) / r2;
}

/* All unordered pairs i<j: forces f (n*3), energy u, virial w. */
int oracle_lj_brute(int64_t n, const double *x, double L, double eps, double sigma, double rc, double *f,
                    double *u, double *w) {
  if (n < 0 || !(L > 0) || !(rc > 0)) return -1;
  double rc2 = rc * rc;
  memset(f, 0, (size_t)n * 3 * sizeof(double));
  double U = 0.0, W = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = i + 1; j < n; ++j) {
      double d[3];
      double r2 = mi_vec(x + 3 * i, x + 3 * j, L, d);
      if (!(r2 <= rc2)) continue;
      double phi, g;
      lj_pair(r2, eps, sigma, &phi, &g);
      U += phi;
      for (int a = 0; a < 3; ++a) {
        f[3 * i + a] -= g * d[a];
        f[3 * j + a] += g * d[a];
      }
      W += g * r2; /* d . F_j */
    }
  }
  *u = U;
  *w = W;
  return 0;
}

/* Per-particle pass: for each selected particle s = sel[t], the complete
 * force f[t] = -grad_s sum_j phi2(s,j) and its pair energy u[t] (each pair's
 * energy counted in full for both members, so sum_t u[t] / 2 = U when all
 * particles are selected). */
int oracle_lj_particles(int64_t n, const double *x, double L, double eps, double sigma, double rc,
                        int64_t nsel, const int64_t *sel, double *f, double *u) {
  if (n < 0 || nsel < 0 || !(L > 0) || !(rc > 0)) return -1;
  double rc2 = rc * rc;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < nsel; ++t) {
    int64_t i = sel[t];
    double fi[3] = {0.0, 0.0, 0.0}, ui = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double d[3];
      double r2 = mi_vec(x + 3 * i, x + 3 * j, L, d);
      if (!(r2 <= rc2)) continue;
      double phi, g;
      lj_pair(r2, eps, sigma, &phi, &g);
      ui += phi;
      for (int a = 0; a < 3; ++a) fi[a] -= g * d[a];
    }
    for (int a = 0; a < 3; ++a) f[3 * t + a] = fi[a];
    u[t] = ui;
  }
  return 0;
}

/* ---------------- Axilrod-Teller-Muto (Sec. 2.1) ---------------- */

/* phi3 for the triangle p, q, r given as explicit (unwrapped) coordinates,
 * written literally with the three cosines. */
static double atm_phi(const double p[3], const double q[3], const double r[3], double nu) {
  double u[3], w[3], z[3];
  for (int a = 0; a < 3; ++a) {
    u[a] = q[a] - p[a]; /* p -> q */
    w[a] = r[a] - p[a]; /* p -> r */
    z[a] = r[a] - q[a]; /* q -> r */
  }
  double rpq = sqrt(dot3(u, u)), rpr = sqrt(dot3(w, w)), rqr = sqrt(dot3(z, z));
  double cp = dot3(u, w) / (rpq * rpr);        /* angle at p between pq and pr */
  double cq = -dot3(u, z) / (rpq * rqr);       /* angle at q between qp and qr */
  double cr = dot3(w, z) / (rpr * rqr);        /* angle at r between rp and rq */
  double prod = rpq * rpr * rqr;
  return nu * (1.0 + 3.0 * cp * cq * cr) / (prod * prod * prod);
}

/* Gradient of phi3(p, q, r) with respect to the first point p.  phi3 is
 * symmetric in its three points, so the gradient with respect to q is
 * atm_grad_first(q, p, r) and with respect to r is atm_grad_first(r, p, q).
 *
 * With u = q - p, w = r - p, z = r - q (dz/dp = 0):
 *   d|u|/dp = -u/|u|,  d|w|/dp = -w/|w|
 *   d cp/dp = -(u + w)/(|u||w|) + cp (u/|u|^2 + w/|w|^2)
 *   d cq/dp =  z/(|u||z|) + cq u/|u|^2
 *   d cr/dp = -z/(|w||z|) + cr w/|w|^2
 *   d(1/D)/dp = (3/D)(u/|u|^2 + w/|w|^2),  D = (|u||w||z|)^3
 *   dphi/dp = nu [ 3 (cq cr dcp + cp cr dcq + cp cq dcr) / D + (1 + 3 cp cq cr) d(1/D) ]
 */
static void atm_grad_first(const double p[3], const double q[3], const double r[3], double nu, double g[3]) {
  double u[3], w[3], z[3];
  for (int a = 0; a < 3; ++a) {
    u[a] = q[a] - p[a];
    w[a] = r[a] - p[a];
    z[a] = r[a] - q[a];
  }
  double u2 = dot3(u, u), w2 = dot3(w, w), z2 = dot3(z, z);
  double ru = sqrt(u2), rw = sqrt(w2), rz = sqrt(z2);
  double cp = dot3(u, w) / (ru * rw);
  double cq = -dot3(u, z) / (ru * rz);
  double cr = dot3(w, z) / (rw * rz);
  double prod = ru * rw * rz;
  double invD = 1.0 / (prod * prod * prod);
  double num = 1.0 + 3.0 * cp * cq * cr;
  for (int a = 0; a < 3; ++a) {
    double dcp = -(u[a] + w[a]) / (ru * rw) + cp * (u[a] / u2 + w[a] / w2);
    double dcq = z[a] / (ru * rz) + cq * u[a] / u2;
    double dcr = -z[a] / (rw * rz) + cr * w[a] / w2;
    double dinvD = 3.0 * invD * (u[a] / u2 + w[a] / w2);
    g[a] = nu * (3.0 * (cq * cr * dcp + cp * cr * dcq + cp * cq * dcr) * invD + num * dinvD);
  }
}

/* Tests whether the unordered triple (i, j, k) interacts: all three
 * minimum-image squared distances <= rc^2.  On success fills the local
 * coordinates p = 0, q = d_ij, r = d_ik. */
static int atm_triple(const double *x, int64_t i, int64_t j, int64_t k, double L, double rc2, double p[3],
                      double q[3], double r[3]) {
  double djk[3];
  if (!(mi_vec(x + 3 * i, x + 3 * j, L, q) <= rc2)) return 0;
  if (!(mi_vec(x + 3 * i, x + 3 * k, L, r) <= rc2)) return 0;
  if (!(mi_vec(x + 3 * j, x + 3 * k, L, djk) <= rc2)) return 0;
  p[0] = p[1] = p[2] = 0.0;
  return 1;
}

/* All unordered triples i<j<k: forces f (n*3), energy u, virial w, and the
 * number of interacting triples. */
int oracle_atm_brute(int64_t n, const double *x, double L, double nu, double rc, double *f, double *u, double *w,
                     int64_t *count) {
  if (n < 0 || !(L > 0) || !(rc > 0)) return -1;
  double rc2 = rc * rc;
  memset(f, 0, (size_t)n * 3 * sizeof(double));
  double U = 0.0, W = 0.0;
  int64_t cnt = 0;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = i + 1; j < n; ++j) {
      double dij[3];
      if (!(mi_vec(x + 3 * i, x + 3 * j, L, dij) <= rc2)) continue; /* cannot interact with any k */
      for (int64_t k = j + 1; k < n; ++k) {
        double p[3], q[3], r[3];
        if (!atm_triple(x, i, j, k, L, rc2, p, q, r)) continue;
        double gi[3], gj[3], gk[3];
        atm_grad_first(p, q, r, nu, gi);
        atm_grad_first(q, p, r, nu, gj);
        atm_grad_first(r, p, q, nu, gk);
        for (int a = 0; a < 3; ++a) {
          f[3 * i + a] -= gi[a];
          f[3 * j + a] -= gj[a];
          f[3 * k + a] -= gk[a];
        }
        U += atm_phi(p, q, r, nu);
        W -= dot3(q, gj) + dot3(r, gk); /* p = 0 contributes nothing */
        ++cnt;
      }
    }
  }
  *u = U;
  *w = W;
  if (count) *count = cnt;
  return 0;
}

/* Per-particle pass: for each selected particle s = sel[t], scan all n
 * particles for its neighbours (r <= rc), then every unordered pair (j, k) of
 * neighbours with r_jk <= rc forms an interacting triple containing s.
 * f[t] = -grad_s of the sum of those phi3, u[t] = their energy sum (each
 * triple counted once per member, so sum_t u[t] / 3 = U when all particles
 * are selected), cnt[t] = number of such triples. */
int oracle_atm_particles(int64_t n, const double *x, double L, double nu, double rc, int64_t nsel,
                         const int64_t *sel, double *f, double *u, int64_t *cnt) {
  if (n < 0 || nsel < 0 || !(L > 0) || !(rc > 0)) return -1;
  double rc2 = rc * rc;
  int ok = 1;
#pragma omp parallel
  {
    /* neighbour scratch: indices and minimum-image vectors of one particle */
    enum { MAXNB = 4096 };
    static __thread int64_t nb[MAXNB];
    static __thread double dv[MAXNB][3];
#pragma omp for schedule(dynamic, 4)
    for (int64_t t = 0; t < nsel; ++t) {
      int64_t s = sel[t];
      int64_t m = 0;
      for (int64_t j = 0; j < n; ++j) {
        if (j == s) continue;
        double d[3];
        if (!(mi_vec(x + 3 * s, x + 3 * j, L, d) <= rc2)) continue;
        if (m >= MAXNB) { ok = 0; break; }
        nb[m] = j;
        dv[m][0] = d[0]; dv[m][1] = d[1]; dv[m][2] = d[2];
        ++m;
      }
      double fs[3] = {0.0, 0.0, 0.0}, us = 0.0;
      int64_t c = 0;
      const double p[3] = {0.0, 0.0, 0.0};
      for (int64_t a = 0; a < m; ++a) {
        for (int64_t b = a + 1; b < m; ++b) {
          double djk[3];
          if (!(mi_vec(x + 3 * nb[a], x + 3 * nb[b], L, djk) <= rc2)) continue;
          double g[3];
          atm_grad_first(p, dv[a], dv[b], nu, g);
          for (int e = 0; e < 3; ++e) fs[e] -= g[e];
          us += atm_phi(p, dv[a], dv[b], nu);
          ++c;
        }
      }
      for (int e = 0; e < 3; ++e) f[3 * t + e] = fs[e];
      u[t] = us;
      if (cnt) cnt[t] = c;
    }
  }
  return ok ? 0 : -1;
}

/* phi3 and the three gradients of one explicit triangle (no cutoff, no box):
 * for closed-form checks.  g is 3x3: rows = gradient w.r.t. p, q, r. */
int oracle_atm_triangle(const double *p, const double *q, const double *r, double nu, double *phi, double *g) {
  *phi = atm_phi(p, q, r, nu);
  atm_grad_first(p, q, r, nu, g);
  atm_grad_first(q, p, r, nu, g + 3);
  atm_grad_first(r, p, q, nu, g + 6);
  return 0;
}

/* Kinetic energy 0.5 m sum v^2. */
double oracle_kinetic(int64_t n, const double *v, double m) {
  double s = 0.0;
  for (int64_t i = 0; i < 3 * n; ++i) s += v[i] * v[i];
  return 0.5 * m * s;
}
