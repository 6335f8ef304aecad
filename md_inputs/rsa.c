/* Random sequential addition (RSA) of points in a periodic cube.
 *
 * Input generator only (no part of the simulated method).  Trial t draws
 * a point from splitmix64 counters 3t, 3t+1, 3t+2 of (seed, stream 4), scaled
 * to [0, L); it is accepted iff every previously accepted point lies at
 * minimum-image distance >= d_min.  A uniform grid of cells of edge >= d_min
 * limits each test to the 27 surrounding cells.  Same stream definition as
 * md_inputs.splitmix64 / uniform.
 *
 * Speed (the result does not depend on it): a cell of edge a >= d_min holds at
 * most 8 accepted points (its 8 sub-cubes of edge a/2 have diagonals
 * sqrt(3) a/2 < d_min, so each holds at most one), so 8 int32 slots per cell;
 * the trial's own cell is tested first (most rejections come from it); the
 * minimum image of a difference |d| < L is d - L, d + L or d, exactly what
 * d - L rint(d / L) gives for such d.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define RSA_STREAM 4u
#define CELL_CAP 8

static uint64_t mix(uint64_t key, uint64_t c) {
  uint64_t z = key + (c + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static double unif(uint64_t key, uint64_t c) { return (double)(mix(key, c) >> 11) * (1.0 / 9007199254740992.0); }

/* minimum image of d, |d| < L (rint(d / L) is -1, 0 or 1 there; ties at |d| = L / 2 round to 0) */
static double mi(double d, double L, double half) {
  if (d > half) return d - L;
  if (d < -half) return d + L;
  return d;
}

/* 1 iff no accepted point of `cell` lies closer than d_min to p */
static int cell_clear(const uint8_t *cnt, const int32_t *slot, const double *out, int64_t cell, const double p[3],
                      double L, double half, double d2) {
  for (int s = 0; s < cnt[cell]; ++s) {
    const double *q = out + 3 * (int64_t)slot[cell * CELL_CAP + s];
    double r2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      double d = mi(q[a] - p[a], L, half);
      r2 += d * d;
    }
    if (r2 < d2) return 0;
  }
  return 1;
}

int64_t rsa_place(int64_t n, double L, double d_min, uint64_t seed, int64_t max_trials, double *out) {
  uint64_t key = seed * 0x100000001B3ull + (uint64_t)RSA_STREAM * 0x9E3779B1ull;
  int64_t ng = (int64_t)floor(L / d_min);
  if (ng < 1) ng = 1;
  if (ng > 1024) ng = 1024;
  if (n > INT32_MAX) return -1;
  double edge = L / (double)ng;
  int64_t ncell = ng * ng * ng;
  uint8_t *cnt = (uint8_t *)calloc((size_t)ncell, sizeof(uint8_t));
  int32_t *slot = (int32_t *)malloc((size_t)ncell * CELL_CAP * sizeof(int32_t));
  if (!cnt || !slot) { free(cnt); free(slot); return -1; }
  double d2 = d_min * d_min, half = 0.5 * L;
  int64_t placed = 0;
  for (int64_t t = 0; t < max_trials && placed < n; ++t) {
    double p[3];
    for (int a = 0; a < 3; ++a) {
      p[a] = unif(key, (uint64_t)(3 * t + a)) * L;
      if (p[a] >= L) p[a] = 0.0;
    }
    int64_t c[3];
    for (int a = 0; a < 3; ++a) {
      c[a] = (int64_t)(p[a] / edge);
      if (c[a] >= ng) c[a] = ng - 1;
    }
    const int64_t own = (c[2] * ng + c[1]) * ng + c[0];
    int ok = cell_clear(cnt, slot, out, own, p, L, half, d2);
    for (int dz = -1; dz <= 1 && ok; ++dz)
      for (int dy = -1; dy <= 1 && ok; ++dy)
        for (int dx = -1; dx <= 1 && ok; ++dx) {
          if (!dx && !dy && !dz) continue;
          int64_t cx = (c[0] + dx + ng) % ng, cy = (c[1] + dy + ng) % ng, cz = (c[2] + dz + ng) % ng;
          int64_t cell = (cz * ng + cy) * ng + cx;
          if (cell != own) ok = cell_clear(cnt, slot, out, cell, p, L, half, d2);
        }
    if (!ok) continue;
    if (cnt[own] >= CELL_CAP) continue; /* cannot happen for edge >= d_min (see above) */
    slot[own * CELL_CAP + cnt[own]++] = (int32_t)placed;
    for (int a = 0; a < 3; ++a) out[3 * placed + a] = p[a];
    ++placed;
  }
  free(cnt);
  free(slot);
  return placed;
}
