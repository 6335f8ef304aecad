/* Random sequential addition (RSA) of points in a periodic cube.
 *
 * Input generator only (no part of the simulated method).  Trial t draws
 * a point from splitmix64 counters 3t, 3t+1, 3t+2 of (seed, stream 4), scaled
 * to [0, L); it is accepted iff every previously accepted point lies at
 * minimum-image distance >= d_min.  A uniform grid of cells of edge >= d_min
 * limits each test to the 27 surrounding cells.  Same stream definition as
 * md_inputs.splitmix64 / uniform.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define RSA_STREAM 4u
#define CELL_CAP 16

static uint64_t mix(uint64_t key, uint64_t c) {
  uint64_t z = key + (c + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static double unif(uint64_t key, uint64_t c) { return (double)(mix(key, c) >> 11) * (1.0 / 9007199254740992.0); }

int64_t rsa_place(int64_t n, double L, double d_min, uint64_t seed, int64_t max_trials, double *out) {
  uint64_t key = seed * 0x100000001B3ull + (uint64_t)RSA_STREAM * 0x9E3779B1ull;
  int64_t ng = (int64_t)floor(L / d_min);
  if (ng < 1) ng = 1;
  if (ng > 1024) ng = 1024;
  double edge = L / (double)ng;
  int64_t ncell = ng * ng * ng;
  int32_t *cnt = (int32_t *)calloc((size_t)ncell, sizeof(int32_t));
  int64_t *slot = (int64_t *)malloc((size_t)ncell * CELL_CAP * sizeof(int64_t));
  if (!cnt || !slot) { free(cnt); free(slot); return -1; }
  double d2 = d_min * d_min;
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
    int ok = 1;
    for (int dz = -1; dz <= 1 && ok; ++dz)
      for (int dy = -1; dy <= 1 && ok; ++dy)
        for (int dx = -1; dx <= 1 && ok; ++dx) {
          int64_t cx = (c[0] + dx + ng) % ng, cy = (c[1] + dy + ng) % ng, cz = (c[2] + dz + ng) % ng;
          int64_t cell = (cz * ng + cy) * ng + cx;
          for (int s = 0; s < cnt[cell]; ++s) {
            const double *q = out + 3 * slot[cell * CELL_CAP + s];
            double r2 = 0.0;
            for (int a = 0; a < 3; ++a) {
              double d = q[a] - p[a];
              d -= L * rint(d / L);
              r2 += d * d;
            }
            if (r2 < d2) { ok = 0; break; }
          }
        }
    if (!ok) continue;
    int64_t cell = (c[2] * ng + c[1]) * ng + c[0];
    if (cnt[cell] >= CELL_CAP) continue; /* cannot happen for edge >= d_min */
    slot[cell * CELL_CAP + cnt[cell]++] = placed;
    for (int a = 0; a < 3; ++a) out[3 * placed + a] = p[a];
    ++placed;
  }
  free(cnt);
  free(slot);
  return placed;
}
