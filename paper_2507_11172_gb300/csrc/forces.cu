// Force and update kernels of the r-RESPA hot path (arXiv 2507.11172):
//   k_lj      Lennard-Jones 12-6 pair forces (Sec. 2.1) from the Verlet pair
//             list (each thread one particle's force, no scatter).
//   k_kick    the inner velocity-Verlet kick/drift of Algorithm 2 after each
//             LJ evaluation (FP64, one thread per particle).
//   k_atm     Axilrod-Teller-Muto triplet forces (Sec. 2.1) with the triplet
//             cutoff "all three distances <= r_c" (Fig. 2 caption, Sec.
//             4.2.2), one CTA per cell, each triplet evaluated once with
//             Newton-3 scatter (cell kernel; the default is k_atm_rot).
//   k_atm_pa  the same forces, each triplet evaluated from each member.
//   k_combine per-particle sum of the triplet kernel's forces and the outer
//             (three-body) kicks of Algorithm 2 (with distance classes: far
//             and near kicks).
//   k_start   opening half kicks and first drift of a call.
#include <stdio.h>

#include "md_internal.cuh"
#include "lj_common.cuh"
#include "sys_stage.cuh"

namespace r3b {

template <typename T> __device__ __forceinline__ T rsqrt_acc(T q);
// FP32: hardware reciprocal square root refined by one Newton step
template <> __device__ __forceinline__ float rsqrt_acc<float>(float q) {
  float t = rsqrtf(q);
  return t * fmaf(-0.5f * q, t * t, 1.5f);
}
template <> __device__ __forceinline__ double rsqrt_acc<double>(double q) { return 1.0 / sqrt(q); }

template <typename T> __device__ __forceinline__ T recip(T x);
template <> __device__ __forceinline__ float recip<float>(float x) { return __frcp_rn(x); }
template <> __device__ __forceinline__ double recip<double>(double x) { return 1.0 / x; }

// Per-particle force accumulator: compensated (hi, lo) pair in FP32 mode,
// plain double in FP64 mode.
template <typename T> struct Acc3;
template <> struct Acc3<float> {
  CompF c[3];
  __device__ Acc3() {
    for (int a = 0; a < 3; ++a) c[a].hi = c[a].lo = 0.f;
  }
  __device__ __forceinline__ void add(float x, float y, float z) {
    c[0].add(x);
    c[1].add(y);
    c[2].add(z);
  }
  __device__ __forceinline__ double get(int a) const { return c[a].value(); }
};
template <> struct Acc3<double> {
  double c[3];
  __device__ Acc3() { c[0] = c[1] = c[2] = 0.0; }
  __device__ __forceinline__ void add(double x, double y, double z) {
    c[0] += x;
    c[1] += y;
    c[2] += z;
  }
  __device__ __forceinline__ double get(int a) const { return c[a]; }
};

template <typename T> struct AccS;
template <> struct AccS<float> {
  CompF c;
  __device__ AccS() { c.hi = c.lo = 0.f; }
  __device__ __forceinline__ void add(float x) { c.add(x); }
  __device__ __forceinline__ double get() const { return c.value(); }
};
template <> struct AccS<double> {
  double c;
  __device__ AccS() : c(0.0) {}
  __device__ __forceinline__ void add(double x) { c += x; }
  __device__ __forceinline__ double get() const { return c; }
};

// finiteness from the exponent bits (integer ALU, not the scarce FP64 pipe)
__device__ __forceinline__ bool finite_bits(double x) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

// Cell-local coordinates are FP64 positions relative to the centre of the particle's cell at the last
// binning.  Positions are folded into [0, L) only at a binning, together with the cell assignment, so
// between two binnings x - centre stays within about half a cell edge plus the displacement: no
// periodic fold is needed, one FP64 subtraction per axis (the centres come from a table; on GB300
// every FP64 instruction is costly).
//
// Centre of cell `cell` (one table row per axis).  The kick/drift and start kernels load it, like every
// other input, before their first store: loads cannot move across stores through pointers that may
// alias, so loading everything first keeps the chain of dependent global round trips short (kick/drift
// 9.5 -> 8.3 us and start 14.5 -> 13.2 us per launch on 100k particles)
__device__ __forceinline__ void cell_centre(const SysDev& S, int cell, double cen[3]) {
  const int nc = S.nc;
  const int cz = cell / (nc * nc);
  const int r = cell - cz * nc * nc;
  const int cy = r / nc;
  const int cx = r - cy * nc;
  cen[0] = S.ccen[cx];
  cen[1] = S.ccen[cy];
  cen[2] = S.ccen[cz];
}

// cell-local coordinates (x - centre) of a new position into buffer buf, and the displacement check
// against r, the particle's coordinates at the last binning (loaded by the caller)
template <typename T>
__device__ __forceinline__ void store_pos_checked(const SysDev& S, int buf, int i, const double x[3],
                                                  const double cen[3], const typename V4<T>::type r) {
  using T4 = typename V4<T>::type;
  T4 h;
  h.x = (T)(x[0] - cen[0]);
  h.y = (T)(x[1] - cen[1]);
  h.z = (T)(x[2] - cen[2]);
  h.w = (T)0;
  reinterpret_cast<T4*>(S.pos[buf])[i] = h;
  const T dx = h.x - r.x, dy = h.y - r.y, dz = h.z - r.z;
  if (dx * dx + dy * dy + dz * dz > Par<T>::half_skin_sq(S)) atomicOr(&S.flags[FLG_SKIN], 1);
}

// cell-local coordinate of an FP64 position relative to the centre of cell `cell` (combine kernel:
// there, loading its inputs before the first store measured slower, so it keeps this form)
__device__ __forceinline__ void cell_rel(const SysDev& S, int cell, const double x[3], double rel[3]) {
  const int nc = S.nc;
  const int cz = cell / (nc * nc);
  const int r = cell - cz * nc * nc;
  const int cy = r / nc;
  const int cx = r - cy * nc;
  rel[0] = x[0] - S.ccen[cx];
  rel[1] = x[1] - S.ccen[cy];
  rel[2] = x[2] - S.ccen[cz];
}

// cell-local coordinates rel into buffer buf, optionally with the displacement check (loads the
// coordinates at the last binning itself, after the store)
template <typename T>
__device__ __forceinline__ void store_pos(const SysDev& S, int buf, int i, const double rel[3], bool check_skin) {
  using T4 = typename V4<T>::type;
  T4 h;
  h.x = (T)rel[0];
  h.y = (T)rel[1];
  h.z = (T)rel[2];
  h.w = (T)0;
  reinterpret_cast<T4*>(S.pos[buf])[i] = h;
  if (check_skin) {  // displacement since the last sort, in the force precision
    const T4 r = reinterpret_cast<const T4*>(S.ref)[i];
    const T dx = h.x - r.x, dy = h.y - r.y, dz = h.z - r.z;
    if (dx * dx + dy * dy + dz * dz > Par<T>::half_skin_sq(S)) atomicOr(&S.flags[FLG_SKIN], 1);
  }
}

// near-class force of particle p from the near-class kernel's sums (read and cleared)
template <typename T>
__device__ __forceinline__ void take_near(const SysDev& S, int p, double f[3]) {
  if (sizeof(T) == 4) {
    fix_take3(S.f3nacc, p, S.fix_unit, f);
  } else {
    double* a = reinterpret_cast<double*>(S.f3nacc) + 4 * (size_t)p;
    f[0] = a[0];
    f[1] = a[1];
    f[2] = a[2];
    a[0] = a[1] = a[2] = 0.0;
  }
}

// ============================================================== LJ pair kernel
// A team of kLjTeam adjacent threads per particle i (F_i only: every pair is evaluated from both
// sides, no scatter).  Thread h of the team walks the groups h, h + kLjTeam, ... of four consecutive
// entries of i's pair-list row with a software pipeline: the row entries of its group after next and
// the neighbour positions of its next group are loaded while its current group is evaluated; a team's
// partial forces are added in FP64 at the end.  On GB300 one thread per particle is fastest (teams of
// 2 and 4 measured 3 % and 1 % slower per outer step on the 100k workload).
// The offset of a neighbour's cell (entry code, one of 27) is computed from the code's bits in FP32
// (off_unit: no shared-memory lookup, which would share the L1 pipe with the gathers; 0.81-0.84 ->
// 0.79 ms per outer step on the 100k workload) and comes from a shared-memory table in FP64; list
// padding uses code 63, whose offset (two cell edges per axis, or a far table entry) is beyond every
// cutoff.  The plain sum of every eight pair
// forces is added to a compensated (hi, lo) accumulator with an error-free TwoSum.  The
// velocity-Verlet kick/drift of Algorithm 2 follows in k_kick.

// read-only cached load of a 4-vector (the position buffer read by a kernel is never written by it)
#ifdef R3B_LJ_POS_EVICT_LAST
__device__ __forceinline__ float4 ldg4(const float4* p) {
  float4 v;
  asm("ld.global.nc.L1::evict_last.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p));
  return v;
}
#else
__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }
#endif
// four pair-list entries: each row is streamed once per launch, so its lines are marked for early
// eviction from L1 (the neighbour positions, reused by many threads of the SM, stay)
__device__ __forceinline__ int4 ld_entries(const int4* p) {
#ifdef R3B_LJ_LIST_PLAIN
  return __ldg(p);
#else
  int4 v;
  asm("ld.global.nc.L1::evict_first.v4.s32 {%0, %1, %2, %3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p));
  return v;
#endif
}
__device__ __forceinline__ double4_32a ldg4(const double4_32a* p) { return *p; }

template <typename T> __device__ __forceinline__ T recip_fast(T x);
// FP32: hardware reciprocal refined by one Newton step (no special-value path: r^2 is a
// normal positive number here)
template <> __device__ __forceinline__ float recip_fast<float>(float x) {
  const float y = __fdividef(1.0f, x);
  return y * fmaf(-x, y, 2.0f);
}
template <> __device__ __forceinline__ double recip_fast<double>(double x) { return 1.0 / x; }

// kE = false: a launch whose items never ask for energies (compiled without the energy terms);
// kPer: threads per block (one per particle), a runtime choice of the autotuner
#ifndef R3B_LJ_THREADS_PER_SM
#define R3B_LJ_THREADS_PER_SM 896  // resident LJ threads per SM the register allocation is sized for
#endif
template <typename T, bool kE, int kPer>
__global__ void __launch_bounds__(kPer, R3B_LJ_THREADS_PER_SM / kPer) k_lj(const SysDev* __restrict__ sys, const PItem* __restrict__ items) {
  static_assert(kPer % 32 == 0 && kLjTeam == 1, "LJ blocks of whole warps, one thread per particle");
  using T4 = typename V4<T>::type;
  __shared__ T4 s_off[64];
  __shared__ double red_u[kPer / 32], red_w[kPer / 32];
  const PItem it = items[blockIdx.x];
#if R3B_STAGE_SYS
  __shared__ StagedSys s_sys;
  stage_sys(s_sys, sys, it.sys);
  pdl_wait();
  __syncthreads();
  const SysDev& S = s_sys.get();
#else
  pdl_wait();
  const SysDev& S = sys[it.sys];
#endif
  const int mode = item_mode(S, it.mode);
  if (mode & M_SKIP) return;  // block-uniform: a block belongs to one system
  const bool energy = kE && (mode & M_ENERGY) != 0;
  for (unsigned c = threadIdx.x; c < 64u; c += blockDim.x) {
    const T e = Par<T>::edge(S);
    T4 o;
    o.x = fma((T)(c & 3u), e, -e);
    o.y = fma((T)((c >> 2) & 3u), e, -e);
    o.z = fma((T)((c >> 4) & 3u), e, -e);
    o.w = (T)0;
    if (c == kPadCode) o.x = o.y = o.z = (T)1e3;
    s_off[c] = o;
  }
  __syncthreads();
  const int n = S.n;
  const int h = threadIdx.x % kLjTeam;  // this thread's share of the row
  const int i = it.begin + threadIdx.x / kLjTeam;
  const bool active = i < n;
  const T4* __restrict__ P = reinterpret_cast<const T4*>(S.pos[it.buf]);
  const double* __restrict__ X = S.X[it.buf];
  Acc3<T> f;
  T uu = 0, ww = 0;  // energy and virial of the current eight pair terms
  AccS<T> ud, wd;    // the thread's energy and virial sums (FP32: compensated; FP64 across threads)
  if (active) {
    const T4 pi = P[i];
    const T rcsq = Par<T>::rc2sq(S), g2 = Par<T>::guard2(S);
    const T lo = rcsq - g2;
    const T sig2 = Par<T>::sig2(S);
    const T eps24 = Par<T>::eps24(S), eps4 = Par<T>::eps4(S);
    const T edge = Par<T>::edge(S);
    const int cnt = S.nbr_cnt[i];
    const int4* __restrict__ row4 = reinterpret_cast<const int4*>(S.nbr + nbr_slot(S.maxnb, i, 0));
    const int4 pad = make_int4((int)(kPadCode << kNbrShift), (int)(kPadCode << kNbrShift),
                               (int)(kPadCode << kNbrShift), (int)(kPadCode << kNbrShift));
    // entries of a group, padded beyond the row's length
    auto entries = [&](int t0) {
      int4 e = t0 < cnt ? ld_entries(row4 + (t0 >> 2)) : pad;
      if (t0 + 1 >= cnt) e.y = pad.y;
      if (t0 + 2 >= cnt) e.z = pad.z;
      if (t0 + 3 >= cnt) e.w = pad.w;
      return e;
    };
    auto gather = [&](const int4 e, T4* pj) {
      pj[0] = ldg4(P + ((unsigned)e.x & kNbrMask));
      pj[1] = ldg4(P + ((unsigned)e.y & kNbrMask));
      pj[2] = ldg4(P + ((unsigned)e.z & kNbrMask));
      pj[3] = ldg4(P + ((unsigned)e.w & kNbrMask));
    };
    constexpr int kStride = 4 * kLjTeam;
    int4 ea = entries(4 * h), eb = entries(4 * h + kStride);
    T4 pa[4], pb[4];
    gather(ea, pa);
    T bmin = (T)1e30;        // smallest |r^2 - r_c^2| met: the guard band is checked once at the end
    T px = 0, py = 0, pz = 0;  // plain sum of the previous group
    bool odd = false;          // a group's plain sum is waiting in (px, py, pz)
    for (int t0 = 4 * h; t0 < cnt; t0 += kStride) {
      gather(eb, pb);  // positions of the next group
      const int4 ec = entries(t0 + 2 * kStride);
      const unsigned e[4] = {(unsigned)ea.x, (unsigned)ea.y, (unsigned)ea.z, (unsigned)ea.w};
      T sx = 0, sy = 0, sz = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        T dx, dy, dz;
        if (R3B_LJ_ARITH_OFF && sizeof(T) == 4) {  // padding (code 63): two edges per axis, beyond r_c
          const unsigned cd = e[u] >> kNbrShift;
          dx = fma((T)off_unit(cd & 3u), edge, pa[u].x - pi.x);
          dy = fma((T)off_unit((cd >> 2) & 3u), edge, pa[u].y - pi.y);
          dz = fma((T)off_unit(cd >> 4), edge, pa[u].z - pi.z);
        } else {
          const T4 o = s_off[e[u] >> kNbrShift];
          dx = (pa[u].x - pi.x) + o.x;
          dy = (pa[u].y - pi.y) + o.y;
          dz = (pa[u].z - pi.z) + o.z;
        }
        const T r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        bmin = fmin(bmin, fabs(r2 - rcsq));
        const T ir2 = recip_fast<T>(r2);
        const T sr2 = sig2 * ir2;
        const T sr6 = sr2 * sr2 * sr2;
        const T sr12 = sr6 * sr6;
        const T g = r2 <= lo ? eps24 * (sr12 + sr12 - sr6) * ir2 : (T)0;  // F_i = -g d
        sx = fma(-g, dx, sx);
        sy = fma(-g, dy, sy);
        sz = fma(-g, dz, sz);
        if (energy) {
          uu += r2 <= lo ? eps4 * (sr12 - sr6) : (T)0;
          ww = fma(g, r2, ww);
        }
      }
      // every eight terms (two groups) are summed plainly, then added exactly
      if (odd || t0 + kStride >= cnt) {
        f.add(sx + px, sy + py, sz + pz);
        px = py = pz = (T)0;
        odd = false;
        if (energy) {
          ud.add(uu);
          wd.add(ww);
          uu = ww = (T)0;
        }
      } else {
        px = sx;
        py = sy;
        pz = sz;
        odd = true;
      }
      ea = eb;
      eb = ec;
#pragma unroll
      for (int u = 0; u < 4; ++u) pa[u] = pb[u];
    }
    if (bmin < g2) {
      // Rare: pairs whose r^2 fell in the guard band around r_c2^2 (left out above) are decided in
      // FP64 with the CPU definition's operation order; the ones inside the cutoff are added.
      for (int t = 0; t < cnt; ++t) {
        if ((t >> 2) % kLjTeam != h) continue;  // this thread's groups only
        const unsigned e = (unsigned)S.nbr[nbr_slot(S.maxnb, i, t)];
        const int j = (int)(e & kNbrMask);
        const T4 pj = P[j];
        const T4 o = s_off[e >> kNbrShift];
        const T dx = (pj.x - pi.x) + o.x, dy = (pj.y - pi.y) + o.y, dz = (pj.z - pi.z) + o.z;
        const T r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        if (!(r2 > lo && r2 < rcsq + g2)) continue;
        atomicAdd(&S.ctr[CTR_GUARD], 1ull);
        if (!exact_within(X, n, i, j, S.L, S.rc2sq)) continue;
        const T ir2 = recip_fast<T>(r2);
        const T sr2 = sig2 * ir2;
        const T sr6 = sr2 * sr2 * sr2;
        const T sr12 = sr6 * sr6;
        const T g = eps24 * (sr12 + sr12 - sr6) * ir2;
        f.add(-g * dx, -g * dy, -g * dz);
        if (energy) {
          ud.add(eps4 * (sr12 - sr6));
          wd.add(g * r2);
        }
      }
    }
  }
  {
    // the team's partial forces, added in FP64 (every thread of the warp takes part in the shuffles)
    double F[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      F[a] = active ? f.get(a) : 0.0;
#pragma unroll
      for (int o = 1; o < kLjTeam; o <<= 1) F[a] += __shfl_xor_sync(0xffffffffu, F[a], o);
    }
    if (active && h == 0) {
      bool bad = false;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        S.f2[a * n + i] = F[a];
        bad |= !finite_bits(F[a]);
      }
      if (bad) atomicOr(&S.flags[FLG_ERR], ERR_NONFINITE);
    }
  }
  if (energy) {  // every pair appears in both members' lists: halve
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double us = warp_sum(ud.get()), ws = warp_sum(wd.get());
    if (lane == 0) {
      red_u[warp] = us;
      red_w[warp] = ws;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double ut = 0.0, wt = 0.0;
#pragma unroll
      for (int q = 0; q < kPer / 32; ++q) {
        ut += red_u[q];
        wt += red_w[q];
      }
      atomicAdd(&S.acc[ACC_U2], 0.5 * ut);
      atomicAdd(&S.acc[ACC_W2], 0.5 * wt);
    }
  }
}

// Velocity-Verlet kick/drift of Algorithm 2 after an LJ evaluation, one thread per particle (FP64):
//   LJ_MID:  v += dt F2 / m (closing half kick of this inner step + opening half kick of the next),
//            x += dt v, cell-local FP32 coordinates of the new positions, displacement check;
//   LJ_LAST: v += dt/2 F2 / m (closing half kick before the three-body evaluation).
// M_NEAR (distance classes, LJ_MID only): the step closes a block of s_near inner steps, so the
// near-class kicks s_near dt/2 F3near / m closing this block and opening the next are added too.
template <typename T>
__global__ void __launch_bounds__(256) k_kick(const SysDev* __restrict__ sys, const PItem* __restrict__ items) {
  const PItem it = items[blockIdx.x];
#if R3B_STAGE_SYS
  __shared__ StagedSys s_sys;
  stage_sys(s_sys, sys, it.sys);
  pdl_wait();
  __syncthreads();
  const SysDev& S = s_sys.get();
#else
  pdl_wait();
  const SysDev& S = sys[it.sys];
#endif
  const int mode = item_mode(S, it.mode);
  if (mode & M_SKIP) return;
  const int kind = mode & M_KIND_MASK;
  if (kind != LJ_MID && kind != LJ_LAST) return;
  const int n = S.n;
  const int i = it.begin + threadIdx.x;
  if (i >= n) return;
  bool bad = false;
  if (kind == LJ_MID) {
    using T4 = typename V4<T>::type;
    const double c = S.dt_in * S.inv_mass;
    const double* X = S.X[it.buf];
    double* Xo = S.X[it.buf ^ 1];
    // inputs first (see cell_centre)
    double vv[3], f[3], x[3], cen[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      vv[a] = S.v[a * n + i];
      f[a] = S.f2[a * n + i];
      x[a] = X[a * n + i];
    }
    const T4 r = reinterpret_cast<const T4*>(S.ref)[i];
    cell_centre(S, S.pcell[i], cen);
#pragma unroll
    for (int a = 0; a < 3; ++a) vv[a] = fma(c, f[a], vv[a]);
    if (mode & M_NEAR) {  // block-uniform; FP64 instructions are costly on GB300: only where needed
      double fn[3];
      take_near<T>(S, i, fn);
      const double cn = S.dt_near * S.inv_mass;
#pragma unroll
      for (int a = 0; a < 3; ++a) vv[a] = fma(cn, fn[a], vv[a]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      S.v[a * n + i] = vv[a];
      x[a] = fma(S.dt_in, vv[a], x[a]);
      Xo[a * n + i] = x[a];
      bad |= !finite_bits(vv[a]);
    }
    store_pos_checked<T>(S, it.buf ^ 1, i, x, cen, r);
  } else {
    const double c = 0.5 * S.dt_in * S.inv_mass;
    double vv[3], f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {  // inputs first (see cell_centre)
      vv[a] = S.v[a * n + i];
      f[a] = S.f2[a * n + i];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      vv[a] = fma(c, f[a], vv[a]);
      S.v[a * n + i] = vv[a];
      bad |= !finite_bits(vv[a]);
    }
  }
  if (bad) atomicOr(&S.flags[FLG_ERR], ERR_NONFINITE);
}

// ============================================================== ATM triplet kernel
//
// One CTA per base cell b (persistent over the work list).  A triplet is
// owned by its member with the smallest sorted index i, which lies in b;
// the other two have larger sorted indices, hence lie in b or in a stencil
// cell whose index is larger than b's.  The CTA stages those cells in
// shared memory with coordinates relative to b's centre (FP32 as a hi + lo
// pair so differences keep full precision), then for each i in b one warp
//   1. compacts i's half list {j : idx_j > idx_i, r_ij <= r_c} (ballot),
//   2. walks all neighbour pairs (j, k) of that list through a k-major pair
//      table, tests r_jk <= r_c and compacts accepted pairs into a queue,
//   3. evaluates 32 queued triplets at a time with all lanes busy:
//      F_i stays in registers (warp-shuffle reduction at the end), F_j and
//      F_k go to the staged particles' shared-memory accumulators.
// The staged accumulators are written to per-stencil-slot partial arrays;
// k_combine adds a particle's (at most 27) partials in a fixed order.
//
// Triplet algebra in squared distances a = r_ij^2, b = r_ik^2, c = r_jk^2:
//   phi = nu [ (abc)^(-3/2) + 3/8 P (abc)^(-5/2) ],
//   P = (a+b-c)(a-b+c)(-a+b+c)   (8 (abc) cos_i cos_j cos_k, law of cosines)
//   dphi/da = nu (abc)^(-5/2) [ 3/8 dP/da - (3/2 abc + 15/16 P) / a ]  (and b, c alike)
//   F_i = 2 (phi_a d_ij + phi_b d_ik),  F_j = 2 (-phi_a d_ij + phi_c d_jk),  F_k = -(F_i + F_j)
// with d_ij = x_j - x_i, d_ik = x_k - x_i, d_jk = x_k - x_j.

struct AtmLayout {
  size_t table, nd, nslot, nidx, queue, aq, sp, sl, acc, sidx, sst, total;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename T>
__host__ __device__ inline AtmLayout atm_layout(int smax) {
  using T4 = typename V4<T>::type;
  AtmLayout l;
  size_t o = 0;
  l.table = o;  // the pair table is read from global memory through L1
  l.nd = o; o = al16(o + sizeof(T4) * kMaxHalf * kAtmWarps);
  l.nslot = o; o = al16(o + sizeof(unsigned short) * kMaxHalf * kAtmWarps);
  l.nidx = o; o = al16(o + sizeof(int) * kMaxHalf * kAtmWarps);
  l.queue = o; o = al16(o + sizeof(unsigned) * kQueue * kAtmWarps);
  l.aq = o; o = al16(o + sizeof(T) * 3 * kMaxHalf * kAtmWarps);
  l.sp = o; o = al16(o + sizeof(T4) * smax);
  l.sl = o; o = al16(o + (sizeof(T) == 4 ? sizeof(T4) * smax : 0));
  l.acc = o; o = al16(o + sizeof(T) * 3 * smax);
  l.sidx = o; o = al16(o + sizeof(int) * smax);
  l.sst = o; o = al16(o + smax);
  l.total = o;
  return l;
}

template <typename T>
struct TripletOut {
  T fi[3], fj[3], fk[3], u;
};

template <typename T>
__device__ __forceinline__ void atm_triplet(const T nu, const typename V4<T>::type dj, const typename V4<T>::type dk,
                                            TripletOut<T>& o) {
  const T ex = dk.x - dj.x, ey = dk.y - dj.y, ez = dk.z - dj.z;  // d_jk
  const T a = dj.w, b = dk.w;
  const T c = ex * ex + ey * ey + ez * ez;
  const T ab = a * b;
  const T q = ab * c;
  const T t = rsqrt_acc<T>(q);
  const T w = t * t;         // 1 / (abc)
  const T t3 = w * t;        // (abc)^(-3/2)
  const T t5 = t3 * w;       // (abc)^(-5/2)
  const T s = a + b + c;
  const T A = s - (c + c), B = s - (b + b), C = s - (a + a);
  const T AB = A * B, AC = A * C, BC = B * C;
  const T P = AB * C;
  const T Pa = (a + a) * C - AB;
  const T Pb = (b + b) * B - AC;
  const T Pc = (c + c) * A - BC;
  const T G = (T)1.5 * q + (T)0.9375 * P;
  const T ia = (b * c) * w, ib = (a * c) * w, ic = ab * w;
  const T nt5 = nu * t5;
  const T pa2 = (T)2 * nt5 * ((T)0.375 * Pa - ia * G);
  const T pb2 = (T)2 * nt5 * ((T)0.375 * Pb - ib * G);
  const T pc2 = (T)2 * nt5 * ((T)0.375 * Pc - ic * G);
  o.fi[0] = pa2 * dj.x + pb2 * dk.x;
  o.fi[1] = pa2 * dj.y + pb2 * dk.y;
  o.fi[2] = pa2 * dj.z + pb2 * dk.z;
  o.fj[0] = pc2 * ex - pa2 * dj.x;
  o.fj[1] = pc2 * ey - pa2 * dj.y;
  o.fj[2] = pc2 * ez - pa2 * dj.z;
  o.fk[0] = -(o.fi[0] + o.fj[0]);
  o.fk[1] = -(o.fi[1] + o.fj[1]);
  o.fk[2] = -(o.fi[2] + o.fj[2]);
  o.u = nu * t3 * ((T)1 + (T)0.375 * P * w);
}

template <typename T>
__global__ void __launch_bounds__(kAtmThreads, 3)
    k_atm(const SysDev* __restrict__ sys, const CItem* __restrict__ items, int nitems,
          const uint16_t* __restrict__ gtable, int smax) {
  pdl_wait();
  using T4 = typename V4<T>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const AtmLayout Ly = atm_layout<T>(smax);
  T4* sp = reinterpret_cast<T4*>(smem + Ly.sp);
  T4* sl = reinterpret_cast<T4*>(smem + Ly.sl);
  T* acc = reinterpret_cast<T*>(smem + Ly.acc);
  int* sidx = reinterpret_cast<int*>(smem + Ly.sidx);
  unsigned char* sst = smem + Ly.sst;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  T4* nd = reinterpret_cast<T4*>(smem + Ly.nd) + warp * kMaxHalf;
  unsigned short* nslot = reinterpret_cast<unsigned short*>(smem + Ly.nslot) + warp * kMaxHalf;
  int* nidx = reinterpret_cast<int*>(smem + Ly.nidx) + warp * kMaxHalf;
  unsigned* queue = reinterpret_cast<unsigned*>(smem + Ly.queue) + warp * kQueue;
  // forces on the neighbours of the warp's current base particle, by list position
  T* aq = reinterpret_cast<T*>(smem + Ly.aq) + warp * 3 * kMaxHalf;

  __shared__ int st_begin[28], st_cnt[27], st_cell[27], st_s[27];
  __shared__ double red[32];
  __shared__ int next_base;


  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const CItem it = items[item];
    const SysDev& S = sys[it.sys];
    const int imode = item_mode(S, it.mode);
    if (imode & M_SKIP) continue;  // CTA-uniform
    const int n = S.n, nc = S.nc, b = it.cell;
    const bool energy = (imode & M_ENERGY) != 0;
    const double* __restrict__ X = S.X[it.buf];
    __syncthreads();  // previous item fully consumed the shared arrays
    // ---- stencil: lane l of warp 0 handles stencil cell s(l); the base cell is first
    if (warp == 0) {
      int s = (lane == 0) ? 13 : (lane <= 13 ? lane - 1 : lane);
      int cnt = 0, cell = 0;
      if (lane < 27) {
        int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
        int bx = b % nc, by = (b / nc) % nc, bz = b / (nc * nc);
        int xx = (bx + dx + nc) % nc, yy = (by + dy + nc) % nc, zz = (bz + dz + nc) % nc;
        cell = (zz * nc + yy) * nc + xx;
        if (cell >= b) cnt = S.cell_start[cell + 1] - S.cell_start[cell];
        st_cnt[lane] = cnt;
        st_cell[lane] = cell;
        st_s[lane] = s;
      }
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (lane < 27) st_begin[lane] = incl - cnt;
      if (lane == 26) st_begin[27] = incl;
    }
    __syncthreads();
    // ---- stage particles with coordinates relative to the base cell centre.  The base cell
    //      fills slots [0, nbase) in sorted order.  A particle of another cell is kept only if
    //      it lies within r_c of the base cell's box (no triplet of a base particle can include
    //      the others) and is appended through a shared counter; a dropped particle receives
    //      zero partial forces from this cell.
    __shared__ int n_kept;
    const int nbase = min(st_cnt[0], smax);
    if (threadIdx.x == 0) {
      n_kept = nbase;
      if (st_cnt[0] > smax) atomicOr(&S.flags[FLG_ERR], ERR_CELL_CAP);
    }
    __syncthreads();
    const T edge_hi = Par<T>::edge(S);
    const T edge_lo = Par<T>::edge_lo(S);
    const T half_e = Par<T>::half_edge(S);
    const T reach2 = Par<T>::reach2(S);
    T* part = reinterpret_cast<T*>(S.partial);
    for (int l = warp; l < 27; l += kAtmWarps) {
      const int cnt = st_cnt[l];
      if (cnt == 0) continue;
      const int s = st_s[l];
      const int c0 = S.cell_start[st_cell[l]];
      const T ox = (T)(s % 3 - 1), oy = (T)((s / 3) % 3 - 1), oz = (T)(s / 9 - 1);
      for (int e0 = 0; e0 < cnt; e0 += 32) {
        const int e = e0 + lane;
        const bool have = e < cnt;
        const int p = c0 + e;
        T4 hs, ls;
        if (have) {
          T4 h = reinterpret_cast<const T4*>(S.pos[it.buf])[p];
          if (sizeof(T) == 4) {
            T4 lo = reinterpret_cast<const T4*>(S.poslo)[p];
            float sx, ex, sy, ey, sz, ez;
            two_sum((float)h.x, (float)(ox * edge_hi), sx, ex);
            two_sum((float)h.y, (float)(oy * edge_hi), sy, ey);
            two_sum((float)h.z, (float)(oz * edge_hi), sz, ez);
            hs.x = sx; hs.y = sy; hs.z = sz; hs.w = 0;
            ls.x = lo.x + (ex + ox * edge_lo);
            ls.y = lo.y + (ey + oy * edge_lo);
            ls.z = lo.z + (ez + oz * edge_lo);
            ls.w = 0;
          } else {
            hs.x = h.x + (T)((double)ox * S.edge);
            hs.y = h.y + (T)((double)oy * S.edge);
            hs.z = h.z + (T)((double)oz * S.edge);
            hs.w = 0;
          }
        }
        bool keep = have;
        int slot = e;
        if (l != 0) {
          if (have) {
            const T bx = max(abs(hs.x) - half_e, (T)0), by = max(abs(hs.y) - half_e, (T)0),
                    bz = max(abs(hs.z) - half_e, (T)0);
            keep = bx * bx + by * by + bz * bz <= reach2;
          }
          const unsigned bal = __ballot_sync(0xffffffffu, keep);
          int base = 0;
          if (lane == 0 && bal) base = atomicAdd(&n_kept, __popc(bal));
          base = __shfl_sync(0xffffffffu, base, 0);
          slot = base + __popc(bal & lt);
        }
        if (keep && slot < smax) {
          if (sizeof(T) == 4) sl[slot] = ls;
          sp[slot] = hs;
          sidx[slot] = p;
          sst[slot] = (unsigned char)s;
          acc[slot] = (T)0;
          acc[smax + slot] = (T)0;
          acc[2 * smax + slot] = (T)0;
        } else if (have && !keep) {
          part[(3 * (size_t)s + 0) * n + p] = (T)0;
          part[(3 * (size_t)s + 1) * n + p] = (T)0;
          part[(3 * (size_t)s + 2) * n + p] = (T)0;
        }
      }
    }
    __syncthreads();
    const int nstaged = min(n_kept, smax);
    if (n_kept > smax && threadIdx.x == 0) atomicOr(&S.flags[FLG_ERR], ERR_CELL_CAP);
    const T rcsq = Par<T>::rc3sq(S);
    const T g3 = Par<T>::guard3(S);
    const T nu = Par<T>::nu(S);
    AccS<T> uacc;
    unsigned long long ntrip = 0;
    // ---- one warp per base particle i.  Warps take particles from a shared counter in
    //      increasing sorted order: the lowest indices own the longest half lists, so the
    //      longest jobs start first and the CTA's warps finish close together.
    if (threadIdx.x == 0) next_base = kAtmWarps;
    __syncthreads();
    for (int is = warp; is < nbase;) {
      const T4 pi = sp[is];
      const int gi = sidx[is];
      // 1. half list: staged particles after i with r_ij <= r_c (hi parts; guard band in FP64)
      int m = 0;
      for (int t0 = is + 1; t0 < nstaged; t0 += 32) {
        const int t = t0 + lane;
        bool ok = false;
        if (t < nstaged) {
          const T4 pt = sp[t];
          const T dx = pt.x - pi.x, dy = pt.y - pi.y, dz = pt.z - pi.z;
          const T r2 = dx * dx + dy * dy + dz * dz;
          if (r2 <= rcsq + g3) {
            if (r2 >= rcsq - g3) {
              atomicAdd(&S.ctr[CTR_GUARD], 1ull);
              ok = exact_within(X, n, gi, sidx[t], S.L, S.rc3sq);
            } else {
              ok = true;
            }
          }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (ok) {
          const int pos = m + __popc(bal & lt);
          if (pos < kMaxHalf) nslot[pos] = (unsigned short)t;
        }
        m += __popc(bal);
      }
      if (m > kMaxHalf) {
        if (lane == 0) atomicOr(&S.flags[FLG_ERR], ERR_HALF_CAP);
        m = kMaxHalf;
      }
      __syncwarp();
      //    full-precision difference vectors of the accepted neighbours: (hi_t - hi_i) exactly
      //    by TwoSum, plus the lo parts (FP32); plain differences in FP64
      {
        T4 li;
        if (sizeof(T) == 4) li = sl[is];
        for (int q = lane; q < m; q += 32) {
          const int t = nslot[q];
          const T4 pt = sp[t];
          T dx, dy, dz;
          if (sizeof(T) == 4) {
            const T4 lt4 = sl[t];
            float s0, e0, s1, e1, s2, e2;
            two_sum((float)pt.x, -(float)pi.x, s0, e0);
            two_sum((float)pt.y, -(float)pi.y, s1, e1);
            two_sum((float)pt.z, -(float)pi.z, s2, e2);
            dx = s0 + (e0 + ((float)lt4.x - (float)li.x));
            dy = s1 + (e1 + ((float)lt4.y - (float)li.y));
            dz = s2 + (e2 + ((float)lt4.z - (float)li.z));
          } else {
            dx = pt.x - pi.x;
            dy = pt.y - pi.y;
            dz = pt.z - pi.z;
          }
          T4 d4;
          d4.x = dx; d4.y = dy; d4.z = dz; d4.w = dx * dx + dy * dy + dz * dz;
          nd[q] = d4;
          nidx[q] = sidx[t];
        }
      }
      __syncwarp();
      // 2. neighbour pairs (j, k) of the half list, k-major through the pair table;
      //    pairs with r_jk <= r_c are compacted into the warp's queue in table order
      T fi0 = 0, fi1 = 0, fi2 = 0;
      const int np = m * (m - 1) / 2;
      int qn = 0;
      for (int q = lane; q < m; q += 32) {
        aq[q] = (T)0;
        aq[kMaxHalf + q] = (T)0;
        aq[2 * kMaxHalf + q] = (T)0;
      }
      __syncwarp();
      // add a force to list position q of the warp-private accumulator.  Plain read-modify-
      // write; lanes of the warp that target the same q in the same step are detected with
      // a match and their values summed by shuffles first, so every slot has one writer.
      auto add_q = [&](unsigned mask, int q, T fx, T fy, T fz) {
        const unsigned grp = __match_any_sync(mask, q);
        const int leader = __ffs(grp) - 1;
        if (grp != (1u << lane)) {
          unsigned others = grp & ~(1u << leader);
          while (others) {
            const int src = __ffs(others) - 1;
            others &= others - 1;
            const T ox = __shfl_sync(grp, fx, src), oy = __shfl_sync(grp, fy, src), oz = __shfl_sync(grp, fz, src);
            if (lane == leader) {
              fx += ox;
              fy += oy;
              fz += oz;
            }
          }
        }
        if (lane == leader) {
          aq[q] += fx;
          aq[kMaxHalf + q] += fy;
          aq[2 * kMaxHalf + q] += fz;
        }
      };
      // 3. queued triplets: lane l takes a contiguous run of the queue, so its pairs mostly
      //    share k (k-major order): F_k and d_k stay in registers until k changes
      auto drain = [&](int count) {
        if (count <= 0) return;
        const int C = ((count + 31) >> 5) | 1;  // odd run length: lanes start in different banks
        const int e0 = lane * C, len = max(0, min(e0 + C, count) - e0);
        // each lane starts its run at a lane-dependent offset: columns list j in ascending
        // order, so lanes that walked their runs in step would hit the same j together
        int off = len ? (lane * 5) % len : 0;
        int curk = -1;
        T4 dk;
        T fk0 = 0, fk1 = 0, fk2 = 0;
        for (int r = 0; r < C; ++r) {  // every lane runs all C steps (warp-wide ballots below)
          const bool act = r < len;
          const unsigned amask = __ballot_sync(0xffffffffu, act);
          if (act) {
            const int e = e0 + off;
            if (++off == len) off = 0;
            const unsigned entry = queue[e];
            const int j = (int)(entry & 0xffffu), k = (int)(entry >> 16);
            const bool change = k != curk;
            const unsigned cmask = __ballot_sync(amask, change && curk >= 0);
            if (change && curk >= 0) add_q(cmask, curk, fk0, fk1, fk2);
            if (change) {
              curk = k;
              dk = nd[k];
              fk0 = fk1 = fk2 = 0;
            }
            TripletOut<T> o;
            atm_triplet<T>(nu, nd[j], dk, o);
            fi0 += o.fi[0];
            fi1 += o.fi[1];
            fi2 += o.fi[2];
            fk0 += o.fk[0];
            fk1 += o.fk[1];
            fk2 += o.fk[2];
            add_q(amask, j, o.fj[0], o.fj[1], o.fj[2]);
            if (energy) uacc.add(o.u);
          }
        }
        __syncwarp();
        const unsigned fmask = __ballot_sync(0xffffffffu, curk >= 0);
        if (curk >= 0) add_q(fmask, curk, fk0, fk1, fk2);
        __syncwarp();
        ntrip += (unsigned long long)count;
      };
      for (int p0 = 0; p0 < np; p0 += 32) {
        const int p = p0 + lane;
        bool ok = false, band = false;
        unsigned entry = 0;
        int jj = 0, kk = 0;
        if (p < np) {
          const unsigned e = __ldg(gtable + p);
          jj = (int)(e & 0xffu);
          kk = (int)(e >> 8);
          const T4 dj = nd[jj], dk = nd[kk];
          const T ex = dk.x - dj.x, ey = dk.y - dj.y, ez = dk.z - dj.z;
          const T c = ex * ex + ey * ey + ez * ez;
          ok = c < rcsq - g3;
          band = (c >= rcsq - g3) && (c <= rcsq + g3);
          entry = (unsigned)jj | ((unsigned)kk << 16);
        }
        if (__any_sync(0xffffffffu, band)) {  // rare: decide the guard band exactly in FP64
          if (band) {
            atomicAdd(&S.ctr[CTR_GUARD], 1ull);
            ok = exact_within(X, n, nidx[jj], nidx[kk], S.L, S.rc3sq);
          }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (ok) queue[qn + __popc(bal & lt)] = entry;
        qn += __popc(bal);
        if (qn > kQueue - 32) {  // next round could overflow: evaluate what is queued
          __syncwarp();
          drain(qn);
          __syncwarp();
          qn = 0;
        }
      }
      __syncwarp();
      drain(qn);
      __syncwarp();
      // neighbours' totals for this base particle -> staged accumulators (one atomic per
      // neighbour and component); F_i by a warp reduction
      for (int q = lane; q < m; q += 32) {
        const int sq = nslot[q];
        atomicAdd(&acc[sq], aq[q]);
        atomicAdd(&acc[smax + sq], aq[kMaxHalf + q]);
        atomicAdd(&acc[2 * smax + sq], aq[2 * kMaxHalf + q]);
      }
      fi0 = warp_sum_t<T>(fi0);
      fi1 = warp_sum_t<T>(fi1);
      fi2 = warp_sum_t<T>(fi2);
      if (lane == 0) {
        atomicAdd(&acc[is], fi0);
        atomicAdd(&acc[smax + is], fi1);
        atomicAdd(&acc[2 * smax + is], fi2);
      }
      __syncwarp();
      int nx = 0;
      if (lane == 0) nx = atomicAdd(&next_base, 1);
      is = __shfl_sync(0xffffffffu, nx, 0);
    }
    __syncthreads();
    // ---- partial forces of every staged particle, one slot per stencil offset
    for (int t = threadIdx.x; t < nstaged; t += blockDim.x) {
      const size_t s = sst[t];
      const int p = sidx[t];
      part[(3 * s + 0) * (size_t)n + p] = acc[t];
      part[(3 * s + 1) * (size_t)n + p] = acc[smax + t];
      part[(3 * s + 2) * (size_t)n + p] = acc[2 * smax + t];
    }
    if (lane == 0 && ntrip) atomicAdd(&S.ctr[CTR_TRIPLETS], ntrip);  // ntrip is warp-uniform
    if (energy) {
      double us = block_sum(uacc.get(), red);
      if (threadIdx.x == 0) {
        atomicAdd(&S.acc[ACC_U3], us);
        atomicAdd(&S.acc[ACC_W3], 9.0 * us);  // phi3 is homogeneous of degree -9: sum r.F = 9 phi3
      }
    }
  }
}

// ============================================================== ATM, one warp per particle
//
// Variant without Newton-3 scatter: warp x gathers x's neighbours within r_c3 from the
// fresh pair list (a superset: r_c2 + skin >= r_c3 is required), tests every unordered
// pair (y, z) of them for r_yz <= r_c3 and evaluates only the force on x,
//   F_x = 2 (phi_a d_xy + phi_b d_xz),  a = r_xy^2, b = r_xz^2, c = r_yz^2,
// so each triplet is evaluated once from each of its three members.  No shared-memory
// accumulation, no staging, no partial buffers: F_x is a warp reduction written directly.
// Energy: each evaluation adds phi / 3.  Triplets are counted where x has the smallest index.

// warp sum of one FP32 value per lane as an error-free (hi, lo) pair (TwoSum tree)
__device__ __forceinline__ void warp_sum_pair(float v, float& hi, float& lo) {
  hi = v;
  lo = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
    float s, e;
    two_sum(hi, oh, s, e);
    hi = s;
    lo = lo + (ol + e);
  }
}

// warp sum of one value per lane: FP32 with compensation (result valid in every lane);
// plain FP64 in the FP64 path
template <typename T> __device__ __forceinline__ double warp_sum_comp(T v);
template <> __device__ __forceinline__ double warp_sum_comp<float>(float v) {
  float hi = v, lo = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
    float s, e;
    two_sum(hi, oh, s, e);
    hi = s;
    lo = lo + (ol + e);
  }
  return (double)hi + (double)lo;
}
template <> __device__ __forceinline__ double warp_sum_comp<double>(double v) { return warp_sum(v); }

template <typename T>
__device__ __forceinline__ void atm_vertex(const T nu, const typename V4<T>::type dy, const typename V4<T>::type dz,
                                           T& fx, T& fy, T& fz, T& u) {
  const T ex = dz.x - dy.x, ey = dz.y - dy.y, ez = dz.z - dy.z;  // d_yz
  const T a = dy.w, b = dz.w;
  const T c = ex * ex + ey * ey + ez * ez;
  const T ab = a * b;
  const T q = ab * c;
  const T t = rsqrt_acc<T>(q);
  const T w = t * t;
  const T t3 = w * t;
  const T t5 = t3 * w;
  const T s = a + b + c;
  const T A = s - (c + c), B = s - (b + b), C = s - (a + a);
  const T AB = A * B, AC = A * C;
  const T P = AB * C;
  const T Pa = (a + a) * C - AB;
  const T Pb = (b + b) * B - AC;
  const T G = (T)1.5 * q + (T)0.9375 * P;
  const T ia = (b * c) * w, ib = (a * c) * w;
  const T nt5 = nu * t5;
  const T pa2 = (T)2 * nt5 * ((T)0.375 * Pa - ia * G);
  const T pb2 = (T)2 * nt5 * ((T)0.375 * Pb - ib * G);
  fx = pa2 * dy.x + pb2 * dz.x;
  fy = pa2 * dy.y + pb2 * dz.y;
  fz = pa2 * dy.z + pb2 * dz.z;
  u = nu * t3 * ((T)1 + (T)0.375 * P * w);
}

constexpr int kPaWarps = 4;
constexpr int kMaxFull = 128;  // neighbours within r_c3 of one particle

template <typename T>
__global__ void __launch_bounds__(32 * kPaWarps)
    k_atm_pa(const SysDev* __restrict__ sys, const PItem* __restrict__ items, const uint16_t* __restrict__ gtable) {
  pdl_wait();
  using T4 = typename V4<T>::type;
  __shared__ T4 s_nd[kPaWarps][kMaxFull];
  __shared__ int s_idx[kPaWarps][kMaxFull];
  __shared__ unsigned s_q[kPaWarps][64];
  const PItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  const int imode = item_mode(S, it.mode);
  if (imode & M_SKIP) return;
  const bool energy = (imode & M_ENERGY) != 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int x = it.begin + warp;
  if (x >= S.n) return;  // whole warp leaves together
  const int n = S.n;
  T4* nd = s_nd[warp];
  int* nidx = s_idx[warp];
  unsigned* queue = s_q[warp];
  const T4* __restrict__ P = reinterpret_cast<const T4*>(S.pos[it.buf]);
  const T4* __restrict__ PL = reinterpret_cast<const T4*>(S.poslo);
  const double* __restrict__ X = S.X[it.buf];
  const T edge = Par<T>::edge(S), edge_lo = Par<T>::edge_lo(S);
  const T rcsq = Par<T>::rc3sq(S), g3 = Par<T>::guard3(S), nu = Par<T>::nu(S);
  const T4 px = P[x];
  T4 lx;
  if (sizeof(T) == 4) lx = PL[x];
  // 1. neighbours within r_c3 from the pair list (full-precision differences)
  const int cnt = S.nbr_cnt[x];
  const int* __restrict__ row = S.nbr + nbr_slot(S.maxnb, x, 0);
  int m = 0;
  for (int t0 = 0; t0 < cnt; t0 += 32) {
    const int t = t0 + lane;
    bool ok = false, band = false;
    int j = x;
    T dx = 0, dy = 0, dz = 0;
    if (t < cnt) {
      const unsigned e = (unsigned)__ldg(row + t);
      j = (int)(e & kNbrMask);
      const unsigned cde = e >> kNbrShift;
      const T ox = (T)(cde & 3u) - (T)1, oy = (T)((cde >> 2) & 3u) - (T)1, oz = (T)(cde >> 4) - (T)1;
      const T4 pj = P[j];
      if (sizeof(T) == 4) {
        const T4 lj = PL[j];
        float s1, e1, s2, e2;
        two_sum((float)pj.x, -(float)px.x, s1, e1);
        two_sum(s1, (float)(ox * edge), s2, e2);
        dx = s2 + ((e1 + e2) + (((float)lj.x - (float)lx.x) + (float)(ox * edge_lo)));
        two_sum((float)pj.y, -(float)px.y, s1, e1);
        two_sum(s1, (float)(oy * edge), s2, e2);
        dy = s2 + ((e1 + e2) + (((float)lj.y - (float)lx.y) + (float)(oy * edge_lo)));
        two_sum((float)pj.z, -(float)px.z, s1, e1);
        two_sum(s1, (float)(oz * edge), s2, e2);
        dz = s2 + ((e1 + e2) + (((float)lj.z - (float)lx.z) + (float)(oz * edge_lo)));
      } else {
        dx = (pj.x - px.x) + ox * edge;
        dy = (pj.y - px.y) + oy * edge;
        dz = (pj.z - px.z) + oz * edge;
      }
      const T r2 = dx * dx + dy * dy + dz * dz;
      ok = r2 < rcsq - g3;
      band = (r2 >= rcsq - g3) && (r2 <= rcsq + g3);
    }
    if (__any_sync(0xffffffffu, band)) {
      if (band) {
        atomicAdd(&S.ctr[CTR_GUARD], 1ull);
        ok = exact_within(X, n, x, j, S.L, S.rc3sq);
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, ok);
    if (ok) {
      const int pos = m + __popc(bal & lt);
      if (pos < kMaxFull) {
        T4 d4;
        d4.x = dx; d4.y = dy; d4.z = dz; d4.w = dx * dx + dy * dy + dz * dz;
        nd[pos] = d4;
        nidx[pos] = j;
      }
    }
    m += __popc(bal);
  }
  if (m > kMaxFull) {
    if (lane == 0) atomicOr(&S.flags[FLG_ERR], ERR_HALF_CAP);
    m = kMaxFull;
  }
  __syncwarp();
  // 2./3. pairs (y, z) of the list through the k-major table; accepted pairs go to a 64-entry
  //        ring and are evaluated 32 at a time (all lanes busy)
  T f0 = 0, f1 = 0, f2 = 0, uu = 0;
  unsigned long long own = 0;
  const int np = m * (m - 1) / 2;
  unsigned head = 0, tail = 0;  // warp-uniform ring positions
  auto eval = [&](unsigned entry) {
    const int y = (int)(entry & 0xffffu), z = (int)(entry >> 16);
    T ax, ay, az, au;
    atm_vertex<T>(nu, nd[y], nd[z], ax, ay, az, au);
    f0 += ax;
    f1 += ay;
    f2 += az;
    uu += au;
    own += (x < nidx[y] && x < nidx[z]) ? 1ull : 0ull;
  };
  for (int p0 = 0; p0 < np; p0 += 32) {
    const int p = p0 + lane;
    bool ok = false, band = false;
    unsigned entry = 0;
    if (p < np) {
      const unsigned e = __ldg(gtable + p);
      const T4 dy = nd[e & 0xffu], dz = nd[e >> 8];
      const T ex = dz.x - dy.x, ey = dz.y - dy.y, ez = dz.z - dy.z;
      const T c = ex * ex + ey * ey + ez * ez;
      ok = c < rcsq - g3;
      band = abs(c - rcsq) <= g3;
      entry = (e & 0xffu) | ((e >> 8) << 16);
    }
    const unsigned bband = __ballot_sync(0xffffffffu, band);
    if (bband) {  // rare: decide the guard band exactly in FP64
      if (band) {
        atomicAdd(&S.ctr[CTR_GUARD], 1ull);
        ok = exact_within(X, n, nidx[entry & 0xffffu], nidx[entry >> 16], S.L, S.rc3sq);
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, ok);
    if (ok) queue[(tail + __popc(bal & lt)) & 63u] = entry;
    tail += __popc(bal);
    if (tail - head >= 32) {
      __syncwarp();
      eval(queue[(head + lane) & 63u]);
      head += 32;
      __syncwarp();
    }
  }
  __syncwarp();
  if (lane < (int)(tail - head)) eval(queue[(head + lane) & 63u]);
  // F_x and the energy share: per-lane FP32 sums combined by an error-free (TwoSum) warp
  // reduction; the (hi, lo) pair is converted to FP64 by the combine kernel on full warps
  // (FP64 arithmetic is scarce on GB300)
  unsigned long long cnt_own = own;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt_own += __shfl_xor_sync(0xffffffffu, cnt_own, o);
  if constexpr (sizeof(T) == 4) {
    float h0, l0, h1, l1, h2, l2, hu = 0.f, lu = 0.f;
    warp_sum_pair(f0, h0, l0);
    warp_sum_pair(f1, h1, l1);
    warp_sum_pair(f2, h2, l2);
    if (energy) warp_sum_pair(uu, hu, lu);
    if (lane == 0) {
      float* pf = reinterpret_cast<float*>(S.partial);  // [6][n]: hi x, y, z then lo x, y, z
      pf[x] = h0;
      pf[n + x] = h1;
      pf[2 * n + x] = h2;
      pf[3 * n + x] = l0;
      pf[4 * n + x] = l1;
      pf[5 * n + x] = l2;
      if (cnt_own) atomicAdd(&S.ctr[CTR_TRIPLETS], cnt_own);
      if (energy) {
        const double U = (double)hu + (double)lu;
        atomicAdd(&S.acc[ACC_U3], U * (1.0 / 3.0));
        atomicAdd(&S.acc[ACC_W3], 3.0 * U);  // 9 * U / 3
      }
    }
  } else {
    const double F0 = warp_sum(f0), F1 = warp_sum(f1), F2 = warp_sum(f2);
    const double U = energy ? warp_sum(uu) : 0.0;
    if (lane == 0) {
      S.f3[x] = F0;
      S.f3[n + x] = F1;
      S.f3[2 * n + x] = F2;
      if (cnt_own) atomicAdd(&S.ctr[CTR_TRIPLETS], cnt_own);
      if (energy) {
        atomicAdd(&S.acc[ACC_U3], U / 3.0);
        atomicAdd(&S.acc[ACC_W3], 3.0 * U);
      }
    }
  }
}

// ============================================================== combine + outer kicks
template <typename T>
__global__ void __launch_bounds__(256) k_combine(const SysDev* __restrict__ sys, const PItem* __restrict__ items) {
  __shared__ double red[32];
  const PItem it = items[blockIdx.x];
#if R3B_STAGE_SYS
  __shared__ StagedSys s_sys;
  stage_sys(s_sys, sys, it.sys);
  pdl_wait();
  __syncthreads();
  const SysDev& S = s_sys.get();
#else
  pdl_wait();
  const SysDev& S = sys[it.sys];
#endif
  const int mode = item_mode(S, it.mode);
  if (mode & M_SKIP) return;
  const int kind = mode & M_KIND_MASK;
  const bool energy = (mode & M_ENERGY) != 0;
  const int n = S.n, nc = S.nc;
  const int p = it.begin + threadIdx.x;
  double ek = 0.0;
  if (p < n) {
    const int cell = S.pcell[p];
    const int cx = cell % nc, cy = (cell / nc) % nc, cz = cell / (nc * nc);
    const T* part = reinterpret_cast<const T*>(S.partial);
    Acc3<T> f;
    const bool ready = (mode & M_F3READY) != 0;  // the per-particle triplet kernel wrote f3
    const bool summed = (mode & M_F3ACC) != 0;   // the rotation kernel's atomic sums
#pragma unroll 1
    for (int s = 0; s < ((ready || summed) ? 0 : 27); ++s) {
      const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
      const int bx = (cx - dx + nc) % nc, by = (cy - dy + nc) % nc, bz = (cz - dz + nc) % nc;
      const int base = (bz * nc + by) * nc + bx;
      if (cell < base) continue;  // the CTA of that base cell did not stage this particle's cell
      f.add(part[(3 * s + 0) * (size_t)n + p], part[(3 * s + 1) * (size_t)n + p], part[(3 * s + 2) * (size_t)n + p]);
    }
    double F[3] = {f.get(0), f.get(1), f.get(2)};
    if (summed) {
      if (sizeof(T) == 4) {
        fix_take3(S.f3acc, p, S.fix_unit, F);
      } else {
        double* a = reinterpret_cast<double*>(S.f3acc) + 4 * (size_t)p;
        F[0] = a[0];
        F[1] = a[1];
        F[2] = a[2];
        a[0] = a[1] = a[2] = 0.0;
      }
    }
    if (ready) {
      if (sizeof(T) == 4) {
        const float* pf = reinterpret_cast<const float*>(S.partial);
        F[0] = (double)pf[p] + (double)pf[3 * n + p];
        F[1] = (double)pf[n + p] + (double)pf[4 * n + p];
        F[2] = (double)pf[2 * n + p] + (double)pf[5 * n + p];
      } else {
        F[0] = S.f3[p];
        F[1] = S.f3[n + p];
        F[2] = S.f3[2 * n + p];
      }
    }
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      S.f3[a * n + p] = F[a];
      bad |= !finite_bits(F[a]);
    }
    // distance classes: F holds near + far; the near part comes from the second evaluation
    const bool classes = S.f3n != nullptr;
    double Fn[3] = {0.0, 0.0, 0.0};
    if (classes) {
      take_near<T>(S, p, Fn);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        S.f3n[a * n + p] = Fn[a];
        bad |= !finite_bits(Fn[a]);
      }
    }
    if (kind != CB_INIT) {
      const double h = 0.5 * S.dt_out * S.inv_mass;
      const double hn = 0.5 * S.dt_near * S.inv_mass;
      double kk[3], vv[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        // far class every outer step, near class every s_near inner steps
        kk[a] = classes ? h * (F[a] - Fn[a]) + hn * Fn[a] : h * F[a];
        vv[a] = S.v[a * n + p] + kk[a];  // closing kicks
      }
      if (energy) ek = 0.5 * S.mass * (vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]);
      if (kind == CB_CONT) {
        const double* X = S.X[it.buf];
        double* Xo = S.X[0];
        double xn[3], rel[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          vv[a] += kk[a] + 0.5 * S.dt_in * S.inv_mass * S.f2[a * n + p];  // opening kicks of the next step
          xn[a] = X[a * n + p] + S.dt_in * vv[a];
          Xo[a * n + p] = xn[a];
        }
        cell_rel(S, cell, xn, rel);
        store_pos<T>(S, 0, p, rel, true);
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        S.v[a * n + p] = vv[a];
        bad |= !finite_bits(vv[a]);
      }
    }
    if (bad) atomicOr(&S.flags[FLG_ERR], ERR_NONFINITE);
  }
  if (energy) {
    double s = block_sum(ek, red);
    if (threadIdx.x == 0) atomicAdd(&S.acc[ACC_EK], s);
  }
}

// opening kicks (outer F3, inner F2) and first drift of a call
template <typename T>
__global__ void __launch_bounds__(256) k_start(const SysDev* __restrict__ sys, const PItem* __restrict__ items) {
  using T4 = typename V4<T>::type;
  const PItem it = items[blockIdx.x];
#if R3B_STAGE_SYS
  __shared__ StagedSys s_sys;
  stage_sys(s_sys, sys, it.sys);
  pdl_wait();
  __syncthreads();
  const SysDev& S = s_sys.get();
#else
  pdl_wait();
  const SysDev& S = sys[it.sys];
#endif
  const int n = S.n;
  const int p = it.begin + threadIdx.x;
  if (p >= n) return;
  const double* X = S.X[it.buf];
  double* Xo = S.X[0];
  // inputs first (see cell_centre)
  double f3[3], f3n[3] = {0.0, 0.0, 0.0}, v[3], f2[3], x[3], cen[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    f3[a] = S.f3[a * n + p];
    if (S.f3n) f3n[a] = S.f3n[a * n + p];
    v[a] = S.v[a * n + p];
    f2[a] = S.f2[a * n + p];
    x[a] = X[a * n + p];
  }
  const T4 r = reinterpret_cast<const T4*>(S.ref)[p];
  cell_centre(S, S.pcell[p], cen);
  bool bad = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // distance classes: far part (f3 - f3n) with the outer step, near part with s_near dt
    const double k3 = S.f3n ? 0.5 * S.dt_out * S.inv_mass * (f3[a] - f3n[a]) + 0.5 * S.dt_near * S.inv_mass * f3n[a]
                            : 0.5 * S.dt_out * S.inv_mass * f3[a];
    const double vv = v[a] + k3 + 0.5 * S.dt_in * S.inv_mass * f2[a];
    S.v[a * n + p] = vv;
    x[a] = x[a] + S.dt_in * vv;
    Xo[a * n + p] = x[a];
    bad |= !finite_bits(vv);
  }
  store_pos_checked<T>(S, 0, p, x, cen, r);
  if (bad) atomicOr(&S.flags[FLG_ERR], ERR_NONFINITE);
}

__global__ void __launch_bounds__(256) k_kinetic(const SysDev* __restrict__ sys, const PItem* __restrict__ items) {
  pdl_wait();
  __shared__ double red[32];
  const PItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  const int p = it.begin + threadIdx.x;
  double ek = 0.0;
  if (p < S.n) {
    const int n = S.n;
    double a = S.v[p], b = S.v[n + p], c = S.v[2 * n + p];
    ek = 0.5 * S.mass * (a * a + b * b + c * c);
  }
  double s = block_sum(ek, red);
  if (threadIdx.x == 0) atomicAdd(&S.acc[ACC_EK], s);
}

// ---------------------------------------------------------------- pair table
// k-major list of index pairs (j, k), j < k < kMaxHalf: the first m (m - 1) / 2
// entries are exactly the pairs of a list of length m.
static uint16_t* g_table = nullptr;

void atm_prepare_table(cudaStream_t s) {
  if (g_table) return;
  static uint16_t h[kPairTable];
  int p = 0;
  for (int k = 1; k < kMaxHalf; ++k)
    for (int j = 0; j < k; ++j) h[p++] = (uint16_t)(j | (k << 8));
  if (cudaMalloc(&g_table, sizeof(h)) != cudaSuccess) {
    g_table = nullptr;
    return;
  }
  cudaMemcpyAsync(g_table, h, sizeof(h), cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);
}

// The dynamic shared-memory limit of a kernel is shared by every system on a device: it is only
// ever raised, never lowered below what another system needs (raise_smem_attr).
int atm_configure(int smax, int precision, int* smem_bytes) {
  int bytes = (int)(precision ? atm_layout<double>(smax).total : atm_layout<float>(smax).total);
  *smem_bytes = bytes;
  int nb = 0;
  const void* kern = precision ? (const void*)k_atm<double> : (const void*)k_atm<float>;
  if (!raise_smem_attr(kern, bytes)) return 0;
  if (precision)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_atm<double>, kAtmThreads, bytes);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_atm<float>, kAtmThreads, bytes);
  return nb;
}

// ---------------------------------------------------------------- launchers
template <typename T, int kPer>
void launch_lj_per(const Launch& L, const PItem* items, int nitems, bool energy) {
  if (energy)
    launch_kernel(L, k_lj<T, true, kPer>, nitems, kPer, 0, L.sys, items);
  else
    launch_kernel(L, k_lj<T, false, kPer>, nitems, kPer, 0, L.sys, items);
}
// items of `block` particles (kLjBlocks), one thread each
template <typename T>
void launch_lj(const Launch& L, const PItem* items, int nitems, bool energy, int block) {
  if (nitems <= 0) return;
  if (block == 32)
    launch_lj_per<T, 32>(L, items, nitems, energy);
  else if (block == 128)
    launch_lj_per<T, 128>(L, items, nitems, energy);
  else
    launch_lj_per<T, 64>(L, items, nitems, energy);
}
template <typename T>
void launch_atm(const Launch& L, const CItem* items, int nitems, int grid, int smax) {
  if (nitems <= 0) return;
  const int bytes = (int)atm_layout<T>(smax).total;
  launch_kernel(L, k_atm<T>, grid, kAtmThreads, bytes, L.sys, items, nitems, (const uint16_t*)g_table, smax);
}
// same launch with a caller-provided pair table (used by the allocation-free entry point)
template <typename T>
void launch_atm_table(const Launch& L, const CItem* items, int nitems, int grid, int smax, const uint16_t* table) {
  if (nitems <= 0) return;
  const int bytes = (int)atm_layout<T>(smax).total;
  k_atm<T><<<grid, kAtmThreads, bytes, L.stream>>>(L.sys, items, nitems, table, smax);
}
template void launch_atm_table<float>(const Launch&, const CItem*, int, int, int, const uint16_t*);

template <typename T>
void launch_atm_pa(const Launch& L, const PItem* items, int nitems) {
  if (nitems > 0) launch_kernel(L, k_atm_pa<T>, nitems, 32 * kPaWarps, 0, L.sys, items, (const uint16_t*)g_table);
}
template void launch_atm_pa<float>(const Launch&, const PItem*, int);
template void launch_atm_pa<double>(const Launch&, const PItem*, int);

template <typename T>
void launch_kick(const Launch& L, const PItem* items, int nitems) {
  if (nitems > 0) launch_kernel(L, k_kick<T>, nitems, 256, 0, L.sys, items);
}
template void launch_kick<float>(const Launch&, const PItem*, int);
template void launch_kick<double>(const Launch&, const PItem*, int);

template <typename T>
void launch_combine(const Launch& L, const PItem* items, int nitems, int block) {
  if (nitems > 0) launch_kernel(L, k_combine<T>, nitems, block, 0, L.sys, items);
}
template <typename T>
void launch_start(const Launch& L, const PItem* items, int nitems, int block) {
  if (nitems > 0) launch_kernel(L, k_start<T>, nitems, block, 0, L.sys, items);
}
void launch_kinetic(const Launch& L, const PItem* items, int nitems, int block) {
  if (nitems > 0) launch_kernel(L, k_kinetic, nitems, block, 0, L.sys, items);
}

template void launch_lj<float>(const Launch&, const PItem*, int, bool, int);
template void launch_lj<double>(const Launch&, const PItem*, int, bool, int);
template void launch_combine<float>(const Launch&, const PItem*, int, int);
template void launch_combine<double>(const Launch&, const PItem*, int, int);
template void launch_start<float>(const Launch&, const PItem*, int, int);
template void launch_start<double>(const Launch&, const PItem*, int, int);
template void launch_atm<float>(const Launch&, const CItem*, int, int, int);
template void launch_atm<double>(const Launch&, const CItem*, int, int, int);

}  // namespace r3b
