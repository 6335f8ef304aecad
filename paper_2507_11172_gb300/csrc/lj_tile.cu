// Lennard-Jones 12-6 pair forces (Sec. 2.1): two alternatives to the row kernel k_lj (forces.cu), all
// three timed by the autotuner.
//
//   k_lj_team  4, 8 or 16 lanes per particle share its pair-list row (end of this file).
//   k_lj_tile  one CTA per block of 2 x 2 x 2 cells (linked cells, Sec. 2.2).  The 4 x 4 x 4 cells around the block (every
//              cell a pair-list entry of the block's particles can point to) are copied into shared
//              memory by bulk asynchronous copies (cp.async.bulk, one per cell: each cell's particles
//              are contiguous in the sorted order) that complete on an mbarrier, then shifted into one
//              frame, the block's centre.  Each thread computes the force on one particle of the block
//              from its pair-list row (F_i only, every pair evaluated from both members, no scatter);
//              the neighbour positions come from shared memory instead of scattered global gathers.
//
// A list entry j | code << 26 (code: offset of j's cell from i's cell, 2 bits per axis) maps to the
// staged slot j + delta(own cell of i, code), delta = first staged slot of that region cell minus the
// cell's first sorted index (a 512-entry table per CTA).  Padding entries (code 63) map to one staged
// slot placed far outside every cutoff.
//
// Precision: the staged FP32 coordinates are the cell-local coordinates plus the FP32-rounded offset
// of their cell's centre from the block's centre (|x| <= about 6 sigma); a pair displacement then
// takes one subtraction, with an absolute error within a factor of about 1.2 of the row kernel's
// (cell-local difference plus a cell offset, rounded at the same magnitudes).
#include "md_internal.cuh"
#include "lj_common.cuh"
#include "sys_stage.cuh"

namespace r3b {

namespace {

constexpr int kLjtWaitLimit = 1 << 19;  // polls of the copy barrier (0.1-0.3 s) before giving up

__device__ __forceinline__ unsigned lt_smem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// mbarrier with an arrival count of one, made visible to the asynchronous proxy
__device__ __forceinline__ void lt_bar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(lt_smem(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// the single arrival, announcing the bytes the copies will deliver
__device__ __forceinline__ void lt_bar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(lt_smem(bar)), "r"(bytes) : "memory");
}
// bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16), completing on bar
__device__ __forceinline__ void lt_bulk(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   lt_smem(dst)),
               "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(lt_smem(bar))
               : "memory");
}
__device__ __forceinline__ bool lt_bar_done(unsigned long long* bar) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(lt_smem(bar))
      : "memory");
  return ok != 0;
}
// wait for phase 0 of bar, polling at most kLjtWaitLimit times
__device__ __forceinline__ bool lt_bar_wait(unsigned long long* bar) {
  for (int k = 0; k < kLjtWaitLimit; ++k) {
    if (lt_bar_done(bar)) return true;
    if (k >= 16) __nanosleep(256);
  }
  return false;
}

// FP32: hardware reciprocal refined by one Newton step (r^2 is a normal positive number here)
template <typename T> __device__ __forceinline__ T lt_recip(T x);
template <> __device__ __forceinline__ float lt_recip<float>(float x) {
  const float y = __fdividef(1.0f, x);
  return y * fmaf(-x, y, 2.0f);
}
template <> __device__ __forceinline__ double lt_recip<double>(double x) { return 1.0 / x; }

// running sum: compensated (hi, lo) in FP32 mode, plain double in FP64 mode
template <typename T> struct LtSum;
template <> struct LtSum<float> {
  CompF c{0.f, 0.f};
  __device__ __forceinline__ void add(float x) { c.add(x); }
  __device__ __forceinline__ double get() const { return c.value(); }
};
template <> struct LtSum<double> {
  double c = 0.0;
  __device__ __forceinline__ void add(double x) { c += x; }
  __device__ __forceinline__ double get() const { return c; }
};

__device__ __forceinline__ bool lt_finite(double x) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

}  // namespace

// kE = false: a launch whose items never ask for energies (compiled without the energy terms).
// Work item: PItem.begin = block index bx + nb (by + nb bz), nb = ceil(nc / 2); smax = staged slots
// available (the block's 4^3 region cells plus the padding slot); more raises ERR_STAGE_CAP.
template <typename T, bool kE>
__global__ void __launch_bounds__(kLjtThreads, kLjtMinBlocks)
    k_lj_tile(const SysDev* __restrict__ sys, const PItem* __restrict__ items, int smax) {
  pdl_wait();
  using T4 = typename V4<T>::type;
  extern __shared__ __align__(128) unsigned char lt_raw[];
  T4* sp = reinterpret_cast<T4*>(lt_raw);
  __shared__ int s_beg[65], s_c0[64];  // staging offset and first sorted index of each region cell
  __shared__ int s_tbl[8 * 64];        // (own cell, entry code) -> staged slot - sorted index
  __shared__ int s_own[9], s_ownr[8];  // own cells: prefix of particle counts, region cell
  __shared__ __align__(8) unsigned long long s_bar;
  __shared__ double red_u[kLjtThreads / 32], red_w[kLjtThreads / 32];
  const PItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  const int mode = item_mode(S, it.mode);
  if (mode & M_SKIP) return;  // block-uniform
  const bool energy = kE && (mode & M_ENERGY) != 0;
  const int nc = S.nc, nb = (nc + 1) >> 1, n = S.n;
  const int bx = it.begin % nb, by = (it.begin / nb) % nb, bz = it.begin / (nb * nb);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T4* __restrict__ P = reinterpret_cast<const T4*>(S.pos[it.buf]);
  // region cell r = rx + 4 ry + 16 rz sits at cell coordinates 2 b - 1 + r per axis (periodic)
  if (warp == 0) {
    int c0v[2], cnt[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int r = 2 * lane + q;
      int g[3] = {2 * bx - 1 + (r & 3), 2 * by - 1 + ((r >> 2) & 3), 2 * bz - 1 + (r >> 4)};
#pragma unroll
      for (int a = 0; a < 3; ++a) g[a] = g[a] < 0 ? g[a] + nc : (g[a] >= nc ? g[a] - nc : g[a]);
      const int c = (g[2] * nc + g[1]) * nc + g[0];
      c0v[q] = S.cell_start[c];
      cnt[q] = S.cell_start[c + 1] - c0v[q];
    }
    const int local = cnt[0] + cnt[1];
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    s_beg[2 * lane] = incl - local;
    s_beg[2 * lane + 1] = incl - local + cnt[0];
    s_c0[2 * lane] = c0v[0];
    s_c0[2 * lane + 1] = c0v[1];
    if (lane == 31) s_beg[64] = incl;
  }
  __syncthreads();
  const int total = s_beg[64];
  if (total + 1 > smax) {  // block-uniform
    if (tid == 0) {
      atomicOr(&S.flags[FLG_ERR], ERR_STAGE_CAP);
      atomicMax(&S.flags[FLG_LJSTAGE], total + 1);
    }
    return;
  }
  if (warp == 0) {
    // own cells o = ox + 2 oy + 4 oz at region (1 + ox, 1 + oy, 1 + oz); those beyond the grid are empty
    int cnt = 0, r = 0;
    if (lane < 8) {
      const int ox = lane & 1, oy = (lane >> 1) & 1, oz = lane >> 2;
      r = (1 + ox) + 4 * (1 + oy) + 16 * (1 + oz);
      if (2 * bx + ox < nc && 2 * by + oy < nc && 2 * bz + oz < nc) cnt = s_beg[r + 1] - s_beg[r];
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane < 8) {
      s_own[lane] = incl - cnt;
      s_ownr[lane] = r;
    }
    if (lane == 7) s_own[8] = incl;
    // bulk copies of the region cells' cell-local positions: one arrival announcing every byte, then
    // one copy per non-empty cell (sorted ranges of 16- or 32-byte records: aligned, whole records)
    if (lane == 0) {
      lt_bar_init(&s_bar);
      lt_bar_expect(&s_bar, (unsigned)total * (unsigned)sizeof(T4) + (unsigned)S.lj_tx_extra);
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int rr = 2 * lane + q;
      const int c = s_beg[rr + 1] - s_beg[rr];
      if (c > 0) lt_bulk(sp + s_beg[rr], P + s_c0[rr], (unsigned)c * (unsigned)sizeof(T4), &s_bar);
    }
  } else if (tid == 32) {
    T4 far;
    far.x = far.y = far.z = (T)1e3;
    far.w = (T)0;
    sp[total] = far;  // target of padding entries
  }
  for (int e = tid; e < 8 * 64; e += kLjtThreads) {
    const int o = e >> 6, code = e & 63;
    const int cx = code & 3, cy = (code >> 2) & 3, cz = code >> 4;
    int v = total;  // padding (entry index 0, code 63): the far slot
    if (cx < 3 && cy < 3 && cz < 3) {
      const int r = ((o & 1) + cx) + 4 * (((o >> 1) & 1) + cy) + 16 * ((o >> 2) + cz);
      v = s_beg[r] - s_c0[r];
    }
    s_tbl[e] = v;
  }
  __syncthreads();  // barrier initialised, tables written
  // every thread waits for the copies; the outcome is made uniform before anyone returns
  const bool ok = __syncthreads_and(lt_bar_wait(&s_bar) ? 1 : 0) != 0;
  if (!ok) {
    if (tid == 0) {
      atomicOr(&S.flags[FLG_ERR], ERR_TIMEOUT);
      lt_bar_wait(&s_bar);  // give copies still in flight a second bounded wait before the CTA exits
    }
    return;
  }
  // shift every region cell into the block's frame (cell centre - block centre, rounded once)
  for (int r = warp; r < 64; r += kLjtThreads / 32) {
    const T ox = (T)(((r & 3) - 1.5) * S.edge), oy = (T)((((r >> 2) & 3) - 1.5) * S.edge),
            oz = (T)(((r >> 4) - 1.5) * S.edge);
    for (int s = s_beg[r] + lane; s < s_beg[r + 1]; s += 32) {
      T4 h = sp[s];
      h.x += ox;
      h.y += oy;
      h.z += oz;
      sp[s] = h;
    }
  }
  __syncthreads();
  const T rcsq = Par<T>::rc2sq(S), g2 = Par<T>::guard2(S);
  const T lo = rcsq - g2;
  const T sig2 = Par<T>::sig2(S);
  const T eps24 = Par<T>::eps24(S), eps4 = Par<T>::eps4(S);
  const double* __restrict__ X = S.X[it.buf];
  const unsigned far_slot = (unsigned)total;
  LtSum<T> ud, wd;  // this thread's energy and virial sums
  const int nown = s_own[8];
  for (int t = tid; t < nown; t += kLjtThreads) {
    int o = 0;
    while (o < 7 && s_own[o + 1] <= t) ++o;
    const int r = s_ownr[o], k = t - s_own[o];
    const int i = s_c0[r] + k;
    const T4 pi = sp[s_beg[r] + k];
    const int* __restrict__ tb = s_tbl + 64 * o;
    // staged slot of an entry (clamped to the staged range: a stale entry cannot leave shared memory)
    auto slot_of = [&](unsigned e) { return min((unsigned)((int)(e & kNbrMask) + tb[e >> kNbrShift]), far_slot); };
    const int cnt = S.nbr_cnt[i];
    const int4* __restrict__ row4 = reinterpret_cast<const int4*>(S.nbr + nbr_slot(S.maxnb, i, 0));
    const int4 pad = make_int4(kNbrPad, kNbrPad, kNbrPad, kNbrPad);
    auto entries = [&](int t0) {
      int4 e = t0 < cnt ? __ldg(row4 + (t0 >> 2)) : pad;
      if (t0 + 1 >= cnt) e.y = pad.y;
      if (t0 + 2 >= cnt) e.z = pad.z;
      if (t0 + 3 >= cnt) e.w = pad.w;
      return e;
    };
    LtSum<T> fx, fy, fz;
    T uu = 0, ww = 0;          // energy and virial of the current eight pair terms
    T bmin = (T)1e30;          // smallest |r^2 - r_c^2| met: the guard band is checked once at the end
    T px = 0, py = 0, pz = 0;  // plain sum of the previous group of four
    bool odd = false;
    int4 ea = entries(0), eb = entries(4);
    for (int t0 = 0; t0 < cnt; t0 += 4) {
      const int4 ec = entries(t0 + 8);  // row entries two groups ahead
      const unsigned e[4] = {(unsigned)ea.x, (unsigned)ea.y, (unsigned)ea.z, (unsigned)ea.w};
      T4 pj[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) pj[u] = sp[slot_of(e[u])];
      T sx = 0, sy = 0, sz = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const T dx = pj[u].x - pi.x, dy = pj[u].y - pi.y, dz = pj[u].z - pi.z;
        const T r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        bmin = fmin(bmin, fabs(r2 - rcsq));
        const T ir2 = lt_recip<T>(r2);
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
      if (odd || t0 + 4 >= cnt) {
        fx.add(sx + px);
        fy.add(sy + py);
        fz.add(sz + pz);
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
    }
    if (bmin < g2) {
      // Rare: pairs whose r^2 fell in the guard band around r_c2^2 (left out above) are decided in FP64
      // with the CPU definition's operation order; the ones inside the cutoff are added.
      const int* __restrict__ row = S.nbr + nbr_slot(S.maxnb, i, 0);
      for (int q = 0; q < cnt; ++q) {
        const unsigned e = (unsigned)row[q];
        const T4 pj = sp[slot_of(e)];
        const T dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
        const T r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        if (!(r2 > lo && r2 < rcsq + g2)) continue;
        atomicAdd(&S.ctr[CTR_GUARD], 1ull);
        if (!exact_within(X, n, i, (int)(e & kNbrMask), S.L, S.rc2sq)) continue;
        const T ir2 = lt_recip<T>(r2);
        const T sr2 = sig2 * ir2;
        const T sr6 = sr2 * sr2 * sr2;
        const T sr12 = sr6 * sr6;
        const T g = eps24 * (sr12 + sr12 - sr6) * ir2;
        fx.add(-g * dx);
        fy.add(-g * dy);
        fz.add(-g * dz);
        if (energy) {
          ud.add(eps4 * (sr12 - sr6));
          wd.add(g * r2);
        }
      }
    }
    const double F[3] = {fx.get(), fy.get(), fz.get()};
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      S.f2[a * n + i] = F[a];
      bad |= !lt_finite(F[a]);
    }
    if (bad) atomicOr(&S.flags[FLG_ERR], ERR_NONFINITE);
  }
  if (energy) {  // every pair appears in both members' lists: halve
    const double us = warp_sum(ud.get()), ws = warp_sum(wd.get());
    if (lane == 0) {
      red_u[warp] = us;
      red_w[warp] = ws;
    }
    __syncthreads();
    if (tid == 0) {
      double ut = 0.0, wt = 0.0;
#pragma unroll
      for (int q = 0; q < kLjtThreads / 32; ++q) {
        ut += red_u[q];
        wt += red_w[q];
      }
      atomicAdd(&S.acc[ACC_U2], 0.5 * ut);
      atomicAdd(&S.acc[ACC_W2], 0.5 * wt);
    }
  }
}

template <typename T>
void launch_lj_tile(const Launch& L, const PItem* items, int nitems, bool energy, int smax) {
  if (nitems <= 0) return;
  const size_t bytes = (size_t)smax * sizeof(typename V4<T>::type);
  if (energy)
    launch_kernel(L, k_lj_tile<T, true>, nitems, kLjtThreads, bytes, L.sys, items, smax);
  else
    launch_kernel(L, k_lj_tile<T, false>, nitems, kLjtThreads, bytes, L.sys, items, smax);
}
// the kernels' dynamic shared-memory limit is shared by every system on a device: only ever raised
int lj_tile_configure(int smax, int precision) {
  const int bytes = smax * (precision ? (int)sizeof(double4_32a) : (int)sizeof(float4));
  const void* kerns[2][2] = {{(const void*)k_lj_tile<float, false>, (const void*)k_lj_tile<float, true>},
                             {(const void*)k_lj_tile<double, false>, (const void*)k_lj_tile<double, true>}};
  for (const void* k : kerns[precision ? 1 : 0])
    if (!raise_smem_attr(k, bytes)) return -1;
  return bytes;
}
template void launch_lj_tile<float>(const Launch&, const PItem*, int, bool, int);
template void launch_lj_tile<double>(const Launch&, const PItem*, int, bool, int);

// ============================================================== team LJ kernel
// kTeam adjacent lanes per particle i: lane h of the team takes the entries h, h + kTeam, ... of i's
// pair-list row (the team reads consecutive entries together: one sector per team and step) and gathers
// their positions from global memory; no software pipeline, the latency is hidden by occupancy (a warp
// holds 32 / kTeam particles, so kTeam times as many warps are resident as with one thread per
// particle).  Each lane adds its plain sums of at most eight pair forces to a compensated (hi, lo)
// pair by TwoSum; the team's pairs are combined by a TwoSum butterfly (the error stays that of the
// compensated sums), and the first lane of the team writes hi + lo in FP64.
namespace {
__device__ __forceinline__ void lt_team_add(CompF& c, unsigned mask, int o) {
  const float h = __shfl_xor_sync(mask, c.hi, o), l = __shfl_xor_sync(mask, c.lo, o);
  float s, e;
  two_sum(c.hi, h, s, e);
  c.hi = s;
  c.lo = __fadd_rn(__fadd_rn(c.lo, l), e);
}
__device__ __forceinline__ void lt_team_add(double& c, unsigned mask, int o) { c += __shfl_xor_sync(mask, c, o); }
template <typename T> struct LtAcc;
template <> struct LtAcc<float> {
  CompF c{0.f, 0.f};
  __device__ __forceinline__ void add(float x) { c.add(x); }
  __device__ __forceinline__ void team(unsigned mask, int o) { lt_team_add(c, mask, o); }
  __device__ __forceinline__ double get() const { return c.value(); }
};
template <> struct LtAcc<double> {
  double c = 0.0;
  __device__ __forceinline__ void add(double x) { c += x; }
  __device__ __forceinline__ void team(unsigned mask, int o) { lt_team_add(c, mask, o); }
  __device__ __forceinline__ double get() const { return c; }
};
__device__ __forceinline__ float4 lt_ldg4(const float4* p) { return __ldg(p); }
__device__ __forceinline__ double4_32a lt_ldg4(const double4_32a* p) { return *p; }
}  // namespace

// items: PItem.begin = first particle of the block (kLjmThreads / kTeam particles per block)
template <typename T, bool kE, int kTeam>
__global__ void __launch_bounds__(kLjmThreads, kLjmMinBlocks) k_lj_team(const SysDev* __restrict__ sys, const PItem* __restrict__ items) {
  static_assert(kTeam == 4 || kTeam == 8 || kTeam == 16, "team of 4, 8 or 16 lanes");
  using T4 = typename V4<T>::type;
  __shared__ T4 s_off[64];
  __shared__ double red_u[kLjmThreads / 32], red_w[kLjmThreads / 32];
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
  if (mode & M_SKIP) return;  // block-uniform
  const bool energy = kE && (mode & M_ENERGY) != 0;
  for (unsigned c = threadIdx.x; c < 64u; c += kLjmThreads) {
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
  const int n = S.n, lane = threadIdx.x & 31;
  const int h = lane % kTeam;
  const unsigned tmask = (kTeam == 32 ? 0xffffffffu : ((1u << kTeam) - 1u)) << (lane - h);
  const int i = it.begin + (int)threadIdx.x / kTeam;
  const bool active = i < n;  // team-uniform
  const T4* __restrict__ P = reinterpret_cast<const T4*>(S.pos[it.buf]);
  LtAcc<T> fx, fy, fz;
  LtSum<T> ud, wd;
  if (active) {
    const T4 pi = P[i];
    const T rcsq = Par<T>::rc2sq(S), g2 = Par<T>::guard2(S);
    const T lo = rcsq - g2;
    const T sig2 = Par<T>::sig2(S);
    const T eps24 = Par<T>::eps24(S), eps4 = Par<T>::eps4(S);
    const T edge = Par<T>::edge(S);
    const int cnt = S.nbr_cnt[i];
    const int* __restrict__ row = S.nbr + nbr_slot(S.maxnb, i, 0);
    T bmin = (T)1e30;
    T sx = 0, sy = 0, sz = 0, uu = 0, ww = 0;
    int m = 0;  // terms in the plain sums
    for (int t = h; t < cnt; t += kTeam) {
      const unsigned e = (unsigned)__ldg(row + t);
      const T4 pj = lt_ldg4(P + (e & kNbrMask));
      T dx, dy, dz;
      if (R3B_LJ_ARITH_OFF && sizeof(T) == 4) {  // padding (code 63): two edges per axis, beyond r_c
        const unsigned cd = e >> kNbrShift;
        dx = fma((T)off_unit(cd & 3u), edge, pj.x - pi.x);
        dy = fma((T)off_unit((cd >> 2) & 3u), edge, pj.y - pi.y);
        dz = fma((T)off_unit(cd >> 4), edge, pj.z - pi.z);
      } else {
        const T4 o = s_off[e >> kNbrShift];
        dx = (pj.x - pi.x) + o.x;
        dy = (pj.y - pi.y) + o.y;
        dz = (pj.z - pi.z) + o.z;
      }
      const T r2 = fma(dz, dz, fma(dy, dy, dx * dx));
      bmin = fmin(bmin, fabs(r2 - rcsq));
      const T ir2 = lt_recip<T>(r2);
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
      if (++m == 8) {
        fx.add(sx);
        fy.add(sy);
        fz.add(sz);
        sx = sy = sz = (T)0;
        if (energy) {
          ud.add(uu);
          wd.add(ww);
          uu = ww = (T)0;
        }
        m = 0;
      }
    }
    fx.add(sx);
    fy.add(sy);
    fz.add(sz);
    if (energy) {
      ud.add(uu);
      wd.add(ww);
    }
    if (bmin < g2) {
      // Rare: this lane's pairs whose r^2 fell in the guard band around r_c2^2 (left out above) are
      // decided in FP64 with the CPU definition's operation order; the ones inside the cutoff are added.
      const double* __restrict__ X = S.X[it.buf];
      for (int t = h; t < cnt; t += kTeam) {
        const unsigned e = (unsigned)row[t];
        const int j = (int)(e & kNbrMask);
        const T4 pj = P[j];
        const T4 o = s_off[e >> kNbrShift];
        const T dx = (pj.x - pi.x) + o.x, dy = (pj.y - pi.y) + o.y, dz = (pj.z - pi.z) + o.z;
        const T r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        if (!(r2 > lo && r2 < rcsq + g2)) continue;
        atomicAdd(&S.ctr[CTR_GUARD], 1ull);
        if (!exact_within(X, n, i, j, S.L, S.rc2sq)) continue;
        const T ir2 = lt_recip<T>(r2);
        const T sr2 = sig2 * ir2;
        const T sr6 = sr2 * sr2 * sr2;
        const T sr12 = sr6 * sr6;
        const T g = eps24 * (sr12 + sr12 - sr6) * ir2;
        fx.add(-g * dx);
        fy.add(-g * dy);
        fz.add(-g * dz);
        if (energy) {
          ud.add(eps4 * (sr12 - sr6));
          wd.add(g * r2);
        }
      }
    }
#pragma unroll
    for (int o = kTeam / 2; o > 0; o >>= 1) {
      fx.team(tmask, o);
      fy.team(tmask, o);
      fz.team(tmask, o);
    }
    if (h == 0) {
      const double F[3] = {fx.get(), fy.get(), fz.get()};
      bool bad = false;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        S.f2[a * n + i] = F[a];
        bad |= !lt_finite(F[a]);
      }
      if (bad) atomicOr(&S.flags[FLG_ERR], ERR_NONFINITE);
    }
  }
  if (energy) {  // every pair appears in both members' lists: halve
    const int warp = threadIdx.x >> 5;
    const double us = warp_sum(ud.get()), ws = warp_sum(wd.get());
    if (lane == 0) {
      red_u[warp] = us;
      red_w[warp] = ws;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double ut = 0.0, wt = 0.0;
#pragma unroll
      for (int q = 0; q < kLjmThreads / 32; ++q) {
        ut += red_u[q];
        wt += red_w[q];
      }
      atomicAdd(&S.acc[ACC_U2], 0.5 * ut);
      atomicAdd(&S.acc[ACC_W2], 0.5 * wt);
    }
  }
}

template <typename T, int kTeam>
static void launch_lj_team_t(const Launch& L, const PItem* items, int nitems, bool energy) {
  if (energy)
    launch_kernel(L, k_lj_team<T, true, kTeam>, nitems, kLjmThreads, 0, L.sys, items);
  else
    launch_kernel(L, k_lj_team<T, false, kTeam>, nitems, kLjmThreads, 0, L.sys, items);
}
template <typename T>
void launch_lj_team(const Launch& L, const PItem* items, int nitems, bool energy, int team) {
  if (nitems <= 0) return;
  if (team == 4)
    launch_lj_team_t<T, 4>(L, items, nitems, energy);
  else if (team == 16)
    launch_lj_team_t<T, 16>(L, items, nitems, energy);
  else
    launch_lj_team_t<T, 8>(L, items, nitems, energy);
}
template void launch_lj_team<float>(const Launch&, const PItem*, int, bool, int);
template void launch_lj_team<double>(const Launch&, const PItem*, int, bool, int);

}  // namespace r3b
