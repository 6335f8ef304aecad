// Rotation triplet kernel: Axilrod-Teller-Muto forces (Sec. 2.1) with the triplet cutoff "all three
// distances <= r_c" (Fig. 2 caption, Sec. 4.2.2), every triplet evaluated once (Newton 3, the
// future-work traversal of Sec. 5).
//
// Ownership.  A triplet belongs to its lowest member in the order "z coordinate of the last binning in
// fixed point, then sorted index".  Displacements come from wrapping 32-bit differences of those
// fixed-point positions, so the order is exactly antisymmetric and transitive on every triangle of
// particles within r_c of each other (L > 3 r_c): each triplet has exactly one owner.  The owner i
// sees the other two in its half list {j : r_ij <= r_c3, j above i}, about half of its neighbours
// (a half ball, so the list length varies little from particle to particle).
//
// Rotation.  One warp per base particle i.  Lane v holds half-list node v (displacement d_v = x_v - x_i
// and a_v = |d_v|^2).  In step s, lane v pairs node v with node (v + s) mod m; steps 1 .. (m - 1) / 2
// (plus s = m / 2 on lanes v < m / 2 for even m) visit every unordered pair of nodes exactly once, and
// within a step every node is the partner of exactly one lane.  Lists of 33 .. 64 nodes are split into
// halves A and B: rotation within A, within B, and a cross rotation pairing A_v with B_(v + s) mod |A|
// (B padded to |A| with far-away dummies).
//
// Forces as edge weights.  With a = |d_j|^2, b = |d_k|^2, c = |e|^2, e = d_k - d_j, and
// pa2 = 2 dphi/da, pb2 = 2 dphi/db, pc2 = 2 dphi/dc:
//   F_i = pa2 d_j + pb2 d_k,  F_j = -pa2 d_j + pc2 e,  F_k = -pb2 d_k - pc2 e.
// Node v collects a scalar W_v (its i-edge weights) and a vector G_v (its j-k edge forces); then
// F_v = G_v - W_v d_v and F_i = sum_v W_v d_v.  The lane of node j keeps j's share in registers; the
// partner's share goes to the partner's shared-memory slot (the rotation makes those writes distinct).
// Per-(base, node) totals are added to the node's force with one vector atomic; the combine kernel
// reads and clears the sums.
//
// Squared-distance algebra (law of cosines; w = 1/(abc), u = w^(1/2), A = a + b - c, B = a - b + c,
// C = -a + b + c, P = ABC = 8 abc cos(g_i) cos(g_j) cos(g_k)):
//   phi = nu u^3 (1 + 3/8 P w),  2 dphi/da = 3/4 nu u^5 (dP/da - bc (4 + 5/2 P w))  (b, c alike),
//   dP/da = 2a C - AB,  dP/db = 2b B - AC,  dP/dc = 2c A - BC.
// The factors 3/4 nu (forces) and nu (energy) are applied once per node, not per pair.
//
// Cutoff decisions.  FP32 decisions are taken on r^2; a pair whose r^2 lies within the guard band
// around r_c^2 is re-decided in FP64 from the FP64 positions with the CPU definition's operation
// order (exact_within).  Pair tests inside the rotation run in FP32 first; a phase that met the band
// is discarded and repeated with exact decisions.
#include "md_internal.cuh"

namespace r3b {

constexpr int kZrMax = 64;    // half-list capacity: two rotation groups of at most 32 nodes
constexpr int kZrWarps = 8;   // warps per CTA
constexpr int kZrPer = 4;     // consecutive bases per warp in one work item
static_assert(kZrWarps * kZrPer == rot_bases_per_item(0), "work items and kernel disagree");

// FP32 reciprocal square root: the hardware approximation (flush-to-zero form; the argument is a
// product of three squared distances, never subnormal) refined by one Newton-Raphson step
__device__ __forceinline__ float zr_rsqrt(float q) {
  float t;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(q));
  return t * fmaf(-0.5f * q, t * t, 1.5f);
}
__device__ __forceinline__ double zr_rsqrt(double q) { return 1.0 / sqrt(q); }

template <typename T>
struct ZrSmem {
  using T4 = typename V4<T>::type;
  T4 nd[kZrMax];          // half list: (d_v, |d_v|^2)
  T4 pn[kZrMax];          // partners of the current phase, doubled (pn[t + m] = pn[t]), far dummies after
  T4 slot[2][kZrMax];     // partner shares (G, W) of odd and even steps, in pn's index space
  T4 tot[kZrMax];         // per-node totals across phases (lists longer than 32)
  int nidx[kZrMax];       // sorted index of each node
  int pidx[kZrMax];       // sorted index of each partner entry (exact repeats)
};
template <typename T>
constexpr size_t zr_smem_bytes() {
  return sizeof(ZrSmem<T>) * kZrWarps;
}

// Far-away dummies: own nodes of lanes without a node sit at +1e3, padding partners at -1e3, so
// every pair involving a dummy is rejected by the cutoff while all intermediates stay finite (no
// pair of dummies coincides).
template <typename T>
__device__ __forceinline__ typename V4<T>::type zr_far(T sgn) {
  typename V4<T>::type f;
  f.x = f.y = f.z = sgn * (T)1e3;
  f.w = (T)3e6;
  return f;
}
template <typename T>
__device__ __forceinline__ typename V4<T>::type zr_zero() {
  typename V4<T>::type f;
  f.x = f.y = f.z = f.w = (T)0;
  return f;
}

// Per-lane running sums of one base (or one phase).
template <typename T>
struct ZrAcc {
  T W, Gx, Gy, Gz;  // own node
  T cnt, u;         // accepted pairs, energy / nu
  T dmin;           // smallest |c - r_c^2| met (FP32 decisions)
};

// One phase: own node J of this lane (J.w = |d_J|^2; far dummy for lanes without a node), partners in
// w.pn / w.pidx.  Full steps s_lo .. s_hi for every lane; then, if half > 0, step `half` for lanes
// v < half only.  Slots must be zero on entry.
template <typename T, bool kE, bool kExact>
__device__ __forceinline__ void zr_steps(const SysDev& S, const double* __restrict__ X, ZrSmem<T>& w,
                                         const typename V4<T>::type J, const int jid, const int s_lo,
                                         const int s_hi, const int half, const int lane, ZrAcc<T>& A) {
  using T4 = typename V4<T>::type;
  const T rcsq = Par<T>::rc3sq(S), g = Par<T>::guard3(S);
  const T a = J.w, a2 = J.w + J.w;
  auto step = [&](const int s, const int par, const T off) {
    const T4 pk = w.pn[lane + s];
    const T ex = pk.x - J.x, ey = pk.y - J.y, ez = pk.z - J.z;
    const T c = fma(ez, ez, fma(ey, ey, ex * ex)) + off;
    const T t = c - rcsq;
    T okf;
    if constexpr (kExact) {
      bool ok = t <= g;
      const bool band = ok && t >= -g;
      if (__any_sync(0xffffffffu, band)) {
        if (band) {
          atomicAdd(&S.ctr[CTR_GUARD], 1ull);
          ok = exact_within(X, S.n, jid, w.pidx[lane + s], S.L, S.rc3sq);
        }
      }
      okf = ok ? (T)1 : (T)0;
    } else {
      okf = (t <= g) ? (T)1 : (T)0;
      A.dmin = fmin(A.dmin, fabs(t));
    }
    const T b = pk.w;
    const T ab = a * b;
    const T u = zr_rsqrt(ab * c);
    const T ww = u * u;
    const T t3 = ww * u;
    const T t5 = t3 * ww;
    const T sum = (a + b) + c;
    const T Aa = fma((T)-2, c, sum);  // a + b - c
    const T Bb = fma((T)-2, b, sum);  // a - b + c
    const T Cc = fma((T)-2, a, sum);  // -a + b + c
    const T AB = Aa * Bb, AC = Aa * Cc, BC = Bb * Cc;
    const T P = AB * Cc;
    const T Pa = fma(a2, Cc, -AB);
    const T Pb = fma(b + b, Bb, -AC);
    const T Pc = fma(c + c, Aa, -BC);
    const T Pw = P * ww;
    const T H = fma((T)2.5, Pw, (T)4);
    const T kk = t5 * okf;
    const T pa2 = kk * fma(-(b * c), H, Pa);
    const T pb2 = kk * fma(-(a * c), H, Pb);
    const T pc2 = kk * fma(-ab, H, Pc);
    A.cnt += okf;
    if constexpr (kE) A.u = fma(t3 * okf, fma((T)0.375, Pw, (T)1), A.u);
    A.W += pa2;
    A.Gx = fma(pc2, ex, A.Gx);
    A.Gy = fma(pc2, ey, A.Gy);
    A.Gz = fma(pc2, ez, A.Gz);
    T4* const sl = &w.slot[par][lane + s];
    T4 q = *sl;
    q.x = fma(-pc2, ex, q.x);
    q.y = fma(-pc2, ey, q.y);
    q.z = fma(-pc2, ez, q.z);
    q.w += pb2;
    *sl = q;
  };
  // two steps per warp barrier: consecutive steps write different slot arrays, steps two apart
  // may write one slot from different lanes
  int s = s_lo;
#pragma unroll 1
  for (; s + 1 <= s_hi; s += 2) {
    step(s, 0, (T)0);
    step(s + 1, 1, (T)0);
    __syncwarp();
  }
  if (s <= s_hi) {
    step(s, 0, (T)0);
    __syncwarp();
  }
  if (half > 0) {
    step(half, 1, lane < half ? (T)0 : (T)1e6);
    __syncwarp();
  }
}

// zero both slot arrays
template <typename T>
__device__ __forceinline__ void zr_clear_slots(ZrSmem<T>& w, int lane) {
  w.slot[0][lane] = zr_zero<T>();
  w.slot[0][lane + 32] = zr_zero<T>();
  w.slot[1][lane] = zr_zero<T>();
  w.slot[1][lane + 32] = zr_zero<T>();
}

// Partner layout of a self rotation over nodes first .. first + mx - 1 (mx <= 32): doubled, then far.
template <typename T>
__device__ __forceinline__ void zr_layout_self(ZrSmem<T>& w, int first, int mx, int lane) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = lane + 32 * h;
    const int v = t < mx ? t : t - mx;
    const bool real = t < 2 * mx;
    w.pn[t] = real ? w.nd[first + v] : zr_far<T>((T)-1);
    w.pidx[t] = real ? w.nidx[first + v] : 0;
  }
}
// Partner layout of a cross rotation: nodes first .. first + mb - 1 padded to mp (mb <= mp <= 32),
// doubled, then far.
template <typename T>
__device__ __forceinline__ void zr_layout_cross(ZrSmem<T>& w, int first, int mb, int mp, int lane) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = lane + 32 * h;
    const int v = t < mp ? t : t - mp;
    const bool real = t < 2 * mp && v < mb;
    w.pn[t] = real ? w.nd[first + v] : zr_far<T>((T)-1);
    w.pidx[t] = real ? w.nidx[first + v] : 0;
  }
}

// Run one phase with FP32 decisions; if a pair met the guard band, discard and repeat it exactly.
// Returns the lane's own-node sums in A (cnt, u are added to the running totals in R).
template <typename T, bool kE>
__device__ __forceinline__ void zr_phase_exact(const SysDev& S, const double* __restrict__ X, ZrSmem<T>& w,
                                            const typename V4<T>::type J, const int jid, const int s_lo,
                                            const int s_hi, const int half, const int lane, ZrAcc<T>& A) {
  __syncwarp();
  zr_clear_slots<T>(w, lane);
  __syncwarp();
  A.W = A.Gx = A.Gy = A.Gz = A.cnt = A.u = (T)0;
  zr_steps<T, kE, true>(S, X, w, J, jid, s_lo, s_hi, half, lane, A);
}
template <typename T, bool kE>
__device__ __forceinline__ void zr_phase(const SysDev& S, const double* __restrict__ X, ZrSmem<T>& w,
                                         const typename V4<T>::type J, const int jid, const int s_lo,
                                         const int s_hi, const int half, const int lane, ZrAcc<T>& A) {
  A.W = A.Gx = A.Gy = A.Gz = A.cnt = A.u = (T)0;
  A.dmin = (T)1e30;
  zr_steps<T, kE, false>(S, X, w, J, jid, s_lo, s_hi, half, lane, A);
  if (__any_sync(0xffffffffu, A.dmin <= Par<T>::guard3(S))) zr_phase_exact<T, kE>(S, X, w, J, jid, s_lo, s_hi, half, lane, A);
}

// Displacement x_j - x_i in the kernel's precision.  FP32: wrapping fixed-point difference (exact
// minimum image), one rounding to FP32, one scaling.  FP64: cell-local coordinates plus cell offset.
__device__ __forceinline__ void zr_disp(const SysDev& S, int, const int4 qi, const int4 qj, unsigned, int, int,
                                        float& dx, float& dy, float& dz) {
  const float sc = S.f_qscale;
  dx = (float)(int)((unsigned)qj.x - (unsigned)qi.x) * sc;
  dy = (float)(int)((unsigned)qj.y - (unsigned)qi.y) * sc;
  dz = (float)(int)((unsigned)qj.z - (unsigned)qi.z) * sc;
}
__device__ __forceinline__ void zr_disp(const SysDev& S, int buf, const int4, const int4, unsigned code, int i,
                                        int j, double& dx, double& dy, double& dz) {
  const double4_32a* P = reinterpret_cast<const double4_32a*>(S.pos[buf]);
  const double4_32a pi = P[i], pj = P[j];
  const double ox = (double)(int)(code & 3u) - 1.0, oy = (double)(int)((code >> 2) & 3u) - 1.0,
               oz = (double)(int)(code >> 4) - 1.0;
  dx = (pj.x - pi.x) + ox * S.edge;
  dy = (pj.y - pi.y) + oy * S.edge;
  dz = (pj.z - pi.z) + oz * S.edge;
}

// Half list of base x into w.nd / w.nidx from its pair-list row; returns its length (entries beyond
// kZrMax are counted, not stored).
template <typename T>
__device__ __forceinline__ int zr_build(const SysDev& S, ZrSmem<T>& w, const int buf, const int x,
                                        const int lane) {
  using T4 = typename V4<T>::type;
  const unsigned lt = (1u << lane) - 1u;
  const unsigned* __restrict__ row = reinterpret_cast<const unsigned*>(S.nbr) + (size_t)x * S.maxnb;
  const int cnt = S.nbr_cnt[x];
  const int4 qi = S.ipos[x];
  const T rcsq = Par<T>::rc3sq(S), g = Par<T>::guard3(S);
  int m = 0;
  for (int t0 = 0; t0 < cnt; t0 += 32) {
    const int t = t0 + lane;
    const bool valid = t < cnt;
    const unsigned e = valid ? __ldg(row + t) : 0u;
    const int j = (int)(e & kNbrMask);
    const int4 qj = valid ? __ldg(S.ipos + j) : qi;
    const int dzq = (int)((unsigned)qj.z - (unsigned)qi.z);
    const bool above = valid && (dzq > 0 || (dzq == 0 && j > x));
    T dx = (T)0, dy = (T)0, dz = (T)0;
    if (above) zr_disp(S, buf, qi, qj, e >> kNbrShift, x, j, dx, dy, dz);
    const T r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    bool ok = above && r2 <= rcsq - g;
    const bool band = above && r2 > rcsq - g && r2 <= rcsq + g;
    if (__any_sync(0xffffffffu, band)) {
      if (band) {
        atomicAdd(&S.ctr[CTR_GUARD], 1ull);
        ok = exact_within(S.X[buf], S.n, x, j, S.L, S.rc3sq);
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, ok);
    const int pos = m + __popc(bal & lt);
    if (ok && pos < kZrMax) {
      T4 d4;
      d4.x = dx;
      d4.y = dy;
      d4.z = dz;
      d4.w = r2;
      w.nd[pos] = d4;
      w.nidx[pos] = j;
    }
    m += __popc(bal);
  }
  __syncwarp();
  return m;
}

// Warp sums of four per-lane values by a transposed butterfly (8 shuffles): afterwards lanes 0-7 hold
// the total of a, lanes 8-15 of b, 16-23 of c, 24-31 of d.
template <typename T>
__device__ __forceinline__ T zr_sum4(T a, T b, T c, T d, int lane) {
  const bool h16 = (lane & 16) != 0;
  T k0 = h16 ? c : a, k1 = h16 ? d : b;
  const T s0 = h16 ? a : c, s1 = h16 ? b : d;
  k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
  k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
  const bool h8 = (lane & 8) != 0;
  T k = h8 ? k1 : k0;
  const T sk = h8 ? k0 : k1;
  k += __shfl_xor_sync(0xffffffffu, sk, 8);
  k += __shfl_xor_sync(0xffffffffu, k, 4);
  k += __shfl_xor_sync(0xffffffffu, k, 2);
  k += __shfl_xor_sync(0xffffffffu, k, 1);
  return k;
}

template <typename T>
__device__ __forceinline__ void zr_atomic_add(void* f3acc, int j, T fx, T fy, T fz) {
  if constexpr (sizeof(T) == 4) {
    atomicAdd(reinterpret_cast<float4*>(f3acc) + j, make_float4(fx, fy, fz, 0.f));
  } else {
    double* q = reinterpret_cast<double*>(f3acc) + 4 * (size_t)j;
    atomicAdd(q, fx);
    atomicAdd(q + 1, fy);
    atomicAdd(q + 2, fz);
  }
}

// node v's final force (scaled by 3/4 nu) to its accumulator; returns W_v d_v (unscaled) for F_i
template <typename T>
__device__ __forceinline__ void zr_emit(const SysDev& S, const typename V4<T>::type d, int j, T W, T Gx, T Gy, T Gz,
                                        T fs, T& fix, T& fiy, T& fiz) {
  fix = fma(W, d.x, fix);
  fiy = fma(W, d.y, fiy);
  fiz = fma(W, d.z, fiz);
  zr_atomic_add<T>(S.f3acc, j, fs * fma(-W, d.x, Gx), fs * fma(-W, d.y, Gy), fs * fma(-W, d.z, Gz));
}

template <typename T>
__device__ __forceinline__ typename V4<T>::type zr_add4(typename V4<T>::type p, typename V4<T>::type q) {
  p.x += q.x;
  p.y += q.y;
  p.z += q.z;
  p.w += q.w;
  return p;
}

// All triplets owned by base x.  Adds forces to S.f3acc; returns (in lane-summed form) count and energy.
template <typename T, bool kE>
__device__ __forceinline__ void zr_base(const SysDev& S, ZrSmem<T>& w, const int buf, const int x, const int lane,
                                        T& cnt_sum, T& u_sum) {
  using T4 = typename V4<T>::type;
  const double* __restrict__ X = S.X[buf];
  const int m_all = zr_build<T>(S, w, buf, x, lane);
  if (m_all > kZrMax) {
    if (lane == 0) atomicOr(&S.flags[FLG_ERR], ERR_HALF_CAP);
    return;
  }
  const int m = m_all;
  const T fs = (T)0.75 * Par<T>::nu(S);
  T fix = (T)0, fiy = (T)0, fiz = (T)0;
  ZrAcc<T> A;
  if (m <= 32) {
    if (m >= 2) {
      zr_clear_slots<T>(w, lane);
      zr_layout_self<T>(w, 0, m, lane);
      __syncwarp();
      const T4 J = lane < m ? w.nd[lane] : zr_far<T>((T)1);
      const int jid = lane < m ? w.nidx[lane] : 0;
      zr_phase<T, kE>(S, X, w, J, jid, 1, (m - 1) >> 1, (m & 1) ? 0 : (m >> 1), lane, A);
      cnt_sum += A.cnt;
      if (kE) u_sum += A.u;
      if (lane < m) {
        const T4 s = zr_add4<T>(zr_add4<T>(w.slot[0][lane], w.slot[1][lane]),
                                zr_add4<T>(w.slot[0][lane + m], w.slot[1][lane + m]));
        zr_emit<T>(S, J, jid, A.W + s.w, A.Gx + s.x, A.Gy + s.y, A.Gz + s.z, fs, fix, fiy, fiz);
      }
    }
  } else {
    // halves A = nodes 0 .. ma-1, B = nodes ma .. m-1 (mb <= ma <= 32)
    const int ma = (m + 1) >> 1, mb = m - ma;
    w.tot[lane] = zr_zero<T>();
    w.tot[lane + 32] = zr_zero<T>();
    // phase 1: within A; phase 2: within B; phase 3: A x B
#pragma unroll 1
    for (int ph = 0; ph < 3; ++ph) {
      __syncwarp();
      zr_clear_slots<T>(w, lane);
      if (ph == 0) zr_layout_self<T>(w, 0, ma, lane);
      else if (ph == 1) zr_layout_self<T>(w, ma, mb, lane);
      else zr_layout_cross<T>(w, ma, mb, ma, lane);
      __syncwarp();
      const int own_first = ph == 1 ? ma : 0, own_n = ph == 1 ? mb : ma;
      const T4 J = lane < own_n ? w.nd[own_first + lane] : zr_far<T>((T)1);
      const int jid = lane < own_n ? w.nidx[own_first + lane] : 0;
      const int mx = ph == 0 ? ma : mb;
      if (ph < 2)
        zr_phase<T, kE>(S, X, w, J, jid, 1, (mx - 1) >> 1, (mx & 1) ? 0 : (mx >> 1), lane, A);
      else
        zr_phase<T, kE>(S, X, w, J, jid, 0, ma - 1, 0, lane, A);
      cnt_sum += A.cnt;
      if (kE) u_sum += A.u;
      // own-node sums and partner slots into the per-node totals
      const int par_first = ph == 0 ? 0 : ma, par_n = ph == 0 ? ma : mb, par_period = ph == 2 ? ma : par_n;
      if (lane < own_n) {
        T4 o;
        o.x = A.Gx;
        o.y = A.Gy;
        o.z = A.Gz;
        o.w = A.W;
        w.tot[own_first + lane] = zr_add4<T>(w.tot[own_first + lane], o);
      }
      __syncwarp();
      if (lane < par_n) {
        const T4 s = zr_add4<T>(zr_add4<T>(w.slot[0][lane], w.slot[1][lane]),
                                zr_add4<T>(w.slot[0][lane + par_period], w.slot[1][lane + par_period]));
        w.tot[par_first + lane] = zr_add4<T>(w.tot[par_first + lane], s);
      }
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int v = lane + 32 * h;
      if (v < m) {
        const T4 t = w.tot[v];
        zr_emit<T>(S, w.nd[v], w.nidx[v], t.w, t.x, t.y, t.z, fs, fix, fiy, fiz);
      }
    }
  }
  // F_i = sum_v W_v d_v (scaled): warp sum
  const T k = zr_sum4<T>(fix, fiy, fiz, (T)0, lane);
  const T Fx = k, Fy = __shfl_sync(0xffffffffu, k, 8), Fz = __shfl_sync(0xffffffffu, k, 16);
  if (lane == 0) zr_atomic_add<T>(S.f3acc, x, fs * Fx, fs * Fy, fs * Fz);
  __syncwarp();  // the next base reuses the warp's shared memory
}

// Work item: 32 consecutive bases, kZrPer per warp.  Counts and energy are summed per CTA and added
// to the system's totals with one atomic each.
template <typename T>
__global__ void __launch_bounds__(32 * kZrWarps, sizeof(T) == 4 ? 4 : 2)
    k_atm_rot(const SysDev* __restrict__ sys, const PItem* __restrict__ items) {
  extern __shared__ __align__(32) unsigned char zr_raw[];
  __shared__ double red_c[kZrWarps], red_u[kZrWarps];
  const PItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  const int imode = item_mode(S, it.mode);
  if (imode & M_SKIP) return;  // block-uniform
  const bool kE = (imode & M_ENERGY) != 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  ZrSmem<T>& w = reinterpret_cast<ZrSmem<T>*>(zr_raw)[warp];
  T cnt = (T)0, u = (T)0;
  for (int k = 0; k < kZrPer; ++k) {
    const int x = it.begin + warp * kZrPer + k;
    if (x >= S.n) break;  // warp-uniform
    if (kE)
      zr_base<T, true>(S, w, it.buf, x, lane, cnt, u);
    else
      zr_base<T, false>(S, w, it.buf, x, lane, cnt, u);
  }
  // per-lane counts are exact small integers in T; sum them in FP64
  double c = warp_sum((double)cnt);
  double uu = kE ? warp_sum((double)u) : 0.0;
  if (lane == 0) {
    red_c[warp] = c;
    red_u[warp] = uu;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ct = 0.0, ut = 0.0;
    for (int q = 0; q < kZrWarps; ++q) {
      ct += red_c[q];
      ut += red_u[q];
    }
    if (ct > 0.0) atomicAdd(&S.ctr[CTR_TRIPLETS], (unsigned long long)(ct + 0.5));
    if (kE) {
      const double U = S.nu * ut;
      atomicAdd(&S.acc[ACC_U3], U);
      atomicAdd(&S.acc[ACC_W3], 9.0 * U);  // sum_a r_a . F_a = 9 phi (phi is homogeneous of degree -9)
    }
  }
}

// dynamic shared memory above the 48 KB default: set once per process and kernel
template <typename T>
static bool zr_configure() {
  static int done = 0;
  if (!done) {
    done = cudaFuncSetAttribute(k_atm_rot<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)zr_smem_bytes<T>()) == cudaSuccess ? 1 : -1;
    if (done < 0) cudaGetLastError();
  }
  return done > 0;
}

template <typename T>
void launch_atm_rot(const Launch& L, const PItem* items, int nitems) {
  if (nitems > 0 && zr_configure<T>())
    k_atm_rot<T><<<nitems, 32 * kZrWarps, zr_smem_bytes<T>(), L.stream>>>(L.sys, items);
}
template void launch_atm_rot<float>(const Launch&, const PItem*, int);
template void launch_atm_rot<double>(const Launch&, const PItem*, int);

}  // namespace r3b
