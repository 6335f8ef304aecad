// Rotation triplet kernel: Axilrod-Teller-Muto forces (Sec. 2.1) with the triplet cutoff "all three
// distances <= r_c" (Fig. 2 caption, Sec. 4.2.2), every triplet evaluated once (Newton 3, the
// future-work traversal of Sec. 5).
//
// Ownership.  A triplet belongs to its lowest member in the order "cell layer along z, then z in fixed
// point (positions of the last binning, box = 2^32 units), then sorted index".  Within a triangle of
// particles closer than r_c the unwrapped cell layers differ by at most one (cell edge >= r_c, at least
// three cells per side) and the fixed-point z differences are exact wrapping 32-bit integers, so the
// order is a total order on every triangle: each triplet has exactly one owner.  The owner i sees the
// other two in its half list {j : r_ij <= r_c3, j above i}, about half of its neighbours (a half ball,
// so the list length varies little from particle to particle).  The pair-list build writes the half
// lists (S.half) with exact cutoff decisions; this kernel takes them as given.
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
// Per-(base, node) totals are added to the node's force sum: FP32 path, in 64-bit fixed point
// (fix_red3: exact, order-independent sums, bitwise reproducible); FP64 path, with FP64 atomics.
// The combine kernel reads and clears the sums.
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

#ifndef R3B_ROT_MINB
#define R3B_ROT_MINB 5  // FP32: CTAs per SM the register allocation is sized for (5-8 measured: 5, without spills, fastest)
#endif
constexpr int kZrMax = 64;    // half-list capacity: two rotation groups of at most 32 nodes
constexpr int kZrWarps = 4;   // warps per CTA
constexpr int kZrPer = 8;     // default number of consecutive bases per warp in one work item
static_assert(kZrMax == kHalfCap, "half-list capacity");
static_assert(kZrWarps * kZrPer == rot_bases_per_item(0) && kZrWarps == kRotWarps, "work items and kernel disagree");

// FP32 reciprocal square root: the hardware approximation (flush-to-zero form; the argument is a
// product of three squared distances, never subnormal) refined by one Newton-Raphson step
__device__ __forceinline__ float zr_rsqrt(float q) {
  float t;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(q));
  return t * fmaf(-0.5f * q, t * t, 1.5f);
}
__device__ __forceinline__ double zr_rsqrt(double q) { return 1.0 / sqrt(q); }

// asynchronous global -> shared copies (completed in commit-group order)
__device__ __forceinline__ unsigned zr_smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void zr_cp16(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(zr_smem_u32(dst)), "l"(__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void zr_cp4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(zr_smem_u32(dst)), "l"(__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void zr_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void zr_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename T>
struct ZrSmem {
  using T4 = typename V4<T>::type;
  T4 pn[kZrMax];            // partners of the current phase, doubled (pn[t + m] = pn[t]), far dummies after;
                            // the half list is built here: (d_v, |d_v|^2)
  T4 slot[2][kZrMax];       // partner shares (G, W) of odd and even steps, in pn's index space
  T4 nd[kZrMax];            // copy of the half list (lists longer than 32 nodes)
  T4 tot[kZrMax];           // per-node totals across phases (lists longer than 32 nodes)
  int nidx[kZrMax];         // sorted index of each node
  int4 cq[kZrMax];          // prefetched fixed-point positions of the next base's half list
  unsigned row[2][kZrMax];  // prefetched half lists (pair-list entries) of the next two bases
  int4 selfq;               // fixed-point position of the prefetched base
  int rcnt[2];              // lengths of the prefetched half lists
  int pad_[2];
};

// Per-CTA copy of the system constants this kernel reads (shared memory: no global reloads)
template <typename T>
struct ZrK {
  const unsigned* half;
  const int* half_cnt;
  const int4* ipos;
  const double* X;       // FP64 positions of the evaluated buffer (exact repeats)
  const void* pos;       // cell-local positions of the evaluated buffer (FP64 path)
  void* f3acc;
  unsigned long long* ctr;
  int* flags;
  double L, rc3sq, nu, edge;
  T rcsq, g, fs;         // r_c3^2, guard half-width, 3/4 nu in the kernel's precision (FP64 path; the
                         // FP32 path's fixed-point sums take unscaled terms)
  float qscale;          // L / 2^32
  int n;
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
template <typename T>
__device__ __forceinline__ typename V4<T>::type zr_add4(typename V4<T>::type p, typename V4<T>::type q) {
  p.x += q.x;
  p.y += q.y;
  p.z += q.z;
  p.w += q.w;
  return p;
}

// Per-lane running sums of one phase.
template <typename T>
struct ZrAcc {
  T W, Gx, Gy, Gz;  // own node
  T cnt, u;         // accepted pairs, energy / nu
  T dmin;           // smallest |c - r_c^2| met (FP32 decisions)
};

// partner entries of a phase: entry t of pn is node pfirst + (t mod period) (exact repeats only)
struct ZrPart {
  int first, period;
};

// One phase: own node J of this lane (J.w = |d_J|^2; far dummy for lanes without a node), partners in
// w.pn.  Full steps s_lo .. s_hi for every lane; then, if half > 0, step `half` for lanes v < half
// only.  Slots must be zero on entry.
template <typename T, bool kE, bool kExact>
__device__ __forceinline__ void zr_steps(const ZrK<T>& K, ZrSmem<T>& w, const typename V4<T>::type J, const int jid,
                                         const ZrPart pp, const int s_lo, const int s_hi, const int half,
                                         const int lane, ZrAcc<T>& A) {
  using T4 = typename V4<T>::type;
  const T rcsq = K.rcsq, g = K.g;
  const T a = J.w, a2 = J.w + J.w;
  auto step = [&](const int s, const int par, const bool masked) {
    const T4 pk = w.pn[lane + s];
    const T ex = pk.x - J.x, ey = pk.y - J.y, ez = pk.z - J.z;
    T c = fma(ez, ez, fma(ey, ey, ex * ex));
    if (masked) c += (T)1e6;  // only the last step of an even list
    const T t = c - rcsq;
    T okf;
    if constexpr (kExact) {
      bool ok = t <= g;
      const bool band = ok && t >= -g;
      if (__any_sync(0xffffffffu, band)) {
        if (band) {
          atomicAdd(&K.ctr[CTR_GUARD], 1ull);
          const int u = lane + s;
          const int kid = w.nidx[pp.first + (u >= pp.period ? u - pp.period : u)];
          ok = exact_within(K.X, K.n, jid, kid, K.L, K.rc3sq);
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
    step(s, 0, false);
    step(s + 1, 1, false);
    __syncwarp();
  }
  if (s <= s_hi) {
    step(s, 0, false);
    __syncwarp();
  }
  if (half > 0) {
    step(half, 1, lane >= half);
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

// Partner layout from w.nd: nodes first .. first + mb - 1 padded to period mp (mb <= mp <= 32),
// doubled, then far dummies (a self rotation has mb = mp).
template <typename T>
__device__ __forceinline__ void zr_layout(ZrSmem<T>& w, int first, int mb, int mp, int lane) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = lane + 32 * h;
    const int v = t < mp ? t : t - mp;
    const bool real = t < 2 * mp && v < mb;
    w.pn[t] = real ? w.nd[first + v] : zr_far<T>((T)-1);
  }
}

// One phase with FP32 decisions; if a pair met the guard band, it is discarded and repeated with
// exact decisions.  The lane's own-node sums, count and energy are left in A.
template <typename T, bool kE>
__device__ __forceinline__ void zr_phase(const ZrK<T>& K, ZrSmem<T>& w, const typename V4<T>::type J, const int jid,
                                         const ZrPart pp, const int s_lo, const int s_hi, const int half,
                                         const int lane, ZrAcc<T>& A) {
  A.W = A.Gx = A.Gy = A.Gz = A.cnt = A.u = (T)0;
  A.dmin = (T)1e30;
  zr_steps<T, kE, false>(K, w, J, jid, pp, s_lo, s_hi, half, lane, A);
  if (__any_sync(0xffffffffu, A.dmin <= K.g)) {
    __syncwarp();
    zr_clear_slots<T>(w, lane);
    __syncwarp();
    A.W = A.Gx = A.Gy = A.Gz = A.cnt = A.u = (T)0;
    zr_steps<T, kE, true>(K, w, J, jid, pp, s_lo, s_hi, half, lane, A);
  }
}

// ---------------------------------------------------------------- paired steps (FP32, m <= 32)
// The rotation over m <= 32 nodes (node v on lane v) with two consecutive steps s, s + 1 evaluated
// together in the two halves of packed FP32x2 instructions (Blackwell FFMA2/FADD2/FMUL2).  Partner
// data of both steps comes from the doubled list in shared memory (pn[t] and pn[t + 1]).
// The partner shares do not go through shared memory: they travel with the partners.  In iteration
// k (steps 2k+1, 2k+2) lane v holds the running shares of nodes v + 2k + 1 (first half) and
// v + 2k + 2 (second half); those nodes are the partners of lane v - 2 in iteration k + 1, so the
// shares move two lanes down after each iteration (shuffles on the ring of m lanes), and after the
// last one they are delivered to the nodes' own lanes.  Steps 1 .. floor(m / 2); for even m the last
// one pairs v with v + m / 2 on lanes v < m / 2 only.  Returns false, with nothing accumulated, if
// some pair fell in the guard band around r_c^2 (the caller repeats with exact decisions).
struct ZrOut32 {
  float W, Gx, Gy, Gz, cnt, u;
};
__device__ __forceinline__ float2 f2s(float x) { return make_float2(x, x); }

template <bool kE>
__device__ __forceinline__ bool zr_self_f2(const ZrK<float>& K, ZrSmem<float>& w, const float4 J, const int m,
                                           const int lane, ZrOut32& o) {
  const float rcsq = K.rcsq, g = K.g;
  const int T = m >> 1;                 // steps
  const int K2 = (T + 1) >> 1;          // iterations (pairs of steps)
  const bool real = lane < m;
  const bool even = (m & 1) == 0;
  const float2 jx = f2s(J.x), jy = f2s(J.y), jz = f2s(J.z), ja = f2s(J.w), ja2 = f2s(J.w + J.w);
  const float2 nrc = f2s(-rcsq), m2 = f2s(-2.f), h25 = f2s(2.5f), c4 = f2s(4.f);
  float2 W = f2s(0.f), Gx = W, Gy = W, Gz = W, cnt = W, uu = W;
  float2 tW = W, tx = W, ty = W, tz = W;  // travelling shares of this lane's two partners
  float dmin = 1e30f;
  const int pass = real ? (lane + 2 < m ? lane + 2 : lane + 2 - m) : lane;
  auto iter = [&](const int s1, const float2 off) {
    const int t = lane + s1;
    const float4 p0 = w.pn[t], p1 = w.pn[t + 1];  // partners of steps s1 and s1 + 1 (t + 1 < 2m + 32)
    const float2 px = make_float2(p0.x, p1.x), py = make_float2(p0.y, p1.y), pz = make_float2(p0.z, p1.z);
    const float2 b = make_float2(p0.w, p1.w);
    const float2 ex = __fadd2_rn(px, make_float2(-jx.x, -jx.y));
    const float2 ey = __fadd2_rn(py, make_float2(-jy.x, -jy.y));
    const float2 ez = __fadd2_rn(pz, make_float2(-jz.x, -jz.y));
    float2 c = __ffma2_rn(ez, ez, __ffma2_rn(ey, ey, __fmul2_rn(ex, ex)));
    c = __fadd2_rn(c, off);
    const float2 tt = __fadd2_rn(c, nrc);
    dmin = fminf(dmin, fminf(fabsf(tt.x), fabsf(tt.y)));
    const float2 okf = make_float2(tt.x <= g ? 1.f : 0.f, tt.y <= g ? 1.f : 0.f);
    const float2 ab = __fmul2_rn(ja, b);
    const float2 q = __fmul2_rn(ab, c);
    float2 u;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(u.x) : "f"(q.x));
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(u.y) : "f"(q.y));
    // one Newton-Raphson step: u (1.5 - 0.5 q u^2)
    u = __fmul2_rn(u, __ffma2_rn(__fmul2_rn(f2s(-0.5f), q), __fmul2_rn(u, u), f2s(1.5f)));
    const float2 ww = __fmul2_rn(u, u);
    const float2 t3 = __fmul2_rn(ww, u);
    const float2 t5 = __fmul2_rn(t3, ww);
    const float2 sum = __fadd2_rn(__fadd2_rn(ja, b), c);
    const float2 Aa = __ffma2_rn(m2, c, sum);   // a + b - c
    const float2 Bb = __ffma2_rn(m2, b, sum);   // a - b + c
    const float2 Cc = __ffma2_rn(m2, ja, sum);  // -a + b + c
    const float2 AB = __fmul2_rn(Aa, Bb), AC = __fmul2_rn(Aa, Cc), BC = __fmul2_rn(Bb, Cc);
    const float2 P = __fmul2_rn(AB, Cc);
    const float2 Pa = __ffma2_rn(ja2, Cc, make_float2(-AB.x, -AB.y));
    const float2 Pb = __ffma2_rn(__fadd2_rn(b, b), Bb, make_float2(-AC.x, -AC.y));
    const float2 Pc = __ffma2_rn(__fadd2_rn(c, c), Aa, make_float2(-BC.x, -BC.y));
    const float2 Pw = __fmul2_rn(P, ww);
    const float2 H = __ffma2_rn(h25, Pw, c4);
    const float2 nH = make_float2(-H.x, -H.y);
    const float2 kk = __fmul2_rn(t5, okf);
    const float2 pa2 = __fmul2_rn(kk, __ffma2_rn(__fmul2_rn(b, c), nH, Pa));
    const float2 pb2 = __fmul2_rn(kk, __ffma2_rn(__fmul2_rn(ja, c), nH, Pb));
    const float2 pc2 = __fmul2_rn(kk, __ffma2_rn(ab, nH, Pc));
    cnt = __fadd2_rn(cnt, okf);
    if constexpr (kE) uu = __ffma2_rn(__fmul2_rn(t3, okf), __ffma2_rn(f2s(0.375f), Pw, f2s(1.f)), uu);
    W = __fadd2_rn(W, pa2);
    Gx = __ffma2_rn(pc2, ex, Gx);
    Gy = __ffma2_rn(pc2, ey, Gy);
    Gz = __ffma2_rn(pc2, ez, Gz);
    const float2 npc = make_float2(-pc2.x, -pc2.y);
    tW = __fadd2_rn(tW, pb2);
    tx = __ffma2_rn(npc, ex, tx);
    ty = __ffma2_rn(npc, ey, ty);
    tz = __ffma2_rn(npc, ez, tz);
  };
  auto shift = [&](float2& v, int src) {
    v.x = __shfl_sync(0xffffffffu, v.x, src);
    v.y = __shfl_sync(0xffffffffu, v.y, src);
  };
  const float2 zero2 = f2s(0.f), big = f2s(1e6f);
  const float2 offr = real ? zero2 : big;
  int k = 0;
#pragma unroll 1
  for (; k < K2 - 1; ++k) {  // full iterations: both steps on every lane with a node
    iter(2 * k + 1, offr);
    shift(tW, pass);
    shift(tx, pass);
    shift(ty, pass);
    shift(tz, pass);
  }
  // last iteration: s1 = 2k + 1 <= T; s2 = s1 + 1 exists iff s2 <= T; the step T is the half step
  // (lanes v < m / 2) when m is even
  const int s1 = 2 * k + 1, s2 = s1 + 1;
  const bool half_ok = lane < (m >> 1);
  const bool v1 = real && (!(even && s1 == T) || half_ok);
  const bool v2 = real && s2 <= T && (!(even && s2 == T) || half_ok);
  iter(s1, make_float2(v1 ? 0.f : 1e6f, v2 ? 0.f : 1e6f));
  if (__any_sync(0xffffffffu, dmin <= g)) return false;
  // deliver the travelling shares to their nodes' lanes: node u's first-half share sits on lane
  // u - s1, its second-half share on lane u - s2 (mod m)
  const int d1 = real ? (lane - s1 >= 0 ? lane - s1 : lane - s1 + m) : lane;
  const int d2 = real ? (lane - s2 >= 0 ? lane - s2 : lane - s2 + m) : lane;
  const float rW = __shfl_sync(0xffffffffu, tW.x, d1) + __shfl_sync(0xffffffffu, tW.y, d2);
  const float rx = __shfl_sync(0xffffffffu, tx.x, d1) + __shfl_sync(0xffffffffu, tx.y, d2);
  const float ry = __shfl_sync(0xffffffffu, ty.x, d1) + __shfl_sync(0xffffffffu, ty.y, d2);
  const float rz = __shfl_sync(0xffffffffu, tz.x, d1) + __shfl_sync(0xffffffffu, tz.y, d2);
  o.W = (W.x + W.y) + rW;
  o.Gx = (Gx.x + Gx.y) + rx;
  o.Gy = (Gy.x + Gy.y) + ry;
  o.Gz = (Gz.x + Gz.y) + rz;
  o.cnt = cnt.x + cnt.y;
  o.u = uu.x + uu.y;
  return true;
}

// ---------------------------------------------------------------- half-list nodes
// FP32 node: displacement from the fixed-point positions (wrapping difference = exact minimum image,
// one rounding to FP32, one scaling) and its squared length
__device__ __forceinline__ float4 zr_qnode(const float sc, const int4 qi, const int4 qj) {
  float4 d;
  d.x = (float)(int)((unsigned)qj.x - (unsigned)qi.x) * sc;
  d.y = (float)(int)((unsigned)qj.y - (unsigned)qi.y) * sc;
  d.z = (float)(int)((unsigned)qj.z - (unsigned)qi.z) * sc;
  d.w = fmaf(d.z, d.z, fmaf(d.y, d.y, d.x * d.x));
  return d;
}

// Half list of base x read from global memory into w.pn / w.nidx (FP64 path); returns its length.
template <typename T>
__device__ __forceinline__ int zr_build_direct(const ZrK<T>& K, ZrSmem<T>& w, const int x, const int lane) {
  const int m = K.half_cnt[x];
  const unsigned* __restrict__ row = K.half + (size_t)x * kHalfCap;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = lane + 32 * h;
    if (t < min(m, kZrMax)) {
      const unsigned e = row[t];
      const int j = (int)(e & kNbrMask);
      typename V4<T>::type d;
      if constexpr (sizeof(T) == 4) {
        d = zr_qnode(K.qscale, K.ipos[x], K.ipos[j]);
      } else {
        const double4_32a* P = reinterpret_cast<const double4_32a*>(K.pos);
        const double4_32a pi = P[x], pj = P[j];
        const unsigned code = e >> kNbrShift;
        d.x = (pj.x - pi.x) + ((double)(int)(code & 3u) - 1.0) * K.edge;
        d.y = (pj.y - pi.y) + ((double)(int)((code >> 2) & 3u) - 1.0) * K.edge;
        d.z = (pj.z - pi.z) + ((double)(int)(code >> 4) - 1.0) * K.edge;
        d.w = fma(d.z, d.z, fma(d.y, d.y, d.x * d.x));
      }
      w.pn[t] = d;
      w.nidx[t] = j;
    }
  }
  __syncwarp();
  return m;
}

// FP32 prefetch, stage 1: the half list (pair-list entries) and its length of base x
__device__ __forceinline__ void zr_fetch_row(const ZrK<float>& K, ZrSmem<float>& w, int slot, int x, int lane) {
  if (lane < kZrMax / 4) zr_cp16(&w.row[slot][4 * lane], K.half + (size_t)x * kHalfCap + 4 * lane);
  if (lane == 0) zr_cp4(&w.rcnt[slot], K.half_cnt + x);
}
// stage 2 (half list already in shared memory): the fixed-point positions of base x and of its
// half-list members
__device__ __forceinline__ void zr_fetch_pos(const ZrK<float>& K, ZrSmem<float>& w, int slot, int x, int lane) {
  if (lane == 0) zr_cp16(&w.selfq, K.ipos + x);
  const int m = min(w.rcnt[slot], kZrMax);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = lane + 32 * h;
    if (t < m) zr_cp16(&w.cq[t], K.ipos + (w.row[slot][t] & kNbrMask));
  }
}
// nodes of base x from the prefetched half list (slot) and positions; returns the list length
__device__ __forceinline__ int zr_build_staged(const ZrK<float>& K, ZrSmem<float>& w, const int slot,
                                               const int lane) {
  const int m = w.rcnt[slot];
  const int4 qi = w.selfq;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = lane + 32 * h;
    if (t < min(m, kZrMax)) {
      w.pn[t] = zr_qnode(K.qscale, qi, w.cq[t]);
      w.nidx[t] = (int)(w.row[slot][t] & kNbrMask);
    }
  }
  __syncwarp();
  return m;
}

// ---------------------------------------------------------------- evaluation of one base
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

// one (base, node) force term to the node's sum: FP32, unscaled into the fixed-point sums (the
// combine kernel applies 3/4 nu); FP64, scaled by 3/4 nu with FP64 atomics
template <typename T>
__device__ __forceinline__ void zr_atomic_add(const ZrK<T>& K, int j, T fx, T fy, T fz) {
  if constexpr (sizeof(T) == 4) {
    if (!fix_red3(K.f3acc, j, fx, fy, fz)) atomicOr(K.flags + FLG_ERR, ERR_NONFINITE);
  } else {
    double* q = reinterpret_cast<double*>(K.f3acc) + 4 * (size_t)j;
    atomicAdd(q, K.fs * fx);
    atomicAdd(q + 1, K.fs * fy);
    atomicAdd(q + 2, K.fs * fz);
  }
}

// A lane's share of the base force F_i.  FP64: the sums of W_v d_v.  FP32: the sums of the lane's
// fixed-point node terms; the triplet forces of a base add up to zero (Newton 3), so F_i is minus the
// sum of its nodes' terms, taken exactly in fixed point (each base's terms then cancel exactly).
template <typename T> struct ZrFi;
template <> struct ZrFi<double> {
  double x = 0.0, y = 0.0, z = 0.0;
};
template <> struct ZrFi<float> {
  long long x = 0, y = 0, z = 0;
};

// node force F_v = G_v - W_v d_v (unscaled) to its sum, and its share of F_i
__device__ __forceinline__ void zr_emit(const ZrK<double>& K, const double4_32a d, int j, double W, double Gx,
                                        double Gy, double Gz, ZrFi<double>& fi) {
  fi.x = fma(W, d.x, fi.x);
  fi.y = fma(W, d.y, fi.y);
  fi.z = fma(W, d.z, fi.z);
  zr_atomic_add<double>(K, j, fma(-W, d.x, Gx), fma(-W, d.y, Gy), fma(-W, d.z, Gz));
}
__device__ __forceinline__ void zr_emit(const ZrK<float>& K, const float4 d, int j, float W, float Gx, float Gy,
                                        float Gz, ZrFi<float>& fi) {
  const float fx = fmaf(-W, d.x, Gx), fy = fmaf(-W, d.y, Gy), fz = fmaf(-W, d.z, Gz);
  if (!(fabsf(fx) < kFixLimit && fabsf(fy) < kFixLimit && fabsf(fz) < kFixLimit)) {
    atomicOr(K.flags + FLG_ERR, ERR_NONFINITE);
    return;
  }
  const long long qx = __float2ll_rn(fx * kFixOne), qy = __float2ll_rn(fy * kFixOne), qz = __float2ll_rn(fz * kFixOne);
  unsigned long long* q = reinterpret_cast<unsigned long long*>(K.f3acc) + 4 * (size_t)j;
  atomicAdd(q, (unsigned long long)qx);
  atomicAdd(q + 1, (unsigned long long)qy);
  atomicAdd(q + 2, (unsigned long long)qz);
  fi.x += qx;
  fi.y += qy;
  fi.z += qz;
}

// exact warp sum of 64-bit integers of magnitude below 2^58: three 21-bit limbs (the 32-bit warp
// reductions of the two low limbs stay below 2^26, the signed high limb below 2^22)
__device__ __forceinline__ long long zr_warp_sum64(long long q) {
  const unsigned lo = (unsigned)q & 0x1FFFFFu;
  const unsigned mid = (unsigned)(q >> 21) & 0x1FFFFFu;
  const int hi = (int)(q >> 42);
  const unsigned slo = __reduce_add_sync(0xffffffffu, lo);
  const unsigned smid = __reduce_add_sync(0xffffffffu, mid);
  const int shi = __reduce_add_sync(0xffffffffu, hi);
  return (long long)shi * (1ll << 42) + (long long)smid * (1ll << 21) + (long long)slo;
}

// F_i of base x to its sum (every lane takes part)
__device__ __forceinline__ void zr_emit_base(const ZrK<double>& K, int x, const ZrFi<double>& fi, int lane) {
  const double k = zr_sum4<double>(fi.x, fi.y, fi.z, 0.0, lane);
  const double Fx = k, Fy = __shfl_sync(0xffffffffu, k, 8), Fz = __shfl_sync(0xffffffffu, k, 16);
  if (lane == 0) zr_atomic_add<double>(K, x, Fx, Fy, Fz);
}
__device__ __forceinline__ void zr_emit_base(const ZrK<float>& K, int x, const ZrFi<float>& fi, int lane) {
  const long long Fx = -zr_warp_sum64(fi.x), Fy = -zr_warp_sum64(fi.y), Fz = -zr_warp_sum64(fi.z);
  if (lane == 0) {
    unsigned long long* q = reinterpret_cast<unsigned long long*>(K.f3acc) + 4 * (size_t)x;
    atomicAdd(q, (unsigned long long)Fx);
    atomicAdd(q + 1, (unsigned long long)Fy);
    atomicAdd(q + 2, (unsigned long long)Fz);
  }
}

// Per-lane energy sum across a warp's bases: FP32 path, a compensated (hi, lo) pair (TwoSum; no FP64
// instruction per base, FP64 being scarce on GB300), converted to FP64 for the warp and CTA sums; FP64
// path, a plain double.
template <typename T> struct ZrU;
template <> struct ZrU<float> {
  CompF c{0.f, 0.f};
  __device__ __forceinline__ void add(float t) { c.add(t); }
  __device__ __forceinline__ double value() const { return c.value(); }
};
template <> struct ZrU<double> {
  double c = 0.0;
  __device__ __forceinline__ void add(double t) { c += t; }
  __device__ __forceinline__ double value() const { return c; }
};

// All triplets owned by base x, whose half list (length m) is in w.pn / w.nidx.  Adds the forces to
// the accumulators and the count and energy (per lane) to cnt_sum, u_sum.
template <typename T, bool kE>
__device__ __forceinline__ void zr_eval(const ZrK<T>& K, ZrSmem<T>& w, const int x, const int m, const int lane,
                                        T& cnt_sum, ZrU<T>& u_sum) {
  using T4 = typename V4<T>::type;
  if (m > kZrMax) {
    if (lane == 0) atomicOr(K.flags + FLG_ERR, ERR_HALF_CAP);
    return;
  }
  if (m < 2) return;
  ZrFi<T> fi;
  ZrAcc<T> A;
  if (m <= 32) {
    // the list in place, doubled (pn[v + m] = pn[v]), then far dummies
    const T4 J = lane < m ? w.pn[lane] : zr_far<T>((T)1);
    const int jid = lane < m ? w.nidx[lane] : 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int t = lane + 32 * h;
      if (t >= m) w.pn[t] = t < 2 * m ? w.pn[t - m] : zr_far<T>((T)-1);
    }
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      __syncwarp();  // the doubled list is read by other lanes
      ZrOut32 r;
      if (zr_self_f2<kE>(K, w, J, m, lane, r)) {
        done = true;
        cnt_sum += r.cnt;
        if (kE) u_sum.add(r.u);
        if (lane < m) zr_emit(K, J, jid, r.W, r.Gx, r.Gy, r.Gz, fi);
      }
    }
    if (!done) {  // FP64 path, or a pair in the guard band: shared-memory rotation (exact repeat if needed)
      zr_clear_slots<T>(w, lane);
      __syncwarp();
      zr_phase<T, kE>(K, w, J, jid, ZrPart{0, m}, 1, (m - 1) >> 1, (m & 1) ? 0 : (m >> 1), lane, A);
      cnt_sum += A.cnt;
      if (kE) u_sum.add(A.u);
      if (lane < m) {
        const T4 s = zr_add4<T>(zr_add4<T>(w.slot[0][lane], w.slot[1][lane]),
                                zr_add4<T>(w.slot[0][lane + m], w.slot[1][lane + m]));
        zr_emit(K, J, jid, A.W + s.w, A.Gx + s.x, A.Gy + s.y, A.Gz + s.z, fi);
      }
    }
  } else {
    // halves A = nodes 0 .. ma-1, B = nodes ma .. m-1 (mb <= ma <= 32): within A, within B, A x B
    const int ma = (m + 1) >> 1, mb = m - ma;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      w.nd[lane + 32 * h] = w.pn[lane + 32 * h];
      w.tot[lane + 32 * h] = zr_zero<T>();
    }
#pragma unroll 1
    for (int ph = 0; ph < 3; ++ph) {
      const int own_first = ph == 1 ? ma : 0, own_n = ph == 1 ? mb : ma;
      const int par_first = ph == 0 ? 0 : ma, par_n = ph == 0 ? ma : mb, par_period = ph == 2 ? ma : par_n;
      __syncwarp();
      zr_clear_slots<T>(w, lane);
      zr_layout<T>(w, par_first, par_n, par_period, lane);
      const T4 J = lane < own_n ? w.nd[own_first + lane] : zr_far<T>((T)1);
      const int jid = lane < own_n ? w.nidx[own_first + lane] : 0;
      __syncwarp();
      const ZrPart pp{par_first, par_period};
      if (ph < 2)
        zr_phase<T, kE>(K, w, J, jid, pp, 1, (own_n - 1) >> 1, (own_n & 1) ? 0 : (own_n >> 1), lane, A);
      else
        zr_phase<T, kE>(K, w, J, jid, pp, 0, ma - 1, 0, lane, A);
      cnt_sum += A.cnt;
      if (kE) u_sum.add(A.u);
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
        zr_emit(K, w.nd[v], w.nidx[v], t.w, t.x, t.y, t.z, fi);
      }
    }
  }
  zr_emit_base(K, x, fi, lane);
}

template <typename T>
__device__ __forceinline__ void zr_eval_any(const ZrK<T>& K, ZrSmem<T>& w, int x, int m, int lane, bool energy, T& cnt,
                                            ZrU<T>& u) {
  if (energy)
    zr_eval<T, true>(K, w, x, m, lane, cnt, u);
  else
    zr_eval<T, false>(K, w, x, m, lane, cnt, u);
  __syncwarp();  // the next base reuses the warp's shared memory
}

// Work item: 4 per consecutive bases, per of them for each warp (the autotuner picks per; 8 by
// default, kZrPer).  FP32: a two-stage cp.async pipeline per warp
// copies the half list of base k + 2 and the positions of base k + 1 into shared memory while base k
// is evaluated.  Counts and energy (compensated per lane, FP64 across lanes) are summed per CTA (the
// last warp to finish adds them to the system's totals with one atomic each).
template <typename T>
__global__ void __launch_bounds__(32 * kZrWarps, sizeof(T) == 4 ? R3B_ROT_MINB : 4)
    k_atm_rot(const SysDev* __restrict__ sys, const PItem* __restrict__ items, const int per) {
  pdl_wait();
  extern __shared__ __align__(32) unsigned char zr_raw[];
  __shared__ ZrK<T> K;
  __shared__ unsigned long long s_cnt;
  __shared__ double s_u;
  __shared__ int s_done;
  const PItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  const int imode = item_mode(S, it.mode);
  if (imode & M_SKIP) return;  // block-uniform
  const bool energy = (imode & M_ENERGY) != 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    K.half = reinterpret_cast<const unsigned*>(S.half);
    K.half_cnt = S.half_cnt;
    K.ipos = S.ipos;
    K.X = S.X[it.buf];
    K.pos = S.pos[it.buf];
    K.f3acc = S.f3acc;
    K.ctr = S.ctr;
    K.flags = S.flags;
    K.L = S.L;
    K.rc3sq = S.rc3sq;
    K.nu = S.nu;
    K.edge = S.edge;
    K.rcsq = Par<T>::rc3sq(S);
    K.g = Par<T>::guard3(S);
    K.fs = (T)0.75 * Par<T>::nu(S);
    K.qscale = S.f_qscale;
    K.n = S.n;
    s_cnt = 0ull;
    s_u = 0.0;
    s_done = 0;
  }
  __syncthreads();
  ZrSmem<T>& w = reinterpret_cast<ZrSmem<T>*>(zr_raw)[warp];
  const int n = K.n;
  const int x0 = it.begin + warp * per;
  const int nb = max(0, min(per, n - x0));  // bases of this warp
  T cnt = (T)0;
  ZrU<T> u;
  if constexpr (sizeof(T) == 4) {
    if (nb > 0) {
      zr_fetch_row(K, w, 0, x0, lane);
      zr_commit();
      zr_wait<0>();
      __syncwarp();
      zr_fetch_pos(K, w, 0, x0, lane);
      zr_commit();
      if (nb > 1) zr_fetch_row(K, w, 1, x0 + 1, lane);
      zr_commit();
    }
    for (int k = 0; k < nb; ++k) {
      zr_wait<1>();  // positions of base k (and every older group) have arrived
      __syncwarp();
      const int m = zr_build_staged(K, w, k & 1, lane);
      if (k + 1 < nb) {  // refill: positions of base k + 1, half list of base k + 2
        zr_wait<0>();
        __syncwarp();
        zr_fetch_pos(K, w, (k + 1) & 1, x0 + k + 1, lane);
      }
      zr_commit();
      __syncwarp();  // every lane has read slot k & 1 before it is refilled
      if (k + 2 < nb) zr_fetch_row(K, w, k & 1, x0 + k + 2, lane);
      zr_commit();
      zr_eval_any<T>(K, w, x0 + k, m, lane, energy, cnt, u);
    }
    zr_wait<0>();
  } else {
    for (int k = 0; k < nb; ++k) {
      const int m = zr_build_direct<T>(K, w, x0 + k, lane);
      zr_eval_any<T>(K, w, x0 + k, m, lane, energy, cnt, u);
    }
  }
  // per-lane counts are exact small integers in T (integer warp reduction: no FP64 instructions)
  const unsigned c = __reduce_add_sync(0xffffffffu, (unsigned)cnt);
  const double uu = energy ? warp_sum(u.value()) : 0.0;
  if (lane == 0) {
    atomicAdd(&s_cnt, (unsigned long long)c);
    if (energy) atomicAdd(&s_u, uu);
    __threadfence_block();
    if (atomicAdd(&s_done, 1) == kZrWarps - 1) {  // last warp of the CTA
      __threadfence_block();
      const unsigned long long ct = atomicAdd(&s_cnt, 0ull);
      if (ct) atomicAdd(K.ctr + CTR_TRIPLETS, ct);
      if (energy) {
        const double U = K.nu * atomicAdd(&s_u, 0.0);
        atomicAdd(S.acc + ACC_U3, U);
        atomicAdd(S.acc + ACC_W3, 9.0 * U);  // sum_a r_a . F_a = 9 phi (phi is homogeneous of degree -9)
      }
    }
  }
}

// dynamic shared memory above the 48 KB default (per device, see raise_smem_attr)
template <typename T>
static bool zr_configure() {
  return raise_smem_attr((const void*)k_atm_rot<T>, (int)zr_smem_bytes<T>());
}

template <typename T>
void launch_atm_rot(const Launch& L, const PItem* items, int nitems, int per) {
  if (nitems > 0 && zr_configure<T>())
    launch_kernel(L, k_atm_rot<T>, nitems, 32 * kZrWarps, zr_smem_bytes<T>(), L.sys, items, per);
}
template void launch_atm_rot<float>(const Launch&, const PItem*, int, int);
template void launch_atm_rot<double>(const Launch&, const PItem*, int, int);

}  // namespace r3b
