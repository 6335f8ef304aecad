// Near-class ATM forces for the distance classes of the three-body force (the multiple-time-stepping
// outlook of Sec. 5; intermediate cutoff r_a after Nakano et al., Sec. 3): every triplet whose three
// pair distances are <= r_a, evaluated once, forces added to S.f3nacc.
//
// Candidates.  At every binning the pair-list build (k_listbuild, pass 2) keeps each particle's
// candidates: the neighbours ranked above it (cell layer along z, fixed-point z of the binning, sorted
// index: the ownership order of the triplet half lists) within (r_a + skin) of it.  A binning happens at
// least once per outer step and whenever a particle has moved more than skin / 2, so every pair that is
// within r_a at any later inner step before the next binning is a candidate pair then.  The ranking is
// frozen at the binning, so it is one total order for every evaluation until the next one, and each
// near triplet has exactly one owner: its lowest-ranked member, whose candidates hold the other two.
//
// Evaluation.  One thread per owner i (near triplets are few per particle: about 8 at density 0.8 and
// r_a = 1.5).  Pass 1 keeps the candidates within r_a of i at the current positions (cell-local
// coordinates plus the entry's cell offset) in shared memory; pass 2 tests every pair of them,
// r_ab <= r_a, and evaluates the triplet with the squared-distance form of the ATM potential:
//   w = 1/(abc), u = w^(1/2), A = a + b - c, B = a - b + c, C = -a + b + c, P = ABC,
//   2 dphi/da = 3/4 nu u^5 (dP/da - bc (4 + 5/2 P w)),  dP/da = 2aC - AB (b, c alike),
//   F_i = pa2 d_a + pb2 d_b,  F_a = -pa2 d_a + pc2 e,  F_b = -pb2 d_b - pc2 e,  e = d_b - d_a.
// F_i and F_a stay in registers (one sum update each per owner / node), F_b goes out with one sum
// update per triplet (FP32 path: 64-bit fixed-point sums, exact and order-independent).  Cutoff decisions within the guard band around r_a^2 are re-decided in FP64
// from the FP64 positions with the CPU definition's operation order (exact_within).
#include "md_internal.cuh"

namespace r3b {

// FP32 reciprocal square root: hardware approximation refined by one Newton-Raphson step
__device__ __forceinline__ float nr_rsqrt(float q) {
  float t;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(q));
  return t * fmaf(-0.5f * q, t * t, 1.5f);
}
__device__ __forceinline__ double nr_rsqrt(double q) { return 1.0 / sqrt(q); }

// one force term to particle j's near-class sum: FP32, unscaled terms into the 64-bit fixed-point sums
// (exact, order-independent; the reader applies 3/4 nu); FP64, terms scaled by 3/4 nu, FP64 atomics
template <typename T>
__device__ __forceinline__ void near_red(const SysDev& S, void* acc, int j, T fx, T fy, T fz) {
  if constexpr (sizeof(T) == 4) {
    if (!fix_red3(acc, j, fx, fy, fz)) atomicOr(&S.flags[FLG_ERR], ERR_NONFINITE);
  } else {
    double* q = reinterpret_cast<double*>(acc) + 4 * (size_t)j;
    atomicAdd(q, fx);
    atomicAdd(q + 1, fy);
    atomicAdd(q + 2, fz);
  }
}

// FP64 re-decision of r_pq <= r_a (out of line: rare, and it keeps the FP64 registers out of the loops)
__device__ __noinline__ bool near_exact(const SysDev& S, const double* X, int p, int q) {
  atomicAdd(&S.ctr[CTR_GUARD], 1ull);
  return exact_within(X, S.n, p, q, S.L, S.rasq);
}

// r^2 <= r_a^2 in the kernel's precision, re-decided in FP64 inside the guard band
template <typename T>
__device__ __forceinline__ bool near_within(const SysDev& S, const double* X, T r2, T ra, T ga, int p, int q) {
  if (r2 <= ra - ga) return true;
  if (r2 > ra + ga) return false;
  return near_exact(S, X, p, q);
}

// one near triplet (i, a, b): a = |d_a|^2, b = |d_b|^2, c = |e|^2, e = d_b - d_a; adds F_i and F_a to
// the running sums and returns F_b
template <typename T>
__device__ __forceinline__ void near_triplet(T fs, T aa, T bb, T cc, T ax, T ay, T az, T bx, T by, T bz, T ex,
                                             T ey, T ez, T& fix, T& fiy, T& fiz, T& fax, T& fay, T& faz, T& fbx,
                                             T& fby, T& fbz) {
  const T ab = aa * bb;
  const T u = nr_rsqrt(ab * cc);
  const T ww = u * u;
  const T t5 = fs * (ww * ww * u);
  const T sum = (aa + bb) + cc;
  const T A = sum - (T)2 * cc, B = sum - (T)2 * bb, C = sum - (T)2 * aa;
  const T AB = A * B, AC = A * C, BC = B * C;
  const T H = (T)4 + (T)2.5 * (AB * C) * ww;
  const T pa2 = t5 * ((aa + aa) * C - AB - bb * cc * H);
  const T pb2 = t5 * ((bb + bb) * B - AC - aa * cc * H);
  const T pc2 = t5 * ((cc + cc) * A - BC - ab * H);
  fix += pa2 * ax + pb2 * bx;
  fiy += pa2 * ay + pb2 * by;
  fiz += pa2 * az + pb2 * bz;
  fax += pc2 * ex - pa2 * ax;
  fay += pc2 * ey - pa2 * ay;
  faz += pc2 * ez - pa2 * az;
  fbx = -pb2 * bx - pc2 * ex;
  fby = -pb2 * by - pc2 * ey;
  fbz = -pb2 * bz - pc2 * ez;
}

// near nodes of a thread kept in shared memory (strided by thread); owners with more use the
// global-memory path
template <typename T> __host__ __device__ constexpr int near_slots() { return sizeof(T) == 4 ? 12 : 8; }

template <typename T>
__global__ void __launch_bounds__(kNearThreads) k_atm_near(const SysDev* __restrict__ sys, const PItem* __restrict__ items) {
  pdl_wait();
  using T4 = typename V4<T>::type;
  constexpr int kSlots = near_slots<T>();
  __shared__ T4 s_nd[kSlots * kNearThreads];  // (d_x, d_y, d_z, |d|^2) of near node v at [v][thread]
  __shared__ int s_ni[kSlots * kNearThreads];
  __shared__ unsigned s_cnt;
  const PItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  if (threadIdx.x == 0) s_cnt = 0u;
  __syncthreads();
  const int tid = threadIdx.x;
  const int i = it.begin + tid;
  unsigned cnt = 0u;
  if (i < S.n) {
    const T4* __restrict__ P = reinterpret_cast<const T4*>(S.pos[it.buf]);
    const double* __restrict__ X = S.X[it.buf];
    const int mc0 = S.half_a_cnt[i];
    if (mc0 > kHalfCap) atomicOr(&S.flags[FLG_ERR], ERR_NEAR_CAP);
    const int mc = min(mc0, kHalfCap);
    const unsigned* __restrict__ row = reinterpret_cast<const unsigned*>(S.half_a) + (size_t)i * kHalfCap;
    const T4 pi = P[i];
    const T edge = Par<T>::edge(S);
    const T ra = Par<T>::rasq(S), ga = Par<T>::guarda(S);
    const T fs = sizeof(T) == 4 ? (T)1 : (T)0.75 * Par<T>::nu(S);  // FP32: unscaled (fixed-point sums)
    // displacement of candidate entry e from i at the current positions
    auto node = [&](unsigned e, T& dx, T& dy, T& dz) {
      const T4 pj = P[e & kNbrMask];
      const unsigned code = e >> kNbrShift;
      dx = (pj.x - pi.x) + (T)((int)(code & 3u) - 1) * edge;
      dy = (pj.y - pi.y) + (T)((int)((code >> 2) & 3u) - 1) * edge;
      dz = (pj.z - pi.z) + (T)((int)(code >> 4) - 1) * edge;
    };
    // pass 1: the candidates within r_a of i now (independent gathers, unrolled for overlap)
    int m = 0;
#pragma unroll 4
    for (int c = 0; c < mc; ++c) {
      const unsigned e = row[c];
      T dx, dy, dz;
      node(e, dx, dy, dz);
      const T d2 = dx * dx + dy * dy + dz * dz;
      if (near_within<T>(S, X, d2, ra, ga, i, (int)(e & kNbrMask))) {
        if (m < kSlots) {
          T4 q;
          q.x = dx;
          q.y = dy;
          q.z = dz;
          q.w = d2;
          s_nd[m * kNearThreads + tid] = q;
          s_ni[m * kNearThreads + tid] = (int)(e & kNbrMask);
        }
        ++m;
      }
    }
    T fix = 0, fiy = 0, fiz = 0;
    if (m <= kSlots) {
      // pass 2: every pair of near nodes, from shared memory
#pragma unroll 1
      for (int a = 0; a + 1 < m; ++a) {
        const T4 na = s_nd[a * kNearThreads + tid];
        const int ja = s_ni[a * kNearThreads + tid];
        T fax = 0, fay = 0, faz = 0;
#pragma unroll 1
        for (int b = a + 1; b < m; ++b) {
          const T4 nb = s_nd[b * kNearThreads + tid];
          const T ex = nb.x - na.x, ey = nb.y - na.y, ez = nb.z - na.z;
          const T cc = ex * ex + ey * ey + ez * ez;
          if (cc > ra + ga) continue;
          const int jb = s_ni[b * kNearThreads + tid];
          if (cc > ra - ga && !near_within<T>(S, X, cc, ra, ga, ja, jb)) continue;
          T fbx, fby, fbz;
          near_triplet<T>(fs, na.w, nb.w, cc, na.x, na.y, na.z, nb.x, nb.y, nb.z, ex, ey, ez, fix, fiy, fiz, fax,
                          fay, faz, fbx, fby, fbz);
          near_red<T>(S, S.f3nacc, jb, fbx, fby, fbz);
          ++cnt;
        }
        if (fax != (T)0 || fay != (T)0 || faz != (T)0) near_red<T>(S, S.f3nacc, ja, fax, fay, faz);
      }
    } else {
      // more near nodes than shared slots: every pair of candidates from global memory
#pragma unroll 1
      for (int a = 0; a + 1 < mc; ++a) {
        const unsigned ea = row[a];
        const int ja = (int)(ea & kNbrMask);
        T ax, ay, az;
        node(ea, ax, ay, az);
        const T aa = ax * ax + ay * ay + az * az;
        if (!near_within<T>(S, X, aa, ra, ga, i, ja)) continue;
        T fax = 0, fay = 0, faz = 0;
#pragma unroll 1
        for (int b = a + 1; b < mc; ++b) {
          const unsigned eb = row[b];
          const int jb = (int)(eb & kNbrMask);
          T bx, by, bz;
          node(eb, bx, by, bz);
          const T bb = bx * bx + by * by + bz * bz;
          if (!near_within<T>(S, X, bb, ra, ga, i, jb)) continue;
          const T ex = bx - ax, ey = by - ay, ez = bz - az;
          const T cc = ex * ex + ey * ey + ez * ez;
          if (!near_within<T>(S, X, cc, ra, ga, ja, jb)) continue;
          T fbx, fby, fbz;
          near_triplet<T>(fs, aa, bb, cc, ax, ay, az, bx, by, bz, ex, ey, ez, fix, fiy, fiz, fax, fay, faz, fbx,
                          fby, fbz);
          near_red<T>(S, S.f3nacc, jb, fbx, fby, fbz);
          ++cnt;
        }
        if (fax != (T)0 || fay != (T)0 || faz != (T)0) near_red<T>(S, S.f3nacc, ja, fax, fay, faz);
      }
    }
    if (fix != (T)0 || fiy != (T)0 || fiz != (T)0) near_red<T>(S, S.f3nacc, i, fix, fiy, fiz);
  }
  const unsigned c = __reduce_add_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s_cnt, c);
  __syncthreads();
  if (threadIdx.x == 0 && s_cnt) atomicAdd(&S.ctr[CTR_NEAR], (unsigned long long)s_cnt);
}

template <typename T>
void launch_atm_near(const Launch& L, const PItem* items, int nitems) {
  if (nitems > 0) launch_kernel(L, k_atm_near<T>, nitems, kNearThreads, 0, L.sys, items);
}
template void launch_atm_near<float>(const Launch&, const PItem*, int);
template void launch_atm_near<double>(const Launch&, const PItem*, int);

}  // namespace r3b
