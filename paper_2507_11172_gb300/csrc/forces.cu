// Force kernels of the r-RESPA hot path (arXiv 2507.11172):
//   k_lj      Lennard-Jones 12-6 pair forces (Sec. 2.1) from the Verlet pair
//             list, fused with the inner velocity-Verlet kick/drift of
//             Algorithm 2 (one launch per inner step).
//   k_atm     Axilrod-Teller-Muto triplet forces (Sec. 2.1) with the triplet
//             cutoff "all three distances <= r_c" (Fig. 2 caption, Sec.
//             4.2.2), each triplet evaluated once with Newton-3 scatter.
//   k_combine per-particle sum of the triplet kernel's partial forces and the
//             outer (three-body) kicks of Algorithm 2.
//   k_start   opening half kicks and first drift of a call.
#include <stdio.h>

#include "md_internal.cuh"

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

// cell-local coordinate of an FP64 position relative to the centre of cell
// `cell`, folded to the nearest image (|rel| <= L/2)
__device__ __forceinline__ void cell_rel(const SysDev& S, int cell, const double x[3], double rel[3]) {
  int cc[3] = {cell % S.nc, (cell / S.nc) % S.nc, cell / (S.nc * S.nc)};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double r = x[a] - (cc[a] + 0.5) * S.edge;
    if (r > S.half_L) r -= S.L;
    if (r < -S.half_L) r += S.L;
    rel[a] = r;
  }
}

template <typename T>
__device__ __forceinline__ void store_pos(const SysDev& S, int buf, int i, const double rel[3], bool check_skin) {
  using T4 = typename V4<T>::type;
  T4 h;
  h.x = (T)rel[0];
  h.y = (T)rel[1];
  h.z = (T)rel[2];
  h.w = (T)0;
  reinterpret_cast<T4*>(S.pos[buf])[i] = h;
  if (check_skin) {
    T4 r = reinterpret_cast<const T4*>(S.ref)[i];
    double dx = (double)h.x - (double)r.x, dy = (double)h.y - (double)r.y, dz = (double)h.z - (double)r.z;
    if (dx * dx + dy * dy + dz * dz > S.half_skin_sq) atomicOr(&S.flags[FLG_SKIN], 1);
  }
}

// ============================================================== LJ pair kernel
// A team of kLjTeam lanes shares one particle i: lane t of the team walks list
// entries t, t + kLjTeam, ... (unrolled so several gathers are in flight), sums
// its share in a compensated (hi, lo) accumulator, and the team combines the
// shares with error-free TwoSum steps.  The team's first lane then applies the
// velocity-Verlet kick/drift of Algorithm 2 for i.
template <typename T>
__device__ __forceinline__ void team_sum(CompF& c) {
#pragma unroll
  for (int o = kLjTeam / 2; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, c.hi, o);
    const float ol = __shfl_xor_sync(0xffffffffu, c.lo, o);
    float s, e;
    two_sum(c.hi, oh, s, e);
    c.hi = s;
    c.lo = c.lo + (ol + e);
  }
}
__device__ __forceinline__ void team_sum_d(double& v) {
#pragma unroll
  for (int o = kLjTeam / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
}

template <typename T>
__global__ void __launch_bounds__(256, 4) k_lj(const SysDev* __restrict__ sys, const PItem* __restrict__ items) {
  using T4 = typename V4<T>::type;
  __shared__ double red[32];
  const PItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  const int kind = it.mode & M_KIND_MASK;
  const bool energy = (it.mode & M_ENERGY) != 0;
  const int n = S.n;
  const int tl = threadIdx.x % kLjTeam;
  const int i = it.begin + threadIdx.x / kLjTeam;
  const bool active = i < n;
  const T4* __restrict__ P = reinterpret_cast<const T4*>(S.pos[it.buf]);
  const double* __restrict__ X = S.X[it.buf];
  Acc3<T> f;
  AccS<T> u, w;
  if (active) {
    const T4 pi = P[i];
    const T edge = (T)S.edge;
    const T rcsq = (T)S.rc2sq;
    const T g2 = (T)S.guard2;
    const T sig2 = (T)S.sig2;
    const T eps24 = (T)(24.0 * S.eps), eps4 = (T)(4.0 * S.eps);
    const int cnt = S.nbr_cnt[i];
    const int* __restrict__ row = S.nbr + (size_t)i * S.maxnb;
#pragma unroll 4
    for (int t = tl; t < cnt; t += kLjTeam) {
      const unsigned e = (unsigned)__ldg(row + t);
      const int j = (int)(e & kNbrMask);
      const int code = (int)(e >> kNbrShift);
      const int ox = code % 3 - 1, oy = (code / 3) % 3 - 1, oz = code / 9 - 1;
      const T4 pj = P[j];
      const T dx = (pj.x - pi.x) + (T)ox * edge;
      const T dy = (pj.y - pi.y) + (T)oy * edge;
      const T dz = (pj.z - pi.z) + (T)oz * edge;
      const T r2 = dx * dx + dy * dy + dz * dz;
      if (r2 > rcsq + g2) continue;
      if (r2 >= rcsq - g2) {  // guard band: decide exactly in FP64
        atomicAdd(&S.ctr[CTR_GUARD], 1ull);
        if (!exact_within(X, n, i, j, S.L, S.rc2sq)) continue;
      }
      const T ir2 = recip<T>(r2);
      const T sr2 = sig2 * ir2;
      const T sr6 = sr2 * sr2 * sr2;
      const T sr12 = sr6 * sr6;
      const T g = eps24 * (sr12 + sr12 - sr6) * ir2;  // F_i = -g d
      f.add(-g * dx, -g * dy, -g * dz);
      if (energy) {
        u.add(eps4 * (sr12 - sr6));
        w.add(g * r2);
      }
    }
  }
  // combine the team's shares (all lanes take part in the shuffles)
  double F[3], uu = 0.0, ww = 0.0;
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      team_sum<T>(f.c[a]);
      F[a] = f.get(a);
    }
    if (energy) {
      team_sum<T>(u.c);
      team_sum<T>(w.c);
      uu = u.get();
      ww = w.get();
    }
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      F[a] = f.get(a);
      team_sum_d(F[a]);
    }
    if (energy) {
      uu = u.get();
      ww = w.get();
      team_sum_d(uu);
      team_sum_d(ww);
    }
  }
  double u_out = 0.0, w_out = 0.0;
  if (active && tl == 0) {
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      S.f2[a * n + i] = F[a];
      bad |= !isfinite(F[a]);
    }
    if (kind == LJ_MID) {
      // closing half kick of this inner step + opening half kick of the next, then the drift
      double xn[3], rel[3];
      double* Xo = S.X[it.buf ^ 1];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        double vv = S.v[a * n + i] + S.dt_in * S.inv_mass * F[a];
        S.v[a * n + i] = vv;
        xn[a] = X[a * n + i] + S.dt_in * vv;
        Xo[a * n + i] = xn[a];
        bad |= !isfinite(vv);
      }
      cell_rel(S, S.pcell[i], xn, rel);
      store_pos<T>(S, it.buf ^ 1, i, rel, true);
    } else if (kind == LJ_LAST) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        double vv = S.v[a * n + i] + 0.5 * S.dt_in * S.inv_mass * F[a];
        S.v[a * n + i] = vv;
        bad |= !isfinite(vv);
      }
    }
    if (bad) atomicOr(&S.flags[FLG_ERR], ERR_NONFINITE);
    u_out = 0.5 * uu;  // every pair appears in both members' lists
    w_out = 0.5 * ww;
  }
  if (energy) {
    double us = block_sum(u_out, red);
    double ws = block_sum(w_out, red);
    if (threadIdx.x == 0) {
      atomicAdd(&S.acc[ACC_U2], us);
      atomicAdd(&S.acc[ACC_W2], ws);
    }
  }
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
  size_t table, nd, nslot, nidx, queue, sp, sl, acc, sidx, sst, total;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename T>
__host__ __device__ inline AtmLayout atm_layout(int smax) {
  using T4 = typename V4<T>::type;
  AtmLayout l;
  size_t o = 0;
  l.table = o; o = al16(o + sizeof(uint16_t) * kPairTable);
  l.nd = o; o = al16(o + sizeof(T4) * kMaxHalf * kAtmWarps);
  l.nslot = o; o = al16(o + sizeof(int) * kMaxHalf * kAtmWarps);
  l.nidx = o; o = al16(o + sizeof(int) * kMaxHalf * kAtmWarps);
  l.queue = o; o = al16(o + sizeof(unsigned) * kQueue * kAtmWarps);
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
__global__ void __launch_bounds__(kAtmThreads, 2)
    k_atm(const SysDev* __restrict__ sys, const CItem* __restrict__ items, int nitems,
          const uint16_t* __restrict__ gtable, int smax) {
  using T4 = typename V4<T>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const AtmLayout Ly = atm_layout<T>(smax);
  uint16_t* table = reinterpret_cast<uint16_t*>(smem + Ly.table);
  T4* sp = reinterpret_cast<T4*>(smem + Ly.sp);
  T4* sl = reinterpret_cast<T4*>(smem + Ly.sl);
  T* acc = reinterpret_cast<T*>(smem + Ly.acc);
  int* sidx = reinterpret_cast<int*>(smem + Ly.sidx);
  unsigned char* sst = smem + Ly.sst;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  T4* nd = reinterpret_cast<T4*>(smem + Ly.nd) + warp * kMaxHalf;
  int* nslot = reinterpret_cast<int*>(smem + Ly.nslot) + warp * kMaxHalf;
  int* nidx = reinterpret_cast<int*>(smem + Ly.nidx) + warp * kMaxHalf;
  unsigned* queue = reinterpret_cast<unsigned*>(smem + Ly.queue) + warp * kQueue;

  __shared__ int st_begin[28], st_cnt[27], st_cell[27], st_s[27];
  __shared__ double red[32];

  for (int t = threadIdx.x; t < kPairTable; t += blockDim.x) table[t] = gtable[t];

  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const CItem it = items[item];
    const SysDev& S = sys[it.sys];
    const int n = S.n, nc = S.nc, b = it.cell;
    const bool energy = (it.mode & M_ENERGY) != 0;
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
    const int nstaged = min(st_begin[27], smax);
    const int nbase = min(st_cnt[0], nstaged);
    if (st_begin[27] > smax && threadIdx.x == 0) atomicOr(&S.flags[FLG_ERR], ERR_CELL_CAP);
    // ---- stage particles (coordinates relative to the base cell centre)
    const T edge_hi = (T)S.edge;
    const T edge_lo = (T)(S.edge - (double)edge_hi);
    for (int l = warp; l < 27; l += kAtmWarps) {
      const int cnt = st_cnt[l];
      if (cnt == 0) continue;
      const int s = st_s[l];
      const int c0 = S.cell_start[st_cell[l]];
      const T ox = (T)(s % 3 - 1), oy = (T)((s / 3) % 3 - 1), oz = (T)(s / 9 - 1);
      for (int e = lane; e < cnt; e += 32) {
        const int slot = st_begin[l] + e;
        if (slot >= smax) break;
        const int p = c0 + e;
        T4 h = reinterpret_cast<const T4*>(S.pos[it.buf])[p];
        T4 hs, ls;
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
          sl[slot] = ls;
        } else {
          hs.x = h.x + (T)((double)ox * S.edge);
          hs.y = h.y + (T)((double)oy * S.edge);
          hs.z = h.z + (T)((double)oz * S.edge);
          hs.w = 0;
        }
        sp[slot] = hs;
        sidx[slot] = p;
        sst[slot] = (unsigned char)s;
        acc[slot] = (T)0;
        acc[smax + slot] = (T)0;
        acc[2 * smax + slot] = (T)0;
      }
    }
    __syncthreads();
    const T rcsq = (T)S.rc3sq;
    const T g3 = (T)S.guard3;
    const T nu = (T)S.nu;
    AccS<T> uacc;
    unsigned long long ntrip = 0;
    // ---- one warp per base particle i
    for (int is = warp; is < nbase; is += kAtmWarps) {
      const T4 pi = sp[is];
      T4 li;
      if (sizeof(T) == 4) li = sl[is];
      const int gi = sidx[is];
      // 1. half list
      int m = 0;
      for (int t0 = is + 1; t0 < nstaged; t0 += 32) {
        const int t = t0 + lane;
        bool ok = false;
        T4 d4;
        if (t < nstaged) {
          const T4 pt = sp[t];
          T dx = pt.x - pi.x, dy = pt.y - pi.y, dz = pt.z - pi.z;
          T r2 = dx * dx + dy * dy + dz * dz;
          if (r2 <= rcsq + g3) {
            if (r2 >= rcsq - g3) {
              atomicAdd(&S.ctr[CTR_GUARD], 1ull);
              ok = exact_within(X, n, gi, sidx[t], S.L, S.rc3sq);
            } else {
              ok = true;
            }
          }
          if (ok && sizeof(T) == 4) {  // full-precision difference: (hi_t - hi_i) exactly + lo terms
            const T4 lt4 = sl[t];
            float s0, e0, s1, e1, s2, e2;
            two_sum((float)pt.x, -(float)pi.x, s0, e0);
            two_sum((float)pt.y, -(float)pi.y, s1, e1);
            two_sum((float)pt.z, -(float)pi.z, s2, e2);
            dx = s0 + (e0 + ((float)lt4.x - (float)li.x));
            dy = s1 + (e1 + ((float)lt4.y - (float)li.y));
            dz = s2 + (e2 + ((float)lt4.z - (float)li.z));
            r2 = dx * dx + dy * dy + dz * dz;
          }
          d4.x = dx; d4.y = dy; d4.z = dz; d4.w = r2;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (ok) {
          const int pos = m + __popc(bal & lt);
          if (pos < kMaxHalf) {
            nd[pos] = d4;
            nslot[pos] = t;
            nidx[pos] = sidx[t];
          }
        }
        m += __popc(bal);
      }
      if (m > kMaxHalf) {
        if (lane == 0) atomicOr(&S.flags[FLG_ERR], ERR_HALF_CAP);
        m = kMaxHalf;
      }
      __syncwarp();
      // 2. neighbour pairs (j, k) of the half list, k-major through the pair table;
      //    pairs with r_jk <= r_c are compacted into the warp's queue in table order
      T fi0 = 0, fi1 = 0, fi2 = 0;
      const int np = m * (m - 1) / 2;
      int qn = 0;
      // 3. queued triplets: lane l takes a contiguous run of the queue, so its pairs mostly
      //    share k (k-major order): F_k and d_k stay in registers until k changes; F_j goes
      //    to the staged accumulator of j (targets rarely coincide across lanes)
      auto drain = [&](int count) {
        if (count <= 0) return;
        const int C = ((count + 31) >> 5) | 1;  // odd run length: lanes start in different banks
        const int e0 = lane * C, e1 = min(e0 + C, count);
        int curk = -1, sk = 0;
        T4 dk;
        T fk0 = 0, fk1 = 0, fk2 = 0;
        for (int e = e0; e < e1; ++e) {
          const unsigned entry = queue[e];
          const int j = (int)(entry & 0xffffu), k = (int)(entry >> 16);
          if (k != curk) {
            if (curk >= 0) {
              atomicAdd(&acc[sk], fk0);
              atomicAdd(&acc[smax + sk], fk1);
              atomicAdd(&acc[2 * smax + sk], fk2);
            }
            curk = k;
            dk = nd[k];
            sk = nslot[k];
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
          const int sj = nslot[j];
          atomicAdd(&acc[sj], o.fj[0]);
          atomicAdd(&acc[smax + sj], o.fj[1]);
          atomicAdd(&acc[2 * smax + sj], o.fj[2]);
          if (energy) uacc.add(o.u);
        }
        if (curk >= 0) {
          atomicAdd(&acc[sk], fk0);
          atomicAdd(&acc[smax + sk], fk1);
          atomicAdd(&acc[2 * smax + sk], fk2);
        }
        ntrip += (unsigned long long)count;
      };
      for (int p0 = 0; p0 < np; p0 += 32) {
        const int p = p0 + lane;
        bool ok = false;
        unsigned entry = 0;
        if (p < np) {
          const unsigned e = table[p];
          const int j = (int)(e & 0xffu), k = (int)(e >> 8);
          const T4 dj = nd[j], dk = nd[k];
          const T ex = dk.x - dj.x, ey = dk.y - dj.y, ez = dk.z - dj.z;
          const T c = ex * ex + ey * ey + ez * ez;
          if (c <= rcsq + g3) {
            if (c >= rcsq - g3) {
              atomicAdd(&S.ctr[CTR_GUARD], 1ull);
              ok = exact_within(X, n, nidx[j], nidx[k], S.L, S.rc3sq);
            } else {
              ok = true;
            }
          }
          entry = (unsigned)j | ((unsigned)k << 16);
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
      fi0 = warp_sum_t<T>(fi0);
      fi1 = warp_sum_t<T>(fi1);
      fi2 = warp_sum_t<T>(fi2);
      if (lane == 0) {
        atomicAdd(&acc[is], fi0);
        atomicAdd(&acc[smax + is], fi1);
        atomicAdd(&acc[2 * smax + is], fi2);
      }
      __syncwarp();
    }
    __syncthreads();
    // ---- partial forces of every staged particle, one slot per stencil offset
    T* part = reinterpret_cast<T*>(S.partial);
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

// ============================================================== combine + outer kicks
template <typename T>
__global__ void __launch_bounds__(256) k_combine(const SysDev* __restrict__ sys, const PItem* __restrict__ items) {
  __shared__ double red[32];
  const PItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  const int kind = it.mode & M_KIND_MASK;
  const bool energy = (it.mode & M_ENERGY) != 0;
  const int n = S.n, nc = S.nc;
  const int p = it.begin + threadIdx.x;
  double ek = 0.0;
  if (p < n) {
    const int cell = S.pcell[p];
    const int cx = cell % nc, cy = (cell / nc) % nc, cz = cell / (nc * nc);
    const T* part = reinterpret_cast<const T*>(S.partial);
    Acc3<T> f;
#pragma unroll 1
    for (int s = 0; s < 27; ++s) {
      const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
      const int bx = (cx - dx + nc) % nc, by = (cy - dy + nc) % nc, bz = (cz - dz + nc) % nc;
      const int base = (bz * nc + by) * nc + bx;
      if (cell < base) continue;  // the CTA of that base cell did not stage this particle's cell
      f.add(part[(3 * s + 0) * (size_t)n + p], part[(3 * s + 1) * (size_t)n + p], part[(3 * s + 2) * (size_t)n + p]);
    }
    double F[3] = {f.get(0), f.get(1), f.get(2)};
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      S.f3[a * n + p] = F[a];
      bad |= !isfinite(F[a]);
    }
    if (kind != CB_INIT) {
      const double h = 0.5 * S.dt_out * S.inv_mass;
      double vv[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) vv[a] = S.v[a * n + p] + h * F[a];  // closing outer kick
      if (energy) ek = 0.5 * S.mass * (vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]);
      if (kind == CB_CONT) {
        const double* X = S.X[it.buf];
        double* Xo = S.X[0];
        double xn[3], rel[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          vv[a] += h * F[a] + 0.5 * S.dt_in * S.inv_mass * S.f2[a * n + p];  // opening kicks of the next step
          xn[a] = X[a * n + p] + S.dt_in * vv[a];
          Xo[a * n + p] = xn[a];
        }
        cell_rel(S, cell, xn, rel);
        store_pos<T>(S, 0, p, rel, true);
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        S.v[a * n + p] = vv[a];
        bad |= !isfinite(vv[a]);
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
  const PItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  const int n = S.n;
  const int p = it.begin + threadIdx.x;
  if (p >= n) return;
  const double* X = S.X[it.buf];
  double* Xo = S.X[0];
  double xn[3], rel[3];
  bool bad = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double vv = S.v[a * n + p] + 0.5 * S.dt_out * S.inv_mass * S.f3[a * n + p] +
                0.5 * S.dt_in * S.inv_mass * S.f2[a * n + p];
    S.v[a * n + p] = vv;
    xn[a] = X[a * n + p] + S.dt_in * vv;
    Xo[a * n + p] = xn[a];
    bad |= !isfinite(vv);
  }
  cell_rel(S, S.pcell[p], xn, rel);
  store_pos<T>(S, 0, p, rel, true);
  if (bad) atomicOr(&S.flags[FLG_ERR], ERR_NONFINITE);
}

__global__ void __launch_bounds__(256) k_kinetic(const SysDev* __restrict__ sys, const PItem* __restrict__ items) {
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

int atm_configure(int smax, int precision, int* smem_bytes) {
  int bytes = (int)(precision ? atm_layout<double>(smax).total : atm_layout<float>(smax).total);
  *smem_bytes = bytes;
  int nb = 0;
  if (precision) {
    if (cudaFuncSetAttribute(k_atm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_atm<double>, kAtmThreads, bytes);
  } else {
    if (cudaFuncSetAttribute(k_atm<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_atm<float>, kAtmThreads, bytes);
  }
  return nb;
}

// ---------------------------------------------------------------- launchers
template <typename T>
void launch_lj(const Launch& L, const PItem* items, int nitems, int block) {
  if (nitems > 0) k_lj<T><<<nitems, block, 0, L.stream>>>(L.sys, items);
}
template <typename T>
void launch_atm(const Launch& L, const CItem* items, int nitems, int grid, int smax) {
  if (nitems <= 0) return;
  const int bytes = (int)atm_layout<T>(smax).total;
  k_atm<T><<<grid, kAtmThreads, bytes, L.stream>>>(L.sys, items, nitems, g_table, smax);
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
void launch_combine(const Launch& L, const PItem* items, int nitems, int block) {
  if (nitems > 0) k_combine<T><<<nitems, block, 0, L.stream>>>(L.sys, items);
}
template <typename T>
void launch_start(const Launch& L, const PItem* items, int nitems, int block) {
  if (nitems > 0) k_start<T><<<nitems, block, 0, L.stream>>>(L.sys, items);
}
void launch_kinetic(const Launch& L, const PItem* items, int nitems, int block) {
  if (nitems > 0) k_kinetic<<<nitems, block, 0, L.stream>>>(L.sys, items);
}

template void launch_lj<float>(const Launch&, const PItem*, int, int);
template void launch_lj<double>(const Launch&, const PItem*, int, int);
template void launch_combine<float>(const Launch&, const PItem*, int, int);
template void launch_combine<double>(const Launch&, const PItem*, int, int);
template void launch_start<float>(const Launch&, const PItem*, int, int);
template void launch_start<double>(const Launch&, const PItem*, int, int);
template void launch_atm<float>(const Launch&, const CItem*, int, int, int);
template void launch_atm<double>(const Launch&, const CItem*, int, int, int);

}  // namespace r3b
