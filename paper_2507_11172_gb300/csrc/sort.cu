// Cell-binning counting sort and Verlet pair-list build (linked cells, Sec. 2.2 / Sec. 4.1).
//
// Per sort: bin_count (wrap into [0, L), cell id, atomic rank within the
// cell, Morton key within the cell) -> scan (exclusive prefix over cells,
// resets counts) -> cell order (rank within the cell by key) -> scatter
// (permute positions, velocities, ids into cell order; write the cell-local
// coordinates used by the force kernels) -> listbuild (pair list with skin,
// copies the permuted state back into place).
#include "md_internal.cuh"
#include "sys_stage.cuh"

#ifndef R3B_LIST_PACKED
#define R3B_LIST_PACKED 1  // pair-list build: two candidate chunks per iteration in packed FP32x2
#endif

namespace r3b {

__global__ void k_bin_count(const SysDev* __restrict__ sys, const PItem* __restrict__ items) {
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
  if (sort_idle(S, it.mode)) return;  // block-uniform
  const int p = it.begin + threadIdx.x;
  const int n = S.n;
  const bool valid = p < n;  // no early return: every lane takes part in the match below
  int cell = -1;
  unsigned key = 0u;
  if (valid) {
    double* X = S.X[it.buf];
    const double inv8 = S.inv_edge * 8.0;  // exact scaling
    const int nc = S.nc;
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double x = wrap_box(X[a * n + p], S.L);
      X[a * n + p] = x;
      // floor(8 x / edge) >= 0: its top bits are the cell coordinate floor(x / edge) (x * 8/edge is
      // exactly 8 (x / edge) rounded), its low three bits the position on the cell's 8 x 8 x 8 grid
      const int q8 = max(0, __double2int_rz(x * inv8));
      int q = q8 & 7;
      c[a] = q8 >> 3;
      if (c[a] >= nc) {
        c[a] = nc - 1;
        q = 7;
      }
#pragma unroll
      for (int bit = 0; bit < 3; ++bit) key |= ((unsigned)(q >> bit) & 1u) << (3 * bit + a);  // Morton order
    }
    cell = (c[2] * nc + c[1]) * nc + c[0];
    S.cell_tmp[p] = cell;
    if (S.skey) S.skey[p] = (int)key;
  }
  // arrival rank within the cell: one atomic per group of lanes with the same cell (consecutive
  // particles mostly share a cell); only a bijection onto 0 .. count - 1 matters
  const unsigned peers = __match_any_sync(0xffffffffu, cell);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (valid && lane == leader) base = atomicAdd(&S.count[cell], __popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (valid) S.rank[p] = base + __popc(peers & ((1u << lane) - 1u));
}

// Order within each cell: every particle's slot in its cell's segment is replaced by its rank by
// (Morton key of its position within the cell, index), so that consecutive particles of a cell lie
// close together (their neighbour sets overlap: gathers of consecutive threads share cache lines) and
// the order no longer depends on the arrival order of the binning's atomics.
// Step 1 (per particle): the members of each cell, in arrival order.
__global__ void k_cell_members(const SysDev* __restrict__ sys, const PItem* __restrict__ items) {
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
  if (sort_idle(S, it.mode)) return;
  const int p = it.begin + threadIdx.x;
  if (p >= S.n) return;
  S.members[S.cell_start[S.cell_tmp[p]] + S.rank[p]] = p;
}
// Step 2 (one warp per cell): rank of each member by (key, index) among its cell's members.
__global__ void k_cell_rank(const SysDev* __restrict__ sys, const CItem* __restrict__ items, int nitems) {
  pdl_wait();
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= nitems) return;  // warp-uniform
  const CItem it = items[w];
  const SysDev& S = sys[it.sys];
  if (sort_idle(S, it.mode)) return;  // warp-uniform
  const int lane = threadIdx.x & 31;
  const int b = S.cell_start[it.cell], cnt = S.cell_start[it.cell + 1] - b;
  for (int a0 = 0; a0 < cnt; a0 += 32) {
    const int a = a0 + lane;
    if (a < cnt) {
      const int pa = S.members[b + a];
      const int ka = S.skey[pa];
      int r = 0;
      for (int q = 0; q < cnt; ++q) {
        const int pq = S.members[b + q];
        const int kq = S.skey[pq];
        r += (kq < ka || (kq == ka && pq < pa)) ? 1 : 0;
      }
      S.rank[pa] = r;
    }
  }
}

// One 1024-thread CTA per system: exclusive scan of count[] into
// cell_start[], count[] reset to zero, largest occupancy checked.
__global__ void __launch_bounds__(1024) k_scan(const SysDev* __restrict__ sys, const SItem* __restrict__ items) {
  pdl_wait();
  const SysDev& S = sys[items[blockIdx.x].sys];
  if (sort_idle(S, items[blockIdx.x].mode)) return;
  __shared__ int wsum[32];
  __shared__ int wmax[32];
  const int ncell = S.ncell;
  const int chunk = (ncell + blockDim.x - 1) / blockDim.x;
  const int b = threadIdx.x * chunk;
  const int e = min(b + chunk, ncell);
  int local = 0, mx = 0;
  for (int c = b; c < e; ++c) {
    int v = S.count[c];
    local += v;
    mx = max(mx, v);
  }
  // block exclusive scan of local
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  int m = mx;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 31) wsum[w] = incl;
  if (lane == 0) wmax[w] = m;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    int s = lane < nw ? wsum[lane] : 0;
    int mm = lane < nw ? wmax[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mm = max(mm, __shfl_xor_sync(0xffffffffu, mm, o));
    if (lane < nw) wsum[lane] = s;  // inclusive warp totals
    if (lane == 0) wmax[0] = mm;
  }
  __syncthreads();
  int run = incl - local + (w > 0 ? wsum[w - 1] : 0);
  for (int c = b; c < e; ++c) {
    int v = S.count[c];
    S.cell_start[c] = run;
    run += v;
    S.count[c] = 0;
  }
  if (threadIdx.x == blockDim.x - 1) S.cell_start[ncell] = run;
  if (threadIdx.x == 0) {
    int mxc = wmax[0];
    atomicMax(&S.flags[FLG_MAXCELL], mxc);
    if (mxc > S.cap_cell) atomicOr(&S.flags[FLG_ERR], ERR_CELL_CAP);
  }
}

template <typename T>
__global__ void k_scatter(const SysDev* __restrict__ sys, const PItem* __restrict__ items) {
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
  if (sort_idle(S, it.mode)) return;
  int p = it.begin + threadIdx.x;
  if (p >= S.n) return;
  const int n = S.n;
  const int cell = S.cell_tmp[p];
  const int q = S.cell_start[cell] + S.rank[p];
  const double* X = S.X[it.buf];
  double* Xa = S.X[it.buf ^ 1];
  int cx = cell % S.nc, cy = (cell / S.nc) % S.nc, cz = cell / (S.nc * S.nc);
  double ctr[3] = {(cx + 0.5) * S.edge, (cy + 0.5) * S.edge, (cz + 0.5) * S.edge};
  T hi[3], lo[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double x = X[a * n + p];
    Xa[a * n + q] = x;
    S.v_alt[a * n + q] = S.v[a * n + p];
    double rel = x - ctr[a];
    hi[a] = (T)rel;
    lo[a] = (T)(rel - (double)hi[a]);
  }
  S.id_alt[q] = S.id[p];
  S.pcell[q] = cell;
  T4 h;
  h.x = hi[0]; h.y = hi[1]; h.z = hi[2]; h.w = (T)0;
  T4 l;
  l.x = lo[0]; l.y = lo[1]; l.z = lo[2]; l.w = (T)0;
  reinterpret_cast<T4*>(S.pos[it.buf])[q] = h;
  reinterpret_cast<T4*>(S.poslo)[q] = l;
  reinterpret_cast<T4*>(S.ref)[q] = h;
  if (S.ipos) S.ipos[q] = make_int4(to_fixed(X[p], S.qinv), to_fixed(X[n + p], S.qinv), to_fixed(X[2 * n + p], S.qinv), 0);
}

// Pair list with skin, one CTA per cell b: the 27 cells around b are staged in
// shared memory with coordinates relative to b's centre; one warp per particle i
// of b tests every staged particle and ballot-compacts those within
// (r_c2 + skin)^2 (slightly widened: the list may hold a superset) into i's row.
// Entry = j | image code << 26, code = (dx+1) | (dy+1) << 2 | (dz+1) << 4 for the
// cell offset from i's cell to j's cell.  The same pass writes i's triplet half list
// (S.half, S.half_cnt): the entries j with r_ij <= r_c3 (guard band around r_c3^2
// re-decided in FP64 with the CPU definition's operation order) that lie above i in the
// order "cell layer along z, then fixed-point z, then sorted index", which makes i the
// owner of every triplet whose other two members are in that list.  With distance classes on, the
// same pass keeps the near-class candidates (S.half_a): the entries above i within r_a + skin (a
// superset test, widened by 1e-4).  The CTA also moves the permuted state of b's particles back into
// place.  FP32: registers sized for 1024 resident threads per SM (64 per thread).
template <typename T, int kListWarps>
__global__ void __launch_bounds__(32 * kListWarps, sizeof(T) == 4 ? 32 / kListWarps : 1)
    k_listbuild(const SysDev* __restrict__ sys, const CItem* __restrict__ items, int smax) {
  pdl_wait();
  using T4 = typename V4<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T4* sp = reinterpret_cast<T4*>(smem_raw);
  int* sj = reinterpret_cast<int*>(sp + smax);
  int* sqz = sj + smax;  // fixed-point z of each staged particle
  __shared__ int st_begin[28], st_cnt[27], st_cell[27];
  const CItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  if (sort_idle(S, it.mode)) return;
  const int b = it.cell, nc = S.nc, n = S.n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  if (warp == 0) {
    int cnt = 0;
    if (lane < 27) {
      const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
      const int bx = b % nc, by = (b / nc) % nc, bz = b / (nc * nc);
      const int c = (((bz + dz + nc) % nc) * nc + (by + dy + nc) % nc) * nc + (bx + dx + nc) % nc;
      cnt = S.cell_start[c + 1] - S.cell_start[c];
      st_cnt[lane] = cnt;
      st_cell[lane] = c;
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
  if (st_begin[27] > smax && threadIdx.x == 0) atomicOr(&S.flags[FLG_ERR], ERR_CELL_CAP);
  const T edge = (T)S.edge;
  const T4* __restrict__ P = reinterpret_cast<const T4*>(S.pos[it.buf]);
  // staging: thread t takes slots t, t + blockDim, ...; the loads of kU slots are issued together
  // before their stores (one round trip to L2 for the kU slots instead of one per stencil cell)
  {
    constexpr int kU = 4;
    __shared__ int st_c0[27];
    if (threadIdx.x < 27) st_c0[threadIdx.x] = S.cell_start[st_cell[threadIdx.x]];
    __syncthreads();
    for (int s0 = threadIdx.x; s0 < nstaged; s0 += kU * (int)blockDim.x) {
      T4 h[kU];
      int qz[kU], l[kU], g[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int slot = s0 + u * (int)blockDim.x;
        l[u] = slot < nstaged ? stencil_cell_of(st_begin, slot) : 0;
        g[u] = st_c0[l[u]] + slot - st_begin[l[u]];
        if (slot < nstaged) {
          h[u] = P[g[u]];
          qz[u] = S.ipos[g[u]].z;
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int slot = s0 + u * (int)blockDim.x;
        if (slot < nstaged) {
          const int lu = l[u];
          h[u].x += (T)(lu % 3 - 1) * edge;
          h[u].y += (T)((lu / 3) % 3 - 1) * edge;
          h[u].z += (T)(lu / 9 - 1) * edge;
          sp[slot] = h[u];
          // image code: cell offset (dx, dy, dz) + 1 per axis in 2 bits each
          const unsigned code = (unsigned)(lu % 3) | ((unsigned)((lu / 3) % 3) << 2) | ((unsigned)(lu / 9) << 4);
          sj[slot] = (int)((unsigned)g[u] | (code << kNbrShift));
          sqz[slot] = qz[u];
        }
      }
    }
  }
  __syncthreads();
  const T rl = (T)(S.rlistsq * (1.0 + 1e-5));
  const int nbase = min(st_cnt[13], max(0, nstaged - st_begin[13]));
  const int i0 = S.cell_start[b];
  const double* Xa = S.X[it.buf ^ 1];
  double* X = S.X[it.buf];
  // staged slot of a list entry: its index plus the offset of its stencil cell in the staging
  __shared__ int st_delta[27];
  if (threadIdx.x < 27) st_delta[threadIdx.x] = st_begin[threadIdx.x] - S.cell_start[st_cell[threadIdx.x]];
  __syncthreads();
  const T rc3 = (T)S.rc3sq, g3 = (T)S.guard3;
  const int b9 = st_begin[9];  // first staged slot of the base cell's own layer
  for (int ib = warp; ib < nbase; ib += kListWarps) {
    const int islot = st_begin[13] + ib;
    const int i = i0 + ib;
    const T4 pi = sp[islot];
    int cnt = 0;
    int* const row = S.nbr + nbr_slot(S.maxnb, i, 0);
    // pass 1: every staged particle within the list radius, in staging order; FP32: two chunks of 32
    // candidates per iteration, their distance tests in packed FP32x2 arithmetic.  The row starts with
    // the entries of the lower cell layer (staged slots below b9), none of which is above i: cnt0, the
    // entries from the chunks that lie wholly below b9, is where pass 2 may start.
    auto compact = [&](const int t, const bool ok) {
      const unsigned bal = __ballot_sync(0xffffffffu, ok);
      const int pos = cnt + __popc(bal & lt);
      if (ok && pos < S.maxnb) row[pos] = sj[t];
      cnt += __popc(bal);
    };
    int t0 = 0, cnt0 = 0;
    if constexpr (sizeof(T) == 4 && R3B_LIST_PACKED) {
      const float2 px = make_float2(-pi.x, -pi.x), py = make_float2(-pi.y, -pi.y), pz = make_float2(-pi.z, -pi.z);
      auto two = [&](const int t0) {
        const int ta = t0 + lane, tb = ta + 32;
        const float4 qa = sp[ta];
        const float4 qb = tb < nstaged ? sp[tb] : make_float4(1e3f, 1e3f, 1e3f, 0.f);
        const float2 dx = __fadd2_rn(make_float2(qa.x, qb.x), px);
        const float2 dy = __fadd2_rn(make_float2(qa.y, qb.y), py);
        const float2 dz = __fadd2_rn(make_float2(qa.z, qb.z), pz);
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        compact(ta, ta != islot && r2.x <= rl);
        compact(tb, tb < nstaged && tb != islot && r2.y <= rl);
      };
      for (; t0 + 32 < nstaged && t0 + 64 <= b9; t0 += 64) two(t0);
      cnt0 = cnt;
      for (; t0 + 32 < nstaged; t0 += 64) two(t0);
    }
    auto one = [&](const int t0) {
      const int t = t0 + lane;
      bool ok = false;
      if (t < nstaged && t != islot) {
        const T4 q = sp[t];
        const T dx = q.x - pi.x, dy = q.y - pi.y, dz = q.z - pi.z;
        ok = dx * dx + dy * dy + dz * dz <= rl;
      }
      compact(t, ok);
    };
    if constexpr (!(sizeof(T) == 4 && R3B_LIST_PACKED)) {
      for (; t0 < nstaged && t0 + 32 <= b9; t0 += 32) one(t0);
      cnt0 = cnt;
    }
    for (; t0 < nstaged; t0 += 32) one(t0);
    if (lane == 0) {
      if (cnt > S.maxnb) atomicOr(&S.flags[FLG_ERR], ERR_NBR_CAP);
      S.nbr_cnt[i] = min(cnt, S.maxnb);
    }
    cnt = min(cnt, S.maxnb);
    cnt0 = min(cnt0, cnt);
    __syncwarp();  // the row written above is read back below by other lanes
    // pass 2: the triplet half list among the list entries
    const int qzi = sqz[islot];
    int* hrow = S.half + (size_t)i * kHalfCap;
    int mh = 0, ma = 0;
    for (int t0 = cnt0; t0 < cnt; t0 += 32) {
      const int t = t0 + lane;
      bool half = false, band = false, cand = false;
      unsigned e = 0u;
      if (t < cnt) {
        e = (unsigned)row[t];
        const unsigned code = e >> kNbrShift;
        const int l = (int)(code & 3u) + 3 * (int)((code >> 2) & 3u) + 9 * (int)(code >> 4);
        const int slot = (int)(e & kNbrMask) + st_delta[l];
        // above i: the upper cell layer, or the same layer with larger fixed-point z (ties: index)
        const unsigned lay = code >> 4;
        const int dqz = (int)((unsigned)sqz[slot] - (unsigned)qzi);
        const bool above = lay == 2u || (lay == 1u && (dqz > 0 || (dqz == 0 && (int)(e & kNbrMask) > i)));
        if (above) {
          const T4 q = sp[slot];
          const T dx = q.x - pi.x, dy = q.y - pi.y, dz = q.z - pi.z;
          const T r2 = dx * dx + dy * dy + dz * dz;
          half = r2 <= rc3 - g3;
          band = !half && r2 <= rc3 + g3;
          cand = r2 <= (T)S.f_nearcand;  // distance classes: near-class candidate (superset test)
        }
      }
      if (__any_sync(0xffffffffu, band)) {
        if (band) {
          atomicAdd(&S.ctr[CTR_GUARD], 1ull);
          half = exact_within(Xa, n, i, (int)(e & kNbrMask), S.L, S.rc3sq);
        }
      }
      const unsigned balh = __ballot_sync(0xffffffffu, half);
      const int hpos = mh + __popc(balh & lt);
      if (half && hpos < kHalfCap) hrow[hpos] = (int)e;
      mh += __popc(balh);
      if (S.half_a) {
        const unsigned bala = __ballot_sync(0xffffffffu, cand);
        const int apos = ma + __popc(bala & lt);
        if (cand && apos < kHalfCap) S.half_a[(size_t)i * kHalfCap + apos] = (int)e;
        ma += __popc(bala);
      }
    }
    if (lane == 0) {  // more than kHalfCap: the triplet kernels report ERR_HALF_CAP / ERR_NEAR_CAP
      S.half_cnt[i] = mh;
      if (S.half_a) S.half_a_cnt[i] = ma;
    }
  }
  // every particle of b: permuted state back into place
  for (int ib = threadIdx.x; ib < st_cnt[13]; ib += blockDim.x) {
    const int i = i0 + ib;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      X[a * n + i] = Xa[a * n + i];
      S.v[a * n + i] = S.v_alt[a * n + i];
    }
    S.id[i] = S.id_alt[i];
  }
}

// save (mode 0) or restore (mode 1) the state a batch cycle changes: positions of buffer
// it.buf, velocities, cached forces, ids and cells
__global__ void k_snapshot(const SysDev* __restrict__ sys, const PItem* __restrict__ items, int restore) {
  const PItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  const int p = it.begin + threadIdx.x;
  if (p >= S.n) return;
  const int n = S.n;
  double* X = S.X[it.buf];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int q = a * n + p;
    if (restore) {
      X[q] = S.snap_x[q];
      S.v[q] = S.snap_v[q];
      S.f2[q] = S.snap_f2[q];
      S.f3[q] = S.snap_f3[q];
    } else {
      S.snap_x[q] = X[q];
      S.snap_v[q] = S.v[q];
      S.snap_f2[q] = S.f2[q];
      S.snap_f3[q] = S.f3[q];
    }
  }
  if (restore) {
    S.id[p] = S.snap_id[p];
    S.pcell[p] = S.snap_cell[p];
  } else {
    S.snap_id[p] = S.id[p];
    S.snap_cell[p] = S.pcell[p];
  }
}

// device time stamp (ns) at a point of the stream
__global__ void k_stamp(unsigned long long* out) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *out = t;
}

// Adaptive binning: a binning is due before the next LJ evaluation if some particle has moved more than
// skin / 2 since the last one (flag set by the drifts); the decision is taken once, for every kernel of
// the binning, and the drift flag starts over.
__global__ void k_sort_decide(const SysDev* __restrict__ sys) {
  pdl_wait();
  const SysDev& S = sys[0];
  S.flags[FLG_DOSORT] = S.flags[FLG_SKIN] != 0 ? 1 : 0;
  S.flags[FLG_SKIN] = 0;
}
void launch_sort_decide(const Launch& L) { launch_kernel(L, k_sort_decide, 1, 1, 0, L.sys); }
// the same for every member of a batch (one thread each)
__global__ void k_sort_decide_all(const SysDev* __restrict__ sys, int ns) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ns) return;
  const SysDev& S = sys[j];
  S.flags[FLG_DOSORT] = S.flags[FLG_SKIN] != 0 ? 1 : 0;
  S.flags[FLG_SKIN] = 0;
}
void launch_sort_decide_all(const Launch& L, int ns) {
  if (ns > 0) k_sort_decide_all<<<(ns + 127) / 128, 128, 0, L.stream>>>(L.sys, ns);
}

void launch_snapshot(const Launch& L, const PItem* items, int nitems, int restore) {
  if (nitems > 0) k_snapshot<<<nitems, 256, 0, L.stream>>>(L.sys, items, restore);
}
void launch_stamp(cudaStream_t s, unsigned long long* out) { k_stamp<<<1, 1, 0, s>>>(out); }

void launch_cell_order(const Launch& L, const PItem* pitems, int npitems, int block, const CItem* citems,
                       int ncitems) {
  if (npitems <= 0 || ncitems <= 0) return;
  launch_kernel(L, k_cell_members, npitems, block, 0, L.sys, pitems);
  launch_kernel(L, k_cell_rank, (ncitems + 7) / 8, 256, 0, L.sys, citems, ncitems);
}
void launch_bin_count(const Launch& L, const PItem* items, int nitems, int block) {
  if (nitems > 0) launch_kernel(L, k_bin_count, nitems, block, 0, L.sys, items);
}
void launch_scan(const Launch& L, const SItem* items, int nitems) {
  if (nitems > 0) launch_kernel(L, k_scan, nitems, 1024, 0, L.sys, items);
}
template <typename T>
void launch_scatter(const Launch& L, const PItem* items, int nitems, int block) {
  if (nitems > 0) launch_kernel(L, k_scatter<T>, nitems, block, 0, L.sys, items);
}
template <typename T, int kW>
static void launch_listbuild_w(const Launch& L, const CItem* items, int nitems, int smax, int bytes) {
  launch_kernel(L, k_listbuild<T, kW>, nitems, 32 * kW, bytes, L.sys, items, smax);
}
// warps: warps per CTA (kListWarpChoices), a runtime choice of the autotuner
template <typename T>
void launch_listbuild(const Launch& L, const CItem* items, int nitems, int smax, int warps) {
  if (nitems <= 0) return;
  const int bytes = (int)(smax * (sizeof(typename V4<T>::type) + 2 * sizeof(int)));
  if (warps == 2)
    launch_listbuild_w<T, 2>(L, items, nitems, smax, bytes);
  else if (warps == 8)
    launch_listbuild_w<T, 8>(L, items, nitems, smax, bytes);
  else
    launch_listbuild_w<T, 4>(L, items, nitems, smax, bytes);
}
// the kernels' dynamic shared-memory limit is shared by every system on a device: only ever raised
int listbuild_configure(int smax, int precision) {
  const int bytes = (int)(smax * ((precision ? sizeof(double4_32a) : sizeof(float4)) + 2 * sizeof(int)));
  const void* kerns[2][3] = {{(const void*)k_listbuild<float, 2>, (const void*)k_listbuild<float, 4>,
                              (const void*)k_listbuild<float, 8>},
                             {(const void*)k_listbuild<double, 2>, (const void*)k_listbuild<double, 4>,
                              (const void*)k_listbuild<double, 8>}};
  for (const void* k : kerns[precision ? 1 : 0])
    if (!raise_smem_attr(k, bytes)) return -1;
  return bytes;
}
template void launch_scatter<float>(const Launch&, const PItem*, int, int);
template void launch_scatter<double>(const Launch&, const PItem*, int, int);
template void launch_listbuild<float>(const Launch&, const CItem*, int, int, int);
template void launch_listbuild<double>(const Launch&, const CItem*, int, int, int);

}  // namespace r3b
