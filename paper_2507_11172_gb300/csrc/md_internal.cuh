// Internal definitions shared by the respa3b CUDA sources (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace r3b {

// ---------------------------------------------------------------- capacities
constexpr int kStencil = 27;        // 3 x 3 x 3 cells: cell edge >= every cutoff
constexpr int kMaxHalf = 128;       // per-particle ATM half list (neighbours with larger sorted index)
constexpr int kNbrShift = 26;       // LJ list entry = j | (image code << 26), code = 2 bits per axis
constexpr unsigned kNbrMask = (1u << kNbrShift) - 1u;
constexpr unsigned kPadCode = 63u;  // image code of a padding entry: an offset far outside every cutoff
constexpr int kNbrPad = (int)(kPadCode << kNbrShift);  // padding entry (index 0, code 63)
constexpr int kPairTable = kMaxHalf * (kMaxHalf - 1) / 2;  // (j, k) pairs, k-major
constexpr int kAtmWarps = 8;
constexpr int kAtmThreads = 32 * kAtmWarps;
constexpr int kQueue = 256;         // per-warp queue of accepted neighbour pairs (j, k)
constexpr int kListWarpsDefault = 4;  // warps per CTA of the pair-list build (autotuned: 2, 4 or 8)
constexpr int kNearThreads = 128;   // owners (one thread each) per CTA of the near-class triplet kernel
constexpr int kHalfCap = 64;        // triplet half list per particle (neighbours above it within r_c3)

// Pair-list layout: row-major, entry t of particle i at int index i * maxnb + t (maxnb is a multiple
// of 4, so every row starts on a 16-byte boundary).
__host__ __device__ __forceinline__ size_t nbr_slot(int maxnb, int i, int t) {
  return (size_t)i * (size_t)maxnb + (size_t)t;
}
__host__ __device__ __forceinline__ size_t nbr_rows(size_t n) { return (n + 31) & ~size_t(31); }

// error bits in SysDev::flags[0]
enum : int {
  ERR_CELL_CAP = 1,   // a cell holds more particles than cap_cell
  ERR_NBR_CAP = 2,    // an LJ neighbour list overflowed
  ERR_HALF_CAP = 4,   // an ATM half list overflowed kMaxHalf
  ERR_NONFINITE = 8,  // NaN / Inf in positions, velocities or forces
  ERR_TIMEOUT = 16,   // a bounded wait on a CTA's own bulk copies gave up (cell-tile LJ kernel)
  ERR_NEAR_CAP = 32,  // distance classes: a near-class candidate list overflowed kHalfCap
  ERR_STAGE_CAP = 64, // cell-tile LJ kernel: a block's region held more particles than its staging
};

// accumulator slots in SysDev::acc (double)
enum : int { ACC_U2 = 0, ACC_W2 = 1, ACC_U3 = 2, ACC_W3 = 3, ACC_EK = 4, ACC_N = 8 };
// counter slots in SysDev::ctr (unsigned long long)
enum : int { CTR_TRIPLETS = 0, CTR_GUARD = 1, CTR_NEAR = 2, CTR_N = 4 };  // CTR_NEAR: near-class triplets
// flag slots in SysDev::flags (int)
// FLG_STATE: state transfer; FLG_DOSORT: adaptive binning, a binning is due before the next LJ evaluation
// FLG_LJSTAGE: largest staging need (particles + 1) of a cell-tile LJ block that overflowed
enum : int { FLG_ERR = 0, FLG_SKIN = 1, FLG_MAXCELL = 2, FLG_STATE = 3, FLG_DOSORT = 4, FLG_LJSTAGE = 5, FLG_N = 8 };

// Device-resident description of one system.  Kernels read it from global
// memory at run time (never from constant memory) so graphs stay valid when
// the host re-points arrays.
struct SysDev {
  // geometry
  double L, half_L, edge, inv_edge;
  double qinv;  // 2^32 / L: fixed-point position units per length unit
  int nc, ncell, n, cap_cell;
  // potentials (squared cutoffs computed on the host as rc * rc)
  double eps, sig2, rc2, rc2sq, rlistsq, nu, rc3, rc3sq, half_skin_sq;
  double guard2, guard3;  // half-width of the r^2 band re-decided in FP64 (pair / triplet)
  // integrator
  double dt_in, dt_out, inv_mass, mass;
  int maxnb, cap_stage;  // pair-list capacity per particle; staged particles per ATM CTA
  // FP32 copies of the parameters used by the FP32 kernels, computed on the host (on GB300 an
  // FP64 conversion in every thread costs as much as a pair evaluation)
  float f_edge, f_edge_lo, f_half_edge, f_rc2sq, f_guard2, f_sig2, f_eps24, f_eps4;
  float f_rc3sq, f_guard3, f_nu, f_reach2, f_half_skin_sq, f_qscale;  // f_qscale = L / 2^32
  int precision;  // 0 = FP32 forces, 1 = FP64
  int lj_tx_extra;  // failure-detection test knob: bytes the cell-tile LJ kernel announces to its copy
                    // barrier beyond those it copies (0 in normal runs; md_inject_copy_shortfall)
  // distance classes of the three-body force (all NULL / zero when off): near = triplets whose three
  // pair distances are <= r_a, integrated every s_near inner steps; far = the rest within r_c3
  double rasq, guarda;        // r_a^2 and the half-width of its FP64 re-decision band
  double dt_near;             // s_near * dt_in
  double fix_unit;            // FP32 path: force per unit of the fixed-point sums f3acc / f3nacc (3/4 nu 2^-32)
  float f_rasq, f_guarda;
  float f_nearcand;           // (r_a + skin)^2 widened by 1e-4: near-class candidate test
  int pad2_;
  int *half_a, *half_a_cnt;   // [n][kHalfCap], [n]: near-class candidates of each particle (neighbours
                              // above it within r_a + skin at the last binning), from k_listbuild
  double *f3n;                // [3][n] cached near-class force (f3 holds near + far)
  void *f3nacc;               // [n][4] like f3acc, for the near-class evaluation
  // state in cell-sorted order, double SoA [3][n] (x block, y block, z block)
  double *X[2];       // positions, ping-pong by inner-step parity
  double *v, *f2, *f3;
  double *v_alt;      // scatter target of the sort
  int *id, *id_alt;   // original index of each sorted slot
  void *pos[2];       // T4 [n]: cell-local coordinates (x, y, z relative to the cell centre of the last sort)
  void *poslo;        // T4 [n]: FP32 mode: the rounding remainder of pos at the sort
  void *ref;          // T4 [n]: pos at the sort (displacement check)
  int *pcell;         // [n] cell of the last sort
  int *cell_tmp, *rank;       // [n] binning scratch
  int *skey, *members;        // [n] binning scratch for the order within a cell (NULL: arrival order)
  int *count, *cell_start;    // [ncell], [ncell + 1]
  int *nbr, *nbr_cnt;         // pair list (layout: nbr_slot, ceil(n / 32) * 32 rows of maxnb), [n]
  int *half, *half_cnt;       // [n][kHalfCap] triplet half list of each particle (pair-list entries), [n]
  void *partial;              // T [27][3][n] per-stencil-slot ATM partial forces
  int4 *ipos;                 // [n] positions of the last binning in fixed point (box = 2^32 units;
                              // x, y, z as wrapping 32-bit integers), NULL where unused
  const double *ccen;         // [nc] cell centres along one axis: (c + 0.5) * edge
  void *f3acc;                // [n][4] rotation-kernel ATM force sums: 64-bit fixed point (FP32 path,
                              // fix_red3) or double (FP64 path); zero between evaluations (the combine
                              // kernel clears what it reads)
  double *acc;                // [ACC_N]
  unsigned long long *ctr;    // [CTR_N]
  int *flags;                 // [FLG_N]
  // batched ensembles: per-tick modes of this member (NULL for a lone system) and the
  // snapshot arrays used to replay a batch cycle
  const int *mode_tab;
  double *snap_x, *snap_v, *snap_f2, *snap_f3;
  int *snap_id, *snap_cell;
};


// particle-range work item: threads handle sorted slots [begin, begin + blockDim)
struct PItem {
  int sys;
  int begin;
  int mode;  // kernel-specific mode bits
  int buf;   // position buffer index read (and, for drifting kernels, the one written is buf_out)
};

// base-cell work item for the ATM kernel
struct CItem {
  int sys;
  int cell;
  int buf;
  int mode;
};

// per-system work item (one CTA per system)
struct SItem {
  int sys;
  int mode;
};

// mode bits
enum : int {
  M_ENERGY = 1 << 8,    // accumulate energies / virials
  M_F3READY = 1 << 9,   // combine: f3 already holds complete forces (per-particle triplet kernel)
  M_SKIP = 1 << 10,     // batch: this member does nothing in this launch
  M_F3ACC = 1 << 11,    // combine: read (and clear) the rotation kernel's per-particle sums
  M_NEAR = 1 << 12,     // distance classes: near-class kick after an LJ step (k_kick)
  M_COND = 1 << 13,     // binning kernels: run only if flags[FLG_DOSORT] is set (adaptive binning)
  M_TABLE = 1 << 30,    // batch: the low bits index SysDev::mode_tab, which holds the real mode
  M_TABLE_MASK = 0xffff,
  M_KIND_MASK = 0xff,
};
enum : int {  // LJ kinds
  LJ_INIT = 0,   // forces (and energy) only
  LJ_MID = 1,    // forces; v += dt F2 / m; x += dt v  (closing half kick of this step + opening of the next)
  LJ_LAST = 2,   // forces; v += dt/2 F2 / m (closing half kick before the ATM evaluation)
};
enum : int {  // combine kinds
  CB_INIT = 0,   // F3 only
  CB_LAST = 1,   // F3; v += dt_outer/2 F3 / m
  CB_CONT = 2,   // F3; v += dt_outer F3 / m + dt/2 F2 / m; x += dt v  (next outer step starts)
};

// mode of a work item: its own, or the member's table entry for batched launches
__device__ __forceinline__ int item_mode(const SysDev& S, int imode) {
  return (imode & M_TABLE) ? S.mode_tab[imode & M_TABLE_MASK] : imode;
}
// binning kernels: nothing to do for a skipped member, or for a conditional binning that is not due
__device__ __forceinline__ bool sort_idle(const SysDev& S, int imode) {
  const int m = item_mode(S, imode);
  return (m & M_SKIP) || ((m & M_COND) && S.flags[FLG_DOSORT] == 0);
}

// ---------------------------------------------------------------- helpers

// parameter in the kernel's precision: the FP32 copy or the FP64 original
template <typename T> struct Par;
template <> struct Par<float> {
  static __device__ __forceinline__ float edge(const SysDev& S) { return S.f_edge; }
  static __device__ __forceinline__ float edge_lo(const SysDev& S) { return S.f_edge_lo; }
  static __device__ __forceinline__ float half_edge(const SysDev& S) { return S.f_half_edge; }
  static __device__ __forceinline__ float rc2sq(const SysDev& S) { return S.f_rc2sq; }
  static __device__ __forceinline__ float guard2(const SysDev& S) { return S.f_guard2; }
  static __device__ __forceinline__ float sig2(const SysDev& S) { return S.f_sig2; }
  static __device__ __forceinline__ float eps24(const SysDev& S) { return S.f_eps24; }
  static __device__ __forceinline__ float eps4(const SysDev& S) { return S.f_eps4; }
  static __device__ __forceinline__ float rc3sq(const SysDev& S) { return S.f_rc3sq; }
  static __device__ __forceinline__ float guard3(const SysDev& S) { return S.f_guard3; }
  static __device__ __forceinline__ float nu(const SysDev& S) { return S.f_nu; }
  static __device__ __forceinline__ float reach2(const SysDev& S) { return S.f_reach2; }
  static __device__ __forceinline__ float half_skin_sq(const SysDev& S) { return S.f_half_skin_sq; }
  static __device__ __forceinline__ float rasq(const SysDev& S) { return S.f_rasq; }
  static __device__ __forceinline__ float guarda(const SysDev& S) { return S.f_guarda; }
};
template <> struct Par<double> {
  static __device__ __forceinline__ double edge(const SysDev& S) { return S.edge; }
  static __device__ __forceinline__ double edge_lo(const SysDev&) { return 0.0; }
  static __device__ __forceinline__ double half_edge(const SysDev& S) { return 0.5 * S.edge; }
  static __device__ __forceinline__ double rc2sq(const SysDev& S) { return S.rc2sq; }
  static __device__ __forceinline__ double guard2(const SysDev& S) { return S.guard2; }
  static __device__ __forceinline__ double sig2(const SysDev& S) { return S.sig2; }
  static __device__ __forceinline__ double eps24(const SysDev& S) { return 24.0 * S.eps; }
  static __device__ __forceinline__ double eps4(const SysDev& S) { return 4.0 * S.eps; }
  static __device__ __forceinline__ double rc3sq(const SysDev& S) { return S.rc3sq; }
  static __device__ __forceinline__ double guard3(const SysDev& S) { return S.guard3; }
  static __device__ __forceinline__ double nu(const SysDev& S) { return S.nu; }
  static __device__ __forceinline__ double reach2(const SysDev& S) {
    const double r = S.rc3 * (1.0 + 1e-5) + 1e-5;
    return r * r;
  }
  static __device__ __forceinline__ double half_skin_sq(const SysDev& S) { return S.half_skin_sq; }
  static __device__ __forceinline__ double rasq(const SysDev& S) { return S.rasq; }
  static __device__ __forceinline__ double guarda(const SysDev& S) { return S.guarda; }
};

template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double4_32a; };

// Fold into [0, L).  Positions are folded at every binning and move far less than L in between, so
// nearly every call finds x inside already (checked on the bit pattern with integer compares: for
// L > 0, 0 <= x < L exactly when the pattern of x lies in [0, pattern of L)) or within one box length
// of it (one exact addition or subtraction); the FP64 division, costly on GB300, is left for the rest.
__device__ __forceinline__ double wrap_box(double x, double L) {
  const long long xb = __double_as_longlong(x);
  if (xb >= 0 && xb < __double_as_longlong(L)) return x;
  double y;
  if (x >= L && x < L + L)
    y = x - L;
  else if (x < 0.0 && x >= -L)
    y = x + L;
  else
    y = x - L * floor(x / L);
  if (y >= L) y -= L;
  if (y < 0.0) y = 0.0;
  return y;
}

// Exact cutoff decision in IEEE double with the same operation order as the
// CPU reference definition: d = xj - xi; d -= L * rint(d / L) per axis;
// r2 = (dx*dx + dy*dy) + dz*dz; counts iff r2 <= rcsq.  The _rn intrinsics
// forbid fused multiply-add contraction, so the result is bit-identical to a
// plain IEEE evaluation.
// fixed-point coordinate (2^32 units per box side): the 64-bit rounding wraps modulo 2^32 for any x
__device__ __forceinline__ int to_fixed(double x, double qinv) {
  return (int)(unsigned)(unsigned long long)__double2ll_rn(x * qinv);
}

__device__ __forceinline__ bool exact_within(const double* __restrict__ X, int n, int i, int j, double L,
                                             double rcsq) {
  double r2 = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double d = __dsub_rn(X[a * n + j], X[a * n + i]);
    d = __dsub_rn(d, __dmul_rn(L, rint(__ddiv_rn(d, L))));
    r2 = (a == 0) ? __dmul_rn(d, d) : __dadd_rn(r2, __dmul_rn(d, d));
  }
  return r2 <= rcsq;
}

// ---------------------------------------------------------------- fixed-point force sums
// The FP32 triplet kernels scatter one force term per (owner, member) to the member's sum.  Those
// sums are kept in 64-bit fixed point (2^32 units per unit of the kernels' unscaled terms, which
// carry no factor nu; after Le Grand, Goetz and Walker, "SPFP: Speed without compromise", Comput.
// Phys. Commun. 184 (2013) 374): every FP32 term is rounded once to a multiple of 2^-32 and then
// added exactly, so the sum of a particle's terms is the same integer in any order (bitwise
// reproducible from run to run and whatever else shares the launch) and carries no accumulation
// error.  A term of magnitude 2^22 or more (or NaN) is not added and raises ERR_NONFINITE: it would
// take distances of about 0.2 sigma, and 2^9 such terms could overflow the sum.
constexpr float kFixOne = 4294967296.0f;  // 2^32 fixed-point units per unit of a term
constexpr float kFixLimit = 4194304.0f;   // 2^22: largest accepted term magnitude
__device__ __forceinline__ bool fix_red3(void* acc, int j, float fx, float fy, float fz) {
  if (!(fabsf(fx) < kFixLimit && fabsf(fy) < kFixLimit && fabsf(fz) < kFixLimit)) return false;
  unsigned long long* q = reinterpret_cast<unsigned long long*>(acc) + 4 * (size_t)j;
  atomicAdd(q, (unsigned long long)__float2ll_rn(fx * kFixOne));
  atomicAdd(q + 1, (unsigned long long)__float2ll_rn(fy * kFixOne));
  atomicAdd(q + 2, (unsigned long long)__float2ll_rn(fz * kFixOne));
  return true;
}
// a particle's fixed-point sum as a force (times unit), then cleared for the next evaluation
__device__ __forceinline__ void fix_take3(void* acc, int p, double unit, double f[3]) {
  long long* q = reinterpret_cast<long long*>(acc) + 4 * (size_t)p;
  const long long a = q[0], b = q[1], c = q[2];
  q[0] = q[1] = q[2] = 0;
  f[0] = (double)a * unit;
  f[1] = (double)b * unit;
  f[2] = (double)c * unit;
}

// error-free transformation s + e = a + b (Knuth TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// compensated accumulator (hi, lo) += t
struct CompF {
  float hi, lo;
  __device__ __forceinline__ void add(float t) {
    float s, e;
    two_sum(hi, t, s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum of one double per thread; every thread must call; result valid in thread 0
__device__ __forceinline__ double block_sum(double v, double* smem32) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) smem32[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    int nw = (blockDim.x + 31) >> 5;
    r = lane < nw ? smem32[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// ---------------------------------------------------------------- 27-cell stencil staging
// Stencil of cell b (called by one full warp): for l = 0..26 (offset (l % 3 - 1, l / 3 % 3 - 1,
// l / 9 - 1)) the particle count, first sorted index and the exclusive prefix of counts (staging
// offset, st_begin[27] = total), and per pair-list entry code (dx+1) | (dy+1) << 2 | (dz+1) << 4 the
// difference "staged slot - sorted index" of that cell.
__device__ __forceinline__ void stencil_table(const SysDev& S, int b, int* st_begin, int* st_cnt, int* st_c0,
                                              int* s_delta) {
  const int lane = threadIdx.x & 31, nc = S.nc;
  int cnt = 0, c0 = 0;
  if (lane < 27) {
    const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
    const int bx = b % nc, by = (b / nc) % nc, bz = b / (nc * nc);
    const int c = (((bz + dz + nc) % nc) * nc + (by + dy + nc) % nc) * nc + (bx + dx + nc) % nc;
    c0 = S.cell_start[c];
    cnt = S.cell_start[c + 1] - c0;
  }
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane < 27) {
    st_begin[lane] = incl - cnt;
    st_cnt[lane] = cnt;
    st_c0[lane] = c0;
    const unsigned code = (unsigned)(lane % 3) | ((unsigned)((lane / 3) % 3) << 2) | ((unsigned)(lane / 9) << 4);
    s_delta[code] = (incl - cnt) - c0;
  }
  if (lane == 26) st_begin[27] = incl;
}
// stencil cell of a staged slot (binary search over the staging offsets)
__device__ __forceinline__ int stencil_cell_of(const int* st_begin, int slot) {
  int lo = 0;
#pragma unroll
  for (int w = 16; w > 0; w >>= 1)
    if (lo + w < 27 && st_begin[lo + w] <= slot) lo += w;
  return lo;
}
// Positions of the 27 cells into sp[0 .. nstaged) relative to b's centre (cell-local coordinates of
// buffer buf plus the cell offset); every thread of the CTA takes slots threadIdx.x + k blockDim.x,
// loads first, so that all loads of a thread are in flight together.
template <typename T>
__device__ __forceinline__ void stage_cells(const SysDev& S, int buf, const int* st_begin, const int* st_c0,
                                            int nstaged, typename V4<T>::type* sp) {
  using T4 = typename V4<T>::type;
  constexpr int kU = 4;
  const T edge = Par<T>::edge(S);
  const T4* __restrict__ P = reinterpret_cast<const T4*>(S.pos[buf]);
  for (int s0 = threadIdx.x; s0 < nstaged; s0 += kU * blockDim.x) {
    T4 h[kU];
    int ls[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int slot = s0 + u * blockDim.x;
      ls[u] = slot < nstaged ? stencil_cell_of(st_begin, slot) : 0;
      if (slot < nstaged) h[u] = P[st_c0[ls[u]] + slot - st_begin[ls[u]]];
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int slot = s0 + u * blockDim.x;
      if (slot < nstaged) {
        const int l = ls[u];
        h[u].x += (T)(l % 3 - 1) * edge;
        h[u].y += (T)((l / 3) % 3 - 1) * edge;
        h[u].z += (T)(l / 9 - 1) * edge;
        sp[slot] = h[u];
      }
    }
  }
}

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the current device.  The
// attribute belongs to the device's context, so the largest value set so far is cached per (device,
// kernel), behind a mutex (first calls may come from several threads); never lowered.  False if the
// device refuses the size.
bool raise_smem_attr(const void* kernel, int bytes);

// message that md_last_error returns on this thread (engine.cu)
void set_last_error(const char* msg);

// ---------------------------------------------------------------- launchers
// pdl: launch with programmatic dependent launch (the kernel's blocks may become resident while the
// previous kernel of the stream drains; each such kernel starts with pdl_wait, which returns once
// that kernel has completed and its memory is visible).  Used by the captured single-system plan.
struct Launch {
  cudaStream_t stream;
  const SysDev* sys;  // device array of systems
  bool pdl = false;
};

// first statement of every kernel of the plan: wait for the previous kernel of the stream (a hardware
// dependency, no spin; a no-op when the kernel was launched without the PDL attribute)
// (The next kernel is released implicitly as this grid's blocks exit: an explicit
// griddepcontrol.launch_dependents at a kernel's start let waiting blocks of the next kernel take SM
// slots and slowed the 100k outer step from 0.856 to 0.981 ms.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_kernel(const Launch& L, void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem,
                          Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = L.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = L.pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// sort.cu
void launch_bin_count(const Launch& L, const PItem* items, int nitems, int block);
void launch_cell_order(const Launch& L, const PItem* pitems, int npitems, int block, const CItem* citems,
                       int ncitems);
void launch_snapshot(const Launch& L, const PItem* items, int nitems, int restore);
void launch_stamp(cudaStream_t s, unsigned long long* out);
void launch_sort_decide(const Launch& L);
void launch_sort_decide_all(const Launch& L, int ns);
// state.cu (one system, sys[0])
void launch_put_state(const Launch& L, int n, const double* pos, const double* vel, int cur, int full);
void launch_take_state(const Launch& L, int n, const double* src, double* out, int fold);
void launch_scan(const Launch& L, const SItem* items, int nitems);
template <typename T> void launch_scatter(const Launch& L, const PItem* items, int nitems, int block);
template <typename T> void launch_listbuild(const Launch& L, const CItem* items, int nitems, int smax, int warps);
template <typename T> void launch_atm_near(const Launch& L, const PItem* items, int nitems);
int listbuild_configure(int smax, int precision);
// forces.cu
// LJ pair forces: blocks of kLjPer threads, teams of kLjTeam threads per particle, so items of
// kLjParticles particles
#ifndef R3B_LJ_PER
#define R3B_LJ_PER 64
#endif
constexpr int kLjPer = R3B_LJ_PER;  // threads per block
#ifndef R3B_LJ_TEAM
#define R3B_LJ_TEAM 1
#endif
constexpr int kLjTeam = R3B_LJ_TEAM;  // a power of two dividing 32
constexpr int kLjParticles = kLjPer / kLjTeam;
constexpr int kLjBlocks[3] = {32, 64, 128};  // LJ block sizes the autotuner tries (kLjPer by default)
template <typename T> void launch_lj(const Launch& L, const PItem* items, int nitems, bool energy, int block);
// cell-tile LJ kernel (lj_tile.cu): one CTA of kLjtThreads threads per block of 2 x 2 x 2 cells, items
// with begin = block index; smax staged slots (lj_tile_capacity)
#ifndef R3B_LJT_THREADS
#define R3B_LJT_THREADS 256
#endif
#ifndef R3B_LJT_MINB
#define R3B_LJT_MINB 4
#endif
constexpr int kLjtThreads = R3B_LJT_THREADS;
constexpr int kLjtMinBlocks = R3B_LJT_MINB;
// staged slots of a block's 4^3 region cells: 64 cells of mean occupancy below 0.8 cap_cell, with a
// margin of several standard deviations, plus the padding slot; more raises ERR_STAGE_CAP (and a
// larger cap_cell)
inline int lj_tile_capacity(int cap_cell) { return 52 * cap_cell + 64; }
inline int lj_tile_blocks(int nc) {
  const int nb = (nc + 1) / 2;
  return nb * nb * nb;
}
template <typename T> void launch_lj_tile(const Launch& L, const PItem* items, int nitems, bool energy, int smax);
// raises the kernels' dynamic shared-memory limit; bytes, or -1 if the device refuses the size
int lj_tile_configure(int smax, int precision);
// team LJ kernel (lj_tile.cu): team lanes (4, 8 or 16) per particle, blocks of kLjmThreads threads, items
// of kLjmThreads / team particles
constexpr int kLjmThreads = 256;
#ifndef R3B_LJM_MINB
#define R3B_LJM_MINB 5
#endif
constexpr int kLjmMinBlocks = R3B_LJM_MINB;  // resident blocks per SM the registers are sized for
constexpr int kLjTeams[3] = {4, 8, 16};
template <typename T> void launch_lj_team(const Launch& L, const PItem* items, int nitems, bool energy, int team);
template <typename T> void launch_atm(const Launch& L, const CItem* items, int nitems, int grid, int smax);
// staged-particle capacity of an ATM CTA: the particles within r_c of a base cell (edge >= r_c)
// occupy at most the volume of about 21 cells (16 cells plus margin is sized for the typical mean
// occupancy); more raises ERR_CELL_CAP and a larger cap_cell
inline int atm_stage_capacity(int cap_cell) { return 16 * cap_cell + 64; }
// dynamic shared memory of the ATM kernel for smax staged particles; sets the kernel attribute
// and returns the resident CTAs per SM (0 if it does not fit)
int atm_configure(int smax, int precision, int* smem_bytes);
// per-particle ATM variant: items of 4 particles (one warp each)
template <typename T> void launch_atm_pa(const Launch& L, const PItem* items, int nitems);
constexpr int kPaPerBlock = 4;
// rotation variant: items of kRotWarps x per particles (per consecutive particles per warp; the
// autotuner picks per, rot_bases_per_item is the default item)
constexpr int kRotWarps = 4;
template <typename T> void launch_atm_rot(const Launch& L, const PItem* items, int nitems, int per);
constexpr int rot_bases_per_item(int) { return 32; }
template <typename T>
void launch_atm_table(const Launch& L, const CItem* items, int nitems, int grid, int smax, const uint16_t* table);
template <typename T> void launch_combine(const Launch& L, const PItem* items, int nitems, int block);
// all-triplet ATM forces, open boundaries (direct.cu): X, F host-order AoS device arrays, U[n]
int direct_max_n(int precision);
cudaError_t launch_atm_direct(const double* X, int n, double nu, int precision, double* F, double* U,
                              cudaStream_t s);
// RDF pair counts (observables.cu): items of 256 particles, nbins <= kRdfMaxBins shared counters
constexpr int kRdfMaxBins = 8192;
void launch_rdf(const Launch& L, const PItem* items, int nitems, int nbins, double dr, unsigned long long* counts);
// FP64 kick/drift after an LJ evaluation: items of 256 particles with the LJ kind as mode
template <typename T> void launch_kick(const Launch& L, const PItem* items, int nitems);
template <typename T> void launch_start(const Launch& L, const PItem* items, int nitems, int block);
void launch_kinetic(const Launch& L, const PItem* items, int nitems, int block);
void launch_nonfinite_check(const Launch& L, const PItem* items, int nitems, int block);
void atm_prepare_table(cudaStream_t s);

}  // namespace r3b
