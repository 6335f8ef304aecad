// Host runtime and C ABI of respa3b: device state of a system, the launch
// plan of Algorithm 2 (arXiv 2507.11172, Sec. 4.1) captured as CUDA graphs,
// snapshot/replay when a particle outruns the pair-list skin (with adaptive
// binning afterwards), the triplet-kernel autotuner, distance classes, and the
// batched ensemble / serving engine.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/respa3b.h"
#include "md_internal.cuh"

using namespace r3b;

namespace {

thread_local std::string g_last_error;

md_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? MD_ERR_OOM : MD_ERR_CUDA;
}

#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

constexpr int kBlock = 256;
constexpr int kSafeCalls = 4;  // initial run of calls started in safe mode after a skin replay

int device_sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// one device allocation carved into aligned sub-arrays
struct Arena {
  char* base = nullptr;
  size_t size = 0, used = 0;
  size_t reserve(size_t bytes) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + bytes;
    return off;
  }
};

}  // namespace

void r3b::set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

// ====================================================================== system
struct md_system {
  // description
  int64_t n = 0;
  double L = 0, mass = 1.0;
  int precision = MD_FP32;
  double eps = 1.0, sigma = 1.0, rc2 = 2.5, nu = 0.0, rc3 = 2.5, skin = 0.3;
  // distance classes of the three-body force (r_a = 0: off, plain Algorithm 2)
  double r_a = 0.0;
  int s_near = 0;
  // grid and capacities
  int nc = 0, ncell = 0, cap_cell = 0, maxnb = 0;
  double edge = 0;
  // device memory
  char* mem = nullptr;
  size_t mem_bytes = 0;
  SysDev h{};              // host copy of the device descriptor
  SysDev* d_sys = nullptr;  // device copy (inside mem)
  // snapshot for replay
  double *snap_x = nullptr, *snap_v = nullptr, *snap_f2 = nullptr, *snap_f3 = nullptr, *snap_f3n = nullptr;
  int *snap_id = nullptr, *snap_cell = nullptr;
  // work items
  std::map<std::tuple<int, int, int>, PItem*> pitems;  // (kernel tag, mode, buf) -> device array
  std::map<std::tuple<int, int>, CItem*> citems;        // (mode, buf)
  SItem* sitem = nullptr;
  SItem* sitem_cond = nullptr;
  std::vector<void*> item_allocs;
  int nblocks = 0;
  // execution
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // second stream of the captured plan: the closing LJ step of each outer step runs on it beside the
  // triplet kernel (F2(x) and F3(x) do not depend on each other); fork / join events
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int cur = 0;               // position buffer holding the current state
  bool forces_valid = false;
  bool energy_valid = false;
  int atm_smem = 0, atm_grid = 0;
  int atm_variant = -1;       // 0: cell kernel with Newton-3 scatter, 1: per-particle kernel, -1: tune
  int atm_variant_req = -1;   // requested by md_set_atm_kernel (-1 = autotune)
  int nblocks_pa = 0;
  int nblocks_rot = 0;
  int rot_per = rot_bases_per_item(0) / kRotWarps;  // rotation kernel: bases per warp in a work item
  int lj_block = kLjPer;                 // LJ row kernel: threads (particles) per block
  int lj_kernel = 1;                     // LJ kernel: 0 row kernel (global gathers), 1 cell-tile kernel,
                                         // 2 team kernel (lj_team lanes per particle)
  int lj_kernel_req = -1;                // md_set_lj_kernel (-1: autotuned)
  int lj_team = 8;                       // team kernel: lanes per particle (autotuned: 4, 8 or 16)
  bool lj_tile_ok = false;               // the cell-tile kernel fits in shared memory for cap_cell
  int list_warps = kListWarpsDefault;    // pair-list build: warps per CTA
  bool tuned_from_cache = false;         // the last tuning reused another system's choices
  int lj_block_req = 0, list_warps_req = 0, rot_per_req = 0;  // md_set_shapes (0: autotuned)
  std::map<std::tuple<int, int, int, int, int>, cudaGraphExec_t> graphs;  // (n_outer, k, cur, safe, profile)
  // host mirrors
  int* h_flags = nullptr;       // pinned [FLG_N]
  double* h_acc = nullptr;      // pinned [ACC_N]
  unsigned long long* h_ctr = nullptr;  // pinned [CTR_N]
  // stats
  md_stats stats{};
  bool profile = false;
  std::vector<cudaEvent_t> events;
  double e_kin = 0, u2 = 0, u3 = 0, w2 = 0, w3 = 0;
  // batch membership
  md_batch* batch = nullptr;
  // in a batch, or being admitted to one: LJ forces come from the batch's LJ kernel (the row kernel) from
  // the admission's first evaluation on, so a request gives the same bits in any mix
  bool batch_lj = false;
  int lj_tx_extra = 0;  // md_inject_copy_shortfall (failure-detection tests)
  // calls since the last skin replay that started in safe mode (0: start with the normal plan), and the
  // length of such a run before the normal plan is tried again
  int safe_calls = 0, safe_span = 4;
  // batch member: the last drift of the previous cycle moved a particle more than skin / 2
  bool skin_carry = false;
  // deferred allocation: state kept on the host until first use
  bool deferred = false;
  std::vector<double> host_x, host_v;
};

namespace {

enum KTag { T_BIN = 1, T_SCATTER, T_LIST, T_LJ, T_COMB, T_START, T_KIN, T_ATMPA, T_ATMROT, T_KICK, T_ATMNEAR, T_LJT,
            T_LJM4, T_LJM8, T_LJM16 };  // T_LJM<team>: team LJ kernel items
int ljm_tag(int team) { return team == 4 ? T_LJM4 : (team == 16 ? T_LJM16 : T_LJM8); }
int ljm_per(int tag) { return kLjmThreads / (tag == T_LJM4 ? 4 : (tag == T_LJM16 ? 16 : 8)); }

void free_items(md_system* s) {
  for (void* p : s->item_allocs) cudaFree(p);
  s->item_allocs.clear();
  s->pitems.clear();
  s->citems.clear();
  s->sitem = nullptr;
  s->sitem_cond = nullptr;
}

void clear_graphs(md_system* s) {
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
  s->graphs.clear();
}

void free_device(md_system* s) {
  clear_graphs(s);
  free_items(s);
  if (s->mem) cudaFree(s->mem);
  s->mem = nullptr;
  s->mem_bytes = 0;
  s->d_sys = nullptr;
}

md_status check_geometry(md_system* s) {
  if (!(s->eps > 0) || !(s->sigma > 0) || !(s->rc2 > 0) || !(s->rc3 > 0) || !(s->skin >= 0) || !(s->nu >= 0))
    return MD_ERR_ARG;
  double reach = std::max(s->rc2 + s->skin, s->rc3);
  if (!(s->L > 3.0 * reach)) return MD_ERR_BOX_TOO_SMALL;
  return MD_OK;
}

// binning grid: cells of edge >= max(r_c2 + skin, r_c3), at least 3 per side
void choose_grid(md_system* s) {
  double reach = std::max(s->rc2 + s->skin, s->rc3);
  int nc = (int)floor(s->L / reach);
  if (nc < 3) nc = 3;
  if (nc > 1024) nc = 1024;
  s->nc = nc;
  s->ncell = nc * nc * nc;
  s->edge = s->L / nc;
  double mean = (double)s->n / s->ncell;
  if (s->cap_cell == 0) s->cap_cell = std::max(16, (int)ceil(1.25 * mean + 10.0));
  double rho = (double)s->n / (s->L * s->L * s->L);
  double rl = s->rc2 + s->skin;
  double nl = rho * 4.18879020478639 * rl * rl * rl;
  if (s->maxnb == 0) s->maxnb = std::max(32, (int)ceil(1.35 * nl + 24.0));
  s->maxnb = std::min(s->maxnb, (int)s->n);
  s->maxnb = (s->maxnb + 3) & ~3;  // rows start on 16-byte boundaries (bulk row copies)
}

size_t arena_bytes(const md_system* s);

md_status alloc_device(md_system* s) {
  free_device(s);
  const size_t n = (size_t)s->n;
  const size_t t4 = s->precision ? sizeof(double4_32a) : sizeof(float4);
  const size_t tsz = s->precision ? 8 : 4;
  Arena a;
  size_t o_sys = a.reserve(sizeof(SysDev));
  size_t o_X0 = a.reserve(24 * n), o_X1 = a.reserve(24 * n);
  size_t o_v = a.reserve(24 * n), o_f2 = a.reserve(24 * n), o_f3 = a.reserve(24 * n), o_va = a.reserve(24 * n);
  size_t o_id = a.reserve(4 * n), o_ida = a.reserve(4 * n);
  size_t o_p0 = a.reserve(t4 * n), o_p1 = a.reserve(t4 * n), o_plo = a.reserve(t4 * n), o_ref = a.reserve(t4 * n);
  size_t o_pcell = a.reserve(4 * n), o_ctmp = a.reserve(4 * n), o_rank = a.reserve(4 * n);
  size_t o_skey = a.reserve(4 * n), o_memb = a.reserve(4 * n);
  size_t o_count = a.reserve(4 * (size_t)s->ncell), o_cstart = a.reserve(4 * ((size_t)s->ncell + 1));
  size_t o_nbr = a.reserve(4 * (size_t)s->maxnb * nbr_rows(n)), o_nbc = a.reserve(4 * n);
  size_t o_half = a.reserve(4 * (size_t)kHalfCap * n), o_hc = a.reserve(4 * n);
  size_t o_part = a.reserve(tsz * 27 * 3 * n);
  size_t o_f3a = a.reserve(32 * n);  // [n][4] fixed-point (FP32) or double (FP64) sums
  size_t o_ipos = a.reserve(16 * n);
  size_t o_ccen = a.reserve(8 * (size_t)s->nc);
  size_t o_acc = a.reserve(8 * ACC_N), o_ctr = a.reserve(8 * CTR_N), o_flg = a.reserve(4 * FLG_N);
  size_t o_sx = a.reserve(24 * n), o_sv = a.reserve(24 * n), o_sf2 = a.reserve(24 * n), o_sf3 = a.reserve(24 * n);
  size_t o_sid = a.reserve(4 * n), o_scell = a.reserve(4 * n);
  const bool classes = s->r_a > 0;
  size_t o_halfa = 0, o_hca = 0, o_f3n = 0, o_f3na = 0, o_sf3n = 0;
  if (classes) {
    o_halfa = a.reserve(4 * (size_t)kHalfCap * n);
    o_hca = a.reserve(4 * n);
    o_f3n = a.reserve(24 * n);
    o_f3na = a.reserve(32 * n);
    o_sf3n = a.reserve(24 * n);
  }
  char* m = nullptr;
  cudaError_t e = cudaMalloc(&m, a.used);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "cudaMalloc(system)");
  }
  s->mem = m;
  s->mem_bytes = a.used;
  CK(cudaMemsetAsync(m, 0, a.used, s->stream));
  SysDev& h = s->h;
  memset(&h, 0, sizeof(h));
  h.X[0] = (double*)(m + o_X0);
  h.X[1] = (double*)(m + o_X1);
  h.v = (double*)(m + o_v);
  h.f2 = (double*)(m + o_f2);
  h.f3 = (double*)(m + o_f3);
  h.v_alt = (double*)(m + o_va);
  h.id = (int*)(m + o_id);
  h.id_alt = (int*)(m + o_ida);
  h.pos[0] = m + o_p0;
  h.pos[1] = m + o_p1;
  h.poslo = m + o_plo;
  h.ref = m + o_ref;
  h.pcell = (int*)(m + o_pcell);
  h.cell_tmp = (int*)(m + o_ctmp);
  h.rank = (int*)(m + o_rank);
  h.skey = (int*)(m + o_skey);
  h.members = (int*)(m + o_memb);
  h.count = (int*)(m + o_count);
  h.cell_start = (int*)(m + o_cstart);
  h.nbr = (int*)(m + o_nbr);
  h.nbr_cnt = (int*)(m + o_nbc);
  h.half = (int*)(m + o_half);
  h.half_cnt = (int*)(m + o_hc);
  h.partial = m + o_part;
  h.f3acc = m + o_f3a;
  h.ipos = (int4*)(m + o_ipos);
  if (classes) {
    h.half_a = (int*)(m + o_halfa);
    h.half_a_cnt = (int*)(m + o_hca);
    h.f3n = (double*)(m + o_f3n);
    h.f3nacc = m + o_f3na;
  }
  s->snap_f3n = classes ? (double*)(m + o_sf3n) : nullptr;
  {
    std::vector<double> cen(s->nc);
    for (int c = 0; c < s->nc; ++c) cen[c] = (c + 0.5) * s->edge;
    CK(cudaMemcpyAsync(m + o_ccen, cen.data(), 8 * cen.size(), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    h.ccen = (const double*)(m + o_ccen);
  }
  h.acc = (double*)(m + o_acc);
  h.ctr = (unsigned long long*)(m + o_ctr);
  h.flags = (int*)(m + o_flg);
  s->d_sys = (SysDev*)(m + o_sys);
  s->snap_x = (double*)(m + o_sx);
  s->snap_v = (double*)(m + o_sv);
  s->snap_f2 = (double*)(m + o_sf2);
  s->snap_f3 = (double*)(m + o_sf3);
  s->snap_id = (int*)(m + o_sid);
  s->snap_cell = (int*)(m + o_scell);
  h.snap_x = s->snap_x;
  h.snap_v = s->snap_v;
  h.snap_f2 = s->snap_f2;
  h.snap_f3 = s->snap_f3;
  h.snap_id = s->snap_id;
  h.snap_cell = s->snap_cell;
  h.mode_tab = nullptr;
  return MD_OK;
}

// device bytes alloc_device would reserve (grid and capacities chosen as for a real build)
size_t arena_bytes(const md_system* s0) {
  md_system tmp;
  tmp.n = s0->n;
  tmp.L = s0->L;
  tmp.rc2 = s0->rc2;
  tmp.rc3 = s0->rc3;
  tmp.skin = s0->skin;
  choose_grid(&tmp);
  const size_t n = (size_t)tmp.n;
  const size_t t4 = s0->precision ? sizeof(double4_32a) : sizeof(float4);
  const size_t tsz = s0->precision ? 8 : 4;
  Arena a;
  a.reserve(sizeof(SysDev));
  for (int i = 0; i < 6; ++i) a.reserve(24 * n);
  a.reserve(4 * n);
  a.reserve(4 * n);
  for (int i = 0; i < 4; ++i) a.reserve(t4 * n);
  for (int i = 0; i < 5; ++i) a.reserve(4 * n);
  a.reserve(4 * (size_t)tmp.ncell);
  a.reserve(4 * ((size_t)tmp.ncell + 1));
  a.reserve(4 * (size_t)tmp.maxnb * nbr_rows(n));
  a.reserve(4 * n);
  a.reserve(4 * (size_t)kHalfCap * n);
  a.reserve(4 * n);
  a.reserve(tsz * 27 * 3 * n);
  a.reserve(32 * n);
  a.reserve(16 * n);
  a.reserve(8 * (size_t)tmp.nc);
  a.reserve(8 * ACC_N);
  a.reserve(8 * CTR_N);
  a.reserve(4 * FLG_N);
  for (int i = 0; i < 4; ++i) a.reserve(24 * n);
  a.reserve(4 * n);
  a.reserve(4 * n);
  if (s0->r_a > 0) {  // distance classes
    a.reserve(4 * (size_t)kHalfCap * n);
    a.reserve(4 * n);
    a.reserve(24 * n);
    a.reserve(32 * n);
    a.reserve(24 * n);
  }
  // work-item arrays (about 30 particle-block variants and 4 cell variants)
  return a.used + 30 * sizeof(PItem) * (n / 32 + 2) + 4 * sizeof(CItem) * (size_t)tmp.ncell;
}

// refresh the parameter fields of the descriptor and upload it
md_status upload_desc(md_system* s, double dt_in, double dt_out) {
  SysDev& h = s->h;
  h.L = s->L;
  h.half_L = 0.5 * s->L;
  h.edge = s->edge;
  h.inv_edge = 1.0 / s->edge;
  h.qinv = 4294967296.0 / s->L;
  h.nc = s->nc;
  h.ncell = s->ncell;
  h.n = (int)s->n;
  h.cap_cell = s->cap_cell;
  h.eps = s->eps;
  h.sig2 = s->sigma * s->sigma;
  h.rc2 = s->rc2;
  h.rc2sq = s->rc2 * s->rc2;
  double rl = s->rc2 + s->skin;
  h.rlistsq = rl * rl;
  h.nu = s->nu;
  h.rc3 = s->rc3;
  h.rc3sq = s->rc3 * s->rc3;
  h.half_skin_sq = 0.25 * s->skin * s->skin;
  // FP32 cutoff decisions are exact outside this band of r^2 around r_c^2 (bound on the
  // FP32 error of r^2 from cell-local coordinates: a few 1e-6 * r_c^2; 2e-5 r_c^2 kept)
  double gfac = s->precision ? 1e-12 : 2e-5;
  h.guard2 = gfac * std::max(1.0, h.rc2sq);
  h.guard3 = gfac * std::max(1.0, h.rc3sq);
  h.dt_in = dt_in;
  h.dt_out = dt_out;
  h.rasq = s->r_a * s->r_a;
  h.guarda = gfac * std::max(1.0, h.rasq);
  h.dt_near = s->s_near * dt_in;
  h.fix_unit = 0.75 * s->nu / 4294967296.0;  // unscaled FP32 triplet terms, 2^32 units each
  h.f_rasq = (float)h.rasq;
  h.f_guarda = (float)h.guarda;
  h.f_nearcand = (float)((s->r_a + s->skin) * (s->r_a + s->skin) * (1.0 + 1e-4));
  h.mass = s->mass;
  h.inv_mass = 1.0 / s->mass;
  h.maxnb = s->maxnb;
  h.cap_stage = atm_stage_capacity(s->cap_cell);
  h.precision = s->precision;
  h.lj_tx_extra = s->lj_tx_extra;
  {
    const double r = h.rc3 * (1.0 + 1e-5) + 1e-5;
    h.f_edge = (float)h.edge;
    h.f_edge_lo = (float)(h.edge - (double)h.f_edge);
    h.f_half_edge = (float)(0.5 * h.edge);
    h.f_rc2sq = (float)h.rc2sq;
    h.f_guard2 = (float)h.guard2;
    h.f_sig2 = (float)h.sig2;
    h.f_eps24 = (float)(24.0 * h.eps);
    h.f_eps4 = (float)(4.0 * h.eps);
    h.f_rc3sq = (float)h.rc3sq;
    h.f_guard3 = (float)h.guard3;
    h.f_nu = (float)h.nu;
    h.f_reach2 = (float)(r * r);
    h.f_half_skin_sq = (float)h.half_skin_sq;
    h.f_qscale = (float)(s->L / 4294967296.0);
  }
  CK(cudaMemcpyAsync(s->d_sys, &h, sizeof(SysDev), cudaMemcpyHostToDevice, s->stream));
  return MD_OK;
}

template <typename I>
I* upload_items(md_system* s, const std::vector<I>& v) {
  I* d = nullptr;
  if (cudaMalloc(&d, sizeof(I) * std::max<size_t>(1, v.size())) != cudaSuccess) return nullptr;
  s->item_allocs.push_back(d);
  cudaMemcpyAsync(d, v.data(), sizeof(I) * v.size(), cudaMemcpyHostToDevice, s->stream);
  return d;
}

// number of items of an SM-interleaved particle launch of nb blocks (a multiple of the SM count)
int padded_blocks(int nb) {
  const int nsm = std::max(1, device_sm_count());
  return nsm * ((nb + nsm - 1) / nsm);
}

PItem* pitems_for(md_system* s, int tag, int mode, int buf) {
  auto key = std::make_tuple(tag, mode, buf);
  auto it = s->pitems.find(key);
  if (it != s->pitems.end()) return it->second;
  std::vector<PItem> v;
  const int per = (tag == T_LJ)      ? s->lj_block
                  : (tag == T_LJT)    ? 1
                  : (tag >= T_LJM4)   ? ljm_per(tag)
                  : (tag == T_ATMPA)  ? kPaPerBlock
                  : (tag == T_ATMROT) ? kRotWarps * s->rot_per
                  : (tag == T_ATMNEAR) ? kNearThreads
                                      : kBlock;
  const int nb = (tag == T_LJ)       ? (int)((s->n + s->lj_block - 1) / s->lj_block)
                 : (tag == T_LJT)    ? lj_tile_blocks(s->nc)
                 : (tag >= T_LJM4)   ? (int)((s->n + ljm_per(tag) - 1) / ljm_per(tag))
                 : (tag == T_ATMPA)  ? s->nblocks_pa
                 : (tag == T_ATMROT) ? s->nblocks_rot
                 : (tag == T_ATMNEAR) ? (int)((s->n + kNearThreads - 1) / kNearThreads)
                                     : s->nblocks;
  if (tag == T_LJ || tag == T_ATMROT || tag == T_KICK || tag == T_ATMNEAR || tag >= T_LJM4) {
    // Gather kernels: the block scheduler hands consecutive blocks to different SMs, so blocks
    // b, b + nsm, b + 2 nsm, ... tend to share an SM.  Giving those blocks adjacent particle ranges
    // keeps each SM's neighbour gathers within one region of the box (L1 reuse); the order of the
    // items changes nothing else.
    const int nsm = std::max(1, device_sm_count());
    const int per_sm = (nb + nsm - 1) / nsm;
    for (int b = 0; b < nsm * per_sm; ++b) {  // padded_blocks(nb) items; those past n do nothing
      const int r = (b % nsm) * per_sm + b / nsm;
      v.push_back(PItem{0, r * per, mode, buf});
    }
  } else {
    for (int b = 0; b < nb; ++b) v.push_back(PItem{0, b * per, mode, buf});
  }
  PItem* d = upload_items(s, v);
  s->pitems[key] = d;
  return d;
}

CItem* citems_for(md_system* s, int mode, int buf) {
  auto key = std::make_tuple(mode, buf);
  auto it = s->citems.find(key);
  if (it != s->citems.end()) return it->second;
  std::vector<CItem> v;
  v.reserve(s->ncell);
  for (int c = 0; c < s->ncell; ++c) v.push_back(CItem{0, c, buf, mode});
  CItem* d = upload_items(s, v);
  s->citems[key] = d;
  return d;
}

// all item variants a call can use, created before any graph capture
md_status prepare_items(md_system* s) {
  s->nblocks = (int)((s->n + kBlock - 1) / kBlock);
  s->nblocks_pa = (int)((s->n + kPaPerBlock - 1) / kPaPerBlock);
  s->nblocks_rot = (int)((s->n + kRotWarps * s->rot_per - 1) / (kRotWarps * s->rot_per));
  for (int b = 0; b < 2; ++b) {
    pitems_for(s, T_BIN, 0, b);
    pitems_for(s, T_SCATTER, 0, b);
    pitems_for(s, T_BIN, M_COND, b);
    pitems_for(s, T_SCATTER, M_COND, b);
    citems_for(s, M_COND, b);
    pitems_for(s, T_START, 0, b);
    for (int e = 0; e < 2; ++e) {
      int E = e ? M_ENERGY : 0;
      pitems_for(s, T_LJ, LJ_INIT | E, b);
      pitems_for(s, T_LJ, LJ_MID | E, b);
      pitems_for(s, T_LJ, LJ_LAST | E, b);
      pitems_for(s, T_LJT, LJ_INIT | E, b);
      pitems_for(s, T_LJT, LJ_MID | E, b);
      pitems_for(s, T_LJT, LJ_LAST | E, b);
      for (int team : kLjTeams)
        for (int kind : {LJ_INIT, LJ_MID, LJ_LAST}) pitems_for(s, ljm_tag(team), kind | E, b);
      pitems_for(s, T_KICK, LJ_MID, b);
      pitems_for(s, T_KICK, LJ_LAST, b);
      pitems_for(s, T_COMB, CB_INIT | E, b);
      pitems_for(s, T_COMB, CB_LAST | E, b);
      pitems_for(s, T_COMB, CB_CONT | E, b);
      pitems_for(s, T_COMB, CB_INIT | E | M_F3READY, b);
      pitems_for(s, T_COMB, CB_LAST | E | M_F3READY, b);
      pitems_for(s, T_COMB, CB_CONT | E | M_F3READY, b);
      pitems_for(s, T_COMB, CB_INIT | E | M_F3ACC, b);
      pitems_for(s, T_COMB, CB_LAST | E | M_F3ACC, b);
      pitems_for(s, T_COMB, CB_CONT | E | M_F3ACC, b);
      pitems_for(s, T_ATMPA, E, b);
      pitems_for(s, T_ATMROT, E, b);
      citems_for(s, E, b);
    }
    if (s->r_a > 0) {  // distance classes
      pitems_for(s, T_KICK, LJ_MID | M_NEAR, b);
      pitems_for(s, T_ATMNEAR, 0, b);
    }
  }
  pitems_for(s, T_KIN, 0, 0);
  if (!s->sitem) {
    std::vector<SItem> v{SItem{0, 0}};
    s->sitem = upload_items(s, v);
  }
  if (!s->sitem_cond) {
    std::vector<SItem> v{SItem{0, M_COND}};
    s->sitem_cond = upload_items(s, v);
  }
  CK(cudaStreamSynchronize(s->stream));
  for (auto& kv : s->pitems)
    if (!kv.second) return MD_ERR_OOM;
  for (auto& kv : s->citems)
    if (!kv.second) return MD_ERR_OOM;
  if (!s->sitem || !s->sitem_cond) return MD_ERR_OOM;
  return MD_OK;
}

md_status configure_atm(md_system* s) {
  atm_prepare_table(s->stream);
  int bytes = 0;
  int per_sm = atm_configure(atm_stage_capacity(s->cap_cell), s->precision, &bytes);
  if (per_sm <= 0) {
    g_last_error = "ATM kernel does not fit in shared memory for cap_cell=" + std::to_string(s->cap_cell);
    return MD_ERR_CAPACITY;
  }
  s->atm_smem = bytes;
  if (listbuild_configure(27 * s->cap_cell, s->precision) < 0) {
    g_last_error = "pair-list build does not fit in shared memory for cap_cell=" + std::to_string(s->cap_cell);
    return MD_ERR_CAPACITY;
  }
  s->atm_grid = std::min(s->ncell, per_sm * device_sm_count());
  // the cell-tile LJ kernel where its staging fits in shared memory (else the row kernel)
  s->lj_tile_ok = lj_tile_configure(lj_tile_capacity(s->cap_cell), s->precision) > 0;
  if (!s->lj_tile_ok) s->lj_kernel = 0;
  return MD_OK;
}

// (re)build everything that depends on the grid and the capacities
md_status rebuild(md_system* s, bool keep_state) {
  std::vector<double> x, v;
  std::vector<int> id;
  const size_t n = (size_t)s->n;
  if (keep_state && s->mem) {  // save the current state (sorted order) on the host
    x.resize(3 * n);
    v.resize(3 * n);
    id.resize(n);
    CK(cudaMemcpyAsync(x.data(), s->h.X[s->cur], 24 * n, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(v.data(), s->h.v, 24 * n, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(id.data(), s->h.id, 4 * n, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
  }
  choose_grid(s);
  md_status st = alloc_device(s);
  if (st != MD_OK) return st;
  st = upload_desc(s, 0.0, 0.0);
  if (st != MD_OK) return st;
  if (!keep_state || x.empty()) {  // fresh arena: zero state in the caller's order
    std::vector<int> ident(n);
    for (size_t i = 0; i < n; ++i) ident[i] = (int)i;
    s->cur = 0;
    CK(cudaMemcpyAsync(s->h.id, ident.data(), 4 * n, cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
  }
  if (keep_state && !x.empty()) {
    s->cur = 0;
    CK(cudaMemcpyAsync(s->h.X[0], x.data(), 24 * n, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->h.v, v.data(), 24 * n, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->h.id, id.data(), 4 * n, cudaMemcpyHostToDevice, s->stream));
  }
  st = prepare_items(s);
  if (st != MD_OK) return st;
  st = configure_atm(s);
  if (st != MD_OK) return st;
  s->forces_valid = false;
  s->energy_valid = false;
  s->stats.cells_per_side = s->nc;
  s->atm_variant = -1;  // re-tune for the new grid / parameters
  memset(s->h_ctr, 0, 8 * CTR_N);  // the device counters restart at zero with the new arena
  return MD_OK;
}

// ---------------------------------------------------------------- launch plan
struct Plan {
  md_system* s;
  Launch L;
  // binning, pair list and half lists; cond: only if the last drifts moved a particle more than
  // skin / 2 since the previous binning (decided on the device, adaptive binning)
  template <typename T>
  void sort(int buf, bool cond = false) {
    const int c = cond ? M_COND : 0;
    if (cond) launch_sort_decide(L);
    launch_bin_count(L, pitems_for(s, T_BIN, c, buf), s->nblocks, kBlock);
    launch_scan(L, cond ? s->sitem_cond : s->sitem, 1);
    launch_cell_order(L, pitems_for(s, T_BIN, c, buf), s->nblocks, kBlock, citems_for(s, c, buf), s->ncell);
    launch_scatter<T>(L, pitems_for(s, T_SCATTER, c, buf), s->nblocks, kBlock);
    launch_listbuild<T>(L, citems_for(s, c, buf), s->ncell, 27 * s->cap_cell, s->list_warps);
  }
  // LJ forces and the velocity-Verlet kick/drift; with near = true (distance classes, LJ_MID) the
  // near-class triplets are evaluated between the two and their kicks join the LJ kick
  template <typename T>
  void lj(int kind, int buf, bool energy, bool near = false) { lj_on<T>(L, kind, buf, energy, near); }
  template <typename T>
  void lj_on(const Launch& Lx, int kind, int buf, bool energy, bool near = false) {
    const int ljk = s->batch_lj ? 0 : s->lj_kernel;
    if (ljk == 2) {
      const int tag = ljm_tag(s->lj_team);
      launch_lj_team<T>(Lx, pitems_for(s, tag, kind | (energy ? M_ENERGY : 0), buf),
                        padded_blocks((int)((s->n + ljm_per(tag) - 1) / ljm_per(tag))), energy, s->lj_team);
    } else if (ljk == 1)
      launch_lj_tile<T>(Lx, pitems_for(s, T_LJT, kind | (energy ? M_ENERGY : 0), buf), lj_tile_blocks(s->nc), energy,
                        lj_tile_capacity(s->cap_cell));
    else
      launch_lj<T>(Lx, pitems_for(s, T_LJ, kind | (energy ? M_ENERGY : 0), buf),
                   padded_blocks((int)((s->n + s->lj_block - 1) / s->lj_block)), energy, s->lj_block);
    if (near) atm_near<T>(buf);
    if (kind != LJ_INIT)
      launch_kick<T>(Lx, pitems_for(s, T_KICK, kind | (near ? M_NEAR : 0), buf), padded_blocks(s->nblocks));
  }
  // distance classes: the near-class triplets at the current positions
  template <typename T>
  void atm_near(int buf) {
    launch_atm_near<T>(L, pitems_for(s, T_ATMNEAR, 0, buf), padded_blocks((int)((s->n + kNearThreads - 1) / kNearThreads)));
  }
  // every triplet within r_c3, with the chosen kernel
  template <typename T>
  void atm_all(int buf, bool energy) {
    if (s->atm_variant == 2)
      launch_atm_rot<T>(L, pitems_for(s, T_ATMROT, energy ? M_ENERGY : 0, buf), padded_blocks(s->nblocks_rot),
                        s->rot_per);
    else if (s->atm_variant == 1)
      launch_atm_pa<T>(L, pitems_for(s, T_ATMPA, energy ? M_ENERGY : 0, buf), s->nblocks_pa);
    else
      launch_atm<T>(L, citems_for(s, energy ? M_ENERGY : 0, buf), s->ncell, s->atm_grid,
                    atm_stage_capacity(s->cap_cell));
  }
  template <typename T>
  void atm(int buf, bool energy, int ev) {
    if (ev >= 0) cudaEventRecord(s->events[2 * ev], L.stream);
    atm_all<T>(buf, energy);
    if (ev >= 0) cudaEventRecord(s->events[2 * ev + 1], L.stream);
    if (s->r_a > 0) atm_near<T>(buf);  // distance classes: the near class of the same configuration
  }
  template <typename T>
  void combine(int kind, int buf, bool energy) {
    const int ready = (s->atm_variant == 1) ? M_F3READY : (s->atm_variant == 2 ? M_F3ACC : 0);
    launch_combine<T>(L, pitems_for(s, T_COMB, kind | ready | (energy ? M_ENERGY : 0), buf), s->nblocks, kBlock);
  }
  template <typename T>
  void start(int buf) {
    launch_start<T>(L, pitems_for(s, T_START, 0, buf), s->nblocks, kBlock);
  }
  void kinetic() { launch_kinetic(L, pitems_for(s, T_KIN, 0, 0), s->nblocks, kBlock); }
  void zero_energy() { cudaMemsetAsync(s->h.acc, 0, 8 * ACC_N, L.stream); }
};

// initial forces F2b(x), F3b(x) and energies at the current positions (buffer cur)
template <typename T>
void enqueue_init(Plan& P, int ev) {
  md_system* s = P.s;
  P.zero_energy();
  P.sort<T>(s->cur);
  P.lj<T>(LJ_INIT, s->cur, true);
  P.atm<T>(s->cur, true, ev);
  P.combine<T>(CB_INIT, s->cur, false);
  P.kinetic();
}

// Algorithm 2 for n_outer outer steps of k inner steps, starting from buffer cur
template <typename T>
void enqueue_steps(Plan& P, int n_outer, int k, int cur, bool safe, bool profile) {
  if (n_outer <= 0) return;
  P.start<T>(cur);  // i % s == 0: F3 half kick; first inner half kick and drift
  for (int o = 0; o < n_outer; ++o) {
    const bool last = (o == n_outer - 1);
    if (last) P.zero_energy();
    for (int t = 0; t < k; ++t) {
      const int b = t & 1;
      // distance classes: iteration t closes a block of s_near inner steps
      const bool near = P.s->r_a > 0 && t < k - 1 && (t + 1) % P.s->s_near == 0;
      // binning + pair list at the outer boundary; in safe mode (after a skin replay) also before any
      // inner step whose positions have moved more than skin / 2 since the last binning
      if (t == k - 1)
        P.sort<T>(b);
      else if (safe)
        P.sort<T>(b, true);
      if (t < k - 1) P.lj<T>(LJ_MID, b, false, near);
    }
    const int b = (k - 1) & 1;
    // F2b(x^{i+1}) with its closing half kick and F3b(x^{i+1}) ((i+1) % s == 0) are independent: the LJ
    // step runs on the side stream beside the triplet kernel, joined before the outer kicks.  A profiled
    // pass launches them one after the other, so the triplet kernel's events time it alone.
    md_system* s = P.s;
    if (profile) {
      P.lj<T>(LJ_LAST, b, last);
      P.atm<T>(b, last, o);
    } else {
      cudaEventRecord(s->ev_fork, P.L.stream);
      cudaStreamWaitEvent(s->side, s->ev_fork, 0);
      P.lj_on<T>(Launch{s->side, P.L.sys}, LJ_LAST, b, last);
      cudaEventRecord(s->ev_join, s->side);
      P.atm<T>(b, last, -1);
      cudaStreamWaitEvent(P.L.stream, s->ev_join, 0);
    }
    P.combine<T>(last ? CB_LAST : CB_CONT, b, last);
  }
}

md_status read_flags(md_system* s) {
  CK(cudaMemcpyAsync(s->h_flags, s->h.flags, 4 * FLG_N, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(s->h_acc, s->h.acc, 8 * ACC_N, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(s->h_ctr, s->h.ctr, 8 * CTR_N, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return MD_OK;
}

md_status clear_flags(md_system* s) {
  CK(cudaMemsetAsync(s->h.flags, 0, 4 * FLG_N, s->stream));
  return MD_OK;
}

md_status snapshot(md_system* s, bool save) {
  const size_t n = (size_t)s->n;
  auto cp = [&](void* dst, const void* src, size_t b) {
    return cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToDevice, s->stream);
  };
  if (save) {
    CK(cp(s->snap_x, s->h.X[s->cur], 24 * n));
    CK(cp(s->snap_v, s->h.v, 24 * n));
    CK(cp(s->snap_f2, s->h.f2, 24 * n));
    CK(cp(s->snap_f3, s->h.f3, 24 * n));
    if (s->snap_f3n) CK(cp(s->snap_f3n, s->h.f3n, 24 * n));
    CK(cp(s->snap_id, s->h.id, 4 * n));
    CK(cp(s->snap_cell, s->h.pcell, 4 * n));
  } else {
    CK(cp(s->h.X[s->cur], s->snap_x, 24 * n));
    CK(cp(s->h.v, s->snap_v, 24 * n));
    CK(cp(s->h.f2, s->snap_f2, 24 * n));
    CK(cp(s->h.f3, s->snap_f3, 24 * n));
    if (s->snap_f3n) CK(cp(s->h.f3n, s->snap_f3n, 24 * n));
    CK(cp(s->h.id, s->snap_id, 4 * n));
    CK(cp(s->h.pcell, s->snap_cell, 4 * n));
  }
  return MD_OK;
}

md_status ensure_events(md_system* s, int count) {
  while ((int)s->events.size() < count) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    s->events.push_back(e);
  }
  return MD_OK;
}

// run n_outer steps (n_outer == 0 with init only), as a cached CUDA graph
md_status run_plan(md_system* s, int n_outer, int k, bool init, bool safe) {
  const bool prof = s->profile;
  const int nev = prof ? std::max(1, n_outer) + 1 : 0;
  md_status st = ensure_events(s, 2 * nev);
  if (st != MD_OK) return st;
  Plan P{s, Launch{s->stream, s->d_sys}};
  P.L.pdl = !prof;  // the captured plan: programmatic dependent launches (section "launchers")
  auto key = std::make_tuple(init ? -1 - n_outer : n_outer, k, s->cur, safe ? 1 : 0, prof ? 1 : 0);
  if (prof) {
    // profiling: direct launches so the ATM kernel can be timed with events recorded on the
    // stream (events recorded by graph nodes cannot be read back with cudaEventElapsedTime)
    if (s->precision) {
      if (init) enqueue_init<double>(P, nev - 1);
      enqueue_steps<double>(P, n_outer, k, s->cur, safe, true);
    } else {
      if (init) enqueue_init<float>(P, nev - 1);
      enqueue_steps<float>(P, n_outer, k, s->cur, safe, true);
    }
    CK(cudaGetLastError());
    return MD_OK;
  }
  cudaGraphExec_t exec = nullptr;
  auto it = s->graphs.find(key);
  if (it != s->graphs.end()) {
    exec = it->second;
  } else {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    if (s->precision) {
      if (init) enqueue_init<double>(P, -1);
      enqueue_steps<double>(P, n_outer, k, s->cur, safe, false);
    } else {
      if (init) enqueue_init<float>(P, -1);
      enqueue_steps<float>(P, n_outer, k, s->cur, safe, false);
    }
    cudaError_t e = cudaStreamEndCapture(s->stream, &g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    if (s->graphs.size() > 32) clear_graphs(s);
    s->graphs[key] = exec;
  }
  CK(cudaGraphLaunch(exec, s->stream));
  return MD_OK;
}

md_status finish_call(md_system* s, int n_outer) {
  md_status st = read_flags(s);
  if (st != MD_OK) return st;
  if (s->profile) {
    for (int o = 0; o < n_outer; ++o) {
      float ms = 0;
      cudaError_t e = cudaEventElapsedTime(&ms, s->events[2 * o], s->events[2 * o + 1]);
      if (e == cudaSuccess) {
        s->stats.atm_ms_total += ms;
        s->stats.atm_timed += 1;
      } else {
        g_last_error = std::string("cudaEventElapsedTime: ") + cudaGetErrorString(e);
        cudaGetLastError();  // non-fatal: do not leave the error pending for other CUDA users
      }
    }
  }
  return MD_OK;
}

md_status status_from_flags(md_system* s) {
  int err = s->h_flags[FLG_ERR];
  if (err & ERR_NONFINITE) return MD_ERR_NONFINITE;
  if (err & ERR_NEAR_CAP) {
    g_last_error = "distance classes: more than 64 near-class candidates (neighbours above within r_a + skin)";
    return MD_ERR_CAPACITY;
  }
  if (err & ERR_TIMEOUT) {
    g_last_error = "LJ cell-tile kernel: a bounded wait for its shared-memory copies gave up";
    return MD_ERR_DEVICE_TIMEOUT;
  }
  if (err & (ERR_CELL_CAP | ERR_NBR_CAP | ERR_HALF_CAP | ERR_STAGE_CAP)) return MD_ERR_CAPACITY;
  return MD_OK;
}

bool variant_allowed(const md_system* s, int v) {
  // the per-particle and rotation kernels read neighbours from the pair list: r_c3 <= r_c2 + skin
  return v == 0 || ((v == 1 || v == 2) && s->rc3 <= s->rc2 + s->skin);
}

// rotation kernel work items of kRotWarps x per bases (the items of the previous shape are dropped
// from the cache; their memory is released with the other items)
md_status set_rot_per(md_system* s, int per) {
  if (per == s->rot_per) return MD_OK;
  s->rot_per = per;
  s->nblocks_rot = (int)((s->n + kRotWarps * per - 1) / (kRotWarps * per));
  for (auto it = s->pitems.begin(); it != s->pitems.end();) {
    if (std::get<0>(it->first) == T_ATMROT)
      it = s->pitems.erase(it);
    else
      ++it;
  }
  for (int b = 0; b < 2; ++b)
    for (int e = 0; e < 2; ++e)
      if (!pitems_for(s, T_ATMROT, e ? M_ENERGY : 0, b)) return MD_ERR_OOM;
  CK(cudaStreamSynchronize(s->stream));
  clear_graphs(s);
  return MD_OK;
}

// LJ work items of `block` particles (the items of the previous size are dropped from the cache; their
// memory is released with the other items)
md_status set_lj_block(md_system* s, int block) {
  if (block == s->lj_block) return MD_OK;
  s->lj_block = block;
  for (auto it = s->pitems.begin(); it != s->pitems.end();) {
    if (std::get<0>(it->first) == T_LJ)
      it = s->pitems.erase(it);
    else
      ++it;
  }
  for (int b = 0; b < 2; ++b)
    for (int e = 0; e < 2; ++e)
      for (int kind : {LJ_INIT, LJ_MID, LJ_LAST})
        if (!pitems_for(s, T_LJ, kind | (e ? M_ENERGY : 0), b)) return MD_ERR_OOM;
  CK(cudaStreamSynchronize(s->stream));
  clear_graphs(s);
  return MD_OK;
}

// Autotuner (the paper's AutoPas tunes its traversal at run time, Sec. 4.1; here the launch shapes).
// Choices: the triplet kernel (cell, per-particle or rotation kernel) and the rotation kernel's work-item
// shape (4, 8 or 16 bases per warp), the LJ block size (32, 64 or 128 particles) and the pair-list
// build's warps per CTA (2, 4 or 8).  None of them changes a result bit except the triplet kernel
// variant (within the FP tolerance).  After one initial evaluation (binning, pair list, forces) each
// candidate is launched four times on the same configuration with CUDA events around each launch
// (the first launch warms caches) and the fastest is kept.  The choices are cached for the process,
// keyed on (device, N in half-octave buckets, density in steps of 0.025, r_c2, r_c3, skin, precision,
// distance classes on/off): a later system with the same key skips the trials.
struct TuneChoice {
  int variant, rot_per, lj_block, list_warps, lj_kernel, lj_team;
};
using TuneKey = std::tuple<int, int, int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune_cache;

TuneKey tune_key(const md_system* s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
  const double rho = (double)s->n / (s->L * s->L * s->L);
  return std::make_tuple(dev, (int)floor(2.0 * log2((double)s->n)), (int)lround(rho * 40.0),
                         (int)lround(s->rc2 * 1000.0), (int)lround(s->rc3 * 1000.0), (int)lround(s->skin * 1000.0),
                         s->precision, s->r_a > 0 ? 1 : 0);
}

md_status tune_apply(md_system* s, const TuneChoice& c) {
  const int req = s->atm_variant_req;
  s->atm_variant = req >= 0 ? (variant_allowed(s, req) ? req : 0) : (variant_allowed(s, c.variant) ? c.variant : 0);
  md_status st = set_rot_per(s, s->rot_per_req ? s->rot_per_req : c.rot_per);
  if (st == MD_OK) st = set_lj_block(s, s->lj_block_req ? s->lj_block_req : c.lj_block);
  if (st != MD_OK) return st;
  s->list_warps = s->list_warps_req ? s->list_warps_req : c.list_warps;
  s->lj_kernel = s->lj_kernel_req >= 0 ? s->lj_kernel_req : c.lj_kernel;
  if (s->lj_kernel == 1 && !s->lj_tile_ok) s->lj_kernel = 0;
  s->lj_team = c.lj_team;
  clear_graphs(s);
  return MD_OK;
}

// mean of launches 2-4 of `launch` (CUDA events on the system's stream)
template <typename F>
md_status time_launches(md_system* s, F launch, float* ms_out) {
  float tot = 0.f;
  for (int r = 0; r < 4; ++r) {
    CK(cudaEventRecord(s->events[0], s->stream));
    launch();
    CK(cudaEventRecord(s->events[1], s->stream));
    CK(cudaEventSynchronize(s->events[1]));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, s->events[0], s->events[1]));
    if (r > 0) tot += ms;
  }
  *ms_out = tot / 3.f;
  return MD_OK;
}

md_status tune(md_system* s) {
  const TuneKey key = tune_key(s);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      s->tuned_from_cache = true;
      return tune_apply(s, it->second);
    }
  }
  s->tuned_from_cache = false;
  md_status st = upload_desc(s, 0.0, 0.0);
  if (st != MD_OK) return st;
  st = ensure_events(s, 2);
  if (st != MD_OK) return st;
  Plan P{s, Launch{s->stream, s->d_sys}};
  const bool prof = s->profile;
  s->profile = false;
  clear_graphs(s);
  s->atm_variant = 0;
  st = run_plan(s, 0, 1, true, false);  // binning + pair list at the current positions
  if (st != MD_OK) return st;
  TuneChoice best{0, s->rot_per, s->lj_block, s->list_warps, 0, s->lj_team};
  float tbest = 1e30f;
  // triplet kernel: (variant, bases per warp of the rotation kernel's work items)
#ifdef R3B_ROT_SHAPE_ONLY  // build-time knob: a single rotation shape instead of the tuned choice
  const int cand[][2] = {{0, 0}, {1, 0}, {2, R3B_ROT_SHAPE_ONLY}};
#else
  const int cand[][2] = {{0, 0}, {1, 0}, {2, 4}, {2, 8}, {2, 16}};
#endif
  for (const auto& c : cand) {
    const int v = c[0];
    if (!variant_allowed(s, v)) continue;
    s->atm_variant = v;
    if (v == 2) {
      st = set_rot_per(s, c[1]);
      if (st != MD_OK) return st;
    }
    float ms = 0.f;
    st = time_launches(s, [&] {
      if (s->precision) P.atm_all<double>(s->cur, false); else P.atm_all<float>(s->cur, false);
    }, &ms);
    if (st != MD_OK) return st;
    if (ms < tbest) {
      tbest = ms;
      best.variant = v;
      if (v == 2) best.rot_per = c[1];
    }
  }
  // the rotation kernel's trial launches left sums that no combine cleared
  CK(cudaMemsetAsync(s->h.f3acc, 0, 32 * (size_t)s->n, s->stream));
  // LJ block size (forces only; every block size gives the same forces)
  tbest = 1e30f;
  for (int block : kLjBlocks) {
    st = set_lj_block(s, block);
    if (st != MD_OK) return st;
    float ms = 0.f;
    st = time_launches(s, [&] {
      const PItem* items = pitems_for(s, T_LJ, LJ_INIT, s->cur);
      const int nb = padded_blocks((int)((s->n + block - 1) / block));
      if (s->precision) launch_lj<double>(P.L, items, nb, false, block); else launch_lj<float>(P.L, items, nb, false, block);
    }, &ms);
    if (st != MD_OK) return st;
    if (ms < tbest) {
      tbest = ms;
      best.lj_block = block;
    }
  }
  // the cell-tile LJ kernel against the best row-kernel block (same forces within rounding)
  if (s->lj_tile_ok) {
    float ms = 0.f;
    st = time_launches(s, [&] {
      const PItem* items = pitems_for(s, T_LJT, LJ_INIT, s->cur);
      const int smax = lj_tile_capacity(s->cap_cell);
      if (s->precision)
        launch_lj_tile<double>(P.L, items, lj_tile_blocks(s->nc), false, smax);
      else
        launch_lj_tile<float>(P.L, items, lj_tile_blocks(s->nc), false, smax);
    }, &ms);
    if (st != MD_OK) return st;
    if (ms < tbest) {
      tbest = ms;
      best.lj_kernel = 1;
    }
  }
  // the team kernel with 4, 8 and 16 lanes per particle (its fastest team is kept even where another
  // kernel wins: md_set_lj_kernel(2) then uses it)
  float tteam = 1e30f;
  for (int team : kLjTeams) {
    float ms = 0.f;
    st = time_launches(s, [&] {
      const int tag = ljm_tag(team);
      const PItem* items = pitems_for(s, tag, LJ_INIT, s->cur);
      const int nb = padded_blocks((int)((s->n + ljm_per(tag) - 1) / ljm_per(tag)));
      if (s->precision)
        launch_lj_team<double>(P.L, items, nb, false, team);
      else
        launch_lj_team<float>(P.L, items, nb, false, team);
    }, &ms);
    if (st != MD_OK) return st;
    if (ms < tteam) {
      tteam = ms;
      best.lj_team = team;
    }
  }
  if (tteam < tbest) {
    tbest = tteam;
    best.lj_kernel = 2;
  }
  // pair-list build warps per CTA (the lists are the same for every choice)
  tbest = 1e30f;
  for (int wps : {2, 4, 8}) {
    float ms = 0.f;
    st = time_launches(s, [&] {
      const CItem* items = citems_for(s, 0, s->cur);
      if (s->precision)
        launch_listbuild<double>(P.L, items, s->ncell, 27 * s->cap_cell, wps);
      else
        launch_listbuild<float>(P.L, items, s->ncell, 27 * s->cap_cell, wps);
    }, &ms);
    if (st != MD_OK) return st;
    if (ms < tbest) {
      tbest = ms;
      best.list_warps = wps;
    }
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best;
  }
  st = tune_apply(s, best);
  if (st != MD_OK) return st;
  s->profile = prof;
  s->forces_valid = false;  // recompute with the chosen kernels
  s->energy_valid = false;
  return read_flags(s);  // refresh the counter baseline (the trial launches counted triplets)
}

// one respa_step call with snapshot / replay
md_status do_call(md_system* s, int n_outer, int k, double dt_outer) {
  if (s->r_a > 0 && ((n_outer > 0 && k % s->s_near != 0) || s->r_a > s->rc2 || s->r_a > s->rc3)) {
    g_last_error = "distance classes: k_inner must be a multiple of s_near and r_a <= min(r_c2, r_c3)";
    return MD_ERR_ARG;
  }
  if (s->atm_variant < 0) {
    md_status st = tune(s);
    if (st != MD_OK) return st;
  }
  const double dt_in = dt_outer / k;
  for (int attempt = 0; attempt < 6; ++attempt) {
    // after a skin replay the next calls start in safe mode (adaptive binning; a first attempt that
    // would be replayed anyway costs a whole call); after safe_span calls the normal plan is tried again
    const bool safe = attempt > 0 ? (s->h_flags[FLG_SKIN] &&
                                     !(s->h_flags[FLG_ERR] & (ERR_CELL_CAP | ERR_NBR_CAP | ERR_STAGE_CAP)))
                                  : s->safe_calls > 0;
    md_status st = upload_desc(s, dt_in, dt_outer);
    if (st != MD_OK) return st;
    st = clear_flags(s);
    if (st != MD_OK) return st;
    // a replay restored positions and order from the snapshot, but the lists are those of the failed
    // attempt's binnings: in safe mode the first inner step bins (the drift flag starts set)
    if (safe && attempt > 0) CK(cudaMemsetAsync(s->h.flags + FLG_SKIN, 1, sizeof(int), s->stream));
    const bool init = !s->forces_valid;
    const int cur0 = s->cur;
    st = snapshot(s, true);
    if (st != MD_OK) return st;
    const unsigned long long trip0 = s->h_ctr[CTR_TRIPLETS];  // device counter as of the last call
    const unsigned long long near0 = s->h_ctr[CTR_NEAR];
    st = run_plan(s, n_outer, k, init, safe);
    if (st != MD_OK) return st;
    st = finish_call(s, n_outer);
    if (st != MD_OK) return st;
    const int err = s->h_flags[FLG_ERR];
    const bool skin_bad = s->h_flags[FLG_SKIN] != 0 && !safe;
    const bool cap_bad = (err & (ERR_CELL_CAP | ERR_NBR_CAP | ERR_STAGE_CAP)) != 0;
    // the rotation and per-particle kernels hold shorter half lists than the cell kernel
    const bool half_bad = (err & ERR_HALF_CAP) != 0 && s->atm_variant != 0;
    s->stats.max_cell_count = s->h_flags[FLG_MAXCELL];
    if (!(skin_bad || cap_bad || half_bad) || (err & ERR_NONFINITE)) {
      md_status fs = status_from_flags(s);
      if (fs != MD_OK) {
        s->cur = cur0;
        snapshot(s, false);
        s->forces_valid = false;
        s->energy_valid = false;
        cudaStreamSynchronize(s->stream);
        return fs;
      }
      // success
      if (safe && n_outer > 0) s->safe_calls = (s->safe_calls + 1) % s->safe_span;
      if (!safe && n_outer > 0) s->safe_span = kSafeCalls;  // the normal plan works again
      unsigned long long trip1 = s->h_ctr[CTR_TRIPLETS];
      int evals = n_outer + (init ? 1 : 0);
      if (evals > 0) s->stats.triplets_last = (trip1 - trip0) / (unsigned long long)evals;
      if (s->r_a > 0) {  // near-class evaluations: every s_near inner steps, plus initial
        const int nevals = n_outer * (k / s->s_near) + (init ? 1 : 0);
        if (nevals > 0) s->stats.near_triplets_last = (s->h_ctr[CTR_NEAR] - near0) / (unsigned long long)nevals;
      }
      s->stats.triplets_total += trip1 - trip0;
      s->stats.atm_evals += evals;
      s->stats.lj_evals += (uint64_t)n_outer * k + (init ? 1 : 0);
      s->stats.outer_steps += n_outer;
      s->stats.guard_rechecks = s->h_ctr[CTR_GUARD];
      if (n_outer > 0) s->cur = (k - 1) & 1;
      s->forces_valid = true;
      if (n_outer > 0 || init) {
        s->e_kin = s->h_acc[ACC_EK];
        s->u2 = s->h_acc[ACC_U2];
        s->w2 = s->h_acc[ACC_W2];
        s->u3 = s->h_acc[ACC_U3];
        s->w3 = s->h_acc[ACC_W3];
        s->energy_valid = true;
      }
      return MD_OK;
    }
    // replay from the snapshot
    s->cur = cur0;
    st = snapshot(s, false);
    if (st != MD_OK) return st;
    if (cap_bad) {
      if (err & ERR_CELL_CAP) s->cap_cell = std::max(s->cap_cell + 8, s->h_flags[FLG_MAXCELL] + 8);
      if (err & ERR_NBR_CAP) s->maxnb = s->maxnb * 3 / 2 + 16;
      if (err & ERR_STAGE_CAP)  // the cell-tile LJ staging follows cap_cell (lj_tile_capacity)
        s->cap_cell = std::max(s->cap_cell + 8, (s->h_flags[FLG_LJSTAGE] - 64 + 51) / 52 + 8);
      st = rebuild(s, true);
      if (st != MD_OK) return st;
    } else if (half_bad) {
      s->atm_variant = 0;  // kept for this system until the next tuning
      clear_graphs(s);
      s->forces_valid = false;  // the failed attempt re-sorted: rebuild the lists from the snapshot
    } else {
      s->stats.replays += 1;
      // back off: each failed return to the normal plan doubles the run of safe calls (up to 64)
      if (s->safe_calls == 0 && s->stats.replays > 1) s->safe_span = std::min(2 * s->safe_span, 64);
      s->safe_calls = 1;
    }
    // a replay must recompute the cached forces only if they were not valid before
    if (init) s->forces_valid = false;
    s->h_flags[FLG_SKIN] = skin_bad ? 1 : 0;
    s->h_flags[FLG_ERR] = cap_bad ? (err & ~ERR_HALF_CAP) : 0;
  }
  g_last_error = "respa_step: replay limit reached";
  return MD_ERR_CAPACITY;
}


// caller-order AoS copy (out_aos, host) of a sorted SoA device array; the permutation runs on the
// device (staged in snap_x, free between calls), the host only receives the result
// (two arrays at once when dsrc2 / out2 are given: staged in snap_x and snap_v, one synchronisation)
md_status fetch_sorted(md_system* s, const double* dsrc, double* out_aos, bool wrap, const double* dsrc2 = nullptr,
                       double* out2 = nullptr, bool wrap2 = false) {
  const size_t n = (size_t)s->n;
  Launch L{s->stream, s->d_sys};
  CK(cudaMemsetAsync(s->h.flags + FLG_STATE, 0, 4, s->stream));
  launch_take_state(L, (int)n, dsrc, s->snap_x, wrap ? 1 : 0);
  if (dsrc2) launch_take_state(L, (int)n, dsrc2, s->snap_v, wrap2 ? 1 : 0);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out_aos, s->snap_x, 24 * n, cudaMemcpyDeviceToHost, s->stream));
  if (dsrc2) CK(cudaMemcpyAsync(out2, s->snap_v, 24 * n, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(s->h_flags + FLG_STATE, s->h.flags + FLG_STATE, 4, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return s->h_flags[FLG_STATE] ? MD_ERR_STATE : MD_OK;
}

// new positions and/or velocities in caller order (host AoS): copied straight into device staging
// (the force arrays: set_state invalidates them), checked and placed into the sorted layout by a
// kernel writing the free buffers, committed only if every value was finite
md_status set_state_impl(md_system* s, const double* pos, const double* vel) {
  const size_t n = (size_t)s->n;
  if (!pos && !vel) return MD_OK;
  const bool full = pos && vel;
  Launch L{s->stream, s->d_sys};
  s->forces_valid = false;
  s->energy_valid = false;
  CK(cudaMemsetAsync(s->h.flags + FLG_STATE, 0, 4, s->stream));
  if (pos) CK(cudaMemcpyAsync(s->h.f2, pos, 24 * n, cudaMemcpyHostToDevice, s->stream));
  if (vel) CK(cudaMemcpyAsync(s->h.f3, vel, 24 * n, cudaMemcpyHostToDevice, s->stream));
  launch_put_state(L, (int)n, pos ? s->h.f2 : nullptr, vel ? s->h.f3 : nullptr, s->cur, full ? 1 : 0);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(s->h_flags + FLG_STATE, s->h.flags + FLG_STATE, 4, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));  // the caller may reuse its buffers after return
  const int f = s->h_flags[FLG_STATE];
  if (f & 2) return MD_ERR_STATE;
  if (f & 1) return MD_ERR_NONFINITE;
  s->cur ^= 1;
  CK(cudaMemcpyAsync(s->h.v, s->h.v_alt, 24 * n, cudaMemcpyDeviceToDevice, s->stream));
  if (full) CK(cudaMemcpyAsync(s->h.id, s->h.id_alt, 4 * n, cudaMemcpyDeviceToDevice, s->stream));
  return MD_OK;
}


// allocate a deferred system's device state and upload its host copy
md_status ensure_resident(md_system* s) {
  if (!s->deferred) return MD_OK;
  md_status st = rebuild(s, false);
  if (st != MD_OK) return st;
  s->deferred = false;
  st = set_state_impl(s, s->host_x.data(), s->host_v.data());
  if (st != MD_OK) return st;
  s->host_x.clear();
  s->host_x.shrink_to_fit();
  s->host_v.clear();
  s->host_v.shrink_to_fit();
  return MD_OK;
}

md_status ensure_forces(md_system* s) {
  md_status st = ensure_resident(s);
  if (st != MD_OK) return st;
  if (s->forces_valid) return MD_OK;
  return do_call(s, 0, 1, 1.0);
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* md_status_string(md_status st) {
  switch (st) {
    case MD_OK: return "ok";
    case MD_ERR_ARG: return "invalid argument";
    case MD_ERR_OOM: return "out of device memory";
    case MD_ERR_BOX_TOO_SMALL: return "box too small: L must exceed 3 * max(r_c2 + skin, r_c3)";
    case MD_ERR_NONFINITE: return "non-finite value in the state";
    case MD_ERR_DEVICE_TIMEOUT: return "a kernel's bounded wait for its own shared-memory copies gave up";
    case MD_ERR_CUDA: return "CUDA error";
    case MD_ERR_STATE: return "invalid state for this call";
    case MD_ERR_CAPACITY: return "capacity exceeded";
    case MD_ERR_CANCELLED: return "request cancelled";
  }
  return "unknown status";
}

const char* md_last_error(void) { return g_last_error.c_str(); }

md_status md_create_system(md_system** out, int64_t n, double box_L, const double* pos, const double* vel,
                           double mass, int precision, void* cuda_stream) {
  if (!out) return MD_ERR_ARG;
  *out = nullptr;
  const bool deferred = (precision & MD_DEFERRED) != 0;
  precision &= ~MD_DEFERRED;
  if (n < 3 || n >= (int64_t)kNbrMask || !pos || !(box_L > 0) || !isfinite(box_L) || !(mass > 0) ||
      !isfinite(mass) || (precision != MD_FP32 && precision != MD_FP64))
    return MD_ERR_ARG;
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!isfinite(pos[i]) || (vel && !isfinite(vel[i]))) return MD_ERR_NONFINITE;
  // every early return (a failed CUDA call included) releases what was made so far
  std::unique_ptr<md_system, md_status (*)(md_system*)> s(new md_system(), md_destroy_system);
  s->n = n;
  s->L = box_L;
  s->mass = mass;
  s->precision = precision;
  // a small box gets a thinner default skin (L must exceed 3 (r_c2 + skin))
  if (!(s->L > 3.0 * (s->rc2 + s->skin))) s->skin = std::max(0.0, s->L / 3.0 - s->rc2 - 1e-6 * s->L);
  md_status st = check_geometry(s.get());
  if (st != MD_OK) return st;
  if (cuda_stream) {
    s->stream = (cudaStream_t)cuda_stream;
  } else {
    CK(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
  }
  CK(cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming));
  CK(cudaMallocHost(&s->h_flags, 4 * FLG_N));
  CK(cudaMallocHost(&s->h_acc, 8 * ACC_N));
  CK(cudaMallocHost(&s->h_ctr, 8 * CTR_N));
  memset(s->h_flags, 0, 4 * FLG_N);
  memset(s->h_ctr, 0, 8 * CTR_N);
  if (deferred) {  // keep the state on the host until first use or batch admission
    s->deferred = true;
    s->host_x.assign(pos, pos + 3 * n);
    s->host_v.assign(3 * n, 0.0);
    if (vel) s->host_v.assign(vel, vel + 3 * n);
    for (int64_t i = 0; i < 3 * n; ++i) {
      double x = s->host_x[i] - box_L * floor(s->host_x[i] / box_L);
      s->host_x[i] = x >= box_L ? x - box_L : x;
    }
    *out = s.release();
    return MD_OK;
  }
  st = rebuild(s.get(), false);
  if (st != MD_OK) {
    md_destroy_system(s.release());
    return st;
  }
  st = md_set_state(s.get(), pos, vel);
  if (st != MD_OK) {
    md_destroy_system(s.release());
    return st;
  }
  *out = s.release();
  return MD_OK;
}

md_status md_set_potentials(md_system* s, double lj_eps, double lj_sigma, double rc_pair, double atm_nu,
                            double rc_triplet) {
  if (!s) return MD_ERR_ARG;
  if (!(lj_eps > 0) || !(lj_sigma > 0) || !(rc_pair > 0) || !(rc_triplet > 0) || !(atm_nu >= 0) ||
      !isfinite(lj_eps) || !isfinite(lj_sigma) || !isfinite(rc_pair) || !isfinite(rc_triplet) || !isfinite(atm_nu))
    return MD_ERR_ARG;
  double e0 = s->eps, s0 = s->sigma, r20 = s->rc2, nu0 = s->nu, r30 = s->rc3;
  s->eps = lj_eps;
  s->sigma = lj_sigma;
  s->rc2 = rc_pair;
  s->nu = atm_nu;
  s->rc3 = rc_triplet;
  md_status st = check_geometry(s);
  if (st != MD_OK) {
    s->eps = e0; s->sigma = s0; s->rc2 = r20; s->nu = nu0; s->rc3 = r30;
    return st;
  }
  s->maxnb = 0;
  s->cap_cell = 0;
  if (s->deferred) return MD_OK;
  if (s->batch) return MD_ERR_STATE;
  return rebuild(s, true);
}

md_status md_set_skin(md_system* s, double skin) {
  if (!s || !(skin >= 0) || !isfinite(skin)) return MD_ERR_ARG;
  double old = s->skin;
  s->skin = skin;
  md_status st = check_geometry(s);
  if (st != MD_OK) {
    s->skin = old;
    return st;
  }
  s->maxnb = 0;
  s->cap_cell = 0;
  if (s->deferred) return MD_OK;
  if (s->batch) return MD_ERR_STATE;
  return rebuild(s, true);
}

md_status md_set_distance_classes(md_system* s, double r_a, int s_near) {
  if (!s || !isfinite(r_a)) return MD_ERR_ARG;
  if (s->batch) return MD_ERR_STATE;
  if (r_a > 0 && (s_near < 1 || r_a > s->rc2 || r_a > s->rc3)) return MD_ERR_ARG;
  s->r_a = r_a > 0 ? r_a : 0.0;
  s->s_near = r_a > 0 ? s_near : 0;
  if (s->deferred) return MD_OK;
  return rebuild(s, true);
}

md_status md_get_near_forces(md_system* s, double* f3near) {
  if (!s || !f3near) return MD_ERR_ARG;
  if (s->batch || !(s->r_a > 0)) return MD_ERR_STATE;
  md_status st = ensure_forces(s);
  if (st != MD_OK) return st;
  return fetch_sorted(s, s->h.f3n, f3near, false);
}

md_status md_respa_step(md_system* s, int n_outer, int k_inner, double dt_outer) {
  if (!s || n_outer < 0 || k_inner < 1 || !(dt_outer > 0) || !isfinite(dt_outer)) return MD_ERR_ARG;
  if (s->batch) return MD_ERR_STATE;
  md_status st = ensure_resident(s);
  if (st != MD_OK) return st;
  return do_call(s, n_outer, k_inner, dt_outer);
}

md_status md_get_forces(md_system* s, double* f2, double* f3) {
  if (!s) return MD_ERR_ARG;
  if (s->batch) return MD_ERR_STATE;
  md_status st = ensure_forces(s);
  if (st != MD_OK) return st;
  if (f2 && f3) return fetch_sorted(s, s->h.f2, f2, false, s->h.f3, f3, false);
  if (f2) return fetch_sorted(s, s->h.f2, f2, false);
  if (f3) return fetch_sorted(s, s->h.f3, f3, false);
  return MD_OK;
}

md_status md_get_energy(md_system* s, double* e_kin, double* u2, double* u3, double* virial) {
  if (!s) return MD_ERR_ARG;
  if (s->batch) return MD_ERR_STATE;
  if (!s->energy_valid) {
    s->forces_valid = false;
    md_status st = ensure_forces(s);
    if (st != MD_OK) return st;
  }
  if (e_kin) *e_kin = s->e_kin;
  if (u2) *u2 = s->u2;
  if (u3) *u3 = s->u3;
  if (virial) *virial = s->w2 + s->w3;
  return MD_OK;
}

md_status md_get_rdf(md_system* s, int nbins, double r_max, uint64_t* counts) {
  if (!s || !counts || nbins < 1 || nbins > kRdfMaxBins || !(r_max > 0) || !isfinite(r_max)) return MD_ERR_ARG;
  if (s->batch) return MD_ERR_STATE;
  if (r_max > s->rc2 + s->skin) return MD_ERR_ARG;  // the pair list holds every pair within r_c2 + skin
  md_status st = ensure_forces(s);  // positions of the last binning, with their pair list
  if (st != MD_OK) return st;
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d), 8 * (size_t)nbins, s->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MD_ERR_OOM;
  }
  const double dr = r_max / nbins;
  Launch L{s->stream, s->d_sys};
  e = cudaMemsetAsync(d, 0, 8 * (size_t)nbins, s->stream);
  if (e == cudaSuccess) {
    launch_rdf(L, pitems_for(s, T_BIN, 0, s->cur), s->nblocks, nbins, dr, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(counts, d, 8 * (size_t)nbins, cudaMemcpyDeviceToHost, s->stream);
  cudaFreeAsync(d, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "md_get_rdf");
  return MD_OK;
}

md_status md_get_state(md_system* s, double* pos, double* vel) {
  if (!s) return MD_ERR_ARG;
  if (s->batch) return MD_ERR_STATE;
  if (s->deferred) {
    if (pos) memcpy(pos, s->host_x.data(), 24 * (size_t)s->n);
    if (vel) memcpy(vel, s->host_v.data(), 24 * (size_t)s->n);
    return MD_OK;
  }
  if (pos && vel) return fetch_sorted(s, s->h.X[s->cur], pos, true, s->h.v, vel, false);
  if (pos) return fetch_sorted(s, s->h.X[s->cur], pos, true);
  if (vel) return fetch_sorted(s, s->h.v, vel, false);
  return MD_OK;
}

md_status md_set_state(md_system* s, const double* pos, const double* vel) {
  if (!s) return MD_ERR_ARG;
  if (s->batch) return MD_ERR_STATE;
  if (s->deferred) {
    const size_t n = (size_t)s->n;
    for (size_t i = 0; i < 3 * n; ++i)
      if ((pos && !isfinite(pos[i])) || (vel && !isfinite(vel[i]))) return MD_ERR_NONFINITE;
    if (pos) {
      for (size_t i = 0; i < 3 * n; ++i) {
        double x = pos[i] - s->L * floor(pos[i] / s->L);
        s->host_x[i] = x >= s->L ? x - s->L : x;
      }
    }
    if (vel) memcpy(s->host_v.data(), vel, 24 * n);
    return MD_OK;
  }
  return set_state_impl(s, pos, vel);
}

md_status md_get_stats(md_system* s, md_stats* out) {
  if (!s || !out) return MD_ERR_ARG;
  s->stats.atm_kernel = s->atm_variant;
  s->stats.atm_bases_per_warp = s->rot_per;
  s->stats.lj_block = s->lj_block;
  s->stats.lj_kernel = s->lj_kernel;
  s->stats.lj_team = s->lj_team;
  s->stats.list_warps = s->list_warps;
  s->stats.tuned_from_cache = s->tuned_from_cache ? 1 : 0;
  *out = s->stats;
  return MD_OK;
}

md_status md_set_profiling(md_system* s, int profile) {
  if (!s) return MD_ERR_ARG;
  s->profile = profile != 0;
  clear_graphs(s);
  return MD_OK;
}

md_status md_set_atm_kernel(md_system* s, int variant) {
  if (!s || variant < -1 || variant > 2) return MD_ERR_ARG;
  s->atm_variant_req = variant;
  s->atm_variant = -1;
  clear_graphs(s);
  s->forces_valid = false;
  s->energy_valid = false;
  return MD_OK;
}

md_status md_set_lj_kernel(md_system* s, int variant) {
  if (!s || variant < -1 || variant > 2) return MD_ERR_ARG;
  if (s->batch) return MD_ERR_STATE;
  s->lj_kernel_req = variant;
  s->atm_variant = -1;  // applied with the next tuning (the cached choices fill the rest)
  clear_graphs(s);
  s->forces_valid = false;
  s->energy_valid = false;
  return MD_OK;
}

md_status md_inject_copy_shortfall(md_system* s, int bytes) {
  if (!s || bytes < 0 || bytes > 4096) return MD_ERR_ARG;
  s->lj_tx_extra = bytes;
  return MD_OK;
}

md_status md_get_memory(md_system* s, size_t* device_bytes) {
  if (!s || !device_bytes) return MD_ERR_ARG;
  *device_bytes = s->deferred ? arena_bytes(s) : s->mem_bytes;  // the figure batch admission uses
  return MD_OK;
}

md_status md_set_shapes(md_system* s, int lj_block, int list_warps, int rot_bases_per_warp) {
  if (!s) return MD_ERR_ARG;
  if (lj_block != 0 && lj_block != 32 && lj_block != 64 && lj_block != 128) return MD_ERR_ARG;
  if (list_warps != 0 && list_warps != 2 && list_warps != 4 && list_warps != 8) return MD_ERR_ARG;
  if (rot_bases_per_warp != 0 && rot_bases_per_warp != 4 && rot_bases_per_warp != 8 && rot_bases_per_warp != 16)
    return MD_ERR_ARG;
  if (s->batch) return MD_ERR_STATE;
  s->lj_block_req = lj_block;
  s->list_warps_req = list_warps;
  s->rot_per_req = rot_bases_per_warp;
  s->atm_variant = -1;  // applied with the next tuning (the cached choices fill the rest)
  clear_graphs(s);
  return MD_OK;
}

md_status md_get_info(md_system* s, int64_t* n, double* box_L, int* precision) {
  if (!s) return MD_ERR_ARG;
  if (n) *n = s->n;
  if (box_L) *box_L = s->L;
  if (precision) *precision = s->precision;
  return MD_OK;
}

md_status md_destroy_system(md_system* s) {
  if (!s) return MD_OK;
  if (s->stream) cudaStreamSynchronize(s->stream);
  free_device(s);
  for (auto e : s->events) cudaEventDestroy(e);
  if (s->h_flags) cudaFreeHost(s->h_flags);
  if (s->h_acc) cudaFreeHost(s->h_acc);
  if (s->h_ctr) cudaFreeHost(s->h_ctr);
  if (s->side) cudaStreamSynchronize(s->side);
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  if (s->side) cudaStreamDestroy(s->side);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
  return MD_OK;
}

}  // extern "C"

// ====================================================================== batch
// Batched ensemble / continuous serving.  Resident members share every launch: on each inner
// tick one launch per kernel covers all members (work items carry the member index).  Members
// join at cycle boundaries; a cycle is P = lcm(k_j) ticks, so every member starts its outer
// steps at t = 0 of a cycle.  The cycle is captured once per composition as a CUDA graph;
// what changes from cycle to cycle (energy on a member's final outer step, closing vs
// continuing outer kick, skip once finished) is a per-member table of modes, uploaded before
// each launch.  %globaltimer stamps at tick boundaries give per-outer-step latencies.
namespace {

enum { KT_SORT = 0, KT_LJ = 1, KT_ATM = 2, KT_COMB = 3, KT_N = 4 };
enum { RQ_QUEUED = 0, RQ_RESIDENT = 1, RQ_DONE = 2, RQ_FAILED = 3, RQ_CANCELLED = 4 };

struct Request {
  md_system* s = nullptr;
  uint64_t ticket = 0;
  int n_outer = 0, k = 1;
  double dt_outer = 0;
  int outer_done = 0;
  int state = RQ_QUEUED;
  bool cancel = false;  // resident request cancelled: it leaves at the end of its current outer step
  md_status status = MD_OK;
  std::vector<double> lat_ms;
  unsigned long long trip0 = 0;
};

struct TickItems {
  size_t bin = 0, scan = 0, list = 0, lj = 0, kick = 0, atm = 0, comb = 0;  // offsets (items) in the pools
  int nbin = 0, nscan = 0, nlist = 0, nlj = 0, nkick = 0, natm = 0, ncomb = 0;
};

}  // namespace

struct md_batch {
  size_t budget = 0;
  int64_t max_particles = 0;  // md_batch_set_limits: resident particles admitted (0: no bound)
  int precision = -1;
  std::map<uint64_t, Request> req;
  std::vector<uint64_t> queue, resident;
  uint64_t next_ticket = 1;
  cudaStream_t stream = nullptr;
  // composition
  bool dirty = true;
  int P = 1, variant = 1, smax = 0, smax_list = 0, atm_grid = 0;
  bool cell_only = false;  // a member's half list overflowed the rotation kernel: cell kernel from now on
  SysDev* d_sys = nullptr;
  int* d_modes = nullptr;
  int* h_modes = nullptr;  // pinned [slots][P][KT_N]
  int* d_flags = nullptr;
  double* d_acc = nullptr;
  unsigned long long* d_ctr = nullptr;
  int* h_flags = nullptr;
  double* h_acc = nullptr;
  unsigned long long* h_ctr = nullptr;
  unsigned long long* d_stamps = nullptr;
  unsigned long long* h_stamps = nullptr;
  PItem* d_pitems = nullptr;
  CItem* d_citems = nullptr;
  SItem* d_sitems = nullptr;
  PItem* d_snap = nullptr;
  int nsnap = 0;
  std::vector<TickItems> ticks, ticks_safe;
  cudaGraphExec_t graph = nullptr, graph_safe = nullptr;
  size_t cap_slots = 0;
  uint64_t cycles = 0, replayed = 0;  // cycles run, and replayed from their start
  int safe_calls = 0, safe_span = 4;  // as for single systems: safe cycles after a skin replay
};

namespace {

void batch_free_composition(md_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->graph_safe) cudaGraphExecDestroy(b->graph_safe);
  b->graph = b->graph_safe = nullptr;
  for (void* p : {(void*)b->d_sys, (void*)b->d_modes, (void*)b->d_flags, (void*)b->d_acc, (void*)b->d_ctr,
                  (void*)b->d_stamps, (void*)b->d_pitems, (void*)b->d_citems, (void*)b->d_sitems, (void*)b->d_snap})
    if (p) cudaFree(p);
  for (void* p : {(void*)b->h_modes, (void*)b->h_flags, (void*)b->h_acc, (void*)b->h_ctr, (void*)b->h_stamps})
    if (p) cudaFreeHost(p);
  b->d_sys = nullptr;
  b->d_modes = b->h_modes = nullptr;
  b->d_flags = b->h_flags = nullptr;
  b->d_acc = b->h_acc = nullptr;
  b->d_ctr = b->h_ctr = nullptr;
  b->d_stamps = b->h_stamps = nullptr;
  b->d_pitems = nullptr;
  b->d_citems = nullptr;
  b->d_sitems = nullptr;
  b->d_snap = nullptr;
  b->ticks.clear();
  b->ticks_safe.clear();
}

long long lcm_ll(long long a, long long b) {
  long long x = a, y = b;
  while (y) {
    long long t = x % y;
    x = y;
    y = t;
  }
  return a / x * b;
}

// enqueue one cycle; with check set (outside capture) every launch is checked and the first
// failing one is named in *failed
template <typename T>
void enqueue_cycle(md_batch* b, const std::vector<TickItems>& ticks, bool with_stamps, std::string* failed = nullptr) {
  Launch L{b->stream, b->d_sys};
  auto chk = [&](const char* what, int t) {
    if (!failed || !failed->empty()) return;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) *failed = std::string(what) + " at tick " + std::to_string(t) + ": " + cudaGetErrorString(e);
  };
  if (with_stamps) launch_stamp(b->stream, b->d_stamps);
  chk("stamp", -1);
  for (int t = 0; t < b->P; ++t) {
    const TickItems& it = ticks[t];
    if (&ticks == &b->ticks_safe) launch_sort_decide_all(L, (int)b->resident.size());
    launch_bin_count(L, b->d_pitems + it.bin, it.nbin, kBlock);
    chk("bin_count", t);
    launch_scan(L, b->d_sitems + it.scan, it.nscan);
    chk("scan", t);
    launch_cell_order(L, b->d_pitems + it.bin, it.nbin, kBlock, b->d_citems + it.list, it.nlist);
    chk("cell_order", t);
    launch_scatter<T>(L, b->d_pitems + it.bin, it.nbin, kBlock);
    chk("scatter", t);
    launch_listbuild<T>(L, b->d_citems + it.list, it.nlist, b->smax_list, kListWarpsDefault);
    chk("listbuild", t);
    launch_lj<T>(L, b->d_pitems + it.lj, it.nlj, true, kLjParticles);  // members' modes decide the energy
    chk("lj", t);
    launch_kick<T>(L, b->d_pitems + it.kick, it.nkick);
    chk("kick", t);
    if (b->variant == 2)
      launch_atm_rot<T>(L, b->d_pitems + it.atm, it.natm, rot_bases_per_item(b->precision) / kRotWarps);
    else if (b->variant == 1)
      launch_atm_pa<T>(L, b->d_pitems + it.atm, it.natm);
    else
      launch_atm<T>(L, b->d_citems + it.atm, it.natm, b->atm_grid, b->smax);
    chk("atm", t);
    launch_combine<T>(L, b->d_pitems + it.comb, it.ncomb, kBlock);
    chk("combine", t);
    if (with_stamps) launch_stamp(b->stream, b->d_stamps + t + 1);
    chk("stamp", t);
  }
}

md_status batch_build(md_batch* b) {
  batch_free_composition(b);
  const int ns = (int)b->resident.size();
  if (ns == 0) {
    b->dirty = false;
    return MD_OK;
  }
  long long P = 1;
  bool pa = true;
  int req = -2;  // the members' common requested triplet kernel (-3: they differ)
  int capmax = 0;
  for (uint64_t tk : b->resident) {
    const Request& r = b->req[tk];
    P = lcm_ll(P, r.k);
    pa = pa && variant_allowed(r.s, 1);
    req = (req == -2 || req == r.s->atm_variant_req) ? r.s->atm_variant_req : -3;
    capmax = std::max(capmax, r.s->cap_cell);
  }
  if (P > 4096) {
    g_last_error = "batch: lcm of the members' k_inner exceeds 4096 ticks";
    return MD_ERR_ARG;
  }
  b->P = (int)P;
  // the members' common request where every member allows it, else the rotation kernel where the
  // pair list covers the triplet cutoff, else the cell kernel
  b->variant = b->cell_only ? 0 : ((req >= 0 && (req == 0 || pa)) ? req : (pa ? 2 : 0));
  b->smax = atm_stage_capacity(capmax);
  b->smax_list = 27 * capmax;  // the pair-list build stages the full 27-cell stencil
  {
    int bytes = 0;
    int per_sm = atm_configure(b->smax, b->precision, &bytes);
    if (per_sm <= 0) return MD_ERR_CAPACITY;
    if (listbuild_configure(27 * capmax, b->precision) < 0) return MD_ERR_CAPACITY;
    b->atm_grid = per_sm * device_sm_count();
  }
  // device descriptors: each member's own, with batch-owned flags / counters / mode tables
  CK(cudaMalloc(&b->d_sys, sizeof(SysDev) * ns));
  CK(cudaMalloc(&b->d_modes, sizeof(int) * ns * P * KT_N));
  CK(cudaMallocHost(&b->h_modes, sizeof(int) * ns * P * KT_N));
  CK(cudaMalloc(&b->d_flags, sizeof(int) * ns * FLG_N));
  CK(cudaMallocHost(&b->h_flags, sizeof(int) * ns * FLG_N));
  CK(cudaMalloc(&b->d_acc, sizeof(double) * ns * ACC_N));
  CK(cudaMallocHost(&b->h_acc, sizeof(double) * ns * ACC_N));
  CK(cudaMalloc(&b->d_ctr, sizeof(unsigned long long) * ns * CTR_N));
  CK(cudaMallocHost(&b->h_ctr, sizeof(unsigned long long) * ns * CTR_N));
  CK(cudaMalloc(&b->d_stamps, sizeof(unsigned long long) * (P + 1)));
  CK(cudaMallocHost(&b->h_stamps, sizeof(unsigned long long) * (P + 1)));
  CK(cudaMemsetAsync(b->d_ctr, 0, sizeof(unsigned long long) * ns * CTR_N, b->stream));
  std::vector<SysDev> hs(ns);
  for (int j = 0; j < ns; ++j) {
    Request& r = b->req[b->resident[j]];
    md_system* s = r.s;
    md_status st = upload_desc(s, r.dt_outer / r.k, r.dt_outer);
    if (st != MD_OK) return st;
    SysDev h = s->h;
    h.flags = b->d_flags + j * FLG_N;
    h.acc = b->d_acc + j * ACC_N;
    h.ctr = b->d_ctr + j * CTR_N;
    h.mode_tab = b->d_modes + (size_t)j * P * KT_N;
    hs[j] = h;
    r.trip0 = 0;
  }
  CK(cudaMemcpyAsync(b->d_sys, hs.data(), sizeof(SysDev) * ns, cudaMemcpyHostToDevice, b->stream));
  // work items for every tick of the cycle (normal, and safe: binning items on every tick, which the
  // members' modes make conditional on their drift flags)
  std::vector<PItem> pit;
  std::vector<CItem> cit;
  std::vector<SItem> sit;
  auto build_ticks = [&](bool safe, std::vector<TickItems>& out) {
    out.assign(P, TickItems{});
    for (int t = 0; t < P; ++t) {
      TickItems& ti = out[t];
      auto tab = [&](int kt) { return M_TABLE | (t * KT_N + kt); };
      ti.bin = pit.size();
      for (int j = 0; j < ns; ++j) {
        const Request& r = b->req[b->resident[j]];
        const int tt = t % r.k;
        if (!(tt == r.k - 1 || safe)) continue;
        for (int q = 0; q < (int)r.s->n; q += kBlock) pit.push_back(PItem{j, q, tab(KT_SORT), tt & 1});
      }
      ti.nbin = (int)(pit.size() - ti.bin);
      ti.scan = sit.size();
      for (int j = 0; j < ns; ++j) {
        const Request& r = b->req[b->resident[j]];
        const int tt = t % r.k;
        if (tt == r.k - 1 || safe) sit.push_back(SItem{j, tab(KT_SORT)});
      }
      ti.nscan = (int)(sit.size() - ti.scan);
      ti.list = cit.size();
      for (int j = 0; j < ns; ++j) {
        const Request& r = b->req[b->resident[j]];
        const int tt = t % r.k;
        if (!(tt == r.k - 1 || safe)) continue;
        for (int c = 0; c < r.s->ncell; ++c) cit.push_back(CItem{j, c, tt & 1, tab(KT_SORT)});
      }
      ti.nlist = (int)(cit.size() - ti.list);
      ti.lj = pit.size();
      for (int j = 0; j < ns; ++j) {
        const Request& r = b->req[b->resident[j]];
        const int tt = t % r.k;
        for (int q = 0; q < (int)r.s->n; q += kLjParticles) pit.push_back(PItem{j, q, tab(KT_LJ), tt & 1});
      }
      ti.nlj = (int)(pit.size() - ti.lj);
      ti.kick = pit.size();
      for (int j = 0; j < ns; ++j) {
        const Request& r = b->req[b->resident[j]];
        const int tt = t % r.k;
        for (int q = 0; q < (int)r.s->n; q += kBlock) pit.push_back(PItem{j, q, tab(KT_LJ), tt & 1});
      }
      ti.nkick = (int)(pit.size() - ti.kick);
      if (b->variant >= 1) {
        const int per = (b->variant == 1) ? kPaPerBlock : rot_bases_per_item(b->precision);
        ti.atm = pit.size();
        for (int j = 0; j < ns; ++j) {
          const Request& r = b->req[b->resident[j]];
          if (t % r.k != r.k - 1) continue;
          for (int q = 0; q < (int)r.s->n; q += per) pit.push_back(PItem{j, q, tab(KT_ATM), (r.k - 1) & 1});
        }
        ti.natm = (int)(pit.size() - ti.atm);
      } else {
        ti.atm = cit.size();
        for (int j = 0; j < ns; ++j) {
          const Request& r = b->req[b->resident[j]];
          if (t % r.k != r.k - 1) continue;
          for (int c = 0; c < r.s->ncell; ++c) cit.push_back(CItem{j, c, (r.k - 1) & 1, tab(KT_ATM)});
        }
        ti.natm = (int)(cit.size() - ti.atm);
      }
      ti.comb = pit.size();
      for (int j = 0; j < ns; ++j) {
        const Request& r = b->req[b->resident[j]];
        if (t % r.k != r.k - 1) continue;
        for (int q = 0; q < (int)r.s->n; q += kBlock) pit.push_back(PItem{j, q, tab(KT_COMB), (r.k - 1) & 1});
      }
      ti.ncomb = (int)(pit.size() - ti.comb);
    }
  };
  build_ticks(false, b->ticks);
  build_ticks(true, b->ticks_safe);
  std::vector<PItem> snap;
  for (int j = 0; j < ns; ++j) {
    const Request& r = b->req[b->resident[j]];
    for (int q = 0; q < (int)r.s->n; q += kBlock) snap.push_back(PItem{j, q, 0, 0});
  }
  b->nsnap = (int)snap.size();
  CK(cudaMalloc(&b->d_pitems, sizeof(PItem) * std::max<size_t>(1, pit.size())));
  CK(cudaMalloc(&b->d_citems, sizeof(CItem) * std::max<size_t>(1, cit.size())));
  CK(cudaMalloc(&b->d_sitems, sizeof(SItem) * std::max<size_t>(1, sit.size())));
  CK(cudaMalloc(&b->d_snap, sizeof(PItem) * std::max<size_t>(1, snap.size())));
  CK(cudaMemcpyAsync(b->d_pitems, pit.data(), sizeof(PItem) * pit.size(), cudaMemcpyHostToDevice, b->stream));
  CK(cudaMemcpyAsync(b->d_citems, cit.data(), sizeof(CItem) * cit.size(), cudaMemcpyHostToDevice, b->stream));
  CK(cudaMemcpyAsync(b->d_sitems, sit.data(), sizeof(SItem) * sit.size(), cudaMemcpyHostToDevice, b->stream));
  CK(cudaMemcpyAsync(b->d_snap, snap.data(), sizeof(PItem) * snap.size(), cudaMemcpyHostToDevice, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  // capture the two cycle graphs
  for (int safe = 0; safe < 2; ++safe) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    if (b->precision)
      enqueue_cycle<double>(b, safe ? b->ticks_safe : b->ticks, true);
    else
      enqueue_cycle<float>(b, safe ? b->ticks_safe : b->ticks, true);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) {
      // name the launch that broke the capture: enqueue the same cycle uncaptured, checked
      cudaGetLastError();
      std::string failed;
      if (b->precision)
        enqueue_cycle<double>(b, safe ? b->ticks_safe : b->ticks, true, &failed);
      else
        enqueue_cycle<float>(b, safe ? b->ticks_safe : b->ticks, true, &failed);
      cudaStreamSynchronize(b->stream);
      cudaGetLastError();
      g_last_error = "batch graph capture failed (" + std::string(cudaGetErrorString(e)) + "); " +
                     (failed.empty() ? std::string("uncaptured launches succeeded") : failed);
      return MD_ERR_CUDA;
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(batch)");
    (safe ? b->graph_safe : b->graph) = ex;
  }
  b->dirty = false;
  return MD_OK;
}

// modes of every member for every tick of the next cycle
void batch_fill_modes(md_batch* b, bool safe) {
  const int ns = (int)b->resident.size();
  const int P = b->P;
  for (int j = 0; j < ns; ++j) {
    const Request& r = b->req[b->resident[j]];
    const int rem = r.n_outer - r.outer_done;
    const int f3r = (b->variant == 1) ? M_F3READY : (b->variant == 2 ? M_F3ACC : 0);
    int* tab = b->h_modes + (size_t)j * P * KT_N;
    for (int t = 0; t < P; ++t) {
      const int q = t / r.k, tt = t % r.k;
      int* e = tab + t * KT_N;
      if (q >= rem) {
        e[KT_SORT] = e[KT_LJ] = e[KT_ATM] = e[KT_COMB] = M_SKIP;
        continue;
      }
      const bool closing = tt == r.k - 1;
      const bool final_step = closing && q == rem - 1;
      const int E = final_step ? M_ENERGY : 0;
      // safe plan: a binning before any tick whose positions moved more than skin / 2 (adaptive)
      e[KT_SORT] = closing ? 0 : (safe ? M_COND : M_SKIP);
      e[KT_LJ] = (closing ? LJ_LAST : LJ_MID) | E;
      e[KT_ATM] = closing ? E : M_SKIP;
      e[KT_COMB] = closing ? ((final_step ? CB_LAST : CB_CONT) | E | f3r) : M_SKIP;
    }
  }
}

md_status batch_admit(md_batch* b) {
  size_t used = 0;
  int64_t used_n = 0;
  for (uint64_t tk : b->resident) {
    used += b->req[tk].s->mem_bytes;
    used_n += b->req[tk].s->n;
  }
  while (!b->queue.empty()) {
    Request& r = b->req[b->queue.front()];
    md_system* s = r.s;
    // particle bound (a latency target, not a capacity): the head of the queue waits while it would take
    // the resident particles past it, and runs alone if it is larger than the bound by itself
    if (b->max_particles > 0 && !b->resident.empty() && used_n + s->n > b->max_particles) break;
    const size_t need = s->deferred ? arena_bytes(s) : s->mem_bytes;
    if (b->budget && used + need > b->budget) {
      if (b->resident.empty()) {  // can never fit: fail the request
        r.state = RQ_FAILED;
        r.status = MD_ERR_OOM;
        b->queue.erase(b->queue.begin());
        continue;
      }
      break;
    }
    b->queue.erase(b->queue.begin());
    if (!s->batch_lj) {  // forces not yet computed are computed with the batch's LJ kernel
      s->batch_lj = true;
      clear_graphs(s);
    }
    md_status st = ensure_resident(s);
    if (st == MD_OK) st = ensure_forces(s);
    if (st == MD_OK && r.n_outer > 0) {
      // opening kicks and first drift of the request (Algorithm 2 at i = 0)
      st = upload_desc(s, r.dt_outer / r.k, r.dt_outer);
      if (st == MD_OK) {
        Plan Pl{s, Launch{s->stream, s->d_sys}};
        if (s->precision) Pl.start<double>(s->cur); else Pl.start<float>(s->cur);
        cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "batch start");
      }
    }
    if (st != MD_OK || r.n_outer == 0) {
      s->batch_lj = false;
      clear_graphs(s);
    }
    if (st != MD_OK) {
      r.state = RQ_FAILED;
      r.status = st;
      continue;
    }
    if (r.n_outer == 0) {
      r.state = RQ_DONE;
      continue;
    }
    s->batch = b;
    s->forces_valid = false;
    r.state = RQ_RESIDENT;
    r.s->skin_carry = false;
    used += s->mem_bytes;
    used_n += s->n;
    b->resident.push_back(r.ticket);
    b->dirty = true;
  }
  return MD_OK;
}

// finished or failed members leave; their state is a full step again
void batch_retire(md_batch* b, std::vector<uint64_t>& leaving) {
  if (leaving.empty()) return;
  std::vector<uint64_t> keep;
  for (uint64_t tk : b->resident)
    if (std::find(leaving.begin(), leaving.end(), tk) == leaving.end()) keep.push_back(tk);
  b->resident.swap(keep);
  for (uint64_t tk : leaving) {
    Request& r = b->req[tk];
    r.s->batch = nullptr;
    r.s->batch_lj = false;
    clear_graphs(r.s);
  }
  b->dirty = true;
}

md_status batch_cycle(md_batch* b) {
  const int ns = (int)b->resident.size();
  b->cycles += 1;
  bool was_safe = false;
  for (int attempt = 0; attempt < 4; ++attempt) {
    const bool safe = attempt > 0 || b->safe_calls > 0;
    was_safe = safe;
    batch_fill_modes(b, safe);
    CK(cudaMemcpyAsync(b->d_modes, b->h_modes, sizeof(int) * ns * b->P * KT_N, cudaMemcpyHostToDevice, b->stream));
    // fresh flags, except a member's drift flag left by the previous cycle's last drift (the first
    // tick's positions already moved more than skin / 2 from the member's last binning)
    memset(b->h_flags, 0, sizeof(int) * ns * FLG_N);
    // (a replay restored positions and order from the snapshot, but the lists are those of the failed
    // attempt's binnings: every member bins before its first tick)
    for (int j = 0; j < ns; ++j)
      b->h_flags[j * FLG_N + FLG_SKIN] = (attempt > 0 || b->req[b->resident[j]].s->skin_carry) ? 1 : 0;
    CK(cudaMemcpyAsync(b->d_flags, b->h_flags, sizeof(int) * ns * FLG_N, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemsetAsync(b->d_acc, 0, sizeof(double) * ns * ACC_N, b->stream));
    Launch L{b->stream, b->d_sys};
    launch_snapshot(L, b->d_snap, b->nsnap, 0);
    CK(cudaGraphLaunch(safe ? b->graph_safe : b->graph, b->stream));
    CK(cudaMemcpyAsync(b->h_flags, b->d_flags, sizeof(int) * ns * FLG_N, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(b->h_acc, b->d_acc, sizeof(double) * ns * ACC_N, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(b->h_ctr, b->d_ctr, sizeof(unsigned long long) * ns * CTR_N, cudaMemcpyDeviceToHost,
                       b->stream));
    CK(cudaMemcpyAsync(b->h_stamps, b->d_stamps, sizeof(unsigned long long) * (b->P + 1), cudaMemcpyDeviceToHost,
                       b->stream));
    CK(cudaStreamSynchronize(b->stream));
    bool skin = false, cap = false, half = false;
    for (int j = 0; j < ns; ++j) {
      const int* f = b->h_flags + j * FLG_N;
      // a member that went non-finite fails alone after this cycle: its other flags (a skin violation or
      // a cell overflow, the usual company of a state blowing up) ask for no replay and no growth
      if (f[FLG_ERR] & ERR_NONFINITE) continue;
      if (f[FLG_SKIN] && !safe) skin = true;
      if (f[FLG_ERR] & (ERR_CELL_CAP | ERR_NBR_CAP)) cap = true;
      if ((f[FLG_ERR] & ERR_HALF_CAP) && b->variant != 0) half = true;
    }
    if (!(skin || cap || half)) break;
    b->replayed += 1;
    if (skin) {  // safe cycles from now on, with back-off before the normal plan is tried again
      if (b->safe_calls == 0 && b->replayed > 1) b->safe_span = std::min(2 * b->safe_span, 64);
      b->safe_calls = 1;
    }
    launch_snapshot(L, b->d_snap, b->nsnap, 1);  // every member back to the cycle start
    CK(cudaStreamSynchronize(b->stream));
    if (half && !cap) {  // the cell kernel takes longer half lists; replay the cycle with it
      b->cell_only = true;
      md_status st = batch_build(b);
      if (st != MD_OK) return st;
    }
    if (cap) {
      std::vector<uint64_t> grow;
      for (int j = 0; j < ns; ++j) {
        const int* f = b->h_flags + j * FLG_N;
        if ((f[FLG_ERR] & (ERR_CELL_CAP | ERR_NBR_CAP)) && !(f[FLG_ERR] & ERR_NONFINITE))
          grow.push_back(b->resident[j]);
      }
      for (uint64_t tk : grow) {
        md_system* s = b->req[tk].s;
        const int* f = b->h_flags + (std::find(b->resident.begin(), b->resident.end(), tk) - b->resident.begin()) * FLG_N;
        if (f[FLG_ERR] & ERR_CELL_CAP) s->cap_cell = std::max(s->cap_cell + 8, f[FLG_MAXCELL] + 8);
        if (f[FLG_ERR] & ERR_NBR_CAP) s->maxnb = s->maxnb * 3 / 2 + 16;
        // The snapshot restored the cycle-start state (buffer 0, cycle-start order): inside an outer step,
        // its opening kicks and first drift already applied, and the cached forces are no longer needed
        // (the cycle's ticks compute every force they use).  The new arena keeps positions, velocities
        // and order; the replay below starts in safe mode, which bins before its first tick.
        s->cur = 0;
        md_status st = rebuild(s, true);
        if (st != MD_OK) return st;
      }
      md_status st = batch_build(b);
      if (st != MD_OK) return st;
      attempt = 0;  // replay in safe mode: the restored members' cell-local coordinates are stale
    }
  }
  if (was_safe)
    b->safe_calls = (b->safe_calls + 1) % b->safe_span;
  else
    b->safe_span = 4;  // the normal plan works again
  for (int j = 0; j < ns; ++j)  // a safe cycle's last drift may already be past skin / 2
    b->req[b->resident[j]].s->skin_carry = b->h_flags[j * FLG_N + FLG_SKIN] != 0;
  // progress, latencies, completion
  std::vector<uint64_t> leaving;
  for (int j = 0; j < ns; ++j) {
    Request& r = b->req[b->resident[j]];
    const int* f = b->h_flags + j * FLG_N;
    const int rem = r.n_outer - r.outer_done;
    const int steps = std::min(rem, b->P / r.k);
    for (int q = 0; q < steps; ++q) {
      const unsigned long long t0 = b->h_stamps[q * r.k], t1 = b->h_stamps[(q + 1) * r.k];
      r.lat_ms.push_back((double)(t1 - t0) * 1e-6);
    }
    r.outer_done += steps;
    md_system* s = r.s;
    const unsigned long long trip = b->h_ctr[j * CTR_N + CTR_TRIPLETS];
    s->stats.triplets_total += trip - r.trip0;
    if (steps > 0) s->stats.triplets_last = (trip - r.trip0) / (unsigned long long)steps;
    r.trip0 = trip;
    s->stats.outer_steps += steps;
    s->stats.atm_evals += steps;
    s->stats.lj_evals += (uint64_t)steps * r.k;
    if (f[FLG_ERR] & (ERR_NONFINITE | ERR_HALF_CAP)) {
      r.state = RQ_FAILED;
      r.status = (f[FLG_ERR] & ERR_NONFINITE) ? MD_ERR_NONFINITE : MD_ERR_CAPACITY;
      s->forces_valid = s->energy_valid = false;
      leaving.push_back(r.ticket);
      continue;
    }
    if (r.outer_done >= r.n_outer) {
      if (r.cancel) {
        r.state = RQ_CANCELLED;
        r.status = MD_ERR_CANCELLED;
      }
      const double* a = b->h_acc + j * ACC_N;
      s->e_kin = a[ACC_EK];
      s->u2 = a[ACC_U2];
      s->w2 = a[ACC_W2];
      s->u3 = a[ACC_U3];
      s->w3 = a[ACC_W3];
      s->energy_valid = true;
      s->forces_valid = true;
      s->cur = (r.k - 1) & 1;
      if (!r.cancel) r.state = RQ_DONE;
      leaving.push_back(r.ticket);
    }
  }
  batch_retire(b, leaving);
  return MD_OK;
}

}  // namespace

extern "C" {

md_status md_batch_create(md_batch** out, size_t hbm_budget_bytes) {
  if (!out) return MD_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<md_batch> b(new md_batch());
  b->budget = hbm_budget_bytes;
  CK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
  *out = b.release();
  return MD_OK;
}

md_status md_batch_set_limits(md_batch* b, int64_t max_resident_particles) {
  if (!b || max_resident_particles < 0) return MD_ERR_ARG;
  b->max_particles = max_resident_particles;
  return MD_OK;
}

md_status md_batch_submit(md_batch* b, md_system* s, int n_outer, int k_inner, double dt_outer, uint64_t* ticket) {
  if (!b || !s || n_outer < 0 || k_inner < 1 || !(dt_outer > 0) || !isfinite(dt_outer)) return MD_ERR_ARG;
  if (s->batch) return MD_ERR_STATE;
  for (auto& kv : b->req)
    if (kv.second.s == s && (kv.second.state == RQ_QUEUED || kv.second.state == RQ_RESIDENT)) return MD_ERR_STATE;
  if (s->r_a > 0) return MD_ERR_ARG;  // distance classes run on single systems only
  if (b->precision < 0) b->precision = s->precision;
  if (s->precision != b->precision) return MD_ERR_ARG;
  Request r;
  r.s = s;
  r.ticket = b->next_ticket++;
  r.n_outer = n_outer;
  r.k = k_inner;
  r.dt_outer = dt_outer;
  b->req[r.ticket] = r;
  b->queue.push_back(r.ticket);
  if (ticket) *ticket = r.ticket;
  return MD_OK;
}

md_status md_batch_run(md_batch* b, int max_ticks) {
  if (!b) return MD_ERR_ARG;
  long long done_ticks = 0;
  for (;;) {
    md_status st = batch_admit(b);
    if (st != MD_OK) return st;
    if (b->resident.empty()) break;
    if (b->dirty) {
      st = batch_build(b);
      if (st != MD_OK) return st;
    }
    st = batch_cycle(b);
    if (st != MD_OK) return st;
    done_ticks += b->P;
    if (max_ticks > 0 && done_ticks >= max_ticks) break;
  }
  return MD_OK;
}

md_status md_batch_poll(md_batch* b, uint64_t ticket, int* done) {
  if (!b || !done) return MD_ERR_ARG;
  auto it = b->req.find(ticket);
  if (it == b->req.end()) return MD_ERR_STATE;
  const int state = it->second.state;
  *done = (state == RQ_DONE || state == RQ_CANCELLED || state == RQ_FAILED) ? 1 : 0;
  if (state == RQ_FAILED || state == RQ_CANCELLED) return it->second.status;
  return MD_OK;
}

md_status md_batch_cancel(md_batch* b, uint64_t ticket) {
  if (!b) return MD_ERR_ARG;
  auto it = b->req.find(ticket);
  if (it == b->req.end()) return MD_ERR_STATE;
  Request& r = it->second;
  if (r.state == RQ_QUEUED) {  // never admitted: the system is untouched
    b->queue.erase(std::find(b->queue.begin(), b->queue.end(), ticket));
    r.state = RQ_CANCELLED;
    r.status = MD_ERR_CANCELLED;
    return MD_OK;
  }
  if (r.state == RQ_RESIDENT) {
    // between md_batch_run calls every member stands at a cycle boundary, inside an outer step (its
    // opening kicks and first drift are done): it finishes that step with the closing kicks, so its
    // state is a full step of Algorithm 2, then leaves
    if (!r.cancel) {
      r.cancel = true;
      r.n_outer = std::min(r.n_outer, r.outer_done + 1);
    }
    return MD_OK;
  }
  return MD_ERR_STATE;  // already finished, failed or cancelled
}

md_status md_batch_latency(md_batch* b, uint64_t ticket, double* ms, int* count) {
  if (!b || !count) return MD_ERR_ARG;
  auto it = b->req.find(ticket);
  if (it == b->req.end()) return MD_ERR_STATE;
  const std::vector<double>& l = it->second.lat_ms;
  const int n = std::min<int>(*count, (int)l.size());
  if (ms)
    for (int i = 0; i < n; ++i) ms[i] = l[i];
  *count = ms ? n : (int)l.size();
  return MD_OK;
}

md_status md_batch_pending(md_batch* b, int* queued, int* resident) {
  if (!b) return MD_ERR_ARG;
  if (queued) *queued = (int)b->queue.size();
  if (resident) *resident = (int)b->resident.size();
  return MD_OK;
}

md_status md_batch_cycles(md_batch* b, uint64_t* cycles, uint64_t* replayed) {
  if (!b) return MD_ERR_ARG;
  if (cycles) *cycles = b->cycles;
  if (replayed) *replayed = b->replayed;
  return MD_OK;
}

md_status md_batch_destroy(md_batch* b) {
  if (!b) return MD_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (uint64_t tk : b->resident) {
    Request& r = b->req[tk];
    r.s->batch = nullptr;
    r.s->batch_lj = false;
    clear_graphs(r.s);
    r.s->forces_valid = false;  // interrupted mid-request: the cached forces are not at a full step
    r.s->energy_valid = false;
  }
  batch_free_composition(b);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return MD_OK;
}

}  // extern "C"
