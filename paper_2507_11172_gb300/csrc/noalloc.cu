// Allocation-free ATM force evaluation.
//
// Some callers cannot allocate device memory: code running inside another
// framework's memory pool, a process whose allocator is locked down, or a
// caller that must not trigger the device synchronisation that cudaMalloc and
// cudaFree imply.  md_atm_forces_noalloc serves them: it computes the
// Axilrod-Teller-Muto forces of one configuration with every intermediate
// array (cell lists, sorted coordinates, per-stencil partial forces, work
// lists, the system descriptor and the pair table) in the file-scope arrays
// below, which every GPU that loads the library holds until the process
// exits.  The caller passes the positions and the force output in device
// memory.  Calls share the arrays, so calls that overlap on the GPU (other
// threads, other streams) race and must be serialised by the caller.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/respa3b.h"
#include "md_internal.cuh"

using namespace r3b;

namespace {

constexpr int kMaxN = MD_NOALLOC_MAX_N;
constexpr int kMaxCellsPerSide = 32;
constexpr int kMaxCells = kMaxCellsPerSide * kMaxCellsPerSide * kMaxCellsPerSide;
constexpr int kMaxItems = kMaxCells + (kMaxN + 255) / 256 + 1;

// byte layout of the scratch array (offsets are multiples of 256)
constexpr size_t up256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffSys = 0;
constexpr size_t kOffX0 = up256(kOffSys + sizeof(SysDev));
constexpr size_t kOffX1 = up256(kOffX0 + 24ull * kMaxN);
constexpr size_t kOffV = up256(kOffX1 + 24ull * kMaxN);
constexpr size_t kOffVa = up256(kOffV + 24ull * kMaxN);
constexpr size_t kOffF3 = up256(kOffVa + 24ull * kMaxN);
constexpr size_t kOffId = up256(kOffF3 + 24ull * kMaxN);
constexpr size_t kOffIda = up256(kOffId + 4ull * kMaxN);
constexpr size_t kOffPcell = up256(kOffIda + 4ull * kMaxN);
constexpr size_t kOffCtmp = up256(kOffPcell + 4ull * kMaxN);
constexpr size_t kOffRank = up256(kOffCtmp + 4ull * kMaxN);
constexpr size_t kOffPos = up256(kOffRank + 4ull * kMaxN);
constexpr size_t kOffPosLo = up256(kOffPos + 16ull * kMaxN);
constexpr size_t kOffRef = up256(kOffPosLo + 16ull * kMaxN);
constexpr size_t kOffCount = up256(kOffRef + 16ull * kMaxN);
constexpr size_t kOffStart = up256(kOffCount + 4ull * kMaxCells);
constexpr size_t kOffPart = up256(kOffStart + 4ull * (kMaxCells + 1));
constexpr size_t kOffAcc = up256(kOffPart + 4ull * 27 * 3 * kMaxN);
constexpr size_t kOffCtr = up256(kOffAcc + 8ull * ACC_N);
constexpr size_t kOffFlags = up256(kOffCtr + 8ull * CTR_N);
constexpr size_t kOffNbrCnt = up256(kOffFlags + 4ull * FLG_N);
constexpr size_t kOffPItems = up256(kOffNbrCnt + 4ull * kMaxN);
constexpr size_t kOffCItems = up256(kOffPItems + sizeof(PItem) * ((kMaxN + 255) / 256));
constexpr size_t kOffSItem = up256(kOffCItems + sizeof(CItem) * kMaxCells);
constexpr size_t kScratchBytes = up256(kOffSItem + sizeof(SItem));
static_assert(kScratchBytes <= (size_t)9 << 20, "the scratch array must stay modest (at most 9 MiB; 8.8 MiB as laid out)");
static_assert(kMaxItems > 0, "");

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];
static __device__ __align__(256) uint16_t g_noalloc_table[kPairTable];

namespace {

// AoS caller positions -> SoA slots in caller order; ids = identity; velocities zero
__global__ void k_noalloc_pack(const double* __restrict__ pos, int n, double* __restrict__ X,
                               double* __restrict__ v, int* __restrict__ id) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    X[a * n + i] = pos[3 * i + a];
    v[a * n + i] = 0.0;
  }
  id[i] = i;
}

// sorted SoA forces -> caller-order AoS output
__global__ void k_noalloc_unpack(const double* __restrict__ f3, const int* __restrict__ id, int n,
                                 double* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int o = id[q];
#pragma unroll
  for (int a = 0; a < 3; ++a) out[3 * o + a] = f3[a * n + q];
}

struct DeviceSetup {
  bool done = false;
  unsigned char* scratch = nullptr;
  uint16_t* table = nullptr;
  int per_sm = 0;
  int smem_cap = 0;
};
std::mutex g_setup_mutex;
DeviceSetup g_setup[64];
// messages go to the string md_last_error returns
void set_error(const std::string& msg) { set_last_error(msg.c_str()); }

md_status fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return MD_ERR_CUDA;
}

// once per device, with that device current: device addresses of the arrays and the pair table
md_status setup_device(int dev, cudaStream_t stream, DeviceSetup** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (dev < 0 || dev >= 64) return MD_ERR_ARG;
  DeviceSetup& d = g_setup[dev];
  if (!d.done) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(e, "cudaGetSymbolAddress(scratch)");
    d.scratch = static_cast<unsigned char*>(p);
    e = cudaGetSymbolAddress(&p, g_noalloc_table);
    if (e != cudaSuccess) return fail(e, "cudaGetSymbolAddress(table)");
    d.table = static_cast<uint16_t*>(p);
    std::vector<uint16_t> h(kPairTable);
    int q = 0;
    for (int k = 1; k < kMaxHalf; ++k)
      for (int j = 0; j < k; ++j) h[q++] = (uint16_t)(j | (k << 8));
    e = cudaMemcpyAsync(d.table, h.data(), sizeof(uint16_t) * kPairTable, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return fail(e, "cudaMemcpyAsync(table)");
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(e, "cudaStreamSynchronize");
    d.done = true;
  }
  *out = &d;
  return MD_OK;
}

}  // namespace

extern "C" md_status md_atm_forces_noalloc(const double* d_pos, int64_t n, double box_L, double atm_nu,
                                           double rc_triplet, double* d_f3, double* u3, uint64_t* triplets,
                                           void* cuda_stream) {
  if (!d_pos || !d_f3 || n < 3 || !(box_L > 0) || !isfinite(box_L) || !(rc_triplet > 0) || !isfinite(rc_triplet) ||
      !(atm_nu >= 0) || !isfinite(atm_nu))
    return MD_ERR_ARG;
  if (n > kMaxN) {
    set_error("md_atm_forces_noalloc: n exceeds MD_NOALLOC_MAX_N");
    return MD_ERR_CAPACITY;
  }
  if (!(box_L > 3.0 * rc_triplet)) return MD_ERR_BOX_TOO_SMALL;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fail(ce, "cudaGetDevice");
  DeviceSetup* D = nullptr;
  md_status st = setup_device(dev, stream, &D);
  if (st != MD_OK) return st;

  const int nn = (int)n;
  int nc = (int)floor(box_L / rc_triplet);
  nc = std::min(std::max(nc, 3), kMaxCellsPerSide);
  const int ncell = nc * nc * nc;
  const double edge = box_L / nc;
  unsigned char* m = D->scratch;

  // work items: particle blocks of 256 and one base cell per ATM item
  std::vector<PItem> pit;
  for (int b = 0; b < (nn + 255) / 256; ++b) pit.push_back(PItem{0, b * 256, CB_INIT, 0});
  std::vector<CItem> cit(ncell);
  for (int c = 0; c < ncell; ++c) cit[c] = CItem{0, c, 0, M_ENERGY};
  SItem sit{0, 0};
  PItem* d_pit = reinterpret_cast<PItem*>(m + kOffPItems);
  CItem* d_cit = reinterpret_cast<CItem*>(m + kOffCItems);
  SItem* d_sit = reinterpret_cast<SItem*>(m + kOffSItem);

  int cap = std::max(16, (int)ceil(1.5 * (double)nn / ncell + 12.0));
  for (int attempt = 0; attempt < 4; ++attempt) {
    int smem = 0;
    const int per_sm = atm_configure(atm_stage_capacity(cap), MD_FP32, &smem);
    if (per_sm <= 0) {
      set_error("md_atm_forces_noalloc: a cell holds more particles than shared memory can stage");
      return MD_ERR_CAPACITY;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::min(ncell, per_sm * std::max(sms, 1));

    SysDev h;
    memset(&h, 0, sizeof(h));
    h.L = box_L;
    h.half_L = 0.5 * box_L;
    h.edge = edge;
    h.inv_edge = 1.0 / edge;
    h.nc = nc;
    h.ncell = ncell;
    h.n = nn;
    h.cap_cell = cap;
    h.nu = atm_nu;
    h.rc3 = rc_triplet;
    h.rc3sq = rc_triplet * rc_triplet;
    h.guard3 = 2e-5 * std::max(1.0, h.rc3sq);
    h.mass = 1.0;
    h.inv_mass = 1.0;
    h.X[0] = reinterpret_cast<double*>(m + kOffX0);
    h.X[1] = reinterpret_cast<double*>(m + kOffX1);
    h.v = reinterpret_cast<double*>(m + kOffV);
    h.v_alt = reinterpret_cast<double*>(m + kOffVa);
    h.f2 = reinterpret_cast<double*>(m + kOffF3);
    h.f3 = reinterpret_cast<double*>(m + kOffF3);
    h.id = reinterpret_cast<int*>(m + kOffId);
    h.id_alt = reinterpret_cast<int*>(m + kOffIda);
    h.pcell = reinterpret_cast<int*>(m + kOffPcell);
    h.cell_tmp = reinterpret_cast<int*>(m + kOffCtmp);
    h.rank = reinterpret_cast<int*>(m + kOffRank);
    h.pos[0] = m + kOffPos;
    h.pos[1] = m + kOffPos;
    h.poslo = m + kOffPosLo;
    h.ref = m + kOffRef;
    h.count = reinterpret_cast<int*>(m + kOffCount);
    h.cell_start = reinterpret_cast<int*>(m + kOffStart);
    h.nbr_cnt = reinterpret_cast<int*>(m + kOffNbrCnt);
    h.partial = m + kOffPart;
    h.acc = reinterpret_cast<double*>(m + kOffAcc);
    h.ctr = reinterpret_cast<unsigned long long*>(m + kOffCtr);
    h.flags = reinterpret_cast<int*>(m + kOffFlags);

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
  }
#define NA_CK(call)                                  \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return fail(e_, #call);   \
  } while (0)
    NA_CK(cudaMemcpyAsync(m + kOffSys, &h, sizeof(SysDev), cudaMemcpyHostToDevice, stream));
    NA_CK(cudaMemcpyAsync(d_pit, pit.data(), sizeof(PItem) * pit.size(), cudaMemcpyHostToDevice, stream));
    NA_CK(cudaMemcpyAsync(d_cit, cit.data(), sizeof(CItem) * cit.size(), cudaMemcpyHostToDevice, stream));
    NA_CK(cudaMemcpyAsync(d_sit, &sit, sizeof(SItem), cudaMemcpyHostToDevice, stream));
    // the arrays keep the previous call's contents: clear what must start at zero
    NA_CK(cudaMemsetAsync(h.count, 0, 4ull * ncell, stream));
    NA_CK(cudaMemsetAsync(m + kOffAcc, 0, kOffNbrCnt - kOffAcc, stream));

    Launch L{stream, reinterpret_cast<const SysDev*>(m + kOffSys)};
    const int nb = (nn + 255) / 256;
    k_noalloc_pack<<<nb, 256, 0, stream>>>(d_pos, nn, h.X[0], h.v, h.id);
    launch_bin_count(L, d_pit, nb, 256);
    launch_scan(L, d_sit, 1);
    launch_scatter<float>(L, d_pit, nb, 256);  // sorted positions land in X[1]
    NA_CK(cudaMemcpyAsync(h.X[0], h.X[1], 24ull * nn, cudaMemcpyDeviceToDevice, stream));
    launch_atm_table<float>(L, d_cit, ncell, grid, atm_stage_capacity(cap), D->table);
    launch_combine<float>(L, d_pit, nb, 256);
    k_noalloc_unpack<<<nb, 256, 0, stream>>>(h.f3, h.id_alt, nn, d_f3);
    NA_CK(cudaGetLastError());
    int flags[FLG_N];
    double acc[ACC_N];
    unsigned long long ctr[CTR_N];
    NA_CK(cudaMemcpyAsync(flags, h.flags, sizeof(flags), cudaMemcpyDeviceToHost, stream));
    NA_CK(cudaMemcpyAsync(acc, h.acc, sizeof(acc), cudaMemcpyDeviceToHost, stream));
    NA_CK(cudaMemcpyAsync(ctr, h.ctr, sizeof(ctr), cudaMemcpyDeviceToHost, stream));
    NA_CK(cudaStreamSynchronize(stream));
#undef NA_CK
    if (flags[FLG_ERR] & ERR_CELL_CAP) {  // a denser cell than assumed: stage more and repeat
      cap = std::max(cap + 8, flags[FLG_MAXCELL] + 8);
      continue;
    }
    if (flags[FLG_ERR] & ERR_HALF_CAP) {
      set_error("md_atm_forces_noalloc: a particle has more than 128 larger-index neighbours");
      return MD_ERR_CAPACITY;
    }
    if (flags[FLG_ERR] & ERR_NONFINITE) return MD_ERR_NONFINITE;
    if (u3) *u3 = acc[ACC_U3];
    if (triplets) *triplets = ctr[CTR_TRIPLETS];
    return MD_OK;
  }
  set_error("md_atm_forces_noalloc: cell capacity retries exhausted");
  return MD_ERR_CAPACITY;
}
