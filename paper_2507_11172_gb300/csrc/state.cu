// State transfer between the caller's order (n x 3 AoS, as the C ABI takes and returns it) and the
// library's cell-sorted SoA layout, on the device: the host only copies the caller's buffers in and
// out (directly, so pinned caller memory moves by DMA without staging).
#include <map>
#include <mutex>
#include <utility>

#include "md_internal.cuh"

namespace r3b {

bool raise_smem_attr(const void* kernel, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> raised;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  std::lock_guard<std::mutex> lock(mu);
  int& cur = raised[std::make_pair(dev, kernel)];
  if (bytes <= cur) return true;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cur = bytes;
  return true;
}

// position folded into [0, L), with the host definition's operation order (no contraction)
__device__ __forceinline__ double fold_box(double x, double L) {
  double y = __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
  return y >= L ? __dsub_rn(y, L) : y;
}

// Phase 1 of md_set_state: slot q of the sorted layout takes its caller particle's new position
// (folded) and velocity, or keeps its own where the caller passes none; written to the free
// position buffer xo and to v_alt, so nothing changes before the host has checked the flag.
// full = both given: the layout becomes the caller's order (ids written to id_alt).
__global__ void k_put_state(const SysDev* __restrict__ sys, const double* __restrict__ pos,
                            const double* __restrict__ vel, int cur, int full) {
  const SysDev& S = sys[0];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = S.n;
  if (q >= n) return;
  const int o = full ? q : S.id[q];
  if ((unsigned)o >= (unsigned)n) {  // never for a consistent layout
    atomicOr(&S.flags[FLG_STATE], 2);
    return;
  }
  const double* X = S.X[cur];
  double* Xo = S.X[cur ^ 1];
  bool bad = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double x = X[a * n + q], v = S.v[a * n + q];
    if (pos) {
      x = pos[3 * (size_t)o + a];
      bad |= !isfinite(x);
      x = fold_box(x, S.L);
    }
    if (vel) {
      v = vel[3 * (size_t)o + a];
      bad |= !isfinite(v);
    }
    Xo[a * n + q] = x;
    S.v_alt[a * n + q] = v;
  }
  if (full) S.id_alt[q] = q;
  if (bad) atomicOr(&S.flags[FLG_STATE], 1);
}

// caller-order AoS copy of a sorted SoA array (optionally folded into the box)
__global__ void k_take_state(const SysDev* __restrict__ sys, const double* __restrict__ src, double* __restrict__ out,
                             int fold) {
  const SysDev& S = sys[0];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = S.n;
  if (q >= n) return;
  const size_t o = (size_t)(unsigned)S.id[q];
  if (o >= (size_t)n) {  // never for a consistent layout; reported instead of written out of bounds
    atomicOr(&S.flags[FLG_STATE], 2);
    return;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double x = src[a * n + q];
    out[3 * o + a] = fold ? fold_box(x, S.L) : x;
  }
}

void launch_put_state(const Launch& L, int n, const double* pos, const double* vel, int cur, int full) {
  if (n > 0) k_put_state<<<(n + 255) / 256, 256, 0, L.stream>>>(L.sys, pos, vel, cur, full);
}
void launch_take_state(const Launch& L, int n, const double* src, double* out, int fold) {
  if (n > 0) k_take_state<<<(n + 255) / 256, 256, 0, L.stream>>>(L.sys, src, out, fold);
}

}  // namespace r3b
