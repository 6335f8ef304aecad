// Staging of a work item's system descriptor in shared memory, ahead of the wait for the previous
// kernel of the stream.  The kernels that use it (LJ, kick/drift, start, combine, binning, cell order
// and scatter) load their work item and descriptor before pdl_wait instead of after it; the rest of
// their loads still follow the wait.
#pragma once

namespace r3b {

// The system descriptor of a block's work item, copied into shared memory before the kernel waits for
// the previous kernel of the stream (pdl_wait).  Work items and descriptors are written by the host
// only, never by a kernel, so these two dependent loads may run while the previous kernel drains;
// after the wait and a block barrier every descriptor field comes from shared memory.
#ifndef R3B_STAGE_SYS
#define R3B_STAGE_SYS 1
#endif
struct StagedSys {
  alignas(16) unsigned char raw[sizeof(SysDev)];
  __device__ __forceinline__ const SysDev& get() const { return *reinterpret_cast<const SysDev*>(raw); }
};
__device__ __forceinline__ void stage_sys(StagedSys& dst, const SysDev* __restrict__ sys, int s) {
  static_assert(sizeof(SysDev) % 8 == 0 && alignof(SysDev) <= 16, "descriptor copied in 8-byte words");
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(sys + s);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(dst.raw);
  for (int i = (int)threadIdx.x; i < (int)(sizeof(SysDev) / 8); i += (int)blockDim.x) d[i] = __ldg(src + i);
}

}  // namespace r3b
