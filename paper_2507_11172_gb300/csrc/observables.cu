// Observables of the paper's evaluation (Sec. 4.2): pair counts of the radial distribution function.
//
// k_rdf counts every unordered pair {i, j} of the pair list (i < j in sorted order) whose
// minimum-image distance r lies in [edge_b, edge_b+1), edge_b = b * dr, in IEEE double with the CPU
// definition's operation order: d = x_j - x_i per axis, folded by +-L (a listed pair is within the
// list radius, far below L / 2, so the fold is the same as d - L rint(d / L)),
// r = sqrt((dx*dx + dy*dy) + dz*dz).  The bin is found against the products b * dr themselves, so
// the integer counts equal those of a plain CPU histogram of the same positions.  One thread per
// particle; a shared-memory histogram per CTA, added to the global counts at the end.
#include "md_internal.cuh"

namespace r3b {

__device__ __forceinline__ double rdf_fold(double d, double L, double half_L) {
  if (d > half_L) return __dsub_rn(d, L);
  if (d < -half_L) return __dadd_rn(d, L);
  return d;
}

__global__ void __launch_bounds__(256) k_rdf(const SysDev* __restrict__ sys, const PItem* __restrict__ items,
                                            int nbins, double dr, unsigned long long* __restrict__ counts) {
  extern __shared__ unsigned int hist[];
  const PItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) hist[b] = 0u;
  __syncthreads();
  const int n = S.n;
  const int i = it.begin + threadIdx.x;
  if (i < n) {
    const double* __restrict__ X = S.X[it.buf];
    const double xi = X[i], yi = X[n + i], zi = X[2 * n + i];
    const double L = S.L, hL = S.half_L;
    const double rmax = __dmul_rn((double)nbins, dr);
    const int cnt = S.nbr_cnt[i];
    const int* __restrict__ row = S.nbr + nbr_slot(S.maxnb, i, 0);
    for (int t = 0; t < cnt; ++t) {
      const int j = (int)((unsigned)row[t] & kNbrMask);
      if (j <= i) continue;  // each unordered pair once
      const double dx = rdf_fold(__dsub_rn(X[j], xi), L, hL);
      const double dy = rdf_fold(__dsub_rn(X[n + j], yi), L, hL);
      const double dz = rdf_fold(__dsub_rn(X[2 * n + j], zi), L, hL);
      const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
      if (!(r < rmax)) continue;
      int b = min(nbins - 1, max(0, (int)(r / dr)));
      while (b + 1 < nbins && __dmul_rn((double)(b + 1), dr) <= r) ++b;
      while (b > 0 && __dmul_rn((double)b, dr) > r) --b;
      atomicAdd(&hist[b], 1u);
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x)
    if (hist[b]) atomicAdd(&counts[b], (unsigned long long)hist[b]);
}

void launch_rdf(const Launch& L, const PItem* items, int nitems, int nbins, double dr, unsigned long long* counts) {
  if (nitems > 0)
    k_rdf<<<nitems, 256, sizeof(unsigned int) * (size_t)nbins, L.stream>>>(L.sys, items, nbins, dr, counts);
}

}  // namespace r3b
