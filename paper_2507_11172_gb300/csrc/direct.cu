// All-triplet ("DirectSum") Axilrod-Teller-Muto forces: open boundaries, no cutoff -- the reference
// method the paper uses for its energy studies (Sec. 4.1: every triplet of the system, no
// periodicity).  Each unordered triplet {i, j, k} of distinct particles contributes once to the
// energy; the force on i is F_i = sum over unordered pairs {j, k} of the other particles of
// pa2 d_j + pb2 d_k (d_v = x_v - x_i, pa2 = 2 dphi/da, a = |d_j|^2, b = |d_k|^2, c = |d_k - d_j|^2),
// so every triplet is evaluated from each of its three members: no scatter, no atomics, and the
// energy of one evaluation is phi / 3.  Same squared-distance algebra as the rotation kernel:
//   phi = nu u^3 (1 + 3/8 P u^2), 2 dphi/da = 3/4 nu u^5 (dP/da - bc (4 + 5/2 P u^2)), u = (abc)^(-1/2).
//
// One CTA per particle i: the displacements of all particles from i (FP64 differences rounded to the
// kernel's precision, with their squared lengths) are staged in shared memory; warp w takes
// j = w, w + W, ... and its lanes k = j + 1 + lane, j + 33 + lane, ...; per j the lane sums
// sum_k pa2 (a scalar, multiplied by d_j once) and sum_k pb2 d_k, and adds the per-j result to a
// compensated (hi, lo) accumulator.  The CTA's lanes are combined in FP64.
#include <math.h>

#include <vector>

#include "../../include/respa3b.h"
#include "md_internal.cuh"

namespace r3b {

constexpr int kDsThreads = 256;

template <typename T>
__device__ __forceinline__ T ds_rsqrt(T q);
template <>
__device__ __forceinline__ float ds_rsqrt<float>(float q) {
  float t;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(q));
  return t * fmaf(-0.5f * q, t * t, 1.5f);  // one Newton-Raphson step
}
template <>
__device__ __forceinline__ double ds_rsqrt<double>(double q) {
  return 1.0 / sqrt(q);
}

template <typename T>
struct DsAcc;
template <>
struct DsAcc<float> {
  CompF c[3];
  __device__ DsAcc() {
    for (int a = 0; a < 3; ++a) c[a].hi = c[a].lo = 0.f;
  }
  __device__ __forceinline__ void add(float x, float y, float z) {
    c[0].add(x);
    c[1].add(y);
    c[2].add(z);
  }
  __device__ __forceinline__ double get(int a) const { return c[a].value(); }
};
template <>
struct DsAcc<double> {
  double c[3];
  __device__ DsAcc() { c[0] = c[1] = c[2] = 0.0; }
  __device__ __forceinline__ void add(double x, double y, double z) {
    c[0] += x;
    c[1] += y;
    c[2] += z;
  }
  __device__ __forceinline__ double get(int a) const { return c[a]; }
};

template <typename T, bool kE>
__global__ void __launch_bounds__(kDsThreads) k_atm_direct(const double* __restrict__ X, int n, double nu_d,
                                                           double* __restrict__ F, double* __restrict__ U) {
  using T4 = typename V4<T>::type;
  extern __shared__ __align__(32) unsigned char ds_raw[];
  T4* D = reinterpret_cast<T4*>(ds_raw);
  __shared__ double red[4][kDsThreads / 32];
  const int i = blockIdx.x;
  const double xi = X[3 * i], yi = X[3 * i + 1], zi = X[3 * i + 2];
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    T4 d;
    if (v == i) {  // i itself: a far, finite stand-in, masked below
      d.x = d.y = d.z = (T)1e3;
      d.w = (T)3e6;
    } else {
      d.x = (T)(X[3 * v] - xi);
      d.y = (T)(X[3 * v + 1] - yi);
      d.z = (T)(X[3 * v + 2] - zi);
      d.w = d.x * d.x + d.y * d.y + d.z * d.z;
    }
    D[v] = d;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int W = kDsThreads / 32;
  DsAcc<T> f;
  T uu = 0;
  for (int j = warp; j < n - 1; j += W) {
    if (j == i) continue;  // warp-uniform
    const T4 dj = D[j];
    const T a = dj.w, a2 = dj.w + dj.w;
    T sa = 0, gx = 0, gy = 0, gz = 0;
    for (int k = j + 1 + lane; k < n; k += 32) {
      const T4 dk = D[k];
      const T okf = k != i ? (T)1 : (T)0;
      const T ex = dk.x - dj.x, ey = dk.y - dj.y, ez = dk.z - dj.z;
      const T c = fma(ez, ez, fma(ey, ey, ex * ex));
      const T b = dk.w;
      const T ab = a * b;
      const T u = ds_rsqrt<T>(ab * c);
      const T ww = u * u;
      const T t3 = ww * u;
      const T t5 = t3 * ww;
      const T sum = (a + b) + c;
      const T Aa = fma((T)-2, c, sum);  // a + b - c
      const T Bb = fma((T)-2, b, sum);  // a - b + c
      const T Cc = fma((T)-2, a, sum);  // -a + b + c
      const T AB = Aa * Bb, AC = Aa * Cc;
      const T P = AB * Cc;
      const T Pa = fma(a2, Cc, -AB);
      const T Pb = fma(b + b, Bb, -AC);
      const T Pw = P * ww;
      const T H = fma((T)2.5, Pw, (T)4);
      const T kk = t5 * okf;
      sa = fma(kk, fma(-(b * c), H, Pa), sa);
      const T pb2 = kk * fma(-(a * c), H, Pb);
      gx = fma(pb2, dk.x, gx);
      gy = fma(pb2, dk.y, gy);
      gz = fma(pb2, dk.z, gz);
      if (kE) uu = fma(t3 * okf, fma((T)0.375, Pw, (T)1), uu);
    }
    f.add(fma(sa, dj.x, gx), fma(sa, dj.y, gy), fma(sa, dj.z, gz));
  }
  // CTA sums in FP64 (3/4 nu for the forces, nu / 3 for the energy)
  double v[4] = {f.get(0), f.get(1), f.get(2), kE ? (double)uu : 0.0};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    v[q] = warp_sum(v[q]);
    if (lane == 0) red[q][warp] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int w = 0; w < W; ++w)
      for (int q = 0; q < 4; ++q) s[q] += red[q][w];
    const double fs = 0.75 * nu_d;
    F[3 * i] = fs * s[0];
    F[3 * i + 1] = fs * s[1];
    F[3 * i + 2] = fs * s[2];
    if (kE) U[i] = nu_d * s[3] / 3.0;
  }
}

// capacity: all displacements staged in shared memory
int direct_max_n(int precision) { return (227 * 1024 - 1024) / (precision ? 32 : 16); }

template <typename T>
static cudaError_t direct_launch(const double* X, int n, double nu, double* F, double* U, cudaStream_t s) {
  const int bytes = n * (int)sizeof(typename V4<T>::type);
  cudaError_t e = cudaFuncSetAttribute(k_atm_direct<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  k_atm_direct<T, true><<<n, kDsThreads, bytes, s>>>(X, n, nu, F, U);
  return cudaGetLastError();
}

cudaError_t launch_atm_direct(const double* X, int n, double nu, int precision, double* F, double* U,
                              cudaStream_t s) {
  return precision ? direct_launch<double>(X, n, nu, F, U, s) : direct_launch<float>(X, n, nu, F, U, s);
}

}  // namespace r3b

extern "C" md_status md_atm_direct(const double* pos, int64_t n, double atm_nu, int precision, double* f3,
                                   double* u3, void* cuda_stream) {
  using namespace r3b;
  if (!pos || !f3 || n < 3 || !(atm_nu >= 0) || !isfinite(atm_nu) || (precision != MD_FP32 && precision != MD_FP64))
    return MD_ERR_ARG;
  if (n > direct_max_n(precision)) return MD_ERR_CAPACITY;
  for (int64_t q = 0; q < 3 * n; ++q)
    if (!isfinite(pos[q])) return MD_ERR_NONFINITE;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const size_t nn = (size_t)n;
  double *X = nullptr, *F = nullptr, *U = nullptr;
  md_status st = MD_OK;
  if (cudaMalloc(&X, 24 * nn) != cudaSuccess || cudaMalloc(&F, 24 * nn) != cudaSuccess ||
      cudaMalloc(&U, 8 * nn) != cudaSuccess) {
    cudaGetLastError();
    st = MD_ERR_OOM;
  }
  std::vector<double> uh(nn);
  cudaError_t e = cudaSuccess;
  if (st == MD_OK) {
    e = cudaMemcpyAsync(X, pos, 24 * nn, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_atm_direct(X, (int)n, atm_nu, precision, F, U, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f3, F, 24 * nn, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(uh.data(), U, 8 * nn, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      st = MD_ERR_CUDA;
    }
  }
  cudaFree(X);
  cudaFree(F);
  cudaFree(U);
  if (st != MD_OK) return st;
  double u = 0.0;
  bool bad = false;
  for (size_t q = 0; q < nn; ++q) u += uh[q];
  for (size_t q = 0; q < 3 * nn; ++q) bad |= !isfinite(f3[q]);
  if (u3) *u3 = u;
  return (bad || !isfinite(u)) ? MD_ERR_NONFINITE : MD_OK;
}
