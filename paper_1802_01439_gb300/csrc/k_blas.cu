// Vector kernels of the solvers: deterministic reductions (fixed grid, fixed
// order, so repeated solves are bit-reproducible), the fused conjugate-gradient
// updates (Sec. 3.3 of arXiv:1802.01439: "vector updates and inner products"
// are a significant part of the CG cost, so each pass does as much as it can),
// precision conversions at the boundary of the mixed-precision V-cycle, and
// the first Chebyshev step from a zero initial guess.
#include <cstdint>
#include "blas.h"

namespace dgns {
namespace {

constexpr int RT = 256;  // threads per reduction block

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of v, result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[RT / 32];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = lane < RT / 32 ? red[lane] : 0.0;
    s = warp_sum(s);
  }
  __syncthreads();
  return s;
}

template <class TA, class TB>
__global__ void __launch_bounds__(RT) dot_partial(const TA* __restrict__ a, const TB* __restrict__ b,
                                                  long long n, double* __restrict__ part) {
  double s = 0.0;
  const long long stride = (long long)gridDim.x * RT;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride)
    s = fma((double)a[i], (double)b[i], s);
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <class T>
__global__ void __launch_bounds__(RT) sum_partial(const T* __restrict__ a, long long n,
                                                  double* __restrict__ part) {
  double s = 0.0;
  const long long stride = (long long)gridDim.x * RT;
  if constexpr (sizeof(T) == 4) {
    // FP32 data: a compensated (Neumaier) FP32 sum per thread, its two parts
    // combined in FP64 for the block (one FP64 addition per thread instead of
    // one per entry, which on this part would bind the kernel to the FP64
    // pipe)
    float hi = 0.f, lo = 0.f;
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride) {
      const float v = (float)a[i], t = hi + v;
      lo += fabsf(hi) >= fabsf(v) ? (hi - t) + v : (v - t) + hi;
      hi = t;
    }
    s = (double)hi + (double)lo;
  } else {
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride) s += (double)a[i];
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out[slot] = sum of the partials (single block, fixed order).
__global__ void __launch_bounds__(RT) finish_sum(const double* __restrict__ part, int np,
                                                 double* __restrict__ scal, int slot) {
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += RT) s += part[i];
  s = block_sum(s);
  if (threadIdx.x == 0) scal[slot] = s;
}

// x += alpha p; r -= alpha Ap; partial sums of r.r, alpha = scal[RZ]/scal[PAP]
__global__ void __launch_bounds__(RT) cg_update_kernel(double* __restrict__ x, double* __restrict__ r,
                                                       const double* __restrict__ p,
                                                       const double* __restrict__ Ap, long long n,
                                                       const double* __restrict__ scal,
                                                       double* __restrict__ part) {
  const double alpha = scal[S_RZ] / scal[S_PAP];
  double s = 0.0;
  const long long stride = (long long)gridDim.x * RT;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, Ap[i], r[i]);
    r[i] = ri;
    s = fma(ri, ri, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// p = z + beta p with beta = scal[RZNEW]/scal[RZ]  (first=1: p = z)
__global__ void __launch_bounds__(RT) cg_direction_kernel(double* __restrict__ p, const double* __restrict__ z,
                                                          long long n, const double* __restrict__ scal,
                                                          int first) {
  const double beta = first ? 0.0 : scal[S_RZNEW] / scal[S_RZ];
  const long long stride = (long long)gridDim.x * RT;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride)
    p[i] = first ? z[i] : fma(beta, p[i], z[i]);
}

__global__ void rotate_kernel(double* scal) { scal[S_RZ] = scal[S_RZNEW]; }

// float -> double without the FP64 pipe (on this part a hardware conversion
// costs the FP64 pipe about as much as an FP64 addition).  For a normal
// float the double has the same sign and significand bits and the exponent
// rebiased from 127 to 1023 (IEEE 754 binary32 -> binary64), so the
// conversion is exact and done on the bit patterns; zeros keep their sign.
// Subnormals, infinities and NaNs take the hardware conversion.
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) {
    if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));
    return (double)f;
  }
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)b);
}
template <class TO, class TI>
__device__ __forceinline__ TO convert_to(TI v) {
  if constexpr (sizeof(TI) == 4 && sizeof(TO) == 8)
    return widen_f32(v);
  else
    return (TO)v;
}

// y = (double) x - mean, mean = scal[slot] / n  (or no shift when slot < 0)
template <class TI, class TO>
__global__ void __launch_bounds__(RT) convert_shift_kernel(const TI* __restrict__ x, TO* __restrict__ y,
                                                           long long n, const double* __restrict__ scal,
                                                           int slot) {
  const long long stride = (long long)gridDim.x * RT;
  if (slot < 0) {
    // no shift: a plain conversion (an FP64 subtraction of zero per entry
    // would cost the FP64 pipe as much as a pass over memory)
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride) y[i] = convert_to<TO>(x[i]);
    return;
  }
  const double mu = scal[slot] / (double)n;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride)
    y[i] = (TO)(convert_to<double>(x[i]) - mu);
}

// z = (double) x - mean (mean = scal[slot] / n; none when slot < 0) and the
// partial sums of (r, z) in the order of dot_partial (same grid, same
// per-thread order), so the sum equals that of a separate dot pass
__global__ void __launch_bounds__(RT) widen_shift_dot_kernel(const float* __restrict__ x, double* __restrict__ z,
                                                             const double* __restrict__ r, long long n,
                                                             const double* __restrict__ scal, int slot,
                                                             double* __restrict__ part) {
  const double mu = slot < 0 ? 0.0 : scal[slot] / (double)n;
  double s = 0.0;
  const long long stride = (long long)gridDim.x * RT;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride) {
    double zi = widen_f32(x[i]);
    if (slot >= 0) zi -= mu;
    z[i] = zi;
    s = fma(r[i], zi, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// x = c * dinv[i % nper] * b  (first Chebyshev step from a zero guess)
template <class T>
__global__ void __launch_bounds__(RT) cheb_first_kernel(const T* __restrict__ b, const T* __restrict__ dinv,
                                                        T* __restrict__ x, long long n, int nper, T c) {
  const long long stride = (long long)gridDim.x * RT;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride)
    x[i] = c * dinv[i % nper] * b[i];
}

// x may alias y (element-wise, each entry read before it is written)
__global__ void __launch_bounds__(RT) axpby_kernel(double* y, const double* x,
                                                   long long n, double a, double b) {
  const long long stride = (long long)gridDim.x * RT;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride)
    y[i] = b == 0.0 ? a * x[i] : fma(a, x[i], b * y[i]);  // b = 0 ignores y's contents
}

// Largest biased exponent of |x_i| over the vector (integer operations on
// the bit patterns; 0 for a zero vector, 2047 when an entry is not finite):
// per-block maximum, then one atomic maximum per block into *out (set to 0
// before the launch).
__global__ void __launch_bounds__(RT) exp_max_kernel(const double* __restrict__ x, long long n,
                                                     unsigned* __restrict__ out) {
  unsigned e = 0;
  const long long stride = (long long)gridDim.x * RT;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride) {
    const unsigned h = (unsigned)((unsigned long long)__double_as_longlong(x[i]) >> 32);
    e = max(e, (h >> 20) & 0x7FFu);
  }
  e = __reduce_max_sync(0xffffffffu, e);
  __shared__ unsigned red[RT / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned m = 0;
    for (int w = 0; w < RT / 32; ++w) m = max(m, red[w]);
    atomicMax(out, m);
  }
}

// y = x * 2^k (exact unless the result leaves the double range); y may be x
__global__ void __launch_bounds__(RT) scale_pow2_kernel(const double* x, double* y, long long n, int k) {
  const long long stride = (long long)gridDim.x * RT;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride) y[i] = ldexp(x[i], k);
}

inline unsigned grid_for(long long n) {
  long long b = (n + RT - 1) / RT;
  if (b > RED_BLOCKS) b = RED_BLOCKS;
  if (b < 1) b = 1;
  return (unsigned)b;
}

inline int status() { return cudaGetLastError() == cudaSuccess ? 0 : 2; }

}  // namespace

int dot(const double* a, const double* b, long long n, Reducer& R, int slot, cudaStream_t s) {
  const unsigned g = grid_for(n);
  dot_partial<double, double><<<g, RT, 0, s>>>(a, b, n, R.part);
  finish_sum<<<1, RT, 0, s>>>(R.part, (int)g, R.scal, slot);
  return status();
}

int dot_f32(const float* a, const float* b, long long n, Reducer& R, int slot, cudaStream_t s) {
  const unsigned g = grid_for(n);
  dot_partial<float, float><<<g, RT, 0, s>>>(a, b, n, R.part);
  finish_sum<<<1, RT, 0, s>>>(R.part, (int)g, R.scal, slot);
  return status();
}

int sum(const double* a, long long n, Reducer& R, int slot, cudaStream_t s) {
  const unsigned g = grid_for(n);
  sum_partial<double><<<g, RT, 0, s>>>(a, n, R.part);
  finish_sum<<<1, RT, 0, s>>>(R.part, (int)g, R.scal, slot);
  return status();
}

int sum_f32(const float* a, long long n, Reducer& R, int slot, cudaStream_t s) {
  const unsigned g = grid_for(n);
  sum_partial<float><<<g, RT, 0, s>>>(a, n, R.part);
  finish_sum<<<1, RT, 0, s>>>(R.part, (int)g, R.scal, slot);
  return status();
}

int cg_update(double* x, double* r, const double* p, const double* Ap, long long n, Reducer& R,
              cudaStream_t s) {
  const unsigned g = grid_for(n);
  cg_update_kernel<<<g, RT, 0, s>>>(x, r, p, Ap, n, R.scal, R.part);
  finish_sum<<<1, RT, 0, s>>>(R.part, (int)g, R.scal, S_RR);
  return status();
}

int cg_direction(double* p, const double* z, long long n, Reducer& R, bool first, cudaStream_t s) {
  cg_direction_kernel<<<grid_for(n), RT, 0, s>>>(p, z, n, R.scal, first ? 1 : 0);
  if (!first) rotate_kernel<<<1, 1, 0, s>>>(R.scal);
  return status();
}

int widen_shift_dot(const float* x, double* z, long long n, Reducer& R, int shift_slot, const double* r,
                    int dot_slot, cudaStream_t s) {
  const unsigned g = grid_for(n);
  widen_shift_dot_kernel<<<g, RT, 0, s>>>(x, z, r, n, R.scal, shift_slot, R.part);
  finish_sum<<<1, RT, 0, s>>>(R.part, (int)g, R.scal, dot_slot);
  return status();
}

int scal_rotate(Reducer& R, cudaStream_t s) {
  rotate_kernel<<<1, 1, 0, s>>>(R.scal);
  return status();
}

int convert_shift(const void* x, bool x32, void* y, bool y32, long long n, const Reducer* R,
                  int slot, cudaStream_t s) {
  const unsigned g = grid_for(n);
  const double* sc = R ? R->scal : nullptr;
  if (!R) slot = -1;
  if (x32 && y32)
    convert_shift_kernel<float, float><<<g, RT, 0, s>>>((const float*)x, (float*)y, n, sc, slot);
  else if (x32)
    convert_shift_kernel<float, double><<<g, RT, 0, s>>>((const float*)x, (double*)y, n, sc, slot);
  else if (y32)
    convert_shift_kernel<double, float><<<g, RT, 0, s>>>((const double*)x, (float*)y, n, sc, slot);
  else
    convert_shift_kernel<double, double><<<g, RT, 0, s>>>((const double*)x, (double*)y, n, sc, slot);
  return status();
}

// The same for FP32 vectors in 16-byte pieces (n and nper multiples of 4,
// 16-byte aligned vectors, n < 2^32): one 32-bit remainder per piece instead
// of a 64-bit one per entry.
__global__ void __launch_bounds__(RT) cheb_first4_kernel(const float4* __restrict__ b, const float* __restrict__ dinv,
                                                         float4* __restrict__ x, unsigned n4, unsigned nper, float c) {
  const unsigned stride = gridDim.x * RT;
  for (unsigned i = blockIdx.x * RT + threadIdx.x; i < n4; i += stride) {
    const unsigned k = (4u * i) % nper;
    const float4 v = b[i];
    x[i] = make_float4(c * dinv[k] * v.x, c * dinv[k + 1] * v.y, c * dinv[k + 2] * v.z, c * dinv[k + 3] * v.w);
  }
}

int cheb_first(bool fp32, const void* b, const void* dinv, void* x, long long n, int nper, double c,
               cudaStream_t s) {
  const unsigned g = grid_for(n);
  const bool v4 = fp32 && n % 4 == 0 && nper % 4 == 0 && n < (1LL << 32) &&
                  ((reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(x)) & 15) == 0;
  if (v4)
    cheb_first4_kernel<<<grid_for(n / 4), RT, 0, s>>>((const float4*)b, (const float*)dinv, (float4*)x,
                                                      (unsigned)(n / 4), (unsigned)nper, (float)c);
  else if (fp32)
    cheb_first_kernel<float><<<g, RT, 0, s>>>((const float*)b, (const float*)dinv, (float*)x, n, nper, (float)c);
  else
    cheb_first_kernel<double><<<g, RT, 0, s>>>((const double*)b, (const double*)dinv, (double*)x, n, nper, c);
  return status();
}

int exp_max(const double* x, long long n, unsigned* out, cudaStream_t s) {
  if (cudaMemsetAsync(out, 0, sizeof(unsigned), s) != cudaSuccess) return 2;
  if (n > 0) exp_max_kernel<<<grid_for(n), RT, 0, s>>>(x, n, out);
  return status();
}

int scale_pow2(const double* x, double* y, long long n, int k, cudaStream_t s) {
  if (n > 0) scale_pow2_kernel<<<grid_for(n), RT, 0, s>>>(x, y, n, k);
  return status();
}

int axpby(double* y, const double* x, long long n, double a, double b, cudaStream_t s) {
  axpby_kernel<<<grid_for(n), RT, 0, s>>>(y, x, n, a, b);
  return status();
}

}  // namespace dgns
