// Solver vector kernels (k_blas.cu).
#pragma once
#include <cuda_runtime.h>

namespace dgns {

constexpr int RED_BLOCKS = 1216;  // 152 SMs x 8: fixed grid of every reduction

// Scalar slots of the device-side CG state.
enum {
  S_RZ = 0,     // (r, z)
  S_RZNEW = 1,  // (r, z) of the new iterate
  S_PAP = 2,    // (p, A p)
  S_RR = 3,     // (r, r)
  S_SUM = 4,    // scratch sum (mean projection)
  S_T0 = 5,
  S_T1 = 6,
  S_NSLOTS = 8
};

struct Reducer {
  double* part = nullptr;  // RED_BLOCKS partial sums
  double* scal = nullptr;  // S_NSLOTS scalars
};

int dot(const double* a, const double* b, long long n, Reducer& R, int slot, cudaStream_t s);
int dot_f32(const float* a, const float* b, long long n, Reducer& R, int slot, cudaStream_t s);
int sum(const double* a, long long n, Reducer& R, int slot, cudaStream_t s);
int sum_f32(const float* a, long long n, Reducer& R, int slot, cudaStream_t s);
// x += alpha p, r -= alpha Ap, scal[S_RR] = (r, r); alpha = scal[S_RZ] / scal[S_PAP]
int cg_update(double* x, double* r, const double* p, const double* Ap, long long n, Reducer& R,
              cudaStream_t s);
// p = z + beta p, beta = scal[S_RZNEW] / scal[S_RZ]; then scal[S_RZ] = scal[S_RZNEW]
int cg_direction(double* p, const double* z, long long n, Reducer& R, bool first, cudaStream_t s);
// y = x - scal[slot] / n  (no shift when R is null), with precision conversion
int convert_shift(const void* x, bool x32, void* y, bool y32, long long n, const Reducer* R,
                  int slot, cudaStream_t s);
// z = (double) x - scal[shift_slot] / n (no shift when shift_slot < 0) and
// scal[dot_slot] = (r, z), summed as dot() sums it
int widen_shift_dot(const float* x, double* z, long long n, Reducer& R, int shift_slot, const double* r,
                    int dot_slot, cudaStream_t s);
// scal[S_RZ] = scal[S_RZNEW]
int scal_rotate(Reducer& R, cudaStream_t s);
// x = c * dinv[i % nper] * b
int cheb_first(bool fp32, const void* b, const void* dinv, void* x, long long n, int nper, double c,
               cudaStream_t s);
// y = a x + b y
int axpby(double* y, const double* x, long long n, double a, double b, cudaStream_t s);
// *out (device) = largest biased exponent of |x_i| (0: all zero, 2047: an
// entry is not finite)
int exp_max(const double* x, long long n, unsigned* out, cudaStream_t s);
// y = x * 2^k, exact; y may alias x
int scale_pow2(const double* x, double* y, long long n, int k, cudaStream_t s);

}  // namespace dgns
