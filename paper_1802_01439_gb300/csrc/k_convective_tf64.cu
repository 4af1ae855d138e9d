// Triple-float (FP64-wide) instantiations of the convective kernels
// (k_convective.cuh), compiled apart from the native and double-float ones
// so that the library's translation units build in parallel.
#include "k_convective.cuh"

namespace dgns {

// The 3/2 rule (Q = floor(3N/2)) for N <= 11: at N = 12 one cell's work
// space in 12-byte values exceeds the shared memory of an SM.  Returns 7 for
// other N or Q (the caller then runs the native kernels).
int convective_launch_tf64(int part, const MeshDims& m, const double* u3, double* rface, double* dst3,
                           const ConvHost& t, cudaStream_t s) {
  const int N = t.N, Q = t.Q;
#define DGNS_CONV_TF(NV) \
  if (N == NV && Q == (3 * NV) / 2) return launch_conv<TF64, NV, (3 * NV) / 2>(part, m, u3, rface, dst3, t, s);
  DGNS_CONV_TF(2)
  DGNS_CONV_TF(3)
  DGNS_CONV_TF(4)
  DGNS_CONV_TF(5)
  DGNS_CONV_TF(6)
  DGNS_CONV_TF(7)
  DGNS_CONV_TF(8)
  DGNS_CONV_TF(9)
  DGNS_CONV_TF(10)
  DGNS_CONV_TF(11)
#undef DGNS_CONV_TF
  return 7;
}

}  // namespace dgns
