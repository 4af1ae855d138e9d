// Convective term c_h of Sec. 3.2 of arXiv:1802.01439 (kernels in
// k_convective.cuh): launchers for native FP64 and double-float, and the
// vector-Jacobian product.  The triple-float instantiations live in
// k_convective_tf64.cu (compiled in parallel).
#include "k_convective.cuh"

namespace dgns {

// Supported: Q = floor(3N/2) (the 3/2 rule) and Q = N; arithmetic FP64,
// double-float or triple-float (the 3/2 rule up to N = 11; otherwise FP64).
int convective_launch(int part, const MeshDims& m, const double* u3, double* rface, double* dst3,
                      const ConvHost& t, int arith, cudaStream_t s) {
  const int N = t.N, Q = t.Q;
  if (arith == ARITH_TF64) {
    const int rc = convective_launch_tf64(part, m, u3, rface, dst3, t, s);
    if (rc != 7) return rc;
  }
  const bool emulated = arith == ARITH_DF64;
#define DGNS_CONV(NV)                                                                                 \
  if (N == NV && Q == (3 * NV) / 2)                                                                   \
    return emulated ? launch_conv<DF64, NV, (3 * NV) / 2>(part, m, u3, rface, dst3, t, s)             \
                    : launch_conv<F64, NV, (3 * NV) / 2>(part, m, u3, rface, dst3, t, s);             \
  if (N == NV && Q == NV)                                                                             \
    return emulated ? launch_conv<DF64, NV, NV>(part, m, u3, rface, dst3, t, s)                       \
                    : launch_conv<F64, NV, NV>(part, m, u3, rface, dst3, t, s);
  DGNS_CONV(2)
  DGNS_CONV(3)
  DGNS_CONV(4)
  DGNS_CONV(5)
  DGNS_CONV(6)
  DGNS_CONV(7)
  DGNS_CONV(8)
  DGNS_CONV(9)
  DGNS_CONV(10)
  DGNS_CONV(11)
  DGNS_CONV(12)
#undef DGNS_CONV
  return 7;
}


}  // namespace dgns
