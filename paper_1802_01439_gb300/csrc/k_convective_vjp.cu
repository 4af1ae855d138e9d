// Vector-Jacobian product of the convective term (dC/du)^T w (the reverse
// mode of the BDF2 step's explicit convective term, Sec. 3.2 c_h with the
// 3/2 over-integration rule and the LLF flux): launches of conv_vjp_kernel
// (k_convective.cuh), in a translation unit of its own.  Up to N = 8 the
// kernel keeps u, w and their whole-cell x and y sweeps in shared memory;
// from N = 9 on it contracts plane by plane (z first), with the same flops
// and per-plane buffers only.
#include "k_convective.cuh"

namespace dgns {

int convective_vjp(const MeshDims& m, const double* u3, const double* w3, double* dst3, const ConvHost& t,
                   cudaStream_t s, bool emulated) {
  const int N = t.N, Q = t.Q;
#define DGNS_CONV_VJP(NV, PFV)                                                                     \
  if (N == NV && Q == (3 * NV) / 2)                                                                \
    return emulated ? launch_conv_vjp<DF64, NV, (3 * NV) / 2, PFV>(m, u3, w3, dst3, t, s)          \
                    : launch_conv_vjp<F64, NV, (3 * NV) / 2, PFV>(m, u3, w3, dst3, t, s);          \
  if (N == NV && Q == NV)                                                                          \
    return emulated ? launch_conv_vjp<DF64, NV, NV, PFV>(m, u3, w3, dst3, t, s)                    \
                    : launch_conv_vjp<F64, NV, NV, PFV>(m, u3, w3, dst3, t, s);
  DGNS_CONV_VJP(2, false)
  DGNS_CONV_VJP(3, false)
  DGNS_CONV_VJP(4, false)
  DGNS_CONV_VJP(5, false)
  DGNS_CONV_VJP(6, false)
  DGNS_CONV_VJP(7, false)
  DGNS_CONV_VJP(8, false)
  DGNS_CONV_VJP(9, true)
  DGNS_CONV_VJP(10, true)
  DGNS_CONV_VJP(11, true)
  DGNS_CONV_VJP(12, true)
#undef DGNS_CONV_VJP
  return 7;
}

}  // namespace dgns
