// FP64-wide convective kernels beyond native FP64 (k_convective.cuh),
// compiled apart from the native and double-float ones so that the
// library's translation units build in parallel: the triple-float kernels,
// and the cell kernel with native-FP64 and triple-float blocks side by side.
#include <atomic>

#include "k_convective.cuh"

namespace dgns {
namespace {

// Blocks of the mixed cell kernel: of every `period` consecutive blocks the
// first `nnative` run native FP64.  period 0 selects the built-in split,
// period -1 runs every kernel in triple-float.
std::atomic<int> g_mix_period{0}, g_mix_native{0};

template <int N, int Q>
int launch_conv_mix(int part, const MeshDims& m, const double* u3, double* rface, double* dst3, const ConvHost& h,
                    cudaStream_t s) {
  if (part & 1) {   // face kernel: native FP64
    const int rc = launch_conv<F64, N, Q>(1, m, u3, rface, dst3, h, s);
    if (rc) return rc;
  }
  if (!(part & 2)) return 0;
  constexpr int EPB = conv_fwd_cells_per_block<N>();
  const size_t smem = ((size_t)EPB * ConvLayout<N, Q>::PER + 6 * Q * N + 2 * Q * ((N + 1) / 2)) * sizeof(tf64);
  if (smem > 232448) return 7;
  if (cudaFuncSetAttribute(conv_kernel_mix<N, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 2;
  if (m.E == 0) return 0;
  int period = g_mix_period.load(), nat = g_mix_native.load();
  if (period <= 0 || nat < 0 || nat > period) {   // measured best splits
    period = N <= 3 ? 5 : 4;
    nat = 3;
  }
  const long long blocks = (m.E + EPB - 1) / EPB;
  conv_kernel_mix<N, Q><<<(unsigned)blocks, conv_groups_per_block<N>() * conv_threads<N>(), smem, s>>>(
      u3, rface, dst3, conv_tables<F64, N, Q>(h), conv_tables<TF64, N, Q>(h), m, period, nat);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // namespace

void convective_set_mix(int period, int nnative) {
  g_mix_period.store(period);
  g_mix_native.store(nnative);
}

// Which FP64-wide arrangement runs each convective kernel (3/2 rule), from
// the measured times at ~16.8M DoFs on GB300: the face kernel in
// triple-float where it beat native FP64 (k = 2, 3, 4, 5: 3.58 vs 4.17,
// 4.34 vs 4.61, 3.31 vs 4.09, 4.04 vs 4.11 ms; at k = 9 the even-odd native
// kernel now wins, 2.98 vs 3.72 ms), the cell kernel
// with mixed blocks where that beat native (k = 2: 3 of every 5 blocks
// native, 5.48 vs 7.29 ms; k = 3: 3 of 4, 9.77 vs 11.59 ms); native FP64
// elsewhere (triple-float alone was 0.6-0.95 of native from k = 3 on, the
// mixed cell kernel slower from k = 4 on).
constexpr bool tf64_faces(int N) { return N >= 3 && N <= 6; }
constexpr bool mixed_cells(int N) { return N == 3 || N == 4; }

template <int N, int Q>
int launch_wide(int part, const MeshDims& m, const double* u3, double* rface, double* dst3, const ConvHost& t,
                cudaStream_t s) {
  if (part & 1) {
    const int rc = tf64_faces(N) ? launch_conv<TF64, N, Q>(1, m, u3, rface, dst3, t, s)
                                 : launch_conv<F64, N, Q>(1, m, u3, rface, dst3, t, s);
    if (rc) return rc;
  }
  if (!(part & 2)) return 0;
  if constexpr (mixed_cells(N))   // (the mixed kernel's geometry is that of N = 3, 4)
    return launch_conv_mix<N, Q>(2, m, u3, rface, dst3, t, s);
  else
    return launch_conv<F64, N, Q>(2, m, u3, rface, dst3, t, s);
}

// The 3/2 rule (Q = floor(3N/2)); returns 7 for other N or Q (the caller
// then runs the native kernels).  With the split set to -1 (measurement) the
// triple-float kernels run wherever they fit.
int convective_launch_tf64(int part, const MeshDims& m, const double* u3, double* rface, double* dst3,
                           const ConvHost& t, cudaStream_t s) {
  const int N = t.N, Q = t.Q;
  const bool all_tf = g_mix_period.load() < 0;
#define DGNS_CONV_TF(NV)                                                                          \
  if (N == NV && Q == (3 * NV) / 2)                                                               \
    return all_tf ? launch_conv<TF64, NV, (3 * NV) / 2>(part, m, u3, rface, dst3, t, s)           \
                  : launch_wide<NV, (3 * NV) / 2>(part, m, u3, rface, dst3, t, s);
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
