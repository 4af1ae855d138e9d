// Velocity divergence d_h and pressure gradient g_h with central fluxes
// (Sec. 3.2 of arXiv:1802.01439), FP64, mixed degrees (k_u, k_p).
//
// With exact Gauss quadrature on affine Cartesian cells both are sums of
// Kronecker products of 1D matrices:
//   D u = Mpu_z [Mpu_y R_x u_x + Mpu_x R_y u_y] + Mpu_y Mpu_x R_z u_z
//   (G p)_x = Mup_z Mup_y G_x p,  (G p)_y = Mup_z Mup_x G_y p,
//   (G p)_z = Mup_y Mup_x G_z p
// R_d / G_d are the 1D derivative-plus-face line operators (scaled by the
// tangential cell sizes) and Mpu / Mup the mixed 1D mass matrices.  The
// neighbour terms of the central flux need only the neighbour's face value
// on the shared face (one entry per line: the LGL basis interpolates there).
// The neighbour-coupled sweep is applied first, on raw data, so that the
// neighbour values need no further transformation.
#include "arith.cuh"
#include "ops.h"

namespace dgns {
namespace {

template <int NU>
constexpr int dg_cells_per_block() {
  return NU * NU >= 128 ? 1 : 128 / (NU * NU);
}

template <class V, int NU, int NP>
struct DivTab {
  V R[3][NP * NU];
  V Mpu[NP * NU];
  V nbr[3], nbl[3];
};

template <class V, int NU, int NP>
struct GradTab {
  V G[3][NU * NP];
  V Mup[NU * NP];
  V nbr[3], nbl[3];
};

// out-line = A (NO x NI) in-line (+ add-line); extents of in and out arrays
// differ only in direction D.
template <class P, int NO, int NI, int D, bool ADD>
__device__ __forceinline__ void rect_line(const typename P::V* in, const typename P::V* add,
                                          typename P::V* out, int l, int i0, int i1, int i2, int o0, int o1,
                                          int o2, const typename P::V* A) {
  typedef typename P::V V;
  typedef typename P::Acc Acc;
  int bi, si, bo, so;
  line_geom<D>(l, i0, i1, i2, bi, si);
  line_geom<D>(l, o0, o1, o2, bo, so);
  V x[NI];
  load_line<V, NI>(in, bi, si, x);
#pragma unroll
  for (int i = 0; i < NO; ++i) {
    Acc y;
    if (ADD)
      P::acc_set(y, add[bo + i * so]);
#pragma unroll
    for (int j = 0; j < NI; ++j) {
      if (ADD || j > 0)
        P::acc_fma(y, A[i * NI + j], x[j]);
      else
        P::acc_first(y, A[i * NI + j], x[j]);
    }
    out[bo + i * so] = P::acc_get(y);
  }
}

// Neighbour-coupled line: y = A x + (nbr * xr[0] into y[NO-1]) + (nbl * xl[NI-1] into y[0])
template <class P, int NO, int NI, int D>
__device__ __forceinline__ void flux_line(const typename P::V* in, const double* __restrict__ nbR,
                                          const double* __restrict__ nbL, typename P::V* out, int l, int i0,
                                          int i1, int i2, int o0, int o1, int o2, const typename P::V* A,
                                          typename P::V cr, typename P::V cl) {
  typedef typename P::V V;
  typedef typename P::Acc Acc;
  int bi, si, bo, so;
  line_geom<D>(l, i0, i1, i2, bi, si);
  line_geom<D>(l, o0, o1, o2, bo, so);
  V x[NI];
  load_line<V, NI>(in, bi, si, x);
  const V vr = P::load(nbR + bi), vl = P::load(nbL + bi + (NI - 1) * si);
#pragma unroll
  for (int i = 0; i < NO; ++i) {
    Acc y;
    P::acc_first(y, A[i * NI], x[0]);
#pragma unroll
    for (int j = 1; j < NI; ++j) P::acc_fma(y, A[i * NI + j], x[j]);
    if (i == NO - 1) P::acc_fma(y, cr, vr);
    if (i == 0) P::acc_fma(y, cl, vl);
    out[bo + i * so] = P::acc_get(y);
  }
}

struct CellPos {
  long long el;
  int ex, ey, ez;
};

__device__ __forceinline__ CellPos cell_pos(long long el, const MeshDims& m) {
  CellPos p;
  p.el = el;
  p.ex = (int)(el % m.nx);
  const long long t = el / m.nx;
  p.ey = (int)(t % m.ny);
  p.ez = (int)(t / m.ny);
  return p;
}

template <class P, int NU, int NP>
__global__ void __launch_bounds__(dg_cells_per_block<NU>() * NU * NU)
    div_kernel(const double* __restrict__ u3, double* __restrict__ dst,
               const __grid_constant__ DivTab<typename P::V, NU, NP> tb, const MeshDims m) {
  typedef typename P::V V;
  constexpr int EPB = dg_cells_per_block<NU>(), NT = NU * NU;
  constexpr int NU3 = NU * NU * NU, NP3 = NP * NP * NP, W = NP * NU * NU;
  // per cell: ux, uy, uz (NU3 each), A, B, C (W each), A2, B2, C2 (NP*NP*NU each)
  constexpr int PER = 3 * NU3 + 3 * W + 3 * NP * NP * NU;
  V* sm = reinterpret_cast<V*>(dyn_smem());
  const int slot = threadIdx.x / NT;
  const int t = threadIdx.x - slot * NT;
  const long long c0 = (long long)blockIdx.x * EPB;
  const long long rem = m.E - c0;
  const int nvalid = rem < EPB ? (int)rem : EPB;
  V* S = sm + slot * PER;
  V* U[3] = {S, S + NU3, S + 2 * NU3};
  V* A = S + 3 * NU3;
  V* B = A + W;
  V* C = B + W;
  V* A2 = C + W;
  V* B2 = A2 + NP * NP * NU;
  V* C2 = B2 + NP * NP * NU;
  const bool active = slot < nvalid;
  CellPos p{};
  if (active) {
    p = cell_pos(c0 + slot, m);
    for (int c = 0; c < 3; ++c)
      for (int i = t; i < NU3; i += NT) U[c][i] = P::load(u3 + (c * m.E + p.el) * NU3 + i);
  }
  __syncthreads();
  if (active) {
    // neighbour-coupled sweeps: R_x u_x (x-lines), R_y u_y, R_z u_z
    const double* cx = u3;
    const double* cy = u3 + m.E * NU3;
    const double* cz = u3 + 2 * m.E * NU3;
    for (int l = t; l < NU * NU; l += NT) {
      flux_line<P, NP, NU, 0>(U[0], cx + neighbor<0>(p.el, p.ex, p.ey, p.ez, +1, m) * NU3,
                           cx + neighbor<0>(p.el, p.ex, p.ey, p.ez, -1, m) * NU3, A, l, NU, NU, NU, NP,
                           NU, NU, tb.R[0], tb.nbr[0], tb.nbl[0]);
      flux_line<P, NP, NU, 1>(U[1], cy + neighbor<1>(p.el, p.ex, p.ey, p.ez, +1, m) * NU3,
                           cy + neighbor<1>(p.el, p.ex, p.ey, p.ez, -1, m) * NU3, B, l, NU, NU, NU, NU,
                           NP, NU, tb.R[1], tb.nbr[1], tb.nbl[1]);
      flux_line<P, NP, NU, 2>(U[2], cz + neighbor<2>(p.el, p.ex, p.ey, p.ez, +1, m) * NU3,
                           cz + neighbor<2>(p.el, p.ex, p.ey, p.ez, -1, m) * NU3, C, l, NU, NU, NU, NU,
                           NU, NP, tb.R[2], tb.nbr[2], tb.nbl[2]);
    }
  }
  __syncthreads();
  if (active) {
    // A: (NP,NU,NU) -y-> A2 (NP,NP,NU); B: (NU,NP,NU) -x-> B2 (NP,NP,NU);
    // C: (NU,NU,NP) -x-> C2 (NP,NU,NP)
    for (int l = t; l < NP * NU; l += NT) {
      rect_line<P, NP, NU, 1, false>(A, nullptr, A2, l, NP, NU, NU, NP, NP, NU, tb.Mpu);
      rect_line<P, NP, NU, 0, false>(B, nullptr, B2, l, NU, NP, NU, NP, NP, NU, tb.Mpu);
      rect_line<P, NP, NU, 0, false>(C, nullptr, C2, l, NU, NU, NP, NP, NU, NP, tb.Mpu);
    }
  }
  __syncthreads();
  if (active) {
    // A2 += B2; C2 (NP,NU,NP) -y-> C (NP,NP,NP)
    for (int i = t; i < NP * NP * NU; i += NT) A2[i] = P::add(A2[i], B2[i]);
    for (int l = t; l < NP * NP; l += NT)
      rect_line<P, NP, NU, 1, false>(C2, nullptr, C, l, NP, NU, NP, NP, NP, NP, tb.Mpu);
  }
  __syncthreads();
  if (active) {
    // out = Mpu_z A2 + C  (z-lines), into B
    for (int l = t; l < NP * NP; l += NT)
      rect_line<P, NP, NU, 2, true>(A2, C, B, l, NP, NP, NU, NP, NP, NP, tb.Mpu);
  }
  __syncthreads();
  if (active)
    for (int i = t; i < NP3; i += NT) dst[p.el * NP3 + i] = P::store(B[i]);
}

template <class P, int NU, int NP>
__global__ void __launch_bounds__(dg_cells_per_block<NU>() * NU * NU)
    grad_kernel(const double* __restrict__ pr, double* __restrict__ dst3,
                const __grid_constant__ GradTab<typename P::V, NU, NP> tb, const MeshDims m) {
  typedef typename P::V V;
  constexpr int EPB = dg_cells_per_block<NU>(), NT = NU * NU;
  constexpr int NU3 = NU * NU * NU, NP3 = NP * NP * NP, W1 = NU * NP * NP, W2 = NU * NU * NP;
  constexpr int PER = NP3 + 3 * W1 + 3 * W2 + 3 * NU3;
  V* sm = reinterpret_cast<V*>(dyn_smem());
  const int slot = threadIdx.x / NT;
  const int t = threadIdx.x - slot * NT;
  const long long c0 = (long long)blockIdx.x * EPB;
  const long long rem = m.E - c0;
  const int nvalid = rem < EPB ? (int)rem : EPB;
  V* S = sm + slot * PER;
  V* Pp = S;
  V* A = Pp + NP3;
  V* B = A + W1;
  V* C = B + W1;
  V* A2 = C + W1;
  V* B2 = A2 + W2;
  V* C2 = B2 + W2;
  V* O = C2 + W2;  // 3 * NU3
  const bool active = slot < nvalid;
  CellPos p{};
  if (active) {
    p = cell_pos(c0 + slot, m);
    for (int i = t; i < NP3; i += NT) Pp[i] = P::load(pr + p.el * NP3 + i);
  }
  __syncthreads();
  if (active) {
    for (int l = t; l < NP * NP; l += NT) {
      flux_line<P, NU, NP, 0>(Pp, pr + neighbor<0>(p.el, p.ex, p.ey, p.ez, +1, m) * NP3,
                           pr + neighbor<0>(p.el, p.ex, p.ey, p.ez, -1, m) * NP3, A, l, NP, NP, NP, NU,
                           NP, NP, tb.G[0], tb.nbr[0], tb.nbl[0]);
      flux_line<P, NU, NP, 1>(Pp, pr + neighbor<1>(p.el, p.ex, p.ey, p.ez, +1, m) * NP3,
                           pr + neighbor<1>(p.el, p.ex, p.ey, p.ez, -1, m) * NP3, B, l, NP, NP, NP, NP,
                           NU, NP, tb.G[1], tb.nbr[1], tb.nbl[1]);
      flux_line<P, NU, NP, 2>(Pp, pr + neighbor<2>(p.el, p.ex, p.ey, p.ez, +1, m) * NP3,
                           pr + neighbor<2>(p.el, p.ex, p.ey, p.ez, -1, m) * NP3, C, l, NP, NP, NP, NP,
                           NP, NU, tb.G[2], tb.nbr[2], tb.nbl[2]);
    }
  }
  __syncthreads();
  if (active) {
    // A (NU,NP,NP) -y-> A2 (NU,NU,NP); B (NP,NU,NP) -x-> B2 (NU,NU,NP);
    // C (NP,NP,NU) -x-> C2 (NU,NP,NU)
    for (int l = t; l < NU * NP; l += NT) {
      rect_line<P, NU, NP, 1, false>(A, nullptr, A2, l, NU, NP, NP, NU, NU, NP, tb.Mup);
      rect_line<P, NU, NP, 0, false>(B, nullptr, B2, l, NP, NU, NP, NU, NU, NP, tb.Mup);
      rect_line<P, NU, NP, 0, false>(C, nullptr, C2, l, NP, NP, NU, NU, NP, NU, tb.Mup);
    }
  }
  __syncthreads();
  if (active) {
    for (int l = t; l < NU * NU; l += NT) {
      rect_line<P, NU, NP, 2, false>(A2, nullptr, O, l, NU, NU, NP, NU, NU, NU, tb.Mup);
      rect_line<P, NU, NP, 2, false>(B2, nullptr, O + NU3, l, NU, NU, NP, NU, NU, NU, tb.Mup);
      rect_line<P, NU, NP, 1, false>(C2, nullptr, O + 2 * NU3, l, NU, NP, NU, NU, NU, NU, tb.Mup);
    }
  }
  __syncthreads();
  if (active)
    for (int c = 0; c < 3; ++c)
      for (int i = t; i < NU3; i += NT) dst3[(c * m.E + p.el) * NU3 + i] = P::store(O[c * NU3 + i]);
}

template <class P, int NU, int NP>
int launch_div(const MeshDims& m, const double* u3, double* dst, const DivHost& h, cudaStream_t s) {
  DivTab<typename P::V, NU, NP> tb;
  for (int d = 0; d < 3; ++d) {
    for (int i = 0; i < NP * NU; ++i) tb.R[d][i] = P::make(h.R[d][i]);
    tb.nbr[d] = P::make(h.nbr[d]);
    tb.nbl[d] = P::make(h.nbl[d]);
  }
  for (int i = 0; i < NP * NU; ++i) tb.Mpu[i] = P::make(h.Mpu[i]);
  constexpr int EPB = dg_cells_per_block<NU>();
  constexpr int PER = 3 * NU * NU * NU + 3 * NP * NU * NU + 3 * NP * NP * NU;
  const size_t smem = (size_t)EPB * PER * sizeof(double);
  if (cudaFuncSetAttribute(div_kernel<P, NU, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 2;
  if (m.E == 0) return 0;
  const long long blocks = (m.E + EPB - 1) / EPB;
  div_kernel<P, NU, NP><<<(unsigned)blocks, EPB * NU * NU, smem, s>>>(u3, dst, tb, m);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

template <class P, int NU, int NP>
int launch_grad(const MeshDims& m, const double* p, double* dst3, const GradHost& h, cudaStream_t s) {
  GradTab<typename P::V, NU, NP> tb;
  for (int d = 0; d < 3; ++d) {
    for (int i = 0; i < NP * NU; ++i) tb.G[d][i] = P::make(h.G[d][i]);
    tb.nbr[d] = P::make(h.nbr[d]);
    tb.nbl[d] = P::make(h.nbl[d]);
  }
  for (int i = 0; i < NP * NU; ++i) tb.Mup[i] = P::make(h.Mup[i]);
  constexpr int EPB = dg_cells_per_block<NU>();
  constexpr int PER = NP * NP * NP + 3 * NU * NP * NP + 3 * NU * NU * NP + 3 * NU * NU * NU;
  const size_t smem = (size_t)EPB * PER * sizeof(double);
  if (cudaFuncSetAttribute(grad_kernel<P, NU, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 2;
  if (m.E == 0) return 0;
  const long long blocks = (m.E + EPB - 1) / EPB;
  grad_kernel<P, NU, NP><<<(unsigned)blocks, EPB * NU * NU, smem, s>>>(p, dst3, tb, m);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // namespace

// Supported pairs: k_p = k_u - 1 (the paper's mixed-order spaces, Sec. 3.2)
// and k_p = k_u (equal order).
#define DGNS_DG_CASES(FN, POL, ...)                                   \
  if (Nu == Np + 1) {                                            \
    switch (Nu) {                                                \
      case 3: return FN<POL, 3, 2>(__VA_ARGS__);                      \
      case 4: return FN<POL, 4, 3>(__VA_ARGS__);                      \
      case 5: return FN<POL, 5, 4>(__VA_ARGS__);                      \
      case 6: return FN<POL, 6, 5>(__VA_ARGS__);                      \
      case 7: return FN<POL, 7, 6>(__VA_ARGS__);                      \
      case 8: return FN<POL, 8, 7>(__VA_ARGS__);                      \
      case 9: return FN<POL, 9, 8>(__VA_ARGS__);                      \
      case 10: return FN<POL, 10, 9>(__VA_ARGS__);                    \
      case 11: return FN<POL, 11, 10>(__VA_ARGS__);                   \
      case 12: return FN<POL, 12, 11>(__VA_ARGS__);                   \
    }                                                            \
  } else if (Nu == Np) {                                         \
    switch (Nu) {                                                \
      case 2: return FN<POL, 2, 2>(__VA_ARGS__);                      \
      case 3: return FN<POL, 3, 3>(__VA_ARGS__);                      \
      case 4: return FN<POL, 4, 4>(__VA_ARGS__);                      \
      case 5: return FN<POL, 5, 5>(__VA_ARGS__);                      \
    }                                                            \
  }                                                              \
  return 7;

template <class POL>
int divergence_apply_p(const MeshDims& m, const double* u3, double* dst, const DivHost& t, cudaStream_t s) {
  const int Nu = t.Nu, Np = t.Np;
  DGNS_DG_CASES(launch_div, POL, m, u3, dst, t, s)
}

template <class POL>
int gradient_apply_p(const MeshDims& m, const double* p, double* dst3, const GradHost& t, cudaStream_t s) {
  const int Nu = t.Nu, Np = t.Np;
  DGNS_DG_CASES(launch_grad, POL, m, p, dst3, t, s)
}

int divergence_apply(const MeshDims& m, const double* u3, double* dst, const DivHost& t, cudaStream_t s,
                     bool emulated) {
  return emulated ? divergence_apply_p<DF64>(m, u3, dst, t, s) : divergence_apply_p<F64>(m, u3, dst, t, s);
}

int gradient_apply(const MeshDims& m, const double* p, double* dst3, const GradHost& t, cudaStream_t s,
                   bool emulated) {
  return emulated ? gradient_apply_p<DF64>(m, p, dst3, t, s) : gradient_apply_p<F64>(m, p, dst3, t, s);
}

}  // namespace dgns
