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
#include <algorithm>
#include <cmath>

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
  // even-odd forms (double-float): E [(NU+1)/2][(NP+1)/2], O [(NU+1)/2][NP/2]
  // of G_d (centro-antisymmetric, A(NU-1-i, NP-1-j) = -A(i, j)) and of Mup
  // (centrosymmetric), see rect_line_eo
  V GE[3][((NU + 1) / 2) * ((NP + 1) / 2)], GO[3][((NU + 1) / 2) * (NP / 2)];
  V ME[((NU + 1) / 2) * ((NP + 1) / 2)], MO[((NU + 1) / 2) * (NP / 2)];
};

// out-line = A in-line for an NO x NI matrix with A(NO-1-i, NI-1-j) =
// S A(i, j) (S = +1 or -1), in even-odd form: with xe(j) = x(j) + x(NI-1-j)
// (x(j) at the middle of odd NI) and xo(j) = x(j) - x(NI-1-j), e = E xe and
// o = O xo give out(i) = e(i) + o(i), out(NO-1-i) = S (e(i) - o(i)),
// out(middle) = e + o, with E(i,j) = (A(i,j) + A(i,NI-1-j)) / 2 (A(i,middle)
// in the middle column) and O(i,j) = (A(i,j) - A(i,NI-1-j)) / 2.  The
// neighbour terms of a flux line (cr x_r(0) into out(NO-1), cl x_l(NI-1) into
// out(0)) are added when nbR is given.
template <class P, int NO, int NI, int D, int S>
__device__ __forceinline__ void rect_line_eo(const typename P::V* in, typename P::V* out, int l, int i0, int i1,
                                             int i2, int o0, int o1, int o2, const typename P::V* E,
                                             const typename P::V* O, const double* __restrict__ nbR = nullptr,
                                             const double* __restrict__ nbL = nullptr,
                                             typename P::V cr = typename P::V(), typename P::V cl = typename P::V()) {
  typedef typename P::V V;
  typedef typename P::Acc Acc;
  constexpr int OH = (NO + 1) / 2, OF = NO / 2, IH = (NI + 1) / 2, IF = NI / 2;
  int bi, si, bo, so;
  line_geom<D>(l, i0, i1, i2, bi, si);
  line_geom<D>(l, o0, o1, o2, bo, so);
  V x[NI], xe[IH], xo[IF];
  load_line<V, NI>(in, bi, si, x);
#pragma unroll
  for (int j = 0; j < IF; ++j) {
    xe[j] = P::add_nr(x[j], x[NI - 1 - j]);
    xo[j] = P::sub_nr(x[j], x[NI - 1 - j]);
  }
  if (NI % 2 == 1) xe[IF] = x[IF];
  V y[NO];
#pragma unroll
  for (int i = 0; i < OH; ++i) {
    Acc e, o;
    P::acc_first(e, E[i * IH], xe[0]);
#pragma unroll
    for (int j = 1; j < IH; ++j) P::acc_fma(e, E[i * IH + j], xe[j]);
    P::acc_first(o, O[i * IF], xo[0]);
#pragma unroll
    for (int j = 1; j < IF; ++j) P::acc_fma(o, O[i * IF + j], xo[j]);
    const V a = P::acc_get(e), b = P::acc_get(o);
    y[i] = P::add_nr(a, b);
    if (i < OF) y[NO - 1 - i] = S > 0 ? P::sub_nr(a, b) : P::sub_nr(b, a);
  }
  if (nbR) {
    const V vr = P::load(nbR + bi), vl = P::load(nbL + bi + (NI - 1) * si);
    Acc t, u;
    P::acc_set(t, y[NO - 1]);
    P::acc_fma(t, cr, vr);
    y[NO - 1] = P::acc_get(t);
    P::acc_set(u, y[0]);
    P::acc_fma(u, cl, vl);
    y[0] = P::acc_get(u);
  }
#pragma unroll
  for (int i = 0; i < NO; ++i) out[bo + i * so] = y[i];
}

// Shared memory per cell (doubles): divergence u (3 NU^3, later the three
// partial results of the first mass sweeps) + A, B, C (3 NP NU^2); gradient
// p + A, B, C (NP^3 + 3 NU NP^2, later the result 3 NU^3) + A2, B2, C2
// (3 NU^2 NP).
template <int NU, int NP>
constexpr int div_per_cell() {
  return 3 * NU * NU * NU + 3 * NP * NU * NU;
}
template <int NU, int NP>
constexpr int grad_per_cell() {
  return (NP * NP * NP + 3 * NU * NP * NP > 3 * NU * NU * NU ? NP * NP * NP + 3 * NU * NP * NP
                                                              : 3 * NU * NU * NU) +
         3 * NU * NU * NP;
}

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
  // 32-bit arithmetic (a 64-bit division is a long software sequence)
  const unsigned eu = (unsigned)el, nxu = (unsigned)m.nx, nyu = (unsigned)m.ny;
  p.ex = (int)(eu % nxu);
  const unsigned t = eu / nxu;
  p.ey = (int)(t % nyu);
  p.ez = (int)(t / nyu);
  return p;
}

template <class P, int NU, int NP>
__global__ void __launch_bounds__(dg_cells_per_block<NU>() * NU * NU)
    div_kernel(const double* __restrict__ u3, double* __restrict__ dst,
               const __grid_constant__ DivTab<typename P::V, NU, NP> tb, const MeshDims m) {
  typedef typename P::V V;
  constexpr int EPB = dg_cells_per_block<NU>(), NT = NU * NU;
  constexpr int NU3 = NU * NU * NU, NP3 = NP * NP * NP, W = NP * NU * NU;
  // per cell: ux, uy, uz (NU3 each; dead after the flux sweeps, then A2, B2,
  // C2: NP*NP*NU each), A, B, C (W each)
  constexpr int PER = div_per_cell<NU, NP>();
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
  V* A2 = S;   // over u (dead after the flux sweeps)
  V* B2 = A2 + NP * NP * NU;
  V* C2 = B2 + NP * NP * NU;
  static_assert(3 * NP * NP * NU <= 3 * NU3, "A2, B2, C2 fit in u's place");
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

// EO: the sweeps in even-odd form (double-float arithmetic; G_d and Mup have
// the reflection symmetries, checked on the host)
template <class P, int NU, int NP, bool EO>
__global__ void __launch_bounds__(dg_cells_per_block<NU>() * NU * NU)
    grad_kernel(const double* __restrict__ pr, double* __restrict__ dst3,
                const __grid_constant__ GradTab<typename P::V, NU, NP> tb, const MeshDims m) {
  typedef typename P::V V;
  constexpr int EPB = dg_cells_per_block<NU>(), NT = NU * NU;
  constexpr int NU3 = NU * NU * NU, NP3 = NP * NP * NP, W1 = NU * NP * NP, W2 = NU * NU * NP;
  constexpr int PER = grad_per_cell<NU, NP>();
  V* sm = reinterpret_cast<V*>(dyn_smem());
  const int slot = threadIdx.x / NT;
  const int t = threadIdx.x - slot * NT;
  const long long c0 = (long long)blockIdx.x * EPB;
  const long long rem = m.E - c0;
  const int nvalid = rem < EPB ? (int)rem : EPB;
  V* S = sm + slot * PER;
  // p, A, B, C (dead after the first mass sweeps), then O (3 NU3) in their
  // place; A2, B2, C2 behind
  constexpr int R1 = (NP3 + 3 * W1 > 3 * NU3) ? NP3 + 3 * W1 : 3 * NU3;
  V* Pp = S;
  V* A = Pp + NP3;
  V* B = A + W1;
  V* C = B + W1;
  V* A2 = S + R1;
  V* B2 = A2 + W2;
  V* C2 = B2 + W2;
  V* O = S;  // 3 * NU3
  const bool active = slot < nvalid;
  CellPos p{};
  if (active) {
    p = cell_pos(c0 + slot, m);
    for (int i = t; i < NP3; i += NT) Pp[i] = P::load(pr + p.el * NP3 + i);
  }
  __syncthreads();
  if (active) {
    for (int l = t; l < NP * NP; l += NT) {
      const double* r0 = pr + neighbor<0>(p.el, p.ex, p.ey, p.ez, +1, m) * NP3;
      const double* l0 = pr + neighbor<0>(p.el, p.ex, p.ey, p.ez, -1, m) * NP3;
      const double* r1 = pr + neighbor<1>(p.el, p.ex, p.ey, p.ez, +1, m) * NP3;
      const double* l1 = pr + neighbor<1>(p.el, p.ex, p.ey, p.ez, -1, m) * NP3;
      const double* r2 = pr + neighbor<2>(p.el, p.ex, p.ey, p.ez, +1, m) * NP3;
      const double* l2 = pr + neighbor<2>(p.el, p.ex, p.ey, p.ez, -1, m) * NP3;
      if constexpr (EO) {
        rect_line_eo<P, NU, NP, 0, -1>(Pp, A, l, NP, NP, NP, NU, NP, NP, tb.GE[0], tb.GO[0], r0, l0, tb.nbr[0],
                                       tb.nbl[0]);
        rect_line_eo<P, NU, NP, 1, -1>(Pp, B, l, NP, NP, NP, NP, NU, NP, tb.GE[1], tb.GO[1], r1, l1, tb.nbr[1],
                                       tb.nbl[1]);
        rect_line_eo<P, NU, NP, 2, -1>(Pp, C, l, NP, NP, NP, NP, NP, NU, tb.GE[2], tb.GO[2], r2, l2, tb.nbr[2],
                                       tb.nbl[2]);
      } else {
        flux_line<P, NU, NP, 0>(Pp, r0, l0, A, l, NP, NP, NP, NU, NP, NP, tb.G[0], tb.nbr[0], tb.nbl[0]);
        flux_line<P, NU, NP, 1>(Pp, r1, l1, B, l, NP, NP, NP, NP, NU, NP, tb.G[1], tb.nbr[1], tb.nbl[1]);
        flux_line<P, NU, NP, 2>(Pp, r2, l2, C, l, NP, NP, NP, NP, NP, NU, tb.G[2], tb.nbr[2], tb.nbl[2]);
      }
    }
  }
  __syncthreads();
  if (active) {
    // A (NU,NP,NP) -y-> A2 (NU,NU,NP); B (NP,NU,NP) -x-> B2 (NU,NU,NP);
    // C (NP,NP,NU) -x-> C2 (NU,NP,NU)
    for (int l = t; l < NU * NP; l += NT) {
      if constexpr (EO) {
        rect_line_eo<P, NU, NP, 1, 1>(A, A2, l, NU, NP, NP, NU, NU, NP, tb.ME, tb.MO);
        rect_line_eo<P, NU, NP, 0, 1>(B, B2, l, NP, NU, NP, NU, NU, NP, tb.ME, tb.MO);
        rect_line_eo<P, NU, NP, 0, 1>(C, C2, l, NP, NP, NU, NU, NP, NU, tb.ME, tb.MO);
      } else {
        rect_line<P, NU, NP, 1, false>(A, nullptr, A2, l, NU, NP, NP, NU, NU, NP, tb.Mup);
        rect_line<P, NU, NP, 0, false>(B, nullptr, B2, l, NP, NU, NP, NU, NU, NP, tb.Mup);
        rect_line<P, NU, NP, 0, false>(C, nullptr, C2, l, NP, NP, NU, NU, NP, NU, tb.Mup);
      }
    }
  }
  __syncthreads();
  if (active) {
    for (int l = t; l < NU * NU; l += NT) {
      if constexpr (EO) {
        rect_line_eo<P, NU, NP, 2, 1>(A2, O, l, NU, NU, NP, NU, NU, NU, tb.ME, tb.MO);
        rect_line_eo<P, NU, NP, 2, 1>(B2, O + NU3, l, NU, NU, NP, NU, NU, NU, tb.ME, tb.MO);
        rect_line_eo<P, NU, NP, 1, 1>(C2, O + 2 * NU3, l, NU, NP, NU, NU, NU, NU, tb.ME, tb.MO);
      } else {
        rect_line<P, NU, NP, 2, false>(A2, nullptr, O, l, NU, NU, NP, NU, NU, NU, tb.Mup);
        rect_line<P, NU, NP, 2, false>(B2, nullptr, O + NU3, l, NU, NU, NP, NU, NU, NU, tb.Mup);
        rect_line<P, NU, NP, 1, false>(C2, nullptr, O + 2 * NU3, l, NU, NP, NU, NU, NU, NU, tb.Mup);
      }
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
  const size_t smem = (size_t)EPB * div_per_cell<NU, NP>() * sizeof(double);
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
  // even-odd forms; used in double-float when every matrix has its
  // reflection symmetry (G_d antisymmetric, Mup symmetric) to 1e-13
  constexpr int OH = (NU + 1) / 2, IH = (NP + 1) / 2, IF = NP / 2;
  auto split = [&](const double* A, typename P::V* E, typename P::V* O) {
    for (int i = 0; i < OH; ++i) {
      for (int j = 0; j < IH; ++j)
        E[i * IH + j] = P::make(j < IF ? 0.5 * (A[i * NP + j] + A[i * NP + NP - 1 - j]) : A[i * NP + j]);
      for (int j = 0; j < IF; ++j) O[i * IF + j] = P::make(0.5 * (A[i * NP + j] - A[i * NP + NP - 1 - j]));
    }
  };
  auto symmetric = [&](const double* A, double sg) {
    double mx = 0.0, dev = 0.0;
    for (int i = 0; i < NU * NP; ++i) {
      mx = std::max(mx, std::fabs(A[i]));
      dev = std::max(dev, std::fabs(A[NU * NP - 1 - i] - sg * A[i]));   // A(NU-1-i', NP-1-j') vs A(i', j')
    }
    return dev <= 1e-13 * mx;
  };
  bool eo = P::emulated && symmetric(h.Mup, 1.0);
  for (int d = 0; d < 3; ++d) {
    split(h.G[d], tb.GE[d], tb.GO[d]);
    eo = eo && symmetric(h.G[d], -1.0);
  }
  split(h.Mup, tb.ME, tb.MO);
  constexpr int EPB = dg_cells_per_block<NU>();
  const size_t smem = (size_t)EPB * grad_per_cell<NU, NP>() * sizeof(double);
  if (cudaFuncSetAttribute(grad_kernel<P, NU, NP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(grad_kernel<P, NU, NP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
    return 2;
  if (m.E == 0) return 0;
  const long long blocks = (m.E + EPB - 1) / EPB;
  if (eo)
    grad_kernel<P, NU, NP, true><<<(unsigned)blocks, EPB * NU * NU, smem, s>>>(p, dst3, tb, m);
  else
    grad_kernel<P, NU, NP, false><<<(unsigned)blocks, EPB * NU * NU, smem, s>>>(p, dst3, tb, m);
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
