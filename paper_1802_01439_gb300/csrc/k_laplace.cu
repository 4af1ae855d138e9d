// SIPG Laplace-type operators: Laplace l_h (pressure Poisson), viscous v_h
// and the Helmholtz operator of the viscous substep (Secs. 3.2 and 3.3 of
// arXiv:1802.01439), FP64 and FP32, with fused epilogues for the multigrid
// smoother.
//
// Factorisation.  On an affine axis-aligned cell with exact Gauss quadrature
// the 3D SIPG matrix is a sum of Kronecker products of 1D matrices:
//     L = T_x (x) M (x) M + M (x) T_y (x) M + M (x) M (x) T_z
// where T_d is the 1D SIPG operator along d (cell stiffness plus the face
// terms, coupling a cell to its two periodic neighbours through the
// neighbours' face value and face derivative) scaled by the tangential cell
// sizes, and M is the 1D reference mass matrix.  Per cell the kernel applies
//     y = M_z [ M_y T_x x + M_x T_y x ] + M_x M_y T_z x
// in 8 line sweeps (3 with neighbour terms), i.e. 8(k+1) + 12 multiply-adds
// per DoF.  The neighbour terms need, per line, the neighbour's face value
// and its face-normal derivative (k+1 products on the neighbour's line).
//
// Mapping.  One thread per line of one cell; EPB cells per block; the cell
// and three work arrays are staged in shared memory; neighbour lines are read
// directly from global memory (they are L2 resident).  Global loads and
// stores of the own cells are coalesced over the block's contiguous cells.
//
// Double-float and triple-float.  M and the cell part of T_d are
// centrosymmetric on the LGL nodes, so every line sweep runs in even-odd form
// (about half the emulated multiply-adds), and the neighbours'
// face-derivative sums are formed in native FP64 on the loaded doubles
// (load_nb_summary).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "arith.cuh"
#include "ops.h"

namespace dgns {
namespace {

// Even-odd form of a centrosymmetric N x N matrix C (C(N-1-i, N-1-j) =
// C(i, j), as the 1D mass matrix and the cell part of the 1D SIPG operator
// on the symmetric LGL nodes): with xe(j) = x(j) + x(N-1-j) (x(j) at the
// middle node of odd N) and xo(j) = x(j) - x(N-1-j), e = E xe, o = O xo give
// y(i) = e(i) + o(i), y(N-1-i) = e(i) - o(i), y(middle) = e(middle);
// E(i,j) = (C(i,j) + C(i,N-1-j)) / 2 (C(i,middle) in the middle column),
// O(i,j) = (C(i,j) - C(i,N-1-j)) / 2.  About N^2/2 instead of N^2
// multiply-adds per line, for 2N additions.
template <class V, int N>
struct EOMat {
  V E[((N + 1) / 2) * ((N + 1) / 2)];
  V O[(N / 2) * (N / 2)];
};

template <class V, int N>
struct LapTab {
  V A0[3][N * N];
  V M[N * N];
  V cr[3][N], cl[3][N], gr[3][N], gl[3][N];
  // even-odd forms (double-float sweeps): A0 and M, and the neighbour
  // coupling columns cr, cl split the same way (vE(i) = (v(i) + v(N-1-i)) / 2,
  // v(middle) at the middle, vO(i) = (v(i) - v(N-1-i)) / 2)
  EOMat<V, N> A0eo[3], Meo;
  V crE[3][(N + 1) / 2], crO[3][N / 2], clE[3][(N + 1) / 2], clO[3][N / 2];
  double grd[3][N], gld[3][N];   // gr, gl in FP64 (double-float sweeps: native face derivatives)
};

// Neighbour data of one line in the double-float sweeps: the neighbours'
// face values r(0) (+ side) and lf(N-1) (- side), split into double-float,
// and the face-derivative sums gr . r and gl . lf, formed natively in FP64 on
// the raw doubles: one split each instead of N splits and N emulated
// multiply-adds per neighbour line (the FP64 pipe is otherwise idle here).
template <class V>
struct NbLine {
  V r0, ln;
  double dr, dl;
};

template <class A, int N, int D>
__device__ __forceinline__ NbLine<typename A::V> load_nb_summary(const double* __restrict__ nbR,
                                                                 const double* __restrict__ nbL, int l,
                                                                 const LapTab<typename A::V, N>& tb) {
  int base, stride;
  line_geom<D>(l, N, N, N, base, stride);
  double dr = 0.0, dl = 0.0, r0 = 0.0, ln = 0.0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const double a = __ldg(nbR + base + j * stride), b = __ldg(nbL + base + j * stride);
    if (j == 0) r0 = a;
    if (j == N - 1) ln = b;
    dr = fma(tb.grd[D][j], a, dr);
    dl = fma(tb.gld[D][j], b, dl);
  }
  NbLine<typename A::V> s;
  s.r0 = A::split(r0);
  s.ln = A::split(ln);
  s.dr = dr;
  s.dl = dl;
  return s;
}

// Double-float sweeps use the even-odd form, and so do native FP64 sweeps
// from N = 5 on: there the N^2/2 multiply-adds and 2N additions of a line
// beat N^2 multiply-adds on the FP64 pipe (measured 6 % at N = 5 up to 23 %
// at N = 12; no gain at N = 3, 4).  In FP32 (the multigrid level operator,
// bound by the L1/shared-memory pipe) the direct form is kept.
template <class A, int N>
constexpr bool eo_sweeps() {
  return A::emulated || (sizeof(typename A::V) == 8 && N >= 5);
}
// even-odd sweeps from N = 7 on loop over their output pairs (code size)
template <int N>
constexpr bool eo_roll() {
  return N >= 7;
}

// Fold of a line into its even and odd parts.
template <class A, int N>
__device__ __forceinline__ void eo_fold(const typename A::V (&x)[N], typename A::V (&xe)[(N + 1) / 2],
                                        typename A::V (&xo)[N / 2]) {
#pragma unroll
  for (int j = 0; j < N / 2; ++j) {
    xe[j] = A::add_nr(x[j], x[N - 1 - j]);
    xo[j] = A::sub_nr(x[j], x[N - 1 - j]);
  }
  if (N % 2 == 1) xe[N / 2] = x[N / 2];
}

template <class G>
struct EpiArgs {
  const G* b;
  const G* xprev;
  const G* dinv;
  G c1, c2;
};

// Cells per block (N^2 threads each).  Natively in FP64 (F64 = true) the
// counts fill the warps: on the FP64 pipe a warp instruction costs the same
// with idle lanes, and N^2 threads leave part of the last warp idle
// (N = 6: 3 cells in 4 warps, 84 % of the lanes busy; 8 cells in 9 warps,
// all busy; N = 12: 1 cell in 5 warps, 90 %; 2 cells in 9 warps, all busy).
template <int N, bool F64 = false>
constexpr int cells_per_block() {
  if constexpr (F64) {
    if constexpr (N == 6) return 8;
    if constexpr (N == 7) return 4;
    if constexpr (N == 9) return 3;
    if constexpr (N == 10) return 2;
    if constexpr (N == 12) return 2;
  }
  return N * N >= 128 ? 1 : 128 / (N * N);
}
template <class A>
constexpr bool native64() {
  return !A::emulated && sizeof(typename A::V) == 8;
}

// Shared-memory layout of a staged cell: x-lines padded to an odd length so
// that the line-per-thread accesses of all three directions hit distinct banks
// (a cell of N = 4 floats: x-lines of stride 5, cell stride 80).
template <int N>
constexpr int padx() {
  return (N % 2 == 0) ? N + 1 : N;
}
template <int N>
constexpr int cell_stride() {
  return padx<N>() * N * N;
}
template <int N, int D>
__device__ __forceinline__ void sline(int l, int& base, int& stride) {
  constexpr int P = padx<N>();
  if (D == 0) {          // l = y + N z
    base = l * P;
    stride = 1;
  } else if (D == 1) {   // l = x + N z
    const int x = l % N, z = l / N;
    base = x + P * N * z;
    stride = P;
  } else {               // l = x + N y
    const int x = l % N, y = l / N;
    base = x + P * y;
    stride = P * N;
  }
}
// One line of T_d x in even-odd form (double-float), with the neighbour
// data nb: the coupling through the neighbours' face values
// (cr r(0) + cl lf(N-1)) goes into the even and odd sums, the face-derivative
// sums (gr . r into y(N-1), gl . lf into y(0)) are added to the outer pair.
template <class A, int N, int D>
__device__ __forceinline__ void sipg_line_eo(const typename A::V* X, typename A::V* out,
                                             const NbLine<typename A::V>& nb, int l,
                                             const LapTab<typename A::V, N>& tb) {
  typedef typename A::V V;
  typedef typename A::Acc Acc;
  constexpr int NH = (N + 1) / 2, NF = N / 2;
  int base, stride;
  sline<N, D>(l, base, stride);
  V x[N], xe[NH], xo[NF];
  load_line<V, N>(X, base, stride, x);
  eo_fold<A, N>(x, xe, xo);
  const V r0 = nb.r0, ln = nb.ln;
#pragma unroll(eo_roll<N>() ? 1 : NH)
  for (int i = 0; i < NH; ++i) {
    Acc e;
    A::acc_first(e, tb.crE[D][i], r0);
    A::acc_fma(e, tb.clE[D][i], ln);
#pragma unroll
    for (int j = 0; j < NH; ++j) A::acc_fma(e, tb.A0eo[D].E[i * NH + j], xe[j]);
    if (i < NF) {
      Acc o;
      A::acc_first(o, tb.crO[D][i], r0);
      A::acc_fma(o, tb.clO[D][i], ln);
#pragma unroll
      for (int j = 0; j < NF; ++j) A::acc_fma(o, tb.A0eo[D].O[i * NF + j], xo[j]);
      const V a = A::acc_get(e), b = A::acc_get(o);
      V lo = A::add_nr(a, b), hi = A::sub_nr(a, b);
      if (i == 0) {
        lo = A::add_nr(lo, A::split(nb.dl));
        hi = A::add_nr(hi, A::split(nb.dr));
      }
      out[base + i * stride] = lo;
      out[base + (N - 1 - i) * stride] = hi;
    } else {
      out[base + i * stride] = A::acc_get(e);
    }
  }
}

// One line of T_d x in the direct form (FP32, and native FP64 below N = 5): the cell part,
// the coupling through the neighbours' face values (cr r(0) + cl lf(N-1)) and
// the face-derivative terms (gr . r into y(N-1), gl . lf into y(0)).
template <class A, int N, int D>
__device__ __forceinline__ void sipg_line_direct(const typename A::V (&x)[N], const typename A::V (&r)[N],
                                                 const typename A::V (&lf)[N], typename A::V* out, int base,
                                                 int stride, const LapTab<typename A::V, N>& tb) {
  typedef typename A::Acc Acc;
  Acc y[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    A::acc_first(y[i], tb.cr[D][i], r[0]);
    A::acc_fma(y[i], tb.cl[D][i], lf[N - 1]);
#pragma unroll
    for (int j = 0; j < N; ++j) A::acc_fma(y[i], tb.A0[D][i * N + j], x[j]);
  }
#pragma unroll
  for (int j = 0; j < N; ++j) {
    A::acc_fma(y[N - 1], tb.gr[D][j], r[j]);
    A::acc_fma(y[0], tb.gl[D][j], lf[j]);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) out[base + i * stride] = A::acc_get(y[i]);
}

// One line of T_d x for the own cell, with the neighbour terms read here.
template <class A, int N, int D>
__device__ __forceinline__ void sipg_line(const typename A::V* X, typename A::V* out,
                                          const typename A::G* __restrict__ nbR,
                                          const typename A::G* __restrict__ nbL, int l,
                                          const LapTab<typename A::V, N>& tb) {
  typedef typename A::V V;
  if constexpr (eo_sweeps<A, N>()) {
    sipg_line_eo<A, N, D>(X, out, load_nb_summary<A, N, D>(nbR, nbL, l, tb), l, tb);
  } else {
    int base, stride, gbase, gstride;
    sline<N, D>(l, base, stride);
    line_geom<D>(l, N, N, N, gbase, gstride);
    V x[N], r[N], lf[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      r[j] = A::load(nbR + gbase + j * gstride);
      lf[j] = A::load(nbL + gbase + j * gstride);
    }
    load_line<V, N>(X, base, stride, x);
    sipg_line_direct<A, N, D>(x, r, lf, out, base, stride, tb);
  }
}

// Same (direct form), with the neighbour lines already in registers.
template <class A, int N, int D>
__device__ __forceinline__ void sipg_line_pre(const typename A::V* X, typename A::V* out,
                                              const typename A::V (&r)[N], const typename A::V (&lf)[N], int l,
                                              const LapTab<typename A::V, N>& tb) {
  typedef typename A::V V;
  int base, stride;
  sline<N, D>(l, base, stride);
  V x[N];
  load_line<V, N>(X, base, stride, x);
  sipg_line_direct<A, N, D>(x, r, lf, out, base, stride, tb);
}

template <class A, int N, int D>
__device__ __forceinline__ void load_nb_lines(const typename A::G* __restrict__ nbR,
                                              const typename A::G* __restrict__ nbL, int l,
                                              typename A::V (&r)[N], typename A::V (&lf)[N]) {
  int base, stride;
  line_geom<D>(l, N, N, N, base, stride);
  if constexpr (D == 0 && !A::emulated && sizeof(typename A::G) == 4 && N % 4 == 0) {
    // FP32 x-lines are contiguous and 16-byte aligned: vector loads
#pragma unroll
    for (int j = 0; j < N; j += 4) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(nbR + base + j));
      const float4 b = __ldg(reinterpret_cast<const float4*>(nbL + base + j));
      r[j] = a.x, r[j + 1] = a.y, r[j + 2] = a.z, r[j + 3] = a.w;
      lf[j] = b.x, lf[j + 1] = b.y, lf[j + 2] = b.z, lf[j + 3] = b.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      r[j] = A::load(nbR + base + j * stride);
      lf[j] = A::load(nbL + base + j * stride);
    }
  }
}

// Neighbour lines are prefetched into registers before the own cells are
// staged, so both global-memory latencies overlap (small N only: 6N values
// per thread).
template <int N>
constexpr bool prefetch_neighbours() {
  return N <= 6;
}

// One line of out = M_d in (+ add); in and out may coincide (the line is
// read whole before it is written).
template <class A, int N, int D, bool ADD>
__device__ __forceinline__ void mass_line(const typename A::V* in, const typename A::V* add,
                                          typename A::V* out, int l, const LapTab<typename A::V, N>& tb) {
  typedef typename A::V V;
  typedef typename A::Acc Acc;
  const V* M = tb.M;
  int base, stride;
  sline<N, D>(l, base, stride);
  V x[N];
  Acc y[N];
  load_line<V, N>(in, base, stride, x);
  if constexpr (eo_sweeps<A, N>()) {
    constexpr int NH = (N + 1) / 2, NF = N / 2;
    V xe[NH], xo[NF];
    eo_fold<A, N>(x, xe, xo);
#pragma unroll(eo_roll<N>() ? 1 : NH)
    for (int i = 0; i < NH; ++i) {
      Acc e;
      A::acc_first(e, tb.Meo.E[i * NH], xe[0]);
#pragma unroll
      for (int j = 1; j < NH; ++j) A::acc_fma(e, tb.Meo.E[i * NH + j], xe[j]);
      if (i < NF) {
        Acc o;
        A::acc_first(o, tb.Meo.O[i * NF], xo[0]);
#pragma unroll
        for (int j = 1; j < NF; ++j) A::acc_fma(o, tb.Meo.O[i * NF + j], xo[j]);
        const V a = A::acc_get(e), b = A::acc_get(o);
        V lo = A::add_nr(a, b), hi = A::sub_nr(a, b);
        if (ADD) {
          lo = A::add_nr(lo, add[base + i * stride]);
          hi = A::add_nr(hi, add[base + (N - 1 - i) * stride]);
        }
        out[base + i * stride] = lo;
        out[base + (N - 1 - i) * stride] = hi;
      } else {
        V v = A::acc_get(e);
        if (ADD) v = A::add_nr(v, add[base + i * stride]);
        out[base + i * stride] = v;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (ADD)
        A::acc_set(y[i], add[base + i * stride]);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        if (ADD || j > 0)
          A::acc_fma(y[i], M[i * N + j], x[j]);
        else
          A::acc_first(y[i], M[i * N + j], x[j]);
      }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) out[base + i * stride] = A::acc_get(y[i]);
  }
}

// Copy of one x-line of a cell between global memory (contiguous) and the
// padded shared layout: vector loads/stores where the line is aligned.
template <class A, int N>
__device__ __forceinline__ void load_xline(const typename A::G* __restrict__ g, typename A::V* sl) {
  typedef typename A::G G;
  if constexpr (!A::emulated && sizeof(G) == 4 && N % 4 == 0) {
#pragma unroll
    for (int j = 0; j < N; j += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(g + j));
      sl[j] = v.x;
      sl[j + 1] = v.y;
      sl[j + 2] = v.z;
      sl[j + 3] = v.w;
    }
  } else if constexpr (!A::emulated && sizeof(G) == 8 && N % 2 == 0) {
#pragma unroll
    for (int j = 0; j < N; j += 2) {
      const double2 v = __ldg(reinterpret_cast<const double2*>(g + j));
      sl[j] = v.x;
      sl[j + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) sl[j] = A::load(g + j);
  }
}

template <class A, int N, int EPI>
__global__ void __launch_bounds__(cells_per_block<N, native64<A>()>() * N * N)
    sipg_kernel(const typename A::G* __restrict__ src, typename A::G* __restrict__ dst,
                const __grid_constant__ LapTab<typename A::V, N> tb, const MeshDims m, const long long ncells,
                const EpiArgs<typename A::G> ea) {
  typedef typename A::V V;
  typedef typename A::G G;
  constexpr int NN = N * N, NNN = NN * N, EPB = cells_per_block<N, native64<A>()>();
  constexpr int CS = cell_stride<N>();
  V* sX = reinterpret_cast<V*>(dyn_smem());
  V* sA = sX + EPB * CS;
  V* sB = sA + EPB * CS;
  V* sC = sB + EPB * CS;
  const int slot = threadIdx.x / NN;
  const int l = threadIdx.x - slot * NN;
  const long long c0 = (long long)blockIdx.x * EPB;
  const long long rem = ncells - c0;
  const int nvalid = rem < EPB ? (int)rem : EPB;
  const G* gsrc = src + c0 * NNN;
  const bool active = slot < nvalid;
  const int off = slot * CS;
  const G* nb[6] = {src, src, src, src, src, src};   // +x, -x, +y, -y, +z, -z
  if (active) {
    const CellXYZ cx = cell_xyz((unsigned)(c0 + slot), m);
    const G* cb = src + (size_t)cx.comp * (size_t)m.E * NNN;
    nb[0] = cb + (size_t)neighbor32<0>(cx, +1, m) * NNN;
    nb[1] = cb + (size_t)neighbor32<0>(cx, -1, m) * NNN;
    nb[2] = cb + (size_t)neighbor32<1>(cx, +1, m) * NNN;
    nb[3] = cb + (size_t)neighbor32<1>(cx, -1, m) * NNN;
    nb[4] = cb + (size_t)neighbor32<2>(cx, +1, m) * NNN;
    nb[5] = cb + (size_t)neighbor32<2>(cx, -1, m) * NNN;
  }
  if constexpr (eo_sweeps<A, N>() && prefetch_neighbours<N>()) {
    // double-float: the neighbour summaries of the three directions first
    NbLine<V> n0{}, n1{}, n2{};
    if (active) {
      n0 = load_nb_summary<A, N, 0>(nb[0], nb[1], l, tb);
      n1 = load_nb_summary<A, N, 1>(nb[2], nb[3], l, tb);
      n2 = load_nb_summary<A, N, 2>(nb[4], nb[5], l, tb);
    }
    if (active) load_xline<A, N>(gsrc + slot * NNN + l * N, sX + off + l * padx<N>());
    __syncthreads();
    if (active) {
      sipg_line_eo<A, N, 0>(sX + off, sA + off, n0, l, tb);
      sipg_line_eo<A, N, 1>(sX + off, sB + off, n1, l, tb);
      sipg_line_eo<A, N, 2>(sX + off, sC + off, n2, l, tb);
    }
  } else if constexpr (prefetch_neighbours<N>()) {
    V r0[N], l0[N], r1[N], l1[N], r2[N], l2[N];
    if (active) {
      load_nb_lines<A, N, 0>(nb[0], nb[1], l, r0, l0);
      load_nb_lines<A, N, 1>(nb[2], nb[3], l, r1, l1);
      load_nb_lines<A, N, 2>(nb[4], nb[5], l, r2, l2);
    }
    if (active) load_xline<A, N>(gsrc + slot * NNN + l * N, sX + off + l * padx<N>());
    __syncthreads();
    if (active) {
      sipg_line_pre<A, N, 0>(sX + off, sA + off, r0, l0, l, tb);
      sipg_line_pre<A, N, 1>(sX + off, sB + off, r1, l1, l, tb);
      sipg_line_pre<A, N, 2>(sX + off, sC + off, r2, l2, l, tb);
    }
  } else {
    if (active) load_xline<A, N>(gsrc + slot * NNN + l * N, sX + off + l * padx<N>());
    __syncthreads();
    if (active) {
      sipg_line<A, N, 0>(sX + off, sA + off, nb[0], nb[1], l, tb);
      sipg_line<A, N, 1>(sX + off, sB + off, nb[2], nb[3], l, tb);
      sipg_line<A, N, 2>(sX + off, sC + off, nb[4], nb[5], l, tb);
    }
  }
  __syncthreads();
  if (active) {
    mass_line<A, N, 0, false>(sB + off, nullptr, sB + off, l, tb);  // M_x T_y x
    mass_line<A, N, 1, false>(sC + off, nullptr, sC + off, l, tb);  // M_y T_z x
  }
  __syncthreads();
  if (active) {
    mass_line<A, N, 1, true>(sA + off, sB + off, sA + off, l, tb);  // M_y T_x x + M_x T_y x
    mass_line<A, N, 0, false>(sC + off, nullptr, sC + off, l, tb);  // M_x M_y T_z x
  }
  __syncthreads();
  if (active) mass_line<A, N, 2, true>(sA + off, sC + off, sB + off, l, tb);
  __syncthreads();
  // each thread writes its own x-line of the result
  if (active) {
    const int li = slot * NNN + l * N;        // block-local index of the line start
    G* gdst = dst + c0 * NNN + li;
    const V* yl = sB + off + l * padx<N>();
    if constexpr (EPI == EPI_NONE) {
      if constexpr (!A::emulated && sizeof(G) == 4 && N % 4 == 0) {
#pragma unroll
        for (int j = 0; j < N; j += 4)
          *reinterpret_cast<float4*>(gdst + j) = make_float4(yl[j], yl[j + 1], yl[j + 2], yl[j + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < N; ++j) gdst[j] = A::store(yl[j]);
      }
    } else if constexpr (sizeof(G) == 4 && N % 4 == 0) {
      // FP32 with 16-byte aligned lines: the same update with vector accesses
      const V* xl = sX + off + l * padx<N>();
      const G* bl = ea.b + c0 * NNN + li;
      const G* pl = ea.xprev ? ea.xprev + c0 * NNN + li : nullptr;
#pragma unroll
      for (int j = 0; j < N; j += 4) {
        const float4 b4 = __ldg(reinterpret_cast<const float4*>(bl + j));
        const float bb[4] = {b4.x, b4.y, b4.z, b4.w};
        float out[4];
        if constexpr (EPI == EPI_RESID) {
#pragma unroll
          for (int q = 0; q < 4; ++q) out[q] = bb[q] - yl[j + q];
        } else {
          const float4 d4 = __ldg(reinterpret_cast<const float4*>(ea.dinv + l * N + j));
          const float dd[4] = {d4.x, d4.y, d4.z, d4.w};
          float pp[4] = {0.f, 0.f, 0.f, 0.f};
          if (ea.c1 != (G)0 && pl) {
            const float4 p4 = __ldg(reinterpret_cast<const float4*>(pl + j));
            pp[0] = p4.x, pp[1] = p4.y, pp[2] = p4.z, pp[3] = p4.w;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const G x = xl[j + q];
            G v = fma(ea.c2 * dd[q], bb[q] - yl[j + q], x);
            if (ea.c1 != (G)0) v = fma(ea.c1, x - pp[q], v);
            out[q] = v;
          }
        }
        *reinterpret_cast<float4*>(gdst + j) = make_float4(out[0], out[1], out[2], out[3]);
      }
    } else {
      // plain float / double policies only
      const V* xl = sX + off + l * padx<N>();
      const G* bl = ea.b + c0 * NNN + li;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const G y = yl[j];
        if constexpr (EPI == EPI_RESID) {
          gdst[j] = bl[j] - y;
        } else {
          const G x = xl[j];
          const G r = bl[j] - y;
          G v = fma(ea.c2 * ea.dinv[l * N + j], r, x);
          // x_{k+1} = x_k + c1 (x_k - x_{k-1}) + c2 D^-1 (b - A x_k); a null
          // xprev stands for a zero previous iterate
          if (ea.c1 != (G)0) v = fma(ea.c1, x - (ea.xprev ? ea.xprev[c0 * NNN + li + j] : (G)0), v);
          gdst[j] = v;
        }
      }
    }
  }
}

template <class A, int N, int EPI>
int launch_sipg(const MeshDims& m, int ncomp, const typename A::G* src, typename A::G* dst, const LapHost& h,
                const EpiHost& eh, cudaStream_t s) {
  typedef typename A::G G;
  constexpr int NN = N * N, EPB = cells_per_block<N, native64<A>()>();
  LapTab<typename A::V, N> tb;
  for (int d = 0; d < 3; ++d) {
    for (int i = 0; i < NN; ++i) tb.A0[d][i] = A::make(h.A0[d][i]);
    for (int i = 0; i < N; ++i) {
      tb.cr[d][i] = A::make(h.cr[d][i]);
      tb.cl[d][i] = A::make(h.cl[d][i]);
      tb.gr[d][i] = A::make(h.gr[d][i]);
      tb.gl[d][i] = A::make(h.gl[d][i]);
    }
  }
  for (int i = 0; i < NN; ++i) tb.M[i] = A::make(h.M[i]);
  if constexpr (eo_sweeps<A, N>()) {
    // the even-odd sweeps need centrosymmetric A0 and M (always so for the
    // operators of this library: uniform cells, LGL nodes, equal penalties on
    // both faces); anything else is refused rather than computed wrongly
    auto centro = [&](const double* C) {
      double mx = 0.0, dev = 0.0;
      for (int i = 0; i < NN; ++i) {
        mx = std::max(mx, std::fabs(C[i]));
        dev = std::max(dev, std::fabs(C[i] - C[NN - 1 - i]));
      }
      return dev <= 1e-13 * mx;
    };
    if (!centro(h.M) || !centro(h.A0[0]) || !centro(h.A0[1]) || !centro(h.A0[2])) return 7;
  }
  {
    constexpr int NH = (N + 1) / 2, NF = N / 2;
    auto split = [&](const double* C, EOMat<typename A::V, N>& eo) {
      for (int i = 0; i < NH; ++i)
        for (int j = 0; j < NH; ++j)
          eo.E[i * NH + j] = A::make(j < NF ? 0.5 * (C[i * N + j] + C[i * N + N - 1 - j]) : C[i * N + j]);
      for (int i = 0; i < NF; ++i)
        for (int j = 0; j < NF; ++j) eo.O[i * NF + j] = A::make(0.5 * (C[i * N + j] - C[i * N + N - 1 - j]));
    };
    for (int d = 0; d < 3; ++d) {
      split(h.A0[d], tb.A0eo[d]);
      for (int i = 0; i < NH; ++i) {
        tb.crE[d][i] = A::make(i < NF ? 0.5 * (h.cr[d][i] + h.cr[d][N - 1 - i]) : h.cr[d][i]);
        tb.clE[d][i] = A::make(i < NF ? 0.5 * (h.cl[d][i] + h.cl[d][N - 1 - i]) : h.cl[d][i]);
      }
      for (int i = 0; i < NF; ++i) {
        tb.crO[d][i] = A::make(0.5 * (h.cr[d][i] - h.cr[d][N - 1 - i]));
        tb.clO[d][i] = A::make(0.5 * (h.cl[d][i] - h.cl[d][N - 1 - i]));
      }
    }
    split(h.M, tb.Meo);
    for (int d = 0; d < 3; ++d)
      for (int i = 0; i < N; ++i) {
        tb.grd[d][i] = h.gr[d][i];
        tb.gld[d][i] = h.gl[d][i];
      }
  }
  if constexpr (std::is_same<A, F32>::value && N == 4) {
    // one thread per cell plane where the pointers allow 256-bit accesses
    const int r = laplace_plane_f32(m, ncomp, src, dst, h, EPI, eh, s);
    if (r >= 0) return r;
  }
  EpiArgs<G> ea{(const G*)eh.b, (const G*)eh.xprev, (const G*)eh.dinv, (G)eh.c1, (G)eh.c2};
  const long long ncells = m.E * ncomp;
  if (ncells == 0) return 0;
  const long long blocks = (ncells + EPB - 1) / EPB;
  const size_t smem = (size_t)4 * EPB * cell_stride<N>() * sizeof(typename A::V);
  static bool attr_done = false;
  if (!attr_done) {
    if (cudaFuncSetAttribute(sipg_kernel<A, N, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return 2;
    attr_done = true;
  }
  sipg_kernel<A, N, EPI><<<(unsigned)blocks, EPB * NN, smem, s>>>(src, dst, tb, m, ncells, ea);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

template <class A, int N>
int launch_sipg_epi(const MeshDims& m, int ncomp, const void* src, void* dst, const LapHost& h,
                    int epi, const EpiHost& eh, cudaStream_t s) {
  typedef typename A::G G;
  if constexpr (A::emulated) {
    if (epi != EPI_NONE) return 7;
    return launch_sipg<A, N, EPI_NONE>(m, ncomp, (const G*)src, (G*)dst, h, eh, s);
  } else {
    switch (epi) {
      case EPI_NONE: return launch_sipg<A, N, EPI_NONE>(m, ncomp, (const G*)src, (G*)dst, h, eh, s);
      case EPI_RESID: return launch_sipg<A, N, EPI_RESID>(m, ncomp, (const G*)src, (G*)dst, h, eh, s);
      case EPI_CHEB: return launch_sipg<A, N, EPI_CHEB>(m, ncomp, (const G*)src, (G*)dst, h, eh, s);
    }
  }
  return 1;
}

template <class T>
__global__ void broadcast_kernel(const T* __restrict__ table, T* __restrict__ dst, long long n,
                                 int nper) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    dst[i] = table[i % nper];
}

}  // namespace

int laplace_apply(bool fp32, const MeshDims& m, int ncomp, const void* src, void* dst,
                  const LapHost& tab, int epi, const EpiHost& ea, cudaStream_t s, int arith) {
#define DGNS_CASE(NV)                                                                           \
  case NV:                                                                                      \
    return fp32                     ? launch_sipg_epi<F32, NV>(m, ncomp, src, dst, tab, epi, ea, s)  \
           : arith == ARITH_DF64 ? launch_sipg_epi<DF64, NV>(m, ncomp, src, dst, tab, epi, ea, s) \
           : arith == ARITH_TF64 ? launch_sipg_epi<TF64, NV>(m, ncomp, src, dst, tab, epi, ea, s) \
                                 : launch_sipg_epi<F64, NV>(m, ncomp, src, dst, tab, epi, ea, s);
  switch (tab.N) {
    DGNS_CASE(2)
    DGNS_CASE(3)
    DGNS_CASE(4)
    DGNS_CASE(5)
    DGNS_CASE(6)
    DGNS_CASE(7)
    DGNS_CASE(8)
    DGNS_CASE(9)
    DGNS_CASE(10)
    DGNS_CASE(11)
    DGNS_CASE(12)
  }
#undef DGNS_CASE
  return 7;
}

int broadcast_cells(bool fp32, long long ncells, int nper, const void* table, void* dst,
                    cudaStream_t s) {
  const long long n = ncells * nper;
  if (n == 0) return 0;
  const int threads = 256;
  long long blocks = (n + threads - 1) / threads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (fp32)
    broadcast_kernel<float><<<(unsigned)blocks, threads, 0, s>>>((const float*)table, (float*)dst, n, nper);
  else
    broadcast_kernel<double><<<(unsigned)blocks, threads, 0, s>>>((const double*)table, (double*)dst, n, nper);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // namespace dgns
