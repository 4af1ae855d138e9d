// Projection substep operator M + A_D + A_C with the divergence and
// continuity penalty terms (Sec. 3.2 and the matrix form of the projection
// step, Sec. 3.3, of arXiv:1802.01439), and the element-wise penalty
// parameters from the volume-averaged norm of the extrapolated velocity.
// FP64 or double-float arithmetic, k <= 11.
//
// Per cell (affine, Gauss rule with k+1 points, exact for both forms):
//   values  V_a = (S (x) S (x) S) u_a,   reference derivatives
//   G_x = (D (x) S (x) S) u_x, G_y = (S (x) D (x) S) u_y, G_z = (S (x) S (x) D) u_z
//   at every point: m_a = w V_a, g = tau_D w sum_a G_a / h_a  (w = quadrature
//   weight times h_x h_y h_z); test: y_b = (S^T)^3 m_b + (1/h_b) (D_b^T ...) g,
//   arranged in phases of sweeps along one direction each (proj_kernel).
// Faces normal to a couple only component a: with LGL nodes the traces are
// the nodal values of the face layers and the Gauss rule integrates the face
// mass exactly, so the own face layer gets
//   {{tau_C}} h_t1 h_t2 (Mhat (x) Mhat) (u_a(own layer) - u_a(neighbour layer)).
#include "arith.cuh"
#include "ops.h"

namespace dgns {
namespace {

// Tables of the operator kernel in the arithmetic policy's value type.
template <class V, int N>
struct ProjTabT {
  V S[N * N], D[N * N], M[N * N];
  V W3[N * N * N];       // w_qx w_qy w_qz h_x h_y h_z
  V hinv[3];             // 1 / h_d
  V area[3];             // face area of faces normal to d
};

template <int N>
constexpr int proj_cells_per_block() {
  return N * N >= 64 ? 1 : 64 / (N * N);
}

// One line sweep in an arithmetic policy, out-line (along D) = A in-line,
// A applied as A (TR = false: y_q = sum_j A[q][j] x_j) or as A^T (TR = true:
// y_j = sum_q A[q][j] x_q), plus A2 in2 when TWO (a second table that
// already carries its scale).
template <class P, int N, int D, bool TR, bool TWO>
__device__ __forceinline__ void psweep(const typename P::V* in, const typename P::V* in2, typename P::V* out,
                                       int l, const typename P::V* A, const typename P::V* A2) {
  typedef typename P::V V;
  typedef typename P::Acc Acc;
  int base, stride;
  line_geom<D>(l, N, N, N, base, stride);
  V x[N], x2[N];
  load_line<V, N>(in, base, stride, x);
  if (TWO) load_line<V, N>(in2, base, stride, x2);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    Acc a;
    P::acc_first(a, TR ? A[i] : A[i * N], x[0]);
#pragma unroll
    for (int j = 1; j < N; ++j) P::acc_fma(a, TR ? A[j * N + i] : A[i * N + j], x[j]);
    if (TWO) {
#pragma unroll
      for (int j = 0; j < N; ++j) P::acc_fma(a, TR ? A2[j * N + i] : A2[i * N + j], x2[j]);
    }
    out[base + i * stride] = P::acc_get(a);
  }
}

// Threads per cell of the operator kernel: one warp up to N = 5, then more
// as a sweep's N^2 lines grow; cells per block fill 128 threads.
template <int N>
constexpr int proj_threads() {
  return N <= 5 ? 32 : (N == 6 ? 64 : 128);
}
template <int N>
constexpr int proj_op_cells_per_block() {
  return proj_threads<N>() >= 128 ? 1 : 128 / proj_threads<N>();
}
// Work space per cell: two regions of 5 and 6 N^3 values, used in turn by the
// phases (u -> x-sweeps -> y-sweeps -> z-sweeps -> tests along x, y, z).
template <int N>
constexpr int proj_per_cell() {
  return 11 * N * N * N;
}

// Operator kernel.  Every phase is a set of line sweeps along one direction;
// its work items are (sweep, line) pairs spread over the cell's threads.
//   forward x: X = (S u_x, D u_x, S u_y, S u_z)                 R1 -> R2
//   forward y: Y = (S X0, S X1, S X2, D X2, S X3)               R2 -> R1
//   forward z: V_x V_y V_z = S (Y0, Y2, Y4), G_x G_y G_z =
//              S Y1, S Y3, D Y4                                  R1 -> R2
//   points:    m_b = W V_b, g = tau_D W sum_a G_a / h_a          in R2
//   test x:    A = (S^T m_x + (D/h_x)^T g, S^T m_y, S^T m_z, S^T g)       R2 -> R1
//   test y:    B = (S^T A0, S^T A1 + (D/h_y)^T A3, S^T A2, S^T A3)        R1 -> R2
//   test z:    O = (S^T B0, S^T B1, S^T B2 + (D/h_z)^T B3)                 R2 -> R1
// then the continuity penalty on the face layers of O and the store.
template <class P, int N>
__global__ void __launch_bounds__(proj_op_cells_per_block<N>() * proj_threads<N>())
    proj_kernel(const double* __restrict__ u3, double* __restrict__ dst3, const double* __restrict__ tau_d,
                const double* __restrict__ tau_c, const __grid_constant__ ProjTabT<typename P::V, N> tb,
                const MeshDims m) {
  typedef typename P::V V;
  typedef typename P::Acc Acc;
  constexpr int NT = proj_threads<N>(), NN = N * N, N3 = N * N * N, EPB = proj_op_cells_per_block<N>();
  V* sm = reinterpret_cast<V*>(dyn_smem());
  const int slot = threadIdx.x / NT;
  const int t = threadIdx.x - slot * NT;
  const long long c0 = (long long)blockIdx.x * EPB;
  const long long rem = m.E - c0;
  const int nvalid = rem < EPB ? (int)rem : EPB;
  const bool active = slot < nvalid;
  // tables: S, D, D/h_x, D/h_y, D/h_z, M
  V* sS = sm + EPB * proj_per_cell<N>();
  V* sD = sS + NN;
  V* sDh = sD + NN;
  V* sM = sDh + 3 * NN;
  for (int i = threadIdx.x; i < NN; i += blockDim.x) {
    sS[i] = tb.S[i];
    sD[i] = tb.D[i];
    sM[i] = tb.M[i];
#pragma unroll
    for (int d = 0; d < 3; ++d) sDh[d * NN + i] = P::mul(tb.D[i], tb.hinv[d]);
  }
  V* R1 = sm + slot * proj_per_cell<N>();   // 5 N^3
  V* R2 = R1 + 5 * N3;                      // 6 N^3
  CellXYZ cx{};
  if (active) {
    cx = cell_xyz((unsigned)(c0 + slot), m);
    for (int i = t; i < 3 * N3; i += NT) {
      const int c = i / N3, r = i - c * N3;
      R1[i] = P::load(u3 + ((size_t)c * m.E + cx.el) * N3 + r);
    }
  }
  __syncthreads();
  if (active)   // forward x
    for (int it = t; it < 4 * NN; it += NT) {
      const int s = it / NN, l = it - s * NN;
      const V* in = R1 + (s == 0 ? 0 : (s - 1) * N3);
      psweep<P, N, 0, false, false>(in, nullptr, R2 + s * N3, l, s == 1 ? sD : sS, nullptr);
    }
  group_sync<NT>();
  if (active)   // forward y
    for (int it = t; it < 5 * NN; it += NT) {
      const int s = it / NN, l = it - s * NN;
      const V* in = R2 + (s < 3 ? s : s - 1) * N3;
      psweep<P, N, 1, false, false>(in, nullptr, R1 + s * N3, l, s == 3 ? sD : sS, nullptr);
    }
  group_sync<NT>();
  if (active)   // forward z
    for (int it = t; it < 6 * NN; it += NT) {
      const int s = it / NN, l = it - s * NN;
      const int src = s == 0 ? 0 : s == 1 ? 2 : s == 2 ? 4 : s == 3 ? 1 : s == 4 ? 3 : 4;
      psweep<P, N, 2, false, false>(R1 + src * N3, nullptr, R2 + s * N3, l, s == 5 ? sD : sS, nullptr);
    }
  group_sync<NT>();
  if (active) {   // quadrature points
    const V td = P::load(tau_d + cx.el);
    for (int i = t; i < N3; i += NT) {
      const V w = tb.W3[i];
      Acc dv;
      P::acc_first(dv, tb.hinv[0], R2[3 * N3 + i]);
      P::acc_fma(dv, tb.hinv[1], R2[4 * N3 + i]);
      P::acc_fma(dv, tb.hinv[2], R2[5 * N3 + i]);
      R2[i] = P::mul(w, R2[i]);
      R2[N3 + i] = P::mul(w, R2[N3 + i]);
      R2[2 * N3 + i] = P::mul(w, R2[2 * N3 + i]);
      R2[3 * N3 + i] = P::mul(P::mul(td, w), P::acc_get(dv));
    }
  }
  group_sync<NT>();
  if (active)   // test x
    for (int it = t; it < 4 * NN; it += NT) {
      const int s = it / NN, l = it - s * NN;
      if (s == 0)
        psweep<P, N, 0, true, true>(R2, R2 + 3 * N3, R1, l, sS, sDh);
      else
        psweep<P, N, 0, true, false>(R2 + (s == 3 ? 3 : s) * N3, nullptr, R1 + s * N3, l, sS, nullptr);
    }
  group_sync<NT>();
  if (active)   // test y
    for (int it = t; it < 4 * NN; it += NT) {
      const int s = it / NN, l = it - s * NN;
      if (s == 1)
        psweep<P, N, 1, true, true>(R1 + N3, R1 + 3 * N3, R2 + N3, l, sS, sDh + NN);
      else
        psweep<P, N, 1, true, false>(R1 + s * N3, nullptr, R2 + s * N3, l, sS, nullptr);
    }
  group_sync<NT>();
  if (active)   // test z
    for (int it = t; it < 3 * NN; it += NT) {
      const int s = it / NN, l = it - s * NN;
      if (s == 2)
        psweep<P, N, 2, true, true>(R2 + 2 * N3, R2 + 3 * N3, R1 + 2 * N3, l, sS, sDh + 2 * NN);
      else
        psweep<P, N, 2, true, false>(R2 + s * N3, nullptr, R1 + s * N3, l, sS, nullptr);
    }
  group_sync<NT>();
  // continuity penalty on the six faces f = 2a + (side < 0), each sum
  // factorised: jump J = u_a(own layer) - u_a(neighbour layer) at the face
  // nodes, T = (M (x) I) J, O += {{tau_C}} |F| (I (x) M) T on the own layer;
  // J and T live in R2.  Faces normal to a change component a only, on the
  // layer of their side, so the items of the last phase write disjoint entries.
  V* sJ = R2;
  V* sT = R2 + 6 * NN;
  if (active)
    for (int it = t; it < 6 * NN; it += NT) {
      const int f = it / NN, r = it - f * NN;
      const int a = f >> 1, side = (f & 1) ? -1 : 1;
      const int sa = a == 0 ? 1 : (a == 1 ? N : NN);
      const int s1 = a == 0 ? N : 1, s2 = a == 2 ? N : NN;
      const unsigned nb = a == 0 ? neighbor32<0>(cx, side, m)
                                 : (a == 1 ? neighbor32<1>(cx, side, m) : neighbor32<2>(cx, side, m));
      const int off = (r % N) * s1 + (r / N) * s2;
      const int aown = side > 0 ? N - 1 : 0, anb = side > 0 ? 0 : N - 1;
      sJ[it] = P::sub(P::load(u3 + ((size_t)a * m.E + cx.el) * N3 + aown * sa + off),
                      P::load(u3 + ((size_t)a * m.E + nb) * N3 + anb * sa + off));
    }
  group_sync<NT>();
  if (active)   // T[j1 + N i2] = sum_i1 M[j1][i1] J[i1 + N i2]
    for (int it = t; it < 6 * NN; it += NT) {
      const int f = it / NN, r = it - f * NN;
      const int j1 = r % N, i2 = r / N;
      const V* J = sJ + f * NN + N * i2;
      Acc acc;
      P::acc_first(acc, sM[j1 * N], J[0]);
#pragma unroll
      for (int i1 = 1; i1 < N; ++i1) P::acc_fma(acc, sM[j1 * N + i1], J[i1]);
      sT[it] = P::acc_get(acc);
    }
  group_sync<NT>();
  if (active) {   // O += {{tau_C}} |F| sum_i2 M[j2][i2] T[j1 + N i2]
    const V half_tc = P::half(P::load(tau_c + cx.el));
    for (int it = t; it < 6 * NN; it += NT) {
      const int f = it / NN, r = it - f * NN;
      const int a = f >> 1, side = (f & 1) ? -1 : 1;
      const int sa = a == 0 ? 1 : (a == 1 ? N : NN);
      const int s1 = a == 0 ? N : 1, s2 = a == 2 ? N : NN;
      const unsigned nb = a == 0 ? neighbor32<0>(cx, side, m)
                                 : (a == 1 ? neighbor32<1>(cx, side, m) : neighbor32<2>(cx, side, m));
      // {{tau_C}} |F| (the halving is exact)
      const V tbar = P::mul(P::add(half_tc, P::half(P::load(tau_c + nb))), tb.area[a]);
      const int j1 = r % N, j2 = r / N;
      const V* T = sT + f * NN + j1;
      Acc acc;
      P::acc_first(acc, sM[j2 * N], T[0]);
#pragma unroll
      for (int i2 = 1; i2 < N; ++i2) P::acc_fma(acc, sM[j2 * N + i2], T[N * i2]);
      const int io = a * N3 + (side > 0 ? N - 1 : 0) * sa + j1 * s1 + j2 * s2;
      Acc o;
      P::acc_set(o, R1[io]);
      P::acc_fma(o, tbar, P::acc_get(acc));
      R1[io] = P::acc_get(o);
    }
  }
  group_sync<NT>();
  if (active)
    for (int i = t; i < 3 * N3; i += NT) {
      const int c = i / N3, r = i - c * N3;
      dst3[((size_t)c * m.E + cx.el) * N3 + r] = P::store(R1[i]);
    }
}

// The terms of the projection operator one at a time, for its
// operator-by-operator evaluation (each term its own pass over memory, the
// form the fused kernel is compared with; the mass term is the mass kernel).
//
// Divergence penalty A_D alone: reference derivatives G_a of u_a at the
// Gauss points, g = tau_D w sum_a G_a / h_a, tested with the derivative of
// the test function's own component:
//   forward x: (D u_x, S u_y, S u_z)            R1 -> R2
//   forward y: (S X0, D X1, S X2)               R2 -> R1
//   forward z: G = (S Y0, S Y1, D Y2)           R1 -> R2, then g in R2
//   test x:    ((D/h_x)^T g, S^T g)             R2 -> R1
//   test y:    (S^T A0, (D/h_y)^T A1, S^T A1)   R1 -> R2
//   test z:    (S^T B0, S^T B1, (D/h_z)^T B2)   R2 -> R1, stored
template <int N>
constexpr int projdiv_per_cell() {
  return 6 * N * N * N;
}
template <class P, int N>
__global__ void __launch_bounds__(proj_op_cells_per_block<N>() * proj_threads<N>())
    projdiv_kernel(const double* __restrict__ u3, double* __restrict__ dst3, const double* __restrict__ tau_d,
                   const __grid_constant__ ProjTabT<typename P::V, N> tb, const MeshDims m) {
  typedef typename P::V V;
  typedef typename P::Acc Acc;
  constexpr int NT = proj_threads<N>(), NN = N * N, N3 = N * N * N, EPB = proj_op_cells_per_block<N>();
  V* sm = reinterpret_cast<V*>(dyn_smem());
  const int slot = threadIdx.x / NT;
  const int t = threadIdx.x - slot * NT;
  const long long c0 = (long long)blockIdx.x * EPB;
  const long long rem = m.E - c0;
  const int nvalid = rem < EPB ? (int)rem : EPB;
  const bool active = slot < nvalid;
  V* sS = sm + EPB * projdiv_per_cell<N>();   // tables: S, D, D/h_x, D/h_y, D/h_z
  V* sD = sS + NN;
  V* sDh = sD + NN;
  for (int i = threadIdx.x; i < NN; i += blockDim.x) {
    sS[i] = tb.S[i];
    sD[i] = tb.D[i];
#pragma unroll
    for (int d = 0; d < 3; ++d) sDh[d * NN + i] = P::mul(tb.D[i], tb.hinv[d]);
  }
  V* R1 = sm + slot * projdiv_per_cell<N>();   // 3 N^3
  V* R2 = R1 + 3 * N3;                         // 3 N^3
  long long el = 0;
  if (active) {
    el = c0 + slot;
    for (int i = t; i < 3 * N3; i += NT) {
      const int c = i / N3, r = i - c * N3;
      R1[i] = P::load(u3 + ((size_t)c * m.E + el) * N3 + r);
    }
  }
  __syncthreads();
  if (active)   // forward x
    for (int it = t; it < 3 * NN; it += NT) {
      const int s = it / NN, l = it - s * NN;
      psweep<P, N, 0, false, false>(R1 + s * N3, nullptr, R2 + s * N3, l, s == 0 ? sD : sS, nullptr);
    }
  group_sync<NT>();
  if (active)   // forward y
    for (int it = t; it < 3 * NN; it += NT) {
      const int s = it / NN, l = it - s * NN;
      psweep<P, N, 1, false, false>(R2 + s * N3, nullptr, R1 + s * N3, l, s == 1 ? sD : sS, nullptr);
    }
  group_sync<NT>();
  if (active)   // forward z
    for (int it = t; it < 3 * NN; it += NT) {
      const int s = it / NN, l = it - s * NN;
      psweep<P, N, 2, false, false>(R1 + s * N3, nullptr, R2 + s * N3, l, s == 2 ? sD : sS, nullptr);
    }
  group_sync<NT>();
  if (active) {   // quadrature points: g = tau_D w sum_a G_a / h_a
    const V td = P::load(tau_d + el);
    for (int i = t; i < N3; i += NT) {
      Acc dv;
      P::acc_first(dv, tb.hinv[0], R2[i]);
      P::acc_fma(dv, tb.hinv[1], R2[N3 + i]);
      P::acc_fma(dv, tb.hinv[2], R2[2 * N3 + i]);
      R2[i] = P::mul(P::mul(td, tb.W3[i]), P::acc_get(dv));
    }
  }
  group_sync<NT>();
  if (active)   // test x
    for (int it = t; it < 2 * NN; it += NT) {
      const int s = it / NN, l = it - s * NN;
      psweep<P, N, 0, true, false>(R2, nullptr, R1 + s * N3, l, s == 0 ? sDh : sS, nullptr);
    }
  group_sync<NT>();
  if (active)   // test y
    for (int it = t; it < 3 * NN; it += NT) {
      const int s = it / NN, l = it - s * NN;
      psweep<P, N, 1, true, false>(R1 + (s == 0 ? 0 : N3), nullptr, R2 + s * N3, l, s == 1 ? sDh + NN : sS,
                                   nullptr);
    }
  group_sync<NT>();
  if (active)   // test z
    for (int it = t; it < 3 * NN; it += NT) {
      const int s = it / NN, l = it - s * NN;
      psweep<P, N, 2, true, false>(R2 + s * N3, nullptr, R1 + s * N3, l, s == 2 ? sDh + 2 * NN : sS, nullptr);
    }
  group_sync<NT>();
  if (active)
    for (int i = t; i < 3 * N3; i += NT) {
      const int c = i / N3, r = i - c * N3;
      dst3[((size_t)c * m.E + el) * N3 + r] = P::store(R1[i]);
    }
}

// Continuity penalty A_C alone: on each of the six faces of the cell the
// jump J of the normal component between the own and the neighbour's face
// layer, T = (M (x) I) J, and {{tau_C}} |F| (I (x) M) T on the own face layer
// of that component; every other entry of the cell is zero.
template <int N>
constexpr int projcont_per_cell() {
  return 3 * N * N * N + 12 * N * N;
}
template <class P, int N>
__global__ void __launch_bounds__(proj_op_cells_per_block<N>() * proj_threads<N>())
    projcont_kernel(const double* __restrict__ u3, double* __restrict__ dst3, const double* __restrict__ tau_c,
                    const __grid_constant__ ProjTabT<typename P::V, N> tb, const MeshDims m) {
  typedef typename P::V V;
  typedef typename P::Acc Acc;
  constexpr int NT = proj_threads<N>(), NN = N * N, N3 = N * N * N, EPB = proj_op_cells_per_block<N>();
  V* sm = reinterpret_cast<V*>(dyn_smem());
  const int slot = threadIdx.x / NT;
  const int t = threadIdx.x - slot * NT;
  const long long c0 = (long long)blockIdx.x * EPB;
  const long long rem = m.E - c0;
  const int nvalid = rem < EPB ? (int)rem : EPB;
  const bool active = slot < nvalid;
  V* sM = sm + EPB * projcont_per_cell<N>();
  for (int i = threadIdx.x; i < NN; i += blockDim.x) sM[i] = tb.M[i];
  V* O = sm + slot * projcont_per_cell<N>();   // 3 N^3
  V* sJ = O + 3 * N3;                          // 6 N^2
  V* sT = sJ + 6 * NN;                         // 6 N^2
  CellXYZ cx{};
  if (active) {
    cx = cell_xyz((unsigned)(c0 + slot), m);
    for (int i = t; i < 3 * N3; i += NT) O[i] = P::zero();
    for (int it = t; it < 6 * NN; it += NT) {
      const int f = it / NN, r = it - f * NN;
      const int a = f >> 1, side = (f & 1) ? -1 : 1;
      const int sa = a == 0 ? 1 : (a == 1 ? N : NN);
      const int s1 = a == 0 ? N : 1, s2 = a == 2 ? N : NN;
      const unsigned nb = a == 0 ? neighbor32<0>(cx, side, m)
                                 : (a == 1 ? neighbor32<1>(cx, side, m) : neighbor32<2>(cx, side, m));
      const int off = (r % N) * s1 + (r / N) * s2;
      const int aown = side > 0 ? N - 1 : 0, anb = side > 0 ? 0 : N - 1;
      sJ[it] = P::sub(P::load(u3 + ((size_t)a * m.E + cx.el) * N3 + aown * sa + off),
                      P::load(u3 + ((size_t)a * m.E + nb) * N3 + anb * sa + off));
    }
  }
  group_sync<NT>();
  if (active)   // T[j1 + N i2] = sum_i1 M[j1][i1] J[i1 + N i2]
    for (int it = t; it < 6 * NN; it += NT) {
      const int f = it / NN, r = it - f * NN;
      const int j1 = r % N, i2 = r / N;
      const V* J = sJ + f * NN + N * i2;
      Acc acc;
      P::acc_first(acc, sM[j1 * N], J[0]);
#pragma unroll
      for (int i1 = 1; i1 < N; ++i1) P::acc_fma(acc, sM[j1 * N + i1], J[i1]);
      sT[it] = P::acc_get(acc);
    }
  group_sync<NT>();
  if (active) {   // O = {{tau_C}} |F| sum_i2 M[j2][i2] T[j1 + N i2] on the face layers
    const V half_tc = P::half(P::load(tau_c + cx.el));
    for (int it = t; it < 6 * NN; it += NT) {
      const int f = it / NN, r = it - f * NN;
      const int a = f >> 1, side = (f & 1) ? -1 : 1;
      const int sa = a == 0 ? 1 : (a == 1 ? N : NN);
      const int s1 = a == 0 ? N : 1, s2 = a == 2 ? N : NN;
      const unsigned nb = a == 0 ? neighbor32<0>(cx, side, m)
                                 : (a == 1 ? neighbor32<1>(cx, side, m) : neighbor32<2>(cx, side, m));
      const V tbar = P::mul(P::add(half_tc, P::half(P::load(tau_c + nb))), tb.area[a]);
      const int j1 = r % N, j2 = r / N;
      const V* T = sT + f * NN + j1;
      Acc acc;
      P::acc_first(acc, sM[j2 * N], T[0]);
#pragma unroll
      for (int i2 = 1; i2 < N; ++i2) P::acc_fma(acc, sM[j2 * N + i2], T[N * i2]);
      O[a * N3 + (side > 0 ? N - 1 : 0) * sa + j1 * s1 + j2 * s2] = P::mul(tbar, P::acc_get(acc));
    }
  }
  group_sync<NT>();
  if (active)
    for (int i = t; i < 3 * N3; i += NT) {
      const int c = i / N3, r = i - c * N3;
      dst3[((size_t)c * m.E + cx.el) * N3 + r] = P::store(O[i]);
    }
}

// Volume-averaged Euclidean norm of u per cell -> penalty parameters, in the
// arithmetic policy P; the per-thread partial sums are added in a fixed order
// in FP64.  W3 carries h_x h_y h_z, divided out at the end.
template <class P, int N>
__global__ void __launch_bounds__(proj_cells_per_block<N>() * N * N)
    speed_kernel(const double* __restrict__ u3, double* __restrict__ tau_d, double* __restrict__ tau_c,
                 const __grid_constant__ ProjTabT<typename P::V, N> tb, const MeshDims m, double fd, double fc,
                 double inv_jac) {
  typedef typename P::V V;
  typedef typename P::Acc Acc;
  constexpr int NT = N * N, N3 = N * N * N, EPB = proj_cells_per_block<N>();
  constexpr int PER = 6 * N3;
  V* sm = reinterpret_cast<V*>(dyn_smem());
  const int slot = threadIdx.x / NT;
  const int l = threadIdx.x - slot * NT;
  const long long c0 = (long long)blockIdx.x * EPB;
  const long long rem = m.E - c0;
  const int nvalid = rem < EPB ? (int)rem : EPB;
  const bool active = slot < nvalid;
  V* U = sm + slot * PER;
  V* A = U + 3 * N3;
  __shared__ double red[EPB][NT];
  const long long el = c0 + slot;
  if (active)
    for (int c = 0; c < 3; ++c)
      for (int i = l; i < N3; i += NT) U[c * N3 + i] = P::load(u3 + ((size_t)c * m.E + el) * N3 + i);
  __syncthreads();
  if (active)
    for (int c = 0; c < 3; ++c) psweep<P, N, 0, false, false>(U + c * N3, nullptr, A + c * N3, l, tb.S, nullptr);
  __syncthreads();
  if (active)
    for (int c = 0; c < 3; ++c) psweep<P, N, 1, false, false>(A + c * N3, nullptr, U + c * N3, l, tb.S, nullptr);
  __syncthreads();
  if (active)
    for (int c = 0; c < 3; ++c) psweep<P, N, 2, false, false>(U + c * N3, nullptr, A + c * N3, l, tb.S, nullptr);
  __syncthreads();
  double s = 0.0;
  if (active) {
    Acc acc;
    P::acc_zero(acc);
    for (int i = l; i < N3; i += NT) {
      Acc q;
      P::acc_first(q, A[i], A[i]);
      P::acc_fma(q, A[N3 + i], A[N3 + i]);
      P::acc_fma(q, A[2 * N3 + i], A[2 * N3 + i]);
      P::acc_fma(acc, tb.W3[i], P::sqrt_(P::acc_get_norm(q)));
    }
    s = P::to_double(P::acc_get_norm(acc));
  }
  red[slot][l] = s;
  __syncthreads();
  if (active && l == 0) {
    double t = 0.0;
    for (int i = 0; i < NT; ++i) t += red[slot][i];   // fixed order
    t *= inv_jac;
    tau_d[el] = fd * t;
    tau_c[el] = fc * t;
  }
}


template <class P, int N>
ProjTabT<typename P::V, N> make_tabT(const ProjHost& h) {
  ProjTabT<typename P::V, N> tb;
  for (int i = 0; i < N * N; ++i) {
    tb.S[i] = P::make(h.S[i]);
    tb.D[i] = P::make(h.D[i]);
  }
  for (int i = 0; i < N * N; ++i) tb.M[i] = P::make(h.M[i]);
  const double jac = h.h[0] * h.h[1] * h.h[2];
  for (int qz = 0; qz < N; ++qz)
    for (int qy = 0; qy < N; ++qy)
      for (int qx = 0; qx < N; ++qx) tb.W3[qx + N * (qy + N * qz)] = P::make(h.w[qx] * h.w[qy] * h.w[qz] * jac);
  for (int d = 0; d < 3; ++d) {
    tb.hinv[d] = P::make(1.0 / h.h[d]);
    tb.area[d] = P::make(jac / h.h[d]);
  }
  return tb;
}

template <class P, int N>
int launch_proj(const MeshDims& m, const double* u3, double* dst3, const double* td, const double* tc,
                const ProjHost& h, cudaStream_t s) {
  constexpr int EPB = proj_op_cells_per_block<N>();
  const size_t smem = ((size_t)EPB * proj_per_cell<N>() + 6 * N * N) * sizeof(double);
  if (smem > 232448) return 7;
  if (cudaFuncSetAttribute(proj_kernel<P, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 2;
  if (m.E == 0) return 0;
  const long long blocks = (m.E + EPB - 1) / EPB;
  proj_kernel<P, N><<<(unsigned)blocks, EPB * proj_threads<N>(), smem, s>>>(u3, dst3, td, tc, make_tabT<P, N>(h),
                                                                             m);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

template <class P, int N>
int launch_proj_term(int terms, const MeshDims& m, const double* u3, double* dst3, const double* td,
                     const double* tc, const ProjHost& h, cudaStream_t s) {
  constexpr int EPB = proj_op_cells_per_block<N>();
  const bool div = terms == PROJ_DIV;
  const size_t smem = div ? ((size_t)EPB * projdiv_per_cell<N>() + 5 * N * N) * sizeof(typename P::V)
                          : ((size_t)EPB * projcont_per_cell<N>() + N * N) * sizeof(typename P::V);
  if (smem > 232448) return 7;
  const cudaError_t e = div ? cudaFuncSetAttribute(projdiv_kernel<P, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem)
                            : cudaFuncSetAttribute(projcont_kernel<P, N>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return 2;
  if (m.E == 0) return 0;
  const long long blocks = (m.E + EPB - 1) / EPB;
  if (div)
    projdiv_kernel<P, N><<<(unsigned)blocks, EPB * proj_threads<N>(), smem, s>>>(u3, dst3, td, make_tabT<P, N>(h), m);
  else
    projcont_kernel<P, N><<<(unsigned)blocks, EPB * proj_threads<N>(), smem, s>>>(u3, dst3, tc, make_tabT<P, N>(h),
                                                                                  m);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

template <class P, int N>
int launch_speed(const MeshDims& m, const double* u3, double* td, double* tc, const ProjHost& h, double fd,
                 double fc, cudaStream_t s) {
  constexpr int EPB = proj_cells_per_block<N>();
  const size_t smem = (size_t)EPB * 6 * N * N * N * sizeof(double);
  if (cudaFuncSetAttribute(speed_kernel<P, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 2;
  if (m.E == 0) return 0;
  const long long blocks = (m.E + EPB - 1) / EPB;
  speed_kernel<P, N><<<(unsigned)blocks, EPB * N * N, smem, s>>>(u3, td, tc, make_tabT<P, N>(h), m, fd, fc,
                                                                  1.0 / (h.h[0] * h.h[1] * h.h[2]));
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // namespace

int projection_apply(const MeshDims& m, const double* u3, double* dst3, const double* tau_d, const double* tau_c,
                     const ProjHost& h, cudaStream_t s, bool emulated, int terms) {
  if (terms != PROJ_ALL && terms != PROJ_DIV && terms != PROJ_CONT) return 1;
#define DGNS_PROJ(NV)                                                                                     \
  case NV:                                                                                                \
    if (terms != PROJ_ALL)                                                                                \
      return emulated ? launch_proj_term<DF64, NV>(terms, m, u3, dst3, tau_d, tau_c, h, s)                \
                      : launch_proj_term<F64, NV>(terms, m, u3, dst3, tau_d, tau_c, h, s);                \
    return emulated ? launch_proj<DF64, NV>(m, u3, dst3, tau_d, tau_c, h, s) : launch_proj<F64, NV>(m, u3, dst3, tau_d, tau_c, h, s);
  switch (h.N) {
    DGNS_PROJ(2)
    DGNS_PROJ(3)
    DGNS_PROJ(4)
    DGNS_PROJ(5)
    DGNS_PROJ(6)
    DGNS_PROJ(7)
    DGNS_PROJ(8)
    DGNS_PROJ(9)
    DGNS_PROJ(10)
    DGNS_PROJ(11)
    DGNS_PROJ(12)
  }
#undef DGNS_PROJ
  return 7;
}

int penalty_parameters(const MeshDims& m, const double* u3, double* tau_d, double* tau_c, const ProjHost& h,
                       double fd, double fc, cudaStream_t s, bool emulated) {
#define DGNS_SPEED(NV) \
  case NV:             \
    return emulated ? launch_speed<DF64, NV>(m, u3, tau_d, tau_c, h, fd, fc, s) : launch_speed<F64, NV>(m, u3, tau_d, tau_c, h, fd, fc, s);
  switch (h.N) {
    DGNS_SPEED(2)
    DGNS_SPEED(3)
    DGNS_SPEED(4)
    DGNS_SPEED(5)
    DGNS_SPEED(6)
    DGNS_SPEED(7)
    DGNS_SPEED(8)
    DGNS_SPEED(9)
    DGNS_SPEED(10)
    DGNS_SPEED(11)
    DGNS_SPEED(12)
  }
#undef DGNS_SPEED
  return 7;
}

}  // namespace dgns
