// Kernels of the convective term (included by the translation units that
// instantiate them for each arithmetic).
//
// Convective term c_h of Sec. 3.2 of arXiv:1802.01439 with the conservative
// flux F_c(u) = u (x) u and the local Lax-Friedrichs numerical flux,
// over-integrated with Q = floor(3(k+1)/2) Gauss points per direction, FP64;
// and its vector-Jacobian product.
//
// Cell term   y_c = - sum_d (D_d (x) S (x) S)^T [W_d u_c u_d]  at Q^3 points,
//             W_d = w_qx w_qy w_qz h_x h_y h_z / h_d, S/D: values/derivatives
//             of the LGL basis at the Gauss points.  The Q^3 data never exist
//             at once: after interpolating along x and y the kernel walks the
//             Q planes of constant z, evaluates the flux on the plane, applies
//             the transposed x and y sweeps and accumulates the z contraction
//             in registers.
// Face terms  per face, traces of both cells at the Q^2 face points (LGL:
//             the face values are the nodal values of the face layer),
//             F* = {{u (x) u}}.n + max(|u-.n|, |u+.n|) (u- - u+), tested
//             with the face-layer basis: +R for the '-' cell, -R for the '+'
//             cell.  A face kernel evaluates every face once and writes R;
//             the cell kernel adds the six R of its faces on its way out.
// Even-odd.   On the symmetric LGL nodes and Gauss points S and S w are
//             symmetric and D w antisymmetric under the reflection
//             (q, j) -> (Q-1-q, N-1-j), so a line of values folds into sums and
//             differences and every interpolation or test of a whole line
//             is two half-size contractions (interp_eo, test_eo, xtest_row).
//
// Accuracy.  For smooth fields the weak-form cell and face sums nearly cancel
// (the result is O(h) smaller than the summed terms, more so at high k), so
// every double-float intermediate is renormalised (acc_get_norm): this halves
// the error against the FP64 oracle at the bench workload (1.1e-12 -> 5.3e-13
// relative max-norm, 32^3 cells, k=3) for ~4 % more time.
#pragma once
#include "arith.cuh"
#include "ops.h"

namespace dgns {
namespace {

template <int N>
constexpr int conv_cells_per_block() {
  return N * N >= 64 ? 1 : 64 / (N * N);
}

// Native FP64 at N = 10: the cell's buffers alias by phase (ConvLayout,
// compact), so that two cells of 8 warps share an SM instead of one of 16;
// one computes while the other waits at its phase barriers.
template <bool EM, int N>
constexpr bool conv_compact() {
  return !EM && N == 10;
}
// Threads per group of the forward convective kernel: one warp up to N = 5;
// above, more threads per cell as the cell's shared memory grows (from
// N = 10 on one cell fills an SM's shared memory, so it gets 16 warps; 8 in
// the compact layout).  EM: emulated arithmetic (the default for callers
// without an arithmetic).
template <int N, bool EM = true>
constexpr int conv_threads() {
  return N <= 5 ? 32 : N == 6 ? 64 : N == 7 ? 128 : (N <= 9 || conv_compact<EM, N>()) ? 256 : 512;
}
// Cells per thread group: two for N = 2, where one cell's plane phases have
// 27, 24, 12 and 24 work items for 32 lanes.  (Two cells per warp at N = 4
// measured 6 % slower than one: it halves the warps per SM.)
template <int N>
constexpr int conv_cells_per_group() {
  return N == 2 ? 2 : 1;
}
template <int N, bool EM = true>
constexpr int conv_groups_per_block() {
  return conv_threads<N, EM>() >= 128 ? 1 : 128 / conv_threads<N, EM>();
}
template <int N, bool EM = true>
constexpr int conv_fwd_cells_per_block() {
  return conv_groups_per_block<N, EM>() * conv_cells_per_group<N>();
}

// Shared memory of one cell; a group's cells lie type by type
// ([CPG x UP][CPG x U1R][CPG x U2]), so that the plane work of the group's
// cells is contiguous.
// Region sizes are even, so that with 12-byte (triple-float) values the
// raw doubles of the face integrals in U1R stay 8-byte aligned.
constexpr int even_up(int v) { return v + (v & 1); }
template <int N, int Q, bool CMP = false, bool SPLIT = (N >= 11)>
struct ConvLayout {
  static constexpr int N3 = N * N * N;
  static constexpr int U = 3 * N3;               // nodal velocity
  static constexpr int U1 = 3 * Q * N * N;       // x-interpolated
  // later: the six face integrals, and with the two-phase x tests the folded
  // products (8 Q^2, see conv_split_xtest)
  static constexpr int R = 18 * N * N + (SPLIT ? 8 * Q * Q : 0);
  static constexpr int U1R = even_up(U1 > R ? U1 : R);
  static constexpr int U2 = even_up(3 * Q * Q * N);   // xy-interpolated
  static constexpr int P = 3 * Q * Q;            // one z-plane: u
  static constexpr int X = 8 * N * Q;            // x-tested plane (eight distinct tests)
  static constexpr int Y = 6 * N * N;            // xy-tested plane
  static constexpr int PXY = P + X + Y;
  static constexpr int UP = even_up(U > PXY ? U : PXY);   // nodal u first, plane work later
  // Compact (one cell per group): [W | U2], W = max(U1, PXY + R + P).  The
  // x-interpolated values lie at 0 in W; in the plane loop W holds the plane
  // work (PXY) and behind it the face integrals and the second plane; the
  // nodal u lies at the start of U2's region (dead before U2 is written).
  static constexpr int W = even_up(U1 > PXY + R + P ? U1 : PXY + R + P);
  static constexpr int PER = CMP ? W + U2 : UP + U1R + U2;
};
// Native FP64 from N = 6 on, the cell kernel takes the quadrature planes q
// and Q-1-q together (see conv_cells); the second plane needs room behind
// the face integrals in the x-interpolation buffer, and its y tests room in
// its place (Q^2 >= 2 N^2: the 3/2 rule, not Q = N).
template <bool EMULATED, int N, int Q>
constexpr bool conv_pair_planes() {
  return !EMULATED && N >= 6 && conv_cells_per_group<N>() == 1 &&
         (conv_compact<EMULATED, N>() || ConvLayout<N, Q>::R + ConvLayout<N, Q>::P <= ConvLayout<N, Q>::U1R) &&
         ConvLayout<N, Q>::Y <= ConvLayout<N, Q>::P;
}

// The face kernel's interpolation and test phases give each thread whole
// lines in even-odd form (`lines`) in double-float arithmetic up to N = 8;
// natively (FP64-pipe bound, where idle lanes still cost pipe time) and for
// N > 8 (too few lines per face for the warps an SM needs) one output per
// thread.
template <bool EM, int N>
constexpr bool face_lines() {
  return EM && N <= 8;
}
// Face kernel groups: one warp for FPG faces (four faces up to N = 3, two at
// N = 4, where one face has too few items per phase for 32 lanes; four at
// N = 4 measured slower: fewer warps per SM); with one output per thread
// four warps for one face from N = 7 on.
template <bool L, int N>
constexpr int face_threads() {
  return (L || N <= 6) ? 32 : 128;
}
template <int N>
constexpr int faces_per_group() {
  return N <= 3 ? 4 : (N == 4 ? 2 : 1);
}
template <bool L, int N, int Q, int VB>
constexpr int face_groups_per_block();

// Face work space; the weighted flux (3 Q^2) reuses the first sweep's
// region and the first test sweep (3 Q N) the face layers' (Q <= 2N).
template <int N, int Q>
struct FaceLayout {
  static_assert(Q <= 2 * N, "aliasing needs Q <= 2N");
  static constexpr int T0 = 6 * N * N;  // face layers of both cells; later the first test sweep
  static constexpr int G1 = 6 * Q * N;  // after the first sweep; later the weighted flux
  static constexpr int G2 = 6 * Q * Q;  // traces at the face points
  static constexpr int PER = T0 + G1 + G2;
};
// values of shared memory per group: the work space of its faces, plus the
// S and SW tables with one output per thread
template <bool L, int N, int Q>
constexpr int face_group_smem() {
  return faces_per_group<N>() * FaceLayout<N, Q>::PER + (L ? 0 : 2 * Q * N);
}
// groups per block, VB: bytes per value
template <bool L, int N, int Q, int VB>
constexpr int face_groups_per_block() {
  return face_threads<L, N>() > 32 ? 1 : face_group_smem<L, N, Q>() * VB * 4 <= 96 * 1024 ? 4 : 2;
}


// One output pair of an even-odd contraction of a folded line v (stride s,
// length LL: sums at i, differences at LL-1-i): e = sum_{i < NE} te[i ts] v(i),
// o = sum_{i < NO} to[i os] v(LL-1-i).
template <class A, int LL, int NE, int NO>
__device__ __forceinline__ void fold_dot(const typename A::V* te, int ts, const typename A::V* to, int os,
                                         const typename A::V* v, int s, typename A::V& e, typename A::V& o) {
  typename A::Acc a, b;
  A::acc_first(a, te[0], v[0]);
#pragma unroll
  for (int i = 1; i < NE; ++i) A::acc_fma(a, te[i * ts], v[i * s]);
  A::acc_first(b, to[0], v[(LL - 1) * s]);
#pragma unroll
  for (int i = 1; i < NO; ++i) A::acc_fma(b, to[i * os], v[(LL - 1 - i) * s]);
  e = A::acc_get_norm(a);
  o = A::acc_get_norm(b);
}
// the pair (x[0], x[k]) -> (x[0] + x[k], x[0] - x[k]) in place
template <class A>
__device__ __forceinline__ void fold_pair(typename A::V* x, int k) {
  const typename A::V a = x[0], b = x[k];
  x[0] = A::add(a, b);
  x[k] = A::sub(a, b);
}

__device__ __forceinline__ int node3(int N, int d, int a, int t1, int j1, int t2, int j2) {
  int c[3];
  c[d] = a;
  c[t1] = j1;
  c[t2] = j2;
  return c[0] + N * (c[1] + N * c[2]);
}

// Tables of the forward kernels.  The quadrature weights of each direction
// sit in that direction's test table and the cell-size factor of the flux
// direction d (h_x h_y h_z / h_d) in the y-test table of path d, so no
// per-point weights are multiplied and the x test of F_12 = F_21 is shared
// by the paths (1, 2) and (2, 1).
template <class V, int N, int Q>
struct ConvTabT {
  V S[Q * N];       // S[q][j] = phi_j(x_q): interpolation to the Gauss points
  V SW[Q * N];      // w_q phi_j(x_q): test with phi
  V DW[Q * N];      // w_q phi_j'(x_q): test with phi'
  V TY[3][Q * N];   // y test of flux direction d: jac_d SW (d = 0, 2) or jac_d DW (d = 1)
  V TYeo[3][Q * ((N + 1) / 2)];   // the same in even-odd form (layout of EO below)
  V area[3];        // h_x h_y h_z / h_d: face area of faces normal to d
  // x tests in even-odd form, [DW, SW][T1: (Q+1)/2 x NH | T2: Q/2 x NH],
  // NH = (N+1)/2: T1(i,x) = (T(i,x) + s T(i,N-1-x)) / 2,
  // T2(i,x) = (T(i,x) - s T(i,N-1-x)) / 2, s = -1 for DW, +1 for SW
  V EO[2][Q * ((N + 1) / 2)];
  // interpolation to the Gauss points in even-odd form: I1 [(Q+1)/2][NH],
  // I1(q,j) = (S(q,j) + S(q,N-1-j)) / 2 (S(q,j) in the middle column of odd
  // N); I2 [Q/2][N/2], I2(q,j) = (S(q,j) - S(q,N-1-j)) / 2
  V IE[((Q + 1) / 2) * ((N + 1) / 2) + (Q / 2) * (N / 2)];
};

// v(q) = sum_j S(q,j) u(j) for one line of N values (stride si) to the Q
// Gauss points (stride so), in even-odd form: S is symmetric under the
// reflection (q, j) -> (Q-1-q, N-1-j), so with ue = u(j) + u(N-1-j) (u(j) at
// the middle node of odd N) and uo = u(j) - u(N-1-j), r1 = I1 ue and
// r2 = I2 uo give v(q) = r1 + r2, v(Q-1-q) = r1 - r2 (r1 at the middle
// point of odd Q).  I1, I2: the tables of ConvTabT::IE.
template <class A, int N, int Q>
__device__ __forceinline__ void interp_eo(const typename A::V* IE, const typename A::V* u, int si,
                                          typename A::V* v, int so) {
  typedef typename A::V V;
  typedef typename A::Acc Acc;
  constexpr int NH = (N + 1) / 2, NF = N / 2, QH = (Q + 1) / 2, QF = Q / 2;
  const V* I1 = IE;
  const V* I2 = IE + QH * NH;
  V ue[NH], uo[NF];
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    const V a = u[j * si], b = u[(N - 1 - j) * si];
    ue[j] = A::add_nr(a, b);
    uo[j] = A::sub_nr(a, b);
  }
  if (N % 2 == 1) ue[NH - 1] = u[NF * si];
  // from N = 10 on the output pairs are looped over (registers: the cell
  // kernel's 512-thread groups allow 128 per thread)
#pragma unroll(N >= 10 ? 1 : QH)
  for (int q = 0; q < QH; ++q) {
    Acc r1;
    A::acc_first(r1, I1[q * NH], ue[0]);
#pragma unroll
    for (int j = 1; j < NH; ++j) A::acc_fma(r1, I1[q * NH + j], ue[j]);
    if (q < QF) {
      Acc r2;
      A::acc_first(r2, I2[q * NF], uo[0]);
#pragma unroll
      for (int j = 1; j < NF; ++j) A::acc_fma(r2, I2[q * NF + j], uo[j]);
      const V a = A::acc_get(r1), b = A::acc_get(r2);
      v[q * so] = A::add(a, b);
      v[(Q - 1 - q) * so] = A::sub(a, b);
    } else {
      v[q * so] = A::acc_get_norm(r1);
    }
  }
}

// out(x) = sum_q SW(q,x) h(q) for one line of Q values (stride si), in
// even-odd form (SW symmetric): he = h(q) + h(Q-1-q) (h(q) at the middle
// point of odd Q), ho = h(q) - h(Q-1-q), r1 = T1^T he, r2 = T2^T ho give
// out(x) = r1 + r2, out(N-1-x) = r1 - r2 (r1 at the middle node of odd N).
// T: ConvTabT::EO[1].
template <class A, int N, int Q>
__device__ __forceinline__ void test_eo(const typename A::V* T, const typename A::V* h, int si,
                                        typename A::V (&out)[N]) {
  typedef typename A::V V;
  typedef typename A::Acc Acc;
  constexpr int NH = (N + 1) / 2, NF = N / 2, QH = (Q + 1) / 2, QF = Q / 2;
  const V* T1 = T;
  const V* T2 = T + QH * NH;
  V he[QH], ho[QF];
#pragma unroll
  for (int i = 0; i < QF; ++i) {
    const V a = h[i * si], b = h[(Q - 1 - i) * si];
    he[i] = A::add_nr(a, b);
    ho[i] = A::sub_nr(a, b);
  }
  if (Q % 2 == 1) he[QH - 1] = h[QF * si];
#pragma unroll
  for (int x = 0; x < NH; ++x) {
    Acc r1;
    A::acc_first(r1, T1[x], he[0]);
#pragma unroll
    for (int i = 1; i < QH; ++i) A::acc_fma(r1, T1[i * NH + x], he[i]);
    if (x < NF) {
      Acc r2;
      A::acc_first(r2, T2[x], ho[0]);
#pragma unroll
      for (int i = 1; i < QF; ++i) A::acc_fma(r2, T2[i * NH + x], ho[i]);
      const V a = A::acc_get(r1), b = A::acc_get(r2);
      out[x] = A::add(a, b);
      out[N - 1 - x] = A::sub(a, b);
    } else {
      out[x] = A::acc_get_norm(r1);
    }
  }
}

// The eight distinct x tests of a plane: test k tests F_cd = u_c u_d with
// DW (k < 3, d = 0) or SW; the path (c, d) of the cell term reads the x test
// xtest(c, d).
__device__ __forceinline__ int test_c(int k) { return k < 3 ? k : (k == 3 || k == 6) ? 0 : (k == 7 ? 2 : 1); }
__device__ __forceinline__ int test_d(int k) { return k < 3 ? 0 : (k < 5 ? 1 : 2); }
__device__ __forceinline__ int xtest2(int c) { return c == 0 ? 6 : (c == 1 ? 5 : 7); }  // path (c, 2)

// x tests of the rows qy and Q-1-qy in one work item, stored folded along y
// (sums and differences), so that the y tests run in even-odd form too: one
// item per output pair and half the multiply-adds.  It halves the number of
// x-test items with twice the work each; measured: 3 % faster at N = 4,
// 5-13 % slower at N = 2, 5, 6 (more registers per lane), no gain where the
// unpaired items fit in one round of the lanes.
template <int N>
constexpr bool conv_pair_rows() {
  return N == 4;
}

// From N = 11 on (512 threads per cell, one cell per SM) the 8 Q x-test rows
// leave most of the SM idle, so the x tests run in two phases: the products
// u_c u_d of every row folded into sums and differences (item
// (k, qy, i < (Q+1)/2)), then the even-odd contraction (item (k, qy, output
// pair)).  Measured: +4-7 % at N = 11, 12; 5-15 % slower at N = 7..10, where
// other blocks on the SM use the issue slots of the idle warps.  Natively
// also at N = 4, with the y tests in even-odd form after a fold pass instead
// of paired rows: the paired-row items keep 24 of 32 lanes busy, the two
// phases nearly all (cell + face operator 15.86 -> 14.68 ms at 16.8M DoFs,
// the same results to the bit).  EM: emulated arithmetic.
template <int N, bool EM = true>
constexpr bool conv_split_xtest() {
  return N >= 11 || (!EM && N == 4);
}

// x test of one row of the plane (Q points u_c u_d -> N outputs) in even-odd
// form with the tables T1 (x fe, (Q+1)/2 rows) and T2 (x fo, Q/2 rows):
// out(x) = r1 + r2, out(N-1-x) = s (r1 - r2) (s = -1 for the antisymmetric
// DW), out(middle) = r1 + r2; outputs not renormalised.
template <class A, int N, int Q>
__device__ __forceinline__ void xtest_row(const typename A::V* T1, const typename A::V* T2, bool anti,
                                          const typename A::V* uc, const typename A::V* ud,
                                          typename A::V (&out)[N]) {
  typedef typename A::V V;
  typedef typename A::Acc Acc;
  constexpr int QH = (Q + 1) / 2, QF = Q / 2, NH = (N + 1) / 2, NF = N / 2;
  V fe[QH], fo[QF];
#pragma unroll
  for (int i = 0; i < QF; ++i) {
    const V f1 = A::mul_nr(uc[i], ud[i]), f2 = A::mul_nr(uc[Q - 1 - i], ud[Q - 1 - i]);
    fe[i] = A::add_nr(f1, f2);
    fo[i] = A::sub_nr(f1, f2);
  }
  if (Q % 2 == 1) fe[QH - 1] = A::mul_nr(uc[QF], ud[QF]);
#pragma unroll
  for (int x = 0; x < NH; ++x) {
    Acc r1, r2;
    A::acc_first(r1, T1[x], fe[0]);
#pragma unroll
    for (int i = 1; i < QH; ++i) A::acc_fma(r1, T1[i * NH + x], fe[i]);
    A::acc_first(r2, T2[x], fo[0]);
#pragma unroll
    for (int i = 1; i < QF; ++i) A::acc_fma(r2, T2[i * NH + x], fo[i]);
    const V a = A::acc_get(r1), b = A::acc_get(r2);
    if (x < NF) {
      out[x] = A::add_nr(a, b);
      const V d = A::sub_nr(a, b);
      out[N - 1 - x] = anti ? A::neg(d) : d;
    } else {
      out[x] = A::add_nr(a, b);
    }
  }
}

// i-th of up to two values, selected without an indexed local array
__device__ __forceinline__ unsigned pick2(int i, unsigned a, unsigned b) { return i == 0 ? a : b; }

// Forward convective cell kernel for an arithmetic policy A (F64, DF64 or TF64):
// loads and stores are double; all arithmetic is A's.  A group of NT threads
// treats CPG cells at once; every phase is split into small independent work
// items (one output or one short line of outputs) spread over the group's
// threads; the 1D tables are copied to shared memory because the items index
// them by thread.  A group past the last cell repeats the last cell and
// stores nothing.
template <class A, int N, int Q>
__device__ __forceinline__ void conv_cells(const double* __restrict__ u3, const double* __restrict__ rface,
                                           double* __restrict__ dst3, const ConvTabT<typename A::V, N, Q>& tb,
                                           const MeshDims& m, const unsigned bid) {
  typedef typename A::V V;
  typedef typename A::Acc Acc;
  constexpr bool CMP = conv_compact<A::emulated, N>();
  typedef ConvLayout<N, Q, CMP, conv_split_xtest<N, A::emulated>()> LY;
  static_assert(sizeof(V) % 4 == 0 && sizeof(V) <= 12, "two or three 4-byte words per value");
  constexpr int NT = conv_threads<N, A::emulated>(), CPG = conv_cells_per_group<N>();
  static_assert(!CMP || CPG == 1, "the compact layout holds one cell per group");
  constexpr int N3 = N * N * N, QQ = Q * Q, NN = N * N, QN = Q * N;
  static_assert(CPG <= 2, "one or two cells per group");
  V* sm = reinterpret_cast<V*>(dyn_smem());
  const int g = threadIdx.x / NT;
  const int t = threadIdx.x - g * NT;
  const long long c0 = ((long long)bid * conv_groups_per_block<N, A::emulated>() + g) * CPG;
  const long long last = m.E - 1;
  constexpr int QH = (Q + 1) / 2, QF = Q / 2, NH = (N + 1) / 2, NF = N / 2;
  constexpr bool PR = conv_pair_rows<N>() && !conv_split_xtest<N, A::emulated>();
  V* sS = sm + conv_fwd_cells_per_block<N, A::emulated>() * LY::PER;   // tables: S, SW, DW, TY[0..2] (or TYeo), EO[0..1]
  V* sSW = sS + QN;
  V* sDW = sSW + QN;
  V* sTY = sDW + QN;
  V* sEO = sTY + 3 * QN;
  // native FP64 from N = 6 on: the quadrature planes q and Q-1-q are
  // interpolated together from z-columns folded into sums and differences
  // (S(Q-1-q, N-1-z) = S(q, z) on the symmetric Gauss points and LGL nodes):
  // u(q) = E + O, u(Q-1-q) = E - O with E = ZE(q) . e, O = ZO(q) . o, about
  // half the multiply-adds of interpolating the two planes apart
  constexpr bool PAIR = conv_pair_planes<A::emulated, N, Q>();
  // with paired planes (and natively at N = 4) the x-tested rows of a plane
  // are also folded along y (sums in row q, differences in row Q-1-q) and the
  // y tests run in even-odd form (one item per output pair, as with paired rows)
  constexpr bool EOY = PAIR || (!A::emulated && N == 4);
  V* sZE = sEO + 2 * Q * NH;   // [q < QH][z < NH]
  V* sZO = sZE + QH * NH;      // [q < QH][z < NF]
  if constexpr (PAIR) {
    for (int i = threadIdx.x; i < QH * NH; i += blockDim.x) {
      const int q = i / NH, z = i - q * NH;
      sZE[i] = z < NF ? A::half(A::add(tb.S[q * N + z], tb.S[q * N + N - 1 - z])) : tb.S[q * N + z];
    }
    for (int i = threadIdx.x; i < QH * NF; i += blockDim.x) {
      const int q = i / NF, z = i - q * NF;
      sZO[i] = A::half(A::sub(tb.S[q * N + z], tb.S[q * N + N - 1 - z]));
    }
  }
  // and the z test of a plane pair in even-odd form: the y-tested values of
  // the two planes folded into sums e and differences o; with
  // Se = -(SW(q) + SW(Q-1-q)) / 2, So = -(SW(q) - SW(Q-1-q)) / 2 (De, Do from DW)
  // S1 = Se e1 + Do o3 and S2 = So o1 + De e3 give out(z) = S1 + S2 and, SW
  // symmetric and DW antisymmetric under (q, z) -> (Q-1-q, N-1-z),
  // out(N-1-z) = S1 - S2.  Tables [Se | So | De | Do][q < QH][z < NH].
  V* sQ4 = sZO + QH * NF;
  if constexpr (PAIR) {
    for (int i = threadIdx.x; i < QH * NH; i += blockDim.x) {
      const int q = i / NH, z = i - q * NH;
      const int a = q * N + z, b = (Q - 1 - q) * N + z;
      sQ4[i] = A::neg(A::half(A::add(tb.SW[a], tb.SW[b])));
      sQ4[QH * NH + i] = A::neg(A::half(A::sub(tb.SW[a], tb.SW[b])));
      sQ4[2 * QH * NH + i] = A::neg(A::half(A::add(tb.DW[a], tb.DW[b])));
      sQ4[3 * QH * NH + i] = A::neg(A::half(A::sub(tb.DW[a], tb.DW[b])));
    }
  }
  for (int i = threadIdx.x; i < QN; i += blockDim.x) {
    sS[i] = tb.S[i];
    sSW[i] = tb.SW[i];
    sDW[i] = tb.DW[i];
    if (!PR && !EOY) {
      sTY[i] = tb.TY[0][i];
      sTY[QN + i] = tb.TY[1][i];
      sTY[2 * QN + i] = tb.TY[2][i];
    }
  }
  if (PR || EOY)
    for (int i = threadIdx.x; i < 3 * Q * NH; i += blockDim.x) sTY[i] = tb.TYeo[i / (Q * NH)][i % (Q * NH)];
  for (int i = threadIdx.x; i < Q * NH; i += blockDim.x) {
    sEO[i] = tb.EO[0][i];
    sEO[Q * NH + i] = tb.EO[1][i];
  }
  V* base = sm + g * CPG * LY::PER;
  V* sUg = base + (CMP ? LY::W : 0);   // nodal u of the group's cells [j][c][N3], dead after the x interpolation
  V* sPg = base;                       // plane work: u [j][c][QQ]
  V* sXg = sPg + CPG * LY::P;          // x tests [j][k][qy][x]
  V* sYg = sXg + CPG * LY::X;          // y tests [j][c][2][y][x]
  V* sU1g = base + (CMP ? 0 : CPG * LY::UP);   // x-interpolated, cell j at j U1R
  V* sU2g = base + (CMP ? LY::W : CPG * (LY::UP + LY::U1R));   // xy-interpolated, cell j at j U2
  // the face integrals (cell j at j U1R), in the plane loop; then the x-test
  // products (from N = 11 on) and the second plane of a pair
  V* sRg = CMP ? base + LY::PXY : sU1g;

  // the group's cells (consecutive ids), clamped to the last cell
  const unsigned el0 = (unsigned)(c0 < last ? c0 : last);
  const unsigned el1 = (unsigned)(c0 + 1 < last ? c0 + 1 : last);
  for (int c = 0; c < 3; ++c)
    for (int it = t; it < CPG * N3; it += NT) {
      const int j = it / N3, i = it - j * N3;
      sUg[j * 3 * N3 + c * N3 + i] = A::load(u3 + ((size_t)c * m.E + pick2(j, el0, el1)) * N3 + i);
    }
  __syncthreads();
  // double-float: whole lines in even-odd form (interp_eo, tables read from
  // the kernel parameter), except at N = 5, 6, 7, where one output per item
  // measured faster (k = 4: 1 %, k = 5: 5 %, k = 6: 15 %); natively with
  // paired planes folded lines and one item per output pair; else one
  // output per item
  if constexpr (A::emulated && (N < 5 || N > 7)) {
    // x interpolation: item (j, c, line (y,z))
    for (int it = t; it < CPG * 3 * NN; it += NT) {
      const int j = it / (3 * NN), r = it - j * 3 * NN;
      interp_eo<A, N, Q>(tb.IE, sUg + j * 3 * N3 + r * N, 1, sU1g + j * LY::U1R + r * Q, 1);
    }
    group_sync<NT>();
    // y interpolation: item (j, c, qx, z)
    for (int it = t; it < CPG * 3 * QN; it += NT) {
      const int j = it / (3 * QN), r = it - j * 3 * QN;
      const int c = r / QN, ll = r - c * QN;
      const int qx = ll % Q, z = ll / Q;
      interp_eo<A, N, Q>(tb.IE, sU1g + j * LY::U1R + c * Q * NN + qx + QN * z, Q,
                         sU2g + j * LY::U2 + c * QQ * N + qx + QQ * z, Q);
    }
    group_sync<NT>();
  } else if constexpr (PAIR) {
    // natively with paired planes: every line folded in place into sums
    // (index i) and differences (index N-1-i), then one item per output
    // pair (q, Q-1-q): u(q) = E + O, u(Q-1-q) = E - O (tables ZE, ZO)
    // x interpolation
    for (int it = t; it < 3 * NN * NF; it += NT) {
      const int r = it / NF, i = it - r * NF;
      V* x = sUg + r * N;
      const V a = x[i], b = x[N - 1 - i];
      x[i] = A::add(a, b);
      x[N - 1 - i] = A::sub(a, b);
    }
    group_sync<NT>();
    for (int it = t; it < 3 * NN * QH; it += NT) {   // item (c, line (y,z), q < QH)
      const int r = it / QH, q = it - r * QH;
      const V* x = sUg + r * N;
      Acc e, o;
      A::acc_first(e, sZE[q * NH], x[0]);
#pragma unroll
      for (int i = 1; i < NH; ++i) A::acc_fma(e, sZE[q * NH + i], x[i]);
      A::acc_first(o, sZO[q * NF], x[N - 1]);
#pragma unroll
      for (int i = 1; i < NF; ++i) A::acc_fma(o, sZO[q * NF + i], x[N - 1 - i]);
      const V ev = A::acc_get_norm(e), od = A::acc_get_norm(o);
      V* y = sU1g + r * Q;
      y[q] = A::add(ev, od);
      if (q != Q - 1 - q) y[Q - 1 - q] = A::sub(ev, od);
    }
    group_sync<NT>();
    // y interpolation: lines (c, z, qx) of stride Q
    for (int it = t; it < 3 * QN * NF; it += NT) {
      const int r = it / NF, i = it - r * NF;
      const int c = r / QN, ll = r - c * QN;
      const int qx = ll % Q, z = ll / Q;
      V* x = sU1g + c * Q * NN + qx + QN * z;
      const V a = x[Q * i], b = x[Q * (N - 1 - i)];
      x[Q * i] = A::add(a, b);
      x[Q * (N - 1 - i)] = A::sub(a, b);
    }
    group_sync<NT>();
    for (int it = t; it < 3 * QN * QH; it += NT) {   // item (c, qx, z, qy < QH)
      const int qy = it % QH, r = it / QH;
      const int c = r / QN, ll = r - c * QN;
      const int qx = ll % Q, z = ll / Q;
      const V* x = sU1g + c * Q * NN + qx + QN * z;
      Acc e, o;
      A::acc_first(e, sZE[qy * NH], x[0]);
#pragma unroll
      for (int i = 1; i < NH; ++i) A::acc_fma(e, sZE[qy * NH + i], x[Q * i]);
      A::acc_first(o, sZO[qy * NF], x[Q * (N - 1)]);
#pragma unroll
      for (int i = 1; i < NF; ++i) A::acc_fma(o, sZO[qy * NF + i], x[Q * (N - 1 - i)]);
      const V ev = A::acc_get_norm(e), od = A::acc_get_norm(o);
      V* y = sU2g + c * QQ * N + qx + QQ * z;
      y[Q * qy] = A::add(ev, od);
      if (qy != Q - 1 - qy) y[Q * (Q - 1 - qy)] = A::sub(ev, od);
    }
    group_sync<NT>();
  } else {
    // x interpolation: item (j, c, line (y,z), q)
    for (int it = t; it < CPG * 3 * NN * Q; it += NT) {
      const int j = it / (3 * NN * Q), l = it - j * 3 * NN * Q;
      const int q = l % Q, r = l / Q;
      const V* x = sUg + j * 3 * N3 + r * N;
      Acc a;
      A::acc_first(a, sS[q * N], x[0]);
#pragma unroll
      for (int i = 1; i < N; ++i) A::acc_fma(a, sS[q * N + i], x[i]);
      sU1g[j * LY::U1R + l] = A::acc_get_norm(a);
    }
    group_sync<NT>();
    // y interpolation: item (j, c, qx, z, qy)
    for (int it = t; it < CPG * 3 * Q * N * Q; it += NT) {
      const int j = it / (3 * QN * Q), l = it - j * 3 * QN * Q;
      const int qy = l % Q, r = l / Q;
      const int c = r / QN, ll = r - c * QN;
      const int qx = ll % Q, z = ll / Q;
      const V* x = sU1g + j * LY::U1R + c * Q * NN + qx + QN * z;
      Acc a;
      A::acc_first(a, sS[qy * N], x[0]);
#pragma unroll
      for (int i = 1; i < N; ++i) A::acc_fma(a, sS[qy * N + i], x[Q * i]);
      sU2g[j * LY::U2 + c * QQ * N + qx + Q * qy + QQ * z] = A::acc_get_norm(a);
    }
    group_sync<NT>();
  }

  // The face integrals of the six faces of each cell (raw doubles), fetched
  // asynchronously into the dead x-interpolation buffer while the plane loop
  // runs: block f = 2 d (+R of face (e, d)) and 2 d + 1 (-R of face (e-1_d, d)).
  {
    const CellXYZ x0 = cell_xyz(el0, m), x1 = cell_xyz(el1, m);
    const unsigned n00 = neighbor32<0>(x0, -1, m), n01 = neighbor32<1>(x0, -1, m), n02 = neighbor32<2>(x0, -1, m);
    const unsigned n10 = neighbor32<0>(x1, -1, m), n11 = neighbor32<1>(x1, -1, m), n12 = neighbor32<2>(x1, -1, m);
    for (int it = t; it < CPG * 18 * NN; it += NT) {
      const int j = it / (18 * NN), l = it - j * 18 * NN;
      const int f = l / (3 * NN), i = l - f * 3 * NN;
      const int dd = f >> 1;
      const unsigned cell = (f & 1) == 0 ? pick2(j, el0, el1)
                            : dd == 0     ? pick2(j, n00, n10)
                            : dd == 1     ? pick2(j, n01, n11)
                                          : pick2(j, n02, n12);
      cp_async8(reinterpret_cast<double*>(sRg + j * LY::U1R) + l, rface + ((size_t)dd * m.E + cell) * 3 * NN + i);
    }
  }
  cp_async_commit();

  // The plane loop: every lane keeps the same work items in all planes, so
  // their offsets are computed once; the lane's outputs (items of P4) stay
  // in registers until the end.
  constexpr int I1 = CPG * 3 * QQ, I2 = CPG * 8 * (PR ? QH : Q), I3 = CPG * 3 * N * (PR || EOY ? NH : N),
                I4 = CPG * 3 * N3;
  constexpr int R1 = (I1 + NT - 1) / NT, R2 = (I2 + NT - 1) / NT, R3 = (I3 + NT - 1) / NT,
                R4 = (I4 + NT - 1) / NT;
  int o1[R1];                                  // P1: offset of the z column in sU2g
  int o2t[R2], o2c[R2], o2d[R2], o2x[R2];      // P2: table, u_c, u_d offsets of the row, output offset
  int o2b[R2];                                 // P2 (paired rows): offset of row Q-1-qy from row qy (0: middle)
  int o3a[R3], o3y[R3], o3o[R3];               // P3: X(c,0) + x in sXg; y (pair) + 16 (xtest2(c) - c); Y1 + x in sYg
  int o4y[R4], o4z[R4];                        // P4: offset into sYg, z
#pragma unroll
  for (int r = 0; r < R1; ++r) {
    const int it = t + NT * r;
    const int j = it / (3 * QQ), l = it - j * 3 * QQ;
    o1[r] = j * LY::U2 + (l / QQ) * QQ * N + (l % QQ);
  }
#pragma unroll
  for (int r = 0; r < R2; ++r) {
    // item (j, k, row): with paired rows the row p < QH stands for p and Q-1-p
    constexpr int RW = PR ? QH : Q;
    const int it = t + NT * r;
    const int j = it / (8 * RW), l = it - j * 8 * RW;
    const int k = l / RW, p = l - k * RW;
    o2t[r] = k < 3 ? 0 : Q * NH;    // even-odd DW or SW tables, relative to sEO
    o2c[r] = j * LY::P + test_c(k) * QQ + Q * p;
    o2d[r] = j * LY::P + test_d(k) * QQ + Q * p;
    o2b[r] = Q * (Q - 1 - 2 * p);
    o2x[r] = ((j * 8 + k) * Q + p) * N;
  }
#pragma unroll
  for (int r = 0; r < R3; ++r) {
    // item (j, c, y, x), with paired rows y < NH stands for y and N-1-y
    constexpr int YW = PR || EOY ? NH : N;
    const int it = t + NT * r;
    const int j = it / (3 * N * YW), l = it - j * 3 * N * YW;
    const int c = l / (N * YW), rr = l - c * N * YW;
    const int x = rr % N, y = rr / N;
    o3a[r] = (j * 8 + c) * QN + x;
    o3y[r] = y + 16 * (xtest2(c) - c);
    o3o[r] = (j * 3 + c) * 2 * NN + x;
  }
#pragma unroll
  for (int r = 0; r < R4; ++r) {
    const int it = t + NT * r;
    const int j = it / (3 * N3), l = it - j * 3 * N3;
    const int c = l / N3, rr = l - c * N3;
    o4y[r] = (j * 3 + c) * 2 * NN + rr % NN;
    o4z[r] = rr / NN;
  }
  Acc out[PAIR ? 1 : R4];
  // with paired planes the z test runs after both planes' y tests, one item
  // per (c, y, x) line, its N outputs as the pairs S1 +- S2 in registers
  constexpr int IL = 3 * NN, RL = (IL + NT - 1) / NT;
  Acc s1[PAIR ? RL : 1][NH], s2[PAIR ? RL : 1][NH];
  // the point loop of the unpaired y tests is unrolled, except for N = 5 and
  // 6 (k = 4, 5), where the rolled loop measured 5 % faster
  constexpr int UQ = (N == 5 || N == 6) ? 1 : Q;

  // the second plane of a pair sits behind the face integrals (and the
  // folded x-test products) in the dead x-interpolation buffer; its y tests
  // later replace it there
  V* sPb = sRg + LY::R;
  static_assert(!PAIR || LY::Y <= LY::P, "room for the second plane's y tests");
  if constexpr (PAIR) {
    // fold every z-column: e_z = u_z + u_{N-1-z} at z, o_z = u_z - u_{N-1-z} at N-1-z
    for (int it = t; it < 3 * QQ * NF; it += NT) {
      const int z = it % NF, col = it / NF;
      V* col_ = sU2g + (col / QQ) * QQ * N + (col % QQ);
      const V lo = col_[QQ * z], hi = col_[QQ * (N - 1 - z)];
      col_[QQ * z] = A::add(lo, hi);
      col_[QQ * (N - 1 - z)] = A::sub(lo, hi);
    }
    group_sync<NT>();
  }

#pragma unroll 1
  for (int pq = 0; pq < (PAIR ? QH : Q); ++pq) {
    const bool two = PAIR && pq != Q - 1 - pq;
    // P1: u on the plane (with PAIR: on the planes pq and Q-1-pq); item (j, c, point)
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      if (I1 % NT != 0 && t + NT * r >= I1) break;
      const V* src = sU2g + o1[r];
      if constexpr (PAIR) {
        Acc e, o;
        A::acc_first(e, sZE[pq * NH], src[0]);
#pragma unroll
        for (int z = 1; z < NH; ++z) A::acc_fma(e, sZE[pq * NH + z], src[QQ * z]);
        A::acc_first(o, sZO[pq * NF], src[QQ * (N - 1)]);
#pragma unroll
        for (int z = 1; z < NF; ++z) A::acc_fma(o, sZO[pq * NF + z], src[QQ * (N - 1 - z)]);
        const V ev = A::acc_get_norm(e), od = A::acc_get_norm(o);
        sPg[t + NT * r] = A::add(ev, od);
        if (two) sPb[t + NT * r] = A::sub(ev, od);
      } else {
        Acc a;
        A::acc_first(a, sS[pq * N], src[0]);
#pragma unroll
        for (int z = 1; z < N; ++z) A::acc_fma(a, sS[pq * N + z], src[QQ * z]);
        sPg[t + NT * r] = A::acc_get_norm(a);
      }
    }
    group_sync<NT>();
#pragma unroll 1
    for (int h = 0; h < (two ? 2 : 1); ++h) {
      const int qz = h == 0 ? pq : Q - 1 - pq;
      const V* sPc = h == 0 ? sPg : sPb;
      V* sYc = h == 0 ? sYg : sPb;   // the second plane's y tests replace its dead u
      // P2: F_cd = u_c u_d on x-lines, x test k in even-odd form (xtest_row:
      // SW is symmetric and DW antisymmetric under the reflection
      // (q, x) -> (Q-1-q, N-1-x) of the Gauss points and nodes).  With paired
      // rows an item tests the rows p and Q-1-p and stores their sum in row p
      // and their difference in row (Q+1)/2 + p of the test's block (the
      // middle row of odd Q alone, in row p); else one row per item.
      if constexpr (conv_split_xtest<N, A::emulated>()) {
        static_assert(CPG == 1, "one cell per group");
        V* sFE = sRg + 18 * NN;   // behind the face integrals
        V* sFO = sFE + 8 * Q * QH;
        for (int it = t; it < 8 * Q * QH; it += NT) {   // item (k, qy, i)
          const int k = it / (Q * QH), l = it - k * Q * QH;
          const int qy = l / QH, i = l - qy * QH;
          const V* uc = sPc + test_c(k) * QQ + Q * qy;
          const V* ud = sPc + test_d(k) * QQ + Q * qy;
          if (i < QF) {
            const V f1 = A::mul_nr(uc[i], ud[i]), f2 = A::mul_nr(uc[Q - 1 - i], ud[Q - 1 - i]);
            sFE[it] = A::add_nr(f1, f2);
            sFO[(k * Q + qy) * QF + i] = A::sub_nr(f1, f2);
          } else {
            sFE[it] = A::mul_nr(uc[QF], ud[QF]);   // middle point of odd Q
          }
        }
        group_sync<NT>();
        for (int it = t; it < 8 * Q * NH; it += NT) {   // item (k, qy, x)
          const int k = it / (Q * NH), l = it - k * Q * NH;
          const int qy = l / NH, x = l - qy * NH;
          const V* T1 = sEO + (k < 3 ? 0 : Q * NH);
          const V* T2 = T1 + QH * NH;
          const V* fe = sFE + (k * Q + qy) * QH;
          const V* fo = sFO + (k * Q + qy) * QF;
          Acc r1, r2;
          A::acc_first(r1, T1[x], fe[0]);
  #pragma unroll
          for (int i = 1; i < QH; ++i) A::acc_fma(r1, T1[i * NH + x], fe[i]);
          A::acc_first(r2, T2[x], fo[0]);
  #pragma unroll
          for (int i = 1; i < QF; ++i) A::acc_fma(r2, T2[i * NH + x], fo[i]);
          const V a = A::acc_get(r1), b = A::acc_get(r2);
          V* xo = sXg + (k * Q + qy) * N;
          xo[x] = A::add(a, b);
          if (x < NF) {
            const V d = A::sub(a, b);
            xo[N - 1 - x] = k < 3 ? A::neg(d) : d;
          }
        }
      } else {
  #pragma unroll
        for (int r = 0; r < R2; ++r) {
          const int it = t + NT * r;
          if (I2 % NT != 0 && it >= I2) break;
          const V* T1 = sEO + o2t[r];
          const V* T2 = T1 + QH * NH;
          const bool anti = o2t[r] == 0;
          V xa[N];
          xtest_row<A, N, Q>(T1, T2, anti, sPc + o2c[r], sPc + o2d[r], xa);
          V* xo = sXg + o2x[r];
          if (PR && (Q % 2 == 0 || o2b[r] != 0)) {
            V xb[N];
            xtest_row<A, N, Q>(T1, T2, anti, sPc + o2c[r] + o2b[r], sPc + o2d[r] + o2b[r], xb);
  #pragma unroll
            for (int x = 0; x < N; ++x) {
              xo[x] = A::add(xa[x], xb[x]);
              xo[QH * N + x] = A::sub(xa[x], xb[x]);
            }
          } else {
  #pragma unroll
            for (int x = 0; x < N; ++x) {
              Acc n;
              A::acc_set(n, xa[x]);
              xo[x] = A::acc_get_norm(n);
            }
          }
        }
      }
      group_sync<NT>();
      if constexpr (EOY) {
        // fold every x-tested column along y: row q <- X(q) + X(Q-1-q),
        // row Q-1-q <- X(q) - X(Q-1-q) (the middle row of odd Q unchanged)
        for (int it = t; it < 8 * QF * N; it += NT) {
          const int k = it / (QF * N), l = it - k * QF * N;
          const int p = l / N, x = l - p * N;
          V* ra = sXg + (k * Q + p) * N + x;
          V* rb = sXg + (k * Q + Q - 1 - p) * N + x;
          const V va = *ra, vb = *rb;
          *ra = A::add(va, vb);
          *rb = A::sub(va, vb);
        }
        group_sync<NT>();
      }
      if constexpr (PR || EOY) {
        // P3 (even-odd): Y1 = TY0^T X(c,0) + TY1^T X(c,1), Y3 = TY2^T X(c,2) from the
        // y-folded x tests (rows q < (Q+1)/2: sums Xe; differences Xo in rows
        // (Q+1)/2 + q with paired rows, else Q-1-q); TY0, TY2 symmetric, TY1 antisymmetric: R1 = TY0_1 X0e + TY1_2 X1o,
        // R2 = TY0_2 X0o + TY1_1 X1e give Y1(y) = R1 + R2, Y1(N-1-y) = R1 - R2;
        // C1 = TY2_1 X2e, C2 = TY2_2 X2o give Y3 the same way; item (j, c, y < NH, x)
  #pragma unroll
        for (int r = 0; r < R3; ++r) {
          if (I3 % NT != 0 && t + NT * r >= I3) break;
          const V* X0 = sXg + o3a[r];
          const V* X1 = X0 + 3 * QN;                  // X(c,1) = test 3 + c
          const V* X2 = X0 + (o3y[r] >> 4) * QN;      // X(c,2)
          const int y = o3y[r] & 15;
          const V* J0 = sTY;
          const V* J1 = sTY + Q * NH;
          const V* J2 = sTY + 2 * Q * NH;
          Acc R1, R2, C1, C2;
          A::acc_first(R1, J0[y], X0[0]);
          A::acc_first(R2, J1[y], X1[0]);
          A::acc_first(C1, J2[y], X2[0]);
          A::acc_first(C2, J2[QH * NH + y], X2[(PR ? QH : Q - 1) * N]);
  #pragma unroll
          for (int q = 1; q < QH; ++q) {
            A::acc_fma(R1, J0[q * NH + y], X0[q * N]);
            A::acc_fma(R2, J1[q * NH + y], X1[q * N]);
            A::acc_fma(C1, J2[q * NH + y], X2[q * N]);
          }
  #pragma unroll
          for (int q = 0; q < QF; ++q) {
            const int o = (PR ? QH + q : Q - 1 - q) * N;
            A::acc_fma(R1, J1[(QH + q) * NH + y], X1[o]);
            A::acc_fma(R2, J0[(QH + q) * NH + y], X0[o]);
            if (q > 0) A::acc_fma(C2, J2[(QH + q) * NH + y], X2[o]);
          }
          const V a = A::acc_get(R1), b = A::acc_get(R2), c = A::acc_get(C1), d = A::acc_get(C2);
          V* Y1 = sYc + o3o[r];
          Y1[N * y] = A::add(a, b);
          Y1[NN + N * y] = A::add(c, d);
          if (N % 2 == 0 || y < NF) {
            Y1[N * (N - 1 - y)] = A::sub(a, b);
            Y1[NN + N * (N - 1 - y)] = A::sub(c, d);
          }
        }
      } else {
        // P3: Y1 = TY0^T X(c,0) + TY1^T X(c,1), Y3 = TY2^T X(c,2); item (j, c, y, x)
  #pragma unroll
        for (int r = 0; r < R3; ++r) {
          if (I3 % NT != 0 && t + NT * r >= I3) break;
          const V* X0 = sXg + o3a[r];
          const V* X1 = X0 + 3 * QN;                  // X(c,1) = test 3 + c
          const V* X2 = X0 + (o3y[r] >> 4) * QN;      // X(c,2)
          const int y = o3y[r] & 15;
          Acc y1, y3;
          A::acc_first(y1, sTY[QN + y], X1[0]);
          A::acc_fma(y1, sTY[y], X0[0]);
          A::acc_first(y3, sTY[2 * QN + y], X2[0]);
  #pragma unroll UQ
          for (int qy = 1; qy < Q; ++qy) {
            const int o = N * qy;
            A::acc_fma(y1, sTY[QN + qy * N + y], X1[o]);
            A::acc_fma(y1, sTY[qy * N + y], X0[o]);
            A::acc_fma(y3, sTY[2 * QN + qy * N + y], X2[o]);
          }
          V* Y1 = sYc + o3o[r];
          Y1[N * y] = A::acc_get_norm(y1);
          Y1[NN + N * y] = A::acc_get_norm(y3);
        }
      }
      group_sync<NT>();
      if constexpr (!PAIR) {
        // P4: out -= SW_z(qz) Y1 + DW_z(qz) Y3; item (j, c, x, y, z), in registers
  #pragma unroll
        for (int r = 0; r < R4; ++r) {
          if (I4 % NT != 0 && t + NT * r >= I4) break;
          const V* Y = sYg + o4y[r];
          const int z = o4z[r];
          if (qz == 0)
            A::acc_first(out[r], A::neg(sDW[z]), Y[NN]);
          else
            A::acc_fma(out[r], A::neg(sDW[qz * N + z]), Y[NN]);
          A::acc_fma(out[r], A::neg(sSW[qz * N + z]), Y[0]);
        }
        group_sync<NT>();
      }
    }
    if constexpr (PAIR) {
      // P4 of the pair (pq, Q-1-pq) in even-odd form (tables sQ4); the
      // middle plane of odd Q alone: e = o = its y tests
      const V* Se = sQ4 + pq * NH;
      const V* So = Se + QH * NH;
      const V* De = So + QH * NH;
      const V* Do = De + QH * NH;
  #pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int l = t + NT * r;
        if (IL % NT != 0 && l >= IL) break;
        const int c = l / NN, yx = l - c * NN;
        const V* Ya = sYg + c * 2 * NN + yx;
        V e1 = Ya[0], o1 = Ya[0], e3 = Ya[NN], o3 = Ya[NN];
        if (two) {
          const V* Yb = sPb + c * 2 * NN + yx;
          e1 = A::add(Ya[0], Yb[0]);
          o1 = A::sub(Ya[0], Yb[0]);
          e3 = A::add(Ya[NN], Yb[NN]);
          o3 = A::sub(Ya[NN], Yb[NN]);
        }
  #pragma unroll
        for (int z = 0; z < NH; ++z) {
          if (pq == 0) {
            A::acc_first(s1[r][z], Se[z], e1);
            A::acc_first(s2[r][z], So[z], o1);
          } else {
            A::acc_fma(s1[r][z], Se[z], e1);
            A::acc_fma(s2[r][z], So[z], o1);
          }
          A::acc_fma(s1[r][z], Do[z], o3);
          A::acc_fma(s2[r][z], De[z], e3);
        }
      }
      group_sync<NT>();
    }
  }
  cp_async_wait_all();
  group_sync<NT>();
  // face integrals from the face kernel: +R on the layer N-1 (this cell is
  // the '-' side of its face), -R of the '-' neighbour on the layer 0
  if constexpr (PAIR) {
    if (c0 > last) return;
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int l = t + NT * r;
      if (IL % NT != 0 && l >= IL) break;
      const int c = l / NN, yx = l - c * NN;
      const int x = yx % N, y = yx / N;
      const double* rc = reinterpret_cast<const double*>(sRg) + c * NN;
      double* d = dst3 + ((size_t)c * m.E + el0) * N3 + yx;
#pragma unroll
      for (int z = 0; z < N; ++z) {
        const int zz = z < NH ? z : N - 1 - z;
        const V a = A::acc_get_norm(s1[r][zz]), b = A::acc_get_norm(s2[r][zz]);
        double v = A::to_double(z < NH ? A::add(a, b) : A::sub(a, b));
        if (x == N - 1) v += rc[0 * 3 * NN + y + N * z];
        if (x == 0) v -= rc[1 * 3 * NN + y + N * z];
        if (y == N - 1) v += rc[2 * 3 * NN + x + N * z];
        if (y == 0) v -= rc[3 * 3 * NN + x + N * z];
        if (z == N - 1) v += rc[4 * 3 * NN + x + N * y];
        if (z == 0) v -= rc[5 * 3 * NN + x + N * y];
        d[NN * z] = v;
      }
    }
  } else {
#pragma unroll
    for (int r = 0; r < R4; ++r) {
      const int it = t + NT * r;
      if (I4 % NT != 0 && it >= I4) break;
      const int j = it / (3 * N3), l = it - j * 3 * N3;
      if (c0 + j > last) break;
      const int c = l / N3, rr = l - c * N3;
      const int x = rr % N, yz = rr / N;
      const int y = yz % N, z = yz / N;
      const double* rc = reinterpret_cast<const double*>(sRg + j * LY::U1R) + c * NN;
      // the face integrals arrive as doubles: added natively after the cell
      // term's conversion (a few FP64 additions instead of splits and
      // emulated additions)
      double v = A::to_double(A::acc_get_norm(out[r]));
      if (x == N - 1) v += rc[0 * 3 * NN + y + N * z];
      if (x == 0) v -= rc[1 * 3 * NN + y + N * z];
      if (y == N - 1) v += rc[2 * 3 * NN + x + N * z];
      if (y == 0) v -= rc[3 * 3 * NN + x + N * z];
      if (z == N - 1) v += rc[4 * 3 * NN + x + N * y];
      if (z == 0) v -= rc[5 * 3 * NN + x + N * y];
      dst3[((size_t)c * m.E + pick2(j, el0, el1)) * N3 + rr] = v;
    }
  }
}

template <class A, int N, int Q>
__global__ void __launch_bounds__(conv_groups_per_block<N, A::emulated>() * conv_threads<N, A::emulated>())
    conv_kernel(const double* __restrict__ u3, const double* __restrict__ rface, double* __restrict__ dst3,
                const __grid_constant__ ConvTabT<typename A::V, N, Q> tb, const MeshDims m) {
  conv_cells<A, N, Q>(u3, rface, dst3, tb, m, blockIdx.x);
}

// Both pipes at once: of every `period` consecutive blocks the first
// `nnative` run the cell kernel in native FP64 (the FP64 pipe, whose
// instructions take few issue slots) and the others in triple-float (the
// FP32 pipe), so that the blocks resident on an SM keep both pipes busy.
// Both arithmetics are at least FP64-wide; the shared memory is sized for
// the larger (triple-float) work space.
template <int N, int Q>
__global__ void __launch_bounds__(conv_groups_per_block<N>() * conv_threads<N>())
    conv_kernel_mix(const double* __restrict__ u3, const double* __restrict__ rface, double* __restrict__ dst3,
                    const __grid_constant__ ConvTabT<double, N, Q> tbn,
                    const __grid_constant__ ConvTabT<tf64, N, Q> tbt, const MeshDims m, const int period,
                    const int nnative) {
  static_assert(conv_threads<N, false>() == conv_threads<N, true>() && !conv_compact<false, N>() &&
                    conv_groups_per_block<N, false>() == conv_groups_per_block<N, true>(),
                "both arithmetics with the same block geometry");
  // the shared memory is sized for the triple-float blocks; the native blocks
  // (with their own layout) must fit in it
  static_assert((conv_fwd_cells_per_block<N>() * ConvLayout<N, Q, false, conv_split_xtest<N, false>()>::PER +
                 6 * Q * N + 2 * Q * ((N + 1) / 2)) * sizeof(double) <=
                    (conv_fwd_cells_per_block<N>() * ConvLayout<N, Q>::PER + 6 * Q * N + 2 * Q * ((N + 1) / 2)) *
                        sizeof(tf64),
                "native blocks fit in the triple-float shared memory");
  if ((int)(blockIdx.x % (unsigned)period) < nnative)
    conv_cells<F64, N, Q>(u3, rface, dst3, tbn, m, blockIdx.x);
  else
    conv_cells<TF64, N, Q>(u3, rface, dst3, tbt, m, blockIdx.x);
}

// Face term of Sec. 3.2, one evaluation per interior face (the mesh is
// periodic, so every face is interior).  Face (e, d) lies between cell e
// ('-', its layer N-1 along d) and its + neighbour along d ('+', layer 0).
// R = (S (x) S)^T [w1 w2 |face| F*] with F* = {{u (x) u}}.n + lambda [[u]],
// n = +e_d, is the face integral against the '-' cell's face-layer basis;
// the '+' cell's is -R (same trace basis, opposite normal).  Written to
// rface[d][e][c][j1 + N j2] (j1, j2: the two tangential directions in
// increasing order).  A group of FT threads treats FPG faces at once and
// synchronises only itself; the interpolation and test phases give each
// thread whole lines (even-odd form, tables read from the kernel parameter:
// every thread uses the same entry at the same time).
template <class A, int N, int Q>
__global__ void __launch_bounds__(face_groups_per_block<face_lines<A::emulated, N>(), N, Q, sizeof(typename A::V)>() *
                                  face_threads<face_lines<A::emulated, N>(), N>())
    conv_face_kernel(const double* __restrict__ u3, double* __restrict__ rface,
                     const __grid_constant__ ConvTabT<typename A::V, N, Q> tb, const MeshDims m) {
  typedef typename A::V V;
  typedef typename A::Acc Acc;
  typedef FaceLayout<N, Q> LY;
  constexpr bool L = face_lines<A::emulated, N>();
  constexpr int FT = face_threads<L, N>(), FPG = faces_per_group<N>(),
                GPB = face_groups_per_block<L, N, Q, sizeof(V)>();
  constexpr int N3 = N * N * N, NN = N * N, QQ = Q * Q, QN = Q * N;
  V* sm = reinterpret_cast<V*>(dyn_smem());
  const int g = threadIdx.x / FT;
  const int t = threadIdx.x - g * FT;
  const int d = blockIdx.y;
  const long long f0 = ((long long)blockIdx.x * GPB + g) * FPG;
  V* base = sm + g * face_group_smem<L, N, Q>();
  V* sS = base + FPG * LY::PER;   // one output per thread: the tables, indexed by thread
  V* sSW = sS + QN;
  // natively from N = 6 on every contraction runs in even-odd form: the
  // lines folded in place into sums (index i) and differences (index
  // L-1-i), then one item per output pair (o, M-1-o) computes E + O and
  // E - O.  Tables (in place of S, SW): interpolation ZE [QH][NH] =
  // (S(q,j) + S(q,N-1-j)) / 2 (S(q,j) in the middle column of odd N),
  // ZO [QH][NF] = (S(q,j) - S(q,N-1-j)) / 2; test TE [QH][NH] =
  // (SW(q,x) + SW(Q-1-q,x)) / 2 (SW in the middle row of odd Q),
  // TO [QF][NH] = (SW(q,x) - SW(Q-1-q,x)) / 2 (S, SW symmetric under
  // (q, j) -> (Q-1-q, N-1-j), so the second output of a pair is E - O).
  constexpr bool EF = !A::emulated && N >= 6;   // at N = 4, 5: 1-3 % slower
  constexpr int NH = (N + 1) / 2, NF = N / 2, QH = (Q + 1) / 2, QF = Q / 2;
  V* sZE = sS;
  V* sZO = sS + QH * NH;
  V* sTE = sSW;
  V* sTO = sSW + QH * NH;
  if constexpr (EF) {
    for (int i = t; i < QH * NH; i += FT) {
      const int q = i / NH, j = i - q * NH;
      sZE[i] = j < NF ? A::half(A::add(tb.S[q * N + j], tb.S[q * N + N - 1 - j])) : tb.S[q * N + j];
      sTE[i] = q < QF ? A::half(A::add(tb.SW[q * N + j], tb.SW[(Q - 1 - q) * N + j])) : tb.SW[q * N + j];
    }
    for (int i = t; i < QH * NF; i += FT) {
      const int q = i / NF, j = i - q * NF;
      sZO[i] = A::half(A::sub(tb.S[q * N + j], tb.S[q * N + N - 1 - j]));
    }
    for (int i = t; i < QF * NH; i += FT) {
      const int q = i / NH, j = i - q * NH;
      sTO[i] = A::half(A::sub(tb.SW[q * N + j], tb.SW[(Q - 1 - q) * N + j]));
    }
  } else if (!L) {
    for (int i = t; i < QN; i += FT) {
      sS[i] = tb.S[i];
      sSW[i] = tb.SW[i];
    }
  }
  const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  static_assert(FPG == 1 || FPG == 2 || FPG == 4, "one, two or four faces per group");
  // cells of the group's faces (scalars, not an array indexed by a runtime
  // face number, which would live in local memory)
  unsigned el0 = 0, nb0 = 0, el1 = 0, nb1 = 0, el2 = 0, nb2 = 0, el3 = 0, nb3 = 0;
  int nact = 0;
#pragma unroll
  for (int f = 0; f < FPG; ++f) {
    if (f0 + f < m.E) {
      const CellXYZ cx = cell_xyz((unsigned)(f0 + f), m);
      const unsigned nbf =
          d == 0 ? neighbor32<0>(cx, 1, m) : (d == 1 ? neighbor32<1>(cx, 1, m) : neighbor32<2>(cx, 1, m));
      if (f == 0) {
        el0 = cx.el;
        nb0 = nbf;
      } else if (f == 1) {
        el1 = cx.el;
        nb1 = nbf;
      } else if (f == 2) {
        el2 = cx.el;
        nb2 = nbf;
      } else {
        el3 = cx.el;
        nb3 = nbf;
      }
      nact = f + 1;
    }
  }
  auto face_el = [&](int f) { return f < 2 ? (f == 0 ? el0 : el1) : (f == 2 ? el2 : el3); };
  auto face_nb = [&](int f) { return f < 2 ? (f == 0 ? nb0 : nb1) : (f == 2 ? nb2 : nb3); };
  // per face f: T0 [s][c][j1 + N j2] (s = 0: '-', 1: '+'), later K1 [c][q1 + Q j2];
  // G1 [s][c][q1 + Q j2], later H [c][q1 + Q q2]; G2 [s][c][q1 + Q q2]
#define FACE_T0(f) (base + (f) * LY::PER)
#define FACE_G1(f) (base + (f) * LY::PER + LY::T0)
#define FACE_G2(f) (base + (f) * LY::PER + LY::T0 + LY::G1)
  // F0: the face layers of both cells
  for (int it = t; it < nact * 6 * NN; it += FT) {
    const int f = it / (6 * NN), i = it - f * 6 * NN;
    const int sc = i / NN, r = i - sc * NN;
    const int sd = sc / 3, c = sc - 3 * sd;
    const int j1 = r % N, j2 = r / N;
    const unsigned cell = sd == 0 ? face_el(f) : face_nb(f);
    FACE_T0(f)[i] = A::load(u3 + ((size_t)c * m.E + cell) * N3 + node3(N, d, sd == 0 ? N - 1 : 0, t1, j1, t2, j2));
  }
  group_sync<FT>();
  // F1: interpolate along t1
  if constexpr (EF) {   // lines (f, sc, j2) folded, then item (f, sc, j2, q1 < QH)
    for (int it = t; it < nact * 6 * N * NF; it += FT) {
      const int r = it / NF, j = it - r * NF;   // r = (f, sc, j2)
      const int f = r / (6 * N);
      fold_pair<A>(FACE_T0(f) + (r - f * 6 * N) * N + j, N - 1 - 2 * j);
    }
    group_sync<FT>();
    for (int it = t; it < nact * 6 * N * QH; it += FT) {
      const int q1 = it % QH, r = it / QH;
      const int f = r / (6 * N), l = r - f * 6 * N;
      const int sc = l / N, j2 = l - sc * N;
      V e, o;
      fold_dot<A, N, NH, NF>(sZE + q1 * NH, 1, sZO + q1 * NF, 1, FACE_T0(f) + l * N, 1, e, o);
      V* g = FACE_G1(f) + sc * QN + Q * j2;
      g[q1] = A::add(e, o);
      if (q1 != Q - 1 - q1) g[Q - 1 - q1] = A::sub(e, o);
    }
  } else if constexpr (L) {   // item (f, sc, j2): one line of N values -> Q
    for (int it = t; it < nact * 6 * N; it += FT) {
      const int f = it / (6 * N), i = it - f * 6 * N;
      const int sc = i / N, j2 = i - sc * N;
      interp_eo<A, N, Q>(tb.IE, FACE_T0(f) + sc * NN + N * j2, 1, FACE_G1(f) + sc * QN + Q * j2, 1);
    }
  } else {   // item (f, sc, j2, q1)
    for (int it = t; it < nact * 6 * QN; it += FT) {
      const int f = it / (6 * QN), i = it - f * 6 * QN;
      const int q1 = i % Q, r = i / Q;
      const int sc = r / N, j2 = r - sc * N;
      const V* v = FACE_T0(f) + sc * NN + N * j2;
      Acc a;
      A::acc_first(a, sS[q1 * N], v[0]);
#pragma unroll
      for (int j = 1; j < N; ++j) A::acc_fma(a, sS[q1 * N + j], v[j]);
      FACE_G1(f)[sc * QN + q1 + Q * j2] = A::acc_get_norm(a);
    }
  }
  group_sync<FT>();
  // F2: along t2 (the traces are compared in F3, so they are normalised)
  if constexpr (EF) {   // columns (f, sc, q1) folded, then item (f, sc, q1, q2 < QH)
    for (int it = t; it < nact * 6 * Q * NF; it += FT) {
      const int r = it / NF, j = it - r * NF;   // r = (f, sc, q1)
      const int f = r / (6 * Q), l = r - f * 6 * Q;
      const int sc = l / Q, q1 = l - sc * Q;
      fold_pair<A>(FACE_G1(f) + sc * QN + q1 + Q * j, Q * (N - 1 - 2 * j));
    }
    group_sync<FT>();
    for (int it = t; it < nact * 6 * Q * QH; it += FT) {
      const int q2 = it % QH, r = it / QH;
      const int f = r / (6 * Q), l = r - f * 6 * Q;
      const int sc = l / Q, q1 = l - sc * Q;
      V e, o;
      fold_dot<A, N, NH, NF>(sZE + q2 * NH, 1, sZO + q2 * NF, 1, FACE_G1(f) + sc * QN + q1, Q, e, o);
      V* g = FACE_G2(f) + sc * QQ + q1;
      g[Q * q2] = A::add(e, o);
      if (q2 != Q - 1 - q2) g[Q * (Q - 1 - q2)] = A::sub(e, o);
    }
  } else if constexpr (L) {   // item (f, sc, q1)
    for (int it = t; it < nact * 6 * Q; it += FT) {
      const int f = it / (6 * Q), i = it - f * 6 * Q;
      const int sc = i / Q, q1 = i - sc * Q;
      interp_eo<A, N, Q>(tb.IE, FACE_G1(f) + sc * QN + q1, Q, FACE_G2(f) + sc * QQ + q1, Q);
    }
  } else {   // item (f, sc, q1, q2)
    for (int it = t; it < nact * 6 * QQ; it += FT) {
      const int f = it / (6 * QQ), i = it - f * 6 * QQ;
      const int q2 = i % Q, r = i / Q;
      const int sc = r / Q, q1 = r - sc * Q;
      const V* v = FACE_G1(f) + sc * QN + q1;
      Acc a;
      A::acc_first(a, sS[q2 * N], v[0]);
#pragma unroll
      for (int j = 1; j < N; ++j) A::acc_fma(a, sS[q2 * N + j], v[Q * j]);
      FACE_G2(f)[sc * QQ + q1 + Q * q2] = A::acc_get_norm(a);
    }
  }
  group_sync<FT>();
  // F3: LLF flux at the face points (weights are in the test tables); item (c, point)
  for (int it = t; it < nact * 3 * QQ; it += FT) {
    const int f = it / (3 * QQ), i = it - f * 3 * QQ;
    const int c = i / QQ, pt = i - c * QQ;
    const V* g2 = FACE_G2(f) + pt;
    const V umc = g2[c * QQ], upc = g2[(3 + c) * QQ];
    const V unm = g2[d * QQ], unp = g2[(3 + d) * QQ];
    if constexpr (!A::emulated) {
      // natively twice the flux, u-_c un- + u+_c un+ + 2 lambda (u-_c - u+_c),
      // in four FP64 operations: lambda = max(|un-|, |un+|) by an integer
      // comparison (the bit patterns of non-negative doubles order as their
      // values), 2 lambda by an exponent increment (normal numbers; else an
      // addition), and the halving moved into the face area of F5.  Scaling
      // by 2 commutes with every rounding, so the results are those of the
      // halved form.
      const long long bm = __double_as_longlong(unm) & 0x7fffffffffffffffLL;
      const long long bp = __double_as_longlong(unp) & 0x7fffffffffffffffLL;
      const long long bl = bm > bp ? bm : bp;
      const long long ex = bl >> 52;
      double lam2;
      if (ex != 0 && ex < 2046) {
        lam2 = __longlong_as_double(bl + (1LL << 52));
      } else {
        const double l = __longlong_as_double(bl);
        lam2 = l + l;
      }
      const double t = fma(upc, unp, umc * unm);
      FACE_G1(f)[i] = fma(lam2, umc - upc, t);
    } else {
      const V am = A::absval(unm), ap = A::absval(unp);
      const V lam = A::greater(am, ap) ? am : ap;
      // 0.5 (u-_c un- + u+_c un+) + lambda (u-_c - u+_c), the halving is exact
      Acc fl;
      A::acc_first(fl, umc, A::half(unm));
      A::acc_fma(fl, upc, A::half(unp));
      A::acc_fma(fl, lam, A::sub(umc, upc));
      FACE_G1(f)[i] = A::acc_get_norm(fl);
    }
  }
  group_sync<FT>();
  // F4: test along t2 (weights w_q2)
  if constexpr (EF) {   // flux columns (f, c, q1) folded, then item (f, c, q1, j2 < NH)
    for (int it = t; it < nact * 3 * Q * QF; it += FT) {
      const int r = it / QF, i = it - r * QF;   // r = (f, c, q1)
      const int f = r / (3 * Q), l = r - f * 3 * Q;
      const int c = l / Q, q1 = l - c * Q;
      fold_pair<A>(FACE_G1(f) + c * QQ + q1 + Q * i, Q * (Q - 1 - 2 * i));
    }
    group_sync<FT>();
    for (int it = t; it < nact * 3 * Q * NH; it += FT) {
      const int j2 = it % NH, r = it / NH;
      const int f = r / (3 * Q), l = r - f * 3 * Q;
      const int c = l / Q, q1 = l - c * Q;
      V e, o;
      fold_dot<A, Q, QH, QF>(sTE + j2, NH, sTO + j2, NH, FACE_G1(f) + c * QQ + q1, Q, e, o);
      V* k = FACE_T0(f) + c * QN + q1;
      k[Q * j2] = A::add(e, o);
      if (j2 != N - 1 - j2) k[Q * (N - 1 - j2)] = A::sub(e, o);
    }
  } else if constexpr (L) {   // item (f, c, q1): Q values -> N
    for (int it = t; it < nact * 3 * Q; it += FT) {
      const int f = it / (3 * Q), i = it - f * 3 * Q;
      const int c = i / Q, q1 = i - c * Q;
      V o[N];
      test_eo<A, N, Q>(tb.EO[1], FACE_G1(f) + c * QQ + q1, Q, o);
      V* k = FACE_T0(f) + c * QN + q1;
#pragma unroll
      for (int j2 = 0; j2 < N; ++j2) k[Q * j2] = o[j2];
    }
  } else {   // item (f, c, j2, q1)
    for (int it = t; it < nact * 3 * QN; it += FT) {
      const int f = it / (3 * QN), i = it - f * 3 * QN;
      const int q1 = i % Q, r = i / Q;
      const int c = r / N, j2 = r - c * N;
      const V* h = FACE_G1(f) + c * QQ + q1;
      Acc a;
      A::acc_first(a, sSW[j2], h[0]);
#pragma unroll
      for (int q2 = 1; q2 < Q; ++q2) A::acc_fma(a, sSW[q2 * N + j2], h[Q * q2]);
      FACE_T0(f)[c * QN + q1 + Q * j2] = A::acc_get_norm(a);
    }
  }
  group_sync<FT>();
  // F5: test along t1 (weights w_q1), times the face area, store
  // the face area scales the stored results in FP64 (one multiplication
  // after the conversion instead of an emulated product)
  const double area = A::to_double(tb.area[d]) * (A::emulated ? 1.0 : 0.5);   // natively F3 doubled the flux
  if constexpr (EF) {   // rows (f, c, j2) folded, then item (f, c, j2, j1 < NH)
    for (int it = t; it < nact * 3 * N * QF; it += FT) {
      const int r = it / QF, i = it - r * QF;   // r = (f, c, j2)
      const int f = r / (3 * N), l = r - f * 3 * N;
      fold_pair<A>(FACE_T0(f) + l * Q + i, Q - 1 - 2 * i);
    }
    group_sync<FT>();
    for (int it = t; it < nact * 3 * N * NH; it += FT) {
      const int j1 = it % NH, r = it / NH;
      const int f = r / (3 * N), l = r - f * 3 * N;   // l = (c, j2)
      V e, o;
      fold_dot<A, Q, QH, QF>(sTE + j1, NH, sTO + j1, NH, FACE_T0(f) + l * Q, 1, e, o);
      double* dst = rface + ((size_t)d * m.E + face_el(f)) * 3 * NN + l * N;
      dst[j1] = area * A::to_double(A::add(e, o));
      if (j1 != N - 1 - j1) dst[N - 1 - j1] = area * A::to_double(A::sub(e, o));
    }
  } else if constexpr (L) {   // item (f, c, j2)
    for (int it = t; it < nact * 3 * N; it += FT) {
      const int f = it / (3 * N), i = it - f * 3 * N;
      const int c = i / N, j2 = i - c * N;
      V o[N];
      test_eo<A, N, Q>(tb.EO[1], FACE_T0(f) + c * QN + Q * j2, 1, o);
      double* dst = rface + ((size_t)d * m.E + face_el(f)) * 3 * NN + c * NN + N * j2;
#pragma unroll
      for (int j1 = 0; j1 < N; ++j1) dst[j1] = area * A::to_double(o[j1]);
    }
  } else {   // item (f, c, j2, j1)
    for (int it = t; it < nact * 3 * NN; it += FT) {
      const int f = it / (3 * NN), i = it - f * 3 * NN;
      const int c = i / NN, r = i - c * NN;
      const int j1 = r % N, j2 = r / N;
      const V* k = FACE_T0(f) + c * QN + Q * j2;
      Acc a;
      A::acc_first(a, sSW[j1], k[0]);
#pragma unroll
      for (int q1 = 1; q1 < Q; ++q1) A::acc_fma(a, sSW[q1 * N + j1], k[q1]);
      rface[((size_t)d * m.E + face_el(f)) * 3 * NN + i] = area * A::to_double(A::acc_get_norm(a));
    }
  }
#undef FACE_T0
#undef FACE_G1
#undef FACE_G2
}

template <class A, int N, int Q>
ConvTabT<typename A::V, N, Q> conv_tables(const ConvHost& h) {
  ConvTabT<typename A::V, N, Q> tb;
  double jac[3];
  for (int d = 0; d < 3; ++d) {
    jac[d] = h.h[0] * h.h[1] * h.h[2] / h.h[d];
    tb.area[d] = A::make(jac[d]);
  }
  for (int q = 0; q < Q; ++q)
    for (int j = 0; j < N; ++j) {
      const int i = q * N + j;
      tb.S[i] = A::make(h.S[i]);
      tb.SW[i] = A::make(h.w[q] * h.S[i]);
      tb.DW[i] = A::make(h.w[q] * h.D[i]);
      tb.TY[0][i] = A::make(jac[0] * h.w[q] * h.S[i]);
      tb.TY[1][i] = A::make(jac[1] * h.w[q] * h.D[i]);
      tb.TY[2][i] = A::make(jac[2] * h.w[q] * h.S[i]);
    }
  {
    constexpr int QH0 = (Q + 1) / 2, NH0 = (N + 1) / 2;
    for (int d = 0; d < 3; ++d) {
      const double* T = d == 1 ? h.D : h.S;   // jac_d w (S or D): DW antisymmetric
      const double sg = d == 1 ? -1.0 : 1.0;
      for (int i = 0; i < Q; ++i)
        for (int x = 0; x < NH0; ++x) {
          const int q = i < QH0 ? i : i - QH0;
          const double a = jac[d] * h.w[q] * T[q * N + x], b = jac[d] * h.w[q] * T[q * N + N - 1 - x];
          tb.TYeo[d][i * NH0 + x] = A::make(i < QH0 ? 0.5 * (a + sg * b) : 0.5 * (a - sg * b));
        }
    }
  }
  constexpr int QH = (Q + 1) / 2, NH = (N + 1) / 2;
  for (int ty = 0; ty < 2; ++ty) {
    const double* T = ty == 0 ? h.D : h.S;   // DW (antisymmetric), SW (symmetric), times w_q
    const double s = ty == 0 ? -1.0 : 1.0;
    for (int i = 0; i < Q; ++i)
      for (int x = 0; x < NH; ++x) {
        // rows 0..QH-1: T1, rows QH..Q-1: T2 (row i - QH)
        const int q = i < QH ? i : i - QH;
        const double a = h.w[q] * T[q * N + x], b = h.w[q] * T[q * N + N - 1 - x];
        tb.EO[ty][i * NH + x] = A::make(i < QH ? 0.5 * (a + s * b) : 0.5 * (a - s * b));
      }
  }
  {
    constexpr int NF = N / 2, QF = Q / 2;
    for (int q = 0; q < QH; ++q)
      for (int j = 0; j < NH; ++j)
        tb.IE[q * NH + j] =
            A::make(j < NF ? 0.5 * (h.S[q * N + j] + h.S[q * N + N - 1 - j]) : h.S[q * N + j]);
    for (int q = 0; q < QF; ++q)
      for (int j = 0; j < NF; ++j)
        tb.IE[QH * NH + q * NF + j] = A::make(0.5 * (h.S[q * N + j] - h.S[q * N + N - 1 - j]));
  }
  return tb;
}

// part: bit 0 the face kernel (u3 -> rface), bit 1 the cell kernel
// (u3, rface -> dst3).
template <class A, int N, int Q>
int launch_conv(int part, const MeshDims& m, const double* u3, double* rface, double* dst3, const ConvHost& h,
                cudaStream_t s) {
  const ConvTabT<typename A::V, N, Q> tb = conv_tables<A, N, Q>(h);
  constexpr bool FL = face_lines<A::emulated, N>();
  typedef typename A::V V;
  constexpr int EPB = conv_fwd_cells_per_block<N, A::emulated>(), GPB = face_groups_per_block<FL, N, Q, sizeof(V)>(),
                FPG = faces_per_group<N>();
  constexpr int FPB = GPB * FPG;
  // tables: S, SW, DW, TY (6 Q N), EO (2 Q (N+1)/2), and natively (paired
  // planes) ZE, ZO ((Q+1)/2 N) and the z-test tables (4 (Q+1)/2 (N+1)/2)
  constexpr int NH = (N + 1) / 2, QH = (Q + 1) / 2;
  constexpr int TABS = 6 * Q * N + 2 * Q * NH + (conv_pair_planes<A::emulated, N, Q>() ? QH * N + 4 * QH * NH : 0);
  const size_t smem =
      ((size_t)EPB * ConvLayout<N, Q, conv_compact<A::emulated, N>(), conv_split_xtest<N, A::emulated>()>::PER + TABS) *
      sizeof(V);
  const size_t fsmem = (size_t)GPB * face_group_smem<FL, N, Q>() * sizeof(V);
  if (smem > 232448 || fsmem > 232448) return 7;
  if (cudaFuncSetAttribute(conv_kernel<A, N, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(conv_face_kernel<A, N, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem) !=
          cudaSuccess)
    return 2;
  if (m.E == 0) return 0;
  if (part & 1) {
    const dim3 fgrid((unsigned)((m.E + FPB - 1) / FPB), 3);
    conv_face_kernel<A, N, Q><<<fgrid, GPB * face_threads<FL, N>(), fsmem, s>>>(u3, rface, tb, m);
  }
  if (part & 2) {
    const long long blocks = (m.E + EPB - 1) / EPB;
    conv_kernel<A, N, Q><<<(unsigned)blocks, conv_groups_per_block<N, A::emulated>() * conv_threads<N, A::emulated>(), smem, s>>>(
        u3, rface, dst3, tb, m);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// ------------------------------------------------------------------- VJP
// grad_u = (dC/du)^T w.  Cell: with g_cd(q) = sum_i w_c,i d_d phi_i(q), the
// cell part of <w, C(u)> is -sum_q W sum_cd g_cd u_c u_d, whose derivative
// in u_e(q) is -W sum_d (g_ed + g_de) u_d, tested with phi.  Faces: the
// product rule on the LLF flux, d|s| = sign(s) (sign(0) = 0), d max sent to
// the larger argument (half to each on a tie).
template <int N, int Q>
struct VjpLayout {
  static constexpr int N3 = N * N * N;
  static constexpr int UW = 6 * N3;              // u and w, nodal
  static constexpr int L1 = 9 * Q * N * N;       // x-sweeps (u: S; w: S, D); later: result
  static constexpr int L2 = 12 * Q * Q * N;      // xy-sweeps (u: SS; w: DS, SD, SS); later: faces
  static constexpr int FACE = 12 * Q * N + 12 * Q * Q + 3 * Q * Q;
  static constexpr int L2F = L2 > FACE ? L2 : FACE;
  static constexpr int P = 12 * Q * Q;           // plane: u (3) and g (9)
  static constexpr int X = 3 * N * Q;
  static constexpr int Y = 3 * N * N;
  static constexpr int PER = UW + L1 + L2F + P + X + Y;
};

// Plane-first layout (from N = 9 on, where the swept layers above exceed the
// shared memory): every quadrature plane z_q contracts u and w over z first
// (9 fields of N^2), then over x (12 fields of Q N) and y (12 fields of Q^2),
// the same flops as sweeping x, y, z over the whole cell, with per-plane
// buffers only.  The result has its own region (the faces read u and w).
template <int N, int Q>
struct VjpLayoutPF {
  static constexpr int N3 = N * N * N;
  static constexpr int UW = 6 * N3;
  static constexpr int OUT = 3 * N3;
  static constexpr int ZB = 9 * N * N;
  static constexpr int XB = 12 * Q * N;
  static constexpr int P = 12 * Q * Q;
  static constexpr int X = 3 * N * Q;
  static constexpr int Y = 3 * N * N;
  static constexpr int CELL = ZB + XB + P + X + Y;
  static constexpr int FACE = 12 * Q * N + 12 * Q * Q + 3 * Q * Q;
  static constexpr int WORK = CELL > FACE ? CELL : FACE;
  static constexpr int PER = UW + OUT + WORK;
};

template <class V, int N, int Q>
struct VjpTab {
  V S[Q * N];   // phi_j(x_q)
  V D[Q * N];   // phi_j'(x_q)
  V w[Q];       // Gauss weights on [0, 1]
  V jac[3];     // h_x h_y h_z / h_d
  V area[3];    // face area of faces normal to d
};

// One cell per N^2 threads, EPB cells per block; arithmetic policy A (F64
// or DF64), loads and stores in double; PF: the plane-first cell stage.
template <class A, int N, int Q, bool PF = false>
__global__ void __launch_bounds__(conv_cells_per_block<N>() * N * N)
    conv_vjp_kernel(const double* __restrict__ u3, const double* __restrict__ w3, double* __restrict__ dst3,
                    const __grid_constant__ VjpTab<typename A::V, N, Q> tb, const MeshDims m) {
  typedef typename A::V V;
  typedef typename A::Acc Acc;
  typedef VjpLayout<N, Q> LY;
  typedef VjpLayoutPF<N, Q> LP;
  static_assert(sizeof(V) == sizeof(double), "8-byte values");
  constexpr int PER = PF ? LP::PER : LY::PER;
  constexpr int NT = N * N, N3 = N * N * N, EPB = conv_cells_per_block<N>();
  constexpr int QNN = Q * N * N, QQN = Q * Q * N, QQ = Q * Q;
  V* sm = reinterpret_cast<V*>(dyn_smem());
  const int slot = threadIdx.x / NT;
  const int t = threadIdx.x - slot * NT;
  const long long c0 = (long long)blockIdx.x * EPB;
  const long long rem = m.E - c0;
  const int nvalid = rem < EPB ? (int)rem : EPB;
  const bool active = slot < nvalid;
  V* sUW = sm + slot * PER;       // u: [0, 3N3), w: [3N3, 6N3)
  // whole-cell sweeps: L1 = u_S (3), w_S (3), w_D (3), each Q N N; L2 = u_SS
  // (3), w_DS (3), w_SD (3), w_SS (3), each Q Q N; the result over L1, the
  // faces over L2.  Plane-first: ZB, XB per plane, result and faces apart.
  V* sL1 = sUW + LY::UW;
  V* sL2 = sL1 + LY::L1;
  V* sZ = sUW + LP::UW + LP::OUT;
  V* sXB = sZ + LP::ZB;
  V* sP = PF ? sXB + LP::XB : sL2 + LY::L2F;   // u (3 Q Q), g (9 Q Q)
  V* sX = sP + LY::P;
  V* sY = sX + LY::X;
  V* sOut = PF ? sUW + LP::UW : sL1;
  V* sFace = PF ? sZ : sL2;

  long long el = 0;
  int ex = 0, ey = 0, ez = 0;
  if (active) {
    el = c0 + slot;
    const unsigned eu = (unsigned)el, nxu = (unsigned)m.nx, nyu = (unsigned)m.ny;
    ex = (int)(eu % nxu);
    const unsigned tt = eu / nxu;
    ey = (int)(tt % nyu);
    ez = (int)(tt / nyu);
    for (int c = 0; c < 3; ++c)
      for (int i = t; i < N3; i += NT) {
        sUW[c * N3 + i] = A::load(u3 + (c * m.E + el) * N3 + i);
        sUW[(3 + c) * N3 + i] = A::load(w3 + (c * m.E + el) * N3 + i);
      }
  }
  __syncthreads();
  // x-sweeps: u_S, w_S, w_D
  if (!PF && active)
    for (int it = t; it < 6 * N * N; it += NT) {
      const int f = it / (N * N), l = it - f * N * N;   // f < 3: u_c, else w_(f-3)
      V x[N];
      load_line<V, N>(sUW + f * N3, l * N, 1, x);
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        Acc a, b;
        A::acc_first(a, tb.S[q * N], x[0]);
        A::acc_first(b, tb.D[q * N], x[0]);
#pragma unroll
        for (int j = 1; j < N; ++j) {
          A::acc_fma(a, tb.S[q * N + j], x[j]);
          A::acc_fma(b, tb.D[q * N + j], x[j]);
        }
        sL1[f * QNN + l * Q + q] = A::acc_get_norm(a);                     // u_S (f<3) or w_S (f>=3)
        if (f >= 3) sL1[(f + 3) * QNN + l * Q + q] = A::acc_get_norm(b);    // w_D
      }
    }
  if (!PF) __syncthreads();
  // y-sweeps: u_SS, w_DS (from w_D), w_SD and w_SS (from w_S)
  if (!PF && active)
    for (int it = t; it < 6 * Q * N; it += NT) {
      const int f = it / (Q * N), l = it - f * Q * N;
      const int qx = l % Q, z = l / Q;
      V x[N];
      if (f < 3) {
        load_line<V, N>(sL1 + f * QNN, qx + Q * N * z, Q, x);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          Acc a;
          A::acc_first(a, tb.S[q * N], x[0]);
#pragma unroll
          for (int j = 1; j < N; ++j) A::acc_fma(a, tb.S[q * N + j], x[j]);
          sL2[f * QQN + qx + Q * q + QQ * z] = A::acc_get_norm(a);
        }
      } else {
        const int c = f - 3;
        V y[N];
        load_line<V, N>(sL1 + (3 + c) * QNN, qx + Q * N * z, Q, x);   // w_S
        load_line<V, N>(sL1 + (6 + c) * QNN, qx + Q * N * z, Q, y);   // w_D
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          Acc ds, sd, ss;
          A::acc_first(ds, tb.S[q * N], y[0]);
          A::acc_first(sd, tb.D[q * N], x[0]);
          A::acc_first(ss, tb.S[q * N], x[0]);
#pragma unroll
          for (int j = 1; j < N; ++j) {
            A::acc_fma(ds, tb.S[q * N + j], y[j]);
            A::acc_fma(sd, tb.D[q * N + j], x[j]);
            A::acc_fma(ss, tb.S[q * N + j], x[j]);
          }
          sL2[(3 + c) * QQN + qx + Q * q + QQ * z] = A::acc_get_norm(ds);
          sL2[(6 + c) * QQN + qx + Q * q + QQ * z] = A::acc_get_norm(sd);
          sL2[(9 + c) * QQN + qx + Q * q + QQ * z] = A::acc_get_norm(ss);
        }
      }
    }
  if (!PF) __syncthreads();

  Acc acc[3][N];
  const int tx = t % N, ty = t / N;
  for (int qz = 0; qz < Q; ++qz) {
    if constexpr (PF) {
      // P1, plane-first: z-contraction at z_q of u (S), w (S) and w (D) ...
      if (active)
        for (int it = t; it < 9 * N * N; it += NT) {
          const int f = it / (N * N), l = it - f * (N * N);
          const V* src = sUW + (f < 3 ? f : 3 + (f - 3) % 3) * N3 + l;
          const V* T = f >= 6 ? tb.D : tb.S;
          Acc a;
          A::acc_first(a, T[qz * N], src[0]);
#pragma unroll
          for (int z = 1; z < N; ++z) A::acc_fma(a, T[qz * N + z], src[N * N * z]);
          sZ[it] = A::acc_get_norm(a);
        }
      __syncthreads();
      // ... then over x: u S; w_S D (-> g_cx), w_S S (-> g_cy), w_D S (-> g_cz)
      if (active)
        for (int it = t; it < 12 * N; it += NT) {
          const int f = it / N, y = it - f * N;
          const int zf = f < 3 ? f : (f < 9 ? 3 + (f - 3) % 3 : 6 + (f - 9));
          const V* T = (f >= 3 && f < 6) ? tb.D : tb.S;
          V x[N];
          load_line<V, N>(sZ + zf * N * N, N * y, 1, x);
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            Acc a;
            A::acc_first(a, T[q * N], x[0]);
#pragma unroll
            for (int j = 1; j < N; ++j) A::acc_fma(a, T[q * N + j], x[j]);
            sXB[f * Q * N + q + Q * y] = A::acc_get_norm(a);
          }
        }
      __syncthreads();
      // ... then over y (D for g_cy), into the plane layout of P1 below
      if (active)
        for (int it = t; it < 12 * Q; it += NT) {
          const int f = it / Q, qx = it - f * Q;
          const int pf = f < 3 ? f : 3 + 3 * ((f - 3) % 3) + (f - 3) / 3;
          const V* T = (f >= 6 && f < 9) ? tb.D : tb.S;
          V x[N];
          load_line<V, N>(sXB + f * Q * N, qx, Q, x);
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            Acc a;
            A::acc_first(a, T[q * N], x[0]);
#pragma unroll
            for (int j = 1; j < N; ++j) A::acc_fma(a, T[q * N + j], x[j]);
            sP[pf * QQ + qx + Q * q] = A::acc_get_norm(a);
          }
        }
    }
    // P1: u (3) and g_cd (9) on the plane; g_cx from w_DS, g_cy from w_SD
    // (both S in z), g_cz from w_SS (D in z)
    if (!PF && active)
      for (int it = t; it < 12 * QQ; it += NT) {
        const int f = it / QQ, l = it - f * QQ;
        const V* src;
        bool dz = false;
        if (f < 3) {
          src = sL2 + f * QQN;
        } else {
          const int c = (f - 3) / 3, d = (f - 3) % 3;
          src = sL2 + (d == 0 ? 3 + c : (d == 1 ? 6 + c : 9 + c)) * QQN;
          dz = d == 2;
        }
        src += l;
        const V* T = dz ? tb.D : tb.S;
        Acc a;
        A::acc_first(a, T[qz * N], src[0]);
#pragma unroll
        for (int z = 1; z < N; ++z) A::acc_fma(a, T[qz * N + z], src[QQ * z]);
        sP[it] = A::acc_get_norm(a);
      }
    __syncthreads();
    // P2: pointwise -W sum_d (g_ed + g_de) u_d, with reference derivatives
    // scaled by jac[d] = h_x h_y h_z / h_d; result overwrites u on the plane
    if (active)
      for (int it = t; it < QQ; it += NT) {
        const int qx = it % Q, qy = it / Q;
        const V w3q = A::mul(A::mul(tb.w[qx], tb.w[qy]), tb.w[qz]);
        V u[3], g[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) u[c] = sP[c * QQ + it];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int d = 0; d < 3; ++d) g[c][d] = A::mul(tb.jac[d], sP[(3 + 3 * c + d) * QQ + it]);
        V r[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          Acc a;
          A::acc_first(a, A::add(g[e][0], g[0][e]), u[0]);
#pragma unroll
          for (int d = 1; d < 3; ++d) A::acc_fma(a, A::add(g[e][d], g[d][e]), u[d]);
          r[e] = A::neg(A::mul(w3q, A::acc_get_norm(a)));
        }
#pragma unroll
        for (int e = 0; e < 3; ++e) sP[e * QQ + it] = r[e];
      }
    __syncthreads();
    // P3: x test
    if (active)
      for (int it = t; it < 3 * Q; it += NT) {
        const int c = it / Q, qy = it - c * Q;
        Acc a[N];
#pragma unroll
        for (int qx = 0; qx < Q; ++qx) {
          const V gv = sP[c * QQ + qx + Q * qy];
#pragma unroll
          for (int x = 0; x < N; ++x) {
            if (qx == 0)
              A::acc_first(a[x], tb.S[x], gv);
            else
              A::acc_fma(a[x], tb.S[qx * N + x], gv);
          }
        }
#pragma unroll
        for (int x = 0; x < N; ++x) sX[c * N * Q + x + N * qy] = A::acc_get_norm(a[x]);
      }
    __syncthreads();
    // P4: y test
    if (active)
      for (int it = t; it < 3 * N; it += NT) {
        const int c = it / N, x = it - c * N;
        Acc a[N];
#pragma unroll
        for (int qy = 0; qy < Q; ++qy) {
          const V b = sX[c * N * Q + x + N * qy];
#pragma unroll
          for (int y = 0; y < N; ++y) {
            if (qy == 0)
              A::acc_first(a[y], tb.S[y], b);
            else
              A::acc_fma(a[y], tb.S[qy * N + y], b);
          }
        }
#pragma unroll
        for (int y = 0; y < N; ++y) sY[c * N * N + x + N * y] = A::acc_get_norm(a[y]);
      }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const V yv = sY[c * N * N + tx + N * ty];
#pragma unroll
        for (int z = 0; z < N; ++z) {
          if (qz == 0)
            A::acc_first(acc[c][z], tb.S[z], yv);
          else
            A::acc_fma(acc[c][z], tb.S[qz * N + z], yv);
        }
      }
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int z = 0; z < N; ++z) sOut[c * N3 + tx + N * ty + N * N * z] = A::acc_get_norm(acc[c][z]);
  }
  __syncthreads();

  // ---------------------------------------------------------------- faces
  // traces: index f = (side s, field v, comp c) -> s*6 + v*3 + c, v: 0 = u, 1 = w
  V* G1 = sFace;                 // [f][q1 + Q j2]   12 Q N
  V* G2 = G1 + 12 * Q * N;       // [f][q1 + Q q2]   12 Q Q
  V* H = G2 + 12 * QQ;           // [c][q1 + Q q2]   3 Q Q
  V* K1 = G1;
  for (int d = 0; d < 3; ++d) {
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    for (int side = 1; side >= -1; side -= 2) {
      long long nb = 0;
      if (active) {
        if (d == 0) nb = neighbor<0>(el, ex, ey, ez, side, m);
        else if (d == 1) nb = neighbor<1>(el, ex, ey, ez, side, m);
        else nb = neighbor<2>(el, ex, ey, ez, side, m);
      }
      const int aown = side > 0 ? N - 1 : 0, anb = side > 0 ? 0 : N - 1;
      if (active)
        for (int it = t; it < 12 * N; it += NT) {
          const int f = it / N, j2 = it - f * N;
          const int s = f / 6, v = (f / 3) % 2, c = f % 3;
          const double* gsrc = v == 0 ? u3 : w3;
          V val[N];
#pragma unroll
          for (int j1 = 0; j1 < N; ++j1)
            val[j1] = s == 0 ? sUW[(v * 3 + c) * N3 + node3(N, d, aown, t1, j1, t2, j2)]
                             : A::load(gsrc + (c * m.E + nb) * N3 + node3(N, d, anb, t1, j1, t2, j2));
#pragma unroll
          for (int q1 = 0; q1 < Q; ++q1) {
            Acc a;
            A::acc_first(a, tb.S[q1 * N], val[0]);
#pragma unroll
            for (int j = 1; j < N; ++j) A::acc_fma(a, tb.S[q1 * N + j], val[j]);
            G1[f * Q * N + q1 + Q * j2] = A::acc_get_norm(a);
          }
        }
      __syncthreads();
      if (active)
        for (int it = t; it < 12 * Q; it += NT) {
          const int f = it / Q, q1 = it - f * Q;
          V val[N];
#pragma unroll
          for (int j2 = 0; j2 < N; ++j2) val[j2] = G1[f * Q * N + q1 + Q * j2];
#pragma unroll
          for (int q2 = 0; q2 < Q; ++q2) {
            Acc a;
            A::acc_first(a, tb.S[q2 * N], val[0]);
#pragma unroll
            for (int j = 1; j < N; ++j) A::acc_fma(a, tb.S[q2 * N + j], val[j]);
            G2[f * QQ + q1 + Q * q2] = A::acc_get_norm(a);   // compared below
          }
        }
      __syncthreads();
      if (active)
        for (int it = t; it < QQ; it += NT) {
          const int q1 = it % Q, q2 = it / Q;
          const int sm_ = side > 0 ? 0 : 1, sp_ = side > 0 ? 1 : 0;  // trace side of '-' / '+'
          V um[3], up[3], jw[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            um[c] = G2[(sm_ * 6 + c) * QQ + it];
            up[c] = G2[(sp_ * 6 + c) * QQ + it];
            jw[c] = A::sub(G2[(sm_ * 6 + 3 + c) * QQ + it], G2[(sp_ * 6 + 3 + c) * QQ + it]);
          }
          const V unm = um[d], unp = up[d];
          const V am = A::absval(unm), ap = A::absval(unp);
          const bool mbig = A::greater(am, ap), pbig = A::greater(ap, am);
          const V lam = mbig ? am : ap;
          // derivative of max(|un-|, |un+|): sign to the larger side, half to
          // each on a tie
          const float smx = mbig ? (float)A::sign(unm) : (pbig ? 0.0f : 0.5f * (float)A::sign(unm));
          const float spx = pbig ? (float)A::sign(unp) : (mbig ? 0.0f : 0.5f * (float)A::sign(unp));
          Acc jum, jup, jdu;
          A::acc_first(jum, jw[0], um[0]);
          A::acc_first(jup, jw[0], up[0]);
          A::acc_first(jdu, jw[0], A::sub(um[0], up[0]));
#pragma unroll
          for (int c = 1; c < 3; ++c) {
            A::acc_fma(jum, jw[c], um[c]);
            A::acc_fma(jup, jw[c], up[c]);
            A::acc_fma(jdu, jw[c], A::sub(um[c], up[c]));
          }
          const V wgt = A::mul(A::mul(tb.w[q1], tb.w[q2]), tb.area[d]);
          const V lead = side > 0 ? A::add(A::half(unm), lam) : A::sub(A::half(unp), lam);
          const V extra = side > 0 ? A::add(A::half(A::acc_get_norm(jum)), A::scale_pow2(A::acc_get_norm(jdu), smx))
                                   : A::add(A::half(A::acc_get_norm(jup)), A::scale_pow2(A::acc_get_norm(jdu), spx));
#pragma unroll
          for (int e = 0; e < 3; ++e) {
            V g = A::mul(lead, jw[e]);
            if (e == d) g = A::add(g, extra);
            H[e * QQ + it] = A::mul(wgt, g);
          }
        }
      __syncthreads();
      if (active)
        for (int it = t; it < 3 * Q; it += NT) {
          const int c = it / Q, q1 = it - c * Q;
          Acc a[N];
#pragma unroll
          for (int q2 = 0; q2 < Q; ++q2) {
            const V h = H[c * QQ + q1 + Q * q2];
#pragma unroll
            for (int j = 0; j < N; ++j) {
              if (q2 == 0)
                A::acc_first(a[j], tb.S[j], h);
              else
                A::acc_fma(a[j], tb.S[q2 * N + j], h);
            }
          }
#pragma unroll
          for (int j2 = 0; j2 < N; ++j2) K1[c * Q * N + q1 + Q * j2] = A::acc_get_norm(a[j2]);
        }
      __syncthreads();
      if (active)
        for (int it = t; it < 3 * N; it += NT) {
          const int c = it / N, j2 = it - c * N;
          Acc a[N];
#pragma unroll
          for (int q1 = 0; q1 < Q; ++q1) {
            const V h = K1[c * Q * N + q1 + Q * j2];
#pragma unroll
            for (int j = 0; j < N; ++j) {
              if (q1 == 0)
                A::acc_first(a[j], tb.S[j], h);
              else
                A::acc_fma(a[j], tb.S[q1 * N + j], h);
            }
          }
#pragma unroll
          for (int j1 = 0; j1 < N; ++j1) {
            V& o = sOut[c * N3 + node3(N, d, aown, t1, j1, t2, j2)];
            o = A::add(o, A::acc_get_norm(a[j1]));
          }
        }
      __syncthreads();
    }
  }
  if (active)
    for (int c = 0; c < 3; ++c)
      for (int i = t; i < N3; i += NT) dst3[(c * m.E + el) * N3 + i] = A::store(sOut[c * N3 + i]);
}

template <class A, int N, int Q, bool PF = false>
int launch_conv_vjp(const MeshDims& m, const double* u3, const double* w3, double* dst3, const ConvHost& h,
                    cudaStream_t s) {
  VjpTab<typename A::V, N, Q> tb;
  for (int i = 0; i < Q * N; ++i) {
    tb.S[i] = A::make(h.S[i]);
    tb.D[i] = A::make(h.D[i]);
  }
  for (int q = 0; q < Q; ++q) tb.w[q] = A::make(h.w[q]);
  for (int d = 0; d < 3; ++d) {
    tb.jac[d] = A::make(h.h[0] * h.h[1] * h.h[2] / h.h[d]);
    tb.area[d] = tb.jac[d];
  }
  constexpr int EPB = conv_cells_per_block<N>();
  const size_t smem = (size_t)EPB * (PF ? VjpLayoutPF<N, Q>::PER : VjpLayout<N, Q>::PER) * sizeof(double);
  if (smem > 232448) return 7;
  if (cudaFuncSetAttribute(conv_vjp_kernel<A, N, Q, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return 2;
  if (m.E == 0) return 0;
  const long long blocks = (m.E + EPB - 1) / EPB;
  conv_vjp_kernel<A, N, Q, PF><<<(unsigned)blocks, EPB * N * N, smem, s>>>(u3, w3, dst3, tb, m);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // namespace
}  // namespace dgns
