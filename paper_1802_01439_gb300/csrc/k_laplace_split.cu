// The SIPG Laplace operator evaluated as separate cell and face kernels (Sec.
// 3.2: the cell integrals of grad q . grad p and the interior-face terms
// -{d_n q}[p] - [q]{d_n p} + tau [q][p]), native FP64: the operator-by-
// operator counterpart of the fused element-centric kernel (k_laplace.cu).
//
// 1. Cell term: the line kernel with the cell stiffness alone (no face
//    coupling), y = (K_x M M + M K_y M + M M K_z) x.
// 2. Face kernel: for every face (direction d, the cell e on its - side, the
//    cell e+ = e + d on its + side) and every line normal to it, the jump
//    J = u^-(1) - u^+(0) and the mean normal derivative
//    A = (u^-'(1) + u^+'(0)) / (2 h_d) of the two lines (u^- of cell e,
//    u^+ of cell e+); both are weighted by the tangential mass M (x) M over
//    the face's lines and by the face area h_t1 h_t2, and stored per face:
//    F[d][e] = (J^, A^), 2 N^2 numbers.
// 3. Face-apply kernel: every node (i along d, tangential index t) of cell e
//    adds, from the face on its + side (its own F[d][e]) and the face on its
//    - side (F[d][e-]),
//        -d1_i J^_r / (2 h_d) + [i = N-1] (tau J^_r - A^_r)
//        -d0_i J^_l / (2 h_d) + [i = 0]   (A^_l - tau J^_l)
//    with d0_i = phi_i'(0), d1_i = phi_i'(1): the test function's jump and
//    mean normal derivative at the face.
// The face kernel reads each cell three times (once per direction) and the
// apply kernel reads and writes y once more: about six times the memory
// traffic of the fused kernel, which is the comparison this path exists for.
#include "common.cuh"
#include "ops.h"

namespace dgns {
namespace {

template <int N>
struct SplitTab {
  double d0[N], d1[N];
  double M[N * N];
  double ih[3], tau[3], area[3];   // 1 / h_d, penalty, h_t1 h_t2
};

template <int N>
constexpr int faces_per_block() {
  return N * N >= 128 ? 1 : 128 / (N * N);
}

// Node index of position i along d and tangential (t1, t2) (the two other
// directions in increasing order).
template <int N>
__device__ __forceinline__ int node_of(int d, int i, int t1, int t2) {
  return d == 0 ? i + N * (t1 + N * t2) : (d == 1 ? t1 + N * (i + N * t2) : t1 + N * (t2 + N * i));
}

template <int N>
__global__ void __launch_bounds__(faces_per_block<N>() * N * N)
    sipg_face_kernel(const double* __restrict__ src, double* __restrict__ fb, const __grid_constant__ SplitTab<N> tb,
                     const MeshDims m, const long long ncells) {
  constexpr int NN = N * N, FPB = faces_per_block<N>(), N3 = NN * N;
  __shared__ double sJ[FPB][NN], sA[FPB][NN], tJ[FPB][NN], tA[FPB][NN];
  const int slot = threadIdx.x / NN, t = threadIdx.x - slot * NN;
  const int t1 = t % N, t2 = t / N;
  const long long face = (long long)blockIdx.x * FPB + slot;   // d * ncells + cell
  const bool active = face < 3 * ncells;
  int d = 0;
  if (active) {
    d = (int)(face / ncells);
    const long long cell = face - (long long)d * ncells;
    const CellXYZ cx = cell_xyz((unsigned)cell, m);
    const long long cfirst = (long long)cx.comp * m.E;
    const unsigned nb = d == 0 ? neighbor32<0>(cx, +1, m) : (d == 1 ? neighbor32<1>(cx, +1, m) : neighbor32<2>(cx, +1, m));
    const double* a = src + (size_t)cell * N3;
    const double* b = src + (size_t)(cfirst + nb) * N3;
    double da = 0.0, db = 0.0, am = 0.0, bp = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const double ai = __ldg(a + node_of<N>(d, i, t1, t2)), bi = __ldg(b + node_of<N>(d, i, t1, t2));
      da = fma(tb.d1[i], ai, da);
      db = fma(tb.d0[i], bi, db);
      if (i == N - 1) am = ai;
      if (i == 0) bp = bi;
    }
    sJ[slot][t] = am - bp;
    sA[slot][t] = 0.5 * tb.ih[d] * (da + db);
  }
  __syncthreads();
  // tangential mass M (x) M: along t1, then along t2
  if (active) {
    double j = 0.0, aa = 0.0;
#pragma unroll
    for (int s = 0; s < N; ++s) {
      j = fma(tb.M[t1 * N + s], sJ[slot][s + N * t2], j);
      aa = fma(tb.M[t1 * N + s], sA[slot][s + N * t2], aa);
    }
    tJ[slot][t] = j;
    tA[slot][t] = aa;
  }
  __syncthreads();
  if (active) {
    double j = 0.0, aa = 0.0;
#pragma unroll
    for (int s = 0; s < N; ++s) {
      j = fma(tb.M[t2 * N + s], tJ[slot][t1 + N * s], j);
      aa = fma(tb.M[t2 * N + s], tA[slot][t1 + N * s], aa);
    }
    double* f = fb + (size_t)face * 2 * NN;
    f[t] = tb.area[d] * j;
    f[NN + t] = tb.area[d] * aa;
  }
}

constexpr int APPLY_THREADS = 256;

// One thread per node of every cell.
template <int N>
__global__ void __launch_bounds__(APPLY_THREADS)
    sipg_face_apply_kernel(const double* __restrict__ fb, double* __restrict__ dst,
                           const __grid_constant__ SplitTab<N> tb, const MeshDims m, const long long ncells) {
  constexpr int NN = N * N, N3 = NN * N;
  const long long id = (long long)blockIdx.x * APPLY_THREADS + threadIdx.x;
  if (id >= ncells * N3) return;
  const long long cell = id / N3;
  const int node = (int)(id - cell * N3);
  const int x = node % N, y = (node / N) % N, z = node / NN;
  const CellXYZ cx = cell_xyz((unsigned)cell, m);
  const long long cfirst = (long long)cx.comp * m.E;
  double v = dst[id];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int i = d == 0 ? x : (d == 1 ? y : z);
    const int t = d == 0 ? y + N * z : (d == 1 ? x + N * z : x + N * y);
    const unsigned em = d == 0 ? neighbor32<0>(cx, -1, m) : (d == 1 ? neighbor32<1>(cx, -1, m) : neighbor32<2>(cx, -1, m));
    const double* fr = fb + ((size_t)d * ncells + cell) * 2 * NN;
    const double* fl = fb + ((size_t)d * ncells + cfirst + em) * 2 * NN;
    const double jr = __ldg(fr + t), ar = __ldg(fr + NN + t);
    const double jl = __ldg(fl + t), al = __ldg(fl + NN + t);
    const double hh = -0.5 * tb.ih[d];
    v = fma(hh * tb.d1[i], jr, v);
    v = fma(hh * tb.d0[i], jl, v);
    if (i == N - 1) v += tb.tau[d] * jr - ar;
    if (i == 0) v += al - tb.tau[d] * jl;
  }
  dst[id] = v;
}

template <int N>
int launch_split(const MeshDims& m, int ncomp, const double* src, double* fbuf, double* dst, const SplitHost& h,
                 cudaStream_t s) {
  SplitTab<N> tb;
  for (int i = 0; i < N; ++i) {
    tb.d0[i] = h.d0[i];
    tb.d1[i] = h.d1[i];
  }
  for (int i = 0; i < N * N; ++i) tb.M[i] = h.M[i];
  for (int d = 0; d < 3; ++d) {
    tb.ih[d] = h.ih[d];
    tb.tau[d] = h.tau[d];
    tb.area[d] = h.area[d];
  }
  const long long ncells = m.E * ncomp;
  if (ncells == 0) return 0;
  constexpr int FPB = faces_per_block<N>();
  sipg_face_kernel<N><<<(unsigned)((3 * ncells + FPB - 1) / FPB), FPB * N * N, 0, s>>>(src, fbuf, tb, m, ncells);
  if (cudaGetLastError() != cudaSuccess) return 2;
  const long long nodes = ncells * N * N * N;
  sipg_face_apply_kernel<N><<<(unsigned)((nodes + APPLY_THREADS - 1) / APPLY_THREADS), APPLY_THREADS, 0, s>>>(
      fbuf, dst, tb, m, ncells);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // namespace

int laplace_faces_apply(const MeshDims& m, int ncomp, const double* src, double* fbuf, double* dst,
                        const SplitHost& h, cudaStream_t s) {
  switch (h.N) {
    case 2: return launch_split<2>(m, ncomp, src, fbuf, dst, h, s);
    case 3: return launch_split<3>(m, ncomp, src, fbuf, dst, h, s);
    case 4: return launch_split<4>(m, ncomp, src, fbuf, dst, h, s);
    case 5: return launch_split<5>(m, ncomp, src, fbuf, dst, h, s);
    case 6: return launch_split<6>(m, ncomp, src, fbuf, dst, h, s);
    case 7: return launch_split<7>(m, ncomp, src, fbuf, dst, h, s);
    case 8: return launch_split<8>(m, ncomp, src, fbuf, dst, h, s);
    case 9: return launch_split<9>(m, ncomp, src, fbuf, dst, h, s);
    case 10: return launch_split<10>(m, ncomp, src, fbuf, dst, h, s);
    case 11: return launch_split<11>(m, ncomp, src, fbuf, dst, h, s);
    case 12: return launch_split<12>(m, ncomp, src, fbuf, dst, h, s);
  }
  return 7;
}

}  // namespace dgns
