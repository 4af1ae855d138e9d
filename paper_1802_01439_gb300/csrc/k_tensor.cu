// Cell-local tensor-product kernels: mass matrix and its exact inverse
// (Secs. 3.2 and 3.3 of arXiv:1802.01439; on an affine Cartesian cell the
// element mass matrix is h_x h_y h_z Mhat (x) Mhat (x) Mhat and its inverse
// the Kronecker product of the 1D inverses, three sweeps per cell), and the
// h-multigrid transfers (embedding of a coarse cell polynomial into its eight
// children and the transpose).
#include <algorithm>
#include <cmath>

#include "arith.cuh"
#include "ops.h"

namespace dgns {
namespace {

template <int N>
constexpr int tcells_per_block() {
  return N * N >= 128 ? 1 : 128 / (N * N);
}

template <class V, int N>
struct Tens3 {
  V Mx[N * N], My[N * N], Mz[N * N];
  // even-odd forms of the three matrices (double-float sweeps of
  // centrosymmetric matrices, C(N-1-i, N-1-j) = C(i, j), as the 1D mass
  // matrix and its inverse on the symmetric LGL nodes): with
  // xe(j) = x(j) + x(N-1-j) (x(j) at the middle of odd N) and
  // xo(j) = x(j) - x(N-1-j), e = E xe and o = O xo give y(i) = e(i) + o(i),
  // y(N-1-i) = e(i) - o(i), y(middle) = e(middle), with
  // E(i,j) = (C(i,j) + C(i,N-1-j)) / 2 (C(i,middle) in the middle column) and
  // O(i,j) = (C(i,j) - C(i,N-1-j)) / 2
  V E[3][((N + 1) / 2) * ((N + 1) / 2)];
  V O[3][(N / 2) * (N / 2)];
};

template <class T, int N, int D>
__device__ __forceinline__ void sweep_line(const T* in, T* out, int l, const T* A) {
  int base, stride;
  line_geom<D>(l, N, N, N, base, stride);
  T x[N], y[N];
  load_line<T, N>(in, base, stride, x);
  matvec<T, N, N>(A, x, y);
  store_line<T, N>(out, base, stride, y);
}

template <class A, int N, int D>
__device__ __forceinline__ void sweep_line_p(const typename A::V* in, typename A::V* out, int l,
                                             const typename A::V* M) {
  typedef typename A::V V;
  typedef typename A::Acc Acc;
  int base, stride;
  line_geom<D>(l, N, N, N, base, stride);
  V x[N];
  load_line<V, N>(in, base, stride, x);
  Acc y[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    A::acc_first(y[i], M[i * N], x[0]);
#pragma unroll
    for (int j = 1; j < N; ++j) A::acc_fma(y[i], M[i * N + j], x[j]);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) out[base + i * stride] = A::acc_get(y[i]);
}

template <class A, int N, int D>
__device__ __forceinline__ void sweep_line_eo(const typename A::V* in, typename A::V* out, int l,
                                              const typename A::V* E, const typename A::V* O) {
  typedef typename A::V V;
  typedef typename A::Acc Acc;
  constexpr int NH = (N + 1) / 2, NF = N / 2;
  int base, stride;
  line_geom<D>(l, N, N, N, base, stride);
  V x[N], xe[NH], xo[NF];
  load_line<V, N>(in, base, stride, x);
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    xe[j] = A::add_nr(x[j], x[N - 1 - j]);
    xo[j] = A::sub_nr(x[j], x[N - 1 - j]);
  }
  if (N % 2 == 1) xe[NF] = x[NF];
#pragma unroll
  for (int i = 0; i < NH; ++i) {
    Acc e;
    A::acc_first(e, E[i * NH], xe[0]);
#pragma unroll
    for (int j = 1; j < NH; ++j) A::acc_fma(e, E[i * NH + j], xe[j]);
    if (i < NF) {
      Acc o;
      A::acc_first(o, O[i * NF], xo[0]);
#pragma unroll
      for (int j = 1; j < NF; ++j) A::acc_fma(o, O[i * NF + j], xo[j]);
      const V a = A::acc_get(e), b = A::acc_get(o);
      out[base + i * stride] = A::add_nr(a, b);
      out[base + (N - 1 - i) * stride] = A::sub_nr(a, b);
    } else {
      out[base + i * stride] = A::acc_get(e);
    }
  }
}

// EO: the sweeps in even-odd form (double-float arithmetic, centrosymmetric
// matrices); natively an addition costs as much as a multiply-add.
template <class A, int N, bool EO>
__global__ void __launch_bounds__(tcells_per_block<N>() * N * N)
    tensor3_kernel(const typename A::G* __restrict__ src, typename A::G* __restrict__ dst,
                   const __grid_constant__ Tens3<typename A::V, N> tb, const long long ncells) {
  typedef typename A::V V;
  constexpr int NN = N * N, NNN = NN * N, EPB = tcells_per_block<N>();
  V* sX = reinterpret_cast<V*>(dyn_smem());
  V* sA = sX + EPB * NNN;
  const int slot = threadIdx.x / NN;
  const int l = threadIdx.x - slot * NN;
  const long long c0 = (long long)blockIdx.x * EPB;
  const long long rem = ncells - c0;
  const int nvalid = rem < EPB ? (int)rem : EPB;
  for (int i = threadIdx.x; i < nvalid * NNN; i += blockDim.x) sX[i] = A::load(src + c0 * NNN + i);
  __syncthreads();
  const bool active = slot < nvalid;
  const int off = slot * NNN;
  if constexpr (EO) {
    if (active) sweep_line_eo<A, N, 0>(sX + off, sA + off, l, tb.E[0], tb.O[0]);
    __syncthreads();
    if (active) sweep_line_eo<A, N, 1>(sA + off, sA + off, l, tb.E[1], tb.O[1]);
    __syncthreads();
    if (active) sweep_line_eo<A, N, 2>(sA + off, sX + off, l, tb.E[2], tb.O[2]);
  } else {
    if (active) sweep_line_p<A, N, 0>(sX + off, sA + off, l, tb.Mx);
    __syncthreads();
    if (active) sweep_line_p<A, N, 1>(sA + off, sA + off, l, tb.My);
    __syncthreads();
    if (active) sweep_line_p<A, N, 2>(sA + off, sX + off, l, tb.Mz);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nvalid * NNN; i += blockDim.x) dst[c0 * NNN + i] = A::store(sX[i]);
}

template <class A, int N>
int launch_tensor3(long long ncells, const double* src, double* dst, const double* Mx, const double* My,
                   const double* Mz, cudaStream_t s) {
  constexpr int NN = N * N, EPB = tcells_per_block<N>(), NH = (N + 1) / 2, NF = N / 2;
  Tens3<typename A::V, N> tb;
  for (int i = 0; i < NN; ++i) {
    tb.Mx[i] = A::make(Mx[i]);
    tb.My[i] = A::make(My[i]);
    tb.Mz[i] = A::make(Mz[i]);
  }
  // even-odd sweeps for double-float arithmetic when all three matrices are
  // centrosymmetric (to 1e-14 of their largest entry)
  bool eo = A::emulated;
  const double* Ms[3] = {Mx, My, Mz};
  for (int d = 0; d < 3 && eo; ++d) {
    double mx = 0.0, dev = 0.0;
    for (int i = 0; i < NN; ++i) {
      mx = std::max(mx, std::fabs(Ms[d][i]));
      dev = std::max(dev, std::fabs(Ms[d][i] - Ms[d][NN - 1 - i]));   // C(N-1-i, N-1-j) is entry NN-1-(iN+j)
    }
    if (dev > 1e-14 * mx) eo = false;
  }
  for (int d = 0; d < 3; ++d) {
    const double* C = Ms[d];
    for (int i = 0; i < NH; ++i)
      for (int j = 0; j < NH; ++j)
        tb.E[d][i * NH + j] = A::make(j < NF ? 0.5 * (C[i * N + j] + C[i * N + N - 1 - j]) : C[i * N + j]);
    for (int i = 0; i < NF; ++i)
      for (int j = 0; j < NF; ++j) tb.O[d][i * NF + j] = A::make(0.5 * (C[i * N + j] - C[i * N + N - 1 - j]));
  }
  if (ncells == 0) return 0;
  const size_t smem = (size_t)2 * EPB * NN * N * sizeof(typename A::V);
  static bool attr_done = false;
  if (!attr_done) {
    if (cudaFuncSetAttribute(tensor3_kernel<A, N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(tensor3_kernel<A, N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return 2;
    attr_done = true;
  }
  const long long blocks = (ncells + EPB - 1) / EPB;
  if (eo)
    tensor3_kernel<A, N, true><<<(unsigned)blocks, EPB * NN, smem, s>>>(src, dst, tb, ncells);
  else
    tensor3_kernel<A, N, false><<<(unsigned)blocks, EPB * NN, smem, s>>>(src, dst, tb, ncells);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// ---------------------------------------------------------------- transfers
template <class T, int N>
struct Prol {
  T P[2][N * N];  // P[c][i*N+j] = phi_j((xi_i + c)/2)
};

// Transfers per coarse cell with the 1D operators factored across the eight
// children (prolongation: x-sweep into the two x-halves, y-sweep into four,
// z-sweep into the eight children, written straight to the fine vector;
// restriction in the reverse order): 14 N^4 multiply-adds per coarse cell
// instead of 24 N^4, every coarse value read or written once.  Threads per
// coarse cell: N^3 (N <= 5) or N^2; the 1D tables sit in shared memory
// (items of a warp index them by different output nodes).
template <int N>
constexpr int xfer_threads() {
  return N * N * N <= 128 ? N * N * N : N * N;
}
template <int N>
constexpr int xfer_cells_per_block() {
  return xfer_threads<N>() >= 256 ? 1 : 256 / xfer_threads<N>();
}

template <class T, int N, bool ADD>
__global__ void __launch_bounds__(xfer_cells_per_block<N>() * xfer_threads<N>())
    prolong_cell_kernel(const T* __restrict__ coarse, T* __restrict__ fine, const __grid_constant__ Prol<T, N> tb,
                        const MeshDims mc, const long long ncoarse) {
  constexpr int NN = N * N, N3 = NN * N, TPC = xfer_threads<N>(), CPB = xfer_cells_per_block<N>();
  T* sP = reinterpret_cast<T*>(dyn_smem());   // P[c][j N + i], 2 N^2
  T* sm = sP + 2 * NN;
  const int slot = threadIdx.x / TPC, t = threadIdx.x - slot * TPC;
  const long long c = (long long)blockIdx.x * CPB + slot;
  const bool active = c < ncoarse;
  T* sC = sm + slot * 7 * N3;   // coarse cell [z][y][x]
  T* sA = sC + N3;              // [cx][z][y][x]
  T* sB = sA + 2 * N3;          // [cx + 2 cy][z][y][x]
  for (int i = threadIdx.x; i < 2 * NN; i += blockDim.x) sP[i] = tb.P[i / NN][i % NN];
  if (active)
    for (int i = t; i < N3; i += TPC) sC[i] = coarse[c * N3 + i];
  __syncthreads();
  if (active)
    for (int it = t; it < 2 * N3; it += TPC) {
      const int cx = it / N3, r = it - cx * N3, j = r % N, line = r / N;
      const T* P = sP + cx * NN + j * N;
      T a = P[0] * sC[line * N];
#pragma unroll
      for (int i = 1; i < N; ++i) a = fma(P[i], sC[line * N + i], a);
      sA[it] = a;
    }
  __syncthreads();
  if (active)
    for (int it = t; it < 4 * N3; it += TPC) {
      const int q = it / N3, r = it - q * N3;
      const int cx = q & 1, cy = q >> 1;
      const int x = r % N, j = (r / N) % N, z = r / NN;
      const T* P = sP + cy * NN + j * N;
      const T* src = sA + cx * N3 + x + NN * z;
      T a = P[0] * src[0];
#pragma unroll
      for (int i = 1; i < N; ++i) a = fma(P[i], src[N * i], a);
      sB[it] = a;
    }
  __syncthreads();
  if (active) {
    const unsigned cu = (unsigned)c, nxu = (unsigned)mc.nx, nyu = (unsigned)mc.ny;
    const int ci = (int)(cu % nxu);
    const unsigned tt = cu / nxu;
    const int cj = (int)(tt % nyu), ck = (int)(tt / nyu);
    const long long nfx = 2 * mc.nx, nfy = 2 * mc.ny;
    for (int it = t; it < 8 * N3; it += TPC) {
      const int ch = it / N3, r = it - ch * N3;
      const int cx = ch & 1, cy = (ch >> 1) & 1, cz = ch >> 2;
      const int xy = r % NN, j = r / NN;
      const T* P = sP + cz * NN + j * N;
      const T* src = sB + (cx + 2 * cy) * N3 + xy;
      T a = P[0] * src[0];
#pragma unroll
      for (int i = 1; i < N; ++i) a = fma(P[i], src[NN * i], a);
      const long long f = (2 * ci + cx) + nfx * ((2 * cj + cy) + nfy * (2 * ck + cz));
      if (ADD)
        fine[f * N3 + r] += a;
      else
        fine[f * N3 + r] = a;
    }
  }
}

template <class T, int N>
__global__ void __launch_bounds__(xfer_cells_per_block<N>() * xfer_threads<N>())
    restrict_cell_kernel(const T* __restrict__ fine, T* __restrict__ coarse, const __grid_constant__ Prol<T, N> tb,
                         const MeshDims mc, const long long ncoarse) {
  constexpr int NN = N * N, N3 = NN * N, TPC = xfer_threads<N>(), CPB = xfer_cells_per_block<N>();
  T* sP = reinterpret_cast<T*>(dyn_smem());
  T* sm = sP + 2 * NN;
  const int slot = threadIdx.x / TPC, t = threadIdx.x - slot * TPC;
  const long long c = (long long)blockIdx.x * CPB + slot;
  const bool active = c < ncoarse;
  T* sC = sm + slot * 14 * N3;   // children [cx + 2 cy + 4 cz][z][y][x]
  T* sB = sC + 8 * N3;           // [cx + 2 cy][z'][y][x]
  T* sA = sB + 4 * N3;           // [cx][z'][y'][x]
  for (int i = threadIdx.x; i < 2 * NN; i += blockDim.x) sP[i] = tb.P[i / NN][i % NN];
  if (active) {
    const unsigned cu = (unsigned)c, nxu = (unsigned)mc.nx, nyu = (unsigned)mc.ny;
    const int ci = (int)(cu % nxu);
    const unsigned tt = cu / nxu;
    const int cj = (int)(tt % nyu), ck = (int)(tt / nyu);
    const long long nfx = 2 * mc.nx, nfy = 2 * mc.ny;
    for (int it = t; it < 8 * N3; it += TPC) {
      const int ch = it / N3, r = it - ch * N3;
      const int cx = ch & 1, cy = (ch >> 1) & 1, cz = ch >> 2;
      const long long f = (2 * ci + cx) + nfx * ((2 * cj + cy) + nfy * (2 * ck + cz));
      sC[it] = fine[f * N3 + r];
    }
  }
  __syncthreads();
  // z: B[q][j][y][x] = sum_cz sum_i P[cz][i][j] C[q + 4 cz][i][y][x]
  if (active)
    for (int it = t; it < 4 * N3; it += TPC) {
      const int q = it / N3, r = it - q * N3;
      const int xy = r % NN, j = r / NN;
      T a = (T)0;
#pragma unroll
      for (int cz = 0; cz < 2; ++cz) {
        const T* src = sC + (q + 4 * cz) * N3 + xy;
#pragma unroll
        for (int i = 0; i < N; ++i) a = fma(sP[cz * NN + i * N + j], src[NN * i], a);
      }
      sB[it] = a;
    }
  __syncthreads();
  // y: A[cx][z][j][x] = sum_cy sum_i P[cy][i][j] B[cx + 2 cy][z][i][x]
  if (active)
    for (int it = t; it < 2 * N3; it += TPC) {
      const int cx = it / N3, r = it - cx * N3;
      const int x = r % N, j = (r / N) % N, z = r / NN;
      T a = (T)0;
#pragma unroll
      for (int cy = 0; cy < 2; ++cy) {
        const T* src = sB + (cx + 2 * cy) * N3 + x + NN * z;
#pragma unroll
        for (int i = 0; i < N; ++i) a = fma(sP[cy * NN + i * N + j], src[N * i], a);
      }
      sA[it] = a;
    }
  __syncthreads();
  // x: coarse[z][y][j] = sum_cx sum_i P[cx][i][j] A[cx][z][y][i]
  if (active)
    for (int r = t; r < N3; r += TPC) {
      const int j = r % N, line = r / N;
      T a = (T)0;
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        const T* src = sA + cx * N3 + line * N;
#pragma unroll
        for (int i = 0; i < N; ++i) a = fma(sP[cx * NN + i * N + j], src[i], a);
      }
      coarse[c * N3 + r] = a;
    }
}

template <class T, int N>
Prol<T, N> make_prol(const double* P0, const double* P1) {
  Prol<T, N> tb;
  for (int i = 0; i < N * N; ++i) {
    tb.P[0][i] = (T)P0[i];
    tb.P[1][i] = (T)P1[i];
  }
  return tb;
}

template <class T, int N>
int launch_prolong(const MeshDims& mc, const T* coarse, T* fine, const double* P0,
                   const double* P1, bool add, cudaStream_t s) {
  constexpr int TPC = xfer_threads<N>(), CPB = xfer_cells_per_block<N>();
  if (mc.E == 0) return 0;
  const size_t smem = (size_t)(2 * N * N + CPB * 7 * N * N * N) * sizeof(T);
  auto kern = add ? prolong_cell_kernel<T, N, true> : prolong_cell_kernel<T, N, false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 2;
  const long long blocks = (mc.E + CPB - 1) / CPB;
  kern<<<(unsigned)blocks, CPB * TPC, smem, s>>>(coarse, fine, make_prol<T, N>(P0, P1), mc, mc.E);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

template <class T, int N>
int launch_restrict(const MeshDims& mc, const T* fine, T* coarse, const double* P0,
                    const double* P1, cudaStream_t s) {
  constexpr int TPC = xfer_threads<N>(), CPB = xfer_cells_per_block<N>();
  if (mc.E == 0) return 0;
  const size_t smem = (size_t)(2 * N * N + CPB * 14 * N * N * N) * sizeof(T);
  if (smem > 232448) return 7;
  if (cudaFuncSetAttribute(restrict_cell_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return 2;
  const long long blocks = (mc.E + CPB - 1) / CPB;
  restrict_cell_kernel<T, N><<<(unsigned)blocks, CPB * TPC, smem, s>>>(fine, coarse, make_prol<T, N>(P0, P1), mc,
                                                                     mc.E);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // namespace

#define DGNS_SWITCH_N(NVAR, ...) \
  switch (NVAR) {                 \
    case 2: { constexpr int NC = 2; __VA_ARGS__; } \
    case 3: { constexpr int NC = 3; __VA_ARGS__; } \
    case 4: { constexpr int NC = 4; __VA_ARGS__; } \
    case 5: { constexpr int NC = 5; __VA_ARGS__; } \
    case 6: { constexpr int NC = 6; __VA_ARGS__; } \
    case 7: { constexpr int NC = 7; __VA_ARGS__; } \
    case 8: { constexpr int NC = 8; __VA_ARGS__; } \
    case 9: { constexpr int NC = 9; __VA_ARGS__; } \
    case 10: { constexpr int NC = 10; __VA_ARGS__; } \
    case 11: { constexpr int NC = 11; __VA_ARGS__; } \
    case 12: { constexpr int NC = 12; __VA_ARGS__; } \
  }

int tensor3_apply(int N, long long ncells, const double* src, double* dst, const double* Mx,
                  const double* My, const double* Mz, cudaStream_t s, int arith) {
  DGNS_SWITCH_N(N, return arith == ARITH_DF64   ? launch_tensor3<DF64, NC>(ncells, src, dst, Mx, My, Mz, s)
                          : arith == ARITH_TF64 ? launch_tensor3<TF64, NC>(ncells, src, dst, Mx, My, Mz, s)
                                                : launch_tensor3<F64, NC>(ncells, src, dst, Mx, My, Mz, s))
  return 7;
}

int prolongate(bool fp32, int N, const MeshDims& mc, const void* coarse, void* fine,
               const double* P0, const double* P1, bool add, cudaStream_t s) {
  DGNS_SWITCH_N(N, return fp32 ? launch_prolong<float, NC>(mc, (const float*)coarse, (float*)fine, P0, P1, add, s)
                               : launch_prolong<double, NC>(mc, (const double*)coarse, (double*)fine, P0, P1, add, s))
  return 7;
}

int restrict_fine(bool fp32, int N, const MeshDims& mc, const void* fine, void* coarse,
                  const double* P0, const double* P1, cudaStream_t s) {
  DGNS_SWITCH_N(N, return fp32 ? launch_restrict<float, NC>(mc, (const float*)fine, (float*)coarse, P0, P1, s)
                               : launch_restrict<double, NC>(mc, (const double*)fine, (double*)coarse, P0, P1, s))
  return 7;
}

}  // namespace dgns
