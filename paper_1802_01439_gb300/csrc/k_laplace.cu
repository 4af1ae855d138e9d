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
#include "ops.h"

namespace dgns {
namespace {

template <class T, int N>
struct LapTab {
  T A0[3][N * N];
  T M[N * N];
  T cr[3][N], cl[3][N], gr[3][N], gl[3][N];
};

template <class T>
struct EpiArgs {
  const T* b;
  const T* xprev;
  const T* dinv;
  T c1, c2;
};

template <int N>
constexpr int cells_per_block() {
  return N * N >= 128 ? 1 : 128 / (N * N);
}

// One line of T_d x for the own cell, with the neighbour terms.
template <class T, int N, int D>
__device__ __forceinline__ void sipg_line(const T* X, T* out, const T* __restrict__ nbR,
                                          const T* __restrict__ nbL, int l,
                                          const LapTab<T, N>& tb) {
  int base, stride;
  line_geom<D>(l, N, N, N, base, stride);
  T x[N], r[N], lf[N], y[N];
  load_line<T, N>(X, base, stride, x);
#pragma unroll
  for (int j = 0; j < N; ++j) {
    r[j] = __ldg(nbR + base + j * stride);
    lf[j] = __ldg(nbL + base + j * stride);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T acc = tb.cr[D][i] * r[0];
    acc = fma(tb.cl[D][i], lf[N - 1], acc);
#pragma unroll
    for (int j = 0; j < N; ++j) acc = fma(tb.A0[D][i * N + j], x[j], acc);
    y[i] = acc;
  }
#pragma unroll
  for (int j = 0; j < N; ++j) {
    y[N - 1] = fma(tb.gr[D][j], r[j], y[N - 1]);
    y[0] = fma(tb.gl[D][j], lf[j], y[0]);
  }
  store_line<T, N>(out, base, stride, y);
}

// One line of out = M_d in (+ add).
template <class T, int N, int D, bool ADD>
__device__ __forceinline__ void mass_line(const T* in, const T* add, T* out, int l, const T* M) {
  int base, stride;
  line_geom<D>(l, N, N, N, base, stride);
  T x[N], y[N];
  load_line<T, N>(in, base, stride, x);
  if (ADD) {
    T z[N];
    load_line<T, N>(add, base, stride, z);
    matvec_add<T, N, N>(M, x, z, y);
  } else {
    matvec<T, N, N>(M, x, y);
  }
  store_line<T, N>(out, base, stride, y);
}

template <class T, int N, int EPI>
__global__ void __launch_bounds__(cells_per_block<N>() * N * N)
    sipg_kernel(const T* __restrict__ src, T* __restrict__ dst, const __grid_constant__ LapTab<T, N> tb,
                const MeshDims m, const long long ncells, const EpiArgs<T> ea) {
  constexpr int NN = N * N, NNN = NN * N, EPB = cells_per_block<N>();
  T* sX = reinterpret_cast<T*>(dyn_smem());
  T* sA = sX + EPB * NNN;
  T* sB = sA + EPB * NNN;
  T* sC = sB + EPB * NNN;
  const int slot = threadIdx.x / NN;
  const int l = threadIdx.x - slot * NN;
  const long long c0 = (long long)blockIdx.x * EPB;
  const long long rem = ncells - c0;
  const int nvalid = rem < EPB ? (int)rem : EPB;
  const T* gsrc = src + c0 * NNN;
  for (int i = threadIdx.x; i < nvalid * NNN; i += blockDim.x) sX[i] = gsrc[i];
  __syncthreads();
  const bool active = slot < nvalid;
  const int off = slot * NNN;
  if (active) {
    const long long cell = c0 + slot;
    const long long comp = cell / m.E;
    const long long el = cell - comp * m.E;
    const int ex = (int)(el % m.nx);
    const long long t = el / m.nx;
    const int ey = (int)(t % m.ny);
    const int ez = (int)(t / m.ny);
    const T* cb = src + comp * m.E * NNN;
    sipg_line<T, N, 0>(sX + off, sA + off, cb + neighbor<0>(el, ex, ey, ez, +1, m) * NNN,
                       cb + neighbor<0>(el, ex, ey, ez, -1, m) * NNN, l, tb);
    sipg_line<T, N, 1>(sX + off, sB + off, cb + neighbor<1>(el, ex, ey, ez, +1, m) * NNN,
                       cb + neighbor<1>(el, ex, ey, ez, -1, m) * NNN, l, tb);
    sipg_line<T, N, 2>(sX + off, sC + off, cb + neighbor<2>(el, ex, ey, ez, +1, m) * NNN,
                       cb + neighbor<2>(el, ex, ey, ez, -1, m) * NNN, l, tb);
  }
  __syncthreads();
  if (active) {
    mass_line<T, N, 0, false>(sB + off, nullptr, sB + off, l, tb.M);  // M_x T_y x
    mass_line<T, N, 1, false>(sC + off, nullptr, sC + off, l, tb.M);  // M_y T_z x
  }
  __syncthreads();
  if (active) {
    mass_line<T, N, 1, true>(sA + off, sB + off, sA + off, l, tb.M);  // M_y T_x x + M_x T_y x
    mass_line<T, N, 0, false>(sC + off, nullptr, sC + off, l, tb.M);  // M_x M_y T_z x
  }
  __syncthreads();
  if (active) mass_line<T, N, 2, true>(sA + off, sC + off, sB + off, l, tb.M);
  __syncthreads();
  T* gdst = dst + c0 * NNN;
  for (int i = threadIdx.x; i < nvalid * NNN; i += blockDim.x) {
    const T y = sB[i];
    if (EPI == EPI_NONE) {
      gdst[i] = y;
    } else if (EPI == EPI_RESID) {
      gdst[i] = ea.b[c0 * NNN + i] - y;
    } else {
      const T x = sX[i];
      const T r = ea.b[c0 * NNN + i] - y;
      T v = fma(ea.c2 * ea.dinv[i % NNN], r, x);
      // x_{k+1} = x_k + c1 (x_k - x_{k-1}) + c2 D^-1 (b - A x_k); a null
      // xprev stands for a zero previous iterate
      if (ea.c1 != (T)0) v = fma(ea.c1, x - (ea.xprev ? ea.xprev[c0 * NNN + i] : (T)0), v);
      gdst[i] = v;
    }
  }
}

template <class T, int N, int EPI>
int launch_sipg(const MeshDims& m, int ncomp, const T* src, T* dst, const LapHost& h,
                const EpiHost& eh, cudaStream_t s) {
  constexpr int NN = N * N, EPB = cells_per_block<N>();
  LapTab<T, N> tb;
  for (int d = 0; d < 3; ++d) {
    for (int i = 0; i < NN; ++i) tb.A0[d][i] = (T)h.A0[d][i];
    for (int i = 0; i < N; ++i) {
      tb.cr[d][i] = (T)h.cr[d][i];
      tb.cl[d][i] = (T)h.cl[d][i];
      tb.gr[d][i] = (T)h.gr[d][i];
      tb.gl[d][i] = (T)h.gl[d][i];
    }
  }
  for (int i = 0; i < NN; ++i) tb.M[i] = (T)h.M[i];
  EpiArgs<T> ea{(const T*)eh.b, (const T*)eh.xprev, (const T*)eh.dinv, (T)eh.c1, (T)eh.c2};
  const long long ncells = m.E * ncomp;
  if (ncells == 0) return 0;
  const long long blocks = (ncells + EPB - 1) / EPB;
  const size_t smem = (size_t)4 * EPB * NN * N * sizeof(T);
  static bool attr_done = false;
  if (!attr_done) {
    if (cudaFuncSetAttribute(sipg_kernel<T, N, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return 2;
    attr_done = true;
  }
  sipg_kernel<T, N, EPI><<<(unsigned)blocks, EPB * NN, smem, s>>>(src, dst, tb, m, ncells, ea);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

template <class T, int N>
int launch_sipg_epi(const MeshDims& m, int ncomp, const void* src, void* dst, const LapHost& h,
                    int epi, const EpiHost& eh, cudaStream_t s) {
  switch (epi) {
    case EPI_NONE: return launch_sipg<T, N, EPI_NONE>(m, ncomp, (const T*)src, (T*)dst, h, eh, s);
    case EPI_RESID: return launch_sipg<T, N, EPI_RESID>(m, ncomp, (const T*)src, (T*)dst, h, eh, s);
    case EPI_CHEB: return launch_sipg<T, N, EPI_CHEB>(m, ncomp, (const T*)src, (T*)dst, h, eh, s);
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
                  const LapHost& tab, int epi, const EpiHost& ea, cudaStream_t s) {
#define DGNS_CASE(NV)                                                                  \
  case NV:                                                                             \
    return fp32 ? launch_sipg_epi<float, NV>(m, ncomp, src, dst, tab, epi, ea, s)      \
                : launch_sipg_epi<double, NV>(m, ncomp, src, dst, tab, epi, ea, s);
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
