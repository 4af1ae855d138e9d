// FP32 SIPG Laplace operator on cells of N = 4 nodes per direction: the
// multigrid level operator of the pressure Poisson solve at k_p = 3 (Secs. 3.2
// and 3.3 of arXiv:1802.01439), with the fused residual and Chebyshev
// epilogues.
//
// Same Kronecker factorisation as the line kernel (k_laplace.cu),
//     y = M_z [ M_y T_x x + M_x T_y x ] + M_x M_y T_z x,
// on a different mapping: one thread per z-plane of a cell, the 4 threads of a
// cell on adjacent lanes of one warp (arithmetic in k_plane_core.cuh).  A
// thread holds its 4 x 4 plane in registers, so the x- and y-sweeps exchange
// no data; the z-direction is a reduce-scatter across the 4 lanes of a cell by
// warp shuffles.  A warp holds 8 consecutive cells: a cell whose x-neighbour
// is in the same warp takes that neighbour's face data by shuffle, the others
// (and every y- and z-neighbour) read plane z of the neighbour, 64 contiguous
// bytes, with two 256-bit loads.  The epilogue's b and previous iterate are
// prefetched into L1 at the start.  No shared memory.
//
// laplace_plane_f32 picks this kernel, or the one staging its data with
// tensor copies (k_laplace_tma.cu), per the variant set by
// laplace_plane_set_variant.
#include <atomic>
#include <cstdint>

#include "k_plane_core.cuh"

namespace dgns {
namespace {

using plane::Epi;
using plane::Tab;
using plane::Tab2;
using plane::XNb;

constexpr int PLANE_THREADS = 256;
constexpr int SMOOTH_MAX_CELLS = 64;

template <int EPI, int ZF, bool PK>
__global__ void __launch_bounds__(PLANE_THREADS, 2)
    sipg_plane_kernel(const float* __restrict__ src, float* __restrict__ dst, const __grid_constant__ Tab tb,
                      const __grid_constant__ Tab2 tp, const MeshDims m, const long long ncells, const Epi ea) {
  const int z = threadIdx.x & 3;
  long long c = ((long long)blockIdx.x * PLANE_THREADS + threadIdx.x) >> 2;
  const bool active = c < ncells;
  // lanes past the last cell work on a valid cell (they take part in the
  // shuffles) and store nothing
  if (!active) c = ncells - 1;
  const CellXYZ cx = cell_xyz((unsigned)c, m);
  const size_t off = (size_t)c * 64 + z * 16;
  const bool hasp = EPI == EPI_CHEB && ea.xprev != nullptr && ea.c1 != 0.f;
  if constexpr (EPI != EPI_NONE) {
    // the epilogue's vectors travel towards L1 while the operator is evaluated
    asm volatile("prefetch.global.L1 [%0];" ::"l"(ea.b + off));
    if (hasp) asm volatile("prefetch.global.L1 [%0];" ::"l"(ea.xprev + off));
  }
  const long long cfirst = (long long)cx.comp * m.E;
  const float* base = src + (size_t)cfirst * 64 + z * 16;
  float X[16], YP[16], YM[16], ZP[16], ZM[16];
  plane::load_plane(src + off, X);
  const unsigned ep = neighbor32<0>(cx, +1, m), em = neighbor32<0>(cx, -1, m);
  plane::load_plane(base + (size_t)neighbor32<1>(cx, +1, m) * 64, YP);
  plane::load_plane(base + (size_t)neighbor32<1>(cx, -1, m) * 64, YM);
  plane::load_plane(base + (size_t)neighbor32<2>(cx, +1, m) * 64, ZP);
  plane::load_plane(base + (size_t)neighbor32<2>(cx, -1, m) * 64, ZM);
  // x-neighbours: by shuffle from lane 4 (cell mod 8) + z where the neighbour
  // is in this warp's 8 cells, else from its plane
  XNb n;
  {
    const long long np = cfirst + ep, nm = cfirst + em;
    plane::xnb_shuffle(tb, X, 4 * (int)(np & 7) + z, 4 * (int)(nm & 7) + z, n);
    if ((np >> 3) != (c >> 3)) {
      float P[16];
      plane::load_plane(base + (size_t)ep * 64, P);
      plane::xnb_from_plane(tb, P, +1, n);
    }
    if ((nm >> 3) != (c >> 3)) {
      float P[16];
      plane::load_plane(base + (size_t)em * 64, P);
      plane::xnb_from_plane(tb, P, -1, n);
    }
  }
  float B[16], D[16], P[16], O[16];
  if constexpr (PK) {
    float2 Y[8];
    plane::apply2<ZF>(tb, tp, z, X, n, YP, YM, ZP, ZM, Y);
    if (!active) return;
    if constexpr (EPI != EPI_NONE) plane::load_plane(ea.b + off, B);
    if constexpr (EPI == EPI_CHEB) plane::load_plane(ea.dinv + z * 16, D);
    if (hasp) plane::load_plane(ea.xprev + off, P);
    plane::epilogue2<EPI>(ea, X, Y, B, D, P, hasp, O);
  } else {
    float Y[16];
    plane::apply<ZF>(tb, z, X, n, YP, YM, ZP, ZM, Y);
    if (!active) return;
    if constexpr (EPI != EPI_NONE) plane::load_plane(ea.b + off, B);
    if constexpr (EPI == EPI_CHEB) plane::load_plane(ea.dinv + z * 16, D);
    if (hasp) plane::load_plane(ea.xprev + off, P);
    plane::epilogue<EPI>(ea, X, Y, B, D, P, hasp, O);
  }
  plane::store_plane(dst + off, O);
}

// Every Chebyshev step of one smoothing call on a level of at most 64 cells,
// in one block (4 threads per cell) with the level in shared memory: three
// buffers (current, previous and next iterate) of 64 floats per cell; the
// neighbour planes come from shared memory, the arithmetic is the register
// kernel's.  Replaces one launch per step on the coarsest levels, where every
// launch is latency-bound.
__global__ void __launch_bounds__(4 * SMOOTH_MAX_CELLS)
    sipg_plane_smooth_kernel(const float* __restrict__ b, const float* __restrict__ x0, float* __restrict__ xout,
                             const float* __restrict__ dinv, const __grid_constant__ Tab tb,
                             const __grid_constant__ Tab2 tp, const MeshDims m, const int ncells,
                             const __grid_constant__ SmoothPlan pl) {
  float* sm = reinterpret_cast<float*>(dyn_smem());
  const int c = threadIdx.x >> 2, z = threadIdx.x & 3;
  const CellXYZ cx = cell_xyz((unsigned)c, m);
  const int own = c * 64 + z * 16;
  const int nb[6] = {(int)neighbor32<0>(cx, +1, m) * 64 + z * 16, (int)neighbor32<0>(cx, -1, m) * 64 + z * 16,
                     (int)neighbor32<1>(cx, +1, m) * 64 + z * 16, (int)neighbor32<1>(cx, -1, m) * 64 + z * 16,
                     (int)neighbor32<2>(cx, +1, m) * 64 + z * 16, (int)neighbor32<2>(cx, -1, m) * 64 + z * 16};
  float* xc = sm;
  float* xp = sm + ncells * 64;
  float* xn = sm + 2 * ncells * 64;
  float B[16], D[16];
  plane::load_plane(b + own, B);
  plane::load_plane(dinv + z * 16, D);
  auto rd = [](const float* q, float (&v)[16]) {
#pragma unroll
    for (int i = 0; i < 16; i += 4) {
      const float4 t = *reinterpret_cast<const float4*>(q + i);
      v[i] = t.x, v[i + 1] = t.y, v[i + 2] = t.z, v[i + 3] = t.w;
    }
  };
  auto wr = [](float* q, const float (&v)[16]) {
#pragma unroll
    for (int i = 0; i < 16; i += 4) *reinterpret_cast<float4*>(q + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
  };
  int k0 = 0;
  {
    float X[16], Z[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) Z[i] = 0.f;
    if (pl.zero_guess) {
      // x_1 = c2 D^-1 b, the first step from x_0 = 0
#pragma unroll
      for (int i = 0; i < 16; ++i) X[i] = pl.c2[0] * D[i] * B[i];
      k0 = 1;
    } else {
      plane::load_plane(x0 + own, X);
    }
    wr(xc + own, X);
    wr(xp + own, Z);
  }
  __syncthreads();
  for (int k = k0; k < pl.nsteps; ++k) {
    float X[16], YP[16], YM[16], ZP[16], ZM[16], P[16];
    rd(xc + own, X);
    rd(xc + nb[2], YP);
    rd(xc + nb[3], YM);
    rd(xc + nb[4], ZP);
    rd(xc + nb[5], ZM);
    XNb n;
    {
      float Q[16];
      rd(xc + nb[0], Q);
      plane::xnb_from_plane(tb, Q, +1, n);
      rd(xc + nb[1], Q);
      plane::xnb_from_plane(tb, Q, -1, n);
    }
    rd(xp + own, P);
    float2 Y[8];
    plane::apply2<1>(tb, tp, z, X, n, YP, YM, ZP, ZM, Y);
    const Epi e{nullptr, nullptr, nullptr, pl.c1[k], pl.c2[k]};
    float O[16];
    plane::epilogue2<EPI_CHEB>(e, X, Y, B, D, P, true, O);
    wr(xn + own, O);
    __syncthreads();
    float* t = xp;
    xp = xc;
    xc = xn;
    xn = t;
  }
  plane::store_plane(xout + own, *reinterpret_cast<const float(*)[16]>(xc + own));
}

std::atomic<int> g_variant{0};

template <int EPI, int ZF, bool PK>
int launch_plane(const MeshDims& m, long long ncells, const float* src, float* dst, const Tab& tb, const Tab2& tp,
                 const Epi& ea, cudaStream_t s) {
  const long long blocks = (ncells * 4 + PLANE_THREADS - 1) / PLANE_THREADS;
  sipg_plane_kernel<EPI, ZF, PK><<<(unsigned)blocks, PLANE_THREADS, 0, s>>>(src, dst, tb, tp, m, ncells, ea);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

template <int ZF, bool PK>
int launch_epi(int epi, const MeshDims& m, long long ncells, const float* src, float* dst, const Tab& tb,
               const Tab2& tp, const Epi& ea, cudaStream_t s) {
  switch (epi) {
    case EPI_NONE: return launch_plane<EPI_NONE, ZF, PK>(m, ncells, src, dst, tb, tp, ea, s);
    case EPI_RESID: return launch_plane<EPI_RESID, ZF, PK>(m, ncells, src, dst, tb, tp, ea, s);
    case EPI_CHEB: return launch_plane<EPI_CHEB, ZF, PK>(m, ncells, src, dst, tb, tp, ea, s);
  }
  return 1;
}

bool aligned32(const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 31) == 0; }

}  // namespace

void laplace_plane_set_variant(int v) { g_variant.store(v); }

int laplace_plane_f32(const MeshDims& m, int ncomp, const float* src, float* dst, const LapHost& h, int epi,
                      const EpiHost& eh, cudaStream_t s) {
  int v = g_variant.load();
  if (h.N != 4 || v < 0) return -1;
  if (v == 0 || v >= 4) {
    // the staged kernel where it applies (nx divisible by 8, 32-byte aligned
    // vectors), else the register one
    const int r = laplace_tma_f32(m, ncomp, src, dst, h, epi, eh, s, v == 5 ? 1 : 0);
    if (r >= 0) return r;
    v = 1;
  }
  if (!aligned32(src) || !aligned32(dst) || !aligned32(eh.b) || !aligned32(eh.xprev) || !aligned32(eh.dinv))
    return -1;
  const long long ncells = m.E * ncomp;
  if (ncells == 0) return 0;
  Tab tb;
  plane::make_tab(h, tb);
  Tab2 tp;
  plane::make_tab2(tb, tp);
  const Epi ea{(const float*)eh.b, (const float*)eh.xprev, (const float*)eh.dinv, (float)eh.c1, (float)eh.c2};
  switch (v) {
    case 1: return launch_epi<1, true>(epi, m, ncells, src, dst, tb, tp, ea, s);
    case 2: return launch_epi<1, false>(epi, m, ncells, src, dst, tb, tp, ea, s);
    case 3: return launch_epi<0, true>(epi, m, ncells, src, dst, tb, tp, ea, s);
  }
  return 1;
}

int laplace_plane_smooth(const MeshDims& m, const float* b, const float* x0, float* xout, const float* dinv,
                         const LapHost& h, const SmoothPlan& plan, cudaStream_t s) {
  const long long ncells = m.E;
  if (h.N != 4 || g_variant.load() < 0 || ncells < 8 || ncells > SMOOTH_MAX_CELLS || ncells % 8 != 0 ||
      plan.nsteps < 1 || plan.nsteps > SMOOTH_MAX_STEPS)
    return -1;
  if (!aligned32(b) || !aligned32(x0) || !aligned32(xout) || !aligned32(dinv)) return -1;
  Tab tb;
  plane::make_tab(h, tb);
  Tab2 tp;
  plane::make_tab2(tb, tp);
  const size_t smem = (size_t)3 * ncells * 64 * sizeof(float);
  sipg_plane_smooth_kernel<<<1, (unsigned)(4 * ncells), smem, s>>>(b, x0, xout, dinv, tb, tp, m, (int)ncells, plan);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // namespace dgns
