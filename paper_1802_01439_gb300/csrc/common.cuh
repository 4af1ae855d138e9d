// Device helpers shared by the operator kernels of libdgns.
//
// Every operator on the periodic Cartesian mesh is a sum of Kronecker products
// of small 1D matrices (the geometry is affine and axis-aligned, so the Gauss
// quadrature of Sec. 3.2 factorises exactly).  A kernel therefore consists of
// "sweeps": for every line of an element along direction d, multiply the line
// by a small matrix whose entries live in the kernel's parameter space.  The
// loops are fully unrolled on the compile-time node count, so the matrix
// entries are uniform constant-bank operands of the FMA instructions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dgns {

// Unsigned division by an invariant divisor d (1 <= d < 2^31) with a
// multiply-high and shifts (Granlund & Montgomery 1994, Fig. 4.1):
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (t + ((n - t) >> min(l,1))) >> max(l-1,0), t = mulhi(m, n).
struct FastDiv {
  unsigned d = 1, m = 1, s1 = 0, s2 = 0;
  __host__ void set(unsigned dv) {
    d = dv;
    unsigned l = 0;
    while ((1ull << l) < dv) ++l;
    m = (unsigned)((((1ull << 32) * ((1ull << l) - dv)) / dv) + 1);
    s1 = l < 1 ? l : 1;
    s2 = l >= 1 ? l - 1 : 0;
  }
  __device__ __forceinline__ unsigned div(unsigned n) const {
    const unsigned t = __umulhi(m, n);
    return (t + ((n - t) >> s1)) >> s2;
  }
};

struct MeshDims {
  int nx, ny, nz;
  long long E;  // cells per component
  FastDiv fE, fx, fy;  // division by E, nx, ny (set by set_divisors)
  __host__ void set_divisors() {
    fE.set((unsigned)E);
    fx.set((unsigned)nx);
    fy.set((unsigned)ny);
  }
};

// Start offset and stride of line `l` (0 <= l < NI*NJ) along direction d in
// a cell array with extents (n0, n1, n2) in x, y, z (x fastest).
template <int D>
__device__ __forceinline__ void line_geom(int l, int n0, int n1, int n2, int& base, int& stride) {
  if (D == 0) {          // x-lines, l = y + n1 * z
    base = l * n0;
    stride = 1;
  } else if (D == 1) {   // y-lines, l = x + n0 * z
    const int x = l % n0, z = l / n0;
    base = x + n0 * n1 * z;
    stride = n0;
  } else {               // z-lines, l = x + n0 * y
    base = l;
    stride = n0 * n1;
  }
}

// Periodic neighbour of local cell `el` along direction D, +1 or -1.
template <int D>
__device__ __forceinline__ long long neighbor(long long el, int ex, int ey, int ez, int sgn,
                                              const MeshDims& m) {
  if (D == 0) {
    int v = ex + sgn;
    v = v < 0 ? m.nx - 1 : (v >= m.nx ? 0 : v);
    return el + (v - ex);
  } else if (D == 1) {
    int v = ey + sgn;
    v = v < 0 ? m.ny - 1 : (v >= m.ny ? 0 : v);
    return el + (long long)(v - ey) * m.nx;
  } else {
    int v = ez + sgn;
    v = v < 0 ? m.nz - 1 : (v >= m.nz ? 0 : v);
    return el + (long long)(v - ez) * m.nx * m.ny;
  }
}

// Cell coordinates with 32-bit integer arithmetic (64-bit division is a long
// integer sequence on the GPU; the library rejects meshes with 2^31 or more
// cells in all components together).
struct CellXYZ {
  unsigned el;    // cell id within its component
  unsigned comp;  // component
  int ex, ey, ez;
};

__device__ __forceinline__ CellXYZ cell_xyz(unsigned cell, const MeshDims& m) {
  CellXYZ c;
  const unsigned E = (unsigned)m.E, nx = (unsigned)m.nx, ny = (unsigned)m.ny;
  c.comp = m.fE.div(cell);
  c.el = cell - c.comp * E;
  const unsigned t = m.fx.div(c.el);
  c.ex = (int)(c.el - t * nx);
  c.ez = (int)m.fy.div(t);
  c.ey = (int)(t - (unsigned)c.ez * ny);
  return c;
}

// Periodic neighbour (cell id within the component) along direction D.
template <int D>
__device__ __forceinline__ unsigned neighbor32(const CellXYZ& c, int sgn, const MeshDims& m) {
  if (D == 0) {
    int v = c.ex + sgn;
    v = v < 0 ? m.nx - 1 : (v >= m.nx ? 0 : v);
    return c.el + (unsigned)(v - c.ex);
  } else if (D == 1) {
    int v = c.ey + sgn;
    v = v < 0 ? m.ny - 1 : (v >= m.ny ? 0 : v);
    return c.el + (unsigned)((v - c.ey) * m.nx);
  } else {
    int v = c.ez + sgn;
    v = v < 0 ? m.nz - 1 : (v >= m.nz ? 0 : v);
    return c.el + (unsigned)((v - c.ez) * m.nx * m.ny);
  }
}

// y[i] = sum_j A[i*NI + j] x[j]   (A row-major NO x NI)
template <class T, int NO, int NI>
__device__ __forceinline__ void matvec(const T* A, const T (&x)[NI], T (&y)[NO]) {
#pragma unroll
  for (int i = 0; i < NO; ++i) {
    T acc = A[i * NI] * x[0];
#pragma unroll
    for (int j = 1; j < NI; ++j) acc = fma(A[i * NI + j], x[j], acc);
    y[i] = acc;
  }
}

template <class T, int N>
__device__ __forceinline__ void load_line(const T* buf, int base, int stride, T (&x)[N]) {
#pragma unroll
  for (int j = 0; j < N; ++j) x[j] = buf[base + j * stride];
}

template <class T, int N>
__device__ __forceinline__ void store_line(T* buf, int base, int stride, const T (&x)[N]) {
#pragma unroll
  for (int j = 0; j < N; ++j) buf[base + j * stride] = x[j];
}

// Asynchronous 8-byte global -> shared copy (cp.async, cached in L1), the
// commit of the copies issued so far, and the wait for all of them.  The
// copied data is visible to other threads after the wait and a barrier.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Barrier of the threads of one cell or face: a warp barrier when they are
// exactly one warp, else a block barrier (then the block holds whole groups
// and every thread reaches it).
template <int NT>
__device__ __forceinline__ void group_sync() {
  if (NT == 32)
    __syncwarp();
  else
    __syncthreads();
}

// Dynamic shared memory, aligned for double2 accesses.
__device__ __forceinline__ unsigned char* dyn_smem() {
  extern __shared__ __align__(16) unsigned char dgns_smem[];
  return dgns_smem;
}

}  // namespace dgns
