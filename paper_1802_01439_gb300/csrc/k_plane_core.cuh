// Arithmetic of the FP32 SIPG operator on cells of N = 4 nodes per direction
// with one thread per z-plane of a cell (Secs. 3.2 and 3.3 of
// arXiv:1802.01439): the Kronecker form
//     y = M_z [ M_y T_x x + M_x T_y x ] + M_x M_y T_z x
// evaluated on a 4 x 4 plane held in registers (index 4 y + x), the 4 planes
// of a cell on adjacent lanes 4 g + z of a warp.  Shared by the kernel that
// reads its planes from global memory (k_laplace_plane.cu) and the one that
// stages them in shared memory with the tensor memory accelerator
// (k_laplace_tma.cu).
#pragma once

#include "common.cuh"
#include "ops.h"

namespace dgns {
namespace plane {

constexpr unsigned FULL = 0xffffffffu;

struct Tab {
  float A0[3][16];
  float M[16];
  float cr[3][4], cl[3][4], gr[3][4], gl[3][4];
};

struct Epi {
  const float* b;
  const float* xprev;
  const float* dinv;
  float c1, c2;
};

inline void make_tab(const LapHost& h, Tab& tb) {
  for (int d = 0; d < 3; ++d) {
    for (int i = 0; i < 16; ++i) tb.A0[d][i] = (float)h.A0[d][i];
    for (int i = 0; i < 4; ++i) {
      tb.cr[d][i] = (float)h.cr[d][i];
      tb.cl[d][i] = (float)h.cl[d][i];
      tb.gr[d][i] = (float)h.gr[d][i];
      tb.gl[d][i] = (float)h.gl[d][i];
    }
  }
  for (int i = 0; i < 16; ++i) tb.M[i] = (float)h.M[i];
}

// One 64-byte plane from global memory with two 256-bit loads.
__device__ __forceinline__ void load_plane(const float* __restrict__ p, float (&v)[16]) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
      : "l"(p));
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8+32];"
      : "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15])
      : "l"(p));
}

__device__ __forceinline__ void store_plane(float* p, const float (&v)[16]) {
  asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
               "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
  asm volatile("st.global.v8.f32 [%0+32], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[8]), "f"(v[9]), "f"(v[10]),
               "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15])
               : "memory");
}

// out = M_x M_y in.
__device__ __forceinline__ void mass_xy(const float (&in)[16], float (&out)[16], const float* M) {
  float t[16];
#pragma unroll
  for (int y = 0; y < 4; ++y)
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      float a = M[4 * y] * in[x];
#pragma unroll
      for (int j = 1; j < 4; ++j) a = fmaf(M[4 * y + j], in[4 * j + x], a);
      t[4 * y + x] = a;
    }
#pragma unroll
  for (int y = 0; y < 4; ++y)
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      float a = M[4 * x] * t[4 * y];
#pragma unroll
      for (int j = 1; j < 4; ++j) a = fmaf(M[4 * x + j], t[4 * y + j], a);
      out[4 * y + x] = a;
    }
}

// Sum of V over the 4 lanes of a cell, plane i to lane i: V[t] of lane j
// holds its contribution to plane t ^ j, so that both butterfly rounds shuffle
// the same registers on every lane; the result is left in V[0].
__device__ __forceinline__ void reduce_scatter4(float (&V)[4][16]) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    V[0][k] += __shfl_xor_sync(FULL, V[2][k], 2);
    V[1][k] += __shfl_xor_sync(FULL, V[3][k], 2);
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) V[0][k] += __shfl_xor_sync(FULL, V[1][k], 1);
}

// x-neighbour data of every row y: the + neighbour's value at x = 0 and
// face-derivative sum gr . row (rp, dp), the - neighbour's value at x = 3 and
// gl . row (lm, dm).
struct XNb {
  float rp[4], dp[4], lm[4], dm[4];
};

// Summaries from a neighbour's plane P: side +1 fills rp, dp; -1 fills lm, dm.
__device__ __forceinline__ void xnb_from_plane(const Tab& tb, const float (&P)[16], int side, XNb& n) {
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    float g = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) g = fmaf(side > 0 ? tb.gr[0][j] : tb.gl[0][j], P[4 * y + j], g);
    if (side > 0) {
      n.rp[y] = P[4 * y];
      n.dp[y] = g;
    } else {
      n.lm[y] = P[4 * y + 3];
      n.dm[y] = g;
    }
  }
}

// Summaries by shuffle from lanes sp (+ neighbour) and sm (- neighbour): every
// lane forms from its own rows what its x-neighbours need.  Every lane of the
// warp takes part.
__device__ __forceinline__ void xnb_shuffle(const Tab& tb, const float (&X)[16], int sp, int sm, XNb& n) {
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    float gsum = 0.f, lsum = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      gsum = fmaf(tb.gr[0][j], X[4 * y + j], gsum);
      lsum = fmaf(tb.gl[0][j], X[4 * y + j], lsum);
    }
    n.rp[y] = __shfl_sync(FULL, X[4 * y], sp);
    n.dp[y] = __shfl_sync(FULL, gsum, sp);
    n.lm[y] = __shfl_sync(FULL, X[4 * y + 3], sm);
    n.dm[y] = __shfl_sync(FULL, lsum, sm);
  }
}

// Y = L x on the own plane z of a cell (lane z of its group): X the own plane,
// n the x-neighbour summaries, YP, YM plane z of the y-neighbours, ZP, ZM plane
// z of the z-neighbours.  The z-direction is one reduce-scatter across the
// cell's lanes (ZF = 0: M_x M_y applied per lane to x and the z-neighbour
// planes first, 48 shuffles) or two (ZF = 1: T_z x reduced first and M_x M_y
// applied once to it, 96 shuffles).  Every lane of the warp takes part.
template <int ZF>
__device__ __forceinline__ void apply(const Tab& tb, int z, const float (&X)[16], const XNb& n,
                                      const float (&YP)[16], const float (&YM)[16], const float (&ZP)[16],
                                      const float (&ZM)[16], float (&Y)[16]) {
  // W = M_y T_x x + M_x T_y x
  float W[16];
  {
    float T[16];   // T_x x, rows y
#pragma unroll
    for (int y = 0; y < 4; ++y) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float a = fmaf(tb.cl[0][i], n.lm[y], tb.cr[0][i] * n.rp[y]);
#pragma unroll
        for (int j = 0; j < 4; ++j) a = fmaf(tb.A0[0][4 * i + j], X[4 * y + j], a);
        T[4 * y + i] = a;
      }
      T[4 * y + 3] += n.dp[y];
      T[4 * y] += n.dm[y];
    }
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        float a = tb.M[4 * y] * T[x];
#pragma unroll
        for (int j = 1; j < 4; ++j) a = fmaf(tb.M[4 * y + j], T[4 * j + x], a);
        W[4 * y + x] = a;
      }
  }
  {
    float T[16];   // T_y x, columns x
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      float dr = 0.f, dl = 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        dr = fmaf(tb.gr[1][j], YP[4 * j + x], dr);
        dl = fmaf(tb.gl[1][j], YM[4 * j + x], dl);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float a = fmaf(tb.cl[1][i], YM[12 + x], tb.cr[1][i] * YP[x]);
#pragma unroll
        for (int j = 0; j < 4; ++j) a = fmaf(tb.A0[1][4 * i + j], X[4 * j + x], a);
        T[4 * i + x] = a;
      }
      T[12 + x] += dr;
      T[x] += dl;
    }
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int j = 0; j < 4; ++j) W[4 * y + x] = fmaf(tb.M[4 * x + j], T[4 * y + j], W[4 * y + x]);
  }
  // z-direction.  Lane j's share of T_z x for output plane i:
  //   A0_z(i, j) x_j + CR(i, j) ZP_j + CL(i, j) ZM_j,
  // CR(i, j) = cr_z(i) [j = 0] + gr_z(j) [i = 3],
  // CL(i, j) = cl_z(i) [j = 3] + gl_z(j) [i = 0]
  // (ZP_j, ZM_j: plane j of the +z and -z neighbours); its share of M_z W
  // for plane i is M(i, j) W_j.
  float mz[4], az[4], crz[4], clz[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int i = t ^ z;
    mz[t] = tb.M[4 * i + z];
    az[t] = tb.A0[2][4 * i + z];
    crz[t] = (z == 0 ? tb.cr[2][i] : 0.f) + (i == 3 ? tb.gr[2][z] : 0.f);
    clz[t] = (z == 3 ? tb.cl[2][i] : 0.f) + (i == 0 ? tb.gl[2][z] : 0.f);
  }
  if constexpr (ZF == 0) {
    float Q[16], R[16], L[16];
    mass_xy(X, Q, tb.M);
    mass_xy(ZP, R, tb.M);
    mass_xy(ZM, L, tb.M);
    float V[4][16];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int k = 0; k < 16; ++k)
        V[t][k] = fmaf(mz[t], W[k], fmaf(az[t], Q[k], fmaf(crz[t], R[k], clz[t] * L[k])));
    reduce_scatter4(V);
#pragma unroll
    for (int k = 0; k < 16; ++k) Y[k] = V[0][k];
  } else {
    float S[16];
    {
      float V[4][16];
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int k = 0; k < 16; ++k) V[t][k] = fmaf(az[t], X[k], fmaf(crz[t], ZP[k], clz[t] * ZM[k]));
      reduce_scatter4(V);
      mass_xy(V[0], S, tb.M);
    }
    float V[4][16];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int k = 0; k < 16; ++k) V[t][k] = mz[t] * W[k];
    reduce_scatter4(V);
#pragma unroll
    for (int k = 0; k < 16; ++k) Y[k] = V[0][k] + S[k];
  }
}

// What the kernel stores for y = L x:  EPI_NONE y;  EPI_RESID b - y;
// EPI_CHEB  x + c1 (x - xprev) + c2 dinv (b - y), a null xprev (hasp false)
// standing for a zero previous iterate.
template <int EPI>
__device__ __forceinline__ void epilogue(const Epi& ea, const float (&X)[16], const float (&Y)[16],
                                         const float (&B)[16], const float (&D)[16], const float (&P)[16],
                                         bool hasp, float (&O)[16]) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if constexpr (EPI == EPI_NONE) {
      O[k] = Y[k];
    } else if constexpr (EPI == EPI_RESID) {
      O[k] = B[k] - Y[k];
    } else {
      float v = fmaf(ea.c2 * D[k], B[k] - Y[k], X[k]);
      if (ea.c1 != 0.f) v = fmaf(ea.c1, X[k] - (hasp ? P[k] : 0.f), v);
      O[k] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// The same arithmetic on packed pairs (fma.rn.f32x2): a plane as 8 float2,
// P[2 y + h] = (x(4 y + 2 h), x(4 y + 2 h + 1)), pairs along x.  Sweeps along
// y and z multiply pairs by a broadcast coefficient; sweeps along x form a
// pair of outputs from a broadcast input and a pair of coefficients.  Every
// element sees the operations of the scalar code in the same order, so the
// results are bit-identical to it, at about half the FP32 instructions.

struct Tab2 {
  float2 Mb[16], A0yb[16];          // (c, c) of M and the cell part of T_y
  float2 A0xp[2][4], Mxp[2][4];     // (c(2h, j), c(2h + 1, j)) of T_x's cell part and M
  float2 crxp[2], clxp[2];          // (cr_x(2h), cr_x(2h + 1)), same for cl_x
  float2 cryb[4], clyb[4], gryb[4], glyb[4];   // (c, c) of T_y's neighbour coupling
};

inline void make_tab2(const Tab& t, Tab2& p) {
  for (int i = 0; i < 16; ++i) {
    p.Mb[i] = make_float2(t.M[i], t.M[i]);
    p.A0yb[i] = make_float2(t.A0[1][i], t.A0[1][i]);
  }
  for (int h = 0; h < 2; ++h) {
    for (int j = 0; j < 4; ++j) {
      p.A0xp[h][j] = make_float2(t.A0[0][4 * (2 * h) + j], t.A0[0][4 * (2 * h + 1) + j]);
      p.Mxp[h][j] = make_float2(t.M[4 * (2 * h) + j], t.M[4 * (2 * h + 1) + j]);
    }
    p.crxp[h] = make_float2(t.cr[0][2 * h], t.cr[0][2 * h + 1]);
    p.clxp[h] = make_float2(t.cl[0][2 * h], t.cl[0][2 * h + 1]);
  }
  for (int i = 0; i < 4; ++i) {
    p.cryb[i] = make_float2(t.cr[1][i], t.cr[1][i]);
    p.clyb[i] = make_float2(t.cl[1][i], t.cl[1][i]);
    p.gryb[i] = make_float2(t.gr[1][i], t.gr[1][i]);
    p.glyb[i] = make_float2(t.gl[1][i], t.gl[1][i]);
  }
}

__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

__device__ __forceinline__ void pack(const float (&v)[16], float2 (&p)[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) p[k] = make_float2(v[2 * k], v[2 * k + 1]);
}

// out = M_x M_y in (M_y on pairs with a broadcast coefficient, then M_x
// forming output pairs).
__device__ __forceinline__ void mass_xy2(const Tab2& tp, const float2 (&in)[8], float2 (&out)[8]) {
  float2 t[8];
#pragma unroll
  for (int y = 0; y < 4; ++y)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float2 a = mul2(tp.Mb[4 * y], in[h]);
#pragma unroll
      for (int j = 1; j < 4; ++j) a = fma2(tp.Mb[4 * y + j], in[2 * j + h], a);
      t[2 * y + h] = a;
    }
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    const float2 tb0 = bc(t[2 * y].x), tb1 = bc(t[2 * y].y), tb2 = bc(t[2 * y + 1].x), tb3 = bc(t[2 * y + 1].y);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float2 a = mul2(tp.Mxp[h][0], tb0);
      a = fma2(tp.Mxp[h][1], tb1, a);
      a = fma2(tp.Mxp[h][2], tb2, a);
      a = fma2(tp.Mxp[h][3], tb3, a);
      out[2 * y + h] = a;
    }
  }
}

__device__ __forceinline__ void reduce_scatter4(float2 (&V)[4][8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    V[0][k] = add2(V[0][k], make_float2(__shfl_xor_sync(FULL, V[2][k].x, 2), __shfl_xor_sync(FULL, V[2][k].y, 2)));
    V[1][k] = add2(V[1][k], make_float2(__shfl_xor_sync(FULL, V[3][k].x, 2), __shfl_xor_sync(FULL, V[3][k].y, 2)));
  }
#pragma unroll
  for (int k = 0; k < 8; ++k)
    V[0][k] = add2(V[0][k], make_float2(__shfl_xor_sync(FULL, V[1][k].x, 1), __shfl_xor_sync(FULL, V[1][k].y, 1)));
}

// Packed form of apply (same results), the neighbour planes fetched where
// they are used: get(i, v) fills v with plane z of the +y (i = 0), -y (1),
// +z (2) or -z (3) neighbour.
// The x- and y-part W = M_y T_x x + M_x T_y x (get(0), get(1) used).
template <class Get>
__device__ __forceinline__ void apply2_xy(const Tab2& tp, const float (&Xs)[16], const XNb& n, Get&& get,
                                          float2 (&W)[8]) {
  float2 X[8];
  pack(Xs, X);
  {
    float2 T[8];   // T_x x: row y, output pair h
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const float2 rb = bc(n.rp[y]), lb = bc(n.lm[y]);
      const float2 xb[4] = {bc(Xs[4 * y]), bc(Xs[4 * y + 1]), bc(Xs[4 * y + 2]), bc(Xs[4 * y + 3])};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float2 a = fma2(tp.clxp[h], lb, mul2(tp.crxp[h], rb));
#pragma unroll
        for (int j = 0; j < 4; ++j) a = fma2(tp.A0xp[h][j], xb[j], a);
        T[2 * y + h] = a;
      }
      T[2 * y + 1].y += n.dp[y];
      T[2 * y].x += n.dm[y];
    }
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float2 a = mul2(tp.Mb[4 * y], T[h]);
#pragma unroll
        for (int j = 1; j < 4; ++j) a = fma2(tp.Mb[4 * y + j], T[2 * j + h], a);
        W[2 * y + h] = a;
      }
  }
  float2 YP[8], YM[8];
  {
    float t[16];
    get(0, t);
    pack(t, YP);
    get(1, t);
    pack(t, YM);
  }
  {
    float2 T[8];   // T_y x: output row i, column pair h
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float2 dr = mul2(tp.gryb[0], YP[h]), dl = mul2(tp.glyb[0], YM[h]);
#pragma unroll
      for (int j = 1; j < 4; ++j) {
        dr = fma2(tp.gryb[j], YP[2 * j + h], dr);
        dl = fma2(tp.glyb[j], YM[2 * j + h], dl);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float2 a = fma2(tp.clyb[i], YM[6 + h], mul2(tp.cryb[i], YP[h]));
#pragma unroll
        for (int j = 0; j < 4; ++j) a = fma2(tp.A0yb[4 * i + j], X[2 * j + h], a);
        T[2 * i + h] = a;
      }
      T[6 + h] = add2(T[6 + h], dr);
      T[h] = add2(T[h], dl);
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const float2 t0 = bc(T[2 * y].x), t1 = bc(T[2 * y].y), t2 = bc(T[2 * y + 1].x), t3 = bc(T[2 * y + 1].y);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float2 a = W[2 * y + h];
        a = fma2(tp.Mxp[h][0], t0, a);
        a = fma2(tp.Mxp[h][1], t1, a);
        a = fma2(tp.Mxp[h][2], t2, a);
        a = fma2(tp.Mxp[h][3], t3, a);
        W[2 * y + h] = a;
      }
    }
  }
}

// The z-part: Y = M_z W + M_x M_y T_z x (get(2), get(3) used).
template <int ZF, class Get>
__device__ __forceinline__ void apply2_z(const Tab& tb, const Tab2& tp, int z, const float (&Xs)[16],
                                         const float2 (&W)[8], Get&& get, float2 (&Y)[8]) {
  float2 X[8];
  pack(Xs, X);
  // z-direction: the slot coefficients of apply, broadcast
  float2 mz[4], az[4], crz[4], clz[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int i = t ^ z;
    mz[t] = bc(tb.M[4 * i + z]);
    az[t] = bc(tb.A0[2][4 * i + z]);
    crz[t] = bc((z == 0 ? tb.cr[2][i] : 0.f) + (i == 3 ? tb.gr[2][z] : 0.f));
    clz[t] = bc((z == 3 ? tb.cl[2][i] : 0.f) + (i == 0 ? tb.gl[2][z] : 0.f));
  }
  float2 ZP[8], ZM[8];
  {
    float t[16];
    get(2, t);
    pack(t, ZP);
    get(3, t);
    pack(t, ZM);
  }
  if constexpr (ZF == 0) {
    float2 Q[8], R[8], L[8];
    mass_xy2(tp, X, Q);
    mass_xy2(tp, ZP, R);
    mass_xy2(tp, ZM, L);
    float2 V[4][8];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int k = 0; k < 8; ++k) V[t][k] = fma2(mz[t], W[k], fma2(az[t], Q[k], fma2(crz[t], R[k], mul2(clz[t], L[k]))));
    reduce_scatter4(V);
#pragma unroll
    for (int k = 0; k < 8; ++k) Y[k] = V[0][k];
  } else {
    float2 S[8];
    {
      float2 V[4][8];
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int k = 0; k < 8; ++k) V[t][k] = fma2(az[t], X[k], fma2(crz[t], ZP[k], mul2(clz[t], ZM[k])));
      reduce_scatter4(V);
      mass_xy2(tp, V[0], S);
    }
    float2 V[4][8];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int k = 0; k < 8; ++k) V[t][k] = mul2(mz[t], W[k]);
    reduce_scatter4(V);
#pragma unroll
    for (int k = 0; k < 8; ++k) Y[k] = add2(V[0][k], S[k]);
  }
}

template <int ZF, class Get>
__device__ __forceinline__ void apply2g(const Tab& tb, const Tab2& tp, int z, const float (&Xs)[16], const XNb& n,
                                        Get&& get, float2 (&Y)[8]) {
  float2 W[8];
  apply2_xy(tp, Xs, n, get, W);
  apply2_z<ZF>(tb, tp, z, Xs, W, get, Y);
}

// Packed form of apply with the neighbour planes in registers.
template <int ZF>
__device__ __forceinline__ void apply2(const Tab& tb, const Tab2& tp, int z, const float (&Xs)[16], const XNb& n,
                                       const float (&YPs)[16], const float (&YMs)[16], const float (&ZPs)[16],
                                       const float (&ZMs)[16], float2 (&Y)[8]) {
  apply2g<ZF>(tb, tp, z, Xs, n,
              [&](int i, float (&v)[16]) {
                const float(&src)[16] = i == 0 ? YPs : (i == 1 ? YMs : (i == 2 ? ZPs : ZMs));
#pragma unroll
                for (int k = 0; k < 16; ++k) v[k] = src[k];
              },
              Y);
}

// Packed form of epilogue.
template <int EPI>
__device__ __forceinline__ void epilogue2(const Epi& ea, const float (&Xs)[16], const float2 (&Y)[8],
                                          const float (&Bs)[16], const float (&Ds)[16], const float (&Ps)[16],
                                          bool hasp, float (&O)[16]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float2 v;
    if constexpr (EPI == EPI_NONE) {
      v = Y[k];
    } else if constexpr (EPI == EPI_RESID) {
      v = sub2(make_float2(Bs[2 * k], Bs[2 * k + 1]), Y[k]);
    } else {
      const float2 x = make_float2(Xs[2 * k], Xs[2 * k + 1]);
      const float2 r = sub2(make_float2(Bs[2 * k], Bs[2 * k + 1]), Y[k]);
      v = fma2(mul2(bc(ea.c2), make_float2(Ds[2 * k], Ds[2 * k + 1])), r, x);
      if (ea.c1 != 0.f) {
        const float2 pv = hasp ? make_float2(Ps[2 * k], Ps[2 * k + 1]) : make_float2(0.f, 0.f);
        v = fma2(bc(ea.c1), sub2(x, pv), v);
      }
    }
    O[2 * k] = v.x;
    O[2 * k + 1] = v.y;
  }
}
}  // namespace plane
}  // namespace dgns
