// Host-side launchers of the libdgns kernels (internal interface between the
// C ABI layer and the kernel translation units).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace dgns {

constexpr int MAXN = 12;  // k + 1 <= 12

// Tables of an SIPG-type operator (Laplace, viscous, Helmholtz) on a Cartesian
// mesh, see laplace_apply below.  All entries already include the geometric
// factors of their direction.
struct LapHost {
  int N = 0;
  double A0[3][MAXN * MAXN];
  double M[MAXN * MAXN];
  double cr[3][MAXN], cl[3][MAXN], gr[3][MAXN], gl[3][MAXN];
};

// What the Laplace-type kernel writes at every node, with y = L x:
enum Epilogue {
  EPI_NONE = 0,   // dst = y
  EPI_RESID = 1,  // dst = b - y
  EPI_CHEB = 2,   // dst = x + c1 (x - xprev) + c2 dinv (b - y)   (Chebyshev step)
};
struct EpiHost {
  const void* b = nullptr;
  const void* xprev = nullptr;
  const void* dinv = nullptr;  // N^3 table, identical for every cell
  double c1 = 0.0, c2 = 0.0;
};

// Arithmetic of the FP64 operator kernels (the context's fp64_mode).
enum Arith {
  ARITH_F64 = 0,    // native FP64
  ARITH_DF64 = 1,   // double-float on the FP32 pipe (48-bit significand)
  ARITH_TF64 = 2,   // triple-float on the FP32 pipe (SIPG and mass kernels; others native FP64)
};

// FP32 Laplace operator on cells of N = 4 with one thread per cell plane
// (k_laplace_plane.cu).  Returns -1, doing nothing, where it does not apply
// (N != 4, a pointer not aligned for its vector accesses, or the line kernel
// selected by laplace_plane_set_variant(-1)); else 0, or 2 on a launch error.
int laplace_plane_f32(const MeshDims& m, int ncomp, const float* src, float* dst, const LapHost& h, int epi,
                      const EpiHost& eh, cudaStream_t s);
// Kernel choice for the FP32 N = 4 operator: 0 built-in (the staged kernel
// where it applies, else the register plane kernel), -1 the line kernel; the
// register plane kernel with packed FP32x2 arithmetic (1), scalar (2), or
// packed with the z-direction as one reduce-scatter (3); the staged kernel
// with one stage and 12 warps per SM (4) or two stages and 7 warps (5), each
// falling back to 1 where it does not apply.
void laplace_plane_set_variant(int v);
// A whole Chebyshev smoothing call on a level of 8..64 cells (multiple of 8)
// at N = 4 in one block (k_laplace_plane.cu): nsteps steps with the
// coefficients c1[k], c2[k] of step k; zero_guess: x_0 = 0 (x0 unused) and
// the first step is x_1 = c2[0] D^-1 b.  xout may be x0.  -1 where it does
// not apply (also under laplace_plane_set_variant(-1)).
constexpr int SMOOTH_MAX_STEPS = 64;
struct SmoothPlan {
  int nsteps = 0;
  int zero_guess = 0;
  float c1[SMOOTH_MAX_STEPS], c2[SMOOTH_MAX_STEPS];
};
int laplace_plane_smooth(const MeshDims& m, const float* b, const float* x0, float* xout, const float* dinv,
                         const LapHost& h, const SmoothPlan& plan, cudaStream_t s);
// The same operator with its data staged in shared memory by tensor copies
// (k_laplace_tma.cu): nx divisible by 8 and 32-byte aligned vectors, else -1;
// variant 0 one stage and 12 warps per SM, 1 two stages and 7 warps.
int laplace_tma_f32(const MeshDims& m, int ncomp, const float* src, float* dst, const LapHost& h, int epi,
                    const EpiHost& eh, cudaStream_t s, int variant);
// Waits of the staged kernel that gave up (device counter; synchronous read).
unsigned laplace_tma_timeouts();

// dst = L src on ncomp scalar fields (cells of component c follow those of
// component c-1); `fp32` selects float data, else double.
// arith (double data only): an Arith; the emulated ones take EPI_NONE only.
// Face data of the split SIPG evaluation (k_laplace_split.cu): phi_i'(0),
// phi_i'(1), the 1D mass, and per direction 1/h_d, the penalty, the face area.
struct SplitHost {
  int N = 0;
  double d0[MAXN], d1[MAXN], M[MAXN * MAXN];
  double ih[3], tau[3], area[3];
};
// dst += the interior-face terms of the SIPG operator on ncomp fields of src
// (the face kernel into fbuf, 6 N^2 doubles per cell, then the apply kernel).
int laplace_faces_apply(const MeshDims& m, int ncomp, const double* src, double* fbuf, double* dst,
                        const SplitHost& h, cudaStream_t s);

int laplace_apply(bool fp32, const MeshDims& m, int ncomp, const void* src, void* dst,
                  const LapHost& tab, int epi, const EpiHost& ea, cudaStream_t s, int arith = ARITH_F64);

// dst[cell][i] = table[i] for every cell (broadcast of a per-cell pattern).
int broadcast_cells(bool fp32, long long ncells, int nper, const void* table, void* dst,
                    cudaStream_t s);

// dst = (Mz (x) My (x) Mx) src per cell, square N x N matrices (mass,
// inverse mass), double data; arith: an Arith.
int tensor3_apply(int N, long long ncells, const double* src, double* dst, const double* Mx,
                  const double* My, const double* Mz, cudaStream_t s, int arith = ARITH_F64);

// Multigrid transfers between a coarse mesh mc and the fine mesh 2*mc.
// prolongate: fine (+)= P coarse; restrict: coarse = P^T fine.
int prolongate(bool fp32, int N, const MeshDims& mc, const void* coarse, void* fine,
               const double* P0, const double* P1, bool add, cudaStream_t s);
int restrict_fine(bool fp32, int N, const MeshDims& mc, const void* fine, void* coarse,
                  const double* P0, const double* P1, cudaStream_t s);

// Divergence and gradient (see k_divgrad.cu for the factorisation).
struct DivHost {
  int Nu = 0, Np = 0;
  double R[3][MAXN * MAXN];    // Np x Nu per direction, scaled by tangential h
  double Mpu[MAXN * MAXN];     // Np x Nu
  double nbr[3], nbl[3];       // neighbour face-value coefficients
};
int divergence_apply(const MeshDims& m, const double* u3, double* dst, const DivHost& t,
                     cudaStream_t s, bool emulated = false);
struct GradHost {
  int Nu = 0, Np = 0;
  double G[3][MAXN * MAXN];    // Nu x Np
  double Mup[MAXN * MAXN];     // Nu x Np
  double nbr[3], nbl[3];
};
int gradient_apply(const MeshDims& m, const double* p, double* dst3, const GradHost& t,
                   cudaStream_t s, bool emulated = false);

// Convective term with local Lax-Friedrichs flux (k_convective.cu).
struct ConvHost {
  int N = 0, Q = 0;
  double S[18 * MAXN];   // Q x N interpolation to Gauss points
  double D[18 * MAXN];   // Q x N derivative at Gauss points (reference)
  double w[18];          // Gauss weights on [0,1]
  double h[3];
};
// part: bit 0 the face kernel (u3 -> rface: the face integrals, 9 E N^2
// doubles, see conv_face_kernel), bit 1 the cell kernel (u3, rface -> dst3).
// arith: an Arith (triple-float for the 3/2 rule up to N = 11, native FP64
// beyond).
int convective_launch(int part, const MeshDims& m, const double* u3, double* rface, double* dst3,
                      const ConvHost& t, int arith, cudaStream_t s);
// The FP64-wide kernels beyond native FP64 (k_convective_tf64.cu): the cell
// kernel with native-FP64 and triple-float blocks side by side, the face
// kernel native; 7 where not instantiated or not fitting.
int convective_launch_tf64(int part, const MeshDims& m, const double* u3, double* rface, double* dst3,
                           const ConvHost& t, cudaStream_t s);
// Split of the mixed cell kernel: of every `period` blocks the first
// `nnative` run native FP64; period 0 restores the built-in split, period
// -1 runs the convective kernels in triple-float throughout.
void convective_set_mix(int period, int nnative);
// emulated: double-float arithmetic (else native FP64)
int convective_vjp(const MeshDims& m, const double* u3, const double* w3, double* dst3,
                   const ConvHost& t, cudaStream_t s, bool emulated = false);

// Projection operator M + A_D + A_C and the penalty parameters
// (k_projection.cu); N = k_u + 1 <= 12.
struct ProjHost {
  int N = 0;
  double S[MAXN * MAXN], D[MAXN * MAXN], M[MAXN * MAXN];
  double w[MAXN];
  double h[3];
};
// Terms of the projection operator: the mass term (the mass kernel), the
// divergence penalty A_D and the continuity penalty A_C; PROJ_ALL is the
// fused operator M + A_D + A_C.
enum ProjTerms { PROJ_MASS = 1, PROJ_DIV = 2, PROJ_CONT = 4, PROJ_ALL = 7 };
// emulated: double-float arithmetic (else native FP64); terms: PROJ_ALL
// (one fused kernel), PROJ_DIV or PROJ_CONT (that term alone)
int projection_apply(const MeshDims& m, const double* u3, double* dst3, const double* tau_d, const double* tau_c,
                     const ProjHost& h, cudaStream_t s, bool emulated = false, int terms = PROJ_ALL);
// tau_d = fd * avg|u|, tau_c = fc * avg|u| per cell
int penalty_parameters(const MeshDims& m, const double* u3, double* tau_d, double* tau_c, const ProjHost& h,
                       double fd, double fc, cudaStream_t s, bool emulated = false);

}  // namespace dgns
