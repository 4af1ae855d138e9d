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

// dst = L src on ncomp scalar fields (cells of component c follow those of
// component c-1); `fp32` selects float data, else double.
// emulated (double data only): double-float arithmetic on the FP32 pipe,
// EPI_NONE only.
int laplace_apply(bool fp32, const MeshDims& m, int ncomp, const void* src, void* dst,
                  const LapHost& tab, int epi, const EpiHost& ea, cudaStream_t s, bool emulated = false);

// dst[cell][i] = table[i] for every cell (broadcast of a per-cell pattern).
int broadcast_cells(bool fp32, long long ncells, int nper, const void* table, void* dst,
                    cudaStream_t s);

// dst = (Mz (x) My (x) Mx) src per cell, square N x N matrices (mass,
// inverse mass), double data; emulated: double-float arithmetic.
int tensor3_apply(int N, long long ncells, const double* src, double* dst, const double* Mx,
                  const double* My, const double* Mz, cudaStream_t s, bool emulated = false);

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
// emulated: double-float arithmetic on the FP32 pipe (else native FP64).
int convective_launch(int part, const MeshDims& m, const double* u3, double* rface, double* dst3,
                      const ConvHost& t, bool emulated, cudaStream_t s);
// emulated: double-float arithmetic (else native FP64)
int convective_vjp(const MeshDims& m, const double* u3, const double* w3, double* dst3,
                   const ConvHost& t, cudaStream_t s, bool emulated = false);

// Projection operator M + A_D + A_C and the penalty parameters
// (k_projection.cu); N = k_u + 1 <= 8.
struct ProjHost {
  int N = 0;
  double S[MAXN * MAXN], D[MAXN * MAXN], M[MAXN * MAXN];
  double w[MAXN];
  double h[3];
};
// emulated: double-float arithmetic (else native FP64)
int projection_apply(const MeshDims& m, const double* u3, double* dst3, const double* tau_d, const double* tau_c,
                     const ProjHost& h, cudaStream_t s, bool emulated = false);
// tau_d = fd * avg|u|, tau_c = fc * avg|u| per cell
int penalty_parameters(const MeshDims& m, const double* u3, double* tau_d, double* tau_c, const ProjHost& h,
                       double fd, double fc, cudaStream_t s, bool emulated = false);

}  // namespace dgns
