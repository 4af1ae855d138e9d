// Host-side 1D tables of the DG discretisation (Sec. 3.2 of Fehn, Wall &
// Kronbichler, arXiv:1802.01439): Gauss and Legendre-Gauss-Lobatto rules,
// Lagrange basis values and derivatives, and the 1D matrices from which the
// device kernels build every 3D operator on a Cartesian mesh.  Everything is
// computed in long double and rounded once to the kernel's precision.
#pragma once
#include <vector>

namespace dgns {

typedef long double ld;
typedef std::vector<ld> vec;

// n-point Gauss-Legendre rule on [0,1] (Newton on the Legendre recurrence).
void gauss_rule(int n, vec& x, vec& w);
// k+1 LGL nodes on [0,1]: end points and the roots of P_k' (Newton).
vec lgl_nodes(int k);
// V[q*N + j] = phi_j(x_q), D[q*N + j] = phi_j'(x_q) of the Lagrange basis
// through `nodes` (product formula).
void lagrange(const vec& nodes, const vec& x, vec& V, vec& D);
// In-place inverse of a dense n x n row-major matrix (Gauss-Jordan with
// partial pivoting).  Returns false when singular.
bool invert(vec& A, int n);

// 1D matrices of one scalar DG space with N = k+1 LGL nodes on [0,1].
struct Space1D {
  int N = 0;
  vec nodes;
  vec mass;      // Mhat[i*N+j] = int_0^1 phi_i phi_j        (N Gauss points, exact)
  vec stiff;     // Khat[i*N+j] = int_0^1 phi_i' phi_j'
  vec d0, d1;    // phi_j'(0), phi_j'(1)
  vec mass_inv;  // Mhat^-1
};
Space1D make_space(int k);

// 1D SIPG Laplace on a periodic line of elements of size h with penalty tau
// (face form -{dq}[p] - [q]{dp} + tau [q][p], Sec. 3.2), split as
//   y_e = A0 x_e + (neighbour terms),
//   neighbour e+1:  y_i += cr_i * x_{e+1}[0],  y_{N-1} += sum_j gr_j x_{e+1}[j]
//   neighbour e-1:  y_i += cl_i * x_{e-1}[N-1], y_0   += sum_j gl_j x_{e-1}[j]
struct Laplace1D {
  vec A0, cr, cl, gr, gl;
};
Laplace1D make_laplace_1d(const Space1D& s, ld h, ld tau);

// 1D divergence line operator for test degree k_p (Np nodes) and trial degree
// k_u (Nu nodes), Nu Gauss points:  y = R x_e + neighbour terms,
//   y_{Np-1} += +1/2 x_{e+1}[0],   y_0 += -1/2 x_{e-1}[Nu-1]
// and the mixed mass Mpu[i*Nu+j] = int phi^p_i phi^u_j.
struct Div1D {
  vec R;    // Np x Nu
  vec Mpu;  // Np x Nu
};
Div1D make_div_1d(const Space1D& su, const Space1D& sp);
// 1D gradient line operator (test degree k_u, trial k_p):
//   y = G x_e + neighbour terms, y_{Nu-1} += 1/2 x_{e+1}[0], y_0 += -1/2 x_{e-1}[Np-1]
struct Grad1D {
  vec G;    // Nu x Np
  vec Mup;  // Nu x Np
};
Grad1D make_grad_1d(const Space1D& su, const Space1D& sp);

// Interpolation to Q Gauss points: S[q*N+j] = phi_j(g_q), D[q*N+j] = phi_j'(g_q),
// w[q] the Gauss weights on [0,1].
struct Quad1D {
  int Q = 0;
  vec S, D, w;
};
Quad1D make_quad_1d(const Space1D& s, int Q);

// Embedding of a coarse cell polynomial into child c (0: left half, 1: right
// half): P[i*N+j] = phi_j((xi_i + c) / 2).
vec make_prolongation_1d(const Space1D& s, int c);

}  // namespace dgns
