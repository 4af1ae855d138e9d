// Projection substep operator M + A_D + A_C with the divergence and
// continuity penalty terms (Sec. 3.2 and the matrix form of the projection
// step, Sec. 3.3, of arXiv:1802.01439), and the element-wise penalty
// parameters from the volume-averaged norm of the extrapolated velocity.
// FP64, k <= 7.
//
// Per cell (affine, Gauss rule with k+1 points, exact for both forms):
//   values  V_a = (S (x) S (x) S) u_a,   reference derivatives
//   G_x = (D (x) S (x) S) u_x, G_y = (S (x) D (x) S) u_y, G_z = (S (x) S (x) D) u_z
//   at every point: m_a = w V_a, g = tau_D w sum_a G_a / h_a  (w = quadrature
//   weight times h_x h_y h_z); test: y_b = (S^T)^3 m_b + (1/h_b) (D_b^T ...) g,
//   each component as one combined sweep along b followed by two S^T sweeps.
// Faces normal to a couple only component a: with LGL nodes the traces are
// the nodal values of the face layers and the Gauss rule integrates the face
// mass exactly, so the own face layer gets
//   {{tau_C}} h_t1 h_t2 (Mhat (x) Mhat) (u_a(own layer) - u_a(neighbour layer)).
#include "ops.h"

namespace dgns {
namespace {

template <int N>
struct ProjTab {
  double S[N * N];   // S[q*N+j] = phi_j(g_q)
  double D[N * N];   // D[q*N+j] = phi_j'(g_q)
  double M[N * N];   // 1D mass
  double w[N];       // Gauss weights on [0,1]
  double h[3];
};

template <int N>
constexpr int proj_cells_per_block() {
  return N * N >= 64 ? 1 : 64 / (N * N);
}

// out-line (along D) = A in-line, A applied as A (TR = false: y_q = sum_j A[q][j] x_j)
// or A^T (TR = true: y_j = sum_q A[q][j] x_q); optional second input and scale.
template <int N, int D, bool TR, bool TWO>
__device__ __forceinline__ void dsweep(const double* in, const double* in2, double* out, int l, const double* A,
                                       const double* A2, double s2) {
  int base, stride;
  line_geom<D>(l, N, N, N, base, stride);
  double x[N], x2[N];
  load_line<double, N>(in, base, stride, x);
  if (TWO) load_line<double, N>(in2, base, stride, x2);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double a = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) a = fma(TR ? A[j * N + i] : A[i * N + j], x[j], a);
    if (TWO) {
      double b = 0.0;
#pragma unroll
      for (int j = 0; j < N; ++j) b = fma(TR ? A2[j * N + i] : A2[i * N + j], x2[j], b);
      a = fma(s2, b, a);
    }
    out[base + i * stride] = a;
  }
}

template <int N>
__global__ void __launch_bounds__(proj_cells_per_block<N>() * N * N)
    proj_kernel(const double* __restrict__ u3, double* __restrict__ dst3, const double* __restrict__ tau_d,
                const double* __restrict__ tau_c, const __grid_constant__ ProjTab<N> tb, const MeshDims m) {
  constexpr int NT = N * N, N3 = N * N * N, EPB = proj_cells_per_block<N>();
  constexpr int PER = 27 * N3;
  double* sm = reinterpret_cast<double*>(dyn_smem());
  const int slot = threadIdx.x / NT;
  const int l = threadIdx.x - slot * NT;
  const long long c0 = (long long)blockIdx.x * EPB;
  const long long rem = m.E - c0;
  const int nvalid = rem < EPB ? (int)rem : EPB;
  const bool active = slot < nvalid;
  double* U = sm + slot * PER;   // 3 N3
  double* X = U + 3 * N3;        // 4 N3: S u_x, D u_x, S u_y, S u_z (x sweeps)
  double* Y = X + 4 * N3;        // 5 N3
  double* Z = Y + 5 * N3;        // 6 N3: V_x V_y V_z G_x G_y G_z -> m_x m_y m_z g
  double* T1 = Z + 6 * N3;       // 3 N3
  double* T2 = T1 + 3 * N3;      // 3 N3
  double* O = T2 + 3 * N3;       // 3 N3
  CellXYZ cx{};
  if (active) {
    cx = cell_xyz((unsigned)(c0 + slot), m);
    for (int c = 0; c < 3; ++c)
      for (int i = l; i < N3; i += NT) U[c * N3 + i] = u3[((size_t)c * m.E + cx.el) * N3 + i];
  }
  __syncthreads();
  if (active) {
    dsweep<N, 0, false, false>(U, nullptr, X, l, tb.S, nullptr, 0.0);
    dsweep<N, 0, false, false>(U, nullptr, X + N3, l, tb.D, nullptr, 0.0);
    dsweep<N, 0, false, false>(U + N3, nullptr, X + 2 * N3, l, tb.S, nullptr, 0.0);
    dsweep<N, 0, false, false>(U + 2 * N3, nullptr, X + 3 * N3, l, tb.S, nullptr, 0.0);
  }
  __syncthreads();
  if (active) {
    dsweep<N, 1, false, false>(X, nullptr, Y, l, tb.S, nullptr, 0.0);               // SS u_x
    dsweep<N, 1, false, false>(X + N3, nullptr, Y + N3, l, tb.S, nullptr, 0.0);     // DS u_x
    dsweep<N, 1, false, false>(X + 2 * N3, nullptr, Y + 2 * N3, l, tb.S, nullptr, 0.0);  // SS u_y
    dsweep<N, 1, false, false>(X + 2 * N3, nullptr, Y + 3 * N3, l, tb.D, nullptr, 0.0);  // SD u_y
    dsweep<N, 1, false, false>(X + 3 * N3, nullptr, Y + 4 * N3, l, tb.S, nullptr, 0.0);  // SS u_z
  }
  __syncthreads();
  if (active) {
    dsweep<N, 2, false, false>(Y, nullptr, Z, l, tb.S, nullptr, 0.0);               // V_x
    dsweep<N, 2, false, false>(Y + 2 * N3, nullptr, Z + N3, l, tb.S, nullptr, 0.0);  // V_y
    dsweep<N, 2, false, false>(Y + 4 * N3, nullptr, Z + 2 * N3, l, tb.S, nullptr, 0.0);  // V_z
    dsweep<N, 2, false, false>(Y + N3, nullptr, Z + 3 * N3, l, tb.S, nullptr, 0.0);      // G_x
    dsweep<N, 2, false, false>(Y + 3 * N3, nullptr, Z + 4 * N3, l, tb.S, nullptr, 0.0);  // G_y
    dsweep<N, 2, false, false>(Y + 4 * N3, nullptr, Z + 5 * N3, l, tb.D, nullptr, 0.0);  // G_z
  }
  __syncthreads();
  if (active) {
    const double td = tau_d[cx.el];
    const double jac = tb.h[0] * tb.h[1] * tb.h[2];
    for (int i = l; i < N3; i += NT) {
      const int qx = i % N, qy = (i / N) % N, qz = i / (N * N);
      const double w = tb.w[qx] * tb.w[qy] * tb.w[qz] * jac;
      const double div = Z[3 * N3 + i] / tb.h[0] + Z[4 * N3 + i] / tb.h[1] + Z[5 * N3 + i] / tb.h[2];
      Z[i] *= w;
      Z[N3 + i] *= w;
      Z[2 * N3 + i] *= w;
      Z[3 * N3 + i] = td * w * div;
    }
  }
  __syncthreads();
  // tests: b = x: (S^T m_x + D^T g / h_x) along x, then S^T y, S^T z
  //        b = y: along y first, then x, z;  b = z: along z first, then x, y
  if (active) {
    dsweep<N, 0, true, true>(Z, Z + 3 * N3, T1, l, tb.S, tb.D, 1.0 / tb.h[0]);
    dsweep<N, 1, true, true>(Z + N3, Z + 3 * N3, T1 + N3, l, tb.S, tb.D, 1.0 / tb.h[1]);
    dsweep<N, 2, true, true>(Z + 2 * N3, Z + 3 * N3, T1 + 2 * N3, l, tb.S, tb.D, 1.0 / tb.h[2]);
  }
  __syncthreads();
  if (active) {
    dsweep<N, 1, true, false>(T1, nullptr, T2, l, tb.S, nullptr, 0.0);
    dsweep<N, 0, true, false>(T1 + N3, nullptr, T2 + N3, l, tb.S, nullptr, 0.0);
    dsweep<N, 0, true, false>(T1 + 2 * N3, nullptr, T2 + 2 * N3, l, tb.S, nullptr, 0.0);
  }
  __syncthreads();
  if (active) {
    dsweep<N, 2, true, false>(T2, nullptr, O, l, tb.S, nullptr, 0.0);
    dsweep<N, 2, true, false>(T2 + N3, nullptr, O + N3, l, tb.S, nullptr, 0.0);
    dsweep<N, 1, true, false>(T2 + 2 * N3, nullptr, O + 2 * N3, l, tb.S, nullptr, 0.0);
  }
  __syncthreads();
  // continuity penalty: faces normal to a, component a
  if (active) {
    for (int a = 0; a < 3; ++a) {
      const int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
      const double area = a == 0 ? tb.h[1] * tb.h[2] : (a == 1 ? tb.h[0] * tb.h[2] : tb.h[0] * tb.h[1]);
      for (int side = 1; side >= -1; side -= 2) {
        const unsigned nb = a == 0 ? neighbor32<0>(cx, side, m) : (a == 1 ? neighbor32<1>(cx, side, m)
                                                                          : neighbor32<2>(cx, side, m));
        const double tbar = 0.5 * (tau_c[cx.el] + tau_c[nb]) * area;
        const int aown = side > 0 ? N - 1 : 0, anb = side > 0 ? 0 : N - 1;
        // thread l handles face node (j1, j2) = (l % N, l / N): (M (x) M) jump
        const int j1 = l % N, j2 = l / N;
        double acc = 0.0;
        const double* ua = u3 + ((size_t)a * m.E) * N3;
#pragma unroll
        for (int i2 = 0; i2 < N; ++i2) {
#pragma unroll
          for (int i1 = 0; i1 < N; ++i1) {
            int co[3], cn[3];
            co[a] = aown;
            co[t1] = i1;
            co[t2] = i2;
            cn[a] = anb;
            cn[t1] = i1;
            cn[t2] = i2;
            const int io = co[0] + N * (co[1] + N * co[2]), in_ = cn[0] + N * (cn[1] + N * cn[2]);
            const double jump = U[a * N3 + io] - __ldg(ua + (size_t)nb * N3 + in_);
            acc = fma(tb.M[j1 * N + i1] * tb.M[j2 * N + i2], jump, acc);
          }
        }
        int co[3];
        co[a] = aown;
        co[t1] = j1;
        co[t2] = j2;
        const int io = co[0] + N * (co[1] + N * co[2]);
        O[a * N3 + io] = fma(tbar, acc, O[a * N3 + io]);
      }
    }
  }
  __syncthreads();
  if (active)
    for (int c = 0; c < 3; ++c)
      for (int i = l; i < N3; i += NT) dst3[((size_t)c * m.E + cx.el) * N3 + i] = O[c * N3 + i];
}

// Volume-averaged Euclidean norm of u per cell -> penalty parameters.
template <int N>
__global__ void __launch_bounds__(proj_cells_per_block<N>() * N * N)
    speed_kernel(const double* __restrict__ u3, double* __restrict__ tau_d, double* __restrict__ tau_c,
                 const __grid_constant__ ProjTab<N> tb, const MeshDims m, double fd, double fc) {
  constexpr int NT = N * N, N3 = N * N * N, EPB = proj_cells_per_block<N>();
  constexpr int PER = 9 * N3;
  double* sm = reinterpret_cast<double*>(dyn_smem());
  const int slot = threadIdx.x / NT;
  const int l = threadIdx.x - slot * NT;
  const long long c0 = (long long)blockIdx.x * EPB;
  const long long rem = m.E - c0;
  const int nvalid = rem < EPB ? (int)rem : EPB;
  const bool active = slot < nvalid;
  double* U = sm + slot * PER;
  double* A = U + 3 * N3;
  double* B = A + 3 * N3;
  __shared__ double red[EPB][NT];
  const long long el = c0 + slot;
  if (active)
    for (int c = 0; c < 3; ++c)
      for (int i = l; i < N3; i += NT) U[c * N3 + i] = u3[((size_t)c * m.E + el) * N3 + i];
  __syncthreads();
  if (active)
    for (int c = 0; c < 3; ++c) dsweep<N, 0, false, false>(U + c * N3, nullptr, A + c * N3, l, tb.S, nullptr, 0.0);
  __syncthreads();
  if (active)
    for (int c = 0; c < 3; ++c) dsweep<N, 1, false, false>(A + c * N3, nullptr, B + c * N3, l, tb.S, nullptr, 0.0);
  __syncthreads();
  if (active)
    for (int c = 0; c < 3; ++c) dsweep<N, 2, false, false>(B + c * N3, nullptr, A + c * N3, l, tb.S, nullptr, 0.0);
  __syncthreads();
  double s = 0.0;
  if (active)
    for (int i = l; i < N3; i += NT) {
      const int qx = i % N, qy = (i / N) % N, qz = i / (N * N);
      const double v = sqrt(A[i] * A[i] + A[N3 + i] * A[N3 + i] + A[2 * N3 + i] * A[2 * N3 + i]);
      s = fma(tb.w[qx] * tb.w[qy] * tb.w[qz], v, s);
    }
  red[slot][l] = s;
  __syncthreads();
  if (active && l == 0) {
    double t = 0.0;
    for (int i = 0; i < NT; ++i) t += red[slot][i];   // fixed order
    tau_d[el] = fd * t;
    tau_c[el] = fc * t;
  }
}

template <int N>
ProjTab<N> make_tab(const ProjHost& h) {
  ProjTab<N> tb;
  for (int i = 0; i < N * N; ++i) {
    tb.S[i] = h.S[i];
    tb.D[i] = h.D[i];
    tb.M[i] = h.M[i];
  }
  for (int q = 0; q < N; ++q) tb.w[q] = h.w[q];
  for (int d = 0; d < 3; ++d) tb.h[d] = h.h[d];
  return tb;
}

template <int N>
int launch_proj(const MeshDims& m, const double* u3, double* dst3, const double* td, const double* tc,
                const ProjHost& h, cudaStream_t s) {
  constexpr int EPB = proj_cells_per_block<N>();
  const size_t smem = (size_t)EPB * 27 * N * N * N * sizeof(double);
  if (smem > 232448) return 7;
  if (cudaFuncSetAttribute(proj_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 2;
  if (m.E == 0) return 0;
  const long long blocks = (m.E + EPB - 1) / EPB;
  proj_kernel<N><<<(unsigned)blocks, EPB * N * N, smem, s>>>(u3, dst3, td, tc, make_tab<N>(h), m);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

template <int N>
int launch_speed(const MeshDims& m, const double* u3, double* td, double* tc, const ProjHost& h, double fd,
                 double fc, cudaStream_t s) {
  constexpr int EPB = proj_cells_per_block<N>();
  const size_t smem = (size_t)EPB * 9 * N * N * N * sizeof(double);
  if (cudaFuncSetAttribute(speed_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 2;
  if (m.E == 0) return 0;
  const long long blocks = (m.E + EPB - 1) / EPB;
  speed_kernel<N><<<(unsigned)blocks, EPB * N * N, smem, s>>>(u3, td, tc, make_tab<N>(h), m, fd, fc);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // namespace

int projection_apply(const MeshDims& m, const double* u3, double* dst3, const double* tau_d, const double* tau_c,
                     const ProjHost& h, cudaStream_t s) {
  switch (h.N) {
    case 2: return launch_proj<2>(m, u3, dst3, tau_d, tau_c, h, s);
    case 3: return launch_proj<3>(m, u3, dst3, tau_d, tau_c, h, s);
    case 4: return launch_proj<4>(m, u3, dst3, tau_d, tau_c, h, s);
    case 5: return launch_proj<5>(m, u3, dst3, tau_d, tau_c, h, s);
    case 6: return launch_proj<6>(m, u3, dst3, tau_d, tau_c, h, s);
    case 7: return launch_proj<7>(m, u3, dst3, tau_d, tau_c, h, s);
    case 8: return launch_proj<8>(m, u3, dst3, tau_d, tau_c, h, s);
  }
  return 7;
}

int penalty_parameters(const MeshDims& m, const double* u3, double* tau_d, double* tau_c, const ProjHost& h,
                       double fd, double fc, cudaStream_t s) {
  switch (h.N) {
    case 2: return launch_speed<2>(m, u3, tau_d, tau_c, h, fd, fc, s);
    case 3: return launch_speed<3>(m, u3, tau_d, tau_c, h, fd, fc, s);
    case 4: return launch_speed<4>(m, u3, tau_d, tau_c, h, fd, fc, s);
    case 5: return launch_speed<5>(m, u3, tau_d, tau_c, h, fd, fc, s);
    case 6: return launch_speed<6>(m, u3, tau_d, tau_c, h, fd, fc, s);
    case 7: return launch_speed<7>(m, u3, tau_d, tau_c, h, fd, fc, s);
    case 8: return launch_speed<8>(m, u3, tau_d, tau_c, h, fd, fc, s);
  }
  return 7;
}

}  // namespace dgns
