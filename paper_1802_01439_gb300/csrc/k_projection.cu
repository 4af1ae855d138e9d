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
#include "arith.cuh"
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

// Tables of the operator kernel in the arithmetic policy's value type.
template <class V, int N>
struct ProjTabT {
  static constexpr bool kMM = N <= 6;   // the N^4 face-mass table fits the parameter space
  V S[N * N], D[N * N], M[N * N];
  V MM[kMM ? N * N * N * N : 1];   // (M (x) M)[(j1 + N j2)][(i1 + N i2)] = M[j1][i1] M[j2][i2]
  V W3[N * N * N];       // w_qx w_qy w_qz h_x h_y h_z
  V hinv[3];             // 1 / h_d
  V area[3];             // face area of faces normal to d
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

// The same sweep in an arithmetic policy: out = A in (+ A2 in2 scaled by the
// second table, which then already carries the scale).
template <class P, int N, int D, bool TR, bool TWO>
__device__ __forceinline__ void psweep(const typename P::V* in, const typename P::V* in2, typename P::V* out,
                                       int l, const typename P::V* A, const typename P::V* A2) {
  typedef typename P::V V;
  typedef typename P::Acc Acc;
  int base, stride;
  line_geom<D>(l, N, N, N, base, stride);
  V x[N], x2[N];
  load_line<V, N>(in, base, stride, x);
  if (TWO) load_line<V, N>(in2, base, stride, x2);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    Acc a;
    P::acc_first(a, TR ? A[i] : A[i * N], x[0]);
#pragma unroll
    for (int j = 1; j < N; ++j) P::acc_fma(a, TR ? A[j * N + i] : A[i * N + j], x[j]);
    if (TWO) {
#pragma unroll
      for (int j = 0; j < N; ++j) P::acc_fma(a, TR ? A2[j * N + i] : A2[i * N + j], x2[j]);
    }
    out[base + i * stride] = P::acc_get(a);
  }
}

template <class P, int N>
__global__ void __launch_bounds__(proj_cells_per_block<N>() * N * N)
    proj_kernel(const double* __restrict__ u3, double* __restrict__ dst3, const double* __restrict__ tau_d,
                const double* __restrict__ tau_c, const __grid_constant__ ProjTabT<typename P::V, N> tb,
                const MeshDims m) {
  typedef typename P::V V;
  typedef typename P::Acc Acc;
  constexpr int NT = N * N, N3 = N * N * N, EPB = proj_cells_per_block<N>();
  constexpr int PER = 27 * N3;
  V* sm = reinterpret_cast<V*>(dyn_smem());
  const int slot = threadIdx.x / NT;
  const int l = threadIdx.x - slot * NT;
  const long long c0 = (long long)blockIdx.x * EPB;
  const long long rem = m.E - c0;
  const int nvalid = rem < EPB ? (int)rem : EPB;
  const bool active = slot < nvalid;
  V* U = sm + slot * PER;   // 3 N3
  V* X = U + 3 * N3;        // 4 N3: S u_x, D u_x, S u_y, S u_z (x sweeps)
  V* Y = X + 4 * N3;        // 5 N3
  V* Z = Y + 5 * N3;        // 6 N3: V_x V_y V_z G_x G_y G_z -> m_x m_y m_z g
  V* T1 = Z + 6 * N3;       // 3 N3
  V* T2 = T1 + 3 * N3;      // 3 N3
  V* O = T2 + 3 * N3;       // 3 N3
  // D^T / h_d tables of the three combined test sweeps
  __shared__ V sDh[3][N * N];
  for (int i = threadIdx.x; i < 3 * N * N; i += blockDim.x)
    sDh[i / (N * N)][i % (N * N)] = P::mul(tb.D[i % (N * N)], tb.hinv[i / (N * N)]);
  CellXYZ cx{};
  if (active) {
    cx = cell_xyz((unsigned)(c0 + slot), m);
    for (int c = 0; c < 3; ++c)
      for (int i = l; i < N3; i += NT) U[c * N3 + i] = P::load(u3 + ((size_t)c * m.E + cx.el) * N3 + i);
  }
  __syncthreads();
  if (active) {
    psweep<P, N, 0, false, false>(U, nullptr, X, l, tb.S, nullptr);
    psweep<P, N, 0, false, false>(U, nullptr, X + N3, l, tb.D, nullptr);
    psweep<P, N, 0, false, false>(U + N3, nullptr, X + 2 * N3, l, tb.S, nullptr);
    psweep<P, N, 0, false, false>(U + 2 * N3, nullptr, X + 3 * N3, l, tb.S, nullptr);
  }
  __syncthreads();
  if (active) {
    psweep<P, N, 1, false, false>(X, nullptr, Y, l, tb.S, nullptr);                  // SS u_x
    psweep<P, N, 1, false, false>(X + N3, nullptr, Y + N3, l, tb.S, nullptr);        // DS u_x
    psweep<P, N, 1, false, false>(X + 2 * N3, nullptr, Y + 2 * N3, l, tb.S, nullptr);  // SS u_y
    psweep<P, N, 1, false, false>(X + 2 * N3, nullptr, Y + 3 * N3, l, tb.D, nullptr);  // SD u_y
    psweep<P, N, 1, false, false>(X + 3 * N3, nullptr, Y + 4 * N3, l, tb.S, nullptr);  // SS u_z
  }
  __syncthreads();
  if (active) {
    psweep<P, N, 2, false, false>(Y, nullptr, Z, l, tb.S, nullptr);                  // V_x
    psweep<P, N, 2, false, false>(Y + 2 * N3, nullptr, Z + N3, l, tb.S, nullptr);    // V_y
    psweep<P, N, 2, false, false>(Y + 4 * N3, nullptr, Z + 2 * N3, l, tb.S, nullptr);  // V_z
    psweep<P, N, 2, false, false>(Y + N3, nullptr, Z + 3 * N3, l, tb.S, nullptr);      // G_x
    psweep<P, N, 2, false, false>(Y + 3 * N3, nullptr, Z + 4 * N3, l, tb.S, nullptr);  // G_y
    psweep<P, N, 2, false, false>(Y + 4 * N3, nullptr, Z + 5 * N3, l, tb.D, nullptr);  // G_z
  }
  __syncthreads();
  if (active) {
    const V td = P::load(tau_d + cx.el);
    for (int i = l; i < N3; i += NT) {
      const V w = tb.W3[i];
      Acc dv;
      P::acc_first(dv, tb.hinv[0], Z[3 * N3 + i]);
      P::acc_fma(dv, tb.hinv[1], Z[4 * N3 + i]);
      P::acc_fma(dv, tb.hinv[2], Z[5 * N3 + i]);
      Z[i] = P::mul(w, Z[i]);
      Z[N3 + i] = P::mul(w, Z[N3 + i]);
      Z[2 * N3 + i] = P::mul(w, Z[2 * N3 + i]);
      Z[3 * N3 + i] = P::mul(P::mul(td, w), P::acc_get(dv));
    }
  }
  __syncthreads();
  // tests: b = x: (S^T m_x + (D/h_x)^T g) along x, then S^T y, S^T z
  //        b = y: along y first, then x, z;  b = z: along z first, then x, y
  if (active) {
    psweep<P, N, 0, true, true>(Z, Z + 3 * N3, T1, l, tb.S, sDh[0]);
    psweep<P, N, 1, true, true>(Z + N3, Z + 3 * N3, T1 + N3, l, tb.S, sDh[1]);
    psweep<P, N, 2, true, true>(Z + 2 * N3, Z + 3 * N3, T1 + 2 * N3, l, tb.S, sDh[2]);
  }
  __syncthreads();
  if (active) {
    psweep<P, N, 1, true, false>(T1, nullptr, T2, l, tb.S, nullptr);
    psweep<P, N, 0, true, false>(T1 + N3, nullptr, T2 + N3, l, tb.S, nullptr);
    psweep<P, N, 0, true, false>(T1 + 2 * N3, nullptr, T2 + 2 * N3, l, tb.S, nullptr);
  }
  __syncthreads();
  if (active) {
    psweep<P, N, 2, true, false>(T2, nullptr, O, l, tb.S, nullptr);
    psweep<P, N, 2, true, false>(T2 + N3, nullptr, O + N3, l, tb.S, nullptr);
    psweep<P, N, 1, true, false>(T2 + 2 * N3, nullptr, O + 2 * N3, l, tb.S, nullptr);
  }
  __syncthreads();
  // continuity penalty: faces normal to a, component a
  if (active) {
    const V half_tc = P::half(P::load(tau_c + cx.el));
    for (int a = 0; a < 3; ++a) {
      // node strides along a and the two tangential directions t1 < t2
      const int sa = a == 0 ? 1 : (a == 1 ? N : N * N);
      const int s1 = a == 0 ? N : 1, s2 = a == 2 ? N : N * N;
      for (int side = 1; side >= -1; side -= 2) {
        const unsigned nb = a == 0 ? neighbor32<0>(cx, side, m) : (a == 1 ? neighbor32<1>(cx, side, m)
                                                                          : neighbor32<2>(cx, side, m));
        // {{tau_C}} |F| (the halving is exact)
        const V tbar = P::mul(P::add(half_tc, P::half(P::load(tau_c + nb))), tb.area[a]);
        const int aown = side > 0 ? N - 1 : 0, anb = side > 0 ? 0 : N - 1;
        // thread l handles face node (j1, j2) = (l % N, l / N): (M (x) M) jump
        const int j1 = l % N, j2 = l / N;
        const double* ua = u3 + ((size_t)a * m.E) * N3;
        Acc acc;
#pragma unroll
        for (int i2 = 0; i2 < N; ++i2) {
#pragma unroll
          for (int i1 = 0; i1 < N; ++i1) {
            const int io = aown * sa + i1 * s1 + i2 * s2, in_ = anb * sa + i1 * s1 + i2 * s2;
            const V jump = P::sub(U[a * N3 + io], P::load(ua + (size_t)nb * N3 + in_));
            const V mm = ProjTabT<V, N>::kMM ? tb.MM[(j1 + N * j2) * N * N + i1 + N * i2]
                                             : P::mul(tb.M[j1 * N + i1], tb.M[j2 * N + i2]);
            if (i1 == 0 && i2 == 0)
              P::acc_first(acc, mm, jump);
            else
              P::acc_fma(acc, mm, jump);
          }
        }
        const int io = aown * sa + j1 * s1 + j2 * s2;
        Acc o;
        P::acc_set(o, O[a * N3 + io]);
        P::acc_fma(o, tbar, P::acc_get(acc));
        O[a * N3 + io] = P::acc_get(o);
      }
    }
  }
  __syncthreads();
  if (active)
    for (int c = 0; c < 3; ++c)
      for (int i = l; i < N3; i += NT) dst3[((size_t)c * m.E + cx.el) * N3 + i] = P::store(O[c * N3 + i]);
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

template <class P, int N>
ProjTabT<typename P::V, N> make_tabT(const ProjHost& h) {
  ProjTabT<typename P::V, N> tb;
  for (int i = 0; i < N * N; ++i) {
    tb.S[i] = P::make(h.S[i]);
    tb.D[i] = P::make(h.D[i]);
  }
  for (int i = 0; i < N * N; ++i) tb.M[i] = P::make(h.M[i]);
  if (ProjTabT<typename P::V, N>::kMM)
    for (int j2 = 0; j2 < N; ++j2)
      for (int j1 = 0; j1 < N; ++j1)
        for (int i2 = 0; i2 < N; ++i2)
          for (int i1 = 0; i1 < N; ++i1)
            tb.MM[(j1 + N * j2) * N * N + i1 + N * i2] = P::make(h.M[j1 * N + i1] * h.M[j2 * N + i2]);
  const double jac = h.h[0] * h.h[1] * h.h[2];
  for (int qz = 0; qz < N; ++qz)
    for (int qy = 0; qy < N; ++qy)
      for (int qx = 0; qx < N; ++qx) tb.W3[qx + N * (qy + N * qz)] = P::make(h.w[qx] * h.w[qy] * h.w[qz] * jac);
  for (int d = 0; d < 3; ++d) {
    tb.hinv[d] = P::make(1.0 / h.h[d]);
    tb.area[d] = P::make(jac / h.h[d]);
  }
  return tb;
}

template <class P, int N>
int launch_proj(const MeshDims& m, const double* u3, double* dst3, const double* td, const double* tc,
                const ProjHost& h, cudaStream_t s) {
  constexpr int EPB = proj_cells_per_block<N>();
  const size_t smem = (size_t)EPB * 27 * N * N * N * sizeof(double);
  if (smem > 232448 - 3 * N * N * sizeof(double)) return 7;
  if (cudaFuncSetAttribute(proj_kernel<P, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 2;
  if (m.E == 0) return 0;
  const long long blocks = (m.E + EPB - 1) / EPB;
  proj_kernel<P, N><<<(unsigned)blocks, EPB * N * N, smem, s>>>(u3, dst3, td, tc, make_tabT<P, N>(h), m);
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
                     const ProjHost& h, cudaStream_t s, bool emulated) {
#define DGNS_PROJ(NV) \
  case NV:            \
    return emulated ? launch_proj<DF64, NV>(m, u3, dst3, tau_d, tau_c, h, s) : launch_proj<F64, NV>(m, u3, dst3, tau_d, tau_c, h, s);
  switch (h.N) {
    DGNS_PROJ(2)
    DGNS_PROJ(3)
    DGNS_PROJ(4)
    DGNS_PROJ(5)
    DGNS_PROJ(6)
    DGNS_PROJ(7)
    DGNS_PROJ(8)
  }
#undef DGNS_PROJ
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
