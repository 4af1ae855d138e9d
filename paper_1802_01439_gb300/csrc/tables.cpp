// Host-side 1D tables (see tables.h).
#include "tables.h"

#include <cmath>

namespace dgns {

namespace {
const ld PI_L = 3.141592653589793238462643383279502884L;

// Legendre P_n and P_n' at x in [-1,1] by the three-term recurrence.
void legendre(int n, ld x, ld& p, ld& dp) {
  ld p0 = 1.0L, p1 = x;
  if (n == 0) { p = 1.0L; dp = 0.0L; return; }
  for (int m = 1; m < n; ++m) {
    ld p2 = ((2 * m + 1) * x * p1 - m * p0) / (m + 1);
    p0 = p1;
    p1 = p2;
  }
  p = p1;
  // n (x P_n - P_{n-1}) = (x^2 - 1) P_n'
  dp = n * (x * p1 - p0) / (x * x - 1.0L);
}
}  // namespace

void gauss_rule(int n, vec& x, vec& w) {
  x.assign(n, 0.0L);
  w.assign(n, 0.0L);
  for (int i = 0; i < n; ++i) {
    ld t = cosl(PI_L * (i + 0.75L) / (n + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld p, dp;
      legendre(n, t, p, dp);
      ld dt = p / dp;
      t -= dt;
      if (fabsl(dt) < 1e-19L) break;
    }
    ld p, dp;
    legendre(n, t, p, dp);
    // t descends with i: store ascending on [0,1]
    x[i] = 0.5L * (1.0L - t);
    w[i] = 1.0L / ((1.0L - t * t) * dp * dp);  // 2/((1-t^2)P'^2) halved
  }
}

vec lgl_nodes(int k) {
  vec x(k + 1);
  x[0] = 0.0L;
  x[k] = 1.0L;
  for (int i = 1; i < k; ++i) {
    ld t = -cosl(PI_L * i / k);
    for (int it = 0; it < 100; ++it) {
      ld p, dp;
      legendre(k, t, p, dp);
      // Newton on P_k': P_k'' = (2t P_k' - k(k+1) P_k) / (1 - t^2)
      ld ddp = (2.0L * t * dp - k * (k + 1.0L) * p) / (1.0L - t * t);
      ld dt = dp / ddp;
      t -= dt;
      if (fabsl(dt) < 1e-19L) break;
    }
    x[i] = 0.5L * (t + 1.0L);
  }
  return x;
}

void lagrange(const vec& nodes, const vec& xs, vec& V, vec& D) {
  const int N = (int)nodes.size();
  const int Q = (int)xs.size();
  V.assign((size_t)Q * N, 0.0L);
  D.assign((size_t)Q * N, 0.0L);
  for (int j = 0; j < N; ++j) {
    ld den = 1.0L;
    for (int m = 0; m < N; ++m)
      if (m != j) den *= nodes[j] - nodes[m];
    for (int q = 0; q < Q; ++q) {
      const ld x = xs[q];
      ld val = 1.0L;
      for (int m = 0; m < N; ++m)
        if (m != j) val *= x - nodes[m];
      ld der = 0.0L;
      for (int l = 0; l < N; ++l) {
        if (l == j) continue;
        ld t = 1.0L;
        for (int m = 0; m < N; ++m)
          if (m != j && m != l) t *= x - nodes[m];
        der += t;
      }
      V[(size_t)q * N + j] = val / den;
      D[(size_t)q * N + j] = der / den;
    }
  }
}

bool invert(vec& A, int n) {
  vec I((size_t)n * n, 0.0L);
  for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0L;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(A[(size_t)r * n + c]) > fabsl(A[(size_t)piv * n + c])) piv = r;
    if (A[(size_t)piv * n + c] == 0.0L) return false;
    if (piv != c)
      for (int j = 0; j < n; ++j) {
        std::swap(A[(size_t)c * n + j], A[(size_t)piv * n + j]);
        std::swap(I[(size_t)c * n + j], I[(size_t)piv * n + j]);
      }
    const ld d = A[(size_t)c * n + c];
    for (int j = 0; j < n; ++j) {
      A[(size_t)c * n + j] /= d;
      I[(size_t)c * n + j] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const ld f = A[(size_t)r * n + c];
      if (f == 0.0L) continue;
      for (int j = 0; j < n; ++j) {
        A[(size_t)r * n + j] -= f * A[(size_t)c * n + j];
        I[(size_t)r * n + j] -= f * I[(size_t)c * n + j];
      }
    }
  }
  A.swap(I);
  return true;
}

Space1D make_space(int k) {
  Space1D s;
  s.N = k + 1;
  const int N = s.N;
  s.nodes = lgl_nodes(k);
  vec g, w, V, D;
  gauss_rule(N, g, w);
  lagrange(s.nodes, g, V, D);
  s.mass.assign((size_t)N * N, 0.0L);
  s.stiff.assign((size_t)N * N, 0.0L);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      ld m = 0.0L, a = 0.0L;
      for (int q = 0; q < N; ++q) {
        m += w[q] * V[(size_t)q * N + i] * V[(size_t)q * N + j];
        a += w[q] * D[(size_t)q * N + i] * D[(size_t)q * N + j];
      }
      s.mass[(size_t)i * N + j] = m;
      s.stiff[(size_t)i * N + j] = a;
    }
  vec e0{0.0L}, e1{1.0L}, V0, D0, V1, D1;
  lagrange(s.nodes, e0, V0, D0);
  lagrange(s.nodes, e1, V1, D1);
  s.d0 = D0;
  s.d1 = D1;
  s.mass_inv = s.mass;
  invert(s.mass_inv, N);
  return s;
}

Laplace1D make_laplace_1d(const Space1D& s, ld h, ld tau) {
  const int N = s.N;
  Laplace1D L;
  L.A0.assign((size_t)N * N, 0.0L);
  L.cr.assign(N, 0.0L);
  L.cl.assign(N, 0.0L);
  L.gr.assign(N, 0.0L);
  L.gl.assign(N, 0.0L);
  const ld ih = 1.0L / h;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      ld a = s.stiff[(size_t)i * N + j] * ih;
      // right face of the element (it is the '-' side): value p(1) = x_{N-1}
      if (j == N - 1) a -= 0.5L * s.d1[i] * ih;
      if (i == N - 1) a -= 0.5L * s.d1[j] * ih;
      if (i == N - 1 && j == N - 1) a += tau;
      // left face (the element is the '+' side): value p(0) = x_0
      if (j == 0) a += 0.5L * s.d0[i] * ih;
      if (i == 0) a += 0.5L * s.d0[j] * ih;
      if (i == 0 && j == 0) a += tau;
      L.A0[(size_t)i * N + j] = a;
    }
  for (int i = 0; i < N; ++i) {
    L.cr[i] = 0.5L * s.d1[i] * ih - (i == N - 1 ? tau : 0.0L);
    L.cl[i] = -0.5L * s.d0[i] * ih - (i == 0 ? tau : 0.0L);
    L.gr[i] = -0.5L * s.d0[i] * ih;
    L.gl[i] = 0.5L * s.d1[i] * ih;
  }
  return L;
}

Div1D make_div_1d(const Space1D& su, const Space1D& sp) {
  const int Nu = su.N, Np = sp.N;
  vec g, w, Vu, Du, Vp, Dp;
  gauss_rule(Nu, g, w);
  lagrange(su.nodes, g, Vu, Du);
  lagrange(sp.nodes, g, Vp, Dp);
  Div1D d;
  d.R.assign((size_t)Np * Nu, 0.0L);
  d.Mpu.assign((size_t)Np * Nu, 0.0L);
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Nu; ++j) {
      ld m = 0.0L, c = 0.0L;
      for (int q = 0; q < Nu; ++q) {
        m += w[q] * Vp[(size_t)q * Np + i] * Vu[(size_t)q * Nu + j];
        c += w[q] * Dp[(size_t)q * Np + i] * Vu[(size_t)q * Nu + j];
      }
      ld r = -c;
      if (i == Np - 1 && j == Nu - 1) r += 0.5L;  // right face, own trace
      if (i == 0 && j == 0) r -= 0.5L;            // left face, own trace
      d.R[(size_t)i * Nu + j] = r;
      d.Mpu[(size_t)i * Nu + j] = m;
    }
  return d;
}

Grad1D make_grad_1d(const Space1D& su, const Space1D& sp) {
  const int Nu = su.N, Np = sp.N;
  vec g, w, Vu, Du, Vp, Dp;
  gauss_rule(Nu, g, w);
  lagrange(su.nodes, g, Vu, Du);
  lagrange(sp.nodes, g, Vp, Dp);
  Grad1D d;
  d.G.assign((size_t)Nu * Np, 0.0L);
  d.Mup.assign((size_t)Nu * Np, 0.0L);
  for (int i = 0; i < Nu; ++i)
    for (int j = 0; j < Np; ++j) {
      ld m = 0.0L, c = 0.0L;
      for (int q = 0; q < Nu; ++q) {
        m += w[q] * Vu[(size_t)q * Nu + i] * Vp[(size_t)q * Np + j];
        c += w[q] * Du[(size_t)q * Nu + i] * Vp[(size_t)q * Np + j];
      }
      ld r = -c;
      if (i == Nu - 1 && j == Np - 1) r += 0.5L;
      if (i == 0 && j == 0) r -= 0.5L;
      d.G[(size_t)i * Np + j] = r;
      d.Mup[(size_t)i * Np + j] = m;
    }
  return d;
}

Quad1D make_quad_1d(const Space1D& s, int Q) {
  Quad1D q;
  q.Q = Q;
  vec g;
  gauss_rule(Q, g, q.w);
  lagrange(s.nodes, g, q.S, q.D);
  return q;
}

vec make_prolongation_1d(const Space1D& s, int c) {
  vec xs(s.N), V, D;
  for (int i = 0; i < s.N; ++i) xs[i] = 0.5L * (s.nodes[i] + c);
  lagrange(s.nodes, xs, V, D);
  return V;
}

}  // namespace dgns
