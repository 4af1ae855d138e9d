// C ABI of libdgns (include/dgns.h): context set-up, table construction,
// host/device pointer staging, operator entry points and the solvers.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

using namespace dgns;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

// Every device allocation of the library goes through dev_malloc / dev_free:
// a test hook can make the n-th allocation from now fail as if the device
// were out of memory, and a count of live allocations lets tests check that
// the failure paths free what they allocated.
std::atomic<long long> g_fail_alloc_in{0};  // 0: disarmed
std::atomic<long long> g_live_allocs{0};

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
  *p = nullptr;
  long long n = g_fail_alloc_in.load();
  while (n > 0 && !g_fail_alloc_in.compare_exchange_weak(n, n - 1)) {
  }
  if (n == 1) return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess && *p) g_live_allocs.fetch_add(1);
  return e;
}
template <class T>
cudaError_t dev_malloc(T** p, size_t bytes) {
  void* v = nullptr;
  const cudaError_t e = dev_malloc_raw(&v, bytes);
  *p = static_cast<T*>(v);
  return e;
}
void dev_free(void* p) {
  if (p && cudaFree(p) == cudaSuccess) g_live_allocs.fetch_sub(1);
}

#define DG_CUDA(call)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? DGNS_ERR_OOM : DGNS_ERR_CUDA,     \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

#define DG_TRY(call)                                                  \
  do {                                                                \
    int rc_ = (call);                                                 \
    if (rc_ != 0) {                                                   \
      if (rc_ == DGNS_ERR_CUDA) {                                     \
        cudaError_t e_ = cudaGetLastError();                          \
        return fail(rc_, std::string(#call) + ": " + cudaGetErrorString(e_)); \
      }                                                               \
      if (g_err.empty()) g_err = #call;                               \
      return rc_;                                                     \
    }                                                                 \
  } while (0)

}  // namespace

namespace dgns {

int set_error(int code, const std::string& msg) { return fail(code, msg); }
void clear_error() { g_err.clear(); }
bool error_empty() { return g_err.empty(); }

void build_lap(const Space1D& s, const double h[3], double pf, double coef, double mass_factor,
               LapHost& L) {
  L.N = s.N;
  const int N = s.N, k = s.N - 1;
  for (int d = 0; d < 3; ++d) {
    const ld tau = (ld)pf * (k + 1) * (k + 1) / (ld)h[d];
    Laplace1D l1 = make_laplace_1d(s, (ld)h[d], tau);
    ld ht = 1.0L;
    for (int e = 0; e < 3; ++e)
      if (e != d) ht *= (ld)h[e];
    const ld f = (ld)coef * ht;
    for (int i = 0; i < N * N; ++i) {
      ld a = f * l1.A0[i];
      if (d == 0 && mass_factor != 0.0) a += (ld)mass_factor * (ld)h[0] * (ld)h[1] * (ld)h[2] * s.mass[i];
      L.A0[d][i] = (double)a;
    }
    for (int i = 0; i < N; ++i) {
      L.cr[d][i] = (double)(f * l1.cr[i]);
      L.cl[d][i] = (double)(f * l1.cl[i]);
      L.gr[d][i] = (double)(f * l1.gr[i]);
      L.gl[d][i] = (double)(f * l1.gl[i]);
    }
  }
  for (int i = 0; i < N * N; ++i) L.M[i] = (double)s.mass[i];
}

}  // namespace dgns

namespace {

// Diagonal pattern (identical for every cell of the uniform mesh), from the
// same factorisation in long double.
std::vector<double> lap_diagonal(const Space1D& s, const double h[3], double pf, const int n[3]) {
  const int N = s.N, k = N - 1;
  std::vector<ld> t[3];
  for (int d = 0; d < 3; ++d) {
    const ld tau = (ld)pf * (k + 1) * (k + 1) / (ld)h[d];
    Laplace1D l1 = make_laplace_1d(s, (ld)h[d], tau);
    ld ht = 1.0L;
    for (int e = 0; e < 3; ++e)
      if (e != d) ht *= (ld)h[e];
    t[d].assign(N, 0.0L);
    for (int a = 0; a < N; ++a) {
      ld v = l1.A0[(size_t)a * N + a];
      if (n[d] == 1) {  // the cell is its own neighbour
        if (a == 0) v += l1.cr[0] + l1.gl[0];
        if (a == N - 1) v += l1.cl[N - 1] + l1.gr[N - 1];
      }
      t[d][a] = ht * v;
    }
  }
  std::vector<double> out((size_t)N * N * N);
  for (int z = 0; z < N; ++z)
    for (int y = 0; y < N; ++y)
      for (int x = 0; x < N; ++x) {
        const ld mx = s.mass[(size_t)x * N + x], my = s.mass[(size_t)y * N + y],
                 mz = s.mass[(size_t)z * N + z];
        out[(size_t)x + N * (y + (size_t)N * z)] =
            (double)(t[0][x] * my * mz + mx * t[1][y] * mz + mx * my * t[2][z]);
      }
  return out;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + nb && pb < pa + na;
}

// Host-pointer staging: device pointers pass through; host pointers are
// copied into context-owned device buffers (grown on demand).
struct Staged {
  dgns_ctx* c;
  bool any_host = false;
  bool in_copied = false;
  struct Out {
    void* host;
    void* dev;
    size_t bytes;
  };
  std::vector<Out> outs;
  int slot = 0;
  explicit Staged(dgns_ctx* ctx) : c(ctx) {}
  int in(const void* p, size_t bytes, const void** dev) {
    if (is_device_ptr(p)) {
      *dev = p;
      return 0;
    }
    void* buf;
    int rc = grab(bytes, &buf);
    if (rc) return rc;
    DG_CUDA(cudaMemcpyAsync(buf, p, bytes, cudaMemcpyHostToDevice, c->s));
    if (!c->stage_ev) DG_CUDA(cudaEventCreateWithFlags(&c->stage_ev, cudaEventDisableTiming));
    DG_CUDA(cudaEventRecord(c->stage_ev, c->s));
    in_copied = true;
    *dev = buf;
    any_host = true;
    return 0;
  }
  int out(void* p, size_t bytes, void** dev) {
    if (is_device_ptr(p)) {
      *dev = p;
      return 0;
    }
    void* buf;
    int rc = grab(bytes, &buf);
    if (rc) return rc;
    outs.push_back({p, buf, bytes});
    *dev = buf;
    any_host = true;
    return 0;
  }
  // read and written: copied in like `in` and back like `out`
  int inout(void* p, size_t bytes, void** dev) {
    if (is_device_ptr(p)) {
      *dev = p;
      return 0;
    }
    const void* d;
    int rc = in(p, bytes, &d);
    if (rc) return rc;
    outs.push_back({p, const_cast<void*>(d), bytes});
    *dev = const_cast<void*>(d);
    return 0;
  }
  int grab(size_t bytes, void** buf) {
    if (slot >= 4) return fail(DGNS_ERR_INVALID_ARG, "too many host-pointer arguments");
    if (c->stage_cap[slot] < bytes) {
      if (c->stage[slot]) {
        cudaStreamSynchronize(c->s);
        dev_free(c->stage[slot]);
        c->stage[slot] = nullptr;
        c->stage_cap[slot] = 0;
      }
      DG_CUDA(dev_malloc(&c->stage[slot], bytes));
      c->stage_cap[slot] = bytes;
    }
    *buf = c->stage[slot++];
    return 0;
  }
  // Host outputs: copied back, complete when the call returns.  Host inputs
  // only: the call returns once they are copied (the caller may reuse them);
  // the kernels run on, stream-ordered before any later use of the staging
  // buffers.
  int finish() {
    for (auto& o : outs) DG_CUDA(cudaMemcpyAsync(o.host, o.dev, o.bytes, cudaMemcpyDeviceToHost, c->s));
    if (!outs.empty())
      DG_CUDA(cudaStreamSynchronize(c->s));
    else if (in_copied)
      DG_CUDA(cudaEventSynchronize(c->stage_ev));
    return 0;
  }
};

int check_space(int space) {
  if (space != DGNS_SPACE_U && space != DGNS_SPACE_P)
    return fail(DGNS_ERR_INVALID_ARG, "space must be DGNS_SPACE_U or DGNS_SPACE_P");
  return 0;
}

void cheb_coeffs(double lam_max, double range, int step, double* rho, double* c1, double* c2) {
  const double lmin = lam_max / range;
  const double theta = 0.5 * (lam_max + lmin), delta = 0.5 * (lam_max - lmin);
  const double sigma = theta / delta;
  if (step == 0) {
    *rho = 1.0 / sigma;
    *c1 = 0.0;
    *c2 = 1.0 / theta;
    return;
  }
  const double rnew = 1.0 / (2.0 * sigma - *rho);
  *c1 = rnew * (*rho);
  *c2 = 2.0 * rnew / delta;
  *rho = rnew;
}

size_t mg_bytes(const dgns_ctx* c) { return c->mg_prec == 32 ? 4 : 8; }

// Chebyshev smoothing on a level; x0 == nullptr means a zero initial guess.
// Returns the buffer holding the result (xa or xb).
int smooth(dgns_ctx* c, Level& L, void* x0, int steps, double range, void** result) {
  const bool f32 = c->mg_prec == 32;
  const int N = c->N[DGNS_SPACE_P];
  double rho = 0, c1 = 0, c2 = 0;
  if (f32 && steps >= 1 && steps <= SMOOTH_MAX_STEPS) {
    // small levels: every step of the call in one launch
    SmoothPlan plan;
    plan.nsteps = steps;
    plan.zero_guess = x0 == nullptr;
    for (int k = 0; k < steps; ++k) {
      cheb_coeffs(L.lambda_max, range, k, &rho, &c1, &c2);
      plan.c1[k] = (float)c1;
      plan.c2[k] = (float)c2;
    }
    void* out = (x0 == nullptr || x0 == L.xb) ? L.xa : L.xb;
    const int rc = laplace_plane_smooth(L.m, (const float*)L.b, (const float*)x0, (float*)out,
                                        (const float*)L.dinv, L.lap, plan, c->s);
    if (rc >= 0) {
      DG_TRY(rc);
      *result = out;
      return 0;
    }
    rho = c1 = c2 = 0;
  }
  void* cur;
  void* oth;
  void* prev = nullptr;
  int first_step;
  if (x0 == nullptr) {
    cheb_coeffs(L.lambda_max, range, 0, &rho, &c1, &c2);
    DG_TRY(cheb_first(f32, L.b, L.dinv, L.xa, L.n, N * N * N, c2, c->s));
    cur = L.xa;
    oth = L.xb;
    first_step = 1;
  } else {
    cur = x0;
    oth = (x0 == L.xa) ? L.xb : L.xa;
    first_step = 0;
  }
  for (int k = first_step; k < steps; ++k) {
    cheb_coeffs(L.lambda_max, range, k, &rho, &c1, &c2);
    EpiHost ea;
    ea.b = L.b;
    ea.dinv = L.dinv;
    // prev is null at k == 1 from a zero guess: the kernel reads it as zero
    ea.xprev = (k == 0) ? nullptr : prev;
    ea.c1 = c1;
    ea.c2 = c2;
    DG_TRY(laplace_apply(f32, L.m, 1, cur, oth, L.lap, EPI_CHEB, ea, c->s));
    prev = cur;
    void* t = cur;
    cur = oth;
    oth = t;
  }
  *result = cur;
  return 0;
}

int vcycle(dgns_ctx* c, int lvl, const dgns_solve_params* prm, void** result) {
  Level& L = c->levels[lvl];
  const bool f32 = c->mg_prec == 32;
  const int N = c->N[DGNS_SPACE_P];
  if (lvl == 0) return smooth(c, L, nullptr, prm->cheb_coarse_iters, prm->smoothing_range, result);
  void* x;
  DG_TRY(smooth(c, L, nullptr, prm->cheb_degree, prm->smoothing_range, &x));
  EpiHost er;
  er.b = L.b;
  DG_TRY(laplace_apply(f32, L.m, 1, x, L.r, L.lap, EPI_RESID, er, c->s));
  Level& C = c->levels[lvl - 1];
  DG_TRY(restrict_fine(f32, N, C.m, L.r, C.b, c->P0, c->P1, c->s));
  void* xc;
  DG_TRY(vcycle(c, lvl - 1, prm, &xc));
  DG_TRY(prolongate(f32, N, C.m, xc, x, c->P0, c->P1, true, c->s));
  return smooth(c, L, x, prm->cheb_degree, prm->smoothing_range, result);
}

int read_scalars(dgns_ctx* c) {
  DG_CUDA(cudaMemcpyAsync(c->h_scal, c->red.scal, S_NSLOTS * sizeof(double), cudaMemcpyDeviceToHost, c->s));
  DG_CUDA(cudaStreamSynchronize(c->s));
  return 0;
}

// Largest eigenvalue of the Lanczos tridiagonal matrix (Sturm bisection).
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int n = (int)a.size();
  double hi = 0.0;
  for (int i = 0; i < n; ++i) {
    double r = fabs(a[i]);
    if (i > 0) r += fabs(b[i - 1]);
    if (i < n - 1) r += fabs(b[i]);
    hi = fmax(hi, r);
  }
  double lo = 0.0;
  auto count_below = [&](double x) {
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < n; ++i) {
      double off = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
      q = (a[i] - x) - (i > 0 ? off / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0) ++cnt;
    }
    return cnt;
  };
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= n) hi = mid;
    else lo = mid;
  }
  return hi;
}

// lambda_max of D^-1 A on a level by the Lanczos process behind CG (FP64).
int estimate_lambda(dgns_ctx* c, Level& L, double* lam) {
  const int iters = 24;
  const long long n = L.n;
  const int N = c->N[DGNS_SPACE_P];
  std::vector<double> hb((size_t)n);
  unsigned long long st = 0x9E3779B97F4A7C15ull;
  double mean = 0.0;
  for (long long i = 0; i < n; ++i) {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    hb[(size_t)i] = (double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    mean += hb[(size_t)i];
  }
  mean /= (double)n;
  for (auto& v : hb) v -= mean;
  double* x = nullptr;
  DG_CUDA(dev_malloc(&x, (size_t)n * sizeof(double)));
  struct FreeOnExit {  // the early returns below must not leak x
    double* p;
    cudaStream_t s;
    ~FreeOnExit() {
      cudaStreamSynchronize(s);
      dev_free(p);
    }
  } guard{x, c->s};
  DG_CUDA(cudaMemsetAsync(x, 0, (size_t)n * sizeof(double), c->s));
  DG_CUDA(cudaMemcpyAsync(c->r, hb.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice, c->s));
  std::vector<double> alpha, beta;
  DG_TRY(cheb_first(false, c->r, L.dinv64, c->z, n, N * N * N, 1.0, c->s));
  DG_TRY(cg_direction(c->p, c->z, n, c->red, true, c->s));
  DG_TRY(dot(c->r, c->z, n, c->red, S_RZ, c->s));
  int rc = 0;
  for (int it = 0; it < iters; ++it) {
    if ((rc = laplace_apply(false, L.m, 1, c->p, c->Ap, L.lap, EPI_NONE, EpiHost(), c->s))) break;
    if ((rc = dot(c->p, c->Ap, n, c->red, S_PAP, c->s))) break;
    if ((rc = read_scalars(c))) break;
    const double rz = c->h_scal[S_RZ], pap = c->h_scal[S_PAP];
    if (!(pap > 0.0) || !(rz > 0.0)) break;
    alpha.push_back(rz / pap);
    if ((rc = cg_update(x, c->r, c->p, c->Ap, n, c->red, c->s))) break;
    if ((rc = cheb_first(false, c->r, L.dinv64, c->z, n, N * N * N, 1.0, c->s))) break;
    if ((rc = dot(c->r, c->z, n, c->red, S_RZNEW, c->s))) break;
    if ((rc = read_scalars(c))) break;
    beta.push_back(c->h_scal[S_RZNEW] / rz);
    if (!(c->h_scal[S_RZNEW] > 1e-300 * rz)) break;
    if ((rc = cg_direction(c->p, c->z, n, c->red, false, c->s))) break;
  }
  if (rc) return rc;
  const int m = (int)alpha.size();
  if (m == 0) return fail(DGNS_ERR_NONFINITE, "eigenvalue estimate: no Lanczos step");
  std::vector<double> ta(m), tb(m > 1 ? m - 1 : 0);
  for (int j = 0; j < m; ++j) {
    ta[j] = 1.0 / alpha[j] + (j > 0 ? beta[j - 1] / alpha[j - 1] : 0.0);
    if (j < m - 1) tb[j] = sqrt(beta[j]) / alpha[j];
  }
  *lam = 1.2 * tridiag_max_eig(ta, tb);
  return 0;
}

void free_ctx(dgns_ctx* c) {
  if (!c) return;
  if (c->s) cudaStreamSynchronize(c->s);
  for (int i = 0; i < 2; ++i) dev_free(c->d_diag[i]);
  for (auto& L : c->levels) {
    dev_free(L.dinv);
    dev_free(L.dinv64);
    dev_free(L.xa);
    dev_free(L.xb);
    dev_free(L.b);
    dev_free(L.r);
  }
  dev_free(c->r);
  dev_free(c->z);
  dev_free(c->p);
  dev_free(c->Ap);
  dev_free(c->conv_face);
  dev_free(c->lap_face);
  dev_free(c->red.part);
  dev_free(c->red.scal);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  for (int i = 0; i < 4; ++i) dev_free(c->stage[i]);
  for (int i = 0; i < 3; ++i) dev_free(c->rwork[i]);
  dev_free(c->d_expmax);
  if (c->stage_ev) cudaEventDestroy(c->stage_ev);
  if (c->vc_exec) cudaGraphExecDestroy(c->vc_exec);
  if (c->gs) cudaStreamDestroy(c->gs);
  delete c;
}

int alloc_cg(dgns_ctx* c, long long n) {
  if (n <= c->cg_cap) return 0;
  // the captured V-cycle graph refers to the old work vectors
  if (c->vc_exec) {
    cudaStreamSynchronize(c->s);
    cudaGraphExecDestroy(c->vc_exec);
    c->vc_exec = nullptr;
  }
  dev_free(c->r);
  dev_free(c->z);
  dev_free(c->p);
  dev_free(c->Ap);
  c->r = c->z = c->p = c->Ap = nullptr;
  const size_t b = (size_t)n * sizeof(double);
  DG_CUDA(dev_malloc(&c->r, b));
  DG_CUDA(dev_malloc(&c->z, b));
  DG_CUDA(dev_malloc(&c->p, b));
  DG_CUDA(dev_malloc(&c->Ap, b));
  c->cg_cap = n;
  return 0;
}

int setup_mg(dgns_ctx* c) {
  const int kp = c->k[DGNS_SPACE_P];
  const int N = kp + 1, N3 = N * N * N;
  const Space1D& s = c->sp1[DGNS_SPACE_P];
  std::vector<int> ns[3];
  int n[3] = {c->m.nx, c->m.ny, c->m.nz};
  std::vector<std::vector<int>> meshes;
  meshes.push_back({n[0], n[1], n[2]});
  const int cn = c->d.mg_coarse_n > 0 ? c->d.mg_coarse_n : 2;
  while (n[0] % 2 == 0 && n[1] % 2 == 0 && n[2] % 2 == 0 && n[0] / 2 >= cn && n[1] / 2 >= cn &&
         n[2] / 2 >= cn && (int)meshes.size() < DGNS_MAX_LEVELS) {
    for (int d = 0; d < 3; ++d) n[d] /= 2;
    meshes.push_back({n[0], n[1], n[2]});
  }
  const int nl = (int)meshes.size();
  c->levels.resize(nl);
  const size_t tb = mg_bytes(c);
  for (int i = 0; i < nl; ++i) {
    const std::vector<int>& mm = meshes[nl - 1 - i];  // level 0 = coarsest
    Level& L = c->levels[i];
    L.m.nx = mm[0];
    L.m.ny = mm[1];
    L.m.nz = mm[2];
    L.m.E = (long long)mm[0] * mm[1] * mm[2];
    L.m.set_divisors();
    L.n = L.m.E * N3;
    for (int d = 0; d < 3; ++d) L.h[d] = (c->d.hi[d] - c->d.lo[d]) / mm[d];
    build_lap(s, L.h, c->d.penalty_factor, 1.0, 0.0, L.lap);
    std::vector<double> dg = lap_diagonal(s, L.h, c->d.penalty_factor, mm.data());
    std::vector<double> inv64(N3);
    std::vector<float> inv32(N3);
    for (int j = 0; j < N3; ++j) {
      inv64[j] = 1.0 / dg[j];
      inv32[j] = (float)inv64[j];
    }
    DG_CUDA(dev_malloc(&L.dinv64, N3 * sizeof(double)));
    DG_CUDA(cudaMemcpy(L.dinv64, inv64.data(), N3 * sizeof(double), cudaMemcpyHostToDevice));
    DG_CUDA(dev_malloc(&L.dinv, N3 * tb));
    DG_CUDA(cudaMemcpy(L.dinv, tb == 4 ? (const void*)inv32.data() : (const void*)inv64.data(), N3 * tb,
                       cudaMemcpyHostToDevice));
    DG_CUDA(dev_malloc(&L.xa, L.n * tb));
    DG_CUDA(dev_malloc(&L.xb, L.n * tb));
    DG_CUDA(dev_malloc(&L.b, L.n * tb));
    DG_CUDA(dev_malloc(&L.r, L.n * tb));
  }
  vec P0 = make_prolongation_1d(s, 0), P1 = make_prolongation_1d(s, 1);
  for (int i = 0; i < N * N; ++i) {
    c->P0[i] = (double)P0[i];
    c->P1[i] = (double)P1[i];
  }
  for (auto& L : c->levels) DG_TRY(estimate_lambda(c, L, &L.lambda_max));
  return 0;
}

// z = M^-1 r; with dot_slot >= 0 also scal[dot_slot] = (r, z) (in the
// FP32 V-cycle's last pass over z, summed as dot() sums it).
int precondition(dgns_ctx* c, const double* r, double* z, const dgns_solve_params* prm, long long n,
                 int dot_slot = -1) {
  if (c->mg_prec == 0 || c->levels.empty()) {
    DG_CUDA(cudaMemcpyAsync(z, r, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
  } else {
    const bool f32 = c->mg_prec == 32;
    Level& F = c->levels.back();
    DG_TRY(convert_shift(r, false, F.b, f32, n, nullptr, 0, c->s));
    void* x;
    DG_TRY(vcycle(c, (int)c->levels.size() - 1, prm, &x));
    if (prm->project_mean) {
      if (f32) DG_TRY(sum_f32((const float*)x, n, c->red, S_SUM, c->s));
      else DG_TRY(sum((const double*)x, n, c->red, S_SUM, c->s));
    }
    const int shift = prm->project_mean ? S_SUM : -1;
    if (f32 && dot_slot >= 0) return widen_shift_dot((const float*)x, z, n, c->red, shift, r, dot_slot, c->s);
    DG_TRY(convert_shift(x, f32, z, false, n, shift >= 0 ? &c->red : nullptr, shift, c->s));
    if (dot_slot >= 0) DG_TRY(dot(r, z, n, c->red, dot_slot, c->s));
    return 0;
  }
  if (prm->project_mean) {
    DG_TRY(sum(z, n, c->red, S_SUM, c->s));
    DG_TRY(convert_shift(z, false, z, false, n, &c->red, S_SUM, c->s));
  }
  if (dot_slot >= 0) DG_TRY(dot(r, z, n, c->red, dot_slot, c->s));
  return 0;
}

// The CG preconditioner r -> z on the context's work vectors, with
// scal[S_RZNEW] = (r, z), replayed from a CUDA graph: one V-cycle is ~10
// launches per level, and on the coarse levels launch latency dominates.
// The first call for a parameter set runs eagerly (it also sets kernel
// attributes), then captures the same sequence.
int precondition_cg(dgns_ctx* c, const dgns_solve_params* prm, long long n) {
  if (c->mg_prec == 0 || c->levels.empty()) return precondition(c, c->r, c->z, prm, n, S_RZNEW);
  const bool same = c->vc_exec && c->vc_key[0] == prm->cheb_degree && c->vc_key[1] == prm->cheb_coarse_iters &&
                    c->vc_key[2] == prm->project_mean && c->vc_range == prm->smoothing_range;
  if (same) {
    DG_CUDA(cudaGraphLaunch(c->vc_exec, c->s));
    return 0;
  }
  DG_TRY(precondition(c, c->r, c->z, prm, n, S_RZNEW));
  if (!c->gs) DG_CUDA(cudaStreamCreateWithFlags(&c->gs, cudaStreamNonBlocking));
  if (c->vc_exec) {
    cudaGraphExecDestroy(c->vc_exec);
    c->vc_exec = nullptr;
  }
  cudaStream_t saved = c->s;
  DG_CUDA(cudaStreamBeginCapture(c->gs, cudaStreamCaptureModeThreadLocal));
  c->s = c->gs;
  const int rc = precondition(c, c->r, c->z, prm, n, S_RZNEW);
  c->s = saved;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->gs, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(DGNS_ERR_CUDA, std::string("V-cycle capture: ") + cudaGetErrorString(e));
  const cudaError_t e2 = cudaGraphInstantiate(&c->vc_exec, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    c->vc_exec = nullptr;
    return fail(DGNS_ERR_CUDA, std::string("V-cycle graph: ") + cudaGetErrorString(e2));
  }
  c->vc_key[0] = prm->cheb_degree;
  c->vc_key[1] = prm->cheb_coarse_iters;
  c->vc_key[2] = prm->project_mean;
  c->vc_range = prm->smoothing_range;
  return 0;
}

}  // namespace

// =============================================================== C ABI ====
extern "C" {

void dgns_default_desc(dgns_mesh_desc* d) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  for (int i = 0; i < 3; ++i) {
    d->n_elem[i] = 4;
    d->lo[i] = -3.14159265358979323846;
    d->hi[i] = 3.14159265358979323846;
  }
  d->degree = 3;
  d->degree_p = -1;
  d->n_q_conv = 0;
  d->penalty_factor = 1.0;
  d->nu = 1.0 / 1600.0;
  d->mg_coarse_n = 2;
  d->mg_precision = 32;
}

void dgns_default_solve_params(dgns_solve_params* p) {
  if (!p) return;
  p->rel_tol = 1e-10;
  p->abs_tol = 0.0;
  p->max_iter = 200;
  p->cheb_degree = 5;
  p->smoothing_range = 20.0;
  p->cheb_coarse_iters = 20;
  p->project_mean = 1;
  p->use_initial_guess = 0;
}

const char* dgns_status_string(int s) {
  switch (s) {
    case DGNS_OK: return "ok";
    case DGNS_ERR_INVALID_ARG: return "invalid argument";
    case DGNS_ERR_CUDA: return "CUDA error";
    case DGNS_ERR_OOM: return "out of device memory";
    case DGNS_ERR_NOT_CONVERGED: return "solver did not converge";
    case DGNS_ERR_NONFINITE: return "non-finite value in solver";
    case DGNS_ERR_ALIAS: return "destination aliases a source";
    case DGNS_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

const char* dgns_last_error(void) { return g_err.c_str(); }

int dgns_create(const dgns_mesh_desc* desc, void* stream, dgns_ctx** out) {
  g_err.clear();
  if (!out) return fail(DGNS_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (!desc) return fail(DGNS_ERR_INVALID_ARG, "desc is null");
  dgns_mesh_desc d = *desc;
  if (d.degree_p < 0) d.degree_p = d.degree - 1;
  if (d.penalty_factor == 0.0) d.penalty_factor = 1.0;
  if (d.degree < 1 || d.degree > DGNS_MAX_DEGREE || d.degree_p < 1 || d.degree_p > DGNS_MAX_DEGREE)
    return fail(DGNS_ERR_INVALID_ARG, "degree and degree_p must lie in 1..11");
  for (int i = 0; i < 3; ++i) {
    if (d.n_elem[i] < 1) return fail(DGNS_ERR_INVALID_ARG, "n_elem must be >= 1");
    if (!(d.hi[i] > d.lo[i])) return fail(DGNS_ERR_INVALID_ARG, "hi must exceed lo");
  }
  if (d.mg_precision != 0 && d.mg_precision != 32 && d.mg_precision != 64)
    return fail(DGNS_ERR_INVALID_ARG, "mg_precision must be 0, 32 or 64");
  if (d.fp64_mode < 0 || d.fp64_mode > 2) return fail(DGNS_ERR_INVALID_ARG, "fp64_mode must be 0, 1 or 2");
  if ((long long)d.n_elem[0] * d.n_elem[1] * d.n_elem[2] * 3 >= (1LL << 31))
    return fail(DGNS_ERR_UNSUPPORTED, "meshes with 3 * cells >= 2^31 are not supported");
  const int Q = d.n_q_conv > 0 ? d.n_q_conv : (3 * (d.degree + 1)) / 2;
  if (Q != (3 * (d.degree + 1)) / 2 && Q != d.degree + 1)
    return fail(DGNS_ERR_UNSUPPORTED, "n_q_conv must be floor(3(k+1)/2) or k+1");
  d.n_q_conv = Q;
  int device = 0;
  DG_CUDA(cudaGetDevice(&device));
  dgns_ctx* c = new dgns_ctx();
  c->d = d;
  c->s = (cudaStream_t)stream;
  c->device = device;
  c->m.nx = d.n_elem[0];
  c->m.ny = d.n_elem[1];
  c->m.nz = d.n_elem[2];
  c->m.E = (long long)d.n_elem[0] * d.n_elem[1] * d.n_elem[2];
  c->m.set_divisors();
  for (int i = 0; i < 3; ++i) c->h[i] = (d.hi[i] - d.lo[i]) / d.n_elem[i];
  c->k[0] = d.degree;
  c->k[1] = d.degree_p;
  for (int sp = 0; sp < 2; ++sp) {
    c->N[sp] = c->k[sp] + 1;
    const int N = c->N[sp];
    c->n[sp] = c->m.E * N * N * N;
    c->sp1[sp] = make_space(c->k[sp]);
    build_lap(c->sp1[sp], c->h, d.penalty_factor, 1.0, 0.0, c->lap[sp]);
    c->diag[sp] = lap_diagonal(c->sp1[sp], c->h, d.penalty_factor, d.n_elem);
    const Space1D& s = c->sp1[sp];
    for (int dd = 0; dd < 3; ++dd)
      for (int i = 0; i < N * N; ++i) {
        // one direction carries the Jacobian h_x h_y h_z
        const ld jac = dd == 0 ? (ld)c->h[0] * c->h[1] * c->h[2] : 1.0L;
        c->mass3[sp][dd][i] = (double)(jac * s.mass[i]);
        c->minv3[sp][dd][i] = (double)(s.mass_inv[i] / jac);
      }
  }
  // divergence / gradient tables (test k_p, trial k_u)
  {
    const Space1D& su = c->sp1[0];
    const Space1D& sp = c->sp1[1];
    Div1D dv = make_div_1d(su, sp);
    Grad1D gr = make_grad_1d(su, sp);
    c->div.Nu = c->grad.Nu = su.N;
    c->div.Np = c->grad.Np = sp.N;
    for (int dd = 0; dd < 3; ++dd) {
      ld ht = 1.0L;
      for (int e = 0; e < 3; ++e)
        if (e != dd) ht *= (ld)c->h[e];
      for (int i = 0; i < su.N * sp.N; ++i) {
        c->div.R[dd][i] = (double)(ht * dv.R[i]);
        c->grad.G[dd][i] = (double)(ht * gr.G[i]);
      }
      c->div.nbr[dd] = c->grad.nbr[dd] = (double)(0.5L * ht);
      c->div.nbl[dd] = c->grad.nbl[dd] = (double)(-0.5L * ht);
    }
    for (int i = 0; i < su.N * sp.N; ++i) {
      c->div.Mpu[i] = (double)dv.Mpu[i];
      c->grad.Mup[i] = (double)gr.Mup[i];
    }
  }
  {
    Quad1D q = make_quad_1d(c->sp1[0], Q);
    c->conv.N = c->sp1[0].N;
    c->conv.Q = Q;
    for (int i = 0; i < Q * c->conv.N; ++i) {
      c->conv.S[i] = (double)q.S[i];
      c->conv.D[i] = (double)q.D[i];
    }
    for (int i = 0; i < Q; ++i) c->conv.w[i] = (double)q.w[i];
    for (int dd = 0; dd < 3; ++dd) c->conv.h[dd] = c->h[dd];
  }
  {
    const Space1D& su = c->sp1[0];
    const int N = su.N;
    Quad1D q = make_quad_1d(su, N);
    c->proj.N = N;
    for (int i = 0; i < N * N; ++i) {
      c->proj.S[i] = (double)q.S[i];
      c->proj.D[i] = (double)q.D[i];
      c->proj.M[i] = (double)su.mass[i];
    }
    for (int i = 0; i < N; ++i) c->proj.w[i] = (double)q.w[i];
    for (int dd = 0; dd < 3; ++dd) c->proj.h[dd] = c->h[dd];
  }
  int rc = 0;
  auto bail = [&](int code) {
    free_ctx(c);
    return code;
  };
  for (int sp = 0; sp < 2; ++sp) {
    const size_t b = c->diag[sp].size() * sizeof(double);
    if (dev_malloc(&c->d_diag[sp], b) != cudaSuccess ||
        cudaMemcpy(c->d_diag[sp], c->diag[sp].data(), b, cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(DGNS_ERR_OOM, "table allocation failed"));
  }
  if (dev_malloc(&c->red.part, RED_BLOCKS * sizeof(double)) != cudaSuccess ||
      dev_malloc(&c->red.scal, S_NSLOTS * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&c->h_scal, S_NSLOTS * sizeof(double)) != cudaSuccess)
    return bail(fail(DGNS_ERR_OOM, "reduction buffers"));
  c->mg_prec = d.mg_precision;
  if (c->mg_prec != 0) {
    if ((rc = alloc_cg(c, c->n[DGNS_SPACE_P]))) return bail(rc);
    if ((rc = setup_mg(c))) return bail(rc);
  }
  *out = c;
  return 0;
}

int dgns_destroy(dgns_ctx* c) {
  free_ctx(c);
  return 0;
}

int dgns_set_stream(dgns_ctx* c, void* stream) {
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  c->s = (cudaStream_t)stream;
  return 0;
}

int dgns_debug_conv_mix(int period, int nnative) {
  if (period < -1 || (period > 0 && (nnative < 0 || nnative > period)))
    return fail(DGNS_ERR_INVALID_ARG, "period >= -1 and 0 <= nnative <= period");
  convective_set_mix(period, nnative);
  return 0;
}

int dgns_debug_laplace_f32_kernel(int variant) {
  if (variant < -1 || variant > 5) return fail(DGNS_ERR_INVALID_ARG, "variant must be in -1..5");
  laplace_plane_set_variant(variant);
  return 0;
}

long long dgns_debug_laplace_f32_timeouts(void) { return (long long)laplace_tma_timeouts(); }

int dgns_debug_fail_alloc(long long n) {
  if (n < 0) return fail(DGNS_ERR_INVALID_ARG, "n must be >= 0");
  g_fail_alloc_in.store(n);
  return 0;
}

long long dgns_debug_live_allocations(void) { return g_live_allocs.load(); }

int dgns_debug_widen_f32(const float* x, double* y, long long n) {
  if (n < 0 || (n > 0 && (!x || !y))) return fail(DGNS_ERR_INVALID_ARG, "widen: bad arguments");
  if (n == 0) return 0;
  DG_TRY(convert_shift(x, true, y, false, n, nullptr, -1, 0));
  DG_CUDA(cudaStreamSynchronize(0));
  return 0;
}

int dgns_sizes(const dgns_ctx* c, long long* nu, long long* np) {
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  if (nu) *nu = c->n[0];
  if (np) *np = c->n[1];
  return 0;
}

int dgns_nodes_1d(const dgns_ctx* c, int space, double* out) {
  if (!c || !out) return fail(DGNS_ERR_INVALID_ARG, "null argument");
  if (check_space(space)) return DGNS_ERR_INVALID_ARG;
  for (int i = 0; i < c->N[space]; ++i) out[i] = (double)c->sp1[space].nodes[i];
  return 0;
}

#define DG_NONNULL(...)                                                          \
  do {                                                                           \
    const void* ps_[] = {__VA_ARGS__};                                           \
    for (const void* p_ : ps_)                                                   \
      if (!p_) return fail(DGNS_ERR_INVALID_ARG, "null pointer argument");       \
  } while (0)

static bool aligned16(const void* a, const void* b) { return (((uintptr_t)a | (uintptr_t)b) & 15u) == 0; }

// Input range of the emulated arithmetic.  Double-float and triple-float
// values carry float's exponent: a loaded double keeps its full significand
// from 2^-74 up and overflows at 2^128.  In those modes every operator call
// measures the largest exponent of its input (one reduction and a read-back
// of one word, so these calls synchronise the stream); an input whose
// largest entry lies outside the window [2^lo, 2^hi] (room for the
// operator's own scaling above, and for entries 2^30 below the largest) is
// multiplied by an exact power of two into a work buffer, the operator runs
// on that copy and its result is scaled back (exactly, unless it leaves the
// double range).  Native FP64 skips all of it.
constexpr int kLinLo = -40, kLinHi = 90;     // linear operators
constexpr int kQuadLo = -20, kQuadHi = 45;   // the convective term (quadratic)

struct Ranged {
  dgns_ctx* c;
  explicit Ranged(dgns_ctx* ctx) : c(ctx) {}
  bool active() const { return c->d.fp64_mode != 0; }
  // shift (the input is to be multiplied by 2^-shift): 0 inside the window
  int measure(const void* x, long long n, int lo, int hi, int* shift) {
    *shift = 0;
    if (!active() || n == 0) return 0;
    if (!c->d_expmax) DG_CUDA(dev_malloc(&c->d_expmax, sizeof(unsigned)));
    if (exp_max((const double*)x, n, c->d_expmax, c->s)) return fail(DGNS_ERR_CUDA, "exp_max launch");
    unsigned e = 0;
    DG_CUDA(cudaMemcpyAsync(&e, c->d_expmax, sizeof(unsigned), cudaMemcpyDeviceToHost, c->s));
    DG_CUDA(cudaStreamSynchronize(c->s));
    if (e == 2047) return fail(DGNS_ERR_NONFINITE, "input holds a non-finite value");
    if (e == 0) return 0;                      // zero (or subnormal only): nothing to keep
    const int E = (int)e - 1023;               // 2^E <= max |x| < 2^(E+1)
    if (E < lo || E > hi) *shift = E;
    return 0;
  }
  // dst = x * 2^k in work buffer `slot` (grown on demand)
  int scaled(const void* x, long long n, int k, int slot, const double** dst) {
    const size_t bytes = (size_t)n * sizeof(double);
    if (c->rwork_cap[slot] < bytes) {
      if (c->rwork[slot]) {
        cudaStreamSynchronize(c->s);
        dev_free(c->rwork[slot]);
        c->rwork[slot] = nullptr;
        c->rwork_cap[slot] = 0;
      }
      DG_CUDA(dev_malloc(&c->rwork[slot], bytes));
      c->rwork_cap[slot] = bytes;
    }
    if (scale_pow2((const double*)x, (double*)c->rwork[slot], n, k, c->s)) return fail(DGNS_ERR_CUDA, "scale launch");
    *dst = (const double*)c->rwork[slot];
    return 0;
  }
  int rescale(void* y, long long n, int k) {
    if (k == 0) return 0;
    if (scale_pow2((const double*)y, (double*)y, n, k, c->s)) return fail(DGNS_ERR_CUDA, "scale launch");
    return 0;
  }
};

static int lap_like(dgns_ctx* c, double* dst, const double* src, int space, int ncomp, double coef,
                    double mass_factor) {
  const size_t bytes = (size_t)c->n[space] * ncomp * sizeof(double);
  if (overlaps(dst, bytes, src, bytes)) return fail(DGNS_ERR_ALIAS, "dst overlaps src");
  Staged st(c);
  const void* s;
  void* d;
  DG_TRY(st.in(src, bytes, &s));
  DG_TRY(st.out(dst, bytes, &d));
  if (!aligned16(d, s)) return fail(DGNS_ERR_INVALID_ARG, "dst and src must be 16-byte aligned");
  const LapHost* tab = &c->lap[space];
  LapHost scaled;
  if (coef != 1.0 || mass_factor != 0.0) {
    const double h[3] = {c->h[0], c->h[1], c->h[2]};
    build_lap(c->sp1[space], h, c->d.penalty_factor, coef, mass_factor, scaled);
    tab = &scaled;
  }
  const long long n = c->n[space] * ncomp;
  Ranged rg(c);
  int sh = 0;
  DG_TRY(rg.measure(s, n, kLinLo, kLinHi, &sh));
  if (sh) {
    const double* sc;
    DG_TRY(rg.scaled(s, n, -sh, 0, &sc));
    s = sc;
  }
  DG_TRY(laplace_apply(false, c->m, ncomp, s, d, *tab, EPI_NONE, EpiHost(), c->s, c->d.fp64_mode));
  DG_TRY(rg.rescale(d, n, sh));
  return st.finish();
}

int dgns_vmult_laplace(dgns_ctx* c, double* dst, const double* src, int space) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(dst, src);
  if (check_space(space)) return DGNS_ERR_INVALID_ARG;
  return lap_like(c, dst, src, space, 1, 1.0, 0.0);
}

static void build_broken_stiffness(const dgns_ctx* c, double coef, LapHost& L, int space);

int dgns_vmult_laplace_split(dgns_ctx* c, double* dst, const double* src, int space) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(dst, src);
  if (check_space(space)) return DGNS_ERR_INVALID_ARG;
  const size_t bytes = (size_t)c->n[space] * sizeof(double);
  if (overlaps(dst, bytes, src, bytes)) return fail(DGNS_ERR_ALIAS, "dst overlaps src");
  const Space1D& s1 = c->sp1[space];
  const int N = s1.N;
  const size_t fbytes = (size_t)6 * c->m.E * N * N * sizeof(double);
  if (c->lap_face_cap < fbytes) {
    dev_free(c->lap_face);
    c->lap_face = nullptr;
    c->lap_face_cap = 0;
    if (dev_malloc(&c->lap_face, fbytes) != cudaSuccess) {
      c->lap_face = nullptr;
      return fail(DGNS_ERR_OOM, "face buffer of the split SIPG evaluation");
    }
    c->lap_face_cap = fbytes;
  }
  Staged st(c);
  const void* sv;
  void* d;
  DG_TRY(st.in(src, bytes, &sv));
  DG_TRY(st.out(dst, bytes, &d));
  if (!aligned16(d, sv)) return fail(DGNS_ERR_INVALID_ARG, "dst and src must be 16-byte aligned");
  LapHost K;
  build_broken_stiffness(c, 1.0, K, space);
  SplitHost sh;
  sh.N = N;
  for (int i = 0; i < N; ++i) {
    sh.d0[i] = (double)s1.d0[i];
    sh.d1[i] = (double)s1.d1[i];
  }
  for (int i = 0; i < N * N; ++i) sh.M[i] = (double)s1.mass[i];
  for (int dd = 0; dd < 3; ++dd) {
    ld ht = 1.0L;
    for (int e = 0; e < 3; ++e)
      if (e != dd) ht *= (ld)c->h[e];
    sh.ih[dd] = (double)(1.0L / (ld)c->h[dd]);
    sh.tau[dd] = (double)((ld)c->d.penalty_factor * N * N / (ld)c->h[dd]);
    sh.area[dd] = (double)ht;
  }
  DG_TRY(laplace_apply(false, c->m, 1, sv, d, K, EPI_NONE, EpiHost(), c->s, ARITH_F64));
  DG_TRY(laplace_faces_apply(c->m, 1, (const double*)sv, c->lap_face, (double*)d, sh, c->s));
  return st.finish();
}

int dgns_vmult_viscous(dgns_ctx* c, double* dst3, const double* src3) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(dst3, src3);
  return lap_like(c, dst3, src3, DGNS_SPACE_U, 3, c->d.nu, 0.0);
}

int dgns_vmult_helmholtz(dgns_ctx* c, double* dst3, const double* src3, double mass_factor) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(dst3, src3);
  return lap_like(c, dst3, src3, DGNS_SPACE_U, 3, c->d.nu, mass_factor);
}

int dgns_vmult_laplace_f32(dgns_ctx* c, float* dst, const float* src, int level) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(dst, src);
  if (level < 0 || level >= (int)c->levels.size())
    return fail(DGNS_ERR_INVALID_ARG, "level out of range (multigrid disabled?)");
  Level& L = c->levels[level];
  const size_t bytes = (size_t)L.n * sizeof(float);
  if (overlaps(dst, bytes, src, bytes)) return fail(DGNS_ERR_ALIAS, "dst overlaps src");
  if (!aligned16(dst, src)) return fail(DGNS_ERR_INVALID_ARG, "dst and src must be 16-byte aligned");
  DG_TRY(laplace_apply(true, L.m, 1, src, dst, L.lap, EPI_NONE, EpiHost(), c->s));
  return 0;
}

int dgns_mg_chebyshev_step_f32(dgns_ctx* c, float* dst, const float* x, const float* xprev, const float* b,
                               double c1, double c2, int level) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(dst, x, b);
  if (c->mg_prec != 32) return fail(DGNS_ERR_UNSUPPORTED, "the FP32 smoother needs mg_precision = 32");
  if (level < 0 || level >= (int)c->levels.size())
    return fail(DGNS_ERR_INVALID_ARG, "level out of range (multigrid disabled?)");
  Level& L = c->levels[level];
  const size_t bytes = (size_t)L.n * sizeof(float);
  if (overlaps(dst, bytes, x, bytes) || overlaps(dst, bytes, b, bytes) || (xprev && overlaps(dst, bytes, xprev, bytes)))
    return fail(DGNS_ERR_ALIAS, "dst overlaps an input");
  if (!aligned16(dst, x) || !aligned16(b, xprev ? xprev : b))
    return fail(DGNS_ERR_INVALID_ARG, "vectors must be 16-byte aligned");
  if (!is_device_ptr(dst) || !is_device_ptr(x) || !is_device_ptr(b) || (xprev && !is_device_ptr(xprev)))
    return fail(DGNS_ERR_INVALID_ARG, "device pointers only");
  EpiHost ea;
  ea.b = b;
  ea.dinv = L.dinv;
  ea.xprev = xprev;
  ea.c1 = c1;
  ea.c2 = c2;
  DG_TRY(laplace_apply(true, L.m, 1, x, dst, L.lap, EPI_CHEB, ea, c->s));
  return 0;
}

int dgns_laplace_diagonal(dgns_ctx* c, double* dst, int space) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(dst);
  if (check_space(space)) return DGNS_ERR_INVALID_ARG;
  const int N = c->N[space];
  Staged st(c);
  void* d;
  DG_TRY(st.out(dst, (size_t)c->n[space] * sizeof(double), &d));
  DG_TRY(broadcast_cells(false, c->m.E, N * N * N, c->d_diag[space], d, c->s));
  return st.finish();
}

static int mass_like(dgns_ctx* c, double* dst, const double* src, int ncomp, int space, bool inverse) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(dst, src);
  if (check_space(space)) return DGNS_ERR_INVALID_ARG;
  if (ncomp < 1) return fail(DGNS_ERR_INVALID_ARG, "ncomp must be >= 1");
  const size_t bytes = (size_t)c->n[space] * ncomp * sizeof(double);
  if (overlaps(dst, bytes, src, bytes)) return fail(DGNS_ERR_ALIAS, "dst overlaps src");
  Staged st(c);
  const void* s;
  void* d;
  DG_TRY(st.in(src, bytes, &s));
  DG_TRY(st.out(dst, bytes, &d));
  const double(*T)[MAXN * MAXN] = inverse ? c->minv3[space] : c->mass3[space];
  const long long n = c->n[space] * ncomp;
  Ranged rg(c);
  int sh = 0;
  DG_TRY(rg.measure(s, n, kLinLo, kLinHi, &sh));
  if (sh) {
    const double* sc;
    DG_TRY(rg.scaled(s, n, -sh, 0, &sc));
    s = sc;
  }
  DG_TRY(tensor3_apply(c->N[space], c->m.E * ncomp, (const double*)s, (double*)d, T[0], T[1], T[2], c->s,
                       c->d.fp64_mode));
  DG_TRY(rg.rescale(d, n, sh));
  return st.finish();
}

int dgns_vmult_mass(dgns_ctx* c, double* dst, const double* src, int ncomp, int space) {
  return mass_like(c, dst, src, ncomp, space, false);
}

int dgns_apply_inverse_mass(dgns_ctx* c, double* dst, const double* src, int ncomp, int space) {
  return mass_like(c, dst, src, ncomp, space, true);
}

int dgns_vmult_divergence(dgns_ctx* c, double* dst_p, const double* u3) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(dst_p, u3);
  const size_t bu = (size_t)c->n[0] * 3 * sizeof(double), bp = (size_t)c->n[1] * sizeof(double);
  if (overlaps(dst_p, bp, u3, bu)) return fail(DGNS_ERR_ALIAS, "dst overlaps src");
  Staged st(c);
  const void* s;
  void* d;
  DG_TRY(st.in(u3, bu, &s));
  DG_TRY(st.out(dst_p, bp, &d));
  Ranged rg(c);
  int sh = 0;
  DG_TRY(rg.measure(s, 3 * c->n[0], kLinLo, kLinHi, &sh));
  if (sh) {
    const double* sc;
    DG_TRY(rg.scaled(s, 3 * c->n[0], -sh, 0, &sc));
    s = sc;
  }
  DG_TRY(divergence_apply(c->m, (const double*)s, (double*)d, c->div, c->s, c->d.fp64_mode == 1));
  DG_TRY(rg.rescale(d, c->n[1], sh));
  return st.finish();
}

int dgns_vmult_gradient(dgns_ctx* c, double* dst3, const double* p) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(dst3, p);
  const size_t bu = (size_t)c->n[0] * 3 * sizeof(double), bp = (size_t)c->n[1] * sizeof(double);
  if (overlaps(dst3, bu, p, bp)) return fail(DGNS_ERR_ALIAS, "dst overlaps src");
  Staged st(c);
  const void* s;
  void* d;
  DG_TRY(st.in(p, bp, &s));
  DG_TRY(st.out(dst3, bu, &d));
  Ranged rg(c);
  int sh = 0;
  DG_TRY(rg.measure(s, c->n[1], kLinLo, kLinHi, &sh));
  if (sh) {
    const double* sc;
    DG_TRY(rg.scaled(s, c->n[1], -sh, 0, &sc));
    s = sc;
  }
  DG_TRY(gradient_apply(c->m, (const double*)s, (double*)d, c->grad, c->s, c->d.fp64_mode == 1));
  DG_TRY(rg.rescale(d, 3 * c->n[0], sh));
  return st.finish();
}

namespace {
int conv_face_buffer(dgns_ctx* c) {
  if (c->conv_face) return 0;
  if (dev_malloc(&c->conv_face, (size_t)9 * c->m.E * c->conv.N * c->conv.N * sizeof(double)) != cudaSuccess) {
    c->conv_face = nullptr;
    cudaGetLastError();
    return fail(DGNS_ERR_OOM, "convective face buffer allocation failed");
  }
  return 0;
}
int conv_status(int rc) {
  if (rc == 7) return fail(DGNS_ERR_UNSUPPORTED, "convective kernel: unsupported (k, n_q_conv)");
  return rc;
}
}  // namespace

int dgns_vmult_convective(dgns_ctx* c, double* dst3, const double* u3) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(dst3, u3);
  const size_t bu = (size_t)c->n[0] * 3 * sizeof(double);
  if (overlaps(dst3, bu, u3, bu)) return fail(DGNS_ERR_ALIAS, "dst overlaps src");
  DG_TRY(conv_face_buffer(c));
  Staged st(c);
  const void* s;
  void* d;
  DG_TRY(st.in(u3, bu, &s));
  DG_TRY(st.out(dst3, bu, &d));
  const long long n = 3 * c->n[0];
  Ranged rg(c);
  int sh = 0;
  DG_TRY(rg.measure(s, n, kQuadLo, kQuadHi, &sh));
  if (sh) {
    const double* sc;
    DG_TRY(rg.scaled(s, n, -sh, 0, &sc));
    s = sc;
  }
  DG_TRY(conv_status(convective_launch(3, c->m, (const double*)s, c->conv_face, (double*)d, c->conv,
                                       c->d.fp64_mode, c->s)));
  DG_TRY(rg.rescale(d, n, 2 * sh));
  return st.finish();
}

int dgns_convective_face_size(const dgns_ctx* c, long long* n) {
  if (!c || !n) return fail(DGNS_ERR_INVALID_ARG, "null argument");
  *n = 9LL * c->m.E * c->conv.N * c->conv.N;
  return 0;
}

int dgns_convective_faces(dgns_ctx* c, double* rface, const double* u3) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(rface, u3);
  const size_t bu = (size_t)c->n[0] * 3 * sizeof(double);
  const size_t bf = (size_t)9 * c->m.E * c->conv.N * c->conv.N * sizeof(double);
  if (overlaps(rface, bf, u3, bu)) return fail(DGNS_ERR_ALIAS, "rface overlaps u3");
  Staged st(c);
  const void* s;
  void* f;
  DG_TRY(st.in(u3, bu, &s));
  DG_TRY(st.out(rface, bf, &f));
  const long long n = 3 * c->n[0], nf = 9LL * c->m.E * c->conv.N * c->conv.N;
  Ranged rg(c);
  int sh = 0;
  DG_TRY(rg.measure(s, n, kQuadLo, kQuadHi, &sh));
  if (sh) {
    const double* sc;
    DG_TRY(rg.scaled(s, n, -sh, 0, &sc));
    s = sc;
  }
  DG_TRY(conv_status(convective_launch(1, c->m, (const double*)s, (double*)f, nullptr, c->conv,
                                       c->d.fp64_mode, c->s)));
  DG_TRY(rg.rescale(f, nf, 2 * sh));
  return st.finish();
}

int dgns_convective_cells(dgns_ctx* c, double* dst3, const double* u3, const double* rface) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(dst3, u3, rface);
  const size_t bu = (size_t)c->n[0] * 3 * sizeof(double);
  const size_t bf = (size_t)9 * c->m.E * c->conv.N * c->conv.N * sizeof(double);
  if (overlaps(dst3, bu, u3, bu) || overlaps(dst3, bu, rface, bf))
    return fail(DGNS_ERR_ALIAS, "dst3 overlaps an input");
  Staged st(c);
  const void* s;
  const void* f;
  void* d;
  DG_TRY(st.in(u3, bu, &s));
  DG_TRY(st.in(rface, bf, &f));
  DG_TRY(st.out(dst3, bu, &d));
  const long long n = 3 * c->n[0], nf = 9LL * c->m.E * c->conv.N * c->conv.N;
  Ranged rg(c);
  int sh = 0;
  DG_TRY(rg.measure(s, n, kQuadLo, kQuadHi, &sh));
  if (sh) {   // the face integrals scale with the square of u
    const double *su, *sf;
    DG_TRY(rg.scaled(s, n, -sh, 0, &su));
    DG_TRY(rg.scaled(f, nf, -2 * sh, 1, &sf));
    s = su;
    f = sf;
  }
  DG_TRY(conv_status(convective_launch(2, c->m, (const double*)s, (double*)f, (double*)d, c->conv,
                                       c->d.fp64_mode, c->s)));
  DG_TRY(rg.rescale(d, n, 2 * sh));
  return st.finish();
}

int dgns_vjp_convective(dgns_ctx* c, double* grad_u3, const double* u3, const double* w3) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(grad_u3, u3, w3);
  const size_t bu = (size_t)c->n[0] * 3 * sizeof(double);
  if (overlaps(grad_u3, bu, u3, bu) || overlaps(grad_u3, bu, w3, bu))
    return fail(DGNS_ERR_ALIAS, "grad_u3 overlaps an input");
  Staged st(c);
  const void* su;
  const void* sw;
  void* d;
  DG_TRY(st.in(u3, bu, &su));
  DG_TRY(st.in(w3, bu, &sw));
  DG_TRY(st.out(grad_u3, bu, &d));
  int rc = convective_vjp(c->m, (const double*)su, (const double*)sw, (double*)d, c->conv, c->s,
                          c->d.fp64_mode == 1);
  if (rc == 7) return fail(DGNS_ERR_UNSUPPORTED, "convective VJP: unsupported degree or quadrature");
  DG_TRY(rc);
  return st.finish();
}

// Broken stiffness (cell terms of the SIPG form only) scaled by `coef`.
static void build_broken_stiffness(const dgns_ctx* c, double coef, LapHost& L, int space = DGNS_SPACE_U) {
  build_lap(c->sp1[space], c->h, c->d.penalty_factor, coef, 0.0, L);
  const Space1D& s = c->sp1[space];
  const int N = s.N;
  for (int d = 0; d < 3; ++d) {
    ld ht = 1.0L;
    for (int e = 0; e < 3; ++e)
      if (e != d) ht *= (ld)c->h[e];
    for (int i = 0; i < N * N; ++i) L.A0[d][i] = (double)((ld)coef * ht * s.stiff[i] / (ld)c->h[d]);
    for (int i = 0; i < N; ++i) L.cr[d][i] = L.cl[d][i] = L.gr[d][i] = L.gl[d][i] = 0.0;
  }
}

int dgns_dissipation_grad(dgns_ctx* c, double* grad3, const double* u3) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(grad3, u3);
  const size_t bu = (size_t)c->n[0] * 3 * sizeof(double);
  if (overlaps(grad3, bu, u3, bu)) return fail(DGNS_ERR_ALIAS, "grad3 overlaps u3");
  Staged st(c);
  const void* s;
  void* d;
  DG_TRY(st.in(u3, bu, &s));
  DG_TRY(st.out(grad3, bu, &d));
  double vol = 1.0;
  for (int i = 0; i < 3; ++i) vol *= c->d.hi[i] - c->d.lo[i];
  LapHost K;
  build_broken_stiffness(c, 2.0 * c->d.nu / vol, K);
  DG_TRY(laplace_apply(false, c->m, 3, s, d, K, EPI_NONE, EpiHost(), c->s, c->d.fp64_mode));
  return st.finish();
}

int dgns_dissipation(dgns_ctx* c, const double* u3, double* eps_out) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(u3, eps_out);
  const long long n = 3 * c->n[0];
  DG_TRY(alloc_cg(c, n));
  Staged st(c);
  const void* s;
  DG_TRY(st.in(u3, (size_t)n * sizeof(double), &s));
  double vol = 1.0;
  for (int i = 0; i < 3; ++i) vol *= c->d.hi[i] - c->d.lo[i];
  LapHost K;
  build_broken_stiffness(c, c->d.nu / vol, K);
  DG_TRY(laplace_apply(false, c->m, 3, s, c->Ap, K, EPI_NONE, EpiHost(), c->s, c->d.fp64_mode));
  DG_TRY(dot((const double*)s, c->Ap, n, c->red, S_T1, c->s));
  DG_TRY(read_scalars(c));
  *eps_out = c->h_scal[S_T1];
  return st.finish();
}

int dgns_axpby(dgns_ctx* c, double* y, const double* x, long long n, double a, double b) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(y, x);
  if (n < 0) return fail(DGNS_ERR_INVALID_ARG, "n < 0");
  if (!is_device_ptr(y) || !is_device_ptr(x)) return fail(DGNS_ERR_INVALID_ARG, "device pointers only");
  if (n == 0) return 0;
  DG_TRY(axpby(y, x, n, a, b, c->s));
  return 0;
}

int dgns_dot(dgns_ctx* c, const double* a, const double* b, long long n, double* out) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(a, b, out);
  if (n < 0) return fail(DGNS_ERR_INVALID_ARG, "n < 0");
  if (!is_device_ptr(a) || !is_device_ptr(b)) return fail(DGNS_ERR_INVALID_ARG, "device pointers only");
  if (n == 0) {
    *out = 0.0;
    return 0;
  }
  DG_TRY(dot(a, b, n, c->red, S_T1, c->s));
  DG_TRY(read_scalars(c));
  *out = c->h_scal[S_T1];
  return 0;
}

int dgns_penalty_parameters(dgns_ctx* c, const double* u_ex3, double dt, double zeta_d, double zeta_c,
                            double* tau_d, double* tau_c) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(u_ex3, tau_d, tau_c);
  if (!is_device_ptr(u_ex3) || !is_device_ptr(tau_d) || !is_device_ptr(tau_c))
    return fail(DGNS_ERR_INVALID_ARG, "device pointers only");
  const double h_eff = cbrt(c->h[0] * c->h[1] * c->h[2]);
  const double fd = zeta_d * h_eff / (c->k[0] + 1) * dt, fc = zeta_c * dt;
  const int rc = penalty_parameters(c->m, u_ex3, tau_d, tau_c, c->proj, fd, fc, c->s, c->d.fp64_mode == 1);
  if (rc == 7) return fail(DGNS_ERR_UNSUPPORTED, "projection operator: degree not supported");
  DG_TRY(rc);
  return 0;
}

int dgns_vmult_projection(dgns_ctx* c, double* dst3, const double* src3, const double* tau_d,
                          const double* tau_c) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(dst3, src3, tau_d, tau_c);
  const size_t bu = (size_t)c->n[0] * 3 * sizeof(double);
  if (overlaps(dst3, bu, src3, bu)) return fail(DGNS_ERR_ALIAS, "dst overlaps src");
  if (!is_device_ptr(dst3) || !is_device_ptr(src3) || !is_device_ptr(tau_d) || !is_device_ptr(tau_c))
    return fail(DGNS_ERR_INVALID_ARG, "device pointers only");
  const long long n = 3 * c->n[0];
  Ranged rg(c);
  int sh = 0;
  DG_TRY(rg.measure(src3, n, kLinLo, kLinHi, &sh));
  if (sh) DG_TRY(rg.scaled(src3, n, -sh, 0, &src3));
  const int rc = projection_apply(c->m, src3, dst3, tau_d, tau_c, c->proj, c->s, c->d.fp64_mode == 1);
  if (rc == 7) return fail(DGNS_ERR_UNSUPPORTED, "projection operator: degree not supported");
  DG_TRY(rc);
  DG_TRY(rg.rescale(dst3, n, sh));
  return 0;
}

int dgns_vmult_projection_terms(dgns_ctx* c, double* dst3, const double* src3, const double* tau_d,
                                const double* tau_c, int terms) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  if (terms == DGNS_PROJ_ALL) return dgns_vmult_projection(c, dst3, src3, tau_d, tau_c);
  if (terms != DGNS_PROJ_MASS && terms != DGNS_PROJ_DIV && terms != DGNS_PROJ_CONT)
    return fail(DGNS_ERR_INVALID_ARG, "terms must be DGNS_PROJ_MASS, _DIV, _CONT or _ALL");
  DG_NONNULL(dst3, src3);
  if (terms == DGNS_PROJ_DIV) DG_NONNULL(tau_d);
  if (terms == DGNS_PROJ_CONT) DG_NONNULL(tau_c);
  const size_t bu = (size_t)c->n[0] * 3 * sizeof(double);
  if (overlaps(dst3, bu, src3, bu)) return fail(DGNS_ERR_ALIAS, "dst overlaps src");
  if (!is_device_ptr(dst3) || !is_device_ptr(src3) || (tau_d && !is_device_ptr(tau_d)) ||
      (tau_c && !is_device_ptr(tau_c)))
    return fail(DGNS_ERR_INVALID_ARG, "device pointers only");
  const long long n = 3 * c->n[0];
  Ranged rg(c);
  int sh = 0;
  DG_TRY(rg.measure(src3, n, kLinLo, kLinHi, &sh));
  if (sh) DG_TRY(rg.scaled(src3, n, -sh, 0, &src3));
  if (terms == DGNS_PROJ_MASS) {
    const double(*T)[MAXN * MAXN] = c->mass3[DGNS_SPACE_U];
    DG_TRY(tensor3_apply(c->N[0], 3 * c->m.E, src3, dst3, T[0], T[1], T[2], c->s, c->d.fp64_mode));
  } else {
    const int rc = projection_apply(c->m, src3, dst3, tau_d, tau_c, c->proj, c->s, c->d.fp64_mode == 1,
                                    terms == DGNS_PROJ_DIV ? PROJ_DIV : PROJ_CONT);
    if (rc == 7) return fail(DGNS_ERR_UNSUPPORTED, "projection operator: degree not supported");
    DG_TRY(rc);
  }
  DG_TRY(rg.rescale(dst3, n, sh));
  return 0;
}

int dgns_cg_projection_solve(dgns_ctx* c, double* x3, const double* b3, const double* tau_d,
                             const double* tau_c, const dgns_solve_params* params, dgns_solve_info* info) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(x3, b3, tau_d, tau_c);
  dgns_solve_params prm;
  if (params) prm = *params;
  else dgns_default_solve_params(&prm);
  if (prm.max_iter < 1) return fail(DGNS_ERR_INVALID_ARG, "invalid solve parameters");
  const long long n = 3 * c->n[DGNS_SPACE_U];
  const size_t bytes = (size_t)n * sizeof(double);
  if (overlaps(x3, bytes, b3, bytes)) return fail(DGNS_ERR_ALIAS, "x overlaps b");
  if (!is_device_ptr(x3) || !is_device_ptr(b3) || !is_device_ptr(tau_d) || !is_device_ptr(tau_c))
    return fail(DGNS_ERR_INVALID_ARG, "device pointers only");
  DG_TRY(alloc_cg(c, n));
  const auto t0 = std::chrono::steady_clock::now();
  const int N = c->N[0];
  const double(*MI)[MAXN * MAXN] = c->minv3[0];
  double* X = x3;
  const double* B = b3;
  // emulated arithmetic: the system is scaled by an exact power of two when b
  // lies outside the input window (the operator is linear:
  // A (x 2^-s) = b 2^-s), and the solution scaled back
  Ranged rg(c);
  int sh = 0;
  DG_TRY(rg.measure(B, n, kLinLo, kLinHi, &sh));
  if (sh) {
    DG_TRY(rg.scaled(B, n, -sh, 2, &B));
    if (prm.use_initial_guess) DG_TRY(rg.rescale(X, n, -sh));
    prm.abs_tol = ldexp(prm.abs_tol, -sh);
  }
  DG_CUDA(cudaMemcpyAsync(c->r, B, bytes, cudaMemcpyDeviceToDevice, c->s));
  if (prm.use_initial_guess) {
    DG_TRY(projection_apply(c->m, X, c->Ap, tau_d, tau_c, c->proj, c->s, c->d.fp64_mode == 1));
    DG_TRY(axpby(c->r, c->Ap, n, -1.0, 1.0, c->s));
    DG_TRY(dot(c->r, c->r, n, c->red, S_T0, c->s));
  } else {
    DG_CUDA(cudaMemsetAsync(X, 0, bytes, c->s));
    DG_TRY(dot(B, B, n, c->red, S_T0, c->s));
  }
  DG_TRY(read_scalars(c));
  const double nb = sqrt(c->h_scal[S_T0]);
  dgns_solve_info inf{};
  inf.initial_res = nb;
  int status = DGNS_OK;
  if (nb > 0.0) {
    DG_TRY(tensor3_apply(N, 3 * c->m.E, c->r, c->z, MI[0], MI[1], MI[2], c->s, c->d.fp64_mode));
    DG_TRY(cg_direction(c->p, c->z, n, c->red, true, c->s));
    DG_TRY(dot(c->r, c->z, n, c->red, S_RZ, c->s));
    int it = 0;
    double res = 1.0;
    status = DGNS_ERR_NOT_CONVERGED;
    while (it < prm.max_iter) {
      DG_TRY(projection_apply(c->m, c->p, c->Ap, tau_d, tau_c, c->proj, c->s, c->d.fp64_mode == 1));
      DG_TRY(dot(c->p, c->Ap, n, c->red, S_PAP, c->s));
      DG_TRY(cg_update(x3, c->r, c->p, c->Ap, n, c->red, c->s));
      DG_TRY(read_scalars(c));
      ++it;
      const double rr = c->h_scal[S_RR];
      if (!std::isfinite(rr)) {
        status = fail(DGNS_ERR_NONFINITE, "non-finite residual");
        break;
      }
      res = sqrt(rr) / nb;
      if (res <= prm.rel_tol || sqrt(rr) <= prm.abs_tol) {
        status = DGNS_OK;
        break;
      }
      DG_TRY(tensor3_apply(N, 3 * c->m.E, c->r, c->z, MI[0], MI[1], MI[2], c->s, c->d.fp64_mode));
      DG_TRY(dot(c->r, c->z, n, c->red, S_RZNEW, c->s));
      DG_TRY(cg_direction(c->p, c->z, n, c->red, false, c->s));
    }
    inf.iterations = it;
    inf.rel_res = res;
    if (status == DGNS_ERR_NOT_CONVERGED) fail(status, "max_iter reached");
  } else if (!std::isfinite(nb)) {
    status = fail(DGNS_ERR_NONFINITE, "non-finite right-hand side");
  }
  DG_TRY(rg.rescale(X, n, sh));
  inf.initial_res = ldexp(inf.initial_res, sh);
  DG_CUDA(cudaStreamSynchronize(c->s));
  inf.status = status;
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  return status;
}

int dgns_mg_info(const dgns_ctx* c, int* n_levels, int* n_elem_per_level, double* lambda_max) {
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  const int nl = (int)c->levels.size();
  if (n_levels) *n_levels = nl;
  for (int i = 0; i < nl; ++i) {
    if (n_elem_per_level) n_elem_per_level[i] = c->levels[i].m.nx;
    if (lambda_max) lambda_max[i] = c->levels[i].lambda_max;
  }
  return 0;
}

int dgns_mg_vcycle(dgns_ctx* c, double* z, const double* r, const dgns_solve_params* params) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(z, r);
  if (c->levels.empty()) return fail(DGNS_ERR_INVALID_ARG, "multigrid disabled");
  dgns_solve_params prm;
  if (params) prm = *params;
  else dgns_default_solve_params(&prm);
  prm.project_mean = 0;
  return precondition(c, r, z, &prm, c->n[DGNS_SPACE_P]);
}

int dgns_mg_prolongate_f32(dgns_ctx* c, float* fine, const float* coarse, int level) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(fine, coarse);
  if (level < 0 || level + 1 >= (int)c->levels.size()) return fail(DGNS_ERR_INVALID_ARG, "level out of range");
  DG_TRY(prolongate(true, c->N[DGNS_SPACE_P], c->levels[level].m, coarse, fine, c->P0, c->P1, false, c->s));
  return 0;
}

int dgns_mg_restrict_f32(dgns_ctx* c, float* coarse, const float* fine, int level) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(fine, coarse);
  if (level < 0 || level + 1 >= (int)c->levels.size()) return fail(DGNS_ERR_INVALID_ARG, "level out of range");
  DG_TRY(restrict_fine(true, c->N[DGNS_SPACE_P], c->levels[level].m, fine, coarse, c->P0, c->P1, c->s));
  return 0;
}

int dgns_cg_mg_solve(dgns_ctx* c, double* x, const double* b, const dgns_solve_params* params,
                     dgns_solve_info* info) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(x, b);
  dgns_solve_params prm;
  if (params) prm = *params;
  else dgns_default_solve_params(&prm);
  if (prm.max_iter < 1 || prm.cheb_degree < 1 || prm.cheb_coarse_iters < 1 || !(prm.smoothing_range > 1.0))
    return fail(DGNS_ERR_INVALID_ARG, "invalid solve parameters");
  const long long n = c->n[DGNS_SPACE_P];
  const size_t bytes = (size_t)n * sizeof(double);
  if (overlaps(x, bytes, b, bytes)) return fail(DGNS_ERR_ALIAS, "x overlaps b");
  DG_TRY(alloc_cg(c, n));
  const auto t0 = std::chrono::steady_clock::now();
  Staged st(c);
  const void* bs;
  void* xs;
  DG_TRY(st.in(b, bytes, &bs));
  DG_TRY(prm.use_initial_guess ? st.inout(x, bytes, &xs) : st.out(x, bytes, &xs));
  double* X = (double*)xs;
  const double* B = (const double*)bs;
  // emulated arithmetic: the system is scaled by an exact power of two when b
  // lies outside the input window (the operator is linear:
  // A (x 2^-s) = b 2^-s), and the solution scaled back
  Ranged rg(c);
  int sh = 0;
  DG_TRY(rg.measure(B, n, kLinLo, kLinHi, &sh));
  if (sh) {
    DG_TRY(rg.scaled(B, n, -sh, 2, &B));
    if (prm.use_initial_guess) DG_TRY(rg.rescale(X, n, -sh));
    prm.abs_tol = ldexp(prm.abs_tol, -sh);
  }
  const LapHost& A = c->lap[DGNS_SPACE_P];
  if (!prm.use_initial_guess) {
    DG_CUDA(cudaMemsetAsync(X, 0, bytes, c->s));
    DG_TRY(dot(B, B, n, c->red, S_T0, c->s));
  }
  if (prm.project_mean) {
    DG_TRY(sum(B, n, c->red, S_SUM, c->s));
    DG_TRY(convert_shift(B, false, c->r, false, n, &c->red, S_SUM, c->s));
  } else {
    DG_CUDA(cudaMemcpyAsync(c->r, B, bytes, cudaMemcpyDeviceToDevice, c->s));
  }
  if (prm.use_initial_guess) {
    // r0 = b - A x0 (A annihilates constants, so the mean shift of b is the one of r0)
    DG_TRY(laplace_apply(false, c->m, 1, X, c->Ap, A, EPI_NONE, EpiHost(), c->s, c->d.fp64_mode));
    DG_TRY(axpby(c->r, c->Ap, n, -1.0, 1.0, c->s));
    DG_TRY(dot(c->r, c->r, n, c->red, S_T0, c->s));
  }
  DG_TRY(read_scalars(c));
  const double nb = sqrt(c->h_scal[S_T0]);
  dgns_solve_info inf{};
  inf.initial_res = nb;
  inf.lambda_max_fine = c->levels.empty() ? 0.0 : c->levels.back().lambda_max;
  int status = DGNS_OK;
  if (!(nb > 0.0)) {
    inf.rel_res = 0.0;
    if (!std::isfinite(nb)) status = fail(DGNS_ERR_NONFINITE, "non-finite right-hand side");
  } else {
    DG_TRY(precondition_cg(c, &prm, n));   // scal[S_RZNEW] = (r, z)
    DG_TRY(cg_direction(c->p, c->z, n, c->red, true, c->s));
    DG_TRY(scal_rotate(c->red, c->s));
    double res = 1.0;
    int it = 0;
    status = DGNS_ERR_NOT_CONVERGED;
    while (it < prm.max_iter) {
      DG_TRY(laplace_apply(false, c->m, 1, c->p, c->Ap, A, EPI_NONE, EpiHost(), c->s, c->d.fp64_mode));
      DG_TRY(dot(c->p, c->Ap, n, c->red, S_PAP, c->s));
      DG_TRY(cg_update(X, c->r, c->p, c->Ap, n, c->red, c->s));
      DG_TRY(read_scalars(c));
      ++it;
      const double rr = c->h_scal[S_RR];
      if (!std::isfinite(rr) || !std::isfinite(c->h_scal[S_PAP])) {
        status = fail(DGNS_ERR_NONFINITE, "non-finite residual");
        break;
      }
      res = sqrt(rr) / nb;
      if (res <= prm.rel_tol || sqrt(rr) <= prm.abs_tol) {
        status = DGNS_OK;
        break;
      }
      DG_TRY(precondition_cg(c, &prm, n));   // scal[S_RZNEW] = (r, z)
      DG_TRY(cg_direction(c->p, c->z, n, c->red, false, c->s));
    }
    inf.iterations = it;
    inf.rel_res = res;
    if (status == DGNS_ERR_NOT_CONVERGED) fail(status, "max_iter reached");
  }
  DG_TRY(rg.rescale(X, n, sh));
  inf.initial_res = ldexp(inf.initial_res, sh);
  DG_TRY(st.finish());
  DG_CUDA(cudaStreamSynchronize(c->s));
  inf.status = status;
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  return status;
}

int dgns_cg_invmass_solve(dgns_ctx* c, double* x3, const double* b3, double mass_factor,
                          const dgns_solve_params* params, dgns_solve_info* info) {
  g_err.clear();
  if (!c) return fail(DGNS_ERR_INVALID_ARG, "ctx is null");
  DG_NONNULL(x3, b3);
  dgns_solve_params prm;
  if (params) prm = *params;
  else dgns_default_solve_params(&prm);
  if (prm.max_iter < 1) return fail(DGNS_ERR_INVALID_ARG, "invalid solve parameters");
  const long long n = 3 * c->n[DGNS_SPACE_U];
  const size_t bytes = (size_t)n * sizeof(double);
  if (overlaps(x3, bytes, b3, bytes)) return fail(DGNS_ERR_ALIAS, "x overlaps b");
  DG_TRY(alloc_cg(c, n));
  const auto t0 = std::chrono::steady_clock::now();
  Staged st(c);
  const void* bs;
  void* xs;
  DG_TRY(st.in(b3, bytes, &bs));
  DG_TRY(prm.use_initial_guess ? st.inout(x3, bytes, &xs) : st.out(x3, bytes, &xs));
  double* X = (double*)xs;
  const double* B = (const double*)bs;
  // emulated arithmetic: the system is scaled by an exact power of two when b
  // lies outside the input window (the operator is linear:
  // A (x 2^-s) = b 2^-s), and the solution scaled back
  Ranged rg(c);
  int sh = 0;
  DG_TRY(rg.measure(B, n, kLinLo, kLinHi, &sh));
  if (sh) {
    DG_TRY(rg.scaled(B, n, -sh, 2, &B));
    if (prm.use_initial_guess) DG_TRY(rg.rescale(X, n, -sh));
    prm.abs_tol = ldexp(prm.abs_tol, -sh);
  }
  LapHost H;
  build_lap(c->sp1[0], c->h, c->d.penalty_factor, c->d.nu, mass_factor, H);
  const int N = c->N[0];
  const double(*MI)[MAXN * MAXN] = c->minv3[0];
  DG_CUDA(cudaMemcpyAsync(c->r, B, bytes, cudaMemcpyDeviceToDevice, c->s));
  if (prm.use_initial_guess) {
    DG_TRY(laplace_apply(false, c->m, 3, X, c->Ap, H, EPI_NONE, EpiHost(), c->s, c->d.fp64_mode));
    DG_TRY(axpby(c->r, c->Ap, n, -1.0, 1.0, c->s));
    DG_TRY(dot(c->r, c->r, n, c->red, S_T0, c->s));
  } else {
    DG_CUDA(cudaMemsetAsync(X, 0, bytes, c->s));
    DG_TRY(dot(B, B, n, c->red, S_T0, c->s));
  }
  DG_TRY(read_scalars(c));
  const double nb = sqrt(c->h_scal[S_T0]);
  dgns_solve_info inf{};
  inf.initial_res = nb;
  int status = DGNS_OK;
  if (nb > 0.0) {
    DG_TRY(tensor3_apply(N, 3 * c->m.E, c->r, c->z, MI[0], MI[1], MI[2], c->s, c->d.fp64_mode));
    DG_TRY(cg_direction(c->p, c->z, n, c->red, true, c->s));
    DG_TRY(dot(c->r, c->z, n, c->red, S_RZ, c->s));
    int it = 0;
    double res = 1.0;
    status = DGNS_ERR_NOT_CONVERGED;
    while (it < prm.max_iter) {
      DG_TRY(laplace_apply(false, c->m, 3, c->p, c->Ap, H, EPI_NONE, EpiHost(), c->s, c->d.fp64_mode));
      DG_TRY(dot(c->p, c->Ap, n, c->red, S_PAP, c->s));
      DG_TRY(cg_update(X, c->r, c->p, c->Ap, n, c->red, c->s));
      DG_TRY(read_scalars(c));
      ++it;
      const double rr = c->h_scal[S_RR];
      if (!std::isfinite(rr)) {
        status = fail(DGNS_ERR_NONFINITE, "non-finite residual");
        break;
      }
      res = sqrt(rr) / nb;
      if (res <= prm.rel_tol || sqrt(rr) <= prm.abs_tol) {
        status = DGNS_OK;
        break;
      }
      DG_TRY(tensor3_apply(N, 3 * c->m.E, c->r, c->z, MI[0], MI[1], MI[2], c->s, c->d.fp64_mode));
      DG_TRY(dot(c->r, c->z, n, c->red, S_RZNEW, c->s));
      DG_TRY(cg_direction(c->p, c->z, n, c->red, false, c->s));
    }
    inf.iterations = it;
    inf.rel_res = res;
    if (status == DGNS_ERR_NOT_CONVERGED) fail(status, "max_iter reached");
  } else if (!std::isfinite(nb)) {
    status = fail(DGNS_ERR_NONFINITE, "non-finite right-hand side");
  }
  DG_TRY(rg.rescale(X, n, sh));
  inf.initial_res = ldexp(inf.initial_res, sh);
  DG_TRY(st.finish());
  DG_CUDA(cudaStreamSynchronize(c->s));
  inf.status = status;
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  return status;
}

}  // extern "C"
