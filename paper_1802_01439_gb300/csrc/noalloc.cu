// Allocation-free variant of the inverse-mass-preconditioned Helmholtz CG
// solve (dgns_cg_invmass_solve_noalloc in include/dgns.h).
//
// Some callers cannot let a library call cudaMalloc: applications that hand
// all device memory to their own pool or allocator up front (a library
// allocation outside that pool can fail or fragment it), and real-time loops
// that must not pay allocation latency or risk an out-of-memory failure in
// the middle of a time step.  This entry point serves them: its CG work
// vectors and reduction scratch live in one file-scope __device__ array of
// fixed size that is part of the loaded module, so the call itself allocates
// nothing.  Like the allocating solve it reads one block of scalars back to
// the host and synchronises the context's stream once per CG iteration.
#include <cmath>
#include <cstring>
#include <mutex>

#include "ctx.h"

namespace {

using namespace dgns;

// Largest work vector (3 velocity components together) the scratch holds.
constexpr long long kMaxEntries = 1LL << 19;  // 524,288 doubles = 4 MiB per vector
constexpr long long kScratch = 4 * kMaxEntries + RED_BLOCKS + S_NSLOTS;

// Four CG vectors (r, z, p, Ap), the reduction partials and the scalars.
// Every GPU that loads the library holds these ~16 MiB until the process exits.
static __device__ __align__(256) double g_cg_scratch[kScratch];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_cg_scratch on the current device.  In host code the
// symbol is only a host-side stand-in, so its address must be queried once per
// device, with that device current.
int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(DGNS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(DGNS_ERR_UNSUPPORTED, "device ordinal too large");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_cg_scratch);
    if (e != cudaSuccess || !p)
      return set_error(DGNS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return 0;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

#define NA_CUDA(call)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return set_error(DGNS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// A failed step keeps the message its callee recorded; where there is none,
// the step's name (and, for CUDA errors, the runtime's message) is recorded.
#define NA_TRY(call)                                                                         \
  do {                                                                                       \
    int rc_ = (call);                                                                        \
    if (rc_ != 0) {                                                                          \
      if (!error_empty()) return rc_;                                                        \
      if (rc_ == DGNS_ERR_CUDA)                                                              \
        return set_error(rc_, std::string(#call) + ": " + cudaGetErrorString(cudaGetLastError())); \
      return set_error(rc_, #call);                                                          \
    }                                                                                        \
  } while (0)

}  // namespace

extern "C" int dgns_cg_invmass_solve_noalloc(dgns_ctx* c, double* x3, const double* b3, double mass_factor,
                                             const dgns_solve_params* params, dgns_solve_info* info) {
  clear_error();
  if (!c || !x3 || !b3) return set_error(DGNS_ERR_INVALID_ARG, "null argument");
  {
    // the scratch address is looked up on the current device, so that must
    // be the device that holds the context (its tables, vectors and stream)
    int dev = -1;
    NA_CUDA(cudaGetDevice(&dev));
    if (dev != c->device)
      return set_error(DGNS_ERR_INVALID_ARG, "dgns_cg_invmass_solve_noalloc: the context's device (" +
                                                 std::to_string(c->device) + ") must be current (is " +
                                                 std::to_string(dev) + ")");
  }
  dgns_solve_params prm;
  if (params) prm = *params;
  else dgns_default_solve_params(&prm);
  if (prm.max_iter < 1) return set_error(DGNS_ERR_INVALID_ARG, "invalid solve parameters");
  const long long n = 3 * c->n[DGNS_SPACE_U];
  if (n > kMaxEntries)
    return set_error(DGNS_ERR_INVALID_ARG,
                     "dgns_cg_invmass_solve_noalloc: 3 x " + std::to_string(c->n[DGNS_SPACE_U]) +
                         " velocity entries exceed the static scratch limit of " + std::to_string(kMaxEntries));
  if (!on_device(x3) || !on_device(b3))
    return set_error(DGNS_ERR_INVALID_ARG, "dgns_cg_invmass_solve_noalloc takes device pointers only");
  const size_t bytes = (size_t)n * sizeof(double);
  const char* px = (const char*)x3;
  const char* pb = (const char*)b3;
  if (px < pb + bytes && pb < px + bytes) return set_error(DGNS_ERR_ALIAS, "x overlaps b");
  double* S = nullptr;
  NA_TRY(scratch_address(&S));
  double* r = S;
  double* z = S + kMaxEntries;
  double* p = S + 2 * kMaxEntries;
  double* Ap = S + 3 * kMaxEntries;
  Reducer red;
  red.part = S + 4 * kMaxEntries;
  red.scal = red.part + RED_BLOCKS;
  double hs[S_NSLOTS];
  auto read_scal = [&]() -> int {
    NA_CUDA(cudaMemcpyAsync(hs, red.scal, sizeof(hs), cudaMemcpyDeviceToHost, c->s));
    NA_CUDA(cudaStreamSynchronize(c->s));
    return 0;
  };
  LapHost H;
  build_lap(c->sp1[0], c->h, c->d.penalty_factor, c->d.nu, mass_factor, H);
  const int N = c->N[0];
  const double(*MI)[MAXN * MAXN] = c->minv3[0];
  // The scratch keeps the previous call's contents; every work vector below
  // is written before it is read, and x (caller-owned) is cleared here
  // unless it holds the initial guess.
  NA_CUDA(cudaMemcpyAsync(r, b3, bytes, cudaMemcpyDeviceToDevice, c->s));
  if (prm.use_initial_guess) {
    NA_TRY(laplace_apply(false, c->m, 3, x3, Ap, H, EPI_NONE, EpiHost(), c->s, c->d.fp64_mode));
    NA_TRY(axpby(r, Ap, n, -1.0, 1.0, c->s));
    NA_TRY(dot(r, r, n, red, S_T0, c->s));
  } else {
    NA_CUDA(cudaMemsetAsync(x3, 0, bytes, c->s));
    NA_TRY(dot(b3, b3, n, red, S_T0, c->s));
  }
  NA_TRY(read_scal());
  const double nb = sqrt(hs[S_T0]);
  dgns_solve_info inf{};
  inf.initial_res = nb;
  int status = DGNS_OK;
  if (nb > 0.0) {
    NA_TRY(tensor3_apply(N, 3 * c->m.E, r, z, MI[0], MI[1], MI[2], c->s, c->d.fp64_mode));
    NA_TRY(cg_direction(p, z, n, red, true, c->s));
    NA_TRY(dot(r, z, n, red, S_RZ, c->s));
    int it = 0;
    double res = 1.0;
    status = DGNS_ERR_NOT_CONVERGED;
    while (it < prm.max_iter) {
      NA_TRY(laplace_apply(false, c->m, 3, p, Ap, H, EPI_NONE, EpiHost(), c->s, c->d.fp64_mode));
      NA_TRY(dot(p, Ap, n, red, S_PAP, c->s));
      NA_TRY(cg_update(x3, r, p, Ap, n, red, c->s));
      NA_TRY(read_scal());
      ++it;
      const double rr = hs[S_RR];
      if (!std::isfinite(rr)) {
        status = set_error(DGNS_ERR_NONFINITE, "non-finite residual");
        break;
      }
      res = sqrt(rr) / nb;
      if (res <= prm.rel_tol || sqrt(rr) <= prm.abs_tol) {
        status = DGNS_OK;
        break;
      }
      NA_TRY(tensor3_apply(N, 3 * c->m.E, r, z, MI[0], MI[1], MI[2], c->s, c->d.fp64_mode));
      NA_TRY(dot(r, z, n, red, S_RZNEW, c->s));
      NA_TRY(cg_direction(p, z, n, red, false, c->s));
    }
    inf.iterations = it;
    inf.rel_res = res;
    if (status == DGNS_ERR_NOT_CONVERGED) set_error(status, "max_iter reached");
  } else if (!std::isfinite(nb)) {
    status = set_error(DGNS_ERR_NONFINITE, "non-finite right-hand side");
  }
  NA_CUDA(cudaStreamSynchronize(c->s));
  inf.status = status;
  if (info) *info = inf;
  return status;
}
