// Internal definition of the libdgns context, shared by the translation
// units that implement C-ABI entry points.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "blas.h"
#include "dgns.h"
#include "ops.h"
#include "tables.h"

namespace dgns {

// One multigrid level of the pressure space.
struct Level {
  MeshDims m{};
  double h[3] = {0, 0, 0};
  LapHost lap;            // FP64 values; rounded by the launcher
  void* dinv = nullptr;   // N^3 table in the V-cycle precision
  double* dinv64 = nullptr;
  void* xa = nullptr;
  void* xb = nullptr;
  void* b = nullptr;
  void* r = nullptr;
  long long n = 0;
  double lambda_max = 0.0;
};

// Records `msg` as the calling thread's last error and returns `code`.
int set_error(int code, const std::string& msg);
// Clears the calling thread's last error (entry points start with it).
void clear_error();
// Whether the calling thread's last error is empty.
bool error_empty();
// SIPG-type tables of space `s` on cells of size h: coef * (Laplace) plus
// mass_factor * (mass), with tau = pf (k+1)^2 / h_d.
void build_lap(const Space1D& s, const double h[3], double pf, double coef, double mass_factor,
               LapHost& L);

}  // namespace dgns

struct dgns_ctx {
  using Level = dgns::Level;
  dgns_mesh_desc d{};
  cudaStream_t s = nullptr;
  int device = -1;  // the CUDA device current at creation, which holds every buffer
  dgns::MeshDims m{};
  double h[3] = {0, 0, 0};
  int k[2] = {0, 0};  // degree of space U, P
  int N[2] = {0, 0};
  long long n[2] = {0, 0};
  dgns::Space1D sp1[2];
  dgns::LapHost lap[2];               // unit-coefficient SIPG tables of U and P
  std::vector<double> diag[2];  // N^3 diagonal pattern of L
  double* d_diag[2] = {nullptr, nullptr};
  double mass3[2][3][dgns::MAXN * dgns::MAXN];
  double minv3[2][3][dgns::MAXN * dgns::MAXN];
  dgns::DivHost div;
  dgns::GradHost grad;
  dgns::ConvHost conv;
  double* conv_face = nullptr;  // face integrals of the convective term, 9 E N^2
  double* lap_face = nullptr;   // face data of the split SIPG evaluation
  size_t lap_face_cap = 0;      // its size in bytes
  dgns::ProjHost proj;
  // multigrid (pressure space)
  int mg_prec = 0;
  std::vector<dgns::Level> levels;
  double P0[dgns::MAXN * dgns::MAXN], P1[dgns::MAXN * dgns::MAXN];
  // FP64 CG work vectors and reductions
  long long cg_cap = 0;
  double *r = nullptr, *z = nullptr, *p = nullptr, *Ap = nullptr;
  dgns::Reducer red;
  double* h_scal = nullptr;  // pinned mirror of the scalars
  // CUDA graph of one preconditioner application (r -> z on the CG work
  // vectors), captured on a private stream and replayed on s
  cudaStream_t gs = nullptr;
  cudaGraphExec_t vc_exec = nullptr;
  int vc_key[3] = {0, 0, 0};
  double vc_range = 0.0;
  // input range of the emulated arithmetic (fp64_mode 1, 2): the largest
  // exponent of an input (device), and work buffers for scaled copies
  unsigned* d_expmax = nullptr;
  void* rwork[3] = {nullptr, nullptr, nullptr};
  size_t rwork_cap[3] = {0, 0, 0};
  // staging of host pointers
  void* stage[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t stage_ev = nullptr;  // recorded after the staging copies of host inputs
  size_t stage_cap[4] = {0, 0, 0, 0};
};
