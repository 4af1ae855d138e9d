/*
 * dgns.h - C ABI of libdgns: matrix-free discontinuous Galerkin operators of
 * the incompressible Navier-Stokes dual-splitting solver of Fehn, Wall &
 * Kronbichler (arXiv:1802.01439), on one NVIDIA GB300 (sm_103a).
 *
 * Discretisation (paper Sec. 3.2): uniform periodic Cartesian mesh of hexahedra,
 * tensor-product Lagrange basis on Legendre-Gauss-Lobatto (LGL) nodes, degree
 * k_u for velocity (space U) and k_p for pressure (space P), Gauss quadrature
 * exact on affine cells, floor(3(k_u+1)/2) points for the convective term.
 *
 * Vector layout (all operators): contiguous, [comp][elem][z][y][x] with x
 * fastest and element id e = i + nx*(j + ny*l).  A scalar field in space S has
 * n_elem * (k_S+1)^3 entries; a velocity field has three such blocks.
 *
 * Pointers: every vector argument is either a device pointer (cudaMalloc,
 * torch CUDA tensor) or a host pointer (pinned or pageable).  With device
 * pointers the call is enqueued on the context's stream and returns at once
 * (in the emulated arithmetic modes 1 and 2 after reading back one word that
 * describes the input's range, see fp64_mode).
 * With host pointers the library stages the data through its own device
 * buffers (allocated at the first such call) and runs the same kernels; a
 * call with a host output copies the result back and returns when it is
 * complete; a call whose only host vectors are inputs returns once they are
 * copied (the caller may then reuse them) while its kernels run on in stream
 * order.
 * The caller owns every vector; the library owns its tables, multigrid levels
 * and scratch.  dst must not alias any source (DGNS_ERR_ALIAS).  Device
 * vectors must be 16-byte aligned (cudaMalloc and torch allocations are; a
 * misaligned view is rejected with DGNS_ERR_INVALID_ARG).
 *
 * Errors: every entry point returns 0 on success or a DGNS_ERR_* code; no C++
 * exception crosses the ABI; dgns_last_error() gives a message for the calling
 * thread.  A context must be used by one host thread at a time.
 */
#ifndef DGNS_H
#define DGNS_H

#ifdef __cplusplus
extern "C" {
#endif

#define DGNS_OK 0
#define DGNS_ERR_INVALID_ARG 1   /* bad size, degree, space, null pointer   */
#define DGNS_ERR_CUDA 2          /* a CUDA runtime call failed             */
#define DGNS_ERR_OOM 3           /* device allocation failed               */
#define DGNS_ERR_NOT_CONVERGED 4 /* solver hit max_iter; info is filled    */
#define DGNS_ERR_NONFINITE 5     /* NaN/Inf residual in a solver, or a      */
                                 /* non-finite input in modes 1 and 2       */
#define DGNS_ERR_ALIAS 6         /* dst overlaps a source                  */
#define DGNS_ERR_UNSUPPORTED 7   /* valid request this build does not do   */

#define DGNS_SPACE_U 0 /* velocity space, degree k_u ("degree")        */
#define DGNS_SPACE_P 1 /* pressure space, degree k_p ("degree_p")      */

#define DGNS_MAX_DEGREE 11
#define DGNS_MAX_LEVELS 16

typedef struct dgns_ctx dgns_ctx;

typedef struct {
  int n_elem[3];         /* elements per direction, >= 1                         */
  double lo[3], hi[3];   /* box; the paper's Taylor-Green box is [-pi, pi]^3      */
  int degree;            /* k_u in 1..11                                          */
  int degree_p;          /* k_p in 1..11; -1 selects k_u - 1 (Sec. 3.2)           */
  int n_q_conv;          /* convective Gauss points per direction; 0 = 3(k+1)/2  */
  double penalty_factor; /* SIPG tau = penalty_factor (k+1)^2 / h; 0 selects 1    */
  double nu;             /* kinematic viscosity of the viscous operator           */
  int mg_coarse_n;       /* coarsest multigrid mesh (elements per direction)      */
  int mg_precision;      /* 32 or 64: arithmetic of the V-cycle; 0 = no multigrid */
  int fp64_mode;         /* arithmetic of every FP64 operator kernel (convective    */
                         /* and its VJP, SIPG-type, mass, divergence, gradient,     */
                         /* projection, penalty parameters, dissipation, the CG     */
                         /* matvecs and inverse-mass preconditioners): 0 native     */
                         /* FP64;                                                   */
                         /* 1 double-float (pairs of FP32 with a 48-bit significand */
                         /* on the FP32 pipe, which GB300 runs 61x faster; parity   */
                         /* with FP64 to 1e-12 relative);                           */
                         /* 2 FP64-wide: triple-float (three FP32, up to 72         */
                         /* significant bits, on the FP32 pipe) in the SIPG-type    */
                         /* and mass kernels and the low-degree convective face     */
                         /* kernels, native-FP64 and triple-float blocks side by    */
                         /* side in the k <= 3 convective cell kernel, native FP64  */
                         /* in all others.  The emulations carry float's exponent: */
                         /* in modes 1 and 2 every operator call and solve measures */
                         /* its input's largest exponent (one reduction and a       */
                         /* read-back, so these calls synchronise the stream) and   */
                         /* scales an input outside [2^-40, 2^90] (convective term:  */
                         /* [2^-20, 2^45]) by an exact power of two, so any FP64    */
                         /* scale is evaluated at full accuracy.  The vector-       */
                         /* Jacobian product, the penalty parameters and the        */
                         /* dissipation take inputs as they are.  The multigrid     */
                         /* V-cycle runs in mg_precision in every mode.             */
} dgns_mesh_desc;

/* Defaults: 4^3 elements on [-pi,pi]^3, k_u = 3, k_p = k_u - 1, 3/2 rule,
 * penalty factor 1, nu = 1/1600, coarse mesh 2, FP32 multigrid. */
void dgns_default_desc(dgns_mesh_desc* desc);

/* Create a context: computes the 1D tables on the host (long double), builds
 * the multigrid hierarchy of the pressure space when mg_precision != 0
 * (levels n, n/2, ... >= mg_coarse_n while every n is even), estimates the
 * Chebyshev eigenvalue bound of every level, and allocates all device memory
 * the operators and solvers need.  stream: a cudaStream_t or NULL (default
 * stream).  On failure *out is NULL and nothing is leaked. */
int dgns_create(const dgns_mesh_desc* desc, void* stream, dgns_ctx** out);
int dgns_destroy(dgns_ctx* ctx);
/* Later calls enqueue on `stream` (a cudaStream_t, NULL for the default
 * stream).  Work already enqueued on the previous stream is not ordered before
 * them: synchronise it, or make the new stream wait on an event, first. */
int dgns_set_stream(dgns_ctx* ctx, void* stream);
const char* dgns_status_string(int status);
const char* dgns_last_error(void);

/* Scalar DoFs per component of space U and space P:
 * n_elem_total * (k+1)^3 (paper Sec. 4, DoF count formula). */
int dgns_sizes(const dgns_ctx* ctx, long long* n_u, long long* n_p);
/* The k+1 LGL nodes on [0,1] of a space, as used by the library (host out). */
int dgns_nodes_1d(const dgns_ctx* ctx, int space, double* out);

/* SIPG Laplace l_h (Sec. 3.2, negative Laplacian of the pressure Poisson
 * equation, matrix L of Sec. 3.3) on one scalar field of `space`:
 * dst = L src.  FP64. */
int dgns_vmult_laplace(dgns_ctx* ctx, double* dst, const double* src, int space);
/* The same operator evaluated operator by operator, as the cell integrals
 * and the interior-face terms of Sec. 3.2 in separate kernels (the cell
 * stiffness term; a face kernel forming each face's jump and mean normal
 * derivative on its lines, weighted by the tangential mass; a kernel adding
 * the six faces' terms to every cell): the counterpart of the fused kernel
 * behind dgns_vmult_laplace, for comparison.  Native FP64 in every
 * fp64_mode.  Allocates a face buffer (6 n_elem_total (k+1)^2 doubles) at its
 * first call, or when a larger space needs one. */
int dgns_vmult_laplace_split(dgns_ctx* ctx, double* dst, const double* src, int space);
/* Same operator in FP32 on multigrid level `level` (0 = coarsest, levels-1 =
 * the pressure space itself).  Device pointers only. */
int dgns_vmult_laplace_f32(dgns_ctx* ctx, float* dst, const float* src, int level);
/* One step of the FP32 Jacobi-Chebyshev smoother on multigrid level `level`
 * (Sec. 3.3), fused into the level operator as the V-cycle runs it:
 * dst = x + c1 (x - xprev) + c2 D^-1 (b - L x), with D the diagonal of the
 * level's L (one N^3 table, identical in every cell) and xprev = NULL read
 * as zero.  Needs mg_precision = 32; device pointers, 16-byte aligned; dst
 * must not overlap an input. */
int dgns_mg_chebyshev_step_f32(dgns_ctx* ctx, float* dst, const float* x, const float* xprev, const float* b,
                               double c1, double c2, int level);
/* Diagonal of L (the Jacobi weights of the Chebyshev smoother, Sec. 3.3). */
int dgns_laplace_diagonal(dgns_ctx* ctx, double* dst, int space);

/* Viscous SIPG v_h (Sec. 3.2, Laplace formulation F_v = nu grad u): dst3 =
 * nu L src3 per velocity component (space U, tau with k_u). */
int dgns_vmult_viscous(dgns_ctx* ctx, double* dst3, const double* src3);
/* Helmholtz operator of the viscous substep (Sec. 3.3):
 * dst3 = (mass_factor M + V) src3 in one pass per component. */
int dgns_vmult_helmholtz(dgns_ctx* ctx, double* dst3, const double* src3, double mass_factor);

/* Mass matrix m_h (Sec. 3.2) and its exact block-diagonal inverse (Sec. 3.3)
 * on ncomp consecutive scalar fields of `space`. */
int dgns_vmult_mass(dgns_ctx* ctx, double* dst, const double* src, int ncomp, int space);
int dgns_apply_inverse_mass(dgns_ctx* ctx, double* dst, const double* src, int ncomp, int space);

/* Velocity divergence d_h (Sec. 3.2, central flux, k_u+1 Gauss points):
 * dst_p (space P) = D u3 (space U, 3 components). */
int dgns_vmult_divergence(dgns_ctx* ctx, double* dst_p, const double* u3);
/* Pressure gradient g_h (Sec. 3.2, central flux): dst3 (space U) = G p. */
int dgns_vmult_gradient(dgns_ctx* ctx, double* dst3, const double* p);

/* Convective term c_h (Sec. 3.2) with F_c = u (x) u and the local
 * Lax-Friedrichs flux, over-integrated with n_q_conv points: dst3 = C(u3),
 * the weak form (not multiplied by M^-1, not negated).  The first call on a
 * context allocates a device scratch buffer of 9 E (k_u+1)^2 doubles for the
 * face integrals (DGNS_ERR_OOM if that fails); make it before capturing
 * calls into a CUDA graph. */
int dgns_vmult_convective(dgns_ctx* ctx, double* dst3, const double* u3);

/* The two phases of dgns_vmult_convective, with a caller-owned face buffer.
 * dgns_convective_face_size: *n = 9 E (k_u+1)^2, the doubles of rface.
 * dgns_convective_faces: every face once (Sec. 3.2, LLF flux), rface =
 * [d][cell e][component c][j1 + (k_u+1) j2]: the flux integral of the face
 * between cell e and its neighbour in +x_d against the face-layer basis of
 * cell e (j1, j2 the node indices along the two other directions, lower
 * direction first); the neighbour's integral is its negative.
 * dgns_convective_cells: the cell term of every cell plus the six face
 * integrals from rface: dst3 = C(u3).  rface must come from
 * dgns_convective_faces on the same u3. */
int dgns_convective_face_size(const dgns_ctx* ctx, long long* n);
int dgns_convective_faces(dgns_ctx* ctx, double* rface, const double* u3);
int dgns_convective_cells(dgns_ctx* ctx, double* dst3, const double* u3, const double* rface);
/* Vector-Jacobian product of the convective term: grad_u3 = (dC/du)^T w3 at
 * u3.  At LLF kinks it uses d|s|/ds = sign(s) (sign(0) = 0) and sends the
 * derivative of max(a, b) to the larger argument (half to each on a tie). */
int dgns_vjp_convective(dgns_ctx* ctx, double* grad_u3, const double* u3, const double* w3);

/* Dissipation rate of the resolved scales, eps = nu / |Omega| int grad u : grad u
 * (Sec. 4.2), with the element-wise (broken) gradient and k_u+1 Gauss points:
 * *eps_out (host) = eps(u3).  Synchronises the stream. */
int dgns_dissipation(dgns_ctx* ctx, const double* u3, double* eps_out);
/* Its gradient: grad3 = d eps / d u3 = (2 nu / |Omega|) K u3 per component,
 * K the broken stiffness matrix (cell terms of l_h only). */
int dgns_dissipation_grad(dgns_ctx* ctx, double* grad3, const double* u3);

/* Vector helpers of the time stepper (device pointers, context stream):
 * y = a x + b y over n entries (b = 0 ignores the prior contents of y; x may
 * equal y), and *out (host) = (a, b) over n entries
 * (deterministic fixed-order reduction; synchronises the stream). */
int dgns_axpby(dgns_ctx* ctx, double* y, const double* x, long long n, double a, double b);
int dgns_dot(dgns_ctx* ctx, const double* a, const double* b, long long n, double* out);

/* Penalty parameters of the projection step (Sec. 3.2, divergence and
 * continuity penalty terms): per cell, with ||u||_e the volume average of the
 * Euclidean norm of the extrapolated velocity u_ex3 (k_u+1 Gauss points) and
 * h = V_e^(1/3):  tau_d[e] = zeta_d ||u||_e h / (k_u+1) dt,
 * tau_c[e] = zeta_c ||u||_e dt.  Device pointers (tau arrays of n_elem
 * doubles). */
int dgns_penalty_parameters(dgns_ctx* ctx, const double* u_ex3, double dt, double zeta_d, double zeta_c,
                            double* tau_d, double* tau_c);
/* Projection operator of the projection substep (Sec. 3.3):
 * dst3 = (M + A_D + A_C) src3 with a_D(v,u) = (div v, tau_D div u)_e and
 * a_C(v,u) = sum_F int {{tau_C}} (v- - v+).n (u- - u+).n, in one fused pass
 * over memory.  Device pointers. */
int dgns_vmult_projection(dgns_ctx* ctx, double* dst3, const double* src3, const double* tau_d,
                          const double* tau_c);
/* The terms of the same operator one at a time, each in its own pass over
 * memory (the operator-by-operator evaluation that the fused operator is
 * compared with in Sec. 4.4): terms = DGNS_PROJ_MASS (dst3 = M src3, the
 * mass kernel; tau arrays unused, may be NULL), DGNS_PROJ_DIV
 * (dst3 = A_D src3; tau_c unused), DGNS_PROJ_CONT (dst3 = A_C src3; tau_d
 * unused) or DGNS_PROJ_ALL (the fused operator, as dgns_vmult_projection).
 * Device pointers; any other terms value returns DGNS_ERR_INVALID_ARG. */
#define DGNS_PROJ_MASS 1
#define DGNS_PROJ_DIV 2
#define DGNS_PROJ_CONT 4
#define DGNS_PROJ_ALL 7
int dgns_vmult_projection_terms(dgns_ctx* ctx, double* dst3, const double* src3, const double* tau_d,
                                const double* tau_c, int terms);

/* CG solves stop when ||r||_2 <= rel_tol ||r_0||_2 or ||r||_2 <= abs_tol,
 * r_0 = b - A x_0 the initial residual (Sec. 3.3: the paper's solvers use
 * abs_tol = 1e-12 and rel_tol = 1e-6 with x_0 extrapolated from previous
 * time steps). */
typedef struct {
  double rel_tol;          /* default 1e-10                                         */
  double abs_tol;          /* default 0                                             */
  int max_iter;            /* default 200                                           */
  int cheb_degree;         /* Chebyshev degree, pre and post (default 5)            */
  double smoothing_range;  /* lambda_max / lambda_min of the smoother (default 20)  */
  int cheb_coarse_iters;   /* Chebyshev steps of the coarse solve (default 20)       */
  int project_mean;        /* 1: remove the Euclidean mean of r0 and of every z      */
  int use_initial_guess;   /* 0 (default): x_0 = 0; 1: x holds x_0 on entry (read
                              and overwritten; host pointers are copied both ways)  */
} dgns_solve_params;

typedef struct {
  int iterations;
  double rel_res;          /* final ||r||_2 / ||r_0||_2 (recursively updated r)     */
  double initial_res;      /* ||r_0||_2 (= ||b||_2 for x_0 = 0)                      */
  int status;
  double lambda_max_fine;  /* Chebyshev upper bound of the finest level             */
  double seconds;          /* wall time of the solve                                */
} dgns_solve_info;

void dgns_default_solve_params(dgns_solve_params* p);

/* Pressure Poisson solve (Sec. 3.3): FP64 conjugate gradients preconditioned
 * by one h-multigrid V-cycle per iteration with Jacobi-Chebyshev smoothing
 * (degree cheb_degree pre and post, range smoothing_range), Chebyshev coarse
 * solve, embedding prolongation and its transpose as restriction; the V-cycle
 * runs in the context's mg_precision.  x (space P) gets the solution;
 * initial guess per params->use_initial_guess.  Returns
 * DGNS_ERR_NOT_CONVERGED with info filled when max_iter is reached. */
int dgns_cg_mg_solve(dgns_ctx* ctx, double* x, const double* b,
                     const dgns_solve_params* params, dgns_solve_info* info);

/* Multigrid hierarchy: number of levels, elements per direction and the
 * Chebyshev upper eigenvalue bound (already including the safety factor) of
 * each level, coarsest first (host outputs, arrays of DGNS_MAX_LEVELS). */
int dgns_mg_info(const dgns_ctx* ctx, int* n_levels, int* n_elem_per_level, double* lambda_max);
/* One V-cycle, z = V(r), on the finest level in the context's precision,
 * FP64 in and out (device pointers). */
int dgns_mg_vcycle(dgns_ctx* ctx, double* z, const double* r, const dgns_solve_params* params);
/* Grid transfers between level `level` and `level`+1 (FP32, device):
 * prolongation = embedding of the coarse polynomials, restriction = its
 * transpose. */
int dgns_mg_prolongate_f32(dgns_ctx* ctx, float* fine, const float* coarse, int level);
int dgns_mg_restrict_f32(dgns_ctx* ctx, float* coarse, const float* fine, int level);

/* Helmholtz solve (viscous substep, Sec. 3.3): CG preconditioned by the
 * inverse mass matrix on (mass_factor M + V) x3 = b3, FP64; initial guess
 * per params->use_initial_guess. */
int dgns_cg_invmass_solve(dgns_ctx* ctx, double* x3, const double* b3, double mass_factor,
                          const dgns_solve_params* params, dgns_solve_info* info);

/* Allocation-free variant of dgns_cg_invmass_solve (the paper has no
 * counterpart: this serves callers that cannot let a library allocate device
 * memory, e.g. applications whose device memory belongs to their own pool or
 * allocator, or real-time loops that must not risk allocation latency or an
 * out-of-memory failure in the middle of a time step).  Same arguments, same
 * arithmetic and the same result.  Differences:
 *   - x3 and b3 must be device pointers (no host staging), and the device that
 *     holds the context must be current (else DGNS_ERR_INVALID_ARG);
 *   - 3 * n_u (the CG vector length) must not exceed 524288, the size of a
 *     fixed scratch array compiled into the library (four work vectors plus
 *     reduction partials, ~16 MiB held by every GPU that loads the library
 *     until the process exits); larger sizes return DGNS_ERR_INVALID_ARG;
 *   - the call performs no cudaMalloc/cudaFree.  Its first call on a device
 *     looks up the device address of that array (cudaGetSymbolAddress, once
 *     per device, under a lock); make that first call before any stream
 *     capture.
 * Like dgns_cg_invmass_solve, it reads one block of scalars back to the host
 * and synchronises the context's stream once per CG iteration, and returns
 * after the solve has finished.
 * All calls share the one array and it keeps the last call's contents:
 * calls that may overlap on the GPU (other streams, other host threads,
 * other contexts) race on it and must be serialised by the caller. */
int dgns_cg_invmass_solve_noalloc(dgns_ctx* ctx, double* x3, const double* b3, double mass_factor,
                                  const dgns_solve_params* params, dgns_solve_info* info);

/* Projection solve (Sec. 3.3): CG preconditioned by the inverse mass
 * matrix on (M + A_D + A_C) x3 = b3, FP64; initial guess per
 * params->use_initial_guess; device pointers. */
int dgns_cg_projection_solve(dgns_ctx* ctx, double* x3, const double* b3, const double* tau_d,
                             const double* tau_c, const dgns_solve_params* params, dgns_solve_info* info);

/* Test hooks for the failure paths (for tests, not for production use).
 * dgns_debug_fail_alloc(n): the n-th device allocation the library makes from
 * now on (n >= 1; any context, any thread) fails as if the device were out of
 * memory, and the hook disarms itself; n = 0 disarms it.  Returns
 * DGNS_ERR_INVALID_ARG for n < 0.
 * dgns_debug_live_allocations: device allocations the library has made and
 * not yet freed, over all contexts. */
int dgns_debug_fail_alloc(long long n);
/* Measurement hook: in fp64_mode 2 the convective cell kernel runs native-FP64
 * and triple-float blocks side by side; of every `period` consecutive blocks
 * the first `nnative` run native FP64.  period = 0 restores the built-in
 * split; period = -1 runs the convective kernels in triple-float throughout.
 * Returns DGNS_ERR_INVALID_ARG unless period >= -1 and 0 <= nnative <= period. */
int dgns_debug_conv_mix(int period, int nnative);
/* Measurement hook: the kernel of the FP32 Laplace operator at k_p = 3 (the
 * multigrid level operator and the Chebyshev step).  0: built-in; -1: one
 * thread per x-line of a cell, data staged in shared memory by the threads;
 * 1: one thread per cell plane, data in registers, packed FP32x2 arithmetic;
 * 2: the same with scalar FP32 arithmetic (bit-identical results); 3: as 1
 * with the z-direction as one reduce-scatter; 4: one thread per cell plane,
 * data staged in shared memory by tensor copies, one stage and 12 warps per
 * SM; 5: as 4 with two stages and 7 warps.  The built-in choice is 4 where it
 * applies (nx divisible by 8, every vector 32-byte aligned), else 1 (every
 * vector 32-byte aligned), else -1; 1..5 fall back the same way.  Returns
 * DGNS_ERR_INVALID_ARG outside -1..5. */
int dgns_debug_laplace_f32_kernel(int variant);
/* Bounded waits of the staged FP32 Laplace kernel that gave up since the
 * library was loaded (0 in a healthy run; a nonzero count means that kernel
 * left results unwritten).  Synchronous device read. */
long long dgns_debug_laplace_f32_timeouts(void);
long long dgns_debug_live_allocations(void);
/* Test hook: y[i] = (double) x[i] for n device floats, by the conversion the
 * FP32 multigrid preconditioner uses on its output (on the bit patterns for
 * normal floats and zeros, by the hardware for the others; exact either way).
 * x, y: device pointers owned by the caller, n >= 0.  Runs on the default
 * stream and synchronises it.  Returns DGNS_ERR_INVALID_ARG for n < 0 or a
 * null pointer with n > 0, DGNS_ERR_CUDA on a launch error. */
int dgns_debug_widen_f32(const float* x, double* y, long long n);

#ifdef __cplusplus
}
#endif
#endif /* DGNS_H */
